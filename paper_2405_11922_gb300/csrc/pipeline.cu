// The whole method (Algorithms 1-3 and Eq. 8) over a batch of stacked graphs,
// the plain single-graph call, the batched call, and the step-level entry
// points of abg.h (each a one-segment batch).
#include <algorithm>
#include <cmath>
#include <cstring>

#include "internal.cuh"

// Z_hat kept on a graph by a solve with ABG_REUSE_PROPAGATION, and the parameters that fix it
// (Z_hat depends on alpha, gamma, d, the BF16 storage option and, through X' of Eq. 15 when
// d < d_u, on the seed, oversample and power_iters; never on k or the NCI options).
struct ZKey {
  double alpha = 0.0;
  int gamma = 0, d = 0, bf16 = 0, oversample = 0, power_iters = 0;
  uint64_t seed = 0;
  bool operator==(const ZKey& o) const {
    return alpha == o.alpha && gamma == o.gamma && d == o.d && bf16 == o.bf16 &&
           oversample == o.oversample && power_iters == o.power_iters && seed == o.seed;
  }
};
struct ZCache {
  ZKey key;
  int device = 0;
  float* buf = nullptr;
  int64_t bytes = 0;
  cudaEvent_t ready = nullptr;  // recorded after the copy into buf
  ~ZCache() {
    cudaSetDevice(device);
    if (ready) cudaEventDestroy(ready);
    if (buf) cudaFree(buf);  // the last solve that read it has finished (it held a reference)
  }
};

// Phi and H at the end of the ONMF steps of a solve with ABG_WARM_START, for a later solve
// on the same graph with the same k and d (the shapes that fix them).
struct PhiCache {
  int k = 0, d = 0;
  int device = 0;
  float* phi = nullptr;  // n_u x round_up(k, 4)
  float* h = nullptr;    // 2d x round_up(k, 4)
  int64_t phi_bytes = 0, h_bytes = 0;
  cudaEvent_t ready = nullptr;  // recorded after the copies into phi and h
  ~PhiCache() {
    cudaSetDevice(device);
    if (ready) cudaEventDestroy(ready);
    if (phi) cudaFree(phi);  // the last solve that read them has finished (it held a reference)
    if (h) cudaFree(h);
  }
};

using namespace abg;

namespace {

struct Ev {
  cudaEvent_t e = nullptr;
  Ev() { cudaEventCreate(&e); }
  ~Ev() {
    if (e) cudaEventDestroy(e);
  }
};

}  // namespace

int abg::check_params(const abg_graph* g, const abg_params* p, int64_t n_rows, int* d_eff) {
  ABG_CHECK(g && p, "null graph or parameters");
  const int d = p->d == 0 ? g->d_u : p->d;
  ABG_CHECK(d >= 1 && d <= g->d_u, "need 1 <= d <= d_u (got d=%d, d_u=%d)", d, g->d_u);
  ABG_CHECK(d <= kMaxD, "d must be <= %d", kMaxD);
  ABG_CHECK(p->alpha >= 0.0 && p->alpha < 1.0, "need 0 <= alpha < 1");
  ABG_CHECK(p->gamma >= 0 && p->t_f >= 0 && p->t_g >= 0, "gamma, t_f, t_g must be >= 0");
  ABG_CHECK(p->oversample >= 0 && p->power_iters >= 0, "oversample, power_iters must be >= 0");
  ABG_CHECK(p->k >= 1 && p->k <= kMaxK && p->k <= 2 * d && p->k <= n_rows,
            "need 1 <= k <= min(|U|, 2d, %d) (got k=%d)", kMaxK, p->k);
  ABG_CHECK(d == g->d_u || (int64_t)d + p->oversample <= 1024,
            "attribute reduction needs d + oversample <= 1024");
  ABG_CHECK((p->nci_flags & ~(ABG_NCI_PROCRUSTES | ABG_NCI_EARLY_STOP)) == 0,
            "unknown nci_flags %d", p->nci_flags);
  ABG_CHECK((p->precision & ~(ABG_BF16_CONTRACT | ABG_BF16_PROPAGATION)) == 0,
            "unknown precision %d", p->precision);
  ABG_CHECK((p->options & ~(ABG_REUSE_PROPAGATION | ABG_WARM_START)) == 0, "unknown options %d",
            p->options);
  *d_eff = d;
  return ABG_OK;
}

namespace {

// Device outputs of one batched solve.
struct SolveOut {
  int reused = 0;                     // Z_hat taken from the graph's ZCache
  std::shared_ptr<ZCache> zhold;      // keeps that ZCache alive until the solve has finished
  int warm = 0;                       // Phi, H taken from the graph's PhiCache
  std::shared_ptr<PhiCache> phold;    // keeps that PhiCache alive until the solve has finished
  int32_t* labels = nullptr;   // rows
  double* obj = nullptr;       // 2 per segment
  int* counters = nullptr;     // 3 per segment: changes, min margin bits, empty clusters
  int* clamped = nullptr;      // per segment
  int* breakdowns = nullptr;   // 1
  std::vector<int> passes;     // NCI passes per segment
};

// Attributes the propagation reads: the graph's own (dense), a densified CSR, or the
// per-segment SVD-reduced X' of Eq. 15. bf16_contract: the products of that SVD read BF16
// attributes directly (BF16 tensor-core kernels, FP32 accumulation).
int prepare_attributes(const abg_graph* g, const RowSpace& rs, int d, int oversample,
                       int power_iters, const std::vector<uint64_t>& seeds, Scratch& scr,
                       cudaStream_t s, const float** xf, const __nv_bfloat16** xb, int64_t* ldx,
                       int* breakdowns, bool bf16_contract = false) {
  *xf = nullptr;
  *xb = nullptr;
  if (d == g->d_u) {
    if (g->x_kind == ABG_X_DENSE_F32) {
      *xf = (const float*)g->x;
      *ldx = g->ldx;
    } else if (g->x_kind == ABG_X_DENSE_BF16) {
      *xb = (const __nv_bfloat16*)g->x;
      *ldx = g->ldx;
    } else {
      float* dense;
      const int64_t ld = round_up(d, 4);
      ABG_TRY(scr.get(&dense, (size_t)g->n_u * ld));
      ABG_TRY(csr_to_dense(g->x_ptr, g->x_col, g->x_val, g->n_u, d, dense, ld, s));
      *xf = dense;
      *ldx = ld;
    }
    return ABG_OK;
  }
  const int64_t ldo = round_up(d, 4);
  float* xr;
  ABG_TRY(scr.get(&xr, (size_t)g->n_u * ldo));
  std::vector<int> kx(rs.nseg, d), lx(rs.nseg);
  for (int i = 0; i < rs.nseg; ++i)
    lx[i] = (int)std::min<int64_t>({(int64_t)d + oversample, (int64_t)g->d_u, rs.h_n[i]});
  for (int i = 0; i < rs.nseg; ++i)
    ABG_CHECK(lx[i] >= d, "attribute reduction of segment %d: d exceeds its row count", i);
  SegSizes ssx;
  ABG_TRY(segsizes_build(&ssx, kx, lx, seeds, scr, s));
  RsvdIn in;
  in.rows = &rs;
  in.m = g->d_u;
  if (g->x_kind == ABG_X_CSR_F32) {
    in.ptr = g->x_ptr;
    in.col = g->xr_col;
    in.val = g->x_val;
    in.tptr = g->xt_ptr;
    in.tcol = g->xt_col;
    in.tval = g->xt_val;
  } else if (g->x_kind == ABG_X_DENSE_F32) {
    in.A = (const float*)g->x;
    in.lda = g->ldx;
  } else {
    float* xf32;
    ABG_TRY(scr.get(&xf32, (size_t)g->n_u * g->ldx));
    ABG_TRY(bf16_to_f32((const __nv_bfloat16*)g->x, g->ldx, g->n_u, (int)g->ldx, xf32, g->ldx, s));
    in.A = xf32;
    in.lda = g->ldx;
    if (bf16_contract) {
      in.A16 = (const __nv_bfloat16*)g->x;
      in.lda16 = g->ldx;
    }
  }
  RsvdOut out;
  out.left = xr;
  out.ldl = ldo;
  out.left_mode = 1;
  ABG_TRY(rsvd(in, ssx, d, power_iters, ABG_STREAM_OMEGA_X, out, breakdowns, s));
  *xf = xr;
  *ldx = ldo;
  return ABG_OK;
}

// R16 (may be null): BF16 copy of R for the two products with R (R^T Phi and R H).
int onmf_iterations(const RowSpace& rs, const SegSizes& ss, const float* R, int m, int64_t ldr,
                    int t_f, float* phi, int64_t ldphi, float* H, int64_t ldh, int64_t hseg,
                    cudaStream_t s, const __nv_bfloat16* R16 = nullptr, int64_t ldr16 = 0) {
  if (t_f == 0) return ABG_OK;
  const int nseg = rs.nseg, kmax = ss.k_max;
  const int64_t kk = round_up(kmax, 4);
  Scratch scr(s);
  float *P, *phi2, *C32;
  double *A, *G, *C;
  ABG_TRY(scr.get(&P, (size_t)rs.rows * ldphi));
  ABG_TRY(scr.get(&phi2, (size_t)rs.rows * ldphi));
  ABG_TRY(scr.get(&C32, (size_t)nseg * kmax * kk));
  ABG_TRY(scr.get(&A, (size_t)nseg * m * kmax));
  ABG_TRY(scr.get(&G, (size_t)nseg * kmax * kmax));
  ABG_TRY(scr.get(&C, (size_t)nseg * kmax * kmax));
  float* cur = phi;
  float* nxt = phi2;
  for (int t = 0; t < t_f; ++t) {
    // Eq. 16: H <- H * (R^T Phi) / (H (Phi^T Phi))
    TN ta;
    ta.A = R;
    ta.lda = ldr;
    ta.A16 = R16;
    ta.lda16 = ldr16;
    ta.B = cur;
    ta.ldb = ldphi;
    ta.K = m;
    ta.N = kmax;
    ta.segN = ss.k;
    ta.C = A;
    ta.ldc = kmax;
    ta.c_seg = (int64_t)m * kmax;
    ABG_TRY(gemm_tn(rs, ta, s));
    TN tg;
    tg.A = tg.B = cur;
    tg.lda = tg.ldb = ldphi;
    tg.K = tg.N = kmax;
    tg.segK = tg.segN = ss.k;
    tg.C = G;
    tg.ldc = kmax;
    tg.c_seg = (int64_t)kmax * kmax;
    ABG_TRY(gemm_tn(rs, tg, s));
    ABG_TRY(nmf_update_h(nseg, m, ss.k, kmax, H, ldh, hseg, A, kmax, (int64_t)m * kmax, G, kmax,
                         (int64_t)kmax * kmax, s));
    // Eq. 17: Phi <- Phi * sqrt((R H) / (Phi (Phi^T (R H))))
    NN pr;
    pr.A = R;
    pr.lda = ldr;
    pr.A16 = R16;
    pr.lda16 = ldr16;
    pr.B = H;
    pr.ldb = ldh;
    pr.b_seg = hseg;
    pr.C = P;
    pr.ldc = ldphi;
    pr.N = kmax;
    pr.K = m;
    pr.segN = ss.k;
    ABG_TRY(gemm_nn(rs, pr, s));
    // Phi^T (R H) = (R^T Phi)^T H: the tall reduction R^T Phi of the H rule (same Phi) is
    // reused, so only a k x 2d x k product remains
    ABG_TRY(small_atb(nseg, m, ss.k, kmax, A, kmax, (int64_t)m * kmax, H, ldh, hseg, C, kmax,
                      (int64_t)kmax * kmax, s));
    ABG_TRY(convert_f64_to_f32(C, (int64_t)nseg * kmax, kmax, kmax, C32, kk, s));
    NN pu;
    pu.A = cur;
    pu.lda = ldphi;
    pu.B = C32;
    pu.ldb = kk;
    pu.b_seg = (int64_t)kmax * kk;
    pu.C = nxt;
    pu.ldc = ldphi;
    pu.N = pu.K = kmax;
    pu.segN = pu.segK = ss.k;
    pu.epi = Epi::PhiUpdate;
    pu.aux = P;
    pu.ldaux = ldphi;
    pu.aux2 = cur;
    pu.ldaux2 = ldphi;
    ABG_TRY(gemm_nn(rs, pu, s));
    std::swap(cur, nxt);
  }
  if (cur != phi)
    ABG_CUDA(cudaMemcpyAsync(phi, cur, sizeof(float) * rs.rows * ldphi, cudaMemcpyDeviceToDevice, s));
  return ABG_OK;
}

// Algorithms 1-3 and Eq. 8 for every segment of g; ev[0..6] (optional) get the phase
// boundaries recorded on s.
// Keeps a copy of zhat (count floats) on g for later solves with the same key, replacing the
// one held before. Best effort: without device memory for the copy nothing is kept.
int zcache_store(abg_graph* g, const ZKey& key, const float* zhat, int64_t count, cudaStream_t s) {
  auto c = std::make_shared<ZCache>();
  c->key = key;
  c->device = g->device;
  c->bytes = count * (int64_t)sizeof(float);
  if (cudaMalloc(&c->buf, (size_t)c->bytes) != cudaSuccess) {
    cudaGetLastError();
    c->buf = nullptr;
    return ABG_OK;
  }
  ABG_CUDA(cudaMemcpyAsync(c->buf, zhat, (size_t)c->bytes, cudaMemcpyDeviceToDevice, s));
  ABG_CUDA(cudaEventCreateWithFlags(&c->ready, cudaEventDisableTiming));
  ABG_CUDA(cudaEventRecord(c->ready, s));
  std::lock_guard<std::mutex> lk(g->zmu);
  if (g->zcache) g->footprint -= g->zcache->bytes;
  g->zcache = c;
  g->footprint += c->bytes;
  return ABG_OK;
}

// Keeps copies of phi (n_u x ldp floats) and h (2d x ldp) on g for later warm-started solves
// with the same k and d, replacing those held before. Best effort, as zcache_store.
int phicache_store(abg_graph* g, int k, int d, const float* phi, int64_t phi_count,
                   const float* h, int64_t h_count, cudaStream_t s) {
  auto c = std::make_shared<PhiCache>();
  c->k = k;
  c->d = d;
  c->device = g->device;
  c->phi_bytes = phi_count * (int64_t)sizeof(float);
  c->h_bytes = h_count * (int64_t)sizeof(float);
  if (cudaMalloc(&c->phi, (size_t)c->phi_bytes) != cudaSuccess ||
      cudaMalloc(&c->h, (size_t)c->h_bytes) != cudaSuccess) {
    cudaGetLastError();
    return ABG_OK;  // the destructor frees whichever allocation succeeded
  }
  ABG_CUDA(cudaMemcpyAsync(c->phi, phi, (size_t)c->phi_bytes, cudaMemcpyDeviceToDevice, s));
  ABG_CUDA(cudaMemcpyAsync(c->h, h, (size_t)c->h_bytes, cudaMemcpyDeviceToDevice, s));
  ABG_CUDA(cudaEventCreateWithFlags(&c->ready, cudaEventDisableTiming));
  ABG_CUDA(cudaEventRecord(c->ready, s));
  std::lock_guard<std::mutex> lk(g->zmu);
  if (g->phicache) g->footprint -= g->phicache->phi_bytes + g->phicache->h_bytes;
  g->phicache = c;
  g->footprint += c->phi_bytes + c->h_bytes;
  return ABG_OK;
}

int solve_batch(abg_graph* g, const RowSpace& rs, const std::vector<int>& ks,
                const std::vector<uint64_t>& seeds, const abg_params& p, int d, SolveOut& o,
                cudaEvent_t* ev, cudaStream_t s) {
  const int nseg = rs.nseg;
  const int64_t n = g->n_u;
  const int m = 2 * d;
  Scratch scr(s);
  // per-segment sizes first: building them waits for their upload
  std::vector<int> ls(nseg);
  for (int i = 0; i < nseg; ++i)
    ls[i] = (int)std::min<int64_t>({(int64_t)ks[i] + p.oversample, (int64_t)m, rs.h_n[i]});
  SegSizes ss;
  ABG_TRY(segsizes_build(&ss, ks, ls, seeds, scr, s));
  if (ev) ABG_CUDA(cudaEventRecord(ev[0], s));
  // ---- Algorithm 1 ----
  const int64_t ldz = round_up(d, 4);
  float* zhat = nullptr;
  const bool reuse = (p.options & ABG_REUSE_PROPAGATION) && nseg == 1;
  const bool reduced = d < g->d_u;
  ZKey key;
  key.alpha = p.alpha;
  key.gamma = p.gamma;
  key.d = d;
  key.bf16 = (p.precision & ABG_BF16_PROPAGATION) ? 1 : 0;
  key.oversample = reduced ? p.oversample : 0;
  key.power_iters = reduced ? p.power_iters : 0;
  key.seed = reduced ? seeds[0] : 0;
  if (reuse) {
    std::lock_guard<std::mutex> lk(g->zmu);
    if (g->zcache && g->zcache->key == key) o.zhold = g->zcache;
  }
  if (o.zhold) {  // Z_hat of an earlier solve with the same key: no reduction, no propagation
    ABG_CUDA(cudaStreamWaitEvent(s, o.zhold->ready, 0));
    zhat = o.zhold->buf;
    o.reused = 1;
    if (ev) ABG_CUDA(cudaEventRecord(ev[1], s));
    if (ev) ABG_CUDA(cudaEventRecord(ev[2], s));
  } else {
    const float* xf;
    const __nv_bfloat16* xb;
    int64_t ldx;
    ABG_TRY(prepare_attributes(g, rs, d, p.oversample, p.power_iters, seeds, scr, s, &xf, &xb,
                               &ldx, o.breakdowns, (p.precision & ABG_BF16_CONTRACT) != 0));
    ABG_TRY(scr.get(&zhat, (size_t)n * ldz));
    if (ev) ABG_CUDA(cudaEventRecord(ev[1], s));
    ABG_TRY(propagate(g, xf, xb, ldx, d, p.alpha, p.gamma, zhat, ldz, s,
                      (p.precision & ABG_BF16_PROPAGATION) != 0));
    if (ev) ABG_CUDA(cudaEventRecord(ev[2], s));
    if (reuse) ABG_TRY(zcache_store(g, key, zhat, n * ldz, s));
  }
  double* q;
  float* qt;
  ABG_TRY(scr.get(&q, (size_t)nseg * d * d));
  ABG_TRY(scr.get(&qt, (size_t)nseg * d * ldz));
  ABG_TRY(orthogonal_matrices(nseg, ss.seed, d, q, s));
  ABG_TRY(transpose_blocks(nseg, d, q, qt, ldz, s));
  const int64_t ldr = round_up(m, 4);
  float* R;
  ABG_TRY(scr.get(&R, (size_t)n * ldr));
  __nv_bfloat16* R16 = nullptr;  // BF16 copy of R for the products with R
  const int64_t ldr16 = round_up(m, 8);
  if (p.precision & ABG_BF16_CONTRACT) ABG_TRY(scr.get(&R16, (size_t)n * ldr16));
  ABG_TRY(random_features(rs, zhat, d, ldz, qt, ldz, R, ldr, o.clamped, s, R16, ldr16));
  if (ev) ABG_CUDA(cudaEventRecord(ev[3], s));
  // ---- Algorithm 2 ----
  const int kmax = ss.k_max;
  const int64_t kk = round_up(kmax, 4);
  const int64_t hseg = (int64_t)m * kk;
  float *phi, *H;
  ABG_TRY(scr.get(&phi, (size_t)n * kk));
  ABG_TRY(scr.get(&H, (size_t)nseg * hseg));
  RsvdIn in;
  in.rows = &rs;
  in.m = m;
  in.A = R;
  in.lda = ldr;
  in.A16 = R16;
  in.lda16 = ldr16;
  RsvdOut out;
  out.left = phi;
  out.ldl = kk;
  out.left_mode = 0;
  out.right = H;
  out.ldr = kk;
  out.rseg = hseg;
  const bool warm = (p.options & ABG_WARM_START) && nseg == 1;
  if (warm) {
    std::lock_guard<std::mutex> lk(g->zmu);
    if (g->phicache && g->phicache->k == kmax && g->phicache->d == d) o.phold = g->phicache;
  }
  if (o.phold) {  // Phi, H at the end of an earlier solve's ONMF steps: no seeding (Eq. 18)
    ABG_CUDA(cudaStreamWaitEvent(s, o.phold->ready, 0));
    ABG_CUDA(cudaMemcpyAsync(phi, o.phold->phi, (size_t)o.phold->phi_bytes,
                             cudaMemcpyDeviceToDevice, s));
    ABG_CUDA(cudaMemcpyAsync(H, o.phold->h, (size_t)o.phold->h_bytes, cudaMemcpyDeviceToDevice,
                             s));
    o.warm = 1;
  } else {
    ABG_TRY(rsvd(in, ss, 0, p.power_iters, ABG_STREAM_OMEGA_R, out, o.breakdowns, s));
  }
  ABG_TRY(onmf_iterations(rs, ss, R, m, ldr, p.t_f, phi, kk, H, kk, hseg, s, R16, ldr16));
  if (warm) ABG_TRY(phicache_store(g, kmax, d, phi, n * kk, H, hseg, s));
  if (ev) ABG_CUDA(cudaEventRecord(ev[4], s));
  // ---- Algorithm 3 ----
  ABG_TRY(nci_run(rs, ss, phi, kk, p.t_g, p.nci_flags, o.labels, nullptr, nullptr, o.counters,
                  &o.passes, s));
  if (ev) ABG_CUDA(cudaEventRecord(ev[5], s));
  // ---- Eq. 8 ----
  ABG_TRY(objective(rs, ss, R, m, ldr, o.labels, o.obj, s));
  if (ev) ABG_CUDA(cudaEventRecord(ev[6], s));
  return ABG_OK;
}

int rowspace_of(const abg_graph* g, RowSpace* rs, Scratch& scr, cudaStream_t s) {
  return rowspace_build(rs, g->seg_row0, g->seg_n, scr, s);
}

// Run the batched solve of g (one parameter set per segment) and bring results to the host.
int cluster_impl(abg_graph* g, const abg_params* ps, int np, cudaStream_t s, int32_t* labels,
                 abg_result* res) {
  SolveHooks hooks;
  ABG_CHECK(g && ps && labels, "null argument");
  ABG_CHECK(np == g->nseg, "need one parameter set per segment (%d given, %d segments)", np, g->nseg);
  int d = 0;
  for (int i = 0; i < np; ++i) {
    int di = 0;
    ABG_TRY(check_params(g, &ps[i], g->seg_n[i], &di));
    if (i == 0) d = di;
    ABG_CHECK(di == d && ps[i].alpha == ps[0].alpha && ps[i].gamma == ps[0].gamma &&
                  ps[i].t_f == ps[0].t_f && ps[i].t_g == ps[0].t_g &&
                  ps[i].oversample == ps[0].oversample && ps[i].power_iters == ps[0].power_iters &&
                  ps[i].nci_flags == ps[0].nci_flags && ps[i].precision == ps[0].precision,
              "batched solves need the same d, alpha, gamma, t_f, t_g, oversample, power_iters, "
              "nci_flags, precision");
  }
  ABG_CUDA(cudaSetDevice(g->device));
  const int nseg = g->nseg;
  std::vector<int> ks(nseg);
  std::vector<uint64_t> seeds(nseg);
  for (int i = 0; i < nseg; ++i) {
    ks[i] = ps[i].k;
    seeds[i] = ps[i].seed;
  }
  Ev e[7];
  cudaEvent_t ev[7];
  for (int i = 0; i < 7; ++i) ev[i] = e[i].e;
  std::vector<double> obj(2 * nseg);
  std::vector<int> cnt(3 * nseg), cl(nseg), passes;
  int reused = 0, warm = 0;
  int bd = 0;
  {
    Scratch scr(s);
    RowSpace rs;
    ABG_TRY(rowspace_of(g, &rs, scr, s));
    SolveOut o;
    ABG_TRY(scr.get(&o.labels, (size_t)g->n_u));
    ABG_TRY(scr.get(&o.obj, (size_t)2 * nseg));
    ABG_TRY(scr.get(&o.counters, (size_t)3 * nseg));
    ABG_TRY(scr.get(&o.clamped, (size_t)nseg));
    ABG_TRY(scr.get(&o.breakdowns, 1));
    ABG_CUDA(cudaMemsetAsync(o.clamped, 0, sizeof(int) * nseg, s));
    ABG_CUDA(cudaMemsetAsync(o.breakdowns, 0, sizeof(int), s));
    int* tc_flag;  // this solve's own report of a tensor-core wait that ran out
    ABG_TRY(scr.get(&tc_flag, 1));
    ABG_CUDA(cudaMemsetAsync(tc_flag, 0, sizeof(int), s));
    TcFlagScope tc_scope(tc_flag);
    const int st = solve_batch(g, rs, ks, seeds, ps[0], d, o, ev, s);
    if (st != ABG_OK) {  // a wait that ran out explains a later failure, and is cleared here
      const int wst = check_wait_flag(g, s);
      return wst != ABG_OK ? wst : st;
    }
    passes = o.passes;
    reused = o.reused;
    warm = o.warm;
    ABG_CUDA(cudaMemcpyAsync(labels, o.labels, sizeof(int32_t) * g->n_u, cudaMemcpyDefault, s));
    ABG_CUDA(cudaMemcpyAsync(obj.data(), o.obj, sizeof(double) * 2 * nseg, cudaMemcpyDeviceToHost, s));
    ABG_CUDA(cudaMemcpyAsync(cnt.data(), o.counters, sizeof(int) * 3 * nseg, cudaMemcpyDeviceToHost, s));
    ABG_CUDA(cudaMemcpyAsync(cl.data(), o.clamped, sizeof(int) * nseg, cudaMemcpyDeviceToHost, s));
    ABG_CUDA(cudaMemcpyAsync(&bd, o.breakdowns, sizeof(int), cudaMemcpyDeviceToHost, s));
    ABG_CUDA(cudaStreamSynchronize(s));
    ABG_TRY(check_wait_flag(g, s));
  }
  ABG_CUDA(cudaStreamSynchronize(s));
  ABG_CUDA(cudaGetLastError());
  float ms[6];
  for (int i = 0; i < 6; ++i) cudaEventElapsedTime(&ms[i], ev[i], ev[i + 1]);
  bool finite = true;
  for (int i = 0; i < nseg; ++i) {
    abg_result r{};
    r.objective = obj[2 * i];
    r.trace_obj = obj[2 * i + 1];
    r.last_changes = ps[i].t_g > 0 ? cnt[i] : 0;
    unsigned b = (unsigned)cnt[nseg + i];
    float f;
    memcpy(&f, &b, sizeof(f));
    r.min_margin = ps[i].t_g > 0 ? f : INFINITY;
    r.empty_clusters = ps[i].t_g > 0 ? cnt[2 * nseg + i] : ps[i].k - 1;
    r.clamped_rows = cl[i];
    r.chol_breakdowns = bd;
    r.nci_passes = i < (int)passes.size() ? passes[i] : ps[i].t_g;
    r.reused_propagation = reused;
    r.warm_started = warm;
    for (int j = 0; j < 6; ++j) r.ms_phase[j] = ms[j];
    finite &= std::isfinite(r.objective);
    if (res) res[i] = r;
  }
  if (!finite) {
    set_error("objective is not finite");
    return ABG_ENUMERIC;
  }
  return ABG_OK;
}

// One-segment row space over n rows.
int single_rows(int64_t n, RowSpace* rs, Scratch& scr, cudaStream_t s) {
  return rowspace_build(rs, std::vector<int64_t>{0}, std::vector<int64_t>{n}, scr, s);
}

}  // namespace

extern "C" {

ABG_API void abg_params_default(abg_params* p) {
  if (!p) return;
  p->k = 2;
  p->gamma = 6;
  p->d = 0;
  p->t_f = 5;
  p->t_g = 20;
  p->oversample = 10;
  p->power_iters = 4;
  p->nci_flags = 0;
  p->alpha = 0.6;
  p->seed = 0;
  p->precision = ABG_PRECISION_FP32;
  p->options = 0;
}

ABG_API int64_t abg_solve_footprint(const abg_graph* g, const abg_params* p) {
  int d = 0;
  if (!g || !p || check_params(g, p, g->n_u, &d) != ABG_OK) return -1;
  const int64_t n = g->n_u;
  const int64_t ld = round_up(d, 4), ldr = round_up(2 * d, 4), kk = round_up(p->k, 4);
  const int64_t l = std::min<int64_t>(p->k + p->oversample, 2 * d);
  const int64_t ll = round_up(l, 4);
  int64_t b = 0;
  b += 4 * n * ld;                       // Z_hat
  if (p->precision & ABG_BF16_PROPAGATION)  // W and the intermediate Z in BF16
    b += 2 * round_up(d, 8) * (g->n_v + (p->gamma > 1 ? n : 0));
  else
    b += 4 * g->n_v * ld;                // W
  b += 4 * n * ldr;                      // R
  if (p->precision & ABG_BF16_CONTRACT) b += 2 * n * round_up(2 * d, 8);  // BF16 copy of R
  b += 4 * n * ll * 2;                   // randomized SVD blocks
  b += 4 * n * kk * 4;                   // Phi (x2), P, spare
  b += 8 * n;                            // labels, row segments
  b += 4 * (ceil_div(n, 2048) + g->nseg) * std::max<int64_t>(2 * d, 128) * std::max<int64_t>(kk, ll);
  if (d < g->d_u) b += 4 * n * (ld + round_up(d + p->oversample, 4) * 2 + g->ldx);
  else if (g->x_kind == ABG_X_CSR_F32) b += 4 * n * ld;
  return b + (64 << 20);
}

ABG_API int abg_cluster(abg_graph* g, const abg_params* p, void* stream, int32_t* labels,
                        abg_result* res) {
  ABG_CHECK(g, "null graph");
  if (g->nseg != 1) {
    set_error("abg_cluster on a batch: use abg_batch_cluster (one parameter set per graph)");
    return ABG_EINVAL;
  }
  return cluster_impl(g, p, 1, (cudaStream_t)stream, labels, res);
}

ABG_API int abg_batch_cluster(abg_graph* batch, const abg_params* params, void* stream,
                              int32_t* labels, abg_result* results) {
  ABG_CHECK(batch, "null batch");
  return cluster_impl(batch, params, batch->nseg, (cudaStream_t)stream, labels, results);
}

ABG_API int abg_reduce_attributes(const abg_graph* g, int32_t d, int32_t oversample,
                                  int32_t power_iters, uint64_t seed, float* x_out, int64_t ldo,
                                  void* stream) {
  ABG_CHECK(g && x_out, "null argument");
  ABG_CHECK(d >= 1 && d < g->d_u && d + oversample <= 1024 && oversample >= 0 && power_iters >= 0,
            "need 1 <= d < d_u, d + oversample <= 1024");
  ABG_CHECK(ldo >= d && ldo % 4 == 0, "ldo must be >= d and a multiple of 4");
  ABG_CUDA(cudaSetDevice(g->device));
  cudaStream_t s = (cudaStream_t)stream;
  Scratch scr(s);
  RowSpace rs;
  ABG_TRY(rowspace_of(g, &rs, scr, s));
  int* bd;
  ABG_TRY(scr.get(&bd, 1));
  ABG_CUDA(cudaMemsetAsync(bd, 0, sizeof(int), s));
  const float* xf;
  const __nv_bfloat16* xb;
  int64_t ldx;
  std::vector<uint64_t> seeds(g->nseg, seed);
  ABG_TRY(prepare_attributes(g, rs, d, oversample, power_iters, seeds, scr, s, &xf, &xb, &ldx, bd));
  ABG_CUDA(cudaMemcpy2DAsync(x_out, sizeof(float) * ldo, xf, sizeof(float) * ldx, sizeof(float) * d,
                             g->n_u, cudaMemcpyDeviceToDevice, s));
  return ABG_OK;
}

ABG_API int abg_propagate(const abg_graph* g, const float* x, int64_t ldx, int32_t d, double alpha,
                          int32_t gamma, int32_t precision, float* zhat, int64_t ldz,
                          void* stream) {
  ABG_CHECK(g && zhat, "null argument");
  ABG_CHECK(precision == ABG_PRECISION_FP32 || precision == ABG_BF16_PROPAGATION,
            "unknown precision %d", precision);
  const bool bf16 = precision == ABG_BF16_PROPAGATION;
  ABG_CUDA(cudaSetDevice(g->device));
  cudaStream_t s = (cudaStream_t)stream;
  if (x) {
    ABG_TRY(propagate(g, x, nullptr, ldx, d, alpha, gamma, zhat, ldz, s, bf16));
    return check_wait_flag(g, s);
  }
  ABG_CHECK(d == g->d_u, "x = NULL needs d == d_u");
  Scratch scr(s);
  RowSpace rs;
  ABG_TRY(rowspace_of(g, &rs, scr, s));
  const float* xf;
  const __nv_bfloat16* xb;
  int64_t lx;
  std::vector<uint64_t> seeds(g->nseg, 0);
  ABG_TRY(prepare_attributes(g, rs, d, 0, 0, seeds, scr, s, &xf, &xb, &lx, nullptr));
  ABG_TRY(propagate(g, xf, xb, lx, d, alpha, gamma, zhat, ldz, s, bf16));
  return check_wait_flag(g, s);
}

ABG_API int abg_orthogonal_matrix(uint64_t seed, int32_t d, double* q_out, void* stream) {
  ABG_CHECK(q_out, "null output");
  cudaStream_t s = (cudaStream_t)stream;
  Scratch scr(s);
  SegSizes ss;
  ABG_TRY(segsizes_build(&ss, {1}, {1}, {seed}, scr, s));
  return orthogonal_matrices(1, ss.seed, d, q_out, s);
}

ABG_API int abg_random_features(const float* zhat, int64_t n, int32_t d, int64_t ldz, uint64_t seed,
                                float* r_out, int64_t ldr, int32_t* clamped, void* stream) {
  ABG_CHECK(zhat && r_out && n >= 1 && d >= 1 && d <= kMaxD, "bad arguments");
  ABG_CHECK(ldz >= d && ldz % 4 == 0, "ldz must be >= d and a multiple of 4");
  cudaStream_t s = (cudaStream_t)stream;
  Scratch scr(s);
  RowSpace rs;
  ABG_TRY(single_rows(n, &rs, scr, s));
  SegSizes ss;
  ABG_TRY(segsizes_build(&ss, {1}, {1}, {seed}, scr, s));
  double* q;
  float* qt;
  const int64_t ldq = round_up(d, 4);
  ABG_TRY(scr.get(&q, (size_t)d * d));
  ABG_TRY(scr.get(&qt, (size_t)d * ldq));
  ABG_TRY(orthogonal_matrices(1, ss.seed, d, q, s));
  ABG_TRY(transpose_blocks(1, d, q, qt, ldq, s));
  int* cl;
  ABG_TRY(scr.get(&cl, 1));
  ABG_CUDA(cudaMemsetAsync(cl, 0, sizeof(int), s));
  ABG_TRY(random_features(rs, zhat, d, ldz, qt, ldq, r_out, ldr, cl, s));
  if (clamped) {
    ABG_CUDA(cudaMemcpyAsync(clamped, cl, sizeof(int), cudaMemcpyDeviceToHost, s));
    ABG_CUDA(cudaStreamSynchronize(s));
  }
  return ABG_OK;
}

ABG_API int abg_seed_factors(const float* r, int64_t n, int32_t m, int64_t ldr, int32_t k,
                             int32_t oversample, int32_t power_iters, uint64_t seed,
                             float* phi_out, int64_t ldphi, float* h_out, int64_t ldh,
                             double* sigma_out, int32_t precision, void* stream) {
  ABG_CHECK(r && phi_out && h_out && n >= 1 && m >= 1, "bad arguments");
  ABG_CHECK(k >= 1 && k <= m && k <= n && k <= kMaxK, "need 1 <= k <= min(n, m, %d)", kMaxK);
  ABG_CHECK(ldr >= m && ldr % 4 == 0 && ldphi >= k && ldphi % 4 == 0 && ldh >= k && ldh % 4 == 0,
            "leading dimensions must cover the width and be multiples of 4");
  ABG_CHECK(oversample >= 0 && power_iters >= 0 && k + oversample <= 1024, "bad SVD parameters");
  cudaStream_t s = (cudaStream_t)stream;
  Scratch scr(s);
  RowSpace rs;
  ABG_TRY(single_rows(n, &rs, scr, s));
  const int l = (int)std::min<int64_t>({(int64_t)k + oversample, (int64_t)m, n});
  SegSizes ss;
  ABG_TRY(segsizes_build(&ss, {k}, {l}, {seed}, scr, s));
  int* bd;
  ABG_TRY(scr.get(&bd, 1));
  ABG_CUDA(cudaMemsetAsync(bd, 0, sizeof(int), s));
  ABG_CHECK(precision == ABG_PRECISION_FP32 || precision == ABG_BF16_CONTRACT,
            "unknown precision %d", precision);
  RsvdIn in;
  in.rows = &rs;
  in.m = m;
  in.A = r;
  in.lda = ldr;
  if (precision == ABG_BF16_CONTRACT) {
    __nv_bfloat16* r16;
    in.lda16 = round_up(m, 8);
    ABG_TRY(scr.get(&r16, (size_t)n * in.lda16));
    ABG_TRY(f32_to_bf16(r, ldr, n, m, r16, in.lda16, s));
    in.A16 = r16;
  }
  RsvdOut out;
  out.left = phi_out;
  out.ldl = ldphi;
  out.left_mode = 0;
  out.right = h_out;
  out.ldr = ldh;
  out.sigma = sigma_out;
  return rsvd(in, ss, 0, power_iters, ABG_STREAM_OMEGA_R, out, bd, s);
}

ABG_API int abg_onmf(const float* r, int64_t n, int32_t m, int64_t ldr, int32_t k, int32_t t_f,
                     float* phi, int64_t ldphi, float* h, int64_t ldh, int32_t precision,
                     void* stream) {
  ABG_CHECK(r && phi && h && n >= 1 && m >= 1 && k >= 1 && k <= kMaxK && t_f >= 0, "bad arguments");
  ABG_CHECK(ldr >= m && ldr % 4 == 0 && ldphi >= k && ldphi % 4 == 0 && ldh >= k && ldh % 4 == 0,
            "leading dimensions must cover the width and be multiples of 4");
  cudaStream_t s = (cudaStream_t)stream;
  Scratch scr(s);
  RowSpace rs;
  ABG_TRY(single_rows(n, &rs, scr, s));
  SegSizes ss;
  ABG_TRY(segsizes_build(&ss, {k}, {k}, {0}, scr, s));
  ABG_CHECK(precision == ABG_PRECISION_FP32 || precision == ABG_BF16_CONTRACT,
            "unknown precision %d", precision);
  __nv_bfloat16* r16 = nullptr;
  const int64_t ld16 = round_up(m, 8);
  if (precision == ABG_BF16_CONTRACT) {
    ABG_TRY(scr.get(&r16, (size_t)n * ld16));
    ABG_TRY(f32_to_bf16(r, ldr, n, m, r16, ld16, s));
  }
  return onmf_iterations(rs, ss, r, m, ldr, t_f, phi, ldphi, h, ldh, (int64_t)m * ldh, s, r16,
                         ld16);
}

ABG_API int abg_nci(const float* phi, int64_t n, int32_t k, int64_t ldphi, int32_t t_g,
                    int32_t nci_flags, int32_t* labels_out, float* margin_out, double* t_out,
                    int32_t* last_changes, int32_t* passes, void* stream) {
  ABG_CHECK(phi && labels_out && n >= 1 && t_g >= 0 && k >= 1 && k <= kMaxK, "bad arguments");
  ABG_CHECK(ldphi >= k && ldphi % 4 == 0, "ldphi must be >= k and a multiple of 4");
  cudaStream_t s = (cudaStream_t)stream;
  Scratch scr(s);
  RowSpace rs;
  ABG_TRY(single_rows(n, &rs, scr, s));
  SegSizes ss;
  ABG_TRY(segsizes_build(&ss, {k}, {k}, {0}, scr, s));
  int* counters;
  ABG_TRY(scr.get(&counters, 3));
  ABG_CHECK((nci_flags & ~(ABG_NCI_PROCRUSTES | ABG_NCI_EARLY_STOP)) == 0, "unknown nci_flags");
  std::vector<int> np;
  ABG_TRY(nci_run(rs, ss, phi, ldphi, t_g, nci_flags, labels_out, margin_out, t_out, counters, &np,
                  s));
  int host[3] = {0, 0, 0};
  ABG_CUDA(cudaMemcpyAsync(host, counters, sizeof(int) * 3, cudaMemcpyDeviceToHost, s));
  ABG_CUDA(cudaStreamSynchronize(s));
  if (last_changes) *last_changes = t_g > 0 ? host[0] : 0;
  if (passes) *passes = np.empty() ? t_g : np[0];
  return ABG_OK;
}

ABG_API int abg_objective(const float* r, int64_t n, int32_t m, int64_t ldr, const int32_t* labels,
                          int32_t k, double* obj, void* stream) {
  ABG_CHECK(r && labels && obj && n >= 1 && m >= 1 && k >= 1 && k <= kMaxK, "bad arguments");
  ABG_CHECK(ldr >= m && ldr % 4 == 0, "ldr must be >= m and a multiple of 4");
  cudaStream_t s = (cudaStream_t)stream;
  Scratch scr(s);
  RowSpace rs;
  ABG_TRY(single_rows(n, &rs, scr, s));
  SegSizes ss;
  ABG_TRY(segsizes_build(&ss, {k}, {k}, {0}, scr, s));
  double* out;
  ABG_TRY(scr.get(&out, 2));
  ABG_TRY(objective(rs, ss, r, m, ldr, labels, out, s));
  ABG_CUDA(cudaMemcpyAsync(obj, out, sizeof(double) * 2, cudaMemcpyDeviceToHost, s));
  ABG_CUDA(cudaStreamSynchronize(s));
  return ABG_OK;
}

}  // extern "C"
