// The whole method (Algorithms 1-3) and the step-level entry points of abg.h.
#include <algorithm>
#include <cmath>

#include "internal.cuh"

using namespace abg;

namespace {

struct Ev {
  cudaEvent_t e = nullptr;
  Ev() { cudaEventCreate(&e); }
  ~Ev() {
    if (e) cudaEventDestroy(e);
  }
};

int check_params(const abg_graph* g, const abg_params* p, int* d_eff) {
  ABG_CHECK(g && p, "null graph or parameters");
  const int d = p->d == 0 ? g->d_u : p->d;
  ABG_CHECK(d >= 1 && d <= g->d_u, "need 1 <= d <= d_u (got d=%d, d_u=%d)", d, g->d_u);
  ABG_CHECK(d <= kMaxD, "d must be <= %d", kMaxD);
  ABG_CHECK(p->alpha >= 0.0 && p->alpha < 1.0, "need 0 <= alpha < 1");
  ABG_CHECK(p->gamma >= 0 && p->t_f >= 0 && p->t_g >= 0, "gamma, t_f, t_g must be >= 0");
  ABG_CHECK(p->oversample >= 0 && p->power_iters >= 0, "oversample, power_iters must be >= 0");
  ABG_CHECK(p->k >= 1 && p->k <= kMaxK && p->k <= 2 * d && p->k <= g->n_u,
            "need 1 <= k <= min(|U|, 2d, %d) (got k=%d)", kMaxK, p->k);
  ABG_CHECK(d == g->d_u || (int64_t)d + p->oversample <= 1024,
            "attribute reduction needs d + oversample <= 1024");
  *d_eff = d;
  return ABG_OK;
}

// Attributes the propagation reads: the graph's own (dense), a densified CSR,
// or the SVD-reduced X' of Eq. 15.
int prepare_attributes(const abg_graph* g, int d, int oversample, int power_iters, uint64_t seed,
                       Scratch& scr, cudaStream_t s, const float** xf, const __nv_bfloat16** xb,
                       int64_t* ldx, int* breakdowns) {
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
  RsvdIn in;
  in.n = g->n_u;
  in.m = g->d_u;
  if (g->x_kind == ABG_X_CSR_F32) {
    in.ptr = g->x_ptr;
    in.col = g->x_col;
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
  }
  RsvdOut out;
  out.left = xr;
  out.ldl = ldo;
  out.left_mode = 1;
  ABG_TRY(rsvd(in, d, oversample, power_iters, seed, ABG_STREAM_OMEGA_X, out, breakdowns, scr, s));
  *xf = xr;
  *ldx = ldo;
  return ABG_OK;
}

int onmf_iterations(const float* R, int64_t n, int m, int64_t ldr, int k, int t_f, float* phi,
                    int64_t ldphi, float* H, int64_t ldh, Scratch& scr, cudaStream_t s) {
  if (t_f == 0) return ABG_OK;
  float *P, *phi2, *C32;
  double *A, *G, *C;
  ABG_TRY(scr.get(&P, (size_t)n * ldphi));
  ABG_TRY(scr.get(&phi2, (size_t)n * ldphi));
  ABG_TRY(scr.get(&C32, (size_t)k * ldphi));
  ABG_TRY(scr.get(&A, (size_t)m * k));
  ABG_TRY(scr.get(&G, (size_t)k * k));
  ABG_TRY(scr.get(&C, (size_t)k * k));
  float* cur = phi;
  float* nxt = phi2;
  for (int t = 0; t < t_f; ++t) {
    // Eq. 16: H <- H * (R^T Phi) / (H (Phi^T Phi))
    ABG_TRY(gemm_tn(n, m, k, R, ldr, cur, ldphi, A, k, scr, s));
    ABG_TRY(gemm_tn(n, k, k, cur, ldphi, cur, ldphi, G, k, scr, s));
    ABG_TRY(nmf_update_h(m, k, H, ldh, A, k, G, k, s));
    // Eq. 17: Phi <- Phi * sqrt((R H) / (Phi (Phi^T (R H))))
    ABG_TRY(gemm_nn(n, k, m, R, ldr, H, ldh, P, ldphi, Epi::Store, nullptr, 0, nullptr, 0, nullptr,
                    s));
    ABG_TRY(gemm_tn(n, k, k, cur, ldphi, P, ldphi, C, k, scr, s));
    ABG_TRY(convert_f64_to_f32(C, k, k, k, C32, ldphi, s));
    ABG_TRY(gemm_nn(n, k, k, cur, ldphi, C32, ldphi, nxt, ldphi, Epi::PhiUpdate, P, ldphi, cur,
                    ldphi, nullptr, s));
    std::swap(cur, nxt);
  }
  if (cur != phi)
    ABG_CUDA(cudaMemcpyAsync(phi, cur, sizeof(float) * n * ldphi, cudaMemcpyDeviceToDevice, s));
  return ABG_OK;
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
  p->reserved0 = 0;
  p->alpha = 0.6;
  p->seed = 0;
}

ABG_API int64_t abg_solve_footprint(const abg_graph* g, const abg_params* p) {
  int d = 0;
  if (!g || !p || check_params(g, p, &d) != ABG_OK) return -1;
  const int64_t n = g->n_u;
  const int64_t ld = round_up(d, 4), ldr = round_up(2 * d, 4), kk = round_up(p->k, 4);
  const int64_t l = std::min<int64_t>(p->k + p->oversample, 2 * d);
  const int64_t ll = round_up(l, 4);
  int64_t b = 0;
  b += 4 * n * ld;                       // Z_hat
  b += 4 * g->n_v * ld;                  // W
  b += 4 * n * ldr;                      // R
  b += 4 * n * ll * 2;                   // randomized SVD blocks
  b += 4 * n * kk * 4;                   // Phi (x2), P, spare
  b += 8 * n;                            // labels
  b += 4 * (ceil_div(n, 2048) + 1) * (int64_t)std::max(2 * d, 128) * 128;  // chunk partials
  if (d < g->d_u) b += 4 * n * (ld + round_up(d + p->oversample, 4) * 2 + g->ldx);
  else if (g->x_kind == ABG_X_CSR_F32) b += 4 * n * ld;
  return b + (64 << 20);
}

ABG_API int abg_cluster(abg_graph* g, const abg_params* p, void* stream, int32_t* labels,
                        abg_result* res) {
  int d = 0;
  ABG_TRY(check_params(g, p, &d));
  ABG_CHECK(labels, "null labels buffer");
  ABG_CUDA(cudaSetDevice(g->device));
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t n = g->n_u;
  const int k = p->k;
  Ev e0, e1, e2, e3, e4, e5, e6;
  int* bd;
  abg_result r{};
  {
    Scratch scr(s);
    ABG_TRY(scr.get(&bd, 1));
    ABG_CUDA(cudaMemsetAsync(bd, 0, sizeof(int), s));
    ABG_CUDA(cudaEventRecord(e0.e, s));
    // ---- Algorithm 1 ----
    const float* xf;
    const __nv_bfloat16* xb;
    int64_t ldx;
    ABG_TRY(prepare_attributes(g, d, p->oversample, p->power_iters, p->seed, scr, s, &xf, &xb, &ldx,
                               bd));
    const int64_t ldz = round_up(d, 4);
    float* zhat;
    ABG_TRY(scr.get(&zhat, (size_t)n * ldz));
    ABG_CUDA(cudaEventRecord(e1.e, s));
    ABG_TRY(propagate(g, xf, xb, ldx, d, p->alpha, p->gamma, zhat, ldz, s));
    ABG_CUDA(cudaEventRecord(e2.e, s));
    double* q;
    float* qt;
    ABG_TRY(scr.get(&q, (size_t)d * d));
    ABG_TRY(scr.get(&qt, (size_t)d * ldz));
    ABG_TRY(orthogonal_matrix(p->seed, d, q, s));
    ABG_TRY(transpose_f64_to_f32(q, d, d, d, qt, ldz, s));
    const int m = 2 * d;
    const int64_t ldr = round_up(m, 4);
    float* R;
    ABG_TRY(scr.get(&R, (size_t)n * ldr));
    int* clamped;
    ABG_TRY(scr.get(&clamped, 1));
    ABG_CUDA(cudaMemsetAsync(clamped, 0, sizeof(int), s));
    ABG_TRY(random_features(zhat, n, d, ldz, qt, R, ldr, clamped, scr, s));
    ABG_CUDA(cudaEventRecord(e3.e, s));
    // ---- Algorithm 2 ----
    const int64_t kk = round_up(k, 4);
    float *phi, *H;
    ABG_TRY(scr.get(&phi, (size_t)n * kk));
    ABG_TRY(scr.get(&H, (size_t)m * kk));
    RsvdIn in;
    in.n = n;
    in.m = m;
    in.A = R;
    in.lda = ldr;
    RsvdOut out;
    out.left = phi;
    out.ldl = kk;
    out.left_mode = 0;
    out.right = H;
    out.ldr = kk;
    ABG_TRY(rsvd(in, k, p->oversample, p->power_iters, p->seed, ABG_STREAM_OMEGA_R, out, bd, scr, s));
    ABG_TRY(onmf_iterations(R, n, m, ldr, k, p->t_f, phi, kk, H, kk, scr, s));
    ABG_CUDA(cudaEventRecord(e4.e, s));
    // ---- Algorithm 3 ----
    int32_t* lab;
    ABG_TRY(scr.get(&lab, (size_t)n));
    float minm = INFINITY;
    ABG_TRY(nci_run(phi, n, k, kk, p->t_g, lab, nullptr, nullptr, &r.last_changes, &minm,
                    &r.empty_clusters, scr, s));
    r.min_margin = minm;
    ABG_CUDA(cudaEventRecord(e5.e, s));
    // ---- Eq. 8 ----
    double obj[2] = {0, 0};
    ABG_TRY(objective(R, n, m, ldr, lab, k, obj, scr, s));
    r.objective = obj[0];
    r.trace_obj = obj[1];
    ABG_CUDA(cudaEventRecord(e6.e, s));
    ABG_CUDA(cudaMemcpyAsync(labels, lab, sizeof(int32_t) * n, cudaMemcpyDefault, s));
    ABG_CUDA(cudaMemcpyAsync(&r.chol_breakdowns, bd, sizeof(int), cudaMemcpyDeviceToHost, s));
    ABG_CUDA(cudaMemcpyAsync(&r.clamped_rows, clamped, sizeof(int), cudaMemcpyDeviceToHost, s));
  }
  ABG_CUDA(cudaStreamSynchronize(s));
  ABG_CUDA(cudaGetLastError());
  cudaEvent_t ev[7] = {e0.e, e1.e, e2.e, e3.e, e4.e, e5.e, e6.e};
  for (int i = 0; i < 6; ++i) cudaEventElapsedTime(&r.ms_phase[i], ev[i], ev[i + 1]);
  if (!std::isfinite(r.objective)) {
    set_error("objective is not finite");
    if (res) *res = r;
    return ABG_ENUMERIC;
  }
  if (res) *res = r;
  return ABG_OK;
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
  int* bd;
  ABG_TRY(scr.get(&bd, 1));
  ABG_CUDA(cudaMemsetAsync(bd, 0, sizeof(int), s));
  const float* xf;
  const __nv_bfloat16* xb;
  int64_t ldx;
  ABG_TRY(prepare_attributes(g, d, oversample, power_iters, seed, scr, s, &xf, &xb, &ldx, bd));
  ABG_CUDA(cudaMemcpy2DAsync(x_out, sizeof(float) * ldo, xf, sizeof(float) * ldx, sizeof(float) * d,
                             g->n_u, cudaMemcpyDeviceToDevice, s));
  return ABG_OK;
}

ABG_API int abg_propagate(const abg_graph* g, const float* x, int64_t ldx, int32_t d, double alpha,
                          int32_t gamma, float* zhat, int64_t ldz, void* stream) {
  ABG_CHECK(g && zhat, "null argument");
  ABG_CUDA(cudaSetDevice(g->device));
  cudaStream_t s = (cudaStream_t)stream;
  if (x) return propagate(g, x, nullptr, ldx, d, alpha, gamma, zhat, ldz, s);
  ABG_CHECK(d == g->d_u, "x = NULL needs d == d_u");
  Scratch scr(s);
  const float* xf;
  const __nv_bfloat16* xb;
  int64_t lx;
  ABG_TRY(prepare_attributes(g, d, 0, 0, 0, scr, s, &xf, &xb, &lx, nullptr));
  return propagate(g, xf, xb, lx, d, alpha, gamma, zhat, ldz, s);
}

ABG_API int abg_orthogonal_matrix(uint64_t seed, int32_t d, double* q_out, void* stream) {
  ABG_CHECK(q_out, "null output");
  return orthogonal_matrix(seed, d, q_out, (cudaStream_t)stream);
}

ABG_API int abg_random_features(const float* zhat, int64_t n, int32_t d, int64_t ldz, uint64_t seed,
                                float* r_out, int64_t ldr, int32_t* clamped, void* stream) {
  ABG_CHECK(zhat && r_out && n >= 1 && d >= 1 && d <= kMaxD, "bad arguments");
  ABG_CHECK(ldz >= d && ldz % 4 == 0, "ldz must be >= d and a multiple of 4");
  cudaStream_t s = (cudaStream_t)stream;
  Scratch scr(s);
  double* q;
  float* qt;
  const int64_t ldq = round_up(d, 4);
  ABG_TRY(scr.get(&q, (size_t)d * d));
  ABG_TRY(scr.get(&qt, (size_t)d * ldq));
  ABG_TRY(orthogonal_matrix(seed, d, q, s));
  ABG_TRY(transpose_f64_to_f32(q, d, d, d, qt, ldq, s));
  int* cl;
  ABG_TRY(scr.get(&cl, 1));
  ABG_CUDA(cudaMemsetAsync(cl, 0, sizeof(int), s));
  ABG_TRY(random_features(zhat, n, d, ldz, qt, r_out, ldr, cl, scr, s));
  if (clamped) {
    ABG_CUDA(cudaMemcpyAsync(clamped, cl, sizeof(int), cudaMemcpyDeviceToHost, s));
    ABG_CUDA(cudaStreamSynchronize(s));
  }
  return ABG_OK;
}

ABG_API int abg_seed_factors(const float* r, int64_t n, int32_t m, int64_t ldr, int32_t k,
                             int32_t oversample, int32_t power_iters, uint64_t seed,
                             float* phi_out, int64_t ldphi, float* h_out, int64_t ldh,
                             double* sigma_out, void* stream) {
  ABG_CHECK(r && phi_out && h_out && n >= 1 && m >= 1, "bad arguments");
  ABG_CHECK(k >= 1 && k <= m && k <= n && k <= kMaxK, "need 1 <= k <= min(n, m, %d)", kMaxK);
  ABG_CHECK(ldr >= m && ldr % 4 == 0 && ldphi >= k && ldphi % 4 == 0 && ldh >= k && ldh % 4 == 0,
            "leading dimensions must cover the width and be multiples of 4");
  ABG_CHECK(oversample >= 0 && power_iters >= 0 && k + oversample <= 1024, "bad SVD parameters");
  cudaStream_t s = (cudaStream_t)stream;
  Scratch scr(s);
  int* bd;
  ABG_TRY(scr.get(&bd, 1));
  ABG_CUDA(cudaMemsetAsync(bd, 0, sizeof(int), s));
  RsvdIn in;
  in.n = n;
  in.m = m;
  in.A = r;
  in.lda = ldr;
  RsvdOut out;
  out.left = phi_out;
  out.ldl = ldphi;
  out.left_mode = 0;
  out.right = h_out;
  out.ldr = ldh;
  out.sigma = sigma_out;
  return rsvd(in, k, oversample, power_iters, seed, ABG_STREAM_OMEGA_R, out, bd, scr, s);
}

ABG_API int abg_onmf(const float* r, int64_t n, int32_t m, int64_t ldr, int32_t k, int32_t t_f,
                     float* phi, int64_t ldphi, float* h, int64_t ldh, void* stream) {
  ABG_CHECK(r && phi && h && n >= 1 && m >= 1 && k >= 1 && k <= kMaxK && t_f >= 0, "bad arguments");
  ABG_CHECK(ldr >= m && ldr % 4 == 0 && ldphi >= k && ldphi % 4 == 0 && ldh >= k && ldh % 4 == 0,
            "leading dimensions must cover the width and be multiples of 4");
  cudaStream_t s = (cudaStream_t)stream;
  Scratch scr(s);
  return onmf_iterations(r, n, m, ldr, k, t_f, phi, ldphi, h, ldh, scr, s);
}

ABG_API int abg_nci(const float* phi, int64_t n, int32_t k, int64_t ldphi, int32_t t_g,
                    int32_t* labels_out, float* margin_out, double* t_out, int32_t* last_changes,
                    void* stream) {
  ABG_CHECK(phi && labels_out && n >= 1 && t_g >= 0, "bad arguments");
  ABG_CHECK(ldphi >= k && ldphi % 4 == 0, "ldphi must be >= k and a multiple of 4");
  cudaStream_t s = (cudaStream_t)stream;
  Scratch scr(s);
  int lc = 0;
  ABG_TRY(nci_run(phi, n, k, ldphi, t_g, labels_out, margin_out, t_out, &lc, nullptr, nullptr, scr,
                  s));
  if (last_changes) *last_changes = lc;
  return ABG_OK;
}

ABG_API int abg_objective(const float* r, int64_t n, int32_t m, int64_t ldr, const int32_t* labels,
                          int32_t k, double* obj, void* stream) {
  ABG_CHECK(r && labels && obj && n >= 1 && m >= 1, "bad arguments");
  ABG_CHECK(ldr >= m && ldr % 4 == 0, "ldr must be >= m and a multiple of 4");
  cudaStream_t s = (cudaStream_t)stream;
  Scratch scr(s);
  return objective(r, n, m, ldr, labels, k, obj, scr, s);
}

}  // extern "C"
