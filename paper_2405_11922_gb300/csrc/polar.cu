// Orthogonal Procrustes factor of Algorithm 3's Phi^T Y (the constraint T T^T = I of
// Eq. 20) by the Newton-Schulz iteration, spread over a thread-block cluster.
//
// X_0 = M / |M|_F, X <- 1.5 X - 0.5 X (X^T X) (Newton-Schulz, Higham 1986 / Bjorck and
// Bowie 1971): every singular value of X follows p(s) = 1.5 s - 0.5 s^3, which takes any
// s in (0, 1] to 1 (quadratically at the end) and keeps 0 at 0, while the singular
// vectors stay those of M. So the limit is U_r V_r^T, the polar factor on M's range.
//
// The library's reading of the factor keeps the singular values above 1e-5 s_1 and drops
// the rest. An iteration stopped after N steps splits the singular values into those that
// reached 1 and those still small, and the stopping rule below makes that split agree with
// the 1e-5 s_1 threshold:
//   * the step norm |X_{N} - X_{N-1}|_F bounds |s - s^3| / 2 for every singular value s of
//     X_{N-1}; once it is <= eps every s lies within eps of 1 or below 2 eps;
//   * p(s) <= 1.5 s, so a value that reached 1 - eps after N steps started at
//     s_0 >= (1 - eps) 1.5^-(N-1) |M|_F, and a value still below 2 eps started at
//     s_0 <= 2 eps 1.5^-(N-1) |M|_F (p(s) ~ 1.5 s for small s);
//   * with eps = 1e-4, 15 <= N <= 28 and s_1 >= |M|_F / sqrt(k) (k <= 128), the first bound
//     is above 1e-5 s_1 and the second below it: kept and dropped values fall on the same
//     sides of the threshold as in the SVD-based factor.
// A segment whose iteration has not met the rule by step 28 (a singular value close to the
// threshold, or a slow one) is left to the Jacobi SVD path, which runs after this kernel
// for the segments flagged here. After the stop one more step and the cube X (X^T X)
// (s -> s^3) take the kept values to 1 to rounding and the dropped ones to ~1e-11.
//
// Layout: the C CTAs of a cluster each hold the whole X (k x k, FP32, row stride ks) and
// X^T X in shared memory; CTA c computes the rows [c r, (c + 1) r) of each product and
// writes them into every CTA's copy (distributed shared memory), then the cluster
// synchronises. Zero columns of M (empty clusters) stay exactly zero.
#include <cooperative_groups.h>

#include "internal.cuh"

namespace cg = cooperative_groups;

namespace abg {

namespace {

constexpr int kNsThreads = 512;
constexpr int kNsMinSteps = 15;
constexpr int kNsMaxSteps = 28;
constexpr float kNsEps = 1e-4f;
constexpr int kNsMaxCluster = 8;

// Rows [r0, r1) of dst = X^T X (every CTA's copy), columns as float4 groups.
__device__ void ns_gram(const float* X, int k, int ks, int r0, int r1, float* const* dst, int C) {
  const int k4 = ks >> 2;
  for (int idx = threadIdx.x; idx < (r1 - r0) * k4; idx += blockDim.x) {
    const int i = r0 + idx / k4, j4 = idx % k4;
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 4
    for (int r = 0; r < k; ++r)
      acc = f4_fma(X[r * ks + i], ld_f4(X + r * ks + 4 * j4), acc);
    for (int q = 0; q < C; ++q) st_f4(dst[q] + i * ks + 4 * j4, acc);
  }
}

// Rows [r0, r1) of X (1.5 I - 0.5 A): the Newton-Schulz step into every CTA's copy of the
// next X, with |X_next - X|^2 of each float4 group in part[(i - r0) k4 + j4]; or with T set,
// the product X A (the cube step) into the FP32 T and the FP64 t64.
__device__ void ns_apply(const float* X, const float* A, int k, int ks, int r0, int r1,
                         float* const* dst, int C, float* part, float* T, int kp, double* t64,
                         int kmax) {
  const int k4 = ks >> 2;
  for (int idx = threadIdx.x; idx < (r1 - r0) * k4; idx += blockDim.x) {
    const int i = r0 + idx / k4, j4 = idx % k4;
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 4
    for (int q = 0; q < k; ++q) acc = f4_fma(X[i * ks + q], ld_f4(A + q * ks + 4 * j4), acc);
    if (T) {
      const float v[4] = {acc.x, acc.y, acc.z, acc.w};
      for (int e = 0; e < 4; ++e) {
        const int j = 4 * j4 + e;
        if (j < k) {
          T[i * kp + j] = v[e];
          if (t64) t64[(int64_t)i * kmax + j] = (double)v[e];
        }
      }
      continue;
    }
    const float4 x = ld_f4(X + i * ks + 4 * j4);
    float4 xn;
    xn.x = fmaf(-0.5f, acc.x, 1.5f * x.x);
    xn.y = fmaf(-0.5f, acc.y, 1.5f * x.y);
    xn.z = fmaf(-0.5f, acc.z, 1.5f * x.z);
    xn.w = fmaf(-0.5f, acc.w, 1.5f * x.w);
    const float ex = xn.x - x.x, ey = xn.y - x.y, ez = xn.z - x.z, ew = xn.w - x.w;
    part[idx] = ex * ex + ey * ey + ez * ez + ew * ew;
    for (int q2 = 0; q2 < C; ++q2) st_f4(dst[q2] + i * ks + 4 * j4, xn);
  }
}

// One cluster of C CTAs per segment. M_s (k_s x k_s of a kmax x kmax slab, FP64) -> T_s
// (FP32, row stride kp) and t64_s (FP64, may be null); done[s] = 1 when the factor was
// written here, 0 when the segment is left to the SVD path.
__global__ void __launch_bounds__(kNsThreads, 1)
    k_polar_ns(const int* __restrict__ segk, int kmax, const double* __restrict__ Mall, int kp,
               float* __restrict__ Tall, double* __restrict__ t64all, int* __restrict__ done) {
  extern __shared__ __align__(16) float ns_smem[];
  __shared__ float s_row[kMaxK];  // |X_next - X|^2 per row, filled by the row's owner
  __shared__ double s_norm;
  cg::cluster_group cluster = cg::this_cluster();
  const int C = (int)cluster.num_blocks();
  const int rank = (int)cluster.block_rank();
  const int sg = blockIdx.x / C;
  const int k = segk[sg];
  const int ks = (int)round_up(kmax, 4);
  const int64_t slab = (int64_t)kmax * kmax;
  const double* M = Mall + sg * slab;
  float* T = Tall + (int64_t)sg * kmax * kp;
  double* t64 = t64all ? t64all + sg * slab : nullptr;
  float* buf[3] = {ns_smem, ns_smem + kmax * ks, ns_smem + 2 * kmax * ks};  // X, X', A
  float* part = ns_smem + 3 * kmax * ks;  // (rows of this CTA) x ks/4 partial step norms
  const int rows = (int)ceil_div(k, C);
  const int r0 = min(k, rank * rows), r1 = min(k, r0 + rows);

  // |M|_F in FP64, the same sum in every CTA
  if (threadIdx.x < 32) {
    double a = 0.0;
    for (int q = threadIdx.x; q < k * k; q += 32) {
      const double v = M[(int64_t)(q / k) * kmax + q % k];
      a += v * v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (threadIdx.x == 0) s_norm = a;
  }
  __syncthreads();
  const double nrm2 = s_norm;
  if (!(nrm2 > 0.0)) {  // M = 0: T = 0
    for (int q = threadIdx.x; q < (r1 - r0) * k; q += blockDim.x) {
      const int i = r0 + q / k, j = q % k;
      T[i * kp + j] = 0.f;
      if (t64) t64[(int64_t)i * kmax + j] = 0.0;
    }
    if (rank == 0 && threadIdx.x == 0) done[sg] = 1;
    cluster.sync();
    return;
  }
  const double inv = 1.0 / sqrt(nrm2);
  for (int q = threadIdx.x; q < kmax * ks; q += blockDim.x) {
    const int i = q / ks, j = q % ks;
    buf[0][q] = (i < k && j < k) ? (float)(M[(int64_t)i * kmax + j] * inv) : 0.f;
    buf[1][q] = 0.f;
    buf[2][q] = 0.f;
  }
  float* nxt[kNsMaxCluster];   // every CTA's copy of the next X
  float* gram[kNsMaxCluster];  // ... and of X^T X
  int ic = 0;  // index of the current X in buf
  auto bind = [&](int c_idx) {
    for (int q = 0; q < C; ++q) {
      nxt[q] = cluster.map_shared_rank(buf[1 - c_idx], q);
      gram[q] = cluster.map_shared_rank(buf[2], q);
    }
  };
  bind(ic);
  cluster.sync();  // every copy initialised before any CTA writes into another

  // One Newton-Schulz step; returns |X_next - X|_F^2 summed group by group within a row and
  // row by row, the same order whatever the cluster size, so the stop (and the result) of a
  // segment does not depend on the batch it is solved in.
  auto step = [&]() -> float {
    ns_gram(buf[ic], k, ks, r0, r1, gram, C);
    cluster.sync();
    ns_apply(buf[ic], buf[2], k, ks, r0, r1, nxt, C, part, nullptr, 0, nullptr, kmax);
    __syncthreads();
    const int k4 = ks >> 2;
    for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
      float t = 0.f;
      for (int j4 = 0; j4 < k4; ++j4) t += part[(i - r0) * k4 + j4];
      for (int q = 0; q < C; ++q) cluster.map_shared_rank(s_row, q)[i] = t;
    }
    cluster.sync();
    float tot = 0.f;
    for (int i = 0; i < k; ++i) tot += s_row[i];
    ic = 1 - ic;
    bind(ic);
    return tot;
  };

  bool ok = false;
  for (int n = 1; n <= kNsMaxSteps; ++n) {
    const float d2 = step();
    if (n >= kNsMinSteps && d2 <= kNsEps * kNsEps) {
      ok = true;
      break;
    }
  }
  if (!ok) {  // uniform over the cluster: every CTA summed the same partials
    if (rank == 0 && threadIdx.x == 0) done[sg] = 0;
    return;   // no CTA writes into another's shared memory after the last cluster barrier
  }
  step();  // polish: kept values to 1 up to rounding
  ns_gram(buf[ic], k, ks, r0, r1, gram, C);
  cluster.sync();
  ns_apply(buf[ic], buf[2], k, ks, r0, r1, nullptr, C, part, T, kp, t64, kmax);  // T = X X^T X
  if (rank == 0 && threadIdx.x == 0) done[sg] = 1;
}

}  // namespace

int polar_newton_schulz(int nseg, const int* segk, int kmax, const double* M, int kp, float* T,
                        double* t64, int* done, cudaStream_t s) {
  ABG_CHECK(kmax >= 1 && kmax <= kMaxK, "polar: need 1 <= k <= %d", kMaxK);
  const int C = kmax <= 32 ? 1 : (kmax <= 64 ? 4 : kNsMaxCluster);
  const size_t ks = (size_t)round_up(kmax, 4);
  const size_t smem = sizeof(float) * (3 * (size_t)kmax * ks + (size_t)ceil_div(kmax, C) * ks / 4);
  ABG_TRY(raise_smem_limit((const void*)k_polar_ns, smem));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(C * nseg));
  cfg.blockDim = dim3(kNsThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  ABG_CUDA(cudaLaunchKernelEx(&cfg, k_polar_ns, segk, kmax, M, kp, T, t64, done));
  note_launch();
  return ABG_OK;
}

}  // namespace abg
