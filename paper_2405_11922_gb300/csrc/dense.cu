// Dense, tall-skinny work of TPO (rows = the |U| target nodes):
//   * gemm_nn: C = A B with A tall (n x K) and B small (K x N <= 128 wide):
//     R Omega, R Q, R H, Phi C, Q_b U (Algorithm 2 and its randomized SVD),
//     Zhat Q^T (Eq. 13), each with a fused element-wise epilogue.
//   * gemm_tn: C = A^T B reduced over the long dimension (R^T Phi, Phi^T Phi,
//     Phi^T (R H), Gram matrices): FP32 products per fixed 2048-row chunk,
//     chunk partials summed in FP64 in a fixed order (deterministic).
//   * random features (Eqs. 13-14), the H rule (Eq. 16), NCI generation
//     (Algorithm 3, Eqs. 21-23) and the objective (Eq. 8).
// All are FP32 SIMT kernels (FMA pipes) tiled through shared memory.
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.cuh"

namespace abg {

constexpr int kTnChunk = 2048;  // rows per partial of a reduction over |U|
constexpr int kRedGroup = 32;   // partials summed per first-level reduction thread

struct EpiNN {
  int mode;
  const float* aux;
  int64_t ldaux;
  const float* aux2;
  int64_t ldaux2;
  const float* sign;
  // random features (mode 5): scale inside sin/cos, factor outside, width d, partial colsums
  float in_scale, out_scale;
  double* colsum_part;  // [gridDim.x][2N]
  // NCI scores (mode 6): row argmax over the N columns (ties -> lowest column), top1 - top2
  int32_t* labels;
  float* margin;
  int first;
  int* changes;
  unsigned* min_margin_bits;
};
constexpr int kEpiSinCos = 5;
constexpr int kEpiArgmax = 6;

struct Best {
  float v;
  int i;
  float s;
};
__device__ __forceinline__ Best merge_best(Best a, Best b) {
  Best r;
  if (a.v > b.v || (a.v == b.v && a.i < b.i)) {
    r = a;
    r.s = fmaxf(a.s, b.v);
  } else {
    r = b;
    r.s = fmaxf(b.s, a.v);
  }
  return r;
}

// ---------------------------------------------------------------------------
// C = A (M x K) * B (K x N), CTA tile 128 x (16*TN), K step 16, 256 threads,
// thread tile 8 rows x TN columns (columns (tx + 16 j) * 4 .. +4 for TN >= 4).
// ---------------------------------------------------------------------------
template <int TN, int EPI>  // EPI: 0 element-wise, 1 sin/cos + column sums, 2 row argmax
__global__ void __launch_bounds__(256) k_gemm_nn(int64_t M, int N, int K,
                                                 const float* __restrict__ A, int64_t lda,
                                                 const float* __restrict__ B, int64_t ldb,
                                                 float* __restrict__ C, int64_t ldc, EpiNN ep) {
  constexpr int BM = 128, BK = 16, BN = 16 * TN, TM = 8;
  constexpr int NQ = TN >= 4 ? TN / 4 : 1;  // float4 column groups per thread
  __shared__ __align__(16) float As[BK][BM];
  __shared__ __align__(16) float Bs[BK][BN];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int64_t m0 = (int64_t)blockIdx.x * BM;
  const int n0 = blockIdx.y * BN;
  float acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = 0.f;

  for (int k0 = 0; k0 < K; k0 += BK) {
    // A tile: thread loads rows r = tid & 127 at k-quads kq and kq+1 (kq = 2*(tid>>7))
#pragma unroll
    for (int rep = 0; rep < 2; ++rep) {
      const int r = tid & 127;
      const int kq = 2 * (tid >> 7) + rep;
      const int64_t gm = m0 + r;
      const int gk = k0 + kq * 4;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (gm < M && gk < K) {
        v = ld_nc_f4(A + gm * lda + gk);
        if (gk + 1 >= K) v.y = 0.f;
        if (gk + 2 >= K) v.z = 0.f;
        if (gk + 3 >= K) v.w = 0.f;
      }
      As[kq * 4 + 0][r] = v.x;
      As[kq * 4 + 1][r] = v.y;
      As[kq * 4 + 2][r] = v.z;
      As[kq * 4 + 3][r] = v.w;
    }
    // B tile: BK rows x BN columns
    constexpr int BQ = BK * BN / 4;
    for (int q = tid; q < BQ; q += 256) {
      const int kk = q / (BN / 4);
      const int nq = q % (BN / 4);
      const int gk = k0 + kk;
      const int gn = n0 + nq * 4;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (gk < K && gn < N) {
        v = ld_nc_f4(B + (int64_t)gk * ldb + gn);
        if (gn + 1 >= N) v.y = 0.f;
        if (gn + 2 >= N) v.z = 0.f;
        if (gn + 3 >= N) v.w = 0.f;
      }
      *reinterpret_cast<float4*>(&Bs[kk][nq * 4]) = v;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < BK; ++k) {
      float a[TM], b[TN];
      float4 a0 = *reinterpret_cast<const float4*>(&As[k][ty * TM]);
      float4 a1 = *reinterpret_cast<const float4*>(&As[k][ty * TM + 4]);
      a[0] = a0.x; a[1] = a0.y; a[2] = a0.z; a[3] = a0.w;
      a[4] = a1.x; a[5] = a1.y; a[6] = a1.z; a[7] = a1.w;
      if (TN >= 4) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
          float4 bv = *reinterpret_cast<const float4*>(&Bs[k][(tx + 16 * q) * 4]);
          b[4 * q + 0] = bv.x; b[4 * q + 1] = bv.y; b[4 * q + 2] = bv.z; b[4 * q + 3] = bv.w;
        }
      } else {
#pragma unroll
        for (int j = 0; j < TN; ++j) b[j] = Bs[k][tx * TN + j];
      }
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }

  // ---- epilogue ----
  auto col_of = [&](int j) -> int {
    return TN >= 4 ? n0 + (tx + 16 * (j / 4)) * 4 + (j & 3) : n0 + tx * TN + j;
  };
  if constexpr (EPI == 1) {
    // R'[i, n] = out_scale * sin(in_scale * acc), R'[i, N + n] = out_scale * cos(...);
    // per-CTA column sums of R' (FP64, fixed order over the 16 row groups)
    __shared__ double csum[16][2 * BN];
    double ls[TN], lc[TN];
#pragma unroll
    for (int j = 0; j < TN; ++j) ls[j] = lc[j] = 0.0;
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      const int64_t gm = m0 + ty * TM + i;
      if (gm >= M) continue;
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        const int gn = col_of(j);
        if (gn >= N) continue;
        float sv, cv;
        sincosf(ep.in_scale * acc[i][j], &sv, &cv);
        sv *= ep.out_scale;
        cv *= ep.out_scale;
        C[gm * ldc + gn] = sv;
        C[gm * ldc + N + gn] = cv;
        ls[j] += (double)sv;
        lc[j] += (double)cv;
      }
    }
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int cl = col_of(j) - n0;
      csum[ty][cl] = ls[j];
      csum[ty][BN + cl] = lc[j];
    }
    __syncthreads();
    for (int c = tid; c < 2 * BN; c += 256) {
      double s = 0.0;
      for (int r = 0; r < 16; ++r) s += csum[r][c];
      const int cl = c % BN;
      const int gn = n0 + cl;
      if (gn < N) ep.colsum_part[(int64_t)blockIdx.x * 2 * N + (c < BN ? gn : N + gn)] = s;
    }
  } else if constexpr (EPI == 2) {
    // Eq. 21: l* = argmax_l (Phi T)[i, l]; the row's columns live on the 16 lanes of equal ty
    // (one grid column covers all N <= 16*TN columns); reduce with shuffles inside 16 lanes
    int old_lab[TM];
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      const int64_t gm = m0 + ty * TM + i;
      old_lab[i] = (!ep.first && tx == 0 && gm < M) ? ep.labels[gm] : -1;
    }
    int local_changes = 0;
    float local_min = INFINITY;
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      Best b{-INFINITY, 0x7fffffff, -INFINITY};
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        const int gn = col_of(j);
        if (gn < N) b = merge_best(b, Best{acc[i][j], gn, -INFINITY});
      }
#pragma unroll
      for (int o = 8; o > 0; o >>= 1) {
        Best other;
        other.v = __shfl_xor_sync(0xffffffffu, b.v, o);
        other.i = __shfl_xor_sync(0xffffffffu, b.i, o);
        other.s = __shfl_xor_sync(0xffffffffu, b.s, o);
        b = merge_best(b, other);
      }
      const int64_t gm = m0 + ty * TM + i;
      if (tx == 0 && gm < M) {
        const float mg = N > 1 ? b.v - b.s : INFINITY;
        if (!ep.first && old_lab[i] != b.i) ++local_changes;
        ep.labels[gm] = b.i;
        if (ep.margin) ep.margin[gm] = mg;
        local_min = fminf(local_min, mg);
      }
    }
    if (local_changes) atomicAdd(ep.changes, local_changes);
    if (local_min < INFINITY) atomicMin(ep.min_margin_bits, __float_as_uint(fmaxf(local_min, 0.f)));
  } else {
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int64_t gm = m0 + ty * TM + i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int gn = col_of(j);
      if (gn >= N) continue;
      float v = acc[i][j];
      switch (ep.mode) {
        case (int)Epi::Relu: v = fmaxf(v, 0.f); break;
        case (int)Epi::SignRelu: v = fmaxf(ep.sign[gn] * v, 0.f); break;
        case (int)Epi::Sign: v = ep.sign[gn] * v; break;
        case (int)Epi::PhiUpdate: {
          const float p = ep.aux[gm * ep.ldaux + gn];
          const float phi = ep.aux2[gm * ep.ldaux2 + gn];
          v = v > 0.f ? phi * sqrtf(fmaxf(p, 0.f) / v) : 0.f;
          break;
        }
        default: break;
      }
      C[gm * ldc + gn] = v;
    }
  }
  }
}

template <int TN>
static void launch_nn(int64_t M, int N, int K, const float* A, int64_t lda, const float* B,
                      int64_t ldb, float* C, int64_t ldc, const EpiNN& ep, cudaStream_t s) {
  dim3 grid((unsigned)ceil_div(M, 128), (unsigned)ceil_div(N, 16 * TN));
  if (ep.mode == kEpiSinCos) {
    k_gemm_nn<TN, 1><<<grid, 256, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc, ep); ::abg::note_launch();
  } else if (ep.mode == kEpiArgmax) {
    k_gemm_nn<TN, 2><<<grid, 256, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc, ep); ::abg::note_launch();
  } else {
    k_gemm_nn<TN, 0><<<grid, 256, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc, ep); ::abg::note_launch();
  }
}

static int gemm_nn_impl(int64_t M, int N, int K, const float* A, int64_t lda, const float* B,
                        int64_t ldb, float* C, int64_t ldc, const EpiNN& ep, cudaStream_t s) {
  ABG_CHECK(M >= 0 && N >= 1 && K >= 1, "gemm_nn: bad sizes");
  ABG_CHECK(lda % 4 == 0 && ldb % 4 == 0 && lda >= K && ldb >= N,
            "gemm_nn: leading dimensions must be multiples of 4 and cover the width");
  if (M == 0) return ABG_OK;
  if (N <= 32)
    launch_nn<2>(M, N, K, A, lda, B, ldb, C, ldc, ep, s);
  else if (N <= 64)
    launch_nn<4>(M, N, K, A, lda, B, ldb, C, ldc, ep, s);
  else
    launch_nn<8>(M, N, K, A, lda, B, ldb, C, ldc, ep, s);
  ABG_LAUNCH_CHECK();
  return ABG_OK;
}

int gemm_nn(int64_t M, int N, int K, const float* A, int64_t lda, const float* B, int64_t ldb,
            float* C, int64_t ldc, Epi epi, const float* aux, int64_t ldaux, const float* aux2,
            int64_t ldaux2, const float* sign, cudaStream_t s) {
  EpiNN ep{(int)epi, aux, ldaux, aux2, ldaux2, sign, 1.f, 1.f, nullptr};
  return gemm_nn_impl(M, N, K, A, lda, B, ldb, C, ldc, ep, s);
}

// ---------------------------------------------------------------------------
// Deterministic FP64 reduction of chunk partials: out[e] = sum_c part[c][e],
// summed in groups of kRedGroup chunks, then over groups, both in index order.
// ---------------------------------------------------------------------------
template <class T>
__global__ void k_reduce_level1(const T* __restrict__ part, int64_t nchunks, int64_t width,
                                double* __restrict__ lvl1) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t g = blockIdx.y;
  if (e >= width) return;
  const int64_t c0 = g * kRedGroup;
  const int64_t c1 = min(nchunks, c0 + kRedGroup);
  double s = 0.0;
  for (int64_t c = c0; c < c1; ++c) s += (double)part[c * width + e];
  lvl1[g * width + e] = s;
}

// out[(e / cols) * ldo + e % cols] = sum over groups
__global__ void k_reduce_level2(const double* __restrict__ lvl1, int64_t ngroups, int64_t width,
                                int cols, double* __restrict__ out, int64_t ldo) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= width) return;
  double s = 0.0;
  for (int64_t g = 0; g < ngroups; ++g) s += lvl1[g * width + e];
  out[(e / cols) * ldo + (e % cols)] = s;
}

template <class T>
static int reduce_partials(const T* part, int64_t nchunks, int64_t width, int cols, double* out,
                           int64_t ldo, Scratch& scr, cudaStream_t s) {
  const int64_t ngroups = ceil_div(nchunks, kRedGroup);
  double* lvl1;
  ABG_TRY(scr.get(&lvl1, (size_t)ngroups * width));
  dim3 g1((unsigned)ceil_div(width, 256), (unsigned)ngroups);
  k_reduce_level1<T><<<g1, 256, 0, s>>>(part, nchunks, width, lvl1); ::abg::note_launch();
  k_reduce_level2<<<(unsigned)ceil_div(width, 256), 256, 0, s>>>(lvl1, ngroups, width, cols, out,
                                                                 ldo); ::abg::note_launch();
  ABG_LAUNCH_CHECK();
  return ABG_OK;
}

// ---------------------------------------------------------------------------
// C = A^T B over a chunk of kTnChunk rows per CTA: output tile 128 (rows = A
// columns) x 16*TN (B columns), 16 rows staged per step; FP32 partial per chunk.
// ---------------------------------------------------------------------------
template <int TN>
__global__ void __launch_bounds__(256) k_gemm_tn_part(int64_t M, int K, int N,
                                                     const float* __restrict__ A, int64_t lda,
                                                     const float* __restrict__ B, int64_t ldb,
                                                     float* __restrict__ part) {
  constexpr int BKo = 128, BN = 16 * TN, SUB = 16, TM = 8;
  constexpr int NQ = TN >= 4 ? TN / 4 : 1;
  __shared__ __align__(16) float As[SUB][BKo];
  __shared__ __align__(16) float Bs[SUB][BN];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int64_t c = blockIdx.x;
  const int k0 = blockIdx.y * BKo;
  const int n0 = blockIdx.z * BN;
  const int64_t r0 = c * kTnChunk;
  const int64_t r1 = min(M, r0 + kTnChunk);
  float acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = 0.f;
  for (int64_t m0 = r0; m0 < r1; m0 += SUB) {
    for (int q = tid; q < SUB * BKo / 4; q += 256) {
      const int mm = q / (BKo / 4), kq = q % (BKo / 4);
      const int64_t gm = m0 + mm;
      const int gk = k0 + kq * 4;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (gm < r1 && gk < K) {
        v = ld_nc_f4(A + gm * lda + gk);
        if (gk + 1 >= K) v.y = 0.f;
        if (gk + 2 >= K) v.z = 0.f;
        if (gk + 3 >= K) v.w = 0.f;
      }
      *reinterpret_cast<float4*>(&As[mm][kq * 4]) = v;
    }
    for (int q = tid; q < SUB * BN / 4; q += 256) {
      const int mm = q / (BN / 4), nq = q % (BN / 4);
      const int64_t gm = m0 + mm;
      const int gn = n0 + nq * 4;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (gm < r1 && gn < N) {
        v = ld_nc_f4(B + gm * ldb + gn);
        if (gn + 1 >= N) v.y = 0.f;
        if (gn + 2 >= N) v.z = 0.f;
        if (gn + 3 >= N) v.w = 0.f;
      }
      *reinterpret_cast<float4*>(&Bs[mm][nq * 4]) = v;
    }
    __syncthreads();
#pragma unroll
    for (int mm = 0; mm < SUB; ++mm) {
      float a[TM], b[TN];
      float4 a0 = *reinterpret_cast<const float4*>(&As[mm][ty * TM]);
      float4 a1 = *reinterpret_cast<const float4*>(&As[mm][ty * TM + 4]);
      a[0] = a0.x; a[1] = a0.y; a[2] = a0.z; a[3] = a0.w;
      a[4] = a1.x; a[5] = a1.y; a[6] = a1.z; a[7] = a1.w;
      if (TN >= 4) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
          float4 bv = *reinterpret_cast<const float4*>(&Bs[mm][(tx + 16 * q) * 4]);
          b[4 * q + 0] = bv.x; b[4 * q + 1] = bv.y; b[4 * q + 2] = bv.z; b[4 * q + 3] = bv.w;
        }
      } else {
#pragma unroll
        for (int j = 0; j < TN; ++j) b[j] = Bs[mm][tx * TN + j];
      }
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
  float* out = part + c * (int64_t)K * N;
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int gk = k0 + ty * TM + i;
    if (gk >= K) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int gn = TN >= 4 ? n0 + (tx + 16 * (j / 4)) * 4 + (j & 3) : n0 + tx * TN + j;
      if (gn < N) out[(int64_t)gk * N + gn] = acc[i][j];
    }
  }
}

int gemm_tn(int64_t M, int K, int N, const float* A, int64_t lda, const float* B, int64_t ldb,
            double* C, int64_t ldc, Scratch& /*caller*/, cudaStream_t s) {
  Scratch scr(s);
  ABG_CHECK(M >= 1 && K >= 1 && N >= 1, "gemm_tn: bad sizes");
  ABG_CHECK(lda % 4 == 0 && ldb % 4 == 0 && lda >= K && ldb >= N,
            "gemm_tn: leading dimensions must be multiples of 4 and cover the width");
  const int64_t nch = ceil_div(M, kTnChunk);
  float* part;
  ABG_TRY(scr.get(&part, (size_t)nch * K * N));
  dim3 grid((unsigned)nch, (unsigned)ceil_div(K, 128), 1);
  if (N <= 32) {
    grid.z = (unsigned)ceil_div(N, 32);
    k_gemm_tn_part<2><<<grid, 256, 0, s>>>(M, K, N, A, lda, B, ldb, part); ::abg::note_launch();
  } else if (N <= 64) {
    grid.z = (unsigned)ceil_div(N, 64);
    k_gemm_tn_part<4><<<grid, 256, 0, s>>>(M, K, N, A, lda, B, ldb, part); ::abg::note_launch();
  } else {
    grid.z = (unsigned)ceil_div(N, 128);
    k_gemm_tn_part<8><<<grid, 256, 0, s>>>(M, K, N, A, lda, B, ldb, part); ::abg::note_launch();
  }
  ABG_LAUNCH_CHECK();
  return reduce_partials<float>(part, nch, (int64_t)K * N, N, C, ldc, scr, s);
}

// column sums of A (M x N): per-chunk FP64 partials, then the ordered reduction
__global__ void k_colsum_part(int64_t M, int N, const float* __restrict__ A, int64_t lda,
                              double* __restrict__ part) {
  const int64_t c = blockIdx.x;
  const int64_t r0 = c * kTnChunk, r1 = min(M, r0 + kTnChunk);
  for (int n = threadIdx.x; n < N; n += blockDim.x) {
    double s = 0.0;
    for (int64_t r = r0; r < r1; ++r) s += (double)A[r * lda + n];
    part[c * N + n] = s;
  }
}

int column_sums(int64_t M, int N, const float* A, int64_t lda, double* out, Scratch& /*caller*/,
                cudaStream_t s) {
  Scratch scr(s);
  const int64_t nch = ceil_div(M, kTnChunk);
  double* part;
  ABG_TRY(scr.get(&part, (size_t)nch * N));
  k_colsum_part<<<(unsigned)nch, 128, 0, s>>>(M, N, A, lda, part); ::abg::note_launch();
  ABG_LAUNCH_CHECK();
  return reduce_partials<double>(part, nch, N, N, out, N, scr, s);
}

// ---------------------------------------------------------------------------
// Random features (Eqs. 13-14)
// ---------------------------------------------------------------------------
// R[i] <- R'[i] / sqrt(max(R'[i].r, 1e-300)); one warp per row.
__global__ void k_rf_normalise(int64_t n, int w2, float* __restrict__ R, int64_t ldr,
                               const double* __restrict__ r, int* __restrict__ clamped) {
  const int64_t row = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  float* rp = R + row * ldr;
  float part = 0.f;
  for (int c = lane; c < w2; c += 32) part = fmaf(rp[c], (float)r[c], part);
  double dot = (double)part;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
  const bool clamp = !(dot > 1e-300);
  if (clamp) dot = 1e-300;
  const float inv = (float)(1.0 / sqrt(dot));
  for (int c = lane; c < w2; c += 32) rp[c] *= inv;
  if (clamp && lane == 0) atomicAdd(clamped, 1);
}

int random_features(const float* zhat, int64_t n, int d, int64_t ldz, const float* qt, float* R,
                    int64_t ldr, int* clamped_dev, Scratch& /*caller*/, cudaStream_t s) {
  Scratch scr(s);
  ABG_CHECK(ldr >= 2 * d && ldr % 4 == 0, "random_features: ldr must be >= 2d, multiple of 4");
  const int64_t ldq = round_up(d, 4);
  const unsigned gx = (unsigned)ceil_div(n, 128);
  double* cpart;
  ABG_TRY(scr.get(&cpart, (size_t)gx * 2 * d));
  EpiNN ep{kEpiSinCos, nullptr, 0, nullptr, 0, nullptr, (float)sqrt((double)d),
           (float)sqrt(exp(1.0) / d), cpart};
  ABG_TRY(gemm_nn_impl(n, d, d, zhat, ldz, qt, ldq, R, ldr, ep, s));
  double* r;
  ABG_TRY(scr.get(&r, (size_t)2 * d));
  ABG_TRY(reduce_partials<double>(cpart, gx, 2 * d, 2 * d, r, 2 * d, scr, s));
  k_rf_normalise<<<(unsigned)ceil_div(n, 8), 256, 0, s>>>(n, 2 * d, R, ldr, r, clamped_dev); ::abg::note_launch();
  ABG_LAUNCH_CHECK();
  return ABG_OK;
}

// ---------------------------------------------------------------------------
// Eq. 16: H <- H * max(R^T Phi, 0) / (H (Phi^T Phi)); a non-positive denominator gives 0
// ---------------------------------------------------------------------------
__global__ void k_nmf_h(int m, int k, const float* __restrict__ H, int64_t ldh,
                        const double* __restrict__ A, int64_t lda, const double* __restrict__ G,
                        int64_t ldg, float* __restrict__ Hn) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= m * k) return;
  const int j = idx / k, l = idx % k;
  double den = 0.0;
  for (int p = 0; p < k; ++p) den += (double)H[(int64_t)j * ldh + p] * G[(int64_t)p * ldg + l];
  const double num = fmax(A[(int64_t)j * lda + l], 0.0);
  Hn[(int64_t)j * ldh + l] = den > 0.0 ? (float)((double)H[(int64_t)j * ldh + l] * num / den) : 0.f;
}

int nmf_update_h(int m, int k, float* H, int64_t ldh, const double* A, int64_t lda,
                 const double* G, int64_t ldg, cudaStream_t s) {
  Scratch scr(s);
  float* Hn;
  ABG_TRY(scr.get(&Hn, (size_t)m * ldh));
  k_nmf_h<<<(unsigned)ceil_div((int64_t)m * k, 256), 256, 0, s>>>(m, k, H, ldh, A, lda, G, ldg, Hn); ::abg::note_launch();
  ABG_LAUNCH_CHECK();
  ABG_CUDA(cudaMemcpyAsync(H, Hn, sizeof(float) * m * ldh, cudaMemcpyDeviceToDevice, s));
  return ABG_OK;
}

// ---------------------------------------------------------------------------
// Algorithm 3: NCI generation
// ---------------------------------------------------------------------------
// Per-chunk cluster sums S[l][m] = sum_{i in chunk, label i = l} Phi[i, m] and counts; one
// thread per column, rows in order (deterministic).
__global__ void k_cluster_sums(int64_t n, int k, int w, const float* __restrict__ X, int64_t ldx,
                               const int32_t* __restrict__ labels, int col0, int wtile,
                               float* __restrict__ part, int64_t chunk_rows) {
  extern __shared__ float accs[];  // [k][wtile] + counts[k]
  const int64_t c = blockIdx.x;
  const int64_t r0 = c * chunk_rows, r1 = min(n, r0 + chunk_rows);
  float* cnt = accs + (int64_t)k * wtile;
  for (int q = threadIdx.x; q < k * wtile + k; q += blockDim.x) accs[q] = 0.f;
  __syncthreads();
  const int m = threadIdx.x;
  const int gm = col0 + m;
  const bool active = m < wtile && gm < w;
  const bool counter = threadIdx.x == 0 && blockIdx.y == 0;
  // 8 rows of loads in flight per thread, then the ordered shared-memory adds
  constexpr int U = 8;
  int64_t r = r0;
  for (; r + U <= r1; r += U) {
    int l[U];
    float v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      l[u] = labels[r + u];
      v[u] = active ? X[(r + u) * ldx + gm] : 0.f;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if ((unsigned)l[u] >= (unsigned)k) continue;  // labels outside [0, k) are skipped
      if (active) accs[l[u] * wtile + m] += v[u];
      if (counter) cnt[l[u]] += 1.f;
    }
  }
  for (; r < r1; ++r) {
    const int l = labels[r];
    if ((unsigned)l >= (unsigned)k) continue;
    if (active) accs[l * wtile + m] += X[r * ldx + gm];
    if (counter) cnt[l] += 1.f;
  }
  __syncthreads();
  // partial layout per chunk: [k][w] sums then [k] counts
  const int64_t width = (int64_t)k * w + k;
  float* out = part + c * width;
  if (active)
    for (int l = 0; l < k; ++l) out[(int64_t)l * w + gm] = accs[l * wtile + m];
  if (blockIdx.y == 0)
    for (int l = threadIdx.x; l < k; l += blockDim.x) out[(int64_t)k * w + l] = cnt[l];
}

static int cluster_sums(const float* X, int64_t n, int w, int64_t ldx, const int32_t* labels,
                        int k, double* sums /* (k+1) x w, last row counts (first k entries) */,
                        Scratch& /*caller*/, cudaStream_t s) {
  Scratch scr(s);
  const int wtile = std::min(w, 256);
  const int ntile = (int)ceil_div(w, wtile);
  // rows per chunk: about 4 CTAs per SM in total
  int64_t chunk_rows = std::max<int64_t>(512, ceil_div(n, (int64_t)num_sms() * 4 / ntile + 1));
  const int64_t nch = ceil_div(n, chunk_rows);
  const int64_t width = (int64_t)k * w + k;
  float* part;
  ABG_TRY(scr.get(&part, (size_t)nch * width));
  const size_t smem = sizeof(float) * ((size_t)k * wtile + k);
  if (smem > 48 * 1024)
    ABG_CUDA(cudaFuncSetAttribute(k_cluster_sums, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem));
  dim3 grid((unsigned)nch, (unsigned)ntile);
  const int threads = (int)round_up(wtile, 32);
  for (int t = 0; t < ntile; ++t) {
    // one launch per column tile keeps blockIdx.y == 0 for the count owner
    k_cluster_sums<<<dim3((unsigned)nch, 1), threads, smem, s>>>(n, k, w, X, ldx, labels,
                                                                 t * wtile, wtile, part,
                                                                 chunk_rows); ::abg::note_launch();
  }
  ABG_LAUNCH_CHECK();
  // reduce: sums[(k) x w] and counts (k) -> write counts into row k of `sums` (stride w)
  return reduce_partials<float>(part, nch, width, (int)width, sums, width, scr, s);
}

// T[m][l] = S[l][m] / sqrt(n_l) (zero for an empty cluster), float with stride kp; FP64 copy.
__global__ void k_nci_finalize(int k, const double* __restrict__ S, int kp, float* __restrict__ T,
                               double* __restrict__ t64, int* __restrict__ empty) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= k * k) return;
  const int m = idx / k, l = idx % k;
  const double cnt = S[(int64_t)k * k + l];
  const double v = cnt > 0 ? S[(int64_t)l * k + m] / sqrt(cnt) : 0.0;
  T[m * kp + l] = (float)v;
  if (t64) t64[m * k + l] = v;
  if (m == 0 && cnt <= 0) atomicAdd(empty, 1);
}

__global__ void k_reset_counters(int* c) {
  c[0] = 0;
  c[1] = 0x7f800000;  // +inf bits: minimum margin so far
  c[2] = 0;
}

__global__ void k_identity(int k, int kp, float* T) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < k * kp) T[idx] = ((idx / kp) == (idx % kp)) ? 1.f : 0.f;
}

int nci_run(const float* phi, int64_t n, int k, int64_t ldphi, int t_g, int32_t* labels,
            float* margin, double* t_out, int* last_changes_host, float* min_margin_host,
            int* empty_host, Scratch& /*caller*/, cudaStream_t s) {
  Scratch scr(s);
  ABG_CHECK(k >= 1 && k <= kMaxK, "nci: need 1 <= k <= %d", kMaxK);
  const int kp = (int)round_up(k, 4);
  float* T;
  ABG_TRY(scr.get(&T, (size_t)k * kp));
  double* S;
  ABG_TRY(scr.get(&S, (size_t)(k + 1) * k));
  int* counters;  // [0] changes, [1] min margin bits, [2] empty clusters
  ABG_TRY(scr.get(&counters, 4));
  k_identity<<<(unsigned)ceil_div(k * kp, 256), 256, 0, s>>>(k, kp, T); ::abg::note_launch();
  auto launch_scores = [&](int first) -> int {
    EpiNN ep{kEpiArgmax, nullptr, 0, nullptr, 0, nullptr, 1.f, 1.f, nullptr,
             labels, margin, first, counters, (unsigned*)(counters + 1)};
    return gemm_nn_impl(n, k, k, phi, ldphi, T, kp, nullptr, 0, ep, s);
  };
  for (int t = 0; t < t_g; ++t) {
    k_reset_counters<<<1, 1, 0, s>>>(counters); ::abg::note_launch();
    ABG_TRY(launch_scores(t == 0));
    ABG_TRY(cluster_sums(phi, n, k, ldphi, labels, k, S, scr, s));
    k_nci_finalize<<<(unsigned)ceil_div(k * k, 256), 256, 0, s>>>(k, S, kp, T, t_out, counters + 2); ::abg::note_launch();
    ABG_LAUNCH_CHECK();
  }
  if (t_g == 0) {  // no pass: every node in cluster 0 (T = I never used)
    ABG_CUDA(cudaMemsetAsync(labels, 0, sizeof(int32_t) * n, s));
  }
  int host[3] = {0, 0x7f800000, 0};
  if (t_g > 0) {
    ABG_CUDA(cudaMemcpyAsync(host, counters, sizeof(int) * 3, cudaMemcpyDeviceToHost, s));
    ABG_CUDA(cudaStreamSynchronize(s));
  }
  if (last_changes_host) *last_changes_host = host[0];
  if (min_margin_host) {
    unsigned b = (unsigned)host[1];
    float f;
    memcpy(&f, &b, sizeof(f));
    *min_margin_host = f;
  }
  if (empty_host) *empty_host = host[2];
  return ABG_OK;
}

// ---------------------------------------------------------------------------
// Eq. 8 through the cluster sums s_l (k x m, FP64) and counts n_l
// ---------------------------------------------------------------------------
__global__ void k_objective_final(int k, int m, const double* __restrict__ S,
                                  double* __restrict__ out) {
  // one CTA: total = sum_l s_l; obj = sum_l s_l.(total - s_l)/n_l; J = sum_l |s_l|^2 / n_l
  __shared__ double red_o[256], red_j[256];
  double o = 0.0, jv = 0.0;
  for (int c = threadIdx.x; c < m; c += blockDim.x) {
    double tot = 0.0;
    for (int l = 0; l < k; ++l) tot += S[(int64_t)l * m + c];
    for (int l = 0; l < k; ++l) {
      const double cnt = S[(int64_t)k * m + l];
      if (cnt > 0) {
        const double sv = S[(int64_t)l * m + c];
        o += sv * (tot - sv) / cnt;
        jv += sv * sv / cnt;
      }
    }
  }
  red_o[threadIdx.x] = o;
  red_j[threadIdx.x] = jv;
  __syncthreads();
  if (threadIdx.x == 0) {
    double so = 0.0, sj = 0.0;
    for (int t = 0; t < (int)blockDim.x; ++t) {
      so += red_o[t];
      sj += red_j[t];
    }
    out[0] = so;
    out[1] = sj;
  }
}

int objective(const float* R, int64_t n, int m, int64_t ldr, const int32_t* labels, int k,
              double* obj_host, Scratch& /*caller*/, cudaStream_t s) {
  Scratch scr(s);
  ABG_CHECK(k >= 1 && k <= kMaxK, "objective: need 1 <= k <= %d", kMaxK);
  double* S;
  ABG_TRY(scr.get(&S, (size_t)(k + 1) * m + k));
  // cluster_sums lays out (k x m) sums then k counts; k_objective_final reads counts at row k
  ABG_TRY(cluster_sums(R, n, m, ldr, labels, k, S, scr, s));
  double* out;
  ABG_TRY(scr.get(&out, 2));
  k_objective_final<<<1, 256, 0, s>>>(k, m, S, out); ::abg::note_launch();
  ABG_LAUNCH_CHECK();
  ABG_CUDA(cudaMemcpyAsync(obj_host, out, sizeof(double) * 2, cudaMemcpyDeviceToHost, s));
  ABG_CUDA(cudaStreamSynchronize(s));
  return ABG_OK;
}

}  // namespace abg
