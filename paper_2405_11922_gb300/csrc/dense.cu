// Dense, tall-skinny work of TPO over a batch row space (rows = U nodes of
// every segment; a plain solve is one segment):
//   * gemm_nn: C = A B_s with A tall and B_s small (per segment): R Omega,
//     R Q, R H, Phi C, Q_b U (Algorithm 2 and its randomized SVD), Zhat Q^T
//     (Eq. 13) and Phi T (Eq. 21), each with a fused epilogue.
//   * gemm_tn: C_s = A^T B reduced over the rows of segment s (R^T Phi,
//     Phi^T Phi, Gram matrices): FP32 products per fixed
//     2048-row chunk, chunk partials summed in FP64 in a fixed order.
//   * random features (Eqs. 13-14), the H rule (Eq. 16), NCI generation
//     (Algorithm 3, Eqs. 21-23) and the objective (Eq. 8).
// All are FP32 SIMT kernels (FMA pipes) tiled through shared memory.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "batch.cuh"
#include "internal.cuh"

namespace abg {

struct NNK {
  const float* A;
  int64_t lda;
  const float* B;
  int64_t ldb, b_seg;
  float* C;
  int64_t ldc;
  int N, K;
  const int* segN;
  const int* segK;
  const int* tile_seg;
  const int64_t* tile_row0;
  const int* tile_rows;
  int epi;
  const float* aux;
  int64_t ldaux;
  const float* aux2;
  int64_t ldaux2;
  const float* sign;
  int64_t sign_seg;
  float in_scale, out_scale;
  double* colsum_part;
  int32_t* labels;
  float* margin;
  int first;
  int* changes;
  unsigned* minbits;
};

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
// C = A (rows of one tile) * B_s, CTA tile 128 x (16*TN), K step 16, 256
// threads, thread tile 8 rows x TN columns (columns (tx + 16 j) * 4 .. +4 for
// TN >= 4). EPI: 0 element-wise, 1 sin/cos + column sums, 2 row argmax.
// ---------------------------------------------------------------------------
template <int TN, int EPI>
__global__ void __launch_bounds__(256) k_gemm_nn(NNK p) {
  constexpr int BM = 128, BK = 16, BN = 16 * TN, TM = 8;
  constexpr int NQ = TN >= 4 ? TN / 4 : 1;
  __shared__ __align__(16) float As[BK][BM];
  __shared__ __align__(16) float Bs[BK][BN];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int sg = p.tile_seg[blockIdx.x];
  const int64_t m0 = p.tile_row0[blockIdx.x];
  const int64_t mend = m0 + p.tile_rows[blockIdx.x];
  const int N = p.segN ? p.segN[sg] : p.N;
  const int K = p.segK ? p.segK[sg] : p.K;
  const float* __restrict__ B = p.B + sg * p.b_seg;
  const float* __restrict__ A = p.A;
  const int n0 = blockIdx.y * BN;
  if (n0 >= N) return;  // uniform over the CTA
  float acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = 0.f;

  for (int k0 = 0; k0 < K; k0 += BK) {
#pragma unroll
    for (int rep = 0; rep < 2; ++rep) {
      const int r = tid & 127;
      const int kq = 2 * (tid >> 7) + rep;
      const int64_t gm = m0 + r;
      const int gk = k0 + kq * 4;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (gm < mend && gk < K) {
        v = ld_nc_f4(A + gm * p.lda + gk);
        if (gk + 1 >= K) v.y = 0.f;
        if (gk + 2 >= K) v.z = 0.f;
        if (gk + 3 >= K) v.w = 0.f;
      }
      As[kq * 4 + 0][r] = v.x;
      As[kq * 4 + 1][r] = v.y;
      As[kq * 4 + 2][r] = v.z;
      As[kq * 4 + 3][r] = v.w;
    }
    constexpr int BQ = BK * BN / 4;
    for (int q = tid; q < BQ; q += 256) {
      const int kk = q / (BN / 4);
      const int nq = q % (BN / 4);
      const int gk = k0 + kk;
      const int gn = n0 + nq * 4;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (gk < K && gn < N) {
        v = ld_nc_f4(B + (int64_t)gk * p.ldb + gn);
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

  auto col_of = [&](int j) -> int {
    return TN >= 4 ? n0 + (tx + 16 * (j / 4)) * 4 + (j & 3) : n0 + tx * TN + j;
  };
  if constexpr (EPI == 1) {
    // R'[i, n] = out_scale sin(in_scale acc), R'[i, N + n] = out_scale cos(...); per-tile FP64
    // column sums of R' in a fixed order over the 16 row groups
    __shared__ double csum[16][2 * BN];
    double ls[TN], lc[TN];
#pragma unroll
    for (int j = 0; j < TN; ++j) ls[j] = lc[j] = 0.0;
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      const int64_t gm = m0 + ty * TM + i;
      if (gm >= mend) continue;
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        const int gn = col_of(j);
        if (gn >= N) continue;
        float sv, cv;
        sincosf(p.in_scale * acc[i][j], &sv, &cv);
        sv *= p.out_scale;
        cv *= p.out_scale;
        p.C[gm * p.ldc + gn] = sv;
        p.C[gm * p.ldc + N + gn] = cv;
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
      const int gn = n0 + c % BN;
      if (gn < N) p.colsum_part[(int64_t)blockIdx.x * 2 * N + (c < BN ? gn : N + gn)] = s;
    }
  } else if constexpr (EPI == 2) {
    // Eq. 21: l* = argmax_l (Phi T)[i, l] over the segment's N clusters; the row's columns
    // live on the 16 lanes of equal ty, reduced with shuffles inside those 16 lanes
    int old_lab[TM];
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      const int64_t gm = m0 + ty * TM + i;
      old_lab[i] = (!p.first && tx == 0 && gm < mend) ? p.labels[gm] : -1;
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
      if (tx == 0 && gm < mend) {
        const float mg = N > 1 ? b.v - b.s : INFINITY;
        if (!p.first && old_lab[i] != b.i) ++local_changes;
        p.labels[gm] = b.i;
        if (p.margin) p.margin[gm] = mg;
        local_min = fminf(local_min, mg);
      }
    }
    if (local_changes) atomicAdd(p.changes + sg, local_changes);
    if (local_min < INFINITY) atomicMin(p.minbits + sg, __float_as_uint(fmaxf(local_min, 0.f)));
  } else {
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      const int64_t gm = m0 + ty * TM + i;
      if (gm >= mend) continue;
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        const int gn = col_of(j);
        if (gn >= N) continue;
        float v = acc[i][j];
        switch (p.epi) {
          case (int)Epi::Relu: v = fmaxf(v, 0.f); break;
          case (int)Epi::SignRelu: v = fmaxf(p.sign[sg * p.sign_seg + gn] * v, 0.f); break;
          case (int)Epi::Sign: v = p.sign[sg * p.sign_seg + gn] * v; break;
          case (int)Epi::PhiUpdate: {
            const float pv = p.aux[gm * p.ldaux + gn];
            const float phi = p.aux2[gm * p.ldaux2 + gn];
            v = v > 0.f ? phi * sqrtf(fmaxf(pv, 0.f) / v) : 0.f;
            break;
          }
          default: break;
        }
        p.C[gm * p.ldc + gn] = v;
      }
    }
  }
}

int gemm_nn(const RowSpace& rs, const NN& a, cudaStream_t s) {
  ABG_CHECK(a.N >= 1 && a.K >= 1, "gemm_nn: bad sizes");
  ABG_CHECK(a.lda % 4 == 0 && a.ldb % 4 == 0 && a.lda >= a.K && a.ldb >= a.N,
            "gemm_nn: leading dimensions must be multiples of 4 and cover the width");
  if (rs.n_tiles == 0) return ABG_OK;
  bool tc = false;
  if (a.A16) ABG_TRY(tc_gemm_nn16(rs, a, s, &tc));
  if (!tc) ABG_TRY(tc_gemm_nn(rs, a, s, &tc));
  if (tc) return ABG_OK;
  NNK p{a.A, a.lda, a.B, a.ldb, a.b_seg, a.C, a.ldc, a.N, a.K, a.segN, a.segK,
        rs.tile_seg, rs.tile_row0, rs.tile_rows, (int)a.epi, a.aux, a.ldaux, a.aux2, a.ldaux2,
        a.sign, a.sign_seg, a.in_scale, a.out_scale, a.colsum_part, a.labels, a.margin, a.first,
        a.changes, a.minbits};
  const int mode = a.sincos ? 1 : (a.argmax ? 2 : 0);
  const int TN = a.N <= 32 ? 2 : (a.N <= 64 ? 4 : 8);
  ABG_CHECK(mode != 2 || a.N <= 16 * TN, "gemm_nn: argmax needs N <= 128");
  dim3 grid((unsigned)rs.n_tiles, (unsigned)ceil_div(a.N, 16 * TN));
#define ABG_NN_CASE(tn, md)                                   \
  if (TN == tn && mode == md) {                               \
    k_gemm_nn<tn, md><<<grid, 256, 0, s>>>(p);                \
    note_launch();                                            \
  }
  ABG_NN_CASE(2, 0) ABG_NN_CASE(4, 0) ABG_NN_CASE(8, 0)
  ABG_NN_CASE(2, 1) ABG_NN_CASE(4, 1) ABG_NN_CASE(8, 1)
  ABG_NN_CASE(2, 2) ABG_NN_CASE(4, 2) ABG_NN_CASE(8, 2)
#undef ABG_NN_CASE
  ABG_LAUNCH_CHECK();
  return ABG_OK;
}

// ---------------------------------------------------------------------------
// Ordered FP64 reduction of per-piece partials (pieces = reduction chunks or
// NN tiles of the row space): out_s[e] = sum over the pieces of segment s, in
// groups of kGroup pieces, then over the groups, both in index order.
// ---------------------------------------------------------------------------
template <class T>
__global__ void k_reduce_l1(const T* __restrict__ part, int64_t width,
                            const int64_t* __restrict__ group_p0, const int* __restrict__ group_np,
                            double* __restrict__ lvl1) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t g = blockIdx.y;
  if (e >= width) return;
  const int64_t p0 = group_p0[g];
  const int np = group_np[g];
  double s = 0.0;
  for (int i = 0; i < np; ++i) s += (double)part[(p0 + i) * width + e];
  lvl1[g * width + e] = s;
}

__global__ void k_reduce_l2(const double* __restrict__ lvl1, int64_t width,
                            const int64_t* __restrict__ seg_g0, int cols,
                            const int* __restrict__ segR, int rmax, const int* __restrict__ segC,
                            int cmax, double* __restrict__ out, int64_t ldo, int64_t oseg) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int sg = blockIdx.y;
  if (e >= width) return;
  const int64_t r = e / cols;
  const int c = (int)(e % cols);
  const int R = segR ? segR[sg] : rmax;
  const int Cc = segC ? segC[sg] : cmax;
  if (r >= R || c >= Cc) return;
  double s = 0.0;
  for (int64_t g = seg_g0[sg]; g < seg_g0[sg + 1]; ++g) s += lvl1[g * width + e];
  out[sg * oseg + r * ldo + c] = s;
}

// out (segment s at out + s*oseg) <- partials reduced; the element e of a piece sits at row
// e / cols, column e % cols; segR/segC (optional) mask rows/columns per segment.
template <class T>
static int reduce_pieces(const RowSpace& rs, bool tiles, const T* part, int64_t width, int cols,
                         const int* segR, int rmax, const int* segC, int cmax, double* out,
                         int64_t ldo, int64_t oseg, cudaStream_t s) {
  Scratch scr(s);
  const int64_t ng = tiles ? rs.n_tgroups : rs.n_groups;
  if (ng == 0) return ABG_OK;
  double* lvl1;
  ABG_TRY(scr.get(&lvl1, (size_t)ng * width));
  dim3 g1((unsigned)ceil_div(width, 256), (unsigned)ng);
  k_reduce_l1<T><<<g1, 256, 0, s>>>(part, width, tiles ? rs.tgroup_tile0 : rs.group_chunk0,
                                     tiles ? rs.tgroup_ntiles : rs.group_nchunks, lvl1);
  note_launch();
  dim3 g2((unsigned)ceil_div(width, 256), (unsigned)rs.nseg);
  k_reduce_l2<<<g2, 256, 0, s>>>(lvl1, width, tiles ? rs.seg_tgroup0 : rs.seg_group0, cols, segR,
                                 rmax, segC, cmax, out, ldo, oseg);
  note_launch();
  ABG_LAUNCH_CHECK();
  return ABG_OK;
}

// ---------------------------------------------------------------------------
// C_s = A^T B over the rows of segment s: one CTA per (chunk, 128-row output
// tile, 16*TN-column output tile), 16 rows staged per step, FP32 partial per chunk.
// ---------------------------------------------------------------------------
template <int TN>
__global__ void __launch_bounds__(256) k_gemm_tn_part(
    const int* __restrict__ chunk_seg, const int64_t* __restrict__ chunk_row0,
    const int* __restrict__ chunk_rows, int Kmax, int Nmax, const int* __restrict__ segK,
    const int* __restrict__ segN, const float* __restrict__ A, int64_t lda,
    const float* __restrict__ B, int64_t ldb, float* __restrict__ part) {
  constexpr int BKo = 128, BN = 16 * TN, SUB = 16, TM = 8;
  constexpr int NQ = TN >= 4 ? TN / 4 : 1;
  __shared__ __align__(16) float As[SUB][BKo];
  __shared__ __align__(16) float Bs[SUB][BN];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int64_t c = blockIdx.x;
  const int sg = chunk_seg[c];
  const int K = segK ? segK[sg] : Kmax;
  const int N = segN ? segN[sg] : Nmax;
  const int k0 = blockIdx.y * BKo;
  const int n0 = blockIdx.z * BN;
  if (k0 >= K || n0 >= N) return;
  const int64_t r0 = chunk_row0[c];
  const int64_t r1 = r0 + chunk_rows[c];
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
  float* out = part + c * (int64_t)Kmax * Nmax;
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int gk = k0 + ty * TM + i;
    if (gk >= K) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int gn = TN >= 4 ? n0 + (tx + 16 * (j / 4)) * 4 + (j & 3) : n0 + tx * TN + j;
      if (gn < N) out[(int64_t)gk * Nmax + gn] = acc[i][j];
    }
  }
}

int gemm_tn(const RowSpace& rs, const TN& a, cudaStream_t s) {
  ABG_CHECK(a.K >= 1 && a.N >= 1, "gemm_tn: bad sizes");
  ABG_CHECK(a.lda % 4 == 0 && a.ldb % 4 == 0 && a.lda >= a.K && a.ldb >= a.N,
            "gemm_tn: leading dimensions must be multiples of 4 and cover the width");
  if (rs.n_chunks == 0) return ABG_OK;
  Scratch scr(s);
  float* part;
  ABG_TRY(scr.get(&part, (size_t)rs.n_chunks * a.K * a.N));
  bool tc = false;
  if (a.A16) ABG_TRY(tc_gemm_tn16(rs, a, part, s, &tc));
  if (!tc) ABG_TRY(tc_gemm_tn(rs, a, part, s, &tc));
  if (tc)
    return reduce_pieces<float>(rs, false, part, (int64_t)a.K * a.N, a.N, a.segK, a.K, a.segN,
                                a.N, a.C, a.ldc, a.c_seg, s);
  const int TNv = a.N <= 32 ? 2 : (a.N <= 64 ? 4 : 8);
  dim3 grid((unsigned)rs.n_chunks, (unsigned)ceil_div(a.K, 128), (unsigned)ceil_div(a.N, 16 * TNv));
#define ABG_TN_CASE(tn)                                                                          \
  if (TNv == tn) {                                                                               \
    k_gemm_tn_part<tn><<<grid, 256, 0, s>>>(rs.chunk_seg, rs.chunk_row0, rs.chunk_rows, a.K,     \
                                            a.N, a.segK, a.segN, a.A, a.lda, a.B, a.ldb, part); \
    note_launch();                                                                               \
  }
  ABG_TN_CASE(2) ABG_TN_CASE(4) ABG_TN_CASE(8)
#undef ABG_TN_CASE
  ABG_LAUNCH_CHECK();
  return reduce_pieces<float>(rs, false, part, (int64_t)a.K * a.N, a.N, a.segK, a.K, a.segN, a.N,
                              a.C, a.ldc, a.c_seg, s);
}

// column sums of A (rows of each segment): per-chunk FP64 partials, ordered reduction
__global__ void k_colsum_part(const int64_t* __restrict__ chunk_row0,
                              const int* __restrict__ chunk_rows, int N,
                              const float* __restrict__ A, int64_t lda,
                              double* __restrict__ part) {
  const int64_t c = blockIdx.x;
  const int64_t r0 = chunk_row0[c], r1 = r0 + chunk_rows[c];
  constexpr int U = 16;  // rows whose loads are in flight together (the adds stay in row order)
  for (int n = threadIdx.x; n < N; n += blockDim.x) {
    double s = 0.0;
    int64_t r = r0;
    for (; r + U <= r1; r += U) {
      float v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) v[u] = A[(r + u) * lda + n];
#pragma unroll
      for (int u = 0; u < U; ++u) s += (double)v[u];
    }
    for (; r < r1; ++r) s += (double)A[r * lda + n];
    part[c * N + n] = s;
  }
}

int column_sums(const RowSpace& rs, int N, const float* A, int64_t lda, double* out,
                int64_t oseg, cudaStream_t s) {
  Scratch scr(s);
  double* part;
  ABG_TRY(scr.get(&part, (size_t)std::max<int64_t>(1, rs.n_chunks) * N));
  if (rs.n_chunks) {
    k_colsum_part<<<(unsigned)rs.n_chunks, 128, 0, s>>>(rs.chunk_row0, rs.chunk_rows, N, A, lda,
                                                         part);
    note_launch();
  }
  ABG_LAUNCH_CHECK();
  return reduce_pieces<double>(rs, false, part, N, N, nullptr, 1, nullptr, N, out, N, oseg, s);
}

// ---------------------------------------------------------------------------
// Random features (Eqs. 13-14)
// ---------------------------------------------------------------------------
// R[i] <- R'[i] / sqrt(max(R'[i].r_s, 1e-300)) with s the row's segment; one warp per row,
// the row held in registers (PER values per lane, all loads in flight together). rf is r in
// FP32 (read through L1); each lane sums its PER products in FP32 and the lanes' partials are
// added exactly in (hi, lo) FP32 pairs (Knuth's TwoSum), so the dot keeps the accuracy of a
// double sum without the GPU's slow FP64 pipe; one lane takes the square root in FP64.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bp = s - a;
  e = (a - (s - bp)) + (b - bp);
}

template <int PER>
__global__ void k_rf_normalise(int64_t n, int w2, float* __restrict__ R, int64_t ldr,
                               const float* __restrict__ rf, const int* __restrict__ row_seg,
                               int* __restrict__ clamped, __nv_bfloat16* __restrict__ R16,
                               int64_t ldr16) {
  const int64_t row = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  const float* rsg = rf + (int64_t)row_seg[row] * w2;
  float* rp = R + row * ldr;
  float x[PER];
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int c = lane + 32 * i;
    x[i] = c < w2 ? rp[c] : 0.f;
  }
  float hi = 0.f, lo = 0.f;
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int c = lane + 32 * i;
    if (c < w2) hi = fmaf(x[i], __ldg(rsg + c), hi);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float ho = __shfl_xor_sync(0xffffffffu, hi, o);
    const float lo2 = __shfl_xor_sync(0xffffffffu, lo, o);
    float e;
    two_sum(hi, ho, hi, e);
    lo += lo2 + e;
  }
  float inv = 0.f;
  int clamp = 0;
  if (lane == 0) {
    double dot = (double)hi + (double)lo;
    clamp = !(dot > 1e-300);
    if (clamp) dot = 1e-300;
    if (dot > 1e-30 && dot < 1e30) {
      // FP32 reciprocal square root and one Newton step (about 1 ulp): an FP64 square root
      // and division per row would occupy the SM's narrow FP64 unit for ~2 ms at 2M rows
      const float df = (float)dot;
      const float y = rsqrtf(df);
      inv = y * fmaf(-0.5f * df * y, y, 1.5f);
    } else {
      inv = (float)(1.0 / sqrt(dot));
    }
  }
  inv = __shfl_sync(0xffffffffu, inv, 0);
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int c = lane + 32 * i;
    if (c >= w2) continue;
    const float v = x[i] * inv;
    rp[c] = v;
    if (R16) R16[row * ldr16 + c] = __float2bfloat16_rn(v);
  }
  if (clamp) atomicAdd(clamped + row_seg[row], 1);
}

__global__ void k_f64_to_f32(int64_t n, const double* __restrict__ a, float* __restrict__ b) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}

int random_features(const RowSpace& rs, const float* zhat, int d, int64_t ldz, const float* qt,
                    int64_t ldq, float* R, int64_t ldr, int* clamped_dev, cudaStream_t s,
                    __nv_bfloat16* R16, int64_t ldr16) {
  ABG_CHECK(ldr >= 2 * d && ldr % 4 == 0, "random_features: ldr must be >= 2d, multiple of 4");
  Scratch scr(s);
  double* cpart;
  ABG_TRY(scr.get(&cpart, (size_t)std::max<int64_t>(1, rs.n_tiles) * 2 * d));
  NN a;
  a.A = zhat;
  a.lda = ldz;
  a.B = qt;
  a.ldb = ldq;
  a.b_seg = (int64_t)d * ldq;
  a.C = R;
  a.ldc = ldr;
  a.N = a.K = d;
  a.sincos = true;
  a.in_scale = (float)sqrt((double)d);
  a.out_scale = (float)sqrt(exp(1.0) / d);
  a.colsum_part = cpart;
  ABG_TRY(gemm_nn(rs, a, s));
  double* r;
  ABG_TRY(scr.get(&r, (size_t)rs.nseg * 2 * d));
  ABG_TRY(reduce_pieces<double>(rs, true, cpart, 2 * d, 2 * d, nullptr, 1, nullptr, 2 * d, r,
                                2 * d, 2 * d, s));
  const unsigned grid = (unsigned)ceil_div(rs.rows, 8);
  const int w2 = 2 * d;
  float* rf;
  ABG_TRY(scr.get(&rf, (size_t)rs.nseg * w2));
  k_f64_to_f32<<<(unsigned)ceil_div((int64_t)rs.nseg * w2, 256), 256, 0, s>>>(
      (int64_t)rs.nseg * w2, r, rf);
  note_launch();
#define ABG_RF_CASE(per)                                                                  \
  if (w2 <= 32 * per) {                                                                   \
    k_rf_normalise<per><<<grid, 256, 0, s>>>(rs.rows, w2, R, ldr, rf, rs.row_seg, clamped_dev, \
                                             R16, ldr16);                                 \
  } else
  ABG_RF_CASE(2) ABG_RF_CASE(4) ABG_RF_CASE(8) ABG_RF_CASE(16) ABG_RF_CASE(32) ABG_RF_CASE(64) {
    set_error("random features: 2d above 2048");
    return ABG_EINVAL;
  }
#undef ABG_RF_CASE
  note_launch();
  ABG_LAUNCH_CHECK();
  return ABG_OK;
}

// ---------------------------------------------------------------------------
// Eq. 16 per segment: H <- H * max(R^T Phi, 0) / (H (Phi^T Phi)); a non-positive denominator
// gives 0. H_s at H + s*hseg (m x k_s, ld ldh), A_s (m x k_s, ld lda), G_s (k_s x k_s, ld ldg).
// ---------------------------------------------------------------------------
__global__ void k_nmf_h(int m, const int* __restrict__ segk, int kmax, const float* __restrict__ H,
                        int64_t ldh, int64_t hseg, const double* __restrict__ A, int64_t lda,
                        int64_t aseg, const double* __restrict__ G, int64_t ldg, int64_t gseg,
                        float* __restrict__ Hn) {
  const int sg = blockIdx.y;
  const int k = segk[sg];
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= m * kmax) return;
  const int j = idx / kmax, l = idx % kmax;
  if (l >= k) return;
  const float* Hs = H + sg * hseg;
  const double* As = A + sg * aseg;
  const double* Gs = G + sg * gseg;
  double den = 0.0;
  for (int p = 0; p < k; ++p) den += (double)Hs[(int64_t)j * ldh + p] * Gs[(int64_t)p * ldg + l];
  const double num = fmax(As[(int64_t)j * lda + l], 0.0);
  Hn[sg * hseg + (int64_t)j * ldh + l] =
      den > 0.0 ? (float)((double)Hs[(int64_t)j * ldh + l] * num / den) : 0.f;
}

int nmf_update_h(int nseg, int m, const int* segk, int kmax, float* H, int64_t ldh, int64_t hseg,
                 const double* A, int64_t lda, int64_t aseg, const double* G, int64_t ldg,
                 int64_t gseg, cudaStream_t s) {
  Scratch scr(s);
  float* Hn;
  ABG_TRY(scr.get(&Hn, (size_t)nseg * hseg));
  ABG_CUDA(cudaMemcpyAsync(Hn, H, sizeof(float) * nseg * hseg, cudaMemcpyDeviceToDevice, s));
  dim3 grid((unsigned)ceil_div((int64_t)m * kmax, 256), (unsigned)nseg);
  k_nmf_h<<<grid, 256, 0, s>>>(m, segk, kmax, H, ldh, hseg, A, lda, aseg, G, ldg, gseg, Hn);
  note_launch();
  ABG_LAUNCH_CHECK();
  ABG_CUDA(cudaMemcpyAsync(H, Hn, sizeof(float) * nseg * hseg, cudaMemcpyDeviceToDevice, s));
  return ABG_OK;
}

// C_s[p][q] = sum_{j < m} A_s[j][p] H_s[j][q] for p, q < k_s (A FP64, H FP32, C FP64)
__global__ void k_small_atb(int m, const int* __restrict__ segk, int kmax,
                            const double* __restrict__ A, int64_t lda, int64_t aseg,
                            const float* __restrict__ H, int64_t ldh, int64_t hseg,
                            double* __restrict__ C, int64_t ldc, int64_t cseg) {
  const int sg = blockIdx.y;
  const int k = segk[sg];
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= kmax * kmax) return;
  const int p = idx / kmax, q = idx % kmax;
  if (p >= k || q >= k) return;
  const double* As = A + sg * aseg;
  const float* Hs = H + sg * hseg;
  double acc = 0.0;
  for (int j = 0; j < m; ++j) acc += As[(int64_t)j * lda + p] * (double)Hs[(int64_t)j * ldh + q];
  C[sg * cseg + (int64_t)p * ldc + q] = acc;
}

int small_atb(int nseg, int m, const int* segk, int kmax, const double* A, int64_t lda,
              int64_t aseg, const float* H, int64_t ldh, int64_t hseg, double* C, int64_t ldc,
              int64_t cseg, cudaStream_t s) {
  dim3 grid((unsigned)ceil_div((int64_t)kmax * kmax, 128), (unsigned)nseg);
  k_small_atb<<<grid, 128, 0, s>>>(m, segk, kmax, A, lda, aseg, H, ldh, hseg, C, ldc, cseg);
  note_launch();
  ABG_LAUNCH_CHECK();
  return ABG_OK;
}

// ---------------------------------------------------------------------------
// Per-chunk cluster sums S[l][m] = sum_{i in chunk, label i = l} X[i, m] and counts.
// The chunk's rows are first bucketed by label with a stable counting sort in shared
// memory; then each warp owns whole clusters and sums their rows in increasing row order
// into registers (a float4 of columns per lane, 128 columns per CTA column tile). Every
// sum is the row-ordered FP32 sum starting from 0, so the result does not depend on the
// launch shape. Labels outside [0, kmax) are skipped.
// ---------------------------------------------------------------------------
constexpr int kCsWarps = 8;
constexpr int kCsCols = 128;  // columns per CTA (32 lanes x 4)

__global__ void __launch_bounds__(kCsWarps * 32) k_cluster_sums(
    const int64_t* __restrict__ chunk_row0, const int* __restrict__ chunk_rows, int kmax, int w,
    const float* __restrict__ X, int64_t ldx, const int32_t* __restrict__ labels,
    float* __restrict__ part) {
  extern __shared__ int cs_smem[];
  int* cnt = cs_smem;      // [kmax] rows per label
  int* off = cnt + kmax;   // [kmax] bucket starts, then (after the scatter) bucket ends
  int* idx = off + kmax;   // [rows] chunk-local row ids, bucketed by label, stable
  const int64_t c = blockIdx.x;
  const int col0 = blockIdx.y * kCsCols;
  const int64_t r0 = chunk_row0[c];
  const int rows = chunk_rows[c];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int l = threadIdx.x; l < kmax; l += blockDim.x) cnt[l] = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < rows; i += blockDim.x) {
    const int l = labels[r0 + i];
    if ((unsigned)l < (unsigned)kmax) atomicAdd(cnt + l, 1);  // counts: order-free
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int run = 0;
    for (int l = 0; l < kmax; ++l) {
      off[l] = run;
      run += cnt[l];
    }
  }
  __syncthreads();
  if (warp == 0) {  // stable scatter: rows in order, 32 at a time, ranks by lane
    for (int base = 0; base < rows; base += 32) {
      const int i = base + lane;
      const int l = i < rows ? labels[r0 + i] : -1;
      const bool ok = (unsigned)l < (unsigned)kmax;
      const unsigned peers = __match_any_sync(0xffffffffu, ok ? l : -1);
      const int rank = __popc(peers & ((1u << lane) - 1u));
      const int pos = ok ? off[l] + rank : 0;
      __syncwarp();
      if (ok) {
        idx[pos] = i;
        if (rank == 0) off[l] += __popc(peers);
      }
      __syncwarp();
    }
  }
  __syncthreads();
  const int64_t width = (int64_t)kmax * w + kmax;
  float* out = part + c * width;
  const int cc = col0 + 4 * lane;
  const bool act = cc < w;
  const float* xc = X + (int64_t)r0 * ldx + cc;
  for (int l = warp; l < kmax; l += kCsWarps) {
    const int end = off[l], beg = end - cnt[l];
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    if (act) {
      int j = beg;
      constexpr int U = 8;  // rows whose loads are in flight together
      for (; j + U <= end; j += U) {
        float4 v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) v[u] = ld_f4(xc + (int64_t)idx[j + u] * ldx);
#pragma unroll
        for (int u = 0; u < U; ++u) {
          acc.x += v[u].x;
          acc.y += v[u].y;
          acc.z += v[u].z;
          acc.w += v[u].w;
        }
      }
      for (; j < end; ++j) {
        const float4 v = ld_f4(xc + (int64_t)idx[j] * ldx);
        acc.x += v.x;
        acc.y += v.y;
        acc.z += v.z;
        acc.w += v.w;
      }
      float* o = out + (int64_t)l * w + cc;
      o[0] = acc.x;
      if (cc + 1 < w) o[1] = acc.y;
      if (cc + 2 < w) o[2] = acc.z;
      if (cc + 3 < w) o[3] = acc.w;
    }
    if (blockIdx.y == 0 && lane == 0) out[(int64_t)kmax * w + l] = (float)cnt[l];
  }
}

// S_s (layout [kmax][w] sums, then kmax counts) at S + s * (kmax*w + kmax)
static int cluster_sums(const RowSpace& rs, const float* X, int w, int64_t ldx,
                        const int32_t* labels, int kmax, double* S, cudaStream_t s) {
  ABG_CHECK(ldx % 4 == 0 && reinterpret_cast<uintptr_t>(X) % 16 == 0,
            "cluster sums: rows must be 16-byte aligned");
  Scratch scr(s);
  const int64_t width = (int64_t)kmax * w + kmax;
  float* part;
  ABG_TRY(scr.get(&part, (size_t)std::max<int64_t>(1, rs.n_chunks) * width));
  const size_t smem = sizeof(int) * (2 * (size_t)kmax + kChunk);
  if (rs.n_chunks) {
    ABG_TRY(raise_smem_limit((const void*)k_cluster_sums, smem));
    dim3 grid((unsigned)rs.n_chunks, (unsigned)ceil_div(w, kCsCols));
    k_cluster_sums<<<grid, kCsWarps * 32, smem, s>>>(rs.chunk_row0, rs.chunk_rows, kmax, w, X,
                                                     ldx, labels, part);
    note_launch();
  }
  ABG_LAUNCH_CHECK();
  return reduce_pieces<float>(rs, false, part, width, (int)width, nullptr, 1, nullptr,
                              (int)width, S, width, width, s);
}

// ---------------------------------------------------------------------------
// Algorithm 3 per segment
// ---------------------------------------------------------------------------
// T_s[m][l] = S_s[l][m] / sqrt(n_l) for m, l < k_s (0 for an empty cluster), float stride kp.
__global__ void k_nci_finalize(const int* __restrict__ segk, int kmax, const double* __restrict__ S,
                               int kp, float* __restrict__ T, double* __restrict__ t64,
                               int* __restrict__ empty, double* __restrict__ mout) {
  const int sg = blockIdx.y;
  const int k = segk[sg];
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= kmax * kmax) return;
  const int m = idx / kmax, l = idx % kmax;
  const double* Ss = S + (int64_t)sg * ((int64_t)kmax * kmax + kmax);
  float* Ts = T + (int64_t)sg * kmax * kp;
  double v = 0.0;
  if (m < k && l < k) {
    const double cnt = Ss[(int64_t)kmax * kmax + l];
    v = cnt > 0 ? Ss[(int64_t)l * kmax + m] / sqrt(cnt) : 0.0;
    if (m == 0 && cnt <= 0) atomicAdd(empty + sg, 1);
    if (t64 && !mout) t64[(int64_t)sg * kmax * kmax + m * kmax + l] = v;
  }
  if (mout)  // Phi^T Y for the Procrustes factor (zero outside k_s x k_s)
    mout[(int64_t)sg * kmax * kmax + (int64_t)m * kmax + l] = v;
  else
    Ts[m * kp + l] = (float)v;
}

// Orthogonal Procrustes factor T = U_r V_r^T of M = Phi^T Y = U S V^T (singular values above
// 1e-5 s_1): W = M V S_r^+, then T = W V^T. evals = s^2 (descending), evecs = V (columns).
__global__ void k_polar_w(const int* __restrict__ segk, int kmax, const double* __restrict__ M,
                          const double* __restrict__ evals, const double* __restrict__ evecs,
                          double* __restrict__ W, const int* __restrict__ skip) {
  const int sg = blockIdx.y;
  if (skip[sg]) return;  // T already written by the Newton-Schulz iteration
  const int k = segk[sg];
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= kmax * kmax) return;
  const int m = idx / kmax, j = idx % kmax;
  const int64_t o = (int64_t)sg * kmax * kmax;
  const double* ev = evals + (int64_t)sg * kmax;
  double v = 0.0;
  if (m < k && j < k && ev[0] > 0.0 && ev[j] > 1e-10 * ev[0]) {
    double acc = 0.0;
    for (int p = 0; p < k; ++p) acc += M[o + (int64_t)m * kmax + p] * evecs[o + (int64_t)p * kmax + j];
    v = acc / sqrt(ev[j]);
  }
  W[o + (int64_t)m * kmax + j] = v;
}

__global__ void k_polar_t(const int* __restrict__ segk, int kmax, const double* __restrict__ W,
                          const double* __restrict__ evecs, int kp, float* __restrict__ T,
                          double* __restrict__ t64, const int* __restrict__ skip) {
  const int sg = blockIdx.y;
  if (skip[sg]) return;
  const int k = segk[sg];
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= kmax * kmax) return;
  const int m = idx / kmax, l = idx % kmax;
  const int64_t o = (int64_t)sg * kmax * kmax;
  double v = 0.0;
  if (m < k && l < k)
    for (int j = 0; j < k; ++j) v += W[o + (int64_t)m * kmax + j] * evecs[o + (int64_t)l * kmax + j];
  if (t64 && m < k && l < k) t64[o + (int64_t)m * kmax + l] = v;
  T[(int64_t)sg * kmax * kp + m * kp + l] = (float)v;
}

// V_s = I (k_s x k_s, column-major with column stride k_s, inside a kmax x kmax slab)
__global__ void k_eye_blocks(const int* __restrict__ segk, int kmax, float* __restrict__ V) {
  const int sg = blockIdx.y;
  const int k = segk[sg];
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= k * k) return;
  V[(int64_t)sg * kmax * kmax + q] = (q / k == q % k) ? 1.f : 0.f;
}

__global__ void k_nci_init(int nseg, const int* __restrict__ segk, int kmax, int kp,
                           float* __restrict__ T) {
  const int64_t total = (int64_t)nseg * kmax * kp;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int sg = (int)(idx / ((int64_t)kmax * kp));
    const int rem = (int)(idx % ((int64_t)kmax * kp));
    const int m = rem / kp, l = rem % kp;
    T[idx] = (m == l && m < segk[sg]) ? 1.f : 0.f;
  }
}

__global__ void k_reset_counters(int nseg, int* __restrict__ c) {
  const int sg = blockIdx.x * blockDim.x + threadIdx.x;
  if (sg >= nseg) return;
  c[sg] = 0;                 // changes
  c[nseg + sg] = 0x7f800000; // minimum margin (+inf bits)
  c[2 * nseg + sg] = 0;      // empty clusters
}

int nci_run(const RowSpace& rs, const SegSizes& ss, const float* phi, int64_t ldphi, int t_g,
            int flags, int32_t* labels, float* margin, double* t_out, int* counters,
            std::vector<int>* passes, cudaStream_t s) {
  const int kmax = ss.k_max, nseg = rs.nseg;
  ABG_CHECK(kmax >= 1 && kmax <= kMaxK, "nci: need 1 <= k <= %d", kMaxK);
  const bool procrustes = flags & ABG_NCI_PROCRUSTES;
  const bool early = flags & ABG_NCI_EARLY_STOP;
  Scratch scr(s);
  const int kp = (int)round_up(kmax, 4);
  float* T;
  ABG_TRY(scr.get(&T, (size_t)nseg * kmax * kp));
  double* S;
  ABG_TRY(scr.get(&S, (size_t)nseg * ((size_t)kmax * kmax + kmax)));
  double *M = nullptr, *W = nullptr, *evals = nullptr, *evecs = nullptr;
  float* warm = nullptr;  // right singular vectors of the last Jacobi pass over Phi^T Y
  int* ns_done = nullptr;  // per segment: the Newton-Schulz iteration gave this pass's T
  // ABG_POLAR=jacobi: every pass through the Jacobi SVD (for comparisons of the two forms)
  const char* pe = std::getenv("ABG_POLAR");
  const bool jacobi_only = pe && std::strcmp(pe, "jacobi") == 0;
  if (procrustes) {
    ABG_TRY(scr.get(&warm, (size_t)nseg * kmax * kmax));
    ABG_TRY(scr.get(&M, (size_t)nseg * kmax * kmax));
    ABG_TRY(scr.get(&W, (size_t)nseg * kmax * kmax));
    ABG_TRY(scr.get(&evals, (size_t)nseg * kmax));
    ABG_TRY(scr.get(&evecs, (size_t)nseg * kmax * kmax));
    ABG_TRY(scr.get(&ns_done, (size_t)nseg));
    ABG_CUDA(cudaMemsetAsync(ns_done, 0, sizeof(int) * nseg, s));
    // the Jacobi sweeps start from the rotations of the last pass that ran them, the first
    // time from the identity (the same as no warm start)
    k_eye_blocks<<<dim3((unsigned)ceil_div((int64_t)kmax * kmax, 256), (unsigned)nseg), 256, 0,
                   s>>>(ss.k, kmax, warm);
    note_launch();
  }
  if (passes) passes->assign(nseg, t_g);
  std::vector<int> done(nseg, 0), host(nseg);
  int n_done = 0;
  k_nci_init<<<(unsigned)std::min<int64_t>(ceil_div((int64_t)nseg * kmax * kp, 256), 4096), 256, 0,
               s>>>(nseg, ss.k, kmax, kp, T);
  note_launch();
  k_reset_counters<<<(unsigned)ceil_div(nseg, 256), 256, 0, s>>>(nseg, counters);
  note_launch();
  for (int t = 0; t < t_g; ++t) {
    k_reset_counters<<<(unsigned)ceil_div(nseg, 256), 256, 0, s>>>(nseg, counters);
    note_launch();
    NN a;
    a.A = phi;
    a.lda = ldphi;
    a.B = T;
    a.ldb = kp;
    a.b_seg = (int64_t)kmax * kp;
    a.N = a.K = kmax;
    a.segN = a.segK = ss.k;
    a.argmax = true;
    a.labels = labels;
    a.margin = margin;
    a.first = t == 0;
    a.changes = counters;
    a.minbits = (unsigned*)(counters + nseg);
    ABG_TRY(gemm_nn(rs, a, s));
    ABG_TRY(cluster_sums(rs, phi, kmax, ldphi, labels, kmax, S, s));
    dim3 g((unsigned)ceil_div(kmax * kmax, 256), (unsigned)nseg);
    k_nci_finalize<<<g, 256, 0, s>>>(ss.k, kmax, S, kp, T, t_out, counters + 2 * nseg, M);
    note_launch();
    if (procrustes) {
      // Newton-Schulz on a thread-block cluster; a segment it leaves (done = 0) goes through
      // the Jacobi SVD, whose sweeps start from the rotations it found last time (consecutive
      // passes move few labels, so Phi^T Y changes little)
      if (!jacobi_only)
        ABG_TRY(polar_newton_schulz(nseg, ss.k, kmax, M, kp, T, t_out, ns_done, s));
      ABG_TRY(svd_right(nseg, kmax, ss.k, kmax, M, evals, evecs, s, warm, true, ns_done, true));
      k_polar_w<<<g, 256, 0, s>>>(ss.k, kmax, M, evals, evecs, W, ns_done);
      note_launch();
      k_polar_t<<<g, 256, 0, s>>>(ss.k, kmax, W, evecs, kp, T, t_out, ns_done);
      note_launch();
    }
    ABG_LAUNCH_CHECK();
    if (early && t >= 1) {  // a pass that changed no label leaves Y and T at a fixed point
      ABG_CUDA(cudaMemcpyAsync(host.data(), counters, sizeof(int) * nseg, cudaMemcpyDeviceToHost,
                               s));
      ABG_CUDA(cudaStreamSynchronize(s));
      for (int i = 0; i < nseg; ++i)
        if (!done[i] && host[i] == 0) {
          done[i] = 1;
          ++n_done;
          if (passes) (*passes)[i] = t + 1;
        }
      if (n_done == nseg) break;
    }
  }
  if (t_g == 0) ABG_CUDA(cudaMemsetAsync(labels, 0, sizeof(int32_t) * rs.rows, s));
  return ABG_OK;
}

// ---------------------------------------------------------------------------
// Eq. 8 per segment through the cluster sums s_l (k x m, FP64) and counts n_l
// ---------------------------------------------------------------------------
__global__ void k_objective_final(const int* __restrict__ segk, int kmax, int m,
                                  const double* __restrict__ S, double* __restrict__ out) {
  // one CTA per segment: total = sum_l s_l; obj = sum_l s_l.(total - s_l)/n_l; J = sum |s_l|^2/n_l
  __shared__ double red_o[256], red_j[256];
  const int sg = blockIdx.x;
  const int k = segk[sg];
  const double* Ss = S + (int64_t)sg * ((int64_t)kmax * m + kmax);
  double o = 0.0, jv = 0.0;
  for (int c = threadIdx.x; c < m; c += blockDim.x) {
    double tot = 0.0;
    for (int l = 0; l < k; ++l) tot += Ss[(int64_t)l * m + c];
    for (int l = 0; l < k; ++l) {
      const double cnt = Ss[(int64_t)kmax * m + l];
      if (cnt > 0) {
        const double sv = Ss[(int64_t)l * m + c];
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
    out[2 * sg] = so;
    out[2 * sg + 1] = sj;
  }
}

int objective(const RowSpace& rs, const SegSizes& ss, const float* R, int m, int64_t ldr,
              const int32_t* labels, double* out_dev, cudaStream_t s) {
  const int kmax = ss.k_max;
  ABG_CHECK(kmax >= 1 && kmax <= kMaxK, "objective: need 1 <= k <= %d", kMaxK);
  Scratch scr(s);
  double* S;
  ABG_TRY(scr.get(&S, (size_t)rs.nseg * ((size_t)kmax * m + kmax)));
  ABG_TRY(cluster_sums(rs, R, m, ldr, labels, kmax, S, s));
  k_objective_final<<<(unsigned)rs.nseg, 256, 0, s>>>(ss.k, kmax, m, S, out_dev);
  note_launch();
  ABG_LAUNCH_CHECK();
  return ABG_OK;
}

}  // namespace abg
