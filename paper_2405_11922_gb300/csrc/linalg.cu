// Random matrices and small dense linear algebra of the method, per segment of
// a batch (a plain solve is one segment):
//   * Gaussian draws from Philox4x32-10 (Salmon et al., SC'11) + Box-Muller
//     on the device (G of Algorithm 1, the randomized-SVD test matrices),
//     keyed by each segment's own seed;
//   * Q = orthogonal factor of QR(G) (Algorithm 1), by CholeskyQR2 in FP64;
//   * CholeskyQR2 of tall FP32 blocks (FP64 Gram / Cholesky, FP32 apply);
//   * the truncated randomized SVD of Halko, Martinsson and Tropp (subspace
//     iteration) used by Algorithm 2's seeding (Eq. 18) and by the attribute
//     reduction of Section 3.2.1 (Eq. 15): the small SVD of B^T = A^T Q runs as
//     a one-sided (Hestenes) Jacobi in FP32, one CTA per segment.
#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.cuh"

namespace abg {

// ---------------------------------------------------------------------------
// Philox4x32-10 and Box-Muller
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k.x += W0;
      k.y += W1;
    }
    const uint32_t lo0 = M0 * c.x, hi0 = __umulhi(M0, c.x);
    const uint32_t lo1 = M1 * c.z, hi1 = __umulhi(M1, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

// Segment blockIdx.y's matrix is rows x cols_s (cols_s = segcols[s], else cols): its entry
// e = r * cols_s + c comes from the counter mapping of abg.h, so a segment draws the same
// numbers whatever the batch's widest segment; columns cols_s..cols-1 are set to 0.
template <class T>
__global__ void k_gaussian(const uint64_t* __restrict__ seeds, uint32_t stream_id, int rows,
                           int cols, const int* __restrict__ segcols, T* out, int64_t ld,
                           int64_t oseg) {
  const int sg = blockIdx.y;
  const uint64_t seed = seeds[sg];
  const int cs = segcols ? segcols[sg] : cols;
  T* o = out + sg * oseg;
  const int64_t total = (int64_t)rows * cs;
  const int64_t nb = (total + 3) / 4;
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < nb;
       b += (int64_t)gridDim.x * blockDim.x) {
    uint4 x = philox4x32_10(make_uint4((uint32_t)b, (uint32_t)(b >> 32), stream_id, 0u),
                            make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
    const double two32 = 4294967296.0;
    double u[4] = {((double)x.x + 0.5) / two32, ((double)x.y + 0.5) / two32,
                   ((double)x.z + 0.5) / two32, ((double)x.w + 0.5) / two32};
    double z[4];
#pragma unroll
    for (int a = 0; a < 4; a += 2) {
      const double rad = sqrt(-2.0 * log(u[a]));
      double sn, cn;
      sincospi(2.0 * u[a + 1], &sn, &cn);
      z[a] = rad * cn;
      z[a + 1] = rad * sn;
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t e = 4 * b + j;
      if (e < total) o[(e / cs) * ld + (e % cs)] = (T)z[j];
    }
  }
  if (cs < cols) {
    const int64_t pad = (int64_t)rows * (cols - cs);
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < pad;
         q += (int64_t)gridDim.x * blockDim.x)
      o[(q / (cols - cs)) * ld + cs + (q % (cols - cs))] = (T)0;
  }
}

int gaussian_f64(int nseg, const uint64_t* seeds, int stream_id, int rows, int cols, double* out,
                 int64_t ld, int64_t oseg, cudaStream_t s) {
  const int64_t nb = ((int64_t)rows * cols + 3) / 4;
  dim3 grid((unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(nb, 256), 2048)),
            (unsigned)nseg);
  k_gaussian<double><<<grid, 256, 0, s>>>(seeds, (uint32_t)stream_id, rows, cols, nullptr, out,
                                          ld, oseg);
  note_launch();
  ABG_LAUNCH_CHECK();
  return ABG_OK;
}

int gaussian_f32(int nseg, const uint64_t* seeds, int stream_id, int rows, int cols,
                 const int* segcols, float* out, int64_t ld, int64_t oseg, cudaStream_t s) {
  const int64_t nb = ((int64_t)rows * cols + 3) / 4;
  dim3 grid((unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(nb, 256), 2048)),
            (unsigned)nseg);
  k_gaussian<float><<<grid, 256, 0, s>>>(seeds, (uint32_t)stream_id, rows, cols, segcols, out,
                                         ld, oseg);
  note_launch();
  ABG_LAUNCH_CHECK();
  return ABG_OK;
}

// ---------------------------------------------------------------------------
// Blocked Cholesky R^T R = G (upper R, FP64) over many SMs, and R^-1 by columns.
// Right-looking, 32-column blocks: the diagonal block is factored by one warp per segment
// (one square root and one division per pivot), the block row to its right is solved with
// the diagonal block's inverse, and the trailing upper triangle is updated by one thread per
// element. A pivot at or below 1e-13 max diag(G) counts as a breakdown: its row of R (and its
// column of R^-1) stays zero, as in the unblocked form. R (and Ri) of segment s use the
// segment's own l_s as row stride inside their slabs.
// ---------------------------------------------------------------------------
constexpr int kCholB = 32;

// R = upper triangle of G (zeros below); tol_s = 1e-13 max_i G_s[i][i]
__global__ void k_chol_init(const int* __restrict__ segl, int lfix, const double* __restrict__ Gall,
                            int64_t ldg, int64_t gseg, double* __restrict__ Rall, int64_t rseg,
                            double* __restrict__ tol) {
  const int sg = blockIdx.y;
  const int l = segl ? segl[sg] : lfix;
  const double* G = Gall + sg * gseg;
  double* R = Rall + sg * rseg;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < (int64_t)l * l;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(q / l), j = (int)(q % l);
    R[q] = j >= i ? G[(int64_t)i * ldg + j] : 0.0;
  }
  if (blockIdx.x == 0 && threadIdx.x < 32) {
    double m = 0.0;
    for (int i = threadIdx.x; i < l; i += 32) m = fmax(m, fabs(G[(int64_t)i * ldg + i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0) tol[sg] = 1e-13 * m;
  }
}

// Diagonal block k of each segment (one CTA of four warps): factor in place, and its
// upper-triangular inverse into D_s (32 x 32, row stride 32). Warp w holds rows w, w + 4, ...
// of the block in registers (lane c = column c), so the FP64 work of every pivot is spread
// over the SM's four sub-partitions: the owner of row j turns it into row j of the factor
// (one reciprocal square root gives the pivot and its inverse) and publishes it in shared
// memory, then every warp updates its rows below j. Each warp updates its rows in ascending
// order, so the next pivot's owner has its row ready first. The inverse X (R X = I) is a back
// substitution over all columns at once: for p descending the owner of row p finishes it,
// x[p] = (delta_pc - acc[p]) / R[p][p], publishes it, and every warp adds R[r][p] x[p] to its
// rows r < p. Pivot and solved rows alternate between two shared buffers, so one barrier per
// step orders them.
constexpr int kCholW = 4;                 // warps per diagonal block
constexpr int kCholR = kCholB / kCholW;  // rows per warp

__global__ void __launch_bounds__(32 * kCholW) k_chol_diag(const int* __restrict__ segl, int lfix,
                                                           int k, double* __restrict__ Rall,
                                                           int64_t rseg,
                                                           const double* __restrict__ tol,
                                                           double* __restrict__ Dall,
                                                           int* __restrict__ breakdowns) {
  __shared__ double row[2][kCholB];  // the pivot row (factor) / the solved row (inverse)
  __shared__ double rinv[kCholB];
  const int sg = blockIdx.x;
  const int l = segl ? segl[sg] : lfix;
  const int o = k * kCholB;
  if (o >= l) return;  // whole CTA
  const int bs = min(kCholB, l - o);
  double* R = Rall + sg * rseg;
  const int w = threadIdx.x >> 5, c = threadIdx.x & 31;  // this lane's column
  double a[kCholR];  // rows w + 4 i of the block, column c
#pragma unroll
  for (int i = 0; i < kCholR; ++i) {
    const int r = w + kCholW * i;
    a[i] = (c < bs && r <= c) ? R[(int64_t)(o + r) * l + o + c] : 0.0;
  }
  const double t = tol[sg];
#pragma unroll
  for (int j = 0; j < kCholB; ++j) {
    if (j >= bs) {  // uniform over the CTA
      if (threadIdx.x == 0) rinv[j] = 0.0;
      continue;
    }
    if (w == j % kCholW) {
      const int ij = j / kCholW;
      const double pv = __shfl_sync(0xffffffffu, a[ij], j);
      const bool ok = pv > t;
      const double rs = ok ? rsqrt(pv) : 0.0;
      if (!ok && c == 0) atomicAdd(breakdowns, 1);
      a[ij] = c == j ? pv * rs : (c > j ? a[ij] * rs : a[ij]);  // row j (0 after a breakdown)
      row[j & 1][c] = a[ij];
      if (c == 0) rinv[j] = rs;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kCholR; ++i) {
      const int r = w + kCholW * i;
      if (r > j && c >= r) a[i] = fma(-row[j & 1][r], row[j & 1][c], a[i]);
    }
  }
#pragma unroll
  for (int i = 0; i < kCholR; ++i) {
    const int r = w + kCholW * i;
    if (c < bs && r <= c) R[(int64_t)(o + r) * l + o + c] = a[i];
  }
  __syncthreads();  // rinv complete; the row buffers are free again
  double x[kCholR];
#pragma unroll
  for (int i = 0; i < kCholR; ++i) x[i] = 0.0;
#pragma unroll
  for (int p = kCholB - 1; p >= 0; --p) {
    if (w == p % kCholW) {
      const int ip = p / kCholW;
      x[ip] = ((c == p ? 1.0 : 0.0) - x[ip]) * rinv[p];
      row[p & 1][c] = x[ip];
    }
    __syncthreads();
    const double xp = row[p & 1][c];
#pragma unroll
    for (int i = 0; i < kCholR; ++i) {
      const int r = w + kCholW * i;
      const double rrp = __shfl_sync(0xffffffffu, a[i], p);  // R[r][p] (lane p of row r)
      if (r < p) x[i] = fma(rrp, xp, x[i]);
    }
  }
  double* D = Dall + (int64_t)sg * kCholB * kCholB;
#pragma unroll
  for (int i = 0; i < kCholR; ++i) {
    const int r = w + kCholW * i;
    D[r * kCholB + c] = c < bs ? x[i] : 0.0;
  }
}

// Block row k to the right of the diagonal block: R[o+t][j] = sum_{s <= t} D[s][t] R[o+s][j]
__global__ void k_chol_panel(const int* __restrict__ segl, int lfix, int k, double* __restrict__ Rall,
                             int64_t rseg, const double* __restrict__ Dall) {
  __shared__ double D[kCholB][kCholB];
  const int sg = blockIdx.y;
  const int l = segl ? segl[sg] : lfix;
  const int o = k * kCholB;
  for (int q = threadIdx.x; q < kCholB * kCholB; q += blockDim.x)
    D[q / kCholB][q % kCholB] = Dall[(int64_t)sg * kCholB * kCholB + q];
  __syncthreads();
  if (o + kCholB >= l) return;
  const int j = o + kCholB + blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= l) return;
  double* R = Rall + sg * rseg;
  double v[kCholB];
#pragma unroll
  for (int s2 = 0; s2 < kCholB; ++s2) v[s2] = R[(int64_t)(o + s2) * l + j];
#pragma unroll
  for (int t = kCholB - 1; t >= 0; --t) {  // top-down would overwrite inputs still needed
    double acc = 0.0;
#pragma unroll
    for (int s2 = 0; s2 <= t; ++s2) acc += D[s2][t] * v[s2];
    R[(int64_t)(o + t) * l + j] = acc;
  }
}

// Trailing update: R[i][j] -= sum_t R[o+t][i] R[o+t][j] for o + 32 <= i <= j < l
__global__ void k_chol_update(const int* __restrict__ segl, int lfix, int k, int m,
                              double* __restrict__ Rall, int64_t rseg) {
  const int sg = blockIdx.y;
  const int l = segl ? segl[sg] : lfix;
  const int o = k * kCholB, base = o + kCholB;
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (int64_t)m * m) return;
  const int i = base + (int)(q / m), j = base + (int)(q % m);
  if (j < i || j >= l) return;
  double* R = Rall + sg * rseg;
  double acc = 0.0;
#pragma unroll 8
  for (int t = 0; t < kCholB; ++t) acc += R[(int64_t)(o + t) * l + i] * R[(int64_t)(o + t) * l + j];
  R[(int64_t)i * l + j] -= acc;
}

// Ri = R^-1 column by column, one warp per column. With the factor staged in shared memory
// (l <= kTriSmemL): for p from c down to 0, x[p] = (delta_pc - acc[p]) / R[p][p], then
// acc[r] += R[r][p] x[p] for all r < p at once (lanes split r), so the chain of c steps has no
// reduction in it. Larger l reads R from global memory by rows: x[r] = -(1/R[r][r])
// sum_{r < p <= c} R[r][p] x[p] with the lanes splitting the sum. A zero pivot gives a zero
// row of R and a zero column of Ri. ri32 (optional) gets an FP32 copy.
constexpr int kTriSmemL = 160;
constexpr int kTriWarps = 8;

__global__ void __launch_bounds__(32 * kTriWarps) k_tri_inv_smem(
    const int* __restrict__ segl, int lfix, const double* __restrict__ Rall, int64_t rseg,
    double* __restrict__ Riall, float* __restrict__ ri32all, int64_t ldr32, int64_t r32seg) {
  extern __shared__ double tri_smem[];
  const int sg = blockIdx.y;
  const int l = segl ? segl[sg] : lfix;
  const int c0 = blockIdx.x * kTriWarps;
  if (c0 >= l) return;
  const int cmax = min(l - 1, c0 + kTriWarps - 1);  // last column of this CTA
  const int ls = (cmax + 1) | 1;  // odd row stride: a column read by 32 lanes takes 2 wavefronts
  double* Rs = tri_smem;                             // rows 0..cmax, columns 0..cmax
  double* rinv = Rs + (int64_t)(cmax + 1) * ls;      // [cmax + 1]
  double* accs = rinv + (cmax + 1);                  // per warp: [cmax + 1]
  const double* R = Rall + sg * rseg;
  for (int q = threadIdx.x; q < (cmax + 1) * (cmax + 1); q += blockDim.x) {
    const int r = q / (cmax + 1), p = q - r * (cmax + 1);
    if (p >= r) Rs[r * ls + p] = R[(int64_t)r * l + p];
  }
  for (int r = threadIdx.x; r <= cmax; r += blockDim.x) {
    const double d = R[(int64_t)r * l + r];
    rinv[r] = d > 0.0 ? 1.0 / d : 0.0;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c = c0 + warp;
  if (c > cmax) return;  // whole warps; no block barrier follows
  double* Ri = Riall + sg * rseg;
  float* ri32 = ri32all ? ri32all + sg * r32seg : nullptr;
  double* acc = accs + warp * (cmax + 1);
  for (int r = lane; r <= c; r += 32) acc[r] = 0.0;
  for (int r = c + 1 + lane; r < l; r += 32) {
    Ri[(int64_t)r * l + c] = 0.0;
    if (ri32) ri32[(int64_t)r * ldr32 + c] = 0.f;
  }
  __syncwarp();
  for (int p = c; p >= 0; --p) {
    const double xp = ((p == c ? 1.0 : 0.0) - acc[p]) * rinv[p];
    if (lane == 0) {
      Ri[(int64_t)p * l + c] = xp;
      if (ri32) ri32[(int64_t)p * ldr32 + c] = (float)xp;
    }
    for (int r = lane; r < p; r += 32) acc[r] = fma(Rs[r * ls + p], xp, acc[r]);
    __syncwarp();
  }
}

__global__ void k_tri_inv_cols(const int* __restrict__ segl, int lfix, const double* __restrict__ Rall,
                               int64_t rseg, double* __restrict__ Riall, float* __restrict__ ri32all,
                               int64_t ldr32, int64_t r32seg) {
  extern __shared__ double xs[];  // per warp: x (l values)
  const int sg = blockIdx.y;
  const int l = segl ? segl[sg] : lfix;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c = blockIdx.x * (blockDim.x >> 5) + warp;
  if (c >= l) return;  // whole warps
  const double* R = Rall + sg * rseg;
  double* Ri = Riall + sg * rseg;
  float* ri32 = ri32all ? ri32all + sg * r32seg : nullptr;
  double* x = xs + (int64_t)warp * l;
  auto inv = [&](int r) {
    const double d = R[(int64_t)r * l + r];
    return d > 0.0 ? 1.0 / d : 0.0;
  };
  for (int r = lane; r < l; r += 32) x[r] = 0.0;
  __syncwarp();
  if (lane == 0) x[c] = inv(c);
  __syncwarp();
  for (int r = c - 1; r >= 0; --r) {
    double acc = 0.0;
    for (int p2 = r + 1 + lane; p2 <= c; p2 += 32) acc += R[(int64_t)r * l + p2] * x[p2];
#pragma unroll
    for (int o2 = 16; o2 > 0; o2 >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o2);
    if (lane == 0) x[r] = -inv(r) * acc;
    __syncwarp();
  }
  for (int r = lane; r < l; r += 32) {
    Ri[(int64_t)r * l + c] = x[r];
    if (ri32) ri32[(int64_t)r * ldr32 + c] = (float)x[r];
  }
}

// Cholesky G_s = R^T R (R upper, positive diagonal) and R^-1 in FP64 per segment. A non-positive
// (or relatively negligible) pivot zeroes that row of R and that column of R^-1 (the column of
// Q it would produce is dropped) and is counted in *breakdowns. Slabs: G_s at G + s*gseg (row
// stride ldg); R_s, Ri_s at R + s*rseg with the segment's own l as row stride; ri32_s
// (optional) at ri32 + s*r32seg (row stride ldr32).
static int chol_inv(int nseg, const int* segl, int lmax, const double* G, int64_t ldg, int64_t gseg,
                    double* R, double* Ri, int64_t rseg, float* ri32, int64_t ldr32, int64_t r32seg,
                    int* breakdowns, cudaStream_t s) {
  Scratch scr(s);
  double *tol, *D;
  ABG_TRY(scr.get(&tol, (size_t)nseg));
  ABG_TRY(scr.get(&D, (size_t)nseg * kCholB * kCholB));
  const int64_t l2 = (int64_t)lmax * lmax;
  k_chol_init<<<dim3((unsigned)std::min<int64_t>(ceil_div(l2, 256), 1024), (unsigned)nseg), 256, 0,
                s>>>(segl, lmax, G, ldg, gseg, R, rseg, tol);
  note_launch();
  const int nb = (int)ceil_div(lmax, kCholB);
  for (int k = 0; k < nb; ++k) {
    k_chol_diag<<<(unsigned)nseg, 32 * kCholW, 0, s>>>(segl, lmax, k, R, rseg, tol, D,
                                                     breakdowns);
    note_launch();
    const int m = lmax - (k + 1) * kCholB;  // trailing columns of the largest segment
    if (m <= 0) continue;
    k_chol_panel<<<dim3((unsigned)ceil_div(m, 128), (unsigned)nseg), 128, 0, s>>>(segl, lmax, k, R,
                                                                                 rseg, D);
    note_launch();
    k_chol_update<<<dim3((unsigned)ceil_div((int64_t)m * m, 256), (unsigned)nseg), 256, 0, s>>>(
        segl, lmax, k, m, R, rseg);
    note_launch();
  }
  if (lmax <= kTriSmemL) {
    // the last CTA stages the most: rows and columns 0..lmax-1 (stride lmax + 1), plus 1/R[p][p]
    // and one accumulator row per warp
    const size_t smem =
        sizeof(double) * ((size_t)lmax * (lmax + 1) + (size_t)lmax * (1 + kTriWarps));
    ABG_TRY(raise_smem_limit((const void*)k_tri_inv_smem, smem));
    k_tri_inv_smem<<<dim3((unsigned)ceil_div(lmax, kTriWarps), (unsigned)nseg), 32 * kTriWarps,
                     smem, s>>>(segl, lmax, R, rseg, Ri, ri32, ldr32, r32seg);
  } else {
    const int wpb = 4;  // columns (warps) per CTA
    const size_t smem = sizeof(double) * wpb * (size_t)lmax;
    ABG_TRY(raise_smem_limit((const void*)k_tri_inv_cols, smem));
    k_tri_inv_cols<<<dim3((unsigned)ceil_div(lmax, wpb), (unsigned)nseg), 32 * wpb, smem, s>>>(
        segl, lmax, R, rseg, Ri, ri32, ldr32, r32seg);
  }
  note_launch();
  ABG_LAUNCH_CHECK();
  return ABG_OK;
}

// ---------------------------------------------------------------------------
// Small FP64 products per segment
// ---------------------------------------------------------------------------
// C_s[i][j] = sum_{r < rows} A_s[r][i] B_s[r][j] for i < ca_s, j < cb_s
__global__ void k_small_tn64(int rows, const int* __restrict__ sca, int ca, const int* __restrict__ scb,
                             int cb, const double* __restrict__ A, int64_t lda, int64_t aseg,
                             const double* __restrict__ B, int64_t ldb, int64_t bseg,
                             double* __restrict__ C, int64_t ldc, int64_t cseg) {
  const int sg = blockIdx.y;
  const int cas = sca ? sca[sg] : ca, cbs = scb ? scb[sg] : cb;
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (int64_t)ca * cb) return;
  const int i = (int)(q / cb), j = (int)(q % cb);
  if (i >= cas || j >= cbs) return;
  const double* As = A + sg * aseg;
  const double* Bs = B + sg * bseg;
  double acc = 0.0;
  for (int r = 0; r < rows; ++r) acc += As[(int64_t)r * lda + i] * Bs[(int64_t)r * ldb + j];
  C[sg * cseg + (int64_t)i * ldc + j] = acc;
}

// C_s[i][j] = sum_{p < inner_s} A_s[i][p] B_s[p][j] for i < ra, j < cb_s
__global__ void k_small_nn64(int ra, const int* __restrict__ sinner, int inner,
                             const int* __restrict__ scb, int cb, const double* __restrict__ A,
                             int64_t lda, int64_t aseg, const double* __restrict__ B, int64_t ldb,
                             int64_t bseg, double* __restrict__ C, int64_t ldc, int64_t cseg) {
  const int sg = blockIdx.y;
  const int ins = sinner ? sinner[sg] : inner, cbs = scb ? scb[sg] : cb;
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (int64_t)ra * cb) return;
  const int i = (int)(q / cb), j = (int)(q % cb);
  if (j >= cbs) return;
  const double* As = A + sg * aseg;
  const double* Bs = B + sg * bseg;
  double acc = 0.0;
  for (int p = 0; p < ins; ++p) acc += As[(int64_t)i * lda + p] * Bs[(int64_t)p * ldb + j];
  C[sg * cseg + (int64_t)i * ldc + j] = acc;
}

__global__ void k_f64_to_f32(int64_t rows, int cols, const double* __restrict__ a, int64_t lda,
                             float* __restrict__ o, int64_t ldo, int transpose) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= rows * cols) return;
  const int64_t i = q / cols;
  const int j = (int)(q % cols);
  if (transpose)
    o[(int64_t)j * ldo + i] = (float)a[i * lda + j];
  else
    o[i * ldo + j] = (float)a[i * lda + j];
}

__global__ void k_f32_to_f64(int64_t rows, int cols, const float* __restrict__ a, int64_t lda,
                             double* __restrict__ o, int64_t ldo) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= rows * cols) return;
  const int64_t i = q / cols;
  const int j = (int)(q % cols);
  o[i * ldo + j] = (double)a[i * lda + j];
}

// Qt_s = Q_s^T (FP32) for nseg d x d FP64 blocks
__global__ void k_transpose_blocks(int nseg, int d, const double* __restrict__ q,
                                   float* __restrict__ qt, int64_t ldo) {
  const int64_t total = (int64_t)nseg * d * d;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t sg = e / ((int64_t)d * d);
    const int rem = (int)(e % ((int64_t)d * d));
    const int i = rem / d, j = rem % d;
    qt[sg * d * ldo + (int64_t)j * ldo + i] = (float)q[e];
  }
}

int transpose_f64_to_f32(const double* a, int rows, int cols, int64_t lda, float* out, int64_t ldo,
                         cudaStream_t s) {
  k_f64_to_f32<<<(unsigned)ceil_div((int64_t)rows * cols, 256), 256, 0, s>>>(rows, cols, a, lda,
                                                                            out, ldo, 1);
  note_launch();
  ABG_LAUNCH_CHECK();
  return ABG_OK;
}

int convert_f64_to_f32(const double* a, int64_t rows, int cols, int64_t lda, float* out,
                       int64_t ldo, cudaStream_t s) {
  if (rows * cols == 0) return ABG_OK;
  k_f64_to_f32<<<(unsigned)ceil_div(rows * cols, 256), 256, 0, s>>>(rows, cols, a, lda, out, ldo,
                                                                   0);
  note_launch();
  ABG_LAUNCH_CHECK();
  return ABG_OK;
}

int transpose_blocks(int nseg, int d, const double* q, float* qt, int64_t ldo, cudaStream_t s) {
  const int64_t total = (int64_t)nseg * d * d;
  k_transpose_blocks<<<(unsigned)std::min<int64_t>(ceil_div(total, 256), 65535), 256, 0, s>>>(
      nseg, d, q, qt, ldo);
  note_launch();
  ABG_LAUNCH_CHECK();
  return ABG_OK;
}

// ---------------------------------------------------------------------------
// Q_s of Algorithm 1: CholeskyQR2 of G_s in FP64 (unique Q with diag(R) > 0)
// ---------------------------------------------------------------------------
int orthogonal_matrices(int nseg, const uint64_t* seeds, int d, double* q, cudaStream_t s) {
  ABG_CHECK(d >= 1 && d <= kMaxD, "orthogonal_matrix: need 1 <= d <= %d", kMaxD);
  Scratch scr(s);
  const int64_t dd = (int64_t)d * d;
  double *G, *Gram, *R, *Ri, *T;
  ABG_TRY(scr.get(&G, (size_t)nseg * dd));
  ABG_TRY(scr.get(&Gram, (size_t)nseg * dd));
  ABG_TRY(scr.get(&R, (size_t)nseg * dd));
  ABG_TRY(scr.get(&Ri, (size_t)nseg * dd));
  ABG_TRY(scr.get(&T, (size_t)nseg * dd));
  int* bd;
  ABG_TRY(scr.get(&bd, 1));
  ABG_CUDA(cudaMemsetAsync(bd, 0, sizeof(int), s));
  ABG_TRY(gaussian_f64(nseg, seeds, ABG_STREAM_G, d, d, G, d, dd, s));
  double* src = G;
  dim3 grid((unsigned)ceil_div(dd, 128), (unsigned)nseg);
  for (int pass = 0; pass < 2; ++pass) {
    k_small_tn64<<<grid, 128, 0, s>>>(d, nullptr, d, nullptr, d, src, d, dd, src, d, dd, Gram, d, dd);
    note_launch();
    ABG_TRY(chol_inv(nseg, nullptr, d, Gram, d, dd, R, Ri, dd, nullptr, 0, 0, bd, s));
    double* dst = pass == 1 ? q : T;
    k_small_nn64<<<grid, 128, 0, s>>>(d, nullptr, d, nullptr, d, src, d, dd, Ri, d, dd, dst, d, dd);
    note_launch();
    src = dst;
  }
  ABG_LAUNCH_CHECK();
  return ABG_OK;
}

// ---------------------------------------------------------------------------
// CholeskyQR2 of tall FP32 blocks per segment: two passes of Gram (FP64, via
// gemm_tn) -> Cholesky -> Y R^-1 (FP32 GEMM).
// ---------------------------------------------------------------------------
// One CholeskyQR pass per segment: dst = src R^-1 with R^T R = src^T src (FP64 Gram and
// Cholesky, FP32 product).
static int cholqr_pass(const RowSpace& rs, const int* segl, int lmax, const float* src,
                       int64_t lds, float* dst, int64_t ldd, int* breakdowns, cudaStream_t s) {
  Scratch scr(s);
  const int64_t ll = round_up(lmax, 4);
  const int64_t l2 = (int64_t)lmax * lmax;
  const int nseg = rs.nseg;
  double *Gram, *R, *Ri;
  float* ri32;
  ABG_TRY(scr.get(&Gram, (size_t)nseg * l2));
  ABG_TRY(scr.get(&R, (size_t)nseg * l2));
  ABG_TRY(scr.get(&Ri, (size_t)nseg * l2));
  ABG_TRY(scr.get(&ri32, (size_t)nseg * lmax * ll));
  TN g;
  g.A = g.B = src;
  g.lda = g.ldb = lds;
  g.K = g.N = lmax;
  g.segK = g.segN = segl;
  g.C = Gram;
  g.ldc = lmax;
  g.c_seg = l2;
  ABG_TRY(gemm_tn(rs, g, s));
  // R_s / Ri_s use the segment's own l_s as row stride inside their l2 slabs
  ABG_TRY(chol_inv(nseg, segl, lmax, Gram, lmax, l2, R, Ri, l2, ri32, ll, lmax * ll, breakdowns, s));
  NN a;
  a.A = src;
  a.lda = lds;
  a.B = ri32;
  a.ldb = ll;
  a.b_seg = lmax * ll;
  a.C = dst;
  a.ldc = ldd;
  a.N = a.K = lmax;
  a.segN = a.segK = segl;
  return gemm_nn(rs, a, s);
}

int cholqr2(const RowSpace& rs, const int* segl, int lmax, float* Y, int64_t ldy, float* tmp,
            int64_t ldt, int* breakdowns, cudaStream_t s) {
  ABG_TRY(cholqr_pass(rs, segl, lmax, Y, ldy, tmp, ldt, breakdowns, s));
  return cholqr_pass(rs, segl, lmax, tmp, ldt, Y, ldy, breakdowns, s);
}

// ---------------------------------------------------------------------------
// One-sided (Hestenes) Jacobi SVD in FP32, one CTA per segment: the columns of
// W_s = Bt_s (m x l_s, FP64 input, row stride lmax inside an m*lmax slab) are
// rotated in round-robin order (the l/2 rotations of a step touch disjoint
// column pairs, a group of lanes per pair) until every pair is orthogonal to
// max(1e-6, 4 sqrt(m) u) of its norms (u = 2^-24); then sigma_j = |w_j| and V holds the accumulated rotations, the
// right singular vectors of Bt_s = the eigenvectors of Bt_s^T Bt_s. FP32 keeps
// the error of sigma_j near 1e-7 sigma_1, the accuracy of the FP32 products
// that formed Bt_s, at a fraction of the cost of FP64 on this GPU.
// evals_s (sigma^2, descending) and evecs_s (columns, row stride lmax) are written.
// Warm start (warm != null, shared-memory case): with warm_in set, the sweeps start from
// W = Bt_s V0 and V = V0 for the orthogonal V0 stored there (the rotations of an earlier,
// nearby matrix, so few sweeps remain); on exit the accumulated V is stored back.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_svd_onesided(int m, const int* __restrict__ segl,
                                                       int lmax, const double* __restrict__ Btall,
                                                       float* __restrict__ Wg_all,
                                                       float* __restrict__ Vg_all, int in_smem,
                                                       int max_sweeps, double* __restrict__ evals,
                                                       double* __restrict__ evecs,
                                                       float* __restrict__ warm, int warm_in,
                                                       const int* __restrict__ skip,
                                                       int square) {
  extern __shared__ float sv_smem[];
  __shared__ int s_rot;
  __shared__ unsigned s_maxr;  // largest |cos| between a pair's columns this sweep (float bits)
  const int sg = blockIdx.x;
  if (skip && skip[sg]) return;  // this segment's factor was found another way
  const int l = segl[sg];
  const double* Bt = Btall + (int64_t)sg * m * lmax;
  // column-major: column j of W at W + j*m, of V at V + j*l
  float* W = in_smem ? sv_smem : Wg_all + (int64_t)sg * m * lmax;
  float* V = in_smem ? sv_smem + (int64_t)m * l : Vg_all + (int64_t)sg * lmax * lmax;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int warp = tid >> 5, lane = tid & 31, nw = nt >> 5;
  float* V0 = warm ? warm + (int64_t)sg * lmax * lmax : nullptr;
  if (V0 && warm_in) {
    // the stored columns, renormalised (FP32 rotations let their norms drift over many calls)
    for (int j = warp; j < l; j += nw) {
      const float* vj = V0 + (int64_t)j * l;
      float acc = 0.f;
      for (int r = lane; r < l; r += 32) acc = fmaf(vj[r], vj[r], acc);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      const float inv = acc > 0.f ? rsqrtf(acc) : 0.f;
      for (int r = lane; r < l; r += 32) V[(int64_t)j * l + r] = vj[r] * inv;
    }
    __syncthreads();
    for (int64_t q = tid; q < (int64_t)m * l; q += nt) {  // W = Bt V0
      const int j = (int)(q / m), r = (int)(q % m);
      const double* br = Bt + (int64_t)r * lmax;
      const float* vj = V + (int64_t)j * l;
      float acc = 0.f;
      for (int p = 0; p < l; ++p) acc = fmaf((float)br[p], vj[p], acc);
      W[q] = acc;
    }
  } else {
    for (int64_t q = tid; q < (int64_t)m * l; q += nt) {
      const int j = (int)(q / m), r = (int)(q % m);
      W[q] = (float)Bt[(int64_t)r * lmax + j];
    }
    for (int64_t q = tid; q < (int64_t)l * l; q += nt) V[q] = (q / l) == (q % l) ? 1.f : 0.f;
  }
  __syncthreads();
  const int mp = (l + 1) & ~1;  // even player count; index l is a bye when l is odd
  const int P = mp / 2;
  // a pair counts as orthogonal below 4 sqrt(m) FP32 ulps of its norms (the rounding level of
  // an m-term FP32 dot product; a fixed 1e-6 sits at that level for m ~ 100 and can keep the
  // sweeps going to max_sweeps), and never above 1e-6 is required
  // (square: the segment's matrix is l x l inside an m x m slab whose other entries are 0,
  // so its columns are l long; the threshold then depends on the segment alone, and a
  // segment gives the same result alone and in a batch)
  const float tol = fmaxf(1e-6f, 4.f * sqrtf((float)(square ? l : m)) * 5.9604645e-8f);
  // G lanes per column pair, so that one pass of the CTA's groups covers a step's P pairs
  // where it can (G >= 8 keeps the column loops a few elements deep per lane)
  const int G = P <= nw ? 32 : (P <= 2 * nw ? 16 : 8);
  const int gpw = 32 / G, gi = lane / G, gl = lane % G;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    if (tid == 0) {
      s_rot = 0;
      s_maxr = 0u;
    }
    __syncthreads();
    int rotated = 0;
    float maxr = 0.f;
    for (int step = 0; step < mp - 1; ++step) {
      // i0 is uniform over the warp, so every lane runs the same trips and the shuffles below
      // see all 32 lanes; groups without a pair carry zeros and rotate nothing
      for (int i0 = warp * gpw; i0 < P; i0 += nw * gpw) {
        const int i = i0 + gi;
        auto player = [&](int pos) {  // round-robin seat pos at this step (seat 0 stays)
          if (pos == 0) return 0;
          int x = pos - 1 + step;       // < 2 (mp - 1)
          if (x >= mp - 1) x -= mp - 1;
          return x + 1;
        };
        int pc = 0, qc = l;
        if (i < P) {
          const int a = player(i), b = player(mp - 1 - i);
          pc = min(a, b);
          qc = max(a, b);
        }
        const bool valid = qc < l;
        float* wp = W + (int64_t)pc * m;
        float* wq = W + (int64_t)(valid ? qc : pc) * m;
        float al = 0.f, be = 0.f, ga = 0.f;
        if (valid)
          for (int r = gl; r < m; r += G) {
            const float x = wp[r], y = wq[r];
            al = fmaf(x, x, al);
            be = fmaf(y, y, be);
            ga = fmaf(x, y, ga);
          }
        for (int o = G / 2; o > 0; o >>= 1) {
          al += __shfl_xor_sync(0xffffffffu, al, o, G);
          be += __shfl_xor_sync(0xffffffffu, be, o, G);
          ga += __shfl_xor_sync(0xffffffffu, ga, o, G);
        }
        if (!valid || !(fabsf(ga) > tol * sqrtf(al * be))) continue;  // uniform over the group
        maxr = fmaxf(maxr, fabsf(ga) * rsqrtf(al * be));
        // the angle only needs to be close: c and s below stay a rotation to rounding
        const float zeta = __fdividef(be - al, 2.f * ga);
        const float t = __fdividef(zeta >= 0.f ? 1.f : -1.f,
                                   fabsf(zeta) + sqrtf(fmaf(zeta, zeta, 1.f)));
        const float c = rsqrtf(fmaf(t, t, 1.f));
        const float sn = c * t;
        for (int r = gl; r < m; r += G) {
          const float x = wp[r], y = wq[r];
          wp[r] = c * x - sn * y;
          wq[r] = sn * x + c * y;
        }
        float* vp = V + (int64_t)pc * l;
        float* vq = V + (int64_t)qc * l;
        for (int r = gl; r < l; r += G) {
          const float x = vp[r], y = vq[r];
          vp[r] = c * x - sn * y;
          vq[r] = sn * x + c * y;
        }
        rotated = 1;
      }
      __syncthreads();
    }
    rotated = __any_sync(0xffffffffu, rotated);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) maxr = fmaxf(maxr, __shfl_xor_sync(0xffffffffu, maxr, o));
    if (lane == 0) {
      if (rotated) atomicOr(&s_rot, 1);
      atomicMax(&s_maxr, __float_as_uint(maxr));  // non-negative floats order as integers
    }
    __syncthreads();
    // done when no pair rotated, or when the largest rotated pair was below sqrt(tol)/4:
    // the sweeps converge quadratically, so the next one would find every pair below tol
    const bool done = s_rot == 0 || __uint_as_float(s_maxr) < 0.25f * sqrtf(tol);
    __syncthreads();  // every thread has read the flags before thread 0 resets them
    if (done) break;
  }
  // sigma_j^2 = |w_j|^2 (one warp per column), then rank descending (ties by index)
  __syncthreads();
  __shared__ float s_norm[kMaxRsvdBlock];
  for (int j = warp; j < l; j += nw) {
    const float* wj = W + (int64_t)j * m;
    float acc = 0.f;
    for (int r = lane; r < m; r += 32) acc = fmaf(wj[r], wj[r], acc);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) s_norm[j] = acc;
  }
  __syncthreads();
  double* ev = evals + (int64_t)sg * lmax;
  double* ec = evecs + (int64_t)sg * lmax * lmax;
  for (int i = tid; i < l; i += nt) {
    const float li = s_norm[i];
    int rank = 0;
    for (int j = 0; j < l; ++j) {
      const float lj = s_norm[j];
      rank += (lj > li) || (lj == li && j < i);
    }
    ev[rank] = (double)li;
    for (int k = 0; k < l; ++k) ec[(int64_t)k * lmax + rank] = (double)V[(int64_t)i * l + k];
  }
  if (V0)
    for (int64_t q = tid; q < (int64_t)l * l; q += nt) V0[q] = V[q];
}

// Rt_s (lmax x lmax, row stride lmax) = R_s (l_s x l_s, row stride l_s), zeros elsewhere
__global__ void k_pad_square(const int* __restrict__ segl, int lmax, const double* __restrict__ R,
                             double* __restrict__ Rt) {
  const int sg = blockIdx.y;
  const int l = segl[sg];
  const int64_t o = (int64_t)sg * lmax * lmax;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < (int64_t)lmax * lmax;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(q / lmax), j = (int)(q % lmax);
    Rt[o + q] = (i < l && j < l) ? R[o + (int64_t)i * l + j] : 0.0;
  }
}

int svd_right(int nseg, int m, const int* segl, int lmax, const double* Bt, double* evals,
              double* evecs, cudaStream_t s, float* warm, bool warm_valid, const int* skip,
              bool square) {
  ABG_CHECK(lmax <= kMaxRsvdBlock, "svd: block width above %d", kMaxRsvdBlock);
  Scratch scr(s);
  const size_t smem = sizeof(float) * ((size_t)m * lmax + (size_t)lmax * lmax);
  const int in_smem = smem <= 200 * 1024;
  const size_t smem_sq = sizeof(float) * 2 * (size_t)lmax * lmax;
  if (!in_smem && m > lmax && smem_sq <= 200 * 1024 && segl) {
    // Tall B^T (m x l) = Q R with R the Cholesky factor of the FP64 Gram B^T^T B^T: R has the
    // same right singular vectors and singular values, and its l x l Jacobi runs in shared
    // memory instead of sweeping m-long columns in global memory
    const int64_t l2 = (int64_t)lmax * lmax;
    double *gram, *R, *Ri, *Rt;
    int* bd;
    ABG_TRY(scr.get(&gram, (size_t)nseg * l2));
    ABG_TRY(scr.get(&R, (size_t)nseg * l2));
    ABG_TRY(scr.get(&Ri, (size_t)nseg * l2));
    ABG_TRY(scr.get(&Rt, (size_t)nseg * l2));
    ABG_TRY(scr.get(&bd, 1));
    ABG_CUDA(cudaMemsetAsync(bd, 0, sizeof(int), s));
    dim3 grid((unsigned)ceil_div(l2, 128), (unsigned)nseg);
    k_small_tn64<<<grid, 128, 0, s>>>(m, segl, lmax, segl, lmax, Bt, lmax, (int64_t)m * lmax, Bt,
                                      lmax, (int64_t)m * lmax, gram, lmax, l2);
    note_launch();
    ABG_TRY(chol_inv(nseg, segl, lmax, gram, lmax, l2, R, Ri, l2, nullptr, 0, 0, bd, s));
    dim3 g2((unsigned)std::min<int64_t>(ceil_div(l2, 256), 1024), (unsigned)nseg);
    k_pad_square<<<g2, 256, 0, s>>>(segl, lmax, R, Rt);
    note_launch();
    ABG_LAUNCH_CHECK();
    return svd_right(nseg, lmax, segl, lmax, Rt, evals, evecs, s, warm, warm_valid, skip,
                     false);
  }
  float *W = nullptr, *V = nullptr;
  if (!in_smem) {
    ABG_TRY(scr.get(&W, (size_t)nseg * m * lmax));
    ABG_TRY(scr.get(&V, (size_t)nseg * lmax * lmax));
  } else {
    ABG_TRY(raise_smem_limit((const void*)k_svd_onesided, smem));
  }
  if (!in_smem) warm = nullptr;  // the warm start keeps V in shared memory
  k_svd_onesided<<<(unsigned)nseg, 1024, in_smem ? smem : 0, s>>>(
      m, segl, lmax, Bt, W, V, in_smem, 40, evals, evecs, warm, warm && warm_valid ? 1 : 0, skip,
      square ? 1 : 0);
  note_launch();
  ABG_LAUNCH_CHECK();
  return ABG_OK;
}

// ---------------------------------------------------------------------------
// Truncated randomized SVD per segment
// ---------------------------------------------------------------------------
// Bm_s[p][j] = U_s[p][j] (x sigma_j in mode 1), Uks_s (FP64), sigma_s; the sign of each
// column is fixed later from the left factor (k_colmax_part, k_colsign).
__global__ void k_rsvd_post(const int* __restrict__ segl, const int* __restrict__ segk, int kfix,
                            int lmax, int kmax, const double* __restrict__ evals,
                            const double* __restrict__ U, int with_sigma, float* __restrict__ Bm,
                            int64_t ldb, double* __restrict__ Uks, double* __restrict__ sigma_out,
                            int64_t sseg) {
  const int sg = blockIdx.y;
  const int l = segl[sg];
  const int k = segk ? segk[sg] : kfix;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= k) return;
  const double* Us = U + (int64_t)sg * lmax * lmax;
  const double sigma = sqrt(fmax(evals[(int64_t)sg * lmax + j], 0.0));
  float* Bs = Bm + (int64_t)sg * lmax * ldb;
  double* Uk = Uks + (int64_t)sg * lmax * kmax;
  for (int p = 0; p < l; ++p) {
    const double u = Us[(int64_t)p * lmax + j];
    Uk[(int64_t)p * kmax + j] = u;
    Bs[(int64_t)p * ldb + j] = (float)(with_sigma ? u * sigma : u);
  }
  if (sigma_out) sigma_out[sg * sseg + j] = sigma;
}

// Sign of each left singular vector (reading R7): its entry of largest magnitude is made
// positive (the first such row on ties). Pass 1: per 2048-row chunk and column j < k_s, the
// signed value of the column's largest-magnitude entry over the chunk's rows, in row order.
__global__ void k_colmax_part(const int* __restrict__ chunk_seg, const int64_t* __restrict__ chunk_row0,
                              const int* __restrict__ chunk_rows, const int* __restrict__ segk,
                              int kfix, int kmax, const float* __restrict__ G, int64_t ldg,
                              float* __restrict__ part) {
  const int64_t c = blockIdx.x;
  const int sg = chunk_seg[c];
  const int k = segk ? segk[sg] : kfix;
  const int64_t r0 = chunk_row0[c], r1 = r0 + chunk_rows[c];
  for (int j = threadIdx.x; j < kmax; j += blockDim.x) {
    float best = 0.f, best_abs = -1.f;
    if (j < k) {
      constexpr int U = 8;  // loads in flight together; the comparisons stay in row order
      int64_t r = r0;
      for (; r + U <= r1; r += U) {
        float v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) v[u] = G[(r + u) * ldg + j];
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (fabsf(v[u]) > best_abs) {
            best_abs = fabsf(v[u]);
            best = v[u];
          }
      }
      for (; r < r1; ++r) {
        const float v = G[r * ldg + j];
        if (fabsf(v) > best_abs) {
          best_abs = fabsf(v);
          best = v;
        }
      }
    }
    part[c * kmax + j] = best;
  }
}

// Pass 2: per segment and column, the chunk winners in chunk order (the first largest
// magnitude over the whole column), giving sign_j = -1 when that entry is negative, else +1.
__global__ void k_colsign(const int* __restrict__ segk, int kfix, int kmax,
                          const int64_t* __restrict__ seg_group0,
                          const int64_t* __restrict__ group_chunk0,
                          const int* __restrict__ group_nchunks, const float* __restrict__ part,
                          float* __restrict__ sign) {
  const int sg = blockIdx.x;
  const int k = segk ? segk[sg] : kfix;
  const int64_t g0 = seg_group0[sg], g1 = seg_group0[sg + 1];
  const int64_t c0 = g1 > g0 ? group_chunk0[g0] : 0;
  const int64_t c1 = g1 > g0 ? group_chunk0[g1 - 1] + group_nchunks[g1 - 1] : 0;
  for (int j = threadIdx.x; j < kmax; j += blockDim.x) {
    float best = 0.f, best_abs = -1.f;
    if (j < k)
      for (int64_t c = c0; c < c1; ++c) {
        const float v = part[c * kmax + j];
        if (fabsf(v) > best_abs) {
          best_abs = fabsf(v);
          best = v;
        }
      }
    sign[(int64_t)sg * kmax + j] = best < 0.f ? -1.f : 1.f;
  }
}

// G[i][j] <- sign_s[j] G[i][j] (then max(., 0) with relu) for j < k_s of the row's segment;
// one warp per row, the lanes over its columns
__global__ void k_apply_sign(int64_t rows, const int* __restrict__ row_seg,
                             const int* __restrict__ segk, int kfix, int kmax,
                             const float* __restrict__ sign, int relu, float* __restrict__ G,
                             int64_t ldg) {
  const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= rows) return;
  const int sg = row_seg[i];
  const int k = segk ? segk[sg] : kfix;
  const float* sgn = sign + (int64_t)sg * kmax;
  float* g = G + i * ldg;
  for (int j = lane; j < k; j += 32) {
    float v = g[j] * sgn[j];
    if (relu) v = fmaxf(v, 0.f);
    g[j] = v;
  }
}

// Uks_s[p][j] *= sign_s[j]: the right factor follows the left one's sign
__global__ void k_sign_cols(const int* __restrict__ segl, const int* __restrict__ segk, int kfix,
                            int lmax, int kmax, const float* __restrict__ sign,
                            double* __restrict__ Uks) {
  const int sg = blockIdx.y;
  const int k = segk ? segk[sg] : kfix;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= segl[sg] * kmax) return;
  const int j = q % kmax;
  if (j >= k) return;
  Uks[(int64_t)sg * lmax * kmax + q] *= (double)sign[(int64_t)sg * kmax + j];
}

__global__ void k_relu_f64_to_f32(int rows, const int* __restrict__ segk, int kmax,
                                  const double* __restrict__ a, int64_t lda, int64_t aseg,
                                  float* __restrict__ o, int64_t ldo, int64_t oseg) {
  const int sg = blockIdx.y;
  const int k = segk[sg];
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (int64_t)rows * kmax) return;
  const int i = (int)(q / kmax), j = (int)(q % kmax);
  if (j >= k) return;
  o[sg * oseg + (int64_t)i * ldo + j] = (float)fmax(a[sg * aseg + (int64_t)i * lda + j], 0.0);
}

// Y (rows of each segment, l_s columns) = A_s * Om_s
static int apply_a(const RsvdIn& in, const int* segl, int lmax, const float* Om, int64_t ldo,
                   float* Y, int64_t ldy, cudaStream_t s) {
  if (in.A) {
    NN a;
    a.A = in.A;
    a.lda = in.lda;
    a.A16 = in.A16;
    a.lda16 = in.lda16;
    a.B = Om;
    a.ldb = ldo;
    a.b_seg = (int64_t)in.m * ldo;
    a.C = Y;
    a.ldc = ldy;
    a.N = lmax;
    a.K = in.m;
    a.segN = segl;
    return gemm_nn(*in.rows, a, s);
  }
  // sparse rows gather rows of the stacked test blocks (column s*m + j)
  return spmm_plain(in.ptr, in.col, in.val, in.rows->rows, Om, ldo, lmax, Y, ldy, s);
}

// Bt_s (m x l_s, FP64, row stride lmax, slab m*lmax) = A_s^T Q_s
static int apply_at(const RsvdIn& in, const int* segl, int lmax, const float* Q, int64_t ldq,
                    double* Bt, float* tmp32, int64_t ldt, cudaStream_t s) {
  const int nseg = in.rows->nseg;
  if (in.A) {
    TN t;
    t.A = in.A;
    t.lda = in.lda;
    t.A16 = in.A16;
    t.lda16 = in.lda16;
    t.B = Q;
    t.ldb = ldq;
    t.K = in.m;
    t.N = lmax;
    t.segN = segl;
    t.C = Bt;
    t.ldc = lmax;
    t.c_seg = (int64_t)in.m * lmax;
    return gemm_tn(*in.rows, t, s);
  }
  ABG_TRY(spmm_plain(in.tptr, in.tcol, in.tval, (int64_t)nseg * in.m, Q, ldq, lmax, tmp32, ldt, s));
  const int64_t rows = (int64_t)nseg * in.m;
  k_f32_to_f64<<<(unsigned)ceil_div(rows * lmax, 256), 256, 0, s>>>(rows, lmax, tmp32, ldt, Bt, lmax);
  note_launch();
  ABG_LAUNCH_CHECK();
  return ABG_OK;
}

int rsvd(const RsvdIn& in, const SegSizes& ss, int kfixed, int power_iters, int stream_id,
         const RsvdOut& out, int* breakdowns, cudaStream_t s) {
  const RowSpace& rs = *in.rows;
  const int nseg = rs.nseg;
  const int m = in.m;
  const int lmax = ss.l_max;
  const int kmax = out.left_mode == 0 ? ss.k_max : kfixed;
  const int* segk = out.left_mode == 0 ? ss.k : nullptr;
  ABG_CHECK(lmax >= 1 && lmax <= 1024, "rsvd: block width must stay in [1, 1024]");
  Scratch scr(s);
  const int64_t ll = round_up(lmax, 4);
  const int64_t kk = round_up(kmax, 4);
  const int64_t l2 = (int64_t)lmax * lmax;
  float *Om, *Y, *T1, *Yt, *T2, *Bm;
  double *Bt, *evals, *evecs, *Uks, *Hd;
  ABG_TRY(scr.get(&Om, (size_t)nseg * m * ll));
  ABG_TRY(scr.get(&Y, (size_t)rs.rows * ll));
  ABG_TRY(scr.get(&T1, (size_t)rs.rows * ll));
  ABG_TRY(scr.get(&Yt, (size_t)nseg * m * ll));
  ABG_TRY(scr.get(&T2, (size_t)nseg * m * ll));
  ABG_TRY(scr.get(&Bt, (size_t)nseg * m * lmax));
  ABG_TRY(scr.get(&evals, (size_t)nseg * lmax));
  ABG_TRY(scr.get(&evecs, (size_t)nseg * l2));
  ABG_TRY(scr.get(&Uks, (size_t)nseg * lmax * kmax));
  ABG_TRY(scr.get(&Hd, (size_t)nseg * m * kmax));
  ABG_TRY(scr.get(&Bm, (size_t)nseg * lmax * kk));
  RowSpace small;  // m rows per segment (the Omega / A^T Q side)
  ABG_TRY(rowspace_uniform(&small, nseg, m, scr, s));
  // range finder: the intermediate bases only need to stay well conditioned (one
  // CholeskyQR pass each); the final tall basis gets CholeskyQR2
  ABG_TRY(gaussian_f32(nseg, ss.seed, stream_id, m, lmax, ss.l, Om, ll, (int64_t)m * ll, s));
  float* Ya = Y;
  float* Yb = T1;
  ABG_TRY(apply_a(in, ss.l, lmax, Om, ll, Ya, ll, s));
  float* cur = Ya;
  if (power_iters == 0) {
    ABG_TRY(cholqr2(rs, ss.l, lmax, Ya, ll, Yb, ll, breakdowns, s));
  } else {
    ABG_TRY(cholqr_pass(rs, ss.l, lmax, Ya, ll, Yb, ll, breakdowns, s));
    cur = Yb;
  }
  for (int it = 0; it < power_iters; ++it) {
    ABG_TRY(apply_at(in, ss.l, lmax, cur, ll, Bt, T2, ll, s));
    ABG_TRY(convert_f64_to_f32(Bt, (int64_t)nseg * m, lmax, lmax, Yt, ll, s));
    ABG_TRY(cholqr_pass(small, ss.l, lmax, Yt, ll, T2, ll, breakdowns, s));
    float* nxt = cur == Ya ? Yb : Ya;
    ABG_TRY(apply_a(in, ss.l, lmax, T2, ll, nxt, ll, s));
    if (it == power_iters - 1) {
      ABG_TRY(cholqr2(rs, ss.l, lmax, nxt, ll, cur, ll, breakdowns, s));
      cur = nxt;
    } else {
      ABG_TRY(cholqr_pass(rs, ss.l, lmax, nxt, ll, cur, ll, breakdowns, s));
    }
  }
  Y = cur;
  // B^T = A^T Q (m x l); its SVD gives sigma and the left singular vectors of B
  ABG_TRY(apply_at(in, ss.l, lmax, Y, ll, Bt, T2, ll, s));
  ABG_TRY(svd_right(nseg, m, ss.l, lmax, Bt, evals, evecs, s));
  {
    dim3 g((unsigned)ceil_div(kmax, 128), (unsigned)nseg);
    k_rsvd_post<<<g, 128, 0, s>>>(ss.l, segk, kfixed, lmax, kmax, evals, evecs, out.left_mode,
                                  Bm, kk, Uks, out.sigma, out.sseg);
    note_launch();
  }
  ABG_LAUNCH_CHECK();
  // left factor Gamma = Q U_k (x Sigma in mode 1), then each column signed so that its entry
  // of largest magnitude is positive, with max(., 0) for Phi (Eq. 18, reading R8)
  {
    NN a;
    a.A = Y;
    a.lda = ll;
    a.B = Bm;
    a.ldb = kk;
    a.b_seg = lmax * kk;
    a.C = out.left;
    a.ldc = out.ldl;
    a.N = kmax;
    a.K = lmax;
    a.segN = segk;
    a.segK = ss.l;
    a.epi = Epi::Store;
    ABG_TRY(gemm_nn(rs, a, s));
  }
  {
    float *part, *sign;
    ABG_TRY(scr.get(&part, (size_t)std::max<int64_t>(1, rs.n_chunks) * kmax));
    ABG_TRY(scr.get(&sign, (size_t)nseg * kmax));
    if (rs.n_chunks) {
      k_colmax_part<<<(unsigned)rs.n_chunks, 128, 0, s>>>(rs.chunk_seg, rs.chunk_row0,
                                                          rs.chunk_rows, segk, kfixed, kmax,
                                                          out.left, out.ldl, part);
      note_launch();
    }
    k_colsign<<<(unsigned)nseg, 128, 0, s>>>(segk, kfixed, kmax, rs.seg_group0, rs.group_chunk0,
                                             rs.group_nchunks, part, sign);
    note_launch();
    k_apply_sign<<<(unsigned)ceil_div(rs.rows, 8), 256, 0, s>>>(
        rs.rows, rs.row_seg, segk, kfixed, kmax, sign, out.left_mode == 0 ? 1 : 0, out.left,
        out.ldl);
    note_launch();
    dim3 g((unsigned)ceil_div((int64_t)lmax * kmax, 256), (unsigned)nseg);
    k_sign_cols<<<g, 256, 0, s>>>(ss.l, segk, kfixed, lmax, kmax, sign, Uks);
    note_launch();
    ABG_LAUNCH_CHECK();
  }
  if (out.right) {  // H_s = max(B_s^T U_k, 0) = max(Psi Sigma, 0)
    dim3 g((unsigned)ceil_div((int64_t)m * kmax, 128), (unsigned)nseg);
    k_small_nn64<<<g, 128, 0, s>>>(m, ss.l, lmax, segk, kmax, Bt, lmax, (int64_t)m * lmax, Uks,
                                   kmax, (int64_t)lmax * kmax, Hd, kmax, (int64_t)m * kmax);
    note_launch();
    dim3 g2((unsigned)ceil_div((int64_t)m * kmax, 256), (unsigned)nseg);
    k_relu_f64_to_f32<<<g2, 256, 0, s>>>(m, ss.k, kmax, Hd, kmax, (int64_t)m * kmax, out.right,
                                         out.ldr, out.rseg);
    note_launch();
    ABG_LAUNCH_CHECK();
  }
  return ABG_OK;
}

}  // namespace abg
