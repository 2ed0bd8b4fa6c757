// Random matrices and small dense linear algebra of the method:
//   * Gaussian draws from Philox4x32-10 (Salmon et al., SC'11) + Box-Muller
//     on the device (G of Algorithm 1, the randomized-SVD test matrices);
//   * Q = orthogonal factor of QR(G) (Algorithm 1), by CholeskyQR2 in FP64;
//   * CholeskyQR2 of tall FP32 blocks (FP64 Gram / Cholesky, FP32 apply);
//   * the truncated randomized SVD of Halko, Martinsson and Tropp (subspace
//     iteration) used by Algorithm 2's seeding (Eq. 18) and by the attribute
//     reduction of Section 3.2.1 (Eq. 15): the small l x l eigenproblem runs
//     as a one-CTA parallel cyclic Jacobi in FP64.
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

template <class T>
__global__ void k_gaussian(uint64_t seed, uint32_t stream_id, int rows, int cols, T* out,
                           int64_t ld) {
  const int64_t total = (int64_t)rows * cols;
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
      double sn, cs;
      sincospi(2.0 * u[a + 1], &sn, &cs);
      z[a] = rad * cs;
      z[a + 1] = rad * sn;
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t e = 4 * b + j;
      if (e < total) out[(e / cols) * ld + (e % cols)] = (T)z[j];
    }
  }
}

int gaussian_f64(uint64_t seed, int stream_id, int rows, int cols, double* out, int64_t ld,
                 cudaStream_t s) {
  const int64_t nb = ((int64_t)rows * cols + 3) / 4;
  k_gaussian<double><<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(nb, 256), 4096)),
                       256, 0, s>>>(seed, (uint32_t)stream_id, rows, cols, out, ld); ::abg::note_launch();
  ABG_LAUNCH_CHECK();
  return ABG_OK;
}

int gaussian_f32(uint64_t seed, int stream_id, int rows, int cols, float* out, int64_t ld,
                 cudaStream_t s) {
  const int64_t nb = ((int64_t)rows * cols + 3) / 4;
  k_gaussian<float><<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(ceil_div(nb, 256), 4096)),
                      256, 0, s>>>(seed, (uint32_t)stream_id, rows, cols, out, ld); ::abg::note_launch();
  ABG_LAUNCH_CHECK();
  return ABG_OK;
}

// ---------------------------------------------------------------------------
// One-CTA Cholesky G = R^T R (R upper, positive diagonal) and R^-1, FP64.
// A non-positive (or relatively negligible) pivot zeroes that row of R and
// that column of R^-1 (the column of Q it would produce is dropped) and is
// counted in *breakdowns.
// work: l*l doubles (R), rinv64: l*l doubles; rinv32 (optional): l x ldr floats.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_chol_inv(int l, const double* __restrict__ G, int64_t ldg,
                                                   double* __restrict__ Rg, double* __restrict__ Rig,
                                                   float* __restrict__ ri32, int64_t ldr32,
                                                   int* __restrict__ breakdowns, int in_smem) {
  extern __shared__ double csm[];
  double* R = in_smem ? csm : Rg;                    // l x l, upper triangle used
  double* Ri = in_smem ? csm + (int64_t)l * l : Rig; // l x l
  const int tid = threadIdx.x, nt = blockDim.x;
  const int warp = tid / 32, lane = tid % 32, nw = nt / 32;
  __shared__ double s_piv;
  __shared__ double s_maxdiag;
  for (int64_t q = tid; q < (int64_t)l * l; q += nt) {
    const int i = (int)(q / l), j = (int)(q % l);
    R[q] = j >= i ? G[(int64_t)i * ldg + j] : 0.0;
  }
  if (tid == 0) {
    double m = 0.0;
    for (int i = 0; i < l; ++i) m = fmax(m, fabs(G[(int64_t)i * ldg + i]));
    s_maxdiag = m;
  }
  __syncthreads();
  const double tol = 1e-13 * s_maxdiag;
  for (int j = 0; j < l; ++j) {
    if (tid == 0) {
      const double p = R[(int64_t)j * l + j];
      if (!(p > tol)) {
        s_piv = 0.0;
        atomicAdd(breakdowns, 1);
      } else {
        s_piv = sqrt(p);
      }
    }
    __syncthreads();
    const double piv = s_piv;
    // row j of R: R[j][j] = piv, R[j][c] = A[j][c] / piv (all zero after a breakdown)
    for (int c = j + tid; c < l; c += nt) {
      const double v = R[(int64_t)j * l + c];
      R[(int64_t)j * l + c] = piv > 0.0 ? (c == j ? piv : v / piv) : 0.0;
    }
    __syncthreads();
    // trailing update A[r][c] -= R[j][r] R[j][c] for j < r <= c: a warp per row
    for (int r = j + 1 + warp; r < l; r += nw) {
      const double rjr = R[(int64_t)j * l + r];
      for (int c = r + lane; c < l; c += 32) R[(int64_t)r * l + c] -= rjr * R[(int64_t)j * l + c];
    }
    __syncthreads();
  }
  // inverse of the upper-triangular R, one warp per column (back substitution)
  for (int j = warp; j < l; j += nw) {
    for (int i = lane; i < l; i += 32) Ri[(int64_t)i * l + j] = 0.0;
    __syncwarp();
    for (int i = j; i >= 0; --i) {
      const double rii = R[(int64_t)i * l + i];
      double acc = 0.0;
      for (int p = i + 1 + lane; p <= j; p += 32) acc += R[(int64_t)i * l + p] * Ri[(int64_t)p * l + j];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) {
        const double rhs = (i == j ? 1.0 : 0.0) - acc;
        Ri[(int64_t)i * l + j] = rii > 0.0 ? rhs / rii : 0.0;
      }
      __syncwarp();
    }
    // a dropped pivot on the diagonal zeroes this column of R^-1
    if (R[(int64_t)j * l + j] <= 0.0)
      for (int i = lane; i < l; i += 32) Ri[(int64_t)i * l + j] = 0.0;
  }
  __syncthreads();
  for (int64_t q = tid; q < (int64_t)l * l; q += nt) {
    const double v = Ri[q];
    if (in_smem) Rig[q] = v;
    if (ri32) ri32[(q / l) * ldr32 + (q % l)] = (float)v;
  }
}

// Launch k_chol_inv with both triangles in shared memory when they fit.
static int chol_inv(int l, const double* G, int64_t ldg, double* R, double* Ri, float* ri32,
                    int64_t ldr32, int* breakdowns, cudaStream_t s) {
  const size_t smem = sizeof(double) * 2 * (size_t)l * l;
  const int in_smem = smem <= 200 * 1024;
  if (in_smem)
    ABG_CUDA(cudaFuncSetAttribute(k_chol_inv, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem));
  k_chol_inv<<<1, 1024, in_smem ? smem : 0, s>>>(l, G, ldg, R, Ri, ri32, ldr32, breakdowns,
                                                 in_smem);
  ::abg::note_launch();
  ABG_LAUNCH_CHECK();
  return ABG_OK;
}

// ---------------------------------------------------------------------------
// Small FP64 products (d x d and l x l matrices)
// ---------------------------------------------------------------------------
// C[i][j] = sum_r A[r][i] B[r][j]   (A: rows x ca, B: rows x cb)
__global__ void k_small_tn64(int rows, int ca, int cb, const double* __restrict__ A, int64_t lda,
                             const double* __restrict__ B, int64_t ldb, double* __restrict__ C,
                             int64_t ldc) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (int64_t)ca * cb) return;
  const int i = (int)(q / cb), j = (int)(q % cb);
  double s = 0.0;
  for (int r = 0; r < rows; ++r) s += A[(int64_t)r * lda + i] * B[(int64_t)r * ldb + j];
  C[(int64_t)i * ldc + j] = s;
}

// C[i][j] = sum_p A[i][p] B[p][j]   (A: ra x inner, B: inner x cb)
__global__ void k_small_nn64(int ra, int inner, int cb, const double* __restrict__ A, int64_t lda,
                             const double* __restrict__ B, int64_t ldb, double* __restrict__ C,
                             int64_t ldc) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (int64_t)ra * cb) return;
  const int i = (int)(q / cb), j = (int)(q % cb);
  double s = 0.0;
  for (int p = 0; p < inner; ++p) s += A[(int64_t)i * lda + p] * B[(int64_t)p * ldb + j];
  C[(int64_t)i * ldc + j] = s;
}

static void small_tn64(int rows, int ca, int cb, const double* A, int64_t lda, const double* B,
                       int64_t ldb, double* C, int64_t ldc, cudaStream_t s) {
  k_small_tn64<<<(unsigned)ceil_div((int64_t)ca * cb, 128), 128, 0, s>>>(rows, ca, cb, A, lda, B,
                                                                        ldb, C, ldc); ::abg::note_launch();
}
static void small_nn64(int ra, int inner, int cb, const double* A, int64_t lda, const double* B,
                       int64_t ldb, double* C, int64_t ldc, cudaStream_t s) {
  k_small_nn64<<<(unsigned)ceil_div((int64_t)ra * cb, 128), 128, 0, s>>>(ra, inner, cb, A, lda, B,
                                                                        ldb, C, ldc); ::abg::note_launch();
}

__global__ void k_f64_to_f32(int rows, int cols, const double* __restrict__ a, int64_t lda,
                             float* __restrict__ o, int64_t ldo, int transpose) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (int64_t)rows * cols) return;
  const int i = (int)(q / cols), j = (int)(q % cols);
  if (transpose)
    o[(int64_t)j * ldo + i] = (float)a[(int64_t)i * lda + j];
  else
    o[(int64_t)i * ldo + j] = (float)a[(int64_t)i * lda + j];
}

__global__ void k_f32_to_f64(int64_t rows, int cols, const float* __restrict__ a, int64_t lda,
                             double* __restrict__ o, int64_t ldo) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= rows * cols) return;
  const int64_t i = q / cols;
  const int j = (int)(q % cols);
  o[i * ldo + j] = (double)a[i * lda + j];
}

int transpose_f64_to_f32(const double* a, int rows, int cols, int64_t lda, float* out, int64_t ldo,
                         cudaStream_t s) {
  k_f64_to_f32<<<(unsigned)ceil_div((int64_t)rows * cols, 256), 256, 0, s>>>(rows, cols, a, lda,
                                                                            out, ldo, 1); ::abg::note_launch();
  ABG_LAUNCH_CHECK();
  return ABG_OK;
}

int convert_f64_to_f32(const double* a, int rows, int cols, int64_t lda, float* out, int64_t ldo,
                       cudaStream_t s) {
  k_f64_to_f32<<<(unsigned)ceil_div((int64_t)rows * cols, 256), 256, 0, s>>>(rows, cols, a, lda,
                                                                            out, ldo, 0); ::abg::note_launch();
  ABG_LAUNCH_CHECK();
  return ABG_OK;
}

// ---------------------------------------------------------------------------
// Q of Algorithm 1: CholeskyQR2 of G in FP64 (unique Q with diag(R) > 0)
// ---------------------------------------------------------------------------
int orthogonal_matrix(uint64_t seed, int d, double* q, cudaStream_t s) {
  ABG_CHECK(d >= 1 && d <= kMaxD, "orthogonal_matrix: need 1 <= d <= %d", kMaxD);
  Scratch scr(s);
  double *G, *Gram, *R, *Ri, *T;
  ABG_TRY(scr.get(&G, (size_t)d * d));
  ABG_TRY(scr.get(&Gram, (size_t)d * d));
  ABG_TRY(scr.get(&R, (size_t)d * d));
  ABG_TRY(scr.get(&Ri, (size_t)d * d));
  ABG_TRY(scr.get(&T, (size_t)d * d));
  int* bd;
  ABG_TRY(scr.get(&bd, 1));
  ABG_CUDA(cudaMemsetAsync(bd, 0, sizeof(int), s));
  ABG_TRY(gaussian_f64(seed, ABG_STREAM_G, d, d, G, d, s));
  double* src = G;
  double* dst = T;
  for (int pass = 0; pass < 2; ++pass) {
    small_tn64(d, d, d, src, d, src, d, Gram, d, s);
    ABG_TRY(chol_inv(d, Gram, d, R, Ri, nullptr, 0, bd, s));
    small_nn64(d, d, d, src, d, Ri, d, pass == 1 ? q : dst, d, s);
    src = dst;
  }
  ABG_LAUNCH_CHECK();
  return ABG_OK;
}

// ---------------------------------------------------------------------------
// CholeskyQR2 of a tall FP32 block Y (M x l): two passes of Gram (FP64, via
// gemm_tn) -> Cholesky -> Y R^-1 (FP32 GEMM).
// ---------------------------------------------------------------------------
int cholqr2(int64_t M, int l, float* Y, int64_t ldy, float* tmp, int64_t ldt, int* breakdowns,
            Scratch& /*caller*/, cudaStream_t s) {
  Scratch scr(s);
  const int64_t ll = round_up(l, 4);
  double *Gram, *R, *Ri;
  float* ri32;
  ABG_TRY(scr.get(&Gram, (size_t)l * l));
  ABG_TRY(scr.get(&R, (size_t)l * l));
  ABG_TRY(scr.get(&Ri, (size_t)l * l));
  ABG_TRY(scr.get(&ri32, (size_t)l * ll));
  for (int pass = 0; pass < 2; ++pass) {
    float* src = pass == 0 ? Y : tmp;
    const int64_t lds = pass == 0 ? ldy : ldt;
    float* dst = pass == 0 ? tmp : Y;
    const int64_t ldd = pass == 0 ? ldt : ldy;
    ABG_TRY(gemm_tn(M, l, l, src, lds, src, lds, Gram, l, scr, s));
    ABG_TRY(chol_inv(l, Gram, l, R, Ri, ri32, ll, breakdowns, s));
    ABG_TRY(gemm_nn(M, l, l, src, lds, ri32, ll, dst, ldd, Epi::Store, nullptr, 0, nullptr, 0,
                    nullptr, s));
  }
  return ABG_OK;
}

// ---------------------------------------------------------------------------
// Parallel cyclic Jacobi for a symmetric l x l FP64 matrix (one CTA, round-
// robin pairing so the l/2 rotations of a step touch disjoint index pairs).
// A is destroyed; evals (descending) and evecs (columns, l x l) are written.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) k_jacobi(int l, double* __restrict__ Ag, double* __restrict__ Vg,
                                                 double* __restrict__ evals,
                                                 double* __restrict__ evecs, int max_sweeps,
                                                 int a_smem, int v_smem) {
  extern __shared__ double js[];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int m = (l + 1) & ~1;  // even player count (index l is a dummy when l is odd)
  const int P = m / 2;
  double* cs = js;
  double* sn = js + P;
  int* pp = reinterpret_cast<int*>(js + 2 * P);
  int* qq = pp + P;
  double* red = js + 3 * P + 1;             // 2 * nt + 1
  double* tail = red + 2 * nt + 2;
  double* A = a_smem ? tail : Ag;
  double* V = v_smem ? tail + (a_smem ? (int64_t)l * l : 0) : Vg;
  if (a_smem)
    for (int64_t q = tid; q < (int64_t)l * l; q += nt) A[q] = Ag[q];
  for (int64_t q = tid; q < (int64_t)l * l; q += nt) V[q] = ((q / l) == (q % l)) ? 1.0 : 0.0;
  __syncthreads();
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int64_t q = tid; q < (int64_t)l * l; q += nt) {
      const double v = A[q] * A[q];
      tot += v;
      if ((q / l) != (q % l)) off += v;
    }
    red[tid] = off;
    red[nt + tid] = tot;
    __syncthreads();
    if (tid == 0) {
      double o = 0.0, t = 0.0;
      for (int i = 0; i < nt; ++i) {
        o += red[i];
        t += red[nt + i];
      }
      red[2 * nt] = (o <= 1e-30 * t || t == 0.0) ? 1.0 : 0.0;
    }
    __syncthreads();
    if (red[2 * nt] != 0.0) break;
    __syncthreads();
    for (int step = 0; step < m - 1; ++step) {
      for (int i = tid; i < P; i += nt) {
        auto player = [&](int pos) { return pos == 0 ? 0 : ((pos - 1 + step) % (m - 1)) + 1; };
        int a = player(i), b = player(m - 1 - i);
        int p = min(a, b), q = max(a, b);
        double c = 1.0, sv = 0.0;
        if (q < l) {
          const double apq = A[(int64_t)p * l + q];
          if (apq != 0.0) {
            const double app = A[(int64_t)p * l + p], aqq = A[(int64_t)q * l + q];
            const double theta = (aqq - app) / (2.0 * apq);
            const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
            c = 1.0 / sqrt(t * t + 1.0);
            sv = t * c;
          }
        }
        cs[i] = c;
        sn[i] = sv;
        pp[i] = p;
        qq[i] = q;
      }
      __syncthreads();
      // rows: A <- J^T A (a warp per pair, lanes over columns)
      const int warp = tid / 32, lane = tid % 32, nw = nt / 32;
      for (int i = warp; i < P; i += nw) {
        const int p = pp[i], q = qq[i];
        if (q >= l) continue;
        const double c = cs[i], sv = sn[i];
        for (int k = lane; k < l; k += 32) {
          const double apk = A[(int64_t)p * l + k], aqk = A[(int64_t)q * l + k];
          A[(int64_t)p * l + k] = c * apk - sv * aqk;
          A[(int64_t)q * l + k] = sv * apk + c * aqk;
        }
      }
      __syncthreads();
      // columns: A <- A J, V <- V J
      for (int i = warp; i < P; i += nw) {
        const int p = pp[i], q = qq[i];
        if (q >= l) continue;
        const double c = cs[i], sv = sn[i];
        for (int k = lane; k < l; k += 32) {
          const double akp = A[(int64_t)k * l + p], akq = A[(int64_t)k * l + q];
          A[(int64_t)k * l + p] = c * akp - sv * akq;
          A[(int64_t)k * l + q] = sv * akp + c * akq;
          const double vkp = V[(int64_t)k * l + p], vkq = V[(int64_t)k * l + q];
          V[(int64_t)k * l + p] = c * vkp - sv * vkq;
          V[(int64_t)k * l + q] = sv * vkp + c * vkq;
        }
      }
      __syncthreads();
    }
  }
  // sort descending (rank by value, ties by index) and write eigenpairs
  for (int i = tid; i < l; i += nt) {
    const double li = A[(int64_t)i * l + i];
    int rank = 0;
    for (int j = 0; j < l; ++j) {
      const double lj = A[(int64_t)j * l + j];
      rank += (lj > li) || (lj == li && j < i);
    }
    evals[rank] = li;
    for (int k = 0; k < l; ++k) evecs[(int64_t)k * l + rank] = V[(int64_t)k * l + i];
  }
}

static int jacobi_eig(int l, double* A, double* evals, double* evecs, Scratch& /*caller*/, cudaStream_t s) {
  Scratch scr(s);
  double* V;
  ABG_TRY(scr.get(&V, (size_t)l * l));
  const int threads = 1024;
  const int P = ((l + 1) & ~1) / 2;
  const size_t base = sizeof(double) * (3 * P + 1 + 2 * threads + 2);
  const size_t mat = sizeof(double) * (size_t)l * l;
  const size_t limit = 220 * 1024;
  const int a_smem = base + mat <= limit;
  const int v_smem = a_smem && base + 2 * mat <= limit;
  const size_t smem = base + (a_smem ? mat : 0) + (v_smem ? mat : 0);
  if (smem > 48 * 1024)
    ABG_CUDA(cudaFuncSetAttribute(k_jacobi, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_jacobi<<<1, threads, smem, s>>>(l, A, V, evals, evecs, 40, a_smem, v_smem);
  ::abg::note_launch();
  ABG_LAUNCH_CHECK();
  return ABG_OK;
}

// ---------------------------------------------------------------------------
// Truncated randomized SVD (subspace iteration) and the factors the method
// needs from it.
// ---------------------------------------------------------------------------
// sign_j = +1 if colsum(Q) . U[:, j] >= 0 else -1 (left vectors summing >= 0);
// Bm[p][j] = U[p][j] * sign_j * (scale ? sigma_j : 1) for j < k (float, ld ldb)
__global__ void k_rsvd_post(int l, int k, const double* __restrict__ evals,
                            const double* __restrict__ U, const double* __restrict__ qsum,
                            int with_sigma, float* __restrict__ Bm, int64_t ldb,
                            double* __restrict__ Uks /* l x k signed, FP64 */,
                            double* __restrict__ sigma_out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= k) return;
  double dot = 0.0;
  for (int p = 0; p < l; ++p) dot += qsum[p] * U[(int64_t)p * l + j];
  const double sg = dot < 0.0 ? -1.0 : 1.0;
  const double sigma = sqrt(fmax(evals[j], 0.0));
  for (int p = 0; p < l; ++p) {
    const double u = U[(int64_t)p * l + j] * sg;
    Uks[(int64_t)p * k + j] = u;
    Bm[(int64_t)p * ldb + j] = (float)(with_sigma ? u * sigma : u);
  }
  if (sigma_out) sigma_out[j] = sigma;
}

__global__ void k_relu_f64_to_f32(int rows, int cols, const double* __restrict__ a, int64_t lda,
                                  float* __restrict__ o, int64_t ldo) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= (int64_t)rows * cols) return;
  const int i = (int)(q / cols), j = (int)(q % cols);
  o[(int64_t)i * ldo + j] = (float)fmax(a[(int64_t)i * lda + j], 0.0);
}

// Y (rows x l) = A * Om (dense: gemm_nn; CSR: SpMM)
static int apply_a(const RsvdIn& in, const float* Om, int64_t ldo, int l, float* Y, int64_t ldy,
                   cudaStream_t s) {
  if (in.A)
    return gemm_nn(in.n, l, in.m, in.A, in.lda, Om, ldo, Y, ldy, Epi::Store, nullptr, 0, nullptr,
                   0, nullptr, s);
  return spmm_plain(in.ptr, in.col, in.val, in.n, Om, ldo, l, Y, ldy, s);
}

// Bt (m x l, FP64) = A^T Q
static int apply_at(const RsvdIn& in, const float* Q, int64_t ldq, int l, double* Bt, float* tmp32,
                    int64_t ldt, Scratch& scr, cudaStream_t s) {
  if (in.A) return gemm_tn(in.n, in.m, l, in.A, in.lda, Q, ldq, Bt, l, scr, s);
  ABG_TRY(spmm_plain(in.tptr, in.tcol, in.tval, in.m, Q, ldq, l, tmp32, ldt, s));
  k_f32_to_f64<<<(unsigned)ceil_div((int64_t)in.m * l, 256), 256, 0, s>>>(in.m, l, tmp32, ldt, Bt, l); ::abg::note_launch();
  ABG_LAUNCH_CHECK();
  return ABG_OK;
}

int rsvd(const RsvdIn& in, int k, int oversample, int power_iters, uint64_t seed, int stream_id,
         const RsvdOut& out, int* breakdowns, Scratch& /*caller*/, cudaStream_t s) {
  Scratch scr(s);
  const int64_t n = in.n;
  const int m = in.m;
  const int l = (int)std::min<int64_t>({(int64_t)k + oversample, (int64_t)m, n});
  ABG_CHECK(k >= 1 && k <= l, "rsvd: need 1 <= k <= min(n, m)");
  ABG_CHECK(l <= 1024, "rsvd: k + oversample must stay <= 1024");
  const int64_t ll = round_up(l, 4);
  float *Om, *Y, *Yt, *T1, *T2, *Bm;
  double *Bt, *M, *evals, *evecs, *qsum, *Uks, *Hd;
  ABG_TRY(scr.get(&Om, (size_t)m * ll));
  ABG_TRY(scr.get(&Y, (size_t)n * ll));
  ABG_TRY(scr.get(&T1, (size_t)n * ll));
  ABG_TRY(scr.get(&Yt, (size_t)m * ll));
  ABG_TRY(scr.get(&T2, (size_t)m * ll));
  ABG_TRY(scr.get(&Bt, (size_t)m * l));
  ABG_TRY(scr.get(&M, (size_t)l * l));
  ABG_TRY(scr.get(&evals, (size_t)l));
  ABG_TRY(scr.get(&evecs, (size_t)l * l));
  ABG_TRY(scr.get(&qsum, (size_t)l));
  ABG_TRY(scr.get(&Uks, (size_t)l * k));
  ABG_TRY(scr.get(&Hd, (size_t)m * k));
  const int64_t kk = round_up(k, 4);
  ABG_TRY(scr.get(&Bm, (size_t)l * kk));
  // range finder
  ABG_TRY(gaussian_f32(seed, stream_id, m, l, Om, ll, s));
  ABG_TRY(apply_a(in, Om, ll, l, Y, ll, s));
  ABG_TRY(cholqr2(n, l, Y, ll, T1, ll, breakdowns, scr, s));
  for (int it = 0; it < power_iters; ++it) {
    ABG_TRY(apply_at(in, Y, ll, l, Bt, T2, ll, scr, s));
    k_f64_to_f32<<<(unsigned)ceil_div((int64_t)m * l, 256), 256, 0, s>>>(m, l, Bt, l, Yt, ll, 0); ::abg::note_launch();
    ABG_LAUNCH_CHECK();
    ABG_TRY(cholqr2(m, l, Yt, ll, T2, ll, breakdowns, scr, s));
    ABG_TRY(apply_a(in, Yt, ll, l, Y, ll, s));
    ABG_TRY(cholqr2(n, l, Y, ll, T1, ll, breakdowns, scr, s));
  }
  // B^T = A^T Q (m x l), B B^T = Bt^T Bt (l x l), eigenpairs
  ABG_TRY(apply_at(in, Y, ll, l, Bt, T2, ll, scr, s));
  small_tn64(m, l, l, Bt, l, Bt, l, M, l, s);
  ABG_LAUNCH_CHECK();
  ABG_TRY(jacobi_eig(l, M, evals, evecs, scr, s));
  ABG_TRY(column_sums(n, l, Y, ll, qsum, scr, s));
  k_rsvd_post<<<(unsigned)ceil_div(k, 128), 128, 0, s>>>(l, k, evals, evecs, qsum, out.left_mode,
                                                         Bm, kk, Uks, out.sigma); ::abg::note_launch();
  ABG_LAUNCH_CHECK();
  // left factor: Q * (U_k signed [* Sigma]) with max(., 0) for Phi
  ABG_TRY(gemm_nn(n, k, l, Y, ll, Bm, kk, out.left, out.ldl,
                  out.left_mode == 0 ? Epi::Relu : Epi::Store, nullptr, 0, nullptr, 0, nullptr, s));
  if (out.right) {  // H = max(B^T U_k, 0) = max(Psi Sigma, 0)
    small_nn64(m, l, k, Bt, l, Uks, k, Hd, k, s);
    k_relu_f64_to_f32<<<(unsigned)ceil_div((int64_t)m * k, 256), 256, 0, s>>>(m, k, Hd, k,
                                                                             out.right, out.ldr); ::abg::note_launch();
    ABG_LAUNCH_CHECK();
  }
  return ABG_OK;
}

}  // namespace abg
