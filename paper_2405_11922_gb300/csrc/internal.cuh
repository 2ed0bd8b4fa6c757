// Internal interfaces between the library's translation units.
#pragma once

#include "common.cuh"

// Device-resident graph (Section 2.1): both CSR (rows = U) and CSC (rows = V)
// with the L_U values of Eq. 7 stored per edge in each order, the degree
// scales, the attributes, and the row schedules of the two SpMMs.
struct abg_graph {
  int device = 0;
  int64_t n_u = 0, n_v = 0, nnz = 0;
  int32_t d_u = 0;
  int32_t x_kind = 0;
  // CSR of L_U (U rows) and CSC (= CSR of L_U^T, V rows)
  int64_t* u_ptr = nullptr;
  int32_t* u_col = nullptr;
  float* u_val = nullptr;
  int64_t* v_ptr = nullptr;
  int32_t* v_col = nullptr;
  float* v_val = nullptr;
  float* su = nullptr;  // D_U^-1/2 (0 for zero degree)
  float* sv = nullptr;  // D_V^-1/2
  // attributes: dense (f32 or bf16, row stride ldx) or CSR (+ its transpose)
  void* x = nullptr;
  int64_t ldx = 0;
  int64_t x_nnz = 0;
  int64_t* x_ptr = nullptr;
  int32_t* x_col = nullptr;
  float* x_val = nullptr;
  int64_t* xt_ptr = nullptr;
  int32_t* xt_col = nullptr;
  float* xt_val = nullptr;
  // SpMM schedules: light rows in decreasing-degree order, heavy rows split
  // into fixed-size edge chunks whose partial sums are reduced in order.
  struct Schedule {
    int64_t n_light = 0;
    int32_t* light = nullptr;        // row ids
    int64_t n_chunks = 0;
    int64_t* chunk_begin = nullptr;  // edge range of each chunk
    int32_t* chunk_row_slot = nullptr;  // heavy-row slot of each chunk
    int64_t n_heavy = 0;
    int32_t* heavy_row = nullptr;    // row id of each heavy slot
    int64_t* heavy_chunk0 = nullptr; // first chunk of each heavy slot (n_heavy + 1)
  } sched_u, sched_v;
  int64_t footprint = 0;
  void* blocks[32] = {};
  int n_blocks = 0;
};

namespace abg {

constexpr int kMaxK = 128;     // clusters supported by the NCI kernels
constexpr int kMaxD = 1024;    // feature width supported by the SpMMs
constexpr int kHeavyChunk = 256;   // edges per chunk of a split row
constexpr int kHeavyRow = 1024;    // rows with more edges are split

// ---- graph.cu ---------------------------------------------------------------
int graph_alloc(abg_graph* g, void** p, size_t bytes, cudaStream_t s);

// ---- spmm.cu ----------------------------------------------------------------
// Algorithm 1 propagation + Eq. 2 on device buffers. Exactly one of x_f32 /
// x_bf16 is non-null (dense attributes, row stride ldx, width d).
int propagate(const abg_graph* g, const float* x_f32, const __nv_bfloat16* x_bf16, int64_t ldx,
              int d, double alpha, int gamma, float* zhat, int64_t ldz, cudaStream_t s);
// C[rows][ldc] = A_csr (rows x K) * B[K][ldb] (width n, plain sum per row).
int spmm_plain(const int64_t* ptr, const int32_t* col, const float* val, int64_t rows,
               const float* B, int64_t ldb, int n, float* C, int64_t ldc, cudaStream_t s);
// dense[rows][ld] (zeroed first) <- CSR
int csr_to_dense(const int64_t* ptr, const int32_t* col, const float* val, int64_t rows, int cols,
                 float* dense, int64_t ld, cudaStream_t s);
int bf16_to_f32(const __nv_bfloat16* x, int64_t ldx, int64_t rows, int cols, float* out,
                int64_t ldo, cudaStream_t s);

// ---- dense.cu ---------------------------------------------------------------
enum class Epi : int {
  Store = 0,        // C = acc
  Relu = 1,         // C = max(acc, 0)
  SignRelu = 2,     // C = max(sign[col] * acc, 0)
  Sign = 3,         // C = sign[col] * acc
  PhiUpdate = 4,    // C = phi * sqrt(max(aux,0)/acc) (acc > 0) else 0   [Eq. 17]
};
// C[M][ldc] = A[M][lda] (M x K) * B[K][ldb] (K x N) with the epilogue.
// aux/aux2: PhiUpdate reads P=aux[M][ldaux] and phi=aux2[M][ldaux2]; sign[N] for Sign*.
int gemm_nn(int64_t M, int N, int K, const float* A, int64_t lda, const float* B, int64_t ldb,
            float* C, int64_t ldc, Epi epi, const float* aux, int64_t ldaux, const float* aux2,
            int64_t ldaux2, const float* sign, cudaStream_t s);
// C[K][N] (FP64, row stride ldc) = A[M][lda]^T (K x M) * B[M][ldb] (M x N), reduction over
// the long dimension M in fixed-size row chunks (FP32 products, FP64 accumulation).
int gemm_tn(int64_t M, int K, int N, const float* A, int64_t lda, const float* B, int64_t ldb,
            double* C, int64_t ldc, Scratch& scr, cudaStream_t s);
// colsum[N] (FP64) of A[M][lda]
int column_sums(int64_t M, int N, const float* A, int64_t lda, double* out, Scratch& scr,
                cudaStream_t s);
// Eqs. 13-14 on zhat (n x d) with Qt[d][d] = Q^T (float), result in R[n][ldr] (2d wide).
int random_features(const float* zhat, int64_t n, int d, int64_t ldz, const float* qt,
                    float* R, int64_t ldr, int* clamped_dev, Scratch& scr, cudaStream_t s);
// Eq. 16 on small matrices: H[m][ldh] <- H * max(A,0) / (H G) (A, G FP64).
int nmf_update_h(int m, int k, float* H, int64_t ldh, const double* A, int64_t lda,
                 const double* G, int64_t ldg, cudaStream_t s);
// Algorithm 3 (all t_g passes) on phi (n x k).
int nci_run(const float* phi, int64_t n, int k, int64_t ldphi, int t_g, int32_t* labels,
            float* margin, double* t_out, int* last_changes_host, float* min_margin_host,
            int* empty_host, Scratch& scr, cudaStream_t s);
// Eq. 8 (objective, trace) through per-cluster sums.
int objective(const float* R, int64_t n, int m, int64_t ldr, const int32_t* labels, int k,
              double* obj_host, Scratch& scr, cudaStream_t s);

// ---- linalg.cu --------------------------------------------------------------
// Gaussian matrix (rows x cols, row stride ld) from (seed, stream id) as described in abg.h.
int gaussian_f64(uint64_t seed, int stream_id, int rows, int cols, double* out, int64_t ld,
                 cudaStream_t s);
int gaussian_f32(uint64_t seed, int stream_id, int rows, int cols, float* out, int64_t ld,
                 cudaStream_t s);
// Q (d x d, FP64) = orthogonal factor of QR(G) with positive diag(R); G from ABG_STREAM_G.
int orthogonal_matrix(uint64_t seed, int d, double* q, cudaStream_t s);
// CholeskyQR2 in place: Y[M][ldy] (M x l) -> orthonormal columns. breakdowns (device int) counts
// non-positive pivots.
int cholqr2(int64_t M, int l, float* Y, int64_t ldy, float* tmp, int64_t ldt, int* breakdowns,
            Scratch& scr, cudaStream_t s);
// Truncated randomized SVD of A (n x m, dense float) or of a CSR matrix (with its transpose).
struct RsvdOut {
  float* left = nullptr;        // n x k, row stride ldl: max(Gamma,0) / Gamma*Sigma / ...
  int64_t ldl = 0;
  int left_mode = 0;            // 0: max(Gamma,0)   1: Gamma*Sigma (signed)
  float* right = nullptr;       // m x k, row stride ldr: max(Psi*Sigma, 0) (may be null)
  int64_t ldr = 0;
  double* sigma = nullptr;      // k (device, may be null)
};
struct RsvdIn {
  int64_t n = 0;
  int m = 0;
  const float* A = nullptr;     // dense n x m
  int64_t lda = 0;
  const int64_t* ptr = nullptr; // or CSR (n x m) + CSR of the transpose (m x n)
  const int32_t* col = nullptr;
  const float* val = nullptr;
  const int64_t* tptr = nullptr;
  const int32_t* tcol = nullptr;
  const float* tval = nullptr;
};
int rsvd(const RsvdIn& in, int k, int oversample, int power_iters, uint64_t seed, int stream_id,
         const RsvdOut& out, int* breakdowns, Scratch& scr, cudaStream_t s);
int transpose_f64_to_f32(const double* a, int rows, int cols, int64_t lda, float* out,
                         int64_t ldo, cudaStream_t s);
int convert_f64_to_f32(const double* a, int rows, int cols, int64_t lda, float* out, int64_t ldo,
                       cudaStream_t s);

}  // namespace abg
