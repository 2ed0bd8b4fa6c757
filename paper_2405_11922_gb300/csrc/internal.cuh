// Internal interfaces between the library's translation units.
#pragma once

#include <memory>
#include <mutex>
#include <vector>

#include "batch.cuh"
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
  int64_t* xt_ptr = nullptr;   // transposed CSR of X per segment: row s*d_u + j lists the
  int32_t* xt_col = nullptr;   //   rows of segment s holding column j (global row ids)
  float* xt_val = nullptr;
  int32_t* xr_col = nullptr;   // X CSR columns as s*d_u + j (the stacked test-block rows)
  // segments: a graph made by abg_batch_create stacks independent graphs
  // (block-diagonal union); segment s owns U rows [seg_row0[s], +seg_n[s])
  int nseg = 1;
  std::vector<int64_t> seg_row0, seg_n;
  // SpMM schedules: light rows in tasks of consecutive rows, heavy rows split
  // into fixed-size edge chunks whose partial sums are reduced in order.
  struct Schedule {
    int64_t n_tasks = 0;
    int2* tasks = nullptr;           // light rows [x, y) of each task, consecutive and in order
    int64_t n_etasks = 0, n_ztasks = 0;
    int2* etasks = nullptr;          // the tasks that hold edges
    int2* ztasks = nullptr;          // the tasks whose rows have no edges
    int64_t n_chunks = 0;
    int64_t* chunk_begin = nullptr;  // edge range of each chunk
    int32_t* chunk_row_slot = nullptr;  // heavy-row slot of each chunk
    int64_t n_heavy = 0;
    int32_t* heavy_row = nullptr;    // row id of each heavy slot
    int64_t* heavy_chunk0 = nullptr; // first chunk of each heavy slot (n_heavy + 1)
  } sched_u, sched_v;
  int* wait_err = nullptr;  // device flag: a bounded wait inside a kernel ran out
  // Z_hat kept by a solve with ABG_REUSE_PROPAGATION (one at a time; see pipeline.cu)
  std::mutex zmu;
  std::shared_ptr<struct ZCache> zcache;
  std::shared_ptr<struct PhiCache> phicache;  // final Phi, H of a solve with ABG_WARM_START
  int64_t footprint = 0;
  void* blocks[64] = {};
  int n_blocks = 0;
};

namespace abg {

constexpr int kMaxK = 128;     // clusters supported by the NCI kernels
constexpr int kMaxRsvdBlock = 1024;  // randomized-SVD block width (and orthogonal-matrix size)
constexpr int kMaxD = 1024;    // feature width supported by the SpMMs
#ifndef ABG_TASK_EDGES
#define ABG_TASK_EDGES 128
#endif
constexpr int kHeavyChunk = ABG_TASK_EDGES;  // edges per chunk of a split row
constexpr int kHeavyRow = ABG_TASK_EDGES;    // rows with more edges are split
constexpr int kTaskRows = 32;                // light rows per task, at most
constexpr int kTaskEdges = ABG_TASK_EDGES;   // edges per task, at most (light rows: <= kHeavyRow)
static_assert(kHeavyRow <= kTaskEdges && kTaskEdges % 4 == 0 && kTaskRows <= 32,
              "task limits must fit the SpMM kernels' staging");

// ---- graph.cu ---------------------------------------------------------------
int graph_alloc(abg_graph* g, void** p, size_t bytes, cudaStream_t s);
// host-only validation of a graph descriptor (CSR, optional CSC, weights, attributes)
int validate_desc(const abg_graph_desc* d);
// Parameters of one solve on g (n_rows clustered nodes): ABG_EINVAL with a message if invalid;
// *d_eff = the attribute width the solve uses.
int check_params(const abg_graph* g, const abg_params* p, int64_t n_rows, int* d_eff);
// A descriptor with side = ABG_SIDE_V seen as the equivalent ABG_SIDE_U descriptor (U and V
// exchanged; a CSC the caller did not give is built into `store`, which must outlive *out).
struct SideSwap {
  abg_graph_desc desc{};
  std::vector<int64_t> vp;
  std::vector<int32_t> ui;
  std::vector<float> wt;
};
int swap_sides(const abg_graph_desc* in, SideSwap* store, const abg_graph_desc** out);

// ---- spmm.cu ----------------------------------------------------------------
// Algorithm 1 propagation + Eq. 2 on device buffers. Exactly one of x_f32 /
// x_bf16 is non-null (dense attributes, row stride ldx, width d).
// Reads (and clears) the graph's wait flag after the stream's work: ABG_EDEVICE when a
// bounded wait inside a kernel ran out. Synchronises s.
int check_wait_flag(const abg_graph* g, cudaStream_t s);
// bf16_rounds: W and the intermediate Z are stored in BF16 between the SpMMs (each gather
// still accumulates in FP32); the final Z-hat is FP32 either way.
int propagate(const abg_graph* g, const float* x_f32, const __nv_bfloat16* x_bf16, int64_t ldx,
              int d, double alpha, int gamma, float* zhat, int64_t ldz, cudaStream_t s,
              bool bf16_rounds = false);
// C[rows][ldc] = A_csr (rows x K) * B[K][ldb] (width n, plain sum per row).
int spmm_plain(const int64_t* ptr, const int32_t* col, const float* val, int64_t rows,
               const float* B, int64_t ldb, int n, float* C, int64_t ldc, cudaStream_t s);
// dense[rows][ld] (zeroed first) <- CSR
int csr_to_dense(const int64_t* ptr, const int32_t* col, const float* val, int64_t rows, int cols,
                 float* dense, int64_t ld, cudaStream_t s);
int bf16_to_f32(const __nv_bfloat16* x, int64_t ldx, int64_t rows, int cols, float* out,
                int64_t ldo, cudaStream_t s);
// out = x rounded to BF16 (nearest even)
int f32_to_bf16(const float* x, int64_t ldx, int64_t rows, int cols, __nv_bfloat16* out,
                int64_t ldo, cudaStream_t s);

// ---- dense.cu (row spaces of batch.cuh; a plain solve is one segment) -------
enum class Epi : int {
  Store = 0,        // C = acc
  Relu = 1,         // C = max(acc, 0)
  SignRelu = 2,     // C = max(sign_s[col] * acc, 0)
  Sign = 3,         // C = sign_s[col] * acc
  PhiUpdate = 4,    // C = phi * sqrt(max(P,0)/acc) (acc > 0) else 0   [Eq. 17]
};
// C = A B_s for the rows of segment s (B_s at B + s*b_seg; per-segment N_s/K_s when segN/segK
// are given, else N/K). aux = P, aux2 = phi for PhiUpdate; sign_s at sign + s*sign_seg.
struct NN {
  const float* A = nullptr;
  int64_t lda = 0;
  // the same A stored in BF16 (row stride lda16): the product may then run on the BF16
  // tensor-core kernel (B rounded to BF16, FP32 accumulation); A is the fallback
  const __nv_bfloat16* A16 = nullptr;
  int64_t lda16 = 0;
  const float* B = nullptr;
  int64_t ldb = 0, b_seg = 0;
  float* C = nullptr;
  int64_t ldc = 0;
  int N = 0, K = 0;
  const int* segN = nullptr;
  const int* segK = nullptr;
  Epi epi = Epi::Store;
  const float* aux = nullptr;
  int64_t ldaux = 0;
  const float* aux2 = nullptr;
  int64_t ldaux2 = 0;
  const float* sign = nullptr;
  int64_t sign_seg = 0;
  // random features: R'[i] = out_scale (sin || cos)(in_scale acc), per-tile column sums
  bool sincos = false;
  float in_scale = 1.f, out_scale = 1.f;
  double* colsum_part = nullptr;
  // NCI scores: row argmax into labels (+ margin), per-segment change / min-margin counters
  bool argmax = false;
  int32_t* labels = nullptr;
  float* margin = nullptr;
  int first = 0;
  int* changes = nullptr;
  unsigned* minbits = nullptr;
};
int gemm_nn(const RowSpace& rs, const NN& a, cudaStream_t s);
// The same product on the tensor cores (tcgen05, three-term tf32 split); *used = false when
// the shape or layout is outside its limits (N <= 256, 16-byte rows; the sin/cos epilogue
// with one N for all segments) or ABG_TENSOR_CORES=0 is set in the environment.
int tc_gemm_nn(const RowSpace& rs, const NN& a, cudaStream_t s, bool* used);
// Chunk partials part[c][K][N] (fp32) of a TN product on the tensor cores; *used = false
// when outside its limits (K, N <= 256, 16-byte rows) or ABG_TENSOR_CORES=0.
struct TN;
int tc_gemm_tn(const RowSpace& rs, const TN& a, float* part, cudaStream_t s, bool* used);
// BF16 forms of the two (kind::f16, FP32 accumulation) for a.A16 != null, no segK, and in
// the TN case K, N <= 256.
int tc_gemm_nn16(const RowSpace& rs, const NN& a, cudaStream_t s, bool* used);
int tc_gemm_tn16(const RowSpace& rs, const TN& a, float* part, cudaStream_t s, bool* used);
// Reads and clears the tensor-core kernels' wait flag (synchronises s): the flag of the solve
// open on this thread (TcFlagScope), else the process-wide flag the step calls use.
int tc_wait_flag(cudaStream_t s, int* flag);
// While alive, the tensor-core kernels launched from this thread report a wait that ran out
// in `flag` (a device int of the caller's solve, zeroed), so concurrent solves on other
// threads and streams neither see nor clear each other's reports.
struct TcFlagScope {
  int* prev;
  explicit TcFlagScope(int* flag);
  ~TcFlagScope();
};
// C_s (K_s x N_s, FP64, at C + s*c_seg, row stride ldc) = A^T B over the rows of segment s.
struct TN {
  const float* A = nullptr;
  int64_t lda = 0;
  const __nv_bfloat16* A16 = nullptr;  // as NN::A16
  int64_t lda16 = 0;
  const float* B = nullptr;
  int64_t ldb = 0;
  int K = 0, N = 0;
  const int* segK = nullptr;
  const int* segN = nullptr;
  double* C = nullptr;
  int64_t ldc = 0, c_seg = 0;
};
int gemm_tn(const RowSpace& rs, const TN& a, cudaStream_t s);
// colsum_s[N] (FP64, at out + s*oseg) of A over the rows of segment s
int column_sums(const RowSpace& rs, int N, const float* A, int64_t lda, double* out, int64_t oseg,
                cudaStream_t s);
// Eqs. 13-14: R (2d wide) from zhat (d wide) with Qt_s = Q_s^T at qt + s*d*ldq; per-segment r;
// clamped_dev[s] counts clamped rows.
// R16 (may be null): a BF16 copy of R (row stride ldr16) written by the same pass.
int random_features(const RowSpace& rs, const float* zhat, int d, int64_t ldz, const float* qt,
                    int64_t ldq, float* R, int64_t ldr, int* clamped_dev, cudaStream_t s,
                    __nv_bfloat16* R16 = nullptr, int64_t ldr16 = 0);
// Eq. 16 per segment (H_s at H + s*hseg, m x k_s; A_s, G_s FP64 slabs).
int nmf_update_h(int nseg, int m, const int* segk, int kmax, float* H, int64_t ldh, int64_t hseg,
                 const double* A, int64_t lda, int64_t aseg, const double* G, int64_t ldg,
                 int64_t gseg, cudaStream_t s);
// C_s (k_s x k_s, FP64) = A_s^T H_s with A_s (m x k_s, FP64) and H_s (m x k_s, FP32).
int small_atb(int nseg, int m, const int* segk, int kmax, const double* A, int64_t lda,
              int64_t aseg, const float* H, int64_t ldh, int64_t hseg, double* C, int64_t ldc,
              int64_t cseg, cudaStream_t s);
// Algorithm 3 per segment (t_g passes; flags = ABG_NCI_*). counters (device, 3*nseg ints):
// last-pass label changes, minimum margin (float bits), empty clusters. passes (host,
// optional): the passes each segment needed (t_g unless it stopped early).
int nci_run(const RowSpace& rs, const SegSizes& ss, const float* phi, int64_t ldphi, int t_g,
            int flags, int32_t* labels, float* margin, double* t_out, int* counters,
            std::vector<int>* passes, cudaStream_t s);
// Eq. 8 per segment: out_dev[2s] = objective, out_dev[2s+1] = Tr(Y^T R R^T Y).
int objective(const RowSpace& rs, const SegSizes& ss, const float* R, int m, int64_t ldr,
              const int32_t* labels, double* out_dev, cudaStream_t s);

// ---- linalg.cu --------------------------------------------------------------
// Right singular vectors and squared singular values (descending) of Bt_s (m x l_s, FP64, row
// stride lmax inside an m*lmax slab): FP32 one-sided Jacobi, results FP64 (l_s x l_s slabs of
// stride lmax). warm (nseg slabs of lmax*lmax floats, optional): the rotations are stored
// there on exit, and with warm_valid the sweeps start from the ones stored by the last call.
// skip (device, per segment, optional): segments with a non-zero entry are left untouched.
// square: segment s is l_s x l_s inside an lmax x lmax slab of zeros (m == lmax), so the
// orthogonality threshold follows l_s (the same result alone and in a batch).
int svd_right(int nseg, int m, const int* segl, int lmax, const double* Bt, double* evals,
              double* evecs, cudaStream_t s, float* warm = nullptr, bool warm_valid = false,
              const int* skip = nullptr, bool square = false);
// Orthogonal Procrustes factor of M_s (k_s x k_s in a kmax x kmax FP64 slab) by the
// Newton-Schulz iteration on a thread-block cluster: T_s (FP32, row stride kp) and t64_s (FP64
// k x k slab, may be null) are written and done[s] = 1 when the iteration meets the stopping
// rule that reproduces the 1e-5 s_1 threshold; done[s] = 0 leaves the segment to svd_right.
int polar_newton_schulz(int nseg, const int* segk, int kmax, const double* M, int kp, float* T,
                        double* t64, int* done, cudaStream_t s);
// Gaussian matrix (rows x cols, row stride ld) of each segment from (seeds[s], stream id); the
// segment's block sits at out + s*oseg; columns >= cols_s (segcols) are set to 0.
int gaussian_f64(int nseg, const uint64_t* seeds, int stream_id, int rows, int cols, double* out,
                 int64_t ld, int64_t oseg, cudaStream_t s);
int gaussian_f32(int nseg, const uint64_t* seeds, int stream_id, int rows, int cols,
                 const int* segcols, float* out, int64_t ld, int64_t oseg, cudaStream_t s);
// Q_s (d x d, FP64, at q + s*d*d) = orthogonal factor of QR(G_s), diag(R) > 0, G_s drawn from
// seeds[s] on ABG_STREAM_G.
int orthogonal_matrices(int nseg, const uint64_t* seeds, int d, double* q, cudaStream_t s);
// CholeskyQR2 in place on Y (rows of each segment, l_s columns, row stride ldy).
int cholqr2(const RowSpace& rs, const int* segl, int lmax, float* Y, int64_t ldy, float* tmp,
            int64_t ldt, int* breakdowns, cudaStream_t s);
// Truncated randomized SVD per segment (randomized subspace iteration).
struct RsvdIn {
  const RowSpace* rows = nullptr;  // rows of A (one segment per problem)
  int m = 0;                       // columns of A (same for every segment)
  const float* A = nullptr;        // dense rows x m
  int64_t lda = 0;
  const __nv_bfloat16* A16 = nullptr;  // optional BF16 copy of A for the BF16 products
  int64_t lda16 = 0;
  // or a CSR whose column j of segment s is stored as s*m + j, and the CSR of the
  // transposes with row s*m + j listing segment s's rows (global row ids)
  const int64_t* ptr = nullptr;
  const int32_t* col = nullptr;
  const float* val = nullptr;
  const int64_t* tptr = nullptr;
  const int32_t* tcol = nullptr;
  const float* tval = nullptr;
};
struct RsvdOut {
  float* left = nullptr;        // rows x (k_s or kfixed), row stride ldl
  int64_t ldl = 0;
  int left_mode = 0;            // 0: max(Gamma, 0)   1: Gamma * Sigma
  float* right = nullptr;       // per segment m x k_s (max(Psi Sigma, 0)), at right + s*rseg
  int64_t ldr = 0, rseg = 0;
  double* sigma = nullptr;      // per segment k_s values at sigma + s*sseg (may be null)
  int64_t sseg = 0;
};
// k per segment: ss.k (left_mode 0) or the uniform kfixed (left_mode 1, ss.k ignored);
// l per segment: ss.l; seeds: ss.seed.
int rsvd(const RsvdIn& in, const SegSizes& ss, int kfixed, int power_iters, int stream_id,
         const RsvdOut& out, int* breakdowns, cudaStream_t s);
int transpose_f64_to_f32(const double* a, int rows, int cols, int64_t lda, float* out,
                         int64_t ldo, cudaStream_t s);
int convert_f64_to_f32(const double* a, int64_t rows, int cols, int64_t lda, float* out,
                       int64_t ldo, cudaStream_t s);
// per-segment transpose of d x d FP64 blocks into FP32 (Qt_s = Q_s^T, row stride ldo)
int transpose_blocks(int nseg, int d, const double* q, float* qt, int64_t ldo, cudaStream_t s);

}  // namespace abg
