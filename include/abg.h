/*
 * abg.h — C ABI of a GB300 (sm_103a) implementation of TPO clustering on
 * attributed bipartite graphs (Yang et al., "Effective Clustering on Large
 * Attributed Bipartite Graphs", KDD'24, arXiv 2405.11922).
 *
 * Conventions for every call
 *   - Returns int status: ABG_OK (0), ABG_PENDING (1) or a negative error.
 *     Nothing throws across this boundary; abg_strerror() names the code and
 *     abg_last_error() gives a one-line detail of the last failure on the
 *     calling thread.
 *   - "host" pointers are read with plain loads; "device" pointers must be
 *     device memory of the graph's device (cudaMalloc / a PyTorch CUDA tensor).
 *     Where a pointer may be either, cudaMemcpy with cudaMemcpyDefault is used.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream). Step calls
 *     only enqueue work on it; abg_cluster synchronises it before returning.
 *   - Dense matrices are row-major with an explicit leading dimension `ld*`
 *     (elements between consecutive rows), ld >= width and ld a multiple of 4
 *     (16-byte rows for float). Every device matrix must be 16-byte aligned.
 *   - Sizes: |U|, |V| < 2^31, nnz < 2^62, 1 <= d <= 1024, 1 <= k <= 128.
 *   - The library allocates its own device memory (stream-ordered, from a
 *     private pool per device); callers own the buffers they pass in.
 *
 * Notation follows the paper: B_U (|U| x |V|) the weighted adjacency,
 * D_U / D_V the weighted degrees (Section 2.1), L_U = D_U^-1/2 B_U D_V^-1/2
 * (Eq. 7), X_U the U attributes, Z_U / Z_hat the propagated / row-normalised
 * features (Eqs. 6, 2), R the random-feature matrix (Eqs. 13-14), Phi and H the
 * NMF factors (Eqs. 11, 16-18), Y the normalised cluster indicator (Eq. 10).
 */
#ifndef ABG_H
#define ABG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define ABG_API __attribute__((visibility("default")))
#else
#define ABG_API
#endif

/* ---- status codes -------------------------------------------------------- */
#define ABG_OK 0
#define ABG_PENDING 1            /* abg_poll: the job has not finished yet      */
#define ABG_EINVAL (-1)          /* bad argument or malformed input             */
#define ABG_ENOMEM (-2)          /* device allocation failed                    */
#define ABG_EDEVICE (-3)         /* CUDA error (launch, copy, bounded wait)     */
#define ABG_ENOTADMITTED (-4)    /* job footprint exceeds the server budget     */
#define ABG_ETIMEDOUT (-5)       /* abg_poll: timeout elapsed                   */
#define ABG_ENOTFOUND (-6)       /* unknown request id                          */
#define ABG_ECANCELLED (-7)      /* request cancelled / server shut down        */
#define ABG_ENUMERIC (-8)        /* non-finite values or a singular Gram matrix */

/* ---- attribute storage kinds (abg_graph_desc.x_kind) --------------------- */
#define ABG_X_DENSE_F32 0        /* x: float [n_u][d_u]                          */
#define ABG_X_DENSE_BF16 1       /* x: uint16 bfloat16 bit patterns [n_u][d_u]   */
#define ABG_X_CSR_F32 2          /* x_ptr[n_u+1], x_idx[x_nnz], x_val[x_nnz]     */

/* ---- random streams of the counter-based generator ----------------------- */
/* Gaussian entry e of a matrix drawn on stream s with key `seed` comes from
 * Philox4x32-10 (Salmon et al., SC'11) at counter (b mod 2^32, b >> 32, s, 0),
 * b = e / 4, key (seed mod 2^32, seed >> 32), through Box-Muller on the two
 * word pairs (u = (x + 0.5) 2^-32; cos / sin of 2 pi u_b times
 * sqrt(-2 ln u_a)); entry e takes output e mod 4. */
#define ABG_STREAM_G 1           /* Algorithm 1: G (d x d) -> Q                  */
#define ABG_STREAM_OMEGA_R 2     /* Algorithm 2: test matrix of the SVD of R     */
#define ABG_STREAM_OMEGA_X 3     /* Section 3.2.1: test matrix of the SVD of X_U */

typedef struct abg_graph abg_graph;

/* Input graph (Definition 1, Section 2.1). All pointers are HOST memory and
 * are copied; the caller keeps ownership. The CSR must have a monotone u_ptr
 * with u_ptr[0] = 0, u_ptr[n_u] = nnz and v_idx in [0, n_v). w == NULL means
 * unit weights; weights must be finite and > 0. The CSC (v_ptr, u_idx, w_t)
 * is optional (all three NULL: it is built by a stable counting sort); when
 * given it must hold exactly the same edges.
 * side: ABG_SIDE_U clusters U with attributes X_U (x rows = n_u). ABG_SIDE_V
 * clusters V instead (the method with the roles of U and V exchanged; x then
 * holds X_V, n_v rows, and every per-node output has n_v entries). */
#define ABG_SIDE_U 0
#define ABG_SIDE_V 1
typedef struct {
  int64_t n_u, n_v, nnz;
  const int64_t* u_ptr;
  const int32_t* v_idx;
  const float* w;
  const int64_t* v_ptr;
  const int32_t* u_idx;
  const float* w_t;
  int32_t d_u;
  int32_t x_kind;
  const void* x;
  const int64_t* x_ptr;
  const int32_t* x_idx;
  const float* x_val;
  int32_t device;
  int32_t side;
} abg_graph_desc;

/* Method parameters (Table 1). d = 0 means d = d_u (no attribute reduction,
 * "TPO (d = d_U)"); 1 <= d < d_u turns on the SVD reduction of Section 3.2.1.
 * alpha in [0, 1), gamma >= 0, 1 <= k <= min(|U|, 2d, 128), t_f, t_g >= 0,
 * oversample >= 0 and power_iters >= 0 configure the truncated randomized
 * SVDs (Halko-Martinsson-Tropp subspace iteration). nci_flags (0 = Algorithm 3
 * as printed) combines:
 *   ABG_NCI_PROCRUSTES  T <- the orthogonal Procrustes factor of Phi^T Y (the
 *                       constraint T T^T = I of Eq. 20 enforced: T = U_r V_r^T
 *                       from Phi^T Y = U S V^T, singular values above 1e-5 s_1)
 *   ABG_NCI_EARLY_STOP  stop after the first pass (other than the first) that
 *                       changes no label: Y and T are then a fixed point, so
 *                       the result equals that of all t_g passes.
 * precision is ABG_PRECISION_FP32 (0, default: FP32 storage, FP32 sparse
 * products, dense products as 3xTF32 on the tensor cores) or a combination of
 *   ABG_BF16_CONTRACT     the dense contractions with the random-feature matrix
 *                         R (Algorithm 2: the randomized SVD's R Omega, R^T Q,
 *                         R Q'; Eqs. 16-17: R^T Phi, R H) and, with d < d_u
 *                         and BF16 attributes, those of the attribute SVD
 *                         (Section 3.2.1) run on the tensor cores with BF16
 *                         operands (R kept as a BF16 copy, the small operand
 *                         rounded to BF16) and FP32 accumulation. Gram
 *                         matrices, Cholesky-QR, the NCI scores and the
 *                         objective stay FP32 / FP64. Applies where the
 *                         BF16 kernels take the shape (2d <= 256 for the
 *                         R^T products); elsewhere the FP32 path runs.
 *   ABG_BF16_PROPAGATION  Algorithm 1 stores W = L^T Z and the intermediate Z
 *                         (rounds 1..gamma-1) in BF16 between its sparse
 *                         products, halving the bytes each gather reads. The
 *                         products accumulate in FP32 and Z_hat (the last
 *                         round, Eq. 2) is FP32.
 * options is 0 or a combination of ABG_REUSE_PROPAGATION and ABG_WARM_START.
 * ABG_REUSE_PROPAGATION: the solve may take Z_hat (Algorithm
 * 1: the propagation of Eq. 6 and the row normalisation of Eq. 2) from an
 * earlier solve on the same graph that had this option and the same alpha,
 * gamma, d and ABG_BF16_PROPAGATION bit (and, with d < d_u, the same seed,
 * oversample and power_iters, which fix X' of Eq. 15), and skip the attribute
 * reduction and the propagation: Z_hat depends on neither k, the NCI options
 * nor the other seeds. A solve with the option that finds no such Z_hat keeps
 * its own on the graph (n_u x round_up(d, 4) floats of device memory, held
 * until abg_destroy or until a solve with other keys replaces it; it counts in
 * abg_graph_footprint). Labels and objective are bitwise those of a solve
 * without the option. Ignored for batches (abg_batch_create). Without the
 * option nothing is kept or reused.
 * ABG_WARM_START (may be combined with the above; an option the paper does not
 * have): a resident re-solve, e.g. with another alpha, starts the T_f ONMF
 * steps of Algorithm 2 (Eqs. 16-17) from the Phi and H that an earlier solve
 * on the same graph with this option and the same k and d ended them with,
 * instead of the randomized-SVD seeding of Eq. 18 (which it skips). The result
 * is that of the ONMF and NCI steps from that start, not the one of a cold
 * solve. A solve with the option that finds no such factors seeds as usual and
 * keeps its final Phi and H on the graph (n_u x round_up(k, 4) and
 * 2d x round_up(k, 4) floats, held like Z_hat above and counted in
 * abg_graph_footprint). Ignored for batches. */
#define ABG_NCI_PROCRUSTES 1
#define ABG_NCI_EARLY_STOP 2
#define ABG_PRECISION_FP32 0
#define ABG_BF16_CONTRACT 1
#define ABG_BF16_PROPAGATION 2
#define ABG_REUSE_PROPAGATION 1
#define ABG_WARM_START 2
typedef struct {
  int32_t k, gamma, d, t_f, t_g, oversample, power_iters;
  int32_t nci_flags;
  double alpha;
  uint64_t seed;
  int32_t precision;
  int32_t options;
} abg_params;

/* Per-solve report. objective = Eq. 8 with s(u_i,u_j) := R[i].R[j] (minimised);
 * trace_obj = Tr(Y^T R R^T Y) (maximised, Lemma obj3); both FP64. min_margin =
 * smallest top1 - top2 score gap of the last NCI pass (Eq. 21). */
typedef struct {
  double objective;
  double trace_obj;
  double min_margin;
  int32_t last_changes;     /* labels changed by the last NCI pass            */
  int32_t empty_clusters;   /* clusters left empty (Eq. 23 leaves them zero)  */
  int32_t clamped_rows;     /* rows with R'[i].r <= 0 before Eq. 14            */
  int32_t chol_breakdowns;  /* Gram pivots that were not positive             */
  /* device time (CUDA events on `stream`, ms) of: attribute preparation (incl.
   * the Eq. 15 reduction), the propagation of Algorithm 1 (both SpMMs, all
   * gamma rounds, Eq. 2), Q and the random features (Eqs. 13-14), the SVD
   * seeding + NMF (Algorithm 2), NCI generation (Algorithm 3), the objective */
  float ms_phase[6];
  int32_t nci_passes;       /* NCI passes run (t_g unless ABG_NCI_EARLY_STOP)   */
  int32_t reused_propagation; /* 1: Z_hat came from an earlier solve (ABG_REUSE_PROPAGATION) */
  int32_t warm_started;       /* 1: ONMF started from an earlier solve's Phi, H (ABG_WARM_START) */
} abg_result;

ABG_API const char* abg_strerror(int status);
ABG_API const char* abg_last_error(void);
ABG_API void abg_params_default(abg_params* p);   /* k=2, gamma=6, alpha=.6, t_f=5, t_g=20, p=10, q=4 */
/* Number of CUDA kernels this library has launched in the calling process so
 * far (a diagnostic counter; every launch site increments it). */
ABG_API int64_t abg_launch_count(void);
/* Of those, the launches of the tensor-core (tcgen05) product kernel. Dense
 * tall-skinny products run there unless the environment variable
 * ABG_TENSOR_CORES is set to 0 (then on the FP32 SIMT kernels). */
ABG_API int64_t abg_tensor_core_launches(void);
/* SpMM autotuner: product shapes measured so far in this process (the first product of a
 * large enough shape times its kernel variants; the outputs are the same bits whichever
 * variant runs). ABG_AUTOTUNE=0 in the environment turns the measuring off. */
ABG_API int64_t abg_spmm_tuned_shapes(void);

/* ---- graph lifetime ------------------------------------------------------ */

/* Validate and upload one ABG, build its CSC if absent, compute the degree
 * scales D^-1/2 (a zero degree gets 0) and the L_U values of Eq. 7 in both
 * CSR and CSC order. Errors: ABG_EINVAL (malformed CSR/CSC, weights, sizes),
 * ABG_ENOMEM, ABG_EDEVICE. On error *out is NULL. */
ABG_API int abg_create(const abg_graph_desc* desc, void* stream, abg_graph** out);
ABG_API void abg_destroy(abg_graph* g);
ABG_API int64_t abg_graph_footprint(const abg_graph* g);   /* device bytes held */
ABG_API int64_t abg_solve_footprint(const abg_graph* g, const abg_params* p); /* bytes one solve adds */

/* ---- the whole method ---------------------------------------------------- */

/* Algorithms 1-3 end to end on `g`: labels[n_u] (host or device memory) get
 * cluster ids in [0, k); `res` (host, may be NULL) the report. Synchronises
 * `stream`. Errors: ABG_EINVAL (parameters), ABG_ENOMEM, ABG_EDEVICE,
 * ABG_ENUMERIC. */
ABG_API int abg_cluster(abg_graph* g, const abg_params* p, void* stream, int32_t* labels,
                        abg_result* res);

/* ---- many graphs per launch ---------------------------------------------- */

/* Stack n graphs (host descriptors as for abg_create; same d_u and x_kind)
 * into one block-diagonal graph whose n segments are solved together: one
 * launch of each kernel serves every graph, and each graph's arithmetic is
 * independent of the others (fixed-size tiles and chunks per graph), so its
 * result is the same alone and in a batch. Segment s owns rows
 * [sum_{t<s} n_u(t), +n_u(s)) of the stacked U. Free with abg_destroy. */
ABG_API int abg_batch_create(const abg_graph_desc* descs, int32_t n, int32_t device, void* stream,
                             abg_graph** out);
ABG_API int32_t abg_graph_segments(const abg_graph* g);   /* 1 for abg_create graphs */

/* Algorithms 1-3 for every segment: params[n] (k and seed may differ per
 * graph; d, alpha, gamma, t_f, t_g, oversample, power_iters must agree),
 * labels (host or device) for all stacked rows, results[n] (host, may be
 * NULL). Synchronises `stream`. */
ABG_API int abg_batch_cluster(abg_graph* batch, const abg_params* params, void* stream,
                              int32_t* labels, abg_result* results);

/* ---- request loop with continuous batching ------------------------------ */

typedef struct abg_server abg_server;
typedef struct {
  int32_t device;
  int32_t workers;            /* batches in flight at once, one CUDA stream each (default 3) */
  int64_t hbm_budget_bytes;   /* admission: estimated device bytes of requests in flight */
  int32_t max_batch_graphs;   /* requests stacked into one batched launch (default 64) */
  int32_t batch_window_us;    /* a free worker waits this long for more requests (default 0) */
  int64_t max_batch_rows;     /* U rows per batch (default 4M; one larger request runs alone) */
} abg_server_opts;
typedef struct {
  int64_t submitted, completed, failed, rejected, batches, max_batch, pending, inflight_bytes;
  int64_t latency_us_last;    /* submit -> completion of the last polled request */
  int64_t propagations_reused; /* completed requests whose solve reused Z_hat */
} abg_server_stats;

ABG_API void abg_server_opts_default(abg_server_opts* o);
ABG_API int abg_server_create(const abg_server_opts* opts, abg_server** out);
/* Cancels requests not yet started (their poll returns ABG_ECANCELLED), waits for the batches
 * in flight, frees everything. */
ABG_API void abg_server_destroy(abg_server* sv);
/* Queue one request. The graph is validated on the host now; its HOST arrays are read when the
 * request's batch is uploaded, so they must stay valid until abg_poll returns a final status
 * for it. Thread-safe. ABG_ENOTADMITTED if its estimated footprint exceeds the budget (the id
 * is still valid for abg_poll). Requests sharing d_u, x_kind, d, alpha, gamma, t_f, t_g,
 * oversample and power_iters may be batched together; k and seed are per request, and a
 * request's result does not depend on what it was batched with. */
ABG_API int abg_submit(abg_server* sv, const abg_graph_desc* graph, const abg_params* params,
                       uint64_t* req_id);
/* Queue a request against a graph already resident on the server's device (abg_create; not a
 * batch): re-solving with another k, alpha, seed or NCI option skips the upload and creation.
 * The caller keeps g alive until abg_poll returns a final status for the request; several
 * requests may share g (solves only read it). Each such request runs alone; its admission
 * footprint is abg_solve_footprint(g, params). Labels have the graph's clustered-side size. */
ABG_API int abg_submit_resident(abg_server* sv, abg_graph* g, const abg_params* params,
                                uint64_t* req_id);
/* Wait up to timeout_us (0: do not wait; < 0: forever) for a request. ABG_OK: labels (host,
 * one per clustered node) and *res are filled and the id is released; ABG_PENDING (timeout 0) or
 * ABG_ETIMEDOUT: not finished; a negative status: the request failed (the id is released). */
ABG_API int abg_poll(abg_server* sv, uint64_t req_id, int64_t timeout_us, int32_t* labels,
                     abg_result* res);
ABG_API int abg_server_get_stats(abg_server* sv, abg_server_stats* out);

/* ---- individual steps (device buffers owned by the caller) --------------- */

/* Eq. 15 / Section 3.2.1: x_out[n_u][ldo] = Gamma Sigma, the top-d SVD of the
 * graph's X_U (randomized, stream ABG_STREAM_OMEGA_X, each left vector signed
 * so that its entry of largest magnitude is positive, the first one on ties). */
ABG_API int abg_reduce_attributes(const abg_graph* g, int32_t d, int32_t oversample,
                                  int32_t power_iters, uint64_t seed, float* x_out, int64_t ldo,
                                  void* stream);

/* Algorithm 1 propagation (Eq. 6 in the restart form Z_0 = (1-a) X,
 * Z <- (1-a) X + a L (L^T Z), gamma times), then Eq. 2: zhat[n_u][ldz] holds
 * the row-normalised Z_U (a zero row stays zero). x = NULL uses the graph's
 * own dense attributes (d must equal d_u); otherwise x[n_u][ldx] (device,
 * float) is the attribute matrix of width d (e.g. abg_reduce_attributes).
 * Returns once the work on `stream` has finished (it then checks the gather
 * pipeline's bounded waits: ABG_EDEVICE if one ran out). precision is
 * ABG_PRECISION_FP32 or ABG_BF16_PROPAGATION (storage of the intermediate
 * blocks, as in abg_params). */
ABG_API int abg_propagate(const abg_graph* g, const float* x, int64_t ldx, int32_t d,
                          double alpha, int32_t gamma, int32_t precision, float* zhat,
                          int64_t ldz, void* stream);

/* Algorithm 1: q_out[d][d] (device, double) = the orthogonal factor of the QR
 * of G ~ N(0,1)^{d x d} drawn on ABG_STREAM_G, with diag(R_qr) > 0. */
ABG_API int abg_orthogonal_matrix(uint64_t seed, int32_t d, double* q_out, void* stream);

/* Eqs. 13-14: r_out[n][ldr] = R for zhat[n][ldz] (width d) and the orthogonal
 * matrix of abg_orthogonal_matrix(seed, d). clamped (host, may be NULL) gets
 * the number of rows whose R'[i].r was <= 0. */
ABG_API int abg_random_features(const float* zhat, int64_t n, int32_t d, int64_t ldz,
                                uint64_t seed, float* r_out, int64_t ldr, int32_t* clamped,
                                void* stream);

/* Algorithm 2 seeding (Eq. 18): truncated randomized SVD of r[n][m] (stream
 * ABG_STREAM_OMEGA_R), phi_out[n][ldphi] = max(Gamma, 0), h_out[m][ldh] =
 * max(Psi Sigma, 0), sigma_out[k] (device, double, may be NULL). precision:
 * ABG_PRECISION_FP32 or ABG_BF16_CONTRACT (the products with r in BF16, as in
 * abg_params). */
ABG_API int abg_seed_factors(const float* r, int64_t n, int32_t m, int64_t ldr, int32_t k,
                             int32_t oversample, int32_t power_iters, uint64_t seed,
                             float* phi_out, int64_t ldphi, float* h_out, int64_t ldh,
                             double* sigma_out, int32_t precision, void* stream);

/* Algorithm 2 loop: t_f times H by Eq. 16 then Phi by Eq. 17, in place on
 * phi[n][ldphi] and h[m][ldh] (max(numerator, 0); a non-positive denominator
 * sets the entry to 0). precision as for abg_seed_factors. */
ABG_API int abg_onmf(const float* r, int64_t n, int32_t m, int64_t ldr, int32_t k, int32_t t_f,
                     float* phi, int64_t ldphi, float* h, int64_t ldh, int32_t precision,
                     void* stream);

/* Algorithm 3: T = I; t_g times l* = argmax_l Phi[i].T[:, l] (ties -> lowest
 * l), Y by Eqs. 22-23, T <- Phi^T Y (or its Procrustes factor, see
 * nci_flags above). labels_out[n] (device int32), margin_out[n] (device float,
 * may be NULL: top1 - top2 of the last pass), t_out[k][k] (device double, may
 * be NULL: T after the last pass), last_changes and passes (host, may be NULL). */
ABG_API int abg_nci(const float* phi, int64_t n, int32_t k, int64_t ldphi, int32_t t_g,
                    int32_t nci_flags, int32_t* labels_out, float* margin_out, double* t_out,
                    int32_t* last_changes, int32_t* passes, void* stream);

/* Eq. 8 with s := R R^T through per-cluster sums (FP64): obj (host) gets
 * {objective, trace_obj}. labels must lie in [0, k). */
ABG_API int abg_objective(const float* r, int64_t n, int32_t m, int64_t ldr,
                          const int32_t* labels, int32_t k, double* obj, void* stream);

/* ---- allocation-free variant (the paper has no counterpart) -------------- */

/* Same result as abg_objective, for callers that must not allocate device
 * memory while they run (an application that gave all GPU memory to its own
 * allocator, a latency-bound loop that cannot absorb an allocation's device
 * synchronisation, a host runtime that forbids libraries to allocate). It calls
 * no cudaMalloc/cudaFree or allocating routine: its scratch is one fixed 24 MiB
 * __device__ array per GPU, held until exit. With CUDA's lazy module loading
 * (the default) that array is reserved by the first call on a device, which
 * also looks it up (cudaGetSymbolAddress): make that first call before the
 * application hands all device memory to its own allocator, and before any
 * stream capture. Limit: k * (m + 1) <= 48,393 (else ABG_EINVAL with the limit
 * in abg_last_error()). All calls share the array and calls that overlapped on
 * the GPU would race on it; each call therefore holds a process-wide lock until
 * `stream` has synchronised, so calls from several host threads run one after
 * another. Labels outside [0, k) are skipped. obj (host) gets
 * {objective, trace_obj}. */
ABG_API int abg_objective_noalloc(const float* r, int64_t n, int32_t m, int64_t ldr,
                                  const int32_t* labels, int32_t k, double* obj, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* ABG_H */
