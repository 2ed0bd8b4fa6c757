// Graph ingestion (Section 2.1, Eq. 7): validation, upload, CSC construction,
// weighted degrees, the D^-1/2 scales and the L_U values in CSR and CSC order,
// and the row schedules the two SpMMs use. Also the library-wide error text
// and the pooled stream-ordered allocator.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "internal.cuh"
#include "tma.cuh"

namespace abg {

static thread_local char g_err[512] = "";
static std::atomic<long long> g_launches{0};

static std::atomic<long long> g_tc_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

static thread_local int t_test_expiry = 0;
int test_wait_expiry() { return t_test_expiry; }
SolveHooks::SolveHooks() : prev(t_test_expiry) {
  const char* e = std::getenv("ABG_TEST_WAIT_EXPIRY");
  t_test_expiry = (e && std::strcmp(e, "spmm") == 0) ? 1 : 0;
}
SolveHooks::~SolveHooks() { t_test_expiry = prev; }
void note_tc_launch() { g_tc_launches.fetch_add(1, std::memory_order_relaxed); }

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

int cuda_status(cudaError_t e, const char* what) {
  set_error("CUDA error %d (%s) in %s", (int)e, cudaGetErrorString(e), what);
  return e == cudaErrorMemoryAllocation ? ABG_ENOMEM : ABG_EDEVICE;
}

// ---- private memory pool per device -------------------------------------------
static std::mutex g_pool_mu;
static cudaMemPool_t g_pool[64] = {};

static int pool_for_current(cudaMemPool_t* out) {
  int dev = 0;
  ABG_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return ABG_EDEVICE;
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if (!g_pool[dev]) {
    cudaMemPoolProps props;
    memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    ABG_CUDA(cudaMemPoolCreate(&g_pool[dev], &props));
    uint64_t thr = UINT64_MAX;
    ABG_CUDA(cudaMemPoolSetAttribute(g_pool[dev], cudaMemPoolAttrReleaseThreshold, &thr));
  }
  *out = g_pool[dev];
  return ABG_OK;
}

// The dynamic shared-memory limit of a kernel is one setting per context, so
// concurrent callers only ever raise it: a launch that needs b bytes finds a
// limit >= b however other threads interleave.
static std::mutex g_smem_mu;
static std::map<std::pair<const void*, int>, size_t> g_smem_limit;

int raise_smem_limit(const void* func, size_t bytes) {
  if (bytes <= 48 * 1024) return ABG_OK;
  int dev = 0;
  ABG_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_smem_mu);
  size_t& cur = g_smem_limit[{func, dev}];
  if (cur >= bytes) return ABG_OK;
  ABG_CUDA(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  cur = bytes;
  return ABG_OK;
}

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static std::once_flag once;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    else
      cudaGetLastError();
  });
  return fn;
}

int dev_alloc(void** p, size_t bytes, cudaStream_t s) {
  cudaMemPool_t pool;
  ABG_TRY(pool_for_current(&pool));
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMallocFromPoolAsync(p, bytes, pool, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    set_error("device allocation of %zu bytes failed (%s)", bytes, cudaGetErrorString(e));
    *p = nullptr;
    return ABG_ENOMEM;
  }
  return ABG_OK;
}

void dev_free(void* p, cudaStream_t s) {
  if (p) cudaFreeAsync(p, s);
}

int graph_alloc(abg_graph* g, void** p, size_t bytes, cudaStream_t s) {
  if (g->n_blocks >= 64) {
    set_error("internal: too many graph blocks");
    return ABG_ENOMEM;
  }
  ABG_TRY(dev_alloc(p, bytes, s));
  g->blocks[g->n_blocks++] = *p;
  g->footprint += (int64_t)bytes;
  return ABG_OK;
}

// ---- kernels --------------------------------------------------------------------

// Weighted degree of each row (Section 2.1), FP64 sums, one warp per row; then
// the scale D^-1/2 with 0 for a zero degree.
// D^-1/2 of one side: scale[row] = (sum of the row's weights)^-1/2, 0 for an empty row.
// A warp takes 32 consecutive rows: a lane sums its own row when it has at most 32 edges,
// the warp sums the longer ones together (lane-strided FP64 partials, then a shuffle tree);
// the FP64 square roots and divisions then run on all lanes at once.
__global__ void k_row_scale(const int64_t* __restrict__ ptr, const float* __restrict__ w,
                            int64_t rows, float* __restrict__ scale) {
  const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t base = row - (threadIdx.x & 31);
  const int lane = threadIdx.x & 31;
  if (base >= rows) return;  // whole warps
  const bool valid = row < rows;
  const int64_t b = valid ? ptr[row] : 0, e = valid ? ptr[row + 1] : 0;
  const bool light = e - b <= 32;
  // weighted rows with more than kHeavyRow edges are summed over their schedule chunks
  // (k_chunk_wsum, k_heavy_scale), so that a hub is spread over many warps
  const bool split = w && e - b > kHeavyRow;
  double acc = 0.0;
  if (!w) {
    acc = (double)(e - b);
  } else {
    if (light)
      for (int64_t j = b; j < e; ++j) acc += (double)w[j];
    unsigned heavy = __ballot_sync(0xffffffffu, valid && !light && !split);
    while (heavy) {
      const int i = __ffs(heavy) - 1;
      heavy &= heavy - 1;
      const int64_t hb = __shfl_sync(0xffffffffu, b, i), he = __shfl_sync(0xffffffffu, e, i);
      double part = 0.0;
      for (int64_t j = hb + lane; j < he; j += 32) part += (double)w[j];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
      if (lane == i) acc = part;
    }
  }
  if (valid && !split) scale[row] = acc > 0.0 ? (float)(1.0 / sqrt(acc)) : 0.0f;
}

// The rows that k_row_scale leaves (weighted, more than kHeavyRow edges): one warp per
// schedule chunk sums its weights (lanes over the chunk, then a shuffle tree) ...
__global__ void k_chunk_wsum(const int64_t* __restrict__ ptr, const float* __restrict__ w,
                             abg_graph::Schedule sc, double* __restrict__ part) {
  const int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (c >= sc.n_chunks) return;  // whole warps
  const int64_t b = sc.chunk_begin[c];
  const int row = sc.heavy_row[sc.chunk_row_slot[c]];
  const int64_t e = min(b + (int64_t)kHeavyChunk, ptr[row + 1]);
  double acc = 0.0;
  for (int64_t j = b + lane; j < e; j += 32) acc += (double)w[j];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) part[c] = acc;
}

// ... and one thread per such row adds its chunks' sums in chunk order
__global__ void k_heavy_scale(abg_graph::Schedule sc, const double* __restrict__ part,
                              float* __restrict__ scale) {
  const int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= sc.n_heavy) return;
  double acc = 0.0;
  for (int64_t c = sc.heavy_chunk0[h]; c < sc.heavy_chunk0[h + 1]; ++c) acc += part[c];
  scale[sc.heavy_row[h]] = acc > 0.0 ? (float)(1.0 / sqrt(acc)) : 0.0f;
}

// L values (Eq. 7) of one storage order: val[e] = w[e] * s_row[row] * s_col[col[e]]. A warp
// takes 32 consecutive rows and walks them one after another, its lanes striding over each
// row's edges (consecutive edges on consecutive lanes).
constexpr int kLvWarps = 8;

__global__ void __launch_bounds__(32 * kLvWarps) k_l_values(
    const int64_t* __restrict__ ptr, const int32_t* __restrict__ col,
    const float* __restrict__ w, int64_t rows, const float* __restrict__ s_row,
    const float* __restrict__ s_col, float* __restrict__ val) {
  __shared__ int64_t start[kLvWarps][33];
  __shared__ double srow[kLvWarps][32];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t r0 = ((int64_t)blockIdx.x * kLvWarps + wid) * 32;
  if (r0 >= rows) return;  // whole warps
  const int nr = rows - r0 < 32 ? (int)(rows - r0) : 32;
  start[wid][lane] = ptr[r0 + min(lane, nr)];
  if (lane == 0) start[wid][32] = ptr[r0 + nr];
  srow[wid][lane] = lane < nr ? (double)s_row[r0 + lane] : 0.0;
  __syncwarp();
  for (int i = 0; i < nr; ++i) {
    const int64_t e = start[wid][i + 1];
    if (e - start[wid][i] > kHeavyRow) continue;  // its schedule chunks (k_l_values_chunks)
    const double sr = srow[wid][i];
    for (int64_t j = start[wid][i] + lane; j < e; j += 32) {
      const double wj = w ? (double)w[j] : 1.0;
      val[j] = (float)(wj * sr * (double)s_col[col[j]]);
    }
  }
}

// L values of the rows with more than kHeavyRow edges: one warp per schedule chunk
__global__ void k_l_values_chunks(const int64_t* __restrict__ ptr, const int32_t* __restrict__ col,
                                  const float* __restrict__ w, abg_graph::Schedule sc,
                                  const float* __restrict__ s_row,
                                  const float* __restrict__ s_col, float* __restrict__ val) {
  const int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (c >= sc.n_chunks) return;  // whole warps
  const int64_t b = sc.chunk_begin[c];
  const int row = sc.heavy_row[sc.chunk_row_slot[c]];
  const int64_t e = min(b + (int64_t)kHeavyChunk, ptr[row + 1]);
  const double sr = (double)s_row[row];
  for (int64_t j = b + lane; j < e; j += 32) {
    const double wj = w ? (double)w[j] : 1.0;
    val[j] = (float)(wj * sr * (double)s_col[col[j]]);
  }
}

// First out-of-range index (first[0]) and first weight that is not finite and positive
// (first[1]) of an edge array; both stay at nnz when there is none.
__global__ void k_check_edges(const int32_t* __restrict__ idx, const float* __restrict__ w,
                              int64_t nnz, int64_t cols, unsigned long long* __restrict__ first) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nnz;
       j += (int64_t)gridDim.x * blockDim.x) {
    if (idx[j] < 0 || idx[j] >= cols) atomicMin(first, (unsigned long long)j);
    if (w && !(isfinite(w[j]) && w[j] > 0.f)) atomicMin(first + 1, (unsigned long long)j);
  }
}

// Column counts of the CSR (to verify a caller-given CSC).
__global__ void k_col_count(const int32_t* __restrict__ col, int64_t nnz, int* __restrict__ cnt) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nnz;
       j += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&cnt[col[j]], 1);
}

__global__ void k_count_mismatch(const int64_t* __restrict__ ptr, const int* __restrict__ cnt,
                                 int64_t rows, int* __restrict__ bad) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < rows;
       r += (int64_t)gridDim.x * blockDim.x)
    if ((int64_t)cnt[r] != ptr[r + 1] - ptr[r]) atomicAdd(bad, 1);
}

}  // namespace abg

using namespace abg;

// ---- host helpers -----------------------------------------------------------------

// First position in [0, n) where bad(i) holds (n if none), scanned by several host threads.
template <class F>
static int64_t first_bad(int64_t n, F bad) {
  const int64_t kMinPerThread = int64_t(1) << 20;
  const int nt = (int)std::max<int64_t>(
      1, std::min<int64_t>({(int64_t)std::max(1u, std::thread::hardware_concurrency()), 32,
                            n / kMinPerThread}));
  if (nt == 1) {
    for (int64_t i = 0; i < n; ++i)
      if (bad(i)) return i;
    return n;
  }
  std::vector<int64_t> found(nt, n);
  std::vector<std::thread> th;
  for (int t = 0; t < nt; ++t)
    th.emplace_back([&, t] {
      const int64_t b = n * t / nt, e = n * (t + 1) / nt;
      for (int64_t i = b; i < e; ++i)
        if (bad(i)) {
          found[t] = i;
          return;
        }
    });
  for (auto& x : th) x.join();
  return *std::min_element(found.begin(), found.end());
}

static int validate_csr(const int64_t* ptr, const int32_t* idx, const float* w, int64_t rows,
                        int64_t cols, int64_t nnz, const char* name) {
  ABG_CHECK(ptr && idx, "%s: null CSR arrays", name);
  ABG_CHECK(ptr[0] == 0 && ptr[rows] == nnz, "%s: ptr[0] must be 0 and ptr[rows] = nnz", name);
  const int64_t r = first_bad(rows, [&](int64_t i) { return ptr[i + 1] < ptr[i]; });
  ABG_CHECK(r == rows, "%s: ptr not monotone at row %lld", name, (long long)r);
  const int64_t j = first_bad(nnz, [&](int64_t i) { return idx[i] < 0 || idx[i] >= cols; });
  ABG_CHECK(j == nnz, "%s: index %d out of range at %lld", name, j < nnz ? idx[j] : 0,
            (long long)j);
  if (w) {
    const int64_t q = first_bad(nnz, [&](int64_t i) { return !(std::isfinite(w[i]) && w[i] > 0.f); });
    ABG_CHECK(q == nnz, "%s: weight %g at %lld not finite/positive", name,
              q < nnz ? (double)w[q] : 0.0, (long long)q);
  }
  return ABG_OK;
}

// The row-pointer half of validate_csr (host); the index and weight half runs on the device
// (k_check_edges) once the arrays are uploaded.
static int validate_ptr(const int64_t* ptr, const int32_t* idx, int64_t rows, int64_t nnz,
                        const char* name) {
  ABG_CHECK(ptr && idx, "%s: null CSR arrays", name);
  ABG_CHECK(ptr[0] == 0 && ptr[rows] == nnz, "%s: ptr[0] must be 0 and ptr[rows] = nnz", name);
  const int64_t r = first_bad(rows, [&](int64_t i) { return ptr[i + 1] < ptr[i]; });
  ABG_CHECK(r == rows, "%s: ptr not monotone at row %lld", name, (long long)r);
  return ABG_OK;
}

// Stable counting sort CSR -> CSC (deterministic edge order inside each column:
// increasing row), parallel over row ranges with per-thread column offsets.
static void build_csc(int64_t n_u, int64_t n_v, int64_t nnz, const int64_t* u_ptr,
                      const int32_t* v_idx, const float* w, std::vector<int64_t>& v_ptr,
                      std::vector<int32_t>& u_idx, std::vector<float>& w_t) {
  v_ptr.assign(n_v + 1, 0);
  u_idx.resize(nnz);
  if (w) w_t.resize(nnz);
  for (int64_t j = 0; j < nnz; ++j) v_ptr[v_idx[j] + 1]++;
  for (int64_t c = 0; c < n_v; ++c) v_ptr[c + 1] += v_ptr[c];
  std::vector<int64_t> cur(v_ptr.begin(), v_ptr.end() - 1);
  for (int64_t r = 0; r < n_u; ++r)
    for (int64_t j = u_ptr[r]; j < u_ptr[r + 1]; ++j) {
      int64_t p = cur[v_idx[j]]++;
      u_idx[p] = (int32_t)r;
      if (w) w_t[p] = w[j];
    }
}

int abg::swap_sides(const abg_graph_desc* in, abg::SideSwap* store, const abg_graph_desc** out) {
  *out = in;
  ABG_CHECK(in, "null descriptor");
  ABG_CHECK(in->side == ABG_SIDE_U || in->side == ABG_SIDE_V, "side must be ABG_SIDE_U or _V");
  if (in->side == ABG_SIDE_U) return ABG_OK;
  // clustering V: the same edges with the roles exchanged (the CSC becomes the CSR)
  ABG_CHECK(in->n_u >= 1 && in->n_v >= 1 && in->n_u < (1ll << 31) && in->n_v < (1ll << 31),
            "need 1 <= |U|, |V| < 2^31");
  ABG_CHECK(in->nnz >= 0, "nnz < 0");
  ABG_TRY(validate_csr(in->u_ptr, in->v_idx, in->w, in->n_u, in->n_v, in->nnz, "CSR"));
  abg_graph_desc& d = store->desc;
  d = *in;
  if (in->v_ptr || in->u_idx || in->w_t) {
    ABG_CHECK(in->v_ptr && in->u_idx && (!in->w == !in->w_t),
              "CSC needs v_ptr, u_idx and (w_t iff w)");
  } else {
    build_csc(in->n_u, in->n_v, in->nnz, in->u_ptr, in->v_idx, in->w, store->vp, store->ui,
              store->wt);
    d.v_ptr = store->vp.data();
    d.u_idx = store->ui.data();
    d.w_t = in->w ? store->wt.data() : nullptr;
  }
  const int64_t* vp = d.v_ptr;
  const int32_t* ui = d.u_idx;
  const float* wt = d.w_t;
  d.n_u = in->n_v;
  d.n_v = in->n_u;
  d.u_ptr = vp;
  d.v_idx = ui;
  d.w = wt;
  d.v_ptr = in->u_ptr;
  d.u_idx = in->v_idx;
  d.w_t = in->w;
  d.side = ABG_SIDE_U;
  *out = &d;
  return ABG_OK;
}

// Row schedule of one SpMM direction: light rows grouped into tasks of at most
// kTaskRows consecutive rows and about kTaskEdges edges (a task never spans a
// heavy row), heavy rows cut into kHeavyChunk-edge chunks.
// Host half of a row schedule: the task and chunk lists (computed from the host row pointers
// only, so it can run while the arrays upload).
struct SchedHost {
  std::vector<int32_t> tasks, et, zt;  // (first row, one past the last row) pairs
  std::vector<int64_t> cb;             // chunk starts
  std::vector<int32_t> cslot;          // heavy slot of each chunk
  std::vector<int32_t> hrow;           // heavy rows
  std::vector<int64_t> hc0;            // first chunk of each heavy row (n_heavy + 1)
};

static void compute_schedule(const int64_t* ptr, int64_t rows, SchedHost& H) {
  // row ranges scanned by several host threads; a task never crosses a range boundary, and
  // results do not depend on task boundaries (every row sums its edges in edge order)
  struct Part {
    std::vector<int32_t> tasks;  // (first row, one past the last row) of each light task
    std::vector<int64_t> cb;     // chunk starts
    std::vector<int32_t> cslot;  // heavy slot (local) of each chunk
    std::vector<int32_t> hrow;   // heavy rows
    std::vector<int64_t> hc0;    // first chunk (local) of each heavy row
  };
  const int64_t kMinRows = int64_t(1) << 18;
  const int nt = (int)std::max<int64_t>(
      1, std::min<int64_t>({(int64_t)std::max(1u, std::thread::hardware_concurrency()), 16,
                            rows / kMinRows}));
  std::vector<Part> parts(nt);
  auto scan = [&](int t) {
    Part& P = parts[t];
    const int64_t rb = rows * t / nt, re = rows * (t + 1) / nt;
    int64_t t_r0 = -1, t_edges = 0;
    auto close_task = [&](int64_t r_end) {
      if (t_r0 >= 0) {
        P.tasks.push_back((int32_t)t_r0);
        P.tasks.push_back((int32_t)r_end);
      }
      t_r0 = -1;
      t_edges = 0;
    };
    for (int64_t r = rb; r < re; ++r) {
      const int64_t deg = ptr[r + 1] - ptr[r];
      if (deg > kHeavyRow) {
        close_task(r);
        P.hc0.push_back((int64_t)P.cb.size());
        const int32_t slot = (int32_t)P.hrow.size();
        P.hrow.push_back((int32_t)r);
        for (int64_t e = ptr[r]; e < ptr[r + 1]; e += kHeavyChunk) {
          P.cb.push_back(e);
          P.cslot.push_back(slot);
        }
        continue;
      }
      if (t_r0 >= 0 && (r - t_r0 >= kTaskRows || t_edges + deg > kTaskEdges)) close_task(r);
      if (t_r0 < 0) t_r0 = r;
      t_edges += deg;
    }
    close_task(re);
  };
  if (nt == 1) {
    scan(0);
  } else {
    std::vector<std::thread> th;
    for (int t = 0; t < nt; ++t) th.emplace_back(scan, t);
    for (auto& x : th) x.join();
  }
  std::vector<int32_t>& tasks = H.tasks;
  std::vector<int64_t>& cb = H.cb;
  std::vector<int32_t>& cslot = H.cslot;
  std::vector<int32_t>& hrow = H.hrow;
  std::vector<int64_t>& hc0 = H.hc0;
  for (const Part& P : parts) {
    const int32_t slot0 = (int32_t)hrow.size();
    const int64_t chunk0 = (int64_t)cb.size();
    tasks.insert(tasks.end(), P.tasks.begin(), P.tasks.end());
    cb.insert(cb.end(), P.cb.begin(), P.cb.end());
    for (int32_t x : P.cslot) cslot.push_back(x + slot0);
    hrow.insert(hrow.end(), P.hrow.begin(), P.hrow.end());
    for (int64_t x : P.hc0) hc0.push_back(x + chunk0);
  }
  hc0.push_back((int64_t)cb.size());
  // the same tasks split by whether they hold edges (the TMA-gather kernel takes those that do)
  std::vector<int32_t>& et = H.et;
  std::vector<int32_t>& zt = H.zt;
  for (size_t i = 0; i < tasks.size(); i += 2) {
    auto& dst = ptr[tasks[i + 1]] > ptr[tasks[i]] ? et : zt;
    dst.push_back(tasks[i]);
    dst.push_back(tasks[i + 1]);
  }
}

// Device half: the lists of H into sc (H must stay alive until the copies have run).
static int upload_schedule(abg_graph* g, const SchedHost& H, abg_graph::Schedule& sc,
                           cudaStream_t s) {
  const std::vector<int32_t>& tasks = H.tasks;
  const std::vector<int32_t>& et = H.et;
  const std::vector<int32_t>& zt = H.zt;
  const std::vector<int64_t>& cb = H.cb;
  const std::vector<int32_t>& cslot = H.cslot;
  const std::vector<int32_t>& hrow = H.hrow;
  const std::vector<int64_t>& hc0 = H.hc0;
  sc.n_tasks = (int64_t)tasks.size() / 2;
  sc.n_etasks = (int64_t)et.size() / 2;
  sc.n_ztasks = (int64_t)zt.size() / 2;
  sc.n_chunks = (int64_t)cb.size();
  sc.n_heavy = (int64_t)hrow.size();
  void* p;
  ABG_TRY(graph_alloc(g, &p, sizeof(int32_t) * 2 * std::max<int64_t>(1, sc.n_tasks), s));
  sc.tasks = (int2*)p;
  ABG_TRY(graph_alloc(g, &p, sizeof(int32_t) * 2 * std::max<int64_t>(1, sc.n_etasks), s));
  sc.etasks = (int2*)p;
  ABG_TRY(graph_alloc(g, &p, sizeof(int32_t) * 2 * std::max<int64_t>(1, sc.n_ztasks), s));
  sc.ztasks = (int2*)p;
  ABG_TRY(graph_alloc(g, &p, sizeof(int64_t) * std::max<int64_t>(1, sc.n_chunks), s));
  sc.chunk_begin = (int64_t*)p;
  ABG_TRY(graph_alloc(g, &p, sizeof(int32_t) * std::max<int64_t>(1, sc.n_chunks), s));
  sc.chunk_row_slot = (int32_t*)p;
  ABG_TRY(graph_alloc(g, &p, sizeof(int32_t) * std::max<int64_t>(1, sc.n_heavy), s));
  sc.heavy_row = (int32_t*)p;
  ABG_TRY(graph_alloc(g, &p, sizeof(int64_t) * (sc.n_heavy + 1), s));
  sc.heavy_chunk0 = (int64_t*)p;
  if (sc.n_tasks)
    ABG_CUDA(cudaMemcpyAsync(sc.tasks, tasks.data(), sizeof(int32_t) * 2 * sc.n_tasks,
                             cudaMemcpyHostToDevice, s));
  if (sc.n_etasks)
    ABG_CUDA(cudaMemcpyAsync(sc.etasks, et.data(), sizeof(int32_t) * 2 * sc.n_etasks,
                             cudaMemcpyHostToDevice, s));
  if (sc.n_ztasks)
    ABG_CUDA(cudaMemcpyAsync(sc.ztasks, zt.data(), sizeof(int32_t) * 2 * sc.n_ztasks,
                             cudaMemcpyHostToDevice, s));
  if (sc.n_chunks) {
    ABG_CUDA(cudaMemcpyAsync(sc.chunk_begin, cb.data(), sizeof(int64_t) * sc.n_chunks,
                             cudaMemcpyHostToDevice, s));
    ABG_CUDA(cudaMemcpyAsync(sc.chunk_row_slot, cslot.data(), sizeof(int32_t) * sc.n_chunks,
                             cudaMemcpyHostToDevice, s));
    ABG_CUDA(cudaMemcpyAsync(sc.heavy_row, hrow.data(), sizeof(int32_t) * sc.n_heavy,
                             cudaMemcpyHostToDevice, s));
  }
  ABG_CUDA(cudaMemcpyAsync(sc.heavy_chunk0, hc0.data(), sizeof(int64_t) * (sc.n_heavy + 1),
                           cudaMemcpyHostToDevice, s));
  return ABG_OK;
}

template <class T>
static int upload(abg_graph* g, T** dst, const T* src, int64_t count, cudaStream_t s) {
  void* p;
  ABG_TRY(graph_alloc(g, &p, sizeof(T) * std::max<int64_t>(1, count), s));
  *dst = (T*)p;
  if (count) ABG_CUDA(cudaMemcpyAsync(p, src, sizeof(T) * count, cudaMemcpyHostToDevice, s));
  return ABG_OK;
}

// Transposed CSR of X per segment (row s*d_u + j lists the rows of segment s with column j,
// in increasing row order) and the stacked column ids s*d_u + j of the row-major CSR.
static void build_segment_transpose(const abg_graph* g, int64_t d_u, const int64_t* x_ptr,
                                    const int32_t* x_idx, const float* x_val,
                                    std::vector<int64_t>& tp, std::vector<int32_t>& ti,
                                    std::vector<float>& tv, std::vector<int32_t>& xr) {
  const int64_t rows_t = (int64_t)g->nseg * d_u;
  const int64_t nnz = x_ptr[g->n_u];
  tp.assign(rows_t + 1, 0);
  ti.resize(nnz);
  tv.resize(nnz);
  xr.resize(nnz);
  for (int sg = 0; sg < g->nseg; ++sg)
    for (int64_t r = g->seg_row0[sg]; r < g->seg_row0[sg] + g->seg_n[sg]; ++r)
      for (int64_t j = x_ptr[r]; j < x_ptr[r + 1]; ++j) {
        const int64_t c = (int64_t)sg * d_u + x_idx[j];
        xr[j] = (int32_t)c;
        tp[c + 1]++;
      }
  for (int64_t c = 0; c < rows_t; ++c) tp[c + 1] += tp[c];
  std::vector<int64_t> cur(tp.begin(), tp.end() - 1);
  for (int64_t r = 0; r < g->n_u; ++r)
    for (int64_t j = x_ptr[r]; j < x_ptr[r + 1]; ++j) {
      const int64_t p = cur[xr[j]]++;
      ti[p] = (int32_t)r;
      tv[p] = x_val[j];
    }
}

namespace abg {
int validate_desc(const abg_graph_desc* d) {
  ABG_CHECK(d, "null descriptor");
  ABG_CHECK(d->n_u >= 1 && d->n_v >= 1 && d->n_u < (1ll << 31) && d->n_v < (1ll << 31),
            "need 1 <= |U|, |V| < 2^31");
  ABG_CHECK(d->nnz >= 0, "nnz < 0");
  ABG_CHECK(d->d_u >= 1 && d->d_u <= 65536, "need 1 <= d_u <= 65536");
  ABG_CHECK(d->x_kind >= ABG_X_DENSE_F32 && d->x_kind <= ABG_X_CSR_F32, "bad x_kind");
  ABG_TRY(validate_csr(d->u_ptr, d->v_idx, d->w, d->n_u, d->n_v, d->nnz, "CSR"));
  if (d->x_kind == ABG_X_CSR_F32) {
    ABG_TRY(validate_csr(d->x_ptr, d->x_idx, nullptr, d->n_u, d->d_u,
                         d->x_ptr ? d->x_ptr[d->n_u] : 0, "X CSR"));
    ABG_CHECK(d->x_val, "X CSR: null values");
  } else {
    ABG_CHECK(d->x, "dense attributes: null x");
  }
  return ABG_OK;
}
}  // namespace abg

static int create_impl(const abg_graph_desc* d, cudaStream_t s, abg_graph* g) {
  ABG_CHECK(d, "null descriptor");
  ABG_CHECK(d->n_u >= 1 && d->n_v >= 1 && d->n_u < (1ll << 31) && d->n_v < (1ll << 31),
            "need 1 <= |U|, |V| < 2^31");
  ABG_CHECK(d->nnz >= 0, "nnz < 0");
  ABG_CHECK(d->d_u >= 1 && d->d_u <= 65536, "need 1 <= d_u <= 65536");
  ABG_CHECK(d->x_kind >= ABG_X_DENSE_F32 && d->x_kind <= ABG_X_CSR_F32, "bad x_kind");
  g->device = d->device;
  if (g->seg_row0.empty()) {
    g->nseg = 1;
    g->seg_row0 = {0};
    g->seg_n = {d->n_u};
  }
  g->n_u = d->n_u;
  g->n_v = d->n_v;
  g->nnz = d->nnz;
  g->d_u = d->d_u;
  g->x_kind = d->x_kind;
  const bool have_csc = d->v_ptr || d->u_idx || d->w_t;
  // with a caller-given CSC the edge arrays are checked on the device after the upload (before
  // any kernel indexes with them); building the CSC here needs them checked first
  if (have_csc)
    ABG_TRY(validate_ptr(d->u_ptr, d->v_idx, d->n_u, d->nnz, "CSR"));
  else
    ABG_TRY(validate_csr(d->u_ptr, d->v_idx, d->w, d->n_u, d->n_v, d->nnz, "CSR"));
  std::vector<int64_t> vp;
  std::vector<int32_t> ui;
  std::vector<float> wt;
  const int64_t* v_ptr = d->v_ptr;
  const int32_t* u_idx = d->u_idx;
  const float* w_t = d->w_t;
  if (have_csc) {
    ABG_CHECK(d->v_ptr && d->u_idx && (!d->w == !d->w_t),
              "CSC needs v_ptr, u_idx and (w_t iff w)");
    ABG_TRY(validate_ptr(d->v_ptr, d->u_idx, d->n_v, d->nnz, "CSC"));
  } else {
    build_csc(d->n_u, d->n_v, d->nnz, d->u_ptr, d->v_idx, d->w, vp, ui, wt);
    v_ptr = vp.data();
    u_idx = ui.data();
    w_t = d->w ? wt.data() : nullptr;
  }
  // the row schedules need only the host row pointers: computed while the arrays upload
  SchedHost sh_u, sh_v;
  std::thread sched_thread([&] {
    compute_schedule(d->u_ptr, d->n_u, sh_u);
    compute_schedule(v_ptr, d->n_v, sh_v);
  });
  struct Joiner {
    std::thread& t;
    ~Joiner() {
      if (t.joinable()) t.join();
    }
  } joiner{sched_thread};
  // attributes
  if (d->x_kind == ABG_X_CSR_F32) {
    ABG_TRY(validate_csr(d->x_ptr, d->x_idx, nullptr, d->n_u, d->d_u, d->x_ptr ? d->x_ptr[d->n_u] : 0,
                         "X CSR"));
    ABG_CHECK(d->x_val, "X CSR: null values");
    g->x_nnz = d->x_ptr[d->n_u];
    const int64_t j = first_bad(g->x_nnz, [&](int64_t i) { return !std::isfinite(d->x_val[i]); });
    ABG_CHECK(j == g->x_nnz, "X CSR: non-finite value at %lld", (long long)j);
  } else {
    ABG_CHECK(d->x, "dense attributes: null x");
  }

  // ---- upload + device work (all validation above is host-only) ----
  ABG_CUDA(cudaSetDevice(d->device));
  ABG_TRY(upload(g, &g->u_ptr, d->u_ptr, d->n_u + 1, s));
  ABG_TRY(upload(g, &g->u_col, d->v_idx, d->nnz, s));
  ABG_TRY(upload(g, &g->v_ptr, v_ptr, d->n_v + 1, s));
  ABG_TRY(upload(g, &g->v_col, u_idx, d->nnz, s));
  float *w_dev = nullptr, *wt_dev = nullptr;
  Scratch scr(s);
  if (d->w) {
    ABG_TRY(scr.get(&w_dev, d->nnz));
    ABG_TRY(scr.get(&wt_dev, d->nnz));
    ABG_CUDA(cudaMemcpyAsync(w_dev, d->w, sizeof(float) * d->nnz, cudaMemcpyHostToDevice, s));
    ABG_CUDA(cudaMemcpyAsync(wt_dev, w_t, sizeof(float) * d->nnz, cudaMemcpyHostToDevice, s));
  }
  if (have_csc && d->nnz) {  // indices in range and weights finite and positive, both orders
    unsigned long long* first;
    ABG_TRY(scr.get(&first, 4));
    const unsigned long long init[4] = {(unsigned long long)d->nnz, (unsigned long long)d->nnz,
                                        (unsigned long long)d->nnz, (unsigned long long)d->nnz};
    ABG_CUDA(cudaMemcpyAsync(first, init, sizeof(init), cudaMemcpyHostToDevice, s));
    const unsigned grid = (unsigned)std::min<int64_t>(ceil_div(d->nnz, 256), num_sms() * 8);
    k_check_edges<<<grid, 256, 0, s>>>(g->u_col, w_dev, d->nnz, d->n_v, first);
    ::abg::note_launch();
    k_check_edges<<<grid, 256, 0, s>>>(g->v_col, wt_dev, d->nnz, d->n_u, first + 2);
    ::abg::note_launch();
    ABG_LAUNCH_CHECK();
    unsigned long long hf[4];
    ABG_CUDA(cudaMemcpyAsync(hf, first, sizeof(hf), cudaMemcpyDeviceToHost, s));
    ABG_CUDA(cudaStreamSynchronize(s));
    const int64_t nz = d->nnz;
    ABG_CHECK((int64_t)hf[0] == nz, "CSR: index %d out of range at %lld", d->v_idx[hf[0]],
              (long long)hf[0]);
    ABG_CHECK((int64_t)hf[1] == nz, "CSR: weight %g at %lld not finite/positive",
              (double)d->w[hf[1]], (long long)hf[1]);
    ABG_CHECK((int64_t)hf[2] == nz, "CSC: index %d out of range at %lld", d->u_idx[hf[2]],
              (long long)hf[2]);
    ABG_CHECK((int64_t)hf[3] == nz, "CSC: weight %g at %lld not finite/positive",
              (double)d->w_t[hf[3]], (long long)hf[3]);
  }
  void* p;
  ABG_TRY(graph_alloc(g, &p, sizeof(float) * std::max<int64_t>(1, d->nnz), s));
  g->u_val = (float*)p;
  ABG_TRY(graph_alloc(g, &p, sizeof(float) * std::max<int64_t>(1, d->nnz), s));
  g->v_val = (float*)p;
  ABG_TRY(graph_alloc(g, &p, sizeof(float) * d->n_u, s));
  g->su = (float*)p;
  ABG_TRY(graph_alloc(g, &p, sizeof(float) * d->n_v, s));
  g->sv = (float*)p;
  if (have_csc) {  // the CSC must hold the CSR's edges: equal per-column counts
    int *cnt, *bad;
    ABG_TRY(scr.get(&cnt, d->n_v));
    ABG_TRY(scr.get(&bad, 1));
    ABG_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int) * d->n_v, s));
    ABG_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
    if (d->nnz) { k_col_count<<<num_sms() * 8, 256, 0, s>>>(g->u_col, d->nnz, cnt); ::abg::note_launch(); }
    k_count_mismatch<<<num_sms() * 4, 256, 0, s>>>(g->v_ptr, cnt, d->n_v, bad); ::abg::note_launch();
    ABG_LAUNCH_CHECK();
    int hbad = 0;
    ABG_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    ABG_CUDA(cudaStreamSynchronize(s));
    ABG_CHECK(hbad == 0, "CSC does not match the CSR (%d columns differ)", hbad);
  }
  // row schedules first: their chunks of the rows with more than kHeavyRow edges spread those
  // rows over many warps in the scales and L values below
  sched_thread.join();
  ABG_TRY(upload_schedule(g, sh_u, g->sched_u, s));
  ABG_TRY(upload_schedule(g, sh_v, g->sched_v, s));
  k_row_scale<<<ceil_div(d->n_u, 256), 256, 0, s>>>(g->u_ptr, w_dev, d->n_u, g->su); ::abg::note_launch();
  k_row_scale<<<ceil_div(d->n_v, 256), 256, 0, s>>>(g->v_ptr, wt_dev, d->n_v, g->sv); ::abg::note_launch();
  if (d->w) {
    double* part;
    ABG_TRY(scr.get(&part, (size_t)std::max<int64_t>(
                               1, std::max(g->sched_u.n_chunks, g->sched_v.n_chunks))));
    const struct {
      const int64_t* ptr;
      const float* w;
      const abg_graph::Schedule* sc;
      float* scale;
    } sides[2] = {{g->u_ptr, w_dev, &g->sched_u, g->su}, {g->v_ptr, wt_dev, &g->sched_v, g->sv}};
    for (const auto& sd : sides) {
      if (sd.sc->n_chunks == 0) continue;
      k_chunk_wsum<<<(unsigned)ceil_div(sd.sc->n_chunks, 8), 256, 0, s>>>(sd.ptr, sd.w, *sd.sc,
                                                                          part);
      ::abg::note_launch();
      k_heavy_scale<<<(unsigned)ceil_div(sd.sc->n_heavy, 256), 256, 0, s>>>(*sd.sc, part,
                                                                            sd.scale);
      ::abg::note_launch();
    }
  }
  k_l_values<<<ceil_div(d->n_u, 32 * kLvWarps), 32 * kLvWarps, 0, s>>>(
      g->u_ptr, g->u_col, w_dev, d->n_u, g->su, g->sv, g->u_val); ::abg::note_launch();
  k_l_values<<<ceil_div(d->n_v, 32 * kLvWarps), 32 * kLvWarps, 0, s>>>(
      g->v_ptr, g->v_col, wt_dev, d->n_v, g->sv, g->su, g->v_val); ::abg::note_launch();
  if (g->sched_u.n_chunks) {
    k_l_values_chunks<<<(unsigned)ceil_div(g->sched_u.n_chunks, 8), 256, 0, s>>>(
        g->u_ptr, g->u_col, w_dev, g->sched_u, g->su, g->sv, g->u_val);
    ::abg::note_launch();
  }
  if (g->sched_v.n_chunks) {
    k_l_values_chunks<<<(unsigned)ceil_div(g->sched_v.n_chunks, 8), 256, 0, s>>>(
        g->v_ptr, g->v_col, wt_dev, g->sched_v, g->sv, g->su, g->v_val);
    ::abg::note_launch();
  }
  ABG_LAUNCH_CHECK();

  // attributes on the device
  if (d->x_kind == ABG_X_DENSE_F32 || d->x_kind == ABG_X_DENSE_BF16) {
    const int esz = d->x_kind == ABG_X_DENSE_F32 ? 4 : 2;
    g->ldx = round_up(d->d_u, 8);
    ABG_TRY(graph_alloc(g, &p, (size_t)esz * g->ldx * d->n_u, s));
    g->x = p;
    ABG_CUDA(cudaMemcpy2DAsync(p, (size_t)esz * g->ldx, d->x, (size_t)esz * d->d_u,
                               (size_t)esz * d->d_u, d->n_u, cudaMemcpyHostToDevice, s));
    if (g->ldx != d->d_u)
      ABG_CUDA(cudaMemset2DAsync((char*)p + (size_t)esz * d->d_u, (size_t)esz * g->ldx, 0,
                                 (size_t)esz * (g->ldx - d->d_u), d->n_u, s));
  } else {
    ABG_TRY(upload(g, &g->x_ptr, d->x_ptr, d->n_u + 1, s));
    ABG_TRY(upload(g, &g->x_col, d->x_idx, g->x_nnz, s));
    ABG_TRY(upload(g, &g->x_val, d->x_val, g->x_nnz, s));
    std::vector<int64_t> tp;
    std::vector<int32_t> ti;
    std::vector<float> tv;
    std::vector<int32_t> xr;
    build_segment_transpose(g, d->d_u, d->x_ptr, d->x_idx, d->x_val, tp, ti, tv, xr);
    ABG_TRY(upload(g, &g->xt_ptr, tp.data(), (int64_t)g->nseg * d->d_u + 1, s));
    ABG_TRY(upload(g, &g->xt_col, ti.data(), g->x_nnz, s));
    ABG_TRY(upload(g, &g->xt_val, tv.data(), g->x_nnz, s));
    if (g->nseg == 1)
      g->xr_col = g->x_col;
    else
      ABG_TRY(upload(g, &g->xr_col, xr.data(), g->x_nnz, s));
    ABG_CUDA(cudaStreamSynchronize(s));  // host vectors go out of scope
  }
  {
    void* p;
    ABG_TRY(graph_alloc(g, &p, sizeof(int), s));
    g->wait_err = (int*)p;
    ABG_CUDA(cudaMemsetAsync(g->wait_err, 0, sizeof(int), s));
  }
  ABG_CUDA(cudaStreamSynchronize(s));
  return ABG_OK;
}

extern "C" {

ABG_API const char* abg_strerror(int st) {
  switch (st) {
    case ABG_OK: return "ok";
    case ABG_PENDING: return "pending";
    case ABG_EINVAL: return "invalid argument";
    case ABG_ENOMEM: return "out of device memory";
    case ABG_EDEVICE: return "CUDA device error";
    case ABG_ENOTADMITTED: return "job does not fit the server's memory budget";
    case ABG_ETIMEDOUT: return "timed out";
    case ABG_ENOTFOUND: return "unknown request";
    case ABG_ECANCELLED: return "cancelled";
    case ABG_ENUMERIC: return "numerical failure";
    default: return "unknown status";
  }
}

ABG_API const char* abg_last_error(void) { return g_err; }

ABG_API int64_t abg_launch_count(void) { return g_launches.load(); }
ABG_API int64_t abg_tensor_core_launches(void) { return g_tc_launches.load(); }

ABG_API int abg_create(const abg_graph_desc* desc, void* stream, abg_graph** out) {
  if (!out) {
    set_error("null output pointer");
    return ABG_EINVAL;
  }
  *out = nullptr;
  abg::SideSwap swap;
  const abg_graph_desc* dd = nullptr;
  int st = abg::swap_sides(desc, &swap, &dd);
  if (st != ABG_OK) return st;
  abg_graph* g = new abg_graph();
  cudaStream_t s = (cudaStream_t)stream;
  st = create_impl(dd, s, g);
  if (st != ABG_OK) {
    abg_destroy(g);
    return st;
  }
  *out = g;
  return ABG_OK;
}

// Stack n graphs into one block-diagonal graph whose segments are the inputs.
ABG_API int abg_batch_create(const abg_graph_desc* descs_in, int32_t n, int32_t device,
                             void* stream, abg_graph** out) {
  if (!out) {
    set_error("null output pointer");
    return ABG_EINVAL;
  }
  *out = nullptr;
  ABG_CHECK(descs_in && n >= 1, "need at least one graph");
  std::vector<SideSwap> swaps(n);
  std::vector<abg_graph_desc> dv(n);
  for (int i = 0; i < n; ++i) {
    const abg_graph_desc* p = nullptr;
    ABG_TRY(swap_sides(&descs_in[i], &swaps[i], &p));
    dv[i] = *p;
  }
  const abg_graph_desc* descs = dv.data();
  const int32_t d_u = descs[0].d_u, kind = descs[0].x_kind;
  int64_t nu = 0, nv = 0, nnz = 0, xnnz = 0;
  bool weighted = false;
  for (int i = 0; i < n; ++i) {
    const abg_graph_desc& e = descs[i];
    ABG_CHECK(e.d_u == d_u && e.x_kind == kind,
              "batched graphs need the same attribute width and storage kind");
    ABG_CHECK(e.n_u >= 1 && e.n_v >= 1 && e.nnz >= 0 && e.u_ptr && e.v_idx, "graph %d: bad sizes", i);
    ABG_CHECK(e.u_ptr[0] == 0 && e.u_ptr[e.n_u] == e.nnz, "graph %d: bad CSR pointers", i);
    if (kind == ABG_X_CSR_F32) {
      ABG_CHECK(e.x_ptr && e.x_idx && e.x_val && e.x_ptr[0] == 0, "graph %d: bad X CSR", i);
      xnnz += e.x_ptr[e.n_u];
    } else {
      ABG_CHECK(e.x, "graph %d: null attributes", i);
    }
    weighted |= e.w != nullptr;
    nu += e.n_u;
    nv += e.n_v;
    nnz += e.nnz;
  }
  ABG_CHECK(nu < (1ll << 31) && nv < (1ll << 31), "batch too large: |U|, |V| must stay < 2^31");
  const size_t esz = kind == ABG_X_DENSE_F32 ? 4 : 2;
  std::vector<int64_t> u_ptr(nu + 1), x_ptr;
  std::vector<int32_t> v_idx(nnz), x_idx;
  std::vector<float> w, x_val;
  std::vector<unsigned char> x_dense;
  if (weighted) w.resize(nnz);
  if (kind == ABG_X_CSR_F32) {
    x_ptr.resize(nu + 1);
    x_idx.resize(xnnz);
    x_val.resize(xnnz);
  } else {
    x_dense.resize(esz * nu * d_u);
  }
  abg_graph* g = new abg_graph();
  int64_t ro = 0, vo = 0, eo = 0, xo = 0;
  u_ptr[0] = 0;
  if (kind == ABG_X_CSR_F32) x_ptr[0] = 0;
  for (int i = 0; i < n; ++i) {
    const abg_graph_desc& e = descs[i];
    g->seg_row0.push_back(ro);
    g->seg_n.push_back(e.n_u);
    for (int64_t r = 0; r < e.n_u; ++r) u_ptr[ro + r + 1] = eo + e.u_ptr[r + 1];
    for (int64_t j = 0; j < e.nnz; ++j) {
      v_idx[eo + j] = (int32_t)(vo + e.v_idx[j]);
      if (weighted) w[eo + j] = e.w ? e.w[j] : 1.f;
    }
    if (kind == ABG_X_CSR_F32) {
      for (int64_t r = 0; r < e.n_u; ++r) x_ptr[ro + r + 1] = xo + e.x_ptr[r + 1];
      const int64_t en = e.x_ptr[e.n_u];
      std::copy(e.x_idx, e.x_idx + en, x_idx.begin() + xo);
      std::copy(e.x_val, e.x_val + en, x_val.begin() + xo);
      xo += en;
    } else {
      memcpy(x_dense.data() + esz * ro * d_u, e.x, esz * e.n_u * d_u);
    }
    ro += e.n_u;
    vo += e.n_v;
    eo += e.nnz;
  }
  g->nseg = n;
  abg_graph_desc u{};
  u.n_u = nu;
  u.n_v = nv;
  u.nnz = nnz;
  u.u_ptr = u_ptr.data();
  u.v_idx = v_idx.data();
  u.w = weighted ? w.data() : nullptr;
  u.d_u = d_u;
  u.x_kind = kind;
  if (kind == ABG_X_CSR_F32) {
    u.x_ptr = x_ptr.data();
    u.x_idx = x_idx.data();
    u.x_val = x_val.data();
  } else {
    u.x = x_dense.data();
  }
  u.device = device;
  int st = create_impl(&u, (cudaStream_t)stream, g);
  if (st != ABG_OK) {
    abg_destroy(g);
    return st;
  }
  *out = g;
  return ABG_OK;
}

ABG_API int32_t abg_graph_segments(const abg_graph* g) { return g ? g->nseg : 0; }

ABG_API void abg_destroy(abg_graph* g) {
  if (!g) return;
  if (g->n_blocks) {
    cudaSetDevice(g->device);
    for (int i = 0; i < g->n_blocks; ++i) cudaFreeAsync(g->blocks[i], 0);
    cudaStreamSynchronize(0);
  }
  delete g;
}

ABG_API int64_t abg_graph_footprint(const abg_graph* g) { return g ? g->footprint : 0; }

}  // extern "C"
