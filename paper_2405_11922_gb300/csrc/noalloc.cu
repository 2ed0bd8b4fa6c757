// abg_objective_noalloc: the objective of abg_objective (per-cluster sums of R,
// then sum_l s_l.(total - s_l)/|C_l| and sum_l |s_l|^2/|C_l| in FP64), for
// callers that must not allocate device memory: a host application that has
// handed the whole GPU to its own allocator up front, a latency-bound loop that
// cannot afford the device-wide synchronisation an allocation may cause, or an
// embedding runtime that forbids libraries from allocating on their own. The
// caller still owns R, the labels and the host result; the only extra memory is
// the fixed array below, which every GPU that loads this library holds until
// the process exits.
#include <mutex>

#include "internal.cuh"

namespace {

constexpr size_t kNoAllocBytes = size_t(24) << 20;  // 24 MiB per device
constexpr int kNoAllocChunks = 128;                 // fixed number of row chunks

// Scratch of every abg_objective_noalloc call on this device. Calls share it
// and it keeps the last call's contents; the kernels below write every element
// they later read, so nothing needs clearing. Calls that overlapped on the GPU
// would race on it, so each call holds a process-wide lock until its stream has
// synchronised: calls from several host threads run one after another. With
// CUDA's lazy module loading the array is reserved when the first call on a
// device loads this file's kernels, not when the library is loaded.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_mu;       // guards g_addr
std::mutex g_call_mu;  // serialises whole calls (see abg_objective_noalloc)
void* g_addr[64] = {};

// Device address of the array for the current device, looked up once per
// device (the first call on a device does this; make that first call before
// any stream capture).
int scratch_address(void** out) {
  int dev = 0;
  ABG_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) {
    abg::set_error("device ordinal %d out of range", dev);
    return ABG_EDEVICE;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return abg::cuda_status(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return ABG_OK;
}

// Bytes of the array one call uses for a per-chunk partial of `width` floats
// (k cluster rows of m sums, then k counts): the chunk partials, the FP64 sums,
// the two results, each block 256-byte aligned.
constexpr int64_t bytes_needed(int64_t width) {
  return ((int64_t)kNoAllocChunks * width * 4 + 255) / 256 * 256 + (width * 8 + 255) / 256 * 256 + 16;
}
// Widest partial that fits in the array.
constexpr int64_t max_width() {
  return (int64_t)((kNoAllocBytes - 1024) / (kNoAllocChunks * sizeof(float) + sizeof(double)));
}
static_assert(bytes_needed(max_width()) <= (int64_t)kNoAllocBytes, "scratch layout overflows");

// Chunk c of rows [c*rows_per, (c+1)*rows_per): per-cluster sums of R columns
// [col0, col0 + 256) and (for col0 == 0) the cluster counts, rows in order.
__global__ void k_na_sums(int64_t n, int k, int m, const float* __restrict__ R, int64_t ldr,
                          const int32_t* __restrict__ labels, int64_t rows_per, int col0,
                          float* __restrict__ part) {
  extern __shared__ float acc[];  // [k][256] then counts[k]
  float* cnt = acc + (int64_t)k * 256;
  const int64_t c = blockIdx.x;
  const int64_t r0 = c * rows_per, r1 = min(n, r0 + rows_per);
  for (int q = threadIdx.x; q < k * 256 + k; q += blockDim.x) acc[q] = 0.f;
  __syncthreads();
  const int col = col0 + threadIdx.x;
  const bool active = col < m;
  constexpr int U = 8;
  int64_t r = r0;
  for (; r + U <= r1; r += U) {
    int l[U];
    float v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      l[u] = labels[r + u];
      v[u] = active ? R[(r + u) * ldr + col] : 0.f;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if ((unsigned)l[u] >= (unsigned)k) continue;  // a label outside [0, k) is skipped
      if (active) acc[l[u] * 256 + threadIdx.x] += v[u];
      if (threadIdx.x == 0 && col0 == 0) cnt[l[u]] += 1.f;
    }
  }
  for (; r < r1; ++r) {
    const int l = labels[r];
    if ((unsigned)l >= (unsigned)k) continue;
    if (active) acc[l * 256 + threadIdx.x] += R[r * ldr + col];
    if (threadIdx.x == 0 && col0 == 0) cnt[l] += 1.f;
  }
  __syncthreads();
  const int64_t width = (int64_t)k * m + k;
  float* out = part + c * width;
  if (active)
    for (int l = 0; l < k; ++l) out[(int64_t)l * m + col] = acc[l * 256 + threadIdx.x];
  if (col0 == 0)
    for (int l = threadIdx.x; l < k; l += blockDim.x) out[(int64_t)k * m + l] = cnt[l];
}

// S[e] = sum over the chunks, in chunk order, in FP64
__global__ void k_na_reduce(const float* __restrict__ part, int64_t width, double* __restrict__ S) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= width) return;
  double s = 0.0;
  for (int c = 0; c < kNoAllocChunks; ++c) s += (double)part[(int64_t)c * width + e];
  S[e] = s;
}

__global__ void k_na_final(int k, int m, const double* __restrict__ S, double* __restrict__ out) {
  __shared__ double ro[256], rj[256];
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
  ro[threadIdx.x] = o;
  rj[threadIdx.x] = jv;
  __syncthreads();
  if (threadIdx.x == 0) {
    double so = 0.0, sj = 0.0;
    for (int t = 0; t < (int)blockDim.x; ++t) {
      so += ro[t];
      sj += rj[t];
    }
    out[0] = so;
    out[1] = sj;
  }
}

}  // namespace

extern "C" ABG_API int abg_objective_noalloc(const float* r, int64_t n, int32_t m, int64_t ldr,
                                             const int32_t* labels, int32_t k, double* obj,
                                             void* stream) {
  using namespace abg;
  ABG_CHECK(r && labels && obj && n >= 1 && m >= 1, "bad arguments");
  ABG_CHECK(ldr >= m && ldr % 4 == 0, "ldr must be >= m and a multiple of 4");
  ABG_CHECK(k >= 1 && k <= kMaxK, "need 1 <= k <= %d", kMaxK);
  const int64_t width = (int64_t)k * m + k;
  ABG_CHECK(width <= max_width(),
            "abg_objective_noalloc: k*(m+1) = %lld exceeds the fixed scratch limit %lld "
            "(use abg_objective)",
            (long long)width, (long long)max_width());
  cudaStream_t s = (cudaStream_t)stream;
  void* base = nullptr;
  ABG_TRY(scratch_address(&base));
  float* part = static_cast<float*>(base);
  double* S = reinterpret_cast<double*>(static_cast<char*>(base) +
                                        round_up((int64_t)kNoAllocChunks * width * 4, 256));
  double* out = S + round_up(width, 32);
  ABG_CHECK(bytes_needed(width) <= (int64_t)kNoAllocBytes, "internal: scratch layout overflow");
  const int64_t rows_per = ceil_div(n, kNoAllocChunks);
  const size_t smem = sizeof(float) * ((size_t)k * 256 + k);
  // One call at a time in this process, from its first launch until its stream has
  // synchronised: the launches of two host threads would otherwise interleave in the
  // array (even on one stream) and one call would read the other's partial sums.
  std::lock_guard<std::mutex> one_call(g_call_mu);
  // the limit is only ever raised, so a small-k call never undercuts a larger one
  ABG_TRY(raise_smem_limit((const void*)k_na_sums, smem));
  for (int col0 = 0; col0 < m; col0 += 256) {
    k_na_sums<<<kNoAllocChunks, 256, smem, s>>>(n, k, m, r, ldr, labels, rows_per, col0, part);
    note_launch();
  }
  k_na_reduce<<<(unsigned)ceil_div(width, 256), 256, 0, s>>>(part, width, S);
  note_launch();
  k_na_final<<<1, 256, 0, s>>>(k, m, S, out);
  note_launch();
  ABG_LAUNCH_CHECK();
  ABG_CUDA(cudaMemcpyAsync(obj, out, sizeof(double) * 2, cudaMemcpyDeviceToHost, s));
  ABG_CUDA(cudaStreamSynchronize(s));
  return ABG_OK;
}
