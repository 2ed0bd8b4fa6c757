// Internal helpers shared by the library's translation units: status
// handling, the stream-ordered allocator, launch helpers and small device
// utilities. Nothing here is part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <cstdio>
#include <string>
#include <vector>

#include "../../include/abg.h"

namespace abg {

// ---------------------------------------------------------------------------
// status / error text
// ---------------------------------------------------------------------------
void set_error(const char* fmt, ...);
int cuda_status(cudaError_t e, const char* what);

#define ABG_TRY(expr)              \
  do {                             \
    int _s = (expr);               \
    if (_s != ABG_OK) return _s;   \
  } while (0)

#define ABG_CUDA(expr)                                            \
  do {                                                            \
    cudaError_t _e = (expr);                                      \
    if (_e != cudaSuccess) return ::abg::cuda_status(_e, #expr);  \
  } while (0)

#define ABG_CHECK(cond, ...)             \
  do {                                   \
    if (!(cond)) {                       \
      ::abg::set_error(__VA_ARGS__);     \
      return ABG_EINVAL;                 \
    }                                    \
  } while (0)

// Launch check: reports the launch error (not asynchronous faults).
#define ABG_LAUNCH_CHECK() ABG_CUDA(cudaGetLastError())

// Test hook of the bounded waits, read from ABG_TEST_WAIT_EXPIRY at the start of each solve
// (abg_cluster, abg_batch_cluster) and held for its duration on the calling thread: with the
// value "spmm" the first wait of every warp of the TMA-gather SpMM for its first gather group
// gets no time at all, so it runs out on a copy still in flight and the error path runs
// (the warp drains its copies under the normal limit). Off (0) by default.
int test_wait_expiry();
struct SolveHooks {
  int prev;
  SolveHooks();
  ~SolveHooks();
};

// kernel launches issued by this library in this process (diagnostic counter)
void note_launch();
void note_tc_launch();  // a tensor-core kernel launch (also counted by note_launch)

// ---------------------------------------------------------------------------
// stream-ordered device memory from a private pool per device
// ---------------------------------------------------------------------------
int dev_alloc(void** p, size_t bytes, cudaStream_t s);
// Raises (never lowers) func's dynamic shared-memory limit on the current device.
int raise_smem_limit(const void* func, size_t bytes);
void dev_free(void* p, cudaStream_t s);

// RAII holder used inside one call: everything is released (stream-ordered)
// when the holder leaves scope.
struct Scratch {
  cudaStream_t stream;
  std::vector<void*> ptrs;
  explicit Scratch(cudaStream_t s) : stream(s) {}
  Scratch(const Scratch&) = delete;
  Scratch& operator=(const Scratch&) = delete;
  ~Scratch() {
    for (void* p : ptrs) dev_free(p, stream);
  }
  template <class T>
  int get(T** out, size_t count) {
    void* p = nullptr;
    int s = dev_alloc(&p, count * sizeof(T) + 16, stream);
    if (s != ABG_OK) return s;
    ptrs.push_back(p);
    *out = static_cast<T*>(p);
    return ABG_OK;
  }
};

__host__ __device__ inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
__host__ __device__ inline int64_t round_up(int64_t a, int64_t b) { return ceil_div(a, b) * b; }
inline int num_sms() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 152;
  }
  return n;
}

// ---------------------------------------------------------------------------
// device utilities
// ---------------------------------------------------------------------------
__device__ __forceinline__ float4 ld_nc_f4(const float* p) {
  return __ldg(reinterpret_cast<const float4*>(p));
}
__device__ __forceinline__ float4 ld_f4(const float* p) {
  return *reinterpret_cast<const float4*>(p);
}
__device__ __forceinline__ void st_f4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }

// 4 consecutive bf16 values (8 bytes) widened to float4.
__device__ __forceinline__ float4 ld_bf16x4(const __nv_bfloat16* p) {
  uint2 raw = __ldg(reinterpret_cast<const uint2*>(p));
  float4 r;
  r.x = __uint_as_float(raw.x << 16);
  r.y = __uint_as_float(raw.x & 0xffff0000u);
  r.z = __uint_as_float(raw.y << 16);
  r.w = __uint_as_float(raw.y & 0xffff0000u);
  return r;
}

__device__ __forceinline__ float4 f4_fma(float a, float4 x, float4 acc) {
  acc.x = fmaf(a, x.x, acc.x);
  acc.y = fmaf(a, x.y, acc.y);
  acc.z = fmaf(a, x.z, acc.z);
  acc.w = fmaf(a, x.w, acc.w);
  return acc;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace abg
