// Algorithm 1 propagation: gamma rounds of the two chained sparse products
//   W = L_U^T Z            (CSC rows = V nodes)
//   Z = (1-a) X + a L_U W  (CSR rows = U nodes, restart fused in the epilogue)
// followed by the row normalisation of Eq. 2 fused into the last round.
//
// Kernel shape: a group of G lanes owns one output row; each lane owns V
// float4 column chunks of that row, so one gathered input row is read with
// G*V coalesced 16-byte loads. The group loads up to G (index, value) pairs
// cooperatively, broadcasts them with shuffles and keeps 8 gathers in flight.
// Light rows run as streaming tasks (runs of consecutive rows, at most
// kTaskRows rows and about kTaskEdges edges); rows with more than kHeavyRow
// edges are split into kHeavyChunk-edge chunks whose partial sums go to a
// scratch buffer and are added back in chunk order, so results do not depend
// on scheduling (no floating-point atomics).
#include <atomic>
#include <cstdlib>
#include <map>
#include <mutex>

#include "internal.cuh"
#include "tma.cuh"

namespace abg {

struct EpiParams {
  int mode;          // 0: C = scale*acc   1: restart   2: restart + Eq. 2 normalisation
  float scale;       // mode 0
  float c_x, c_p;    // modes 1/2: C = c_x * X + c_p * acc
  const void* x;     // restart attributes (float or bf16), row stride ldx
  int x_bf16;
  int64_t ldx;
  int d;             // row width: components at or beyond d are treated as 0 and written as 0
  int out_bf16;      // C holds BF16 values (rounded to nearest even), row stride ldc elements
};

template <class T>
__device__ __forceinline__ float4 load4(const T* p);
template <>
__device__ __forceinline__ float4 load4<float>(const float* p) {
  return ld_nc_f4(p);
}
template <>
__device__ __forceinline__ float4 load4<__nv_bfloat16>(const __nv_bfloat16* p) {
  return ld_bf16x4(p);
}

template <int G>
__device__ __forceinline__ unsigned group_mask() {
  if constexpr (G == 32) {
    return 0xffffffffu;
  } else {
    unsigned lane = threadIdx.x & 31;
    return ((1u << G) - 1u) << (lane & ~(unsigned)(G - 1));
  }
}

// acc[v] += sum over edges [b, e) of val * B[col] (chunks of this lane)
template <int G, int V, class TIn>
__device__ __forceinline__ void gather_range(int64_t b, int64_t e, const int32_t* __restrict__ col,
                                             const float* __restrict__ val,
                                             const TIn* __restrict__ B, int64_t ldb, int nchunk,
                                             int lig, unsigned mask, float4 (&acc)[V]) {
  constexpr int UNR = (V >= 4) ? 4 : (G < 8 ? G : 8);
  for (int64_t base = b; base < e; base += G) {
    int64_t j = base + lig;
    int c = 0;
    float w = 0.f;
    if (j < e) {
      c = __ldg(col + j);
      w = __ldg(val + j);
    }
    const int64_t rem = e - base;
    const int cnt = rem < G ? (int)rem : G;
    for (int t = 0; t < cnt; t += UNR) {
      float4 x[UNR][V];
      float ws[UNR];
#pragma unroll
      for (int u = 0; u < UNR; ++u) {
        int src = (t + u) & (G - 1);
        int ct = __shfl_sync(mask, c, src, G);
        float wt = __shfl_sync(mask, w, src, G);
        bool ok = (t + u) < cnt;
        ws[u] = ok ? wt : 0.f;
        const TIn* rowp = B + (int64_t)ct * ldb;
#pragma unroll
        for (int v = 0; v < V; ++v) {
          int ch = lig + G * v;
          if (ok && ch < nchunk)
            x[u][v] = load4<TIn>(rowp + 4 * ch);
          else
            x[u][v] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
      }
#pragma unroll
      for (int u = 0; u < UNR; ++u)
#pragma unroll
        for (int v = 0; v < V; ++v) acc[v] = f4_fma(ws[u], x[u][v], acc[v]);
    }
  }
}

// zero the components of chunk ch that lie at or beyond column d (row padding)
__device__ __forceinline__ float4 mask_tail(float4 v, int ch, int d) {
  const int c0 = 4 * ch;
  if (c0 + 1 >= d) v.y = 0.f;
  if (c0 + 2 >= d) v.z = 0.f;
  if (c0 + 3 >= d) v.w = 0.f;
  if (c0 >= d) v.x = 0.f;
  return v;
}

// restart attributes of one row (modes 1/2), zero beyond column d
template <int G, int V>
__device__ __forceinline__ void load_x_row(int64_t row, int nchunk, int lig, const EpiParams& ep,
                                           float4 (&xv)[V]) {
#pragma unroll
  for (int v = 0; v < V; ++v) {
    const int ch = lig + G * v;
    xv[v] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (ep.mode != 0 && ch < nchunk) {
      if (ep.x_bf16)
        xv[v] = ld_bf16x4(reinterpret_cast<const __nv_bfloat16*>(ep.x) + row * ep.ldx + 4 * ch);
      else
        xv[v] = ld_nc_f4(reinterpret_cast<const float*>(ep.x) + row * ep.ldx + 4 * ch);
      xv[v] = mask_tail(xv[v], ch, ep.d);
    }
  }
}

// C[row] = scale * acc (mode 0), c_x X[row] + c_p acc (mode 1), the same normalised (mode 2)
template <int G, int V>
__device__ __forceinline__ void epilogue_core(int64_t row, const float4 (&acc_in)[V],
                                              const float4 (&xv)[V], float* C, int64_t ldc,
                                              int nchunk, int lig, unsigned mask,
                                              const EpiParams& ep) {
  float4 acc[V];
#pragma unroll
  for (int v = 0; v < V; ++v) acc[v] = mask_tail(acc_in[v], lig + G * v, ep.d);
  float4 out[V];
  if (ep.mode == 0) {
#pragma unroll
    for (int v = 0; v < V; ++v)
      out[v] = make_float4(ep.scale * acc[v].x, ep.scale * acc[v].y, ep.scale * acc[v].z,
                           ep.scale * acc[v].w);
  } else {
    float ss = 0.f;
#pragma unroll
    for (int v = 0; v < V; ++v) {
      float4 z;
      z.x = fmaf(ep.c_p, acc[v].x, ep.c_x * xv[v].x);
      z.y = fmaf(ep.c_p, acc[v].y, ep.c_x * xv[v].y);
      z.z = fmaf(ep.c_p, acc[v].z, ep.c_x * xv[v].z);
      z.w = fmaf(ep.c_p, acc[v].w, ep.c_x * xv[v].w);
      out[v] = z;
      // explicit FMAs: every inlined copy of this epilogue rounds the same way
      ss = fmaf(z.x, z.x, ss);
      ss = fmaf(z.y, z.y, ss);
      ss = fmaf(z.z, z.z, ss);
      ss = fmaf(z.w, z.w, ss);
    }
    if (ep.mode == 2) {
#pragma unroll
      for (int o = G / 2; o > 0; o >>= 1) ss += __shfl_xor_sync(mask, ss, o, G);
      float inv = ss > 0.f ? 1.0f / sqrtf(ss) : 0.f;
#pragma unroll
      for (int v = 0; v < V; ++v) {
        out[v].x *= inv;
        out[v].y *= inv;
        out[v].z *= inv;
        out[v].w *= inv;
      }
    }
  }
#pragma unroll
  for (int v = 0; v < V; ++v) {
    int ch = lig + G * v;
    if (ch >= nchunk) continue;
    if (ep.out_bf16) {
      const __nv_bfloat162 lo = __floats2bfloat162_rn(out[v].x, out[v].y);
      const __nv_bfloat162 hi = __floats2bfloat162_rn(out[v].z, out[v].w);
      uint2 u;
      u.x = *reinterpret_cast<const uint32_t*>(&lo);
      u.y = *reinterpret_cast<const uint32_t*>(&hi);
      *reinterpret_cast<uint2*>(reinterpret_cast<__nv_bfloat16*>(C) + row * ldc + 4 * ch) = u;
    } else {
      st_f4(C + row * ldc + 4 * ch, out[v]);
    }
  }
}

template <int G, int V>
__device__ __forceinline__ void epilogue_store(int64_t row, const float4 (&acc)[V], float* C,
                                               int64_t ldc, int nchunk, int lig, unsigned mask,
                                               const EpiParams& ep) {
  float4 xv[V];
  load_x_row<G, V>(row, nchunk, lig, ep, xv);
  epilogue_core<G, V>(row, acc, xv, C, ldc, nchunk, lig, mask, ep);
}

// Light rows: one group per listed row (rows == nullptr: row = group index).
template <int G, int V, class TIn>
__global__ void __launch_bounds__(256) k_spmm_rows(const int32_t* __restrict__ rows, int64_t n_rows,
                                                   const int64_t* __restrict__ ptr,
                                                   const int32_t* __restrict__ col,
                                                   const float* __restrict__ val,
                                                   const TIn* __restrict__ B, int64_t ldb,
                                                   float* __restrict__ C, int64_t ldc, int nchunk,
                                                   EpiParams ep) {
  int64_t grp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
  int lig = threadIdx.x & (G - 1);
  if (grp >= n_rows) return;  // whole groups exit together
  unsigned mask = group_mask<G>();
  int64_t row = rows ? (int64_t)rows[grp] : grp;
  float4 acc[V];
#pragma unroll
  for (int v = 0; v < V; ++v) acc[v] = make_float4(0.f, 0.f, 0.f, 0.f);
  gather_range<G, V, TIn>(ptr[row], ptr[row + 1], col, val, B, ldb, nchunk, lig, mask, acc);
  epilogue_store<G, V>(row, acc, C, ldc, nchunk, lig, mask, ep);
}

// Light rows, streamed: one group per task, a run of consecutive light rows whose
// edges are contiguous. The group walks the task's edge list G edges at a time,
// keeping UNR gathers in flight across row boundaries, and finishes a row (epilogue)
// when the edge cursor passes its end. Each row still sums its edges in edge
// order, so results equal the one-row-per-group kernel.
template <int G, int V, class TIn>
__global__ void __launch_bounds__(256) k_spmm_stream(const int2* __restrict__ tasks,
                                                     int64_t n_tasks,
                                                     const int64_t* __restrict__ ptr,
                                                     const int32_t* __restrict__ col,
                                                     const float* __restrict__ val,
                                                     const TIn* __restrict__ B, int64_t ldb,
                                                     float* __restrict__ C, int64_t ldc,
                                                     int nchunk, EpiParams ep) {
  constexpr int UNR = (V >= 4) ? 4 : (G < 8 ? G : 8);
  const int64_t grp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
  const int lig = threadIdx.x & (G - 1);
  if (grp >= n_tasks) return;  // whole groups exit together
  const unsigned mask = group_mask<G>();
  const int2 tk = tasks[grp];
  const int64_t r0 = tk.x;
  const int nrows = tk.y - tk.x;
  const int64_t e_begin = ptr[r0];
  const int64_t e_end = ptr[tk.y];
  // lane i of the window holds the end of row wbase + i
  int wbase = 0;
  int64_t rp = lig < nrows ? ptr[r0 + 1 + lig] : e_end;
  int cur = 0;
  int64_t rend = __shfl_sync(mask, rp, 0, G);
  float4 acc[V];
#pragma unroll
  for (int v = 0; v < V; ++v) acc[v] = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int64_t base = e_begin; base < e_end; base += G) {
    const int64_t j = base + lig;
    int c = 0;
    float w = 0.f;
    if (j < e_end) {
      c = __ldg(col + j);
      w = __ldg(val + j);
    }
    const int64_t rem = e_end - base;
    const int cnt = rem < G ? (int)rem : G;
    for (int t = 0; t < cnt; t += UNR) {
      float4 x[UNR][V];
      float ws[UNR];
#pragma unroll
      for (int u = 0; u < UNR; ++u) {
        const int src = (t + u) & (G - 1);
        const int ct = __shfl_sync(mask, c, src, G);
        ws[u] = __shfl_sync(mask, w, src, G);
        const bool ok = (t + u) < cnt;
        const TIn* rowp = B + (int64_t)ct * ldb;
#pragma unroll
        for (int v = 0; v < V; ++v) {
          const int ch = lig + G * v;
          x[u][v] = (ok && ch < nchunk) ? load4<TIn>(rowp + 4 * ch)
                                        : make_float4(0.f, 0.f, 0.f, 0.f);
        }
      }
#pragma unroll
      for (int u = 0; u < UNR; ++u) {
        if (t + u >= cnt) break;  // uniform over the group
        const int64_t e = base + t + u;
        while (e >= rend) {  // rows before the one edge e belongs to are complete
          epilogue_store<G, V>(r0 + cur, acc, C, ldc, nchunk, lig, mask, ep);
#pragma unroll
          for (int v = 0; v < V; ++v) acc[v] = make_float4(0.f, 0.f, 0.f, 0.f);
          ++cur;  // stays < nrows: e < e_end, the end of the last row
          if (cur - wbase >= G) {
            wbase += G;
            rp = wbase + lig < nrows ? ptr[r0 + 1 + wbase + lig] : e_end;
          }
          rend = __shfl_sync(mask, rp, cur - wbase, G);
        }
#pragma unroll
        for (int v = 0; v < V; ++v) acc[v] = f4_fma(ws[u], x[u][v], acc[v]);
      }
    }
  }
  // the row holding the last edge, then the empty rows after it
  for (; cur < nrows; ++cur) {
    epilogue_store<G, V>(r0 + cur, acc, C, ldc, nchunk, lig, mask, ep);
#pragma unroll
    for (int v = 0; v < V; ++v) acc[v] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

// ---------------------------------------------------------------------------
// Light tasks (or heavy-row chunks) for rows of 17..64 float4 chunks: one warp
// per work item, lane c owning chunk c (+32). Edge indices are relative to the
// item's first edge (32-bit); the (column, value) pairs of the next 32 edges
// are fetched while the current 32 are gathered, UNR row gathers are in flight
// per step, a step whose UNR edges lie in the current row skips the boundary
// checks, and the restart row of X is fetched when a row starts. Each row sums
// its edges in edge order, as in the other SpMM kernels.
// CHUNK: item c sums the kHeavyChunk edges of chunk c into row c of `C` (the
// partial buffer) with the raw epilogue.
// ---------------------------------------------------------------------------
struct SpmmItems {
  const int2* tasks;
  const int64_t* chunk_begin;
  const int32_t* chunk_slot;
  const int32_t* heavy_row;
};

template <int V, class TIn, bool CHUNK, int MODE, int UNR, int MINB>
__global__ void __launch_bounds__(256, MINB)
    k_spmm_warp(const SpmmItems items, int64_t n_items, const int64_t* __restrict__ ptr,
                const int32_t* __restrict__ col, const float* __restrict__ val,
                const TIn* __restrict__ B, int ldb, float* __restrict__ C, int ldc, int nchunk,
                EpiParams ep) {
  const int64_t item = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (item >= n_items) return;  // whole warps
  ep.mode = MODE;  // a compile-time mode lets the compiler drop the other epilogues
  int64_t r0, e0;
  int nrows, ne, rend_l;
  if constexpr (CHUNK) {
    const int64_t row = items.heavy_row[items.chunk_slot[item]];
    r0 = item;
    nrows = 1;
    e0 = items.chunk_begin[item];
    const int64_t rest = ptr[row + 1] - e0;
    ne = rest < kHeavyChunk ? (int)rest : kHeavyChunk;
    rend_l = ne;
  } else {
    const int2 tk = items.tasks[item];
    r0 = tk.x;
    nrows = tk.y - tk.x;
    e0 = ptr[tk.x];
    ne = (int)(ptr[tk.y] - e0);
    rend_l = lane < nrows ? (int)(ptr[tk.x + 1 + lane] - e0) : ne;
  }
  const int32_t* __restrict__ colp = col + e0;
  const float* __restrict__ valp = val + e0;
  float4 acc[V], xv[V];
#pragma unroll
  for (int v = 0; v < V; ++v) acc[v] = make_float4(0.f, 0.f, 0.f, 0.f);
  load_x_row<32, V>(r0, nchunk, lane, ep, xv);
  int cur = 0;
  int rend = __shfl_sync(0xffffffffu, rend_l, 0);
  int c_next = lane < ne ? __ldg(colp + lane) : 0;
  float w_next = lane < ne ? __ldg(valp + lane) : 0.f;
  for (int base = 0; base < ne; base += 32) {
    const int c = c_next;
    const float w = w_next;
    if (base + 32 + lane < ne) {  // the next 32 pairs, fetched while these are gathered
      c_next = __ldg(colp + base + 32 + lane);
      w_next = __ldg(valp + base + 32 + lane);
    }
    const int cnt = ne - base < 32 ? ne - base : 32;
    for (int t = 0; t < cnt; t += UNR) {
      float4 x[UNR][V];
      float ws[UNR];
#pragma unroll
      for (int u = 0; u < UNR; ++u) {
        const int src = t + u;
        const int ct = __shfl_sync(0xffffffffu, c, src & 31);
        ws[u] = __shfl_sync(0xffffffffu, w, src & 31);
        const TIn* rowp = B + (int64_t)ct * ldb;
#pragma unroll
        for (int v = 0; v < V; ++v) {
          const int ch = lane + 32 * v;
          x[u][v] = (src < cnt && ch < nchunk) ? load4<TIn>(rowp + 4 * ch)
                                               : make_float4(0.f, 0.f, 0.f, 0.f);
        }
      }
      if (base + t + UNR <= rend) {  // all UNR edges in the current row
#pragma unroll
        for (int u = 0; u < UNR; ++u)
#pragma unroll
          for (int v = 0; v < V; ++v) acc[v] = f4_fma(ws[u], x[u][v], acc[v]);
      } else {
#pragma unroll
        for (int u = 0; u < UNR; ++u) {
          const int e = base + t + u;
          if (e >= ne) break;  // uniform
          while (e >= rend) {  // rows ending before edge e are complete
            epilogue_core<32, V>(r0 + cur, acc, xv, C, ldc, nchunk, lane, 0xffffffffu, ep);
#pragma unroll
            for (int v = 0; v < V; ++v) acc[v] = make_float4(0.f, 0.f, 0.f, 0.f);
            ++cur;  // < nrows: e < ne, the end of the last row
            rend = __shfl_sync(0xffffffffu, rend_l, cur);
            load_x_row<32, V>(r0 + cur, nchunk, lane, ep, xv);
          }
#pragma unroll
          for (int v = 0; v < V; ++v) acc[v] = f4_fma(ws[u], x[u][v], acc[v]);
        }
      }
    }
  }
  // the row holding the last edge, then the empty rows after it
  for (; cur < nrows; ++cur) {
    epilogue_core<32, V>(r0 + cur, acc, xv, C, ldc, nchunk, lane, 0xffffffffu, ep);
#pragma unroll
    for (int v = 0; v < V; ++v) acc[v] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (cur + 1 < nrows) load_x_row<32, V>(r0 + cur + 1, nchunk, lane, ep, xv);
  }
}

#ifndef ABG_WARP_UNR
#define ABG_WARP_UNR 4
#endif
#ifndef ABG_WARP_MINB
#define ABG_WARP_MINB 5
#endif

// ---------------------------------------------------------------------------
// Light rows with TMA gathers (rows of at most 64 float4 chunks).
//
// One warp per task at a time, tasks gw, gw + W, ... of the warp's own list.
// The task's (column, value) pairs are staged in shared memory; lane 0 issues
// tile::gather4 copies (four gathered rows, one box row each) into a ring of
// slots guarded by one mbarrier each, running up to `slots` groups ahead of
// the consumer and at most one task ahead. All 32 lanes consume a slot in
// edge order (lane c owns float4 chunk c (+32) of every row), so each output
// row sums its edges in the same order as the other SpMM kernels. The restart
// row of X is fetched when a row starts, so its latency hides behind the
// row's gathers. Waits are bounded: a wait that runs out sets *wait_err,
// drains this warp's copies (again bounded) and stops the warp.
// ---------------------------------------------------------------------------
#ifndef ABG_TMA_WARPS
#define ABG_TMA_WARPS 28
#endif
#ifndef ABG_TMA_RING
#define ABG_TMA_RING 4096
#endif
constexpr int kTmaWarps = ABG_TMA_WARPS;     // warps (independent pipelines) per CTA
constexpr int kTmaRingBytes = ABG_TMA_RING;  // gather ring per warp
template <class TIn>
__device__ __forceinline__ float4 smem_chunk(const unsigned char* row, int ch);
template <>
__device__ __forceinline__ float4 smem_chunk<float>(const unsigned char* row, int ch) {
  return *reinterpret_cast<const float4*>(row + 16 * ch);
}
template <>
__device__ __forceinline__ float4 smem_chunk<__nv_bfloat16>(const unsigned char* row, int ch) {
  const uint2 u = *reinterpret_cast<const uint2*>(row + 8 * ch);
  return make_float4(__uint_as_float(u.x << 16), __uint_as_float(u.x & 0xffff0000u),
                     __uint_as_float(u.y << 16), __uint_as_float(u.y & 0xffff0000u));
}

struct TaskMeta {
  int64_t r0;   // first row
  int64_t e0;   // first edge
  int nrows;
  int ne;       // edges (>= 1)
  int rend;     // this lane's row end (lane < nrows), relative to e0
};

// Work items of k_spmm_tma: light tasks (row ranges), or the chunks of heavy rows
// (CHUNK: item c sums kHeavyChunk edges of one row into row c of the partial buffer).
struct TmaItems {
  const int2* tasks;
  const int64_t* chunk_begin;
  const int32_t* chunk_slot;
  const int32_t* heavy_row;
};

template <int V, class TIn, bool CHUNK>
__global__ void __launch_bounds__(kTmaWarps * 32, 1)
    k_spmm_tma(const __grid_constant__ CUtensorMap bmap, const TmaItems items,
               int64_t n_tasks, const int64_t* __restrict__ ptr, const int32_t* __restrict__ col,
               const float* __restrict__ val, float* __restrict__ C, int64_t ldc, int nchunk,
               int row_bytes, int slot_bytes, int slots, int warp_bytes, EpiParams ep,
               int* __restrict__ wait_err, int test_expiry) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int64_t gw = (int64_t)blockIdx.x * kTmaWarps + warp;
  const int64_t nw = (int64_t)gridDim.x * kTmaWarps;
  if (gw >= n_tasks) return;  // whole warps; the kernel has no CTA-wide barrier
  const int64_t n_mine = (n_tasks - gw + nw - 1) / nw;
  unsigned char* ring = smem + (size_t)warp * warp_bytes;
  int* idx = reinterpret_cast<int*>(ring + (size_t)slots * slot_bytes);  // [2][kTaskEdges]
  float* wv = reinterpret_cast<float*>(idx + 2 * kTaskEdges);            // [2][kTaskEdges]
  uint64_t* bars = reinterpret_cast<uint64_t*>(wv + 2 * kTaskEdges);      // [slots]
  const uint32_t ring_s = smem_addr(ring);
  const uint32_t bar_s = smem_addr(bars);
  if (lane == 0)
    for (int i = 0; i < slots; ++i) mbar_init(bar_s + 8 * i, 1);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  __syncwarp();

  // task k of this warp: row range, edge range, row ends, staged (column, value) pairs
  auto load_task = [&](int64_t k, TaskMeta& m) {
    if constexpr (CHUNK) {
      const int64_t c = gw + k * nw;
      const int64_t row = items.heavy_row[items.chunk_slot[c]];
      m.r0 = c;
      m.nrows = 1;
      m.e0 = items.chunk_begin[c];
      const int64_t rest = ptr[row + 1] - m.e0;
      m.ne = rest < kHeavyChunk ? (int)rest : kHeavyChunk;
      m.rend = m.ne;
    } else {
      const int2 tk = items.tasks[gw + k * nw];
      m.r0 = tk.x;
      m.nrows = tk.y - tk.x;
      m.e0 = ptr[tk.x];
      m.ne = (int)(ptr[tk.y] - m.e0);
      m.rend = lane < m.nrows ? (int)(ptr[tk.x + 1 + lane] - m.e0) : m.ne;
    }
    int* ib = idx + (k & 1) * kTaskEdges;
    float* wb = wv + (k & 1) * kTaskEdges;
    const int n4 = (m.ne + 3) & ~3;
    for (int j = lane; j < n4; j += 32) {
      const int jj = j < m.ne ? j : m.ne - 1;  // a padded slot re-gathers the last row
      ib[j] = __ldg(col + m.e0 + jj);
      wb[j] = j < m.ne ? __ldg(val + m.e0 + j) : 0.f;
    }
    __syncwarp();
  };

  TaskMeta mp, mc;
  load_task(0, mp);
  mc = mp;
  int64_t pk = 0, ck = 0;  // producer / consumer task
  int pg = 0, cg = 0;      // next group of the task to issue / consume
  int inflight = 0;        // groups issued and not yet consumed
  int p_slot = 0;          // ring slot of the next issue
  int c_slot = 0;          // ring slot of the next group to consume, and its phase parity
  uint32_t c_phase = 0;
  bool bad = false;

  auto produce = [&]() -> bool {
    if (pk >= n_mine) return false;
    if (pg == ((mp.ne + 3) >> 2)) {
      if (pk + 1 >= n_mine || pk + 1 > ck + 1) return false;
      ++pk;
      load_task(pk, mp);
      pg = 0;
    }
    if (lane == 0) {
      const int4 rows = *reinterpret_cast<const int4*>(idx + (pk & 1) * kTaskEdges + 4 * pg);
      const uint32_t bar = bar_s + 8 * p_slot;
      mbar_expect_tx(bar, 4 * row_bytes);
      tma_gather4(ring_s + p_slot * slot_bytes, &bmap, rows, bar);
    }
    ++pg;
    ++inflight;
    p_slot = p_slot + 1 == slots ? 0 : p_slot + 1;
    return true;
  };

  float4 acc[V], xv[V];
#pragma unroll
  for (int v = 0; v < V; ++v) acc[v] = make_float4(0.f, 0.f, 0.f, 0.f);
  int cur = 0;
  int rend = __shfl_sync(0xffffffffu, mc.rend, 0);
  load_x_row<32, V>(mc.r0, nchunk, lane, ep, xv);

  while (ck < n_mine) {
    while (inflight < slots && produce()) {
    }
    const int sl = c_slot;
    if (test_expiry) {  // test hook: the warp's first wait gets no time (see SolveHooks)
      bad = !mbar_test_wait(bar_s + 8 * sl, c_phase);
      test_expiry = 0;
    } else {
      bad = !mbar_wait_bounded(bar_s + 8 * sl, c_phase);
    }
    if (__any_sync(0xffffffffu, bad)) {
      bad = true;
      break;
    }
    const unsigned char* slot = ring + (size_t)sl * slot_bytes;
    const float* wb = wv + (ck & 1) * kTaskEdges;
    if (4 * cg + 4 <= rend) {  // common case: the four edges lie in the current row
      const float4 w4 = *reinterpret_cast<const float4*>(wb + 4 * cg);
#pragma unroll
      for (int v = 0; v < V; ++v) {
        const int ch = lane + 32 * v;
        if (ch < nchunk) {
          acc[v] = f4_fma(w4.x, smem_chunk<TIn>(slot, ch), acc[v]);
          acc[v] = f4_fma(w4.y, smem_chunk<TIn>(slot + row_bytes, ch), acc[v]);
          acc[v] = f4_fma(w4.z, smem_chunk<TIn>(slot + 2 * row_bytes, ch), acc[v]);
          acc[v] = f4_fma(w4.w, smem_chunk<TIn>(slot + 3 * row_bytes, ch), acc[v]);
        }
      }
    } else
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int j = 4 * cg + i;
      if (j >= mc.ne) break;  // uniform
      while (j >= rend) {     // rows ending before edge j are complete
        epilogue_core<32, V>(mc.r0 + cur, acc, xv, C, ldc, nchunk, lane, 0xffffffffu, ep);
#pragma unroll
        for (int v = 0; v < V; ++v) acc[v] = make_float4(0.f, 0.f, 0.f, 0.f);
        ++cur;  // < nrows: j < ne, the end of the last row
        rend = __shfl_sync(0xffffffffu, mc.rend, cur);
        load_x_row<32, V>(mc.r0 + cur, nchunk, lane, ep, xv);
      }
      const float w = wb[j];
#pragma unroll
      for (int v = 0; v < V; ++v) {
        const int ch = lane + 32 * v;
        if (ch < nchunk) acc[v] = f4_fma(w, smem_chunk<TIn>(slot + i * row_bytes, ch), acc[v]);
      }
    }
    __syncwarp();  // the slot is free once every lane has read it
    --inflight;
    if (++c_slot == slots) {
      c_slot = 0;
      c_phase ^= 1u;
    }
    ++cg;
    if (cg == ((mc.ne + 3) >> 2)) {
      // the row holding the task's last edge, then the empty rows after it
      for (; cur < mc.nrows; ++cur) {
        epilogue_core<32, V>(mc.r0 + cur, acc, xv, C, ldc, nchunk, lane, 0xffffffffu, ep);
#pragma unroll
        for (int v = 0; v < V; ++v) acc[v] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (cur + 1 < mc.nrows) load_x_row<32, V>(mc.r0 + cur + 1, nchunk, lane, ep, xv);
      }
      ++ck;
      cg = 0;
      if (ck < n_mine) {
        while (pk < ck && produce()) {
        }
        mc = mp;  // pk == ck: the producer has staged task ck
        cur = 0;
        rend = __shfl_sync(0xffffffffu, mc.rend, 0);
        load_x_row<32, V>(mc.r0, nchunk, lane, ep, xv);
      }
    }
  }
  if (bad) {
    if (lane == 0) atomicExch(wait_err, 1);
    for (; inflight > 0; --inflight) {  // copies still in flight into this ring
      if (!mbar_wait_bounded(bar_s + 8 * c_slot, c_phase)) break;
      if (++c_slot == slots) {
        c_slot = 0;
        c_phase ^= 1u;
      }
    }
  }
}

// Heavy rows, phase 1: one group per chunk, raw partial sums.
template <int G, int V, class TIn>
__global__ void __launch_bounds__(256) k_spmm_chunks(
    const int64_t* __restrict__ chunk_begin, const int32_t* __restrict__ chunk_slot,
    const int32_t* __restrict__ heavy_row, int64_t n_chunks, const int64_t* __restrict__ ptr,
    const int32_t* __restrict__ col, const float* __restrict__ val, const TIn* __restrict__ B,
    int64_t ldb, float* __restrict__ part, int64_t ldp, int nchunk) {
  int64_t grp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
  int lig = threadIdx.x & (G - 1);
  if (grp >= n_chunks) return;
  unsigned mask = group_mask<G>();
  int64_t row = heavy_row[chunk_slot[grp]];
  int64_t b = chunk_begin[grp];
  int64_t e = min(b + (int64_t)kHeavyChunk, ptr[row + 1]);
  float4 acc[V];
#pragma unroll
  for (int v = 0; v < V; ++v) acc[v] = make_float4(0.f, 0.f, 0.f, 0.f);
  gather_range<G, V, TIn>(b, e, col, val, B, ldb, nchunk, lig, mask, acc);
#pragma unroll
  for (int v = 0; v < V; ++v) {
    int ch = lig + G * v;
    if (ch < nchunk) st_f4(part + grp * ldp + 4 * ch, acc[v]);
  }
}

// Heavy rows, phase 2: add the chunk partials of each heavy row in order, then the epilogue.
template <int G, int V>
__global__ void __launch_bounds__(256) k_spmm_reduce(const int32_t* __restrict__ heavy_row,
                                                     const int64_t* __restrict__ heavy_chunk0,
                                                     int64_t n_heavy,
                                                     const float* __restrict__ part, int64_t ldp,
                                                     float* __restrict__ C, int64_t ldc,
                                                     int nchunk, EpiParams ep) {
  int64_t grp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
  int lig = threadIdx.x & (G - 1);
  if (grp >= n_heavy) return;
  unsigned mask = group_mask<G>();
  float4 acc[V];
#pragma unroll
  for (int v = 0; v < V; ++v) acc[v] = make_float4(0.f, 0.f, 0.f, 0.f);
  const int64_t c1 = heavy_chunk0[grp + 1];
  int64_t c = heavy_chunk0[grp];
  // partials added in chunk order; eight loads in flight at a time
  for (; c + 8 <= c1; c += 8) {
#pragma unroll
    for (int v = 0; v < V; ++v) {
      const int ch = lig + G * v;
      if (ch < nchunk) {
        float4 p[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) p[u] = ld_f4(part + (c + u) * ldp + 4 * ch);
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          acc[v].x += p[u].x;
          acc[v].y += p[u].y;
          acc[v].z += p[u].z;
          acc[v].w += p[u].w;
        }
      }
    }
  }
  for (; c < c1; ++c) {
#pragma unroll
    for (int v = 0; v < V; ++v) {
      const int ch = lig + G * v;
      if (ch < nchunk) {
        const float4 p = ld_f4(part + c * ldp + 4 * ch);
        acc[v].x += p.x;
        acc[v].y += p.y;
        acc[v].z += p.z;
        acc[v].w += p.w;
      }
    }
  }
  epilogue_store<G, V>((int64_t)heavy_row[grp], acc, C, ldc, nchunk, lig, mask, ep);
}

// gamma = 0: Z = (1-a) X, normalised (Eq. 2)
template <int G, int V>
__global__ void __launch_bounds__(256) k_scale_rows(int64_t n_rows, float* __restrict__ C,
                                                    int64_t ldc, int nchunk, EpiParams ep) {
  int64_t grp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
  int lig = threadIdx.x & (G - 1);
  if (grp >= n_rows) return;
  unsigned mask = group_mask<G>();
  float4 acc[V];
#pragma unroll
  for (int v = 0; v < V; ++v) acc[v] = make_float4(0.f, 0.f, 0.f, 0.f);
  epilogue_store<G, V>(grp, acc, C, ldc, nchunk, lig, mask, ep);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

struct Shape {
  int G, V;
};
static Shape shape_for(int nchunk) {
  if (nchunk <= 4) return {4, 1};
  if (nchunk <= 8) return {8, 1};
  if (nchunk <= 16) return {16, 1};
  if (nchunk <= 32) return {32, 1};
  if (nchunk <= 64) return {32, 2};
  if (nchunk <= 128) return {32, 4};
  return {32, 8};
}

static inline unsigned blocks_for(int64_t groups, int G) {
  return (unsigned)ceil_div(groups * G, 256);
}

// Light tasks with edges through k_spmm_tma; *used stays false when the shape does not
// fit its limits (row box of at most 256 elements, 16-byte rows and base).
template <int V, class TIn>
static int run_spmm_tma(const abg_graph::Schedule& sc, const int64_t* ptr, const int32_t* col,
                        const float* val, const TIn* B, int64_t ldb, int64_t b_rows, float* C,
                        int64_t ldc, int nchunk, const EpiParams& ep, float* part, int64_t ldp,
                        int* wait_err, cudaStream_t s, bool* used) {
  *used = false;
  if (sc.n_etasks + sc.n_chunks == 0 || !wait_err) return ABG_OK;
  const auto enc = tensor_map_encoder();
  const int box_w = 4 * nchunk;
  const int row_bytes = box_w * (int)sizeof(TIn);
  const int64_t stride = ldb * (int64_t)sizeof(TIn);
  if (!enc || b_rows < 1 || b_rows > INT32_MAX || box_w > 256 || stride % 16 != 0 ||
      row_bytes % 16 != 0 || reinterpret_cast<uintptr_t>(B) % 16 != 0)
    return ABG_OK;
  CUtensorMap map;
  const cuuint64_t dims[2] = {(cuuint64_t)box_w, (cuuint64_t)b_rows};
  const cuuint64_t strides[1] = {(cuuint64_t)stride};
  const cuuint32_t box[2] = {(cuuint32_t)box_w, 1};  // one row per box: gather4 fetches four
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r =
      enc(&map, sizeof(TIn) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16,
          2, const_cast<TIn*>(B), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
          CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return ABG_OK;
  const int slot_bytes = (int)round_up(4 * row_bytes, 128);
  const int slots = std::max(2, std::min(32, kTmaRingBytes / slot_bytes));
  const int warp_bytes = (int)round_up(slots * slot_bytes + 4 * kTaskEdges * 4 + slots * 8, 1024);
  const size_t smem = (size_t)kTmaWarps * warp_bytes;
  if (smem > 220 * 1024) return ABG_OK;
  ABG_TRY(raise_smem_limit((const void*)k_spmm_tma<V, TIn, false>, smem));
  ABG_TRY(raise_smem_limit((const void*)k_spmm_tma<V, TIn, true>, smem));
  const TmaItems items{sc.etasks, sc.chunk_begin, sc.chunk_row_slot, sc.heavy_row};
  if (sc.n_chunks > 0) {  // raw partial sums of the heavy rows' chunks
    const EpiParams raw{0, 1.f, 0.f, 0.f, nullptr, 0, 0, ep.d};
    const int64_t blocks = std::min<int64_t>(ceil_div(sc.n_chunks, kTmaWarps), num_sms());
    k_spmm_tma<V, TIn, true><<<(unsigned)blocks, kTmaWarps * 32, smem, s>>>(
        map, items, sc.n_chunks, ptr, col, val, part, ldp, nchunk, row_bytes, slot_bytes, slots,
        warp_bytes, raw, wait_err, test_wait_expiry());
    ::abg::note_launch();
  }
  if (sc.n_etasks > 0) {
    const int64_t blocks = std::min<int64_t>(ceil_div(sc.n_etasks, kTmaWarps), num_sms());
    k_spmm_tma<V, TIn, false><<<(unsigned)blocks, kTmaWarps * 32, smem, s>>>(
        map, items, sc.n_etasks, ptr, col, val, C, ldc, nchunk, row_bytes, slot_bytes, slots,
        warp_bytes, ep, wait_err, test_wait_expiry());
    ::abg::note_launch();
  }
  ABG_LAUNCH_CHECK();
  *used = true;
  return ABG_OK;
}

// Light-task variants of one product (rows of 17..64 float4 chunks, where all three apply):
//   0  TMA gather4 ring (k_spmm_tma)          1  register gathers, one warp per task
//   2  a lane group per row over all tasks (k_spmm_stream), heavy chunks by k_spmm_chunks
// Every variant sums each row's edges in edge order, so they give the same bits.
enum SpmmVariant { kVarTma = 0, kVarWarp = 1, kVarRows = 2 };

template <int G, int V, class TIn>
static int run_variant(int vid, bool* ran, const abg_graph::Schedule* sc, const int32_t* rows,
                       int64_t n_rows, const int64_t* ptr, const int32_t* col, const float* val,
                       const TIn* B, int64_t ldb, int64_t b_rows, float* C, int64_t ldc,
                       int nchunk, const EpiParams& ep, float* part, int64_t ldp, int* wait_err,
                       cudaStream_t s) {
  *ran = true;
  bool light = false;  // light tasks with edges and the heavy chunks are done
  if constexpr (G == 32 && V <= 2) {
    if (sc && vid == kVarTma) {
      const int st = run_spmm_tma<V, TIn>(*sc, ptr, col, val, B, ldb, b_rows, C, ldc, nchunk, ep,
                                          part, ldp, wait_err, s, &light);
      if (st != ABG_OK) return st;
      if (!light) {  // the TMA path declined this shape
        *ran = false;
        return ABG_OK;
      }
    }
    if (sc && vid == kVarWarp) {  // register gathers, one warp per item
      constexpr int U = ABG_WARP_UNR, MB = ABG_WARP_MINB;
      const SpmmItems items{sc->etasks, sc->chunk_begin, sc->chunk_row_slot, sc->heavy_row};
      if (sc->n_chunks > 0) {
        const EpiParams raw{0, 1.f, 0.f, 0.f, nullptr, 0, 0, ep.d};
        k_spmm_warp<V, TIn, true, 0, U, MB><<<(unsigned)ceil_div(sc->n_chunks, 8), 256, 0, s>>>(
            items, sc->n_chunks, ptr, col, val, B, (int)ldb, part, (int)ldp, nchunk, raw);
        ::abg::note_launch();
      }
      if (sc->n_etasks > 0) {
        const unsigned grid = (unsigned)ceil_div(sc->n_etasks, 8);
        if (ep.mode == 0)
          k_spmm_warp<V, TIn, false, 0, U, MB><<<grid, 256, 0, s>>>(
              items, sc->n_etasks, ptr, col, val, B, (int)ldb, C, (int)ldc, nchunk, ep);
        else if (ep.mode == 1)
          k_spmm_warp<V, TIn, false, 1, U, MB><<<grid, 256, 0, s>>>(
              items, sc->n_etasks, ptr, col, val, B, (int)ldb, C, (int)ldc, nchunk, ep);
        else
          k_spmm_warp<V, TIn, false, 2, U, MB><<<grid, 256, 0, s>>>(
              items, sc->n_etasks, ptr, col, val, B, (int)ldb, C, (int)ldc, nchunk, ep);
        ::abg::note_launch();
      }
      light = true;
    }
  }
  if (light) {
    if (sc->n_ztasks > 0) {
      k_spmm_stream<G, V, TIn><<<blocks_for(sc->n_ztasks, G), 256, 0, s>>>(
          sc->ztasks, sc->n_ztasks, ptr, col, val, B, ldb, C, ldc, nchunk, ep); ::abg::note_launch();
    }
  } else if (sc && sc->n_tasks > 0) {
    k_spmm_stream<G, V, TIn><<<blocks_for(sc->n_tasks, G), 256, 0, s>>>(
        sc->tasks, sc->n_tasks, ptr, col, val, B, ldb, C, ldc, nchunk, ep); ::abg::note_launch();
  } else if (!sc && n_rows > 0) {
    k_spmm_rows<G, V, TIn><<<blocks_for(n_rows, G), 256, 0, s>>>(rows, n_rows, ptr, col, val, B,
                                                                 ldb, C, ldc, nchunk, ep); ::abg::note_launch();
  }
  if (sc && sc->n_chunks > 0) {
    if (!light) {
      k_spmm_chunks<G, V, TIn><<<blocks_for(sc->n_chunks, G), 256, 0, s>>>(
          sc->chunk_begin, sc->chunk_row_slot, sc->heavy_row, sc->n_chunks, ptr, col, val, B, ldb,
          part, ldp, nchunk); ::abg::note_launch();
    }
    k_spmm_reduce<G, V><<<blocks_for(sc->n_heavy, G), 256, 0, s>>>(
        sc->heavy_row, sc->heavy_chunk0, sc->n_heavy, part, ldp, C, ldc, nchunk, ep); ::abg::note_launch();
  }
  ABG_LAUNCH_CHECK();
  return ABG_OK;
}

// ---------------------------------------------------------------------------
// SpMM autotuner: the first product of a shape (the schedule's task, edge-task and chunk
// counts, the row width and the operand type) runs every variant twice and times the second
// run with CUDA events on its stream; later products of that shape, in this graph or another
// one of the same structure (the same graph uploaded again), use the fastest. The outputs are
// the same bits whichever variant runs, so the choice only moves time. Products with fewer
// than kTuneMinItems tasks and chunks (where the measuring would cost more than it can save)
// and ABG_AUTOTUNE=0 in the environment keep the fixed order (TMA ring, else register
// gathers).
// ---------------------------------------------------------------------------
namespace {
struct TuneKey {
  int64_t n_tasks, n_etasks, n_chunks;
  int nchunk, tsize;
  bool operator<(const TuneKey& o) const {
    if (n_tasks != o.n_tasks) return n_tasks < o.n_tasks;
    if (n_etasks != o.n_etasks) return n_etasks < o.n_etasks;
    if (n_chunks != o.n_chunks) return n_chunks < o.n_chunks;
    if (nchunk != o.nchunk) return nchunk < o.nchunk;
    return tsize < o.tsize;
  }
};
constexpr size_t kTuneCap = 4096;  // shapes remembered (the table is cleared beyond this)
constexpr int64_t kTuneMinItems = 1 << 15;
std::mutex g_tune_mu;
std::map<TuneKey, int> g_tune;
std::atomic<int64_t> g_tuned{0};  // shapes measured

bool autotune_enabled() {
  const char* e = std::getenv("ABG_AUTOTUNE");
  return !(e && e[0] == '0');
}
}  // namespace

template <int G, int V, class TIn>
static int run_spmm(const abg_graph::Schedule* sc, const int32_t* rows, int64_t n_rows,
                    const int64_t* ptr, const int32_t* col, const float* val, const TIn* B,
                    int64_t ldb, int64_t b_rows, float* C, int64_t ldc, int nchunk,
                    const EpiParams& ep, float* part, int64_t ldp, int* wait_err, cudaStream_t s) {
  bool ran = false;
  auto run = [&](int vid) {
    return run_variant<G, V, TIn>(vid, &ran, sc, rows, n_rows, ptr, col, val, B, ldb, b_rows, C,
                                  ldc, nchunk, ep, part, ldp, wait_err, s);
  };
  if constexpr (G == 32 && V <= 2) {
    if (sc && sc->n_etasks + sc->n_chunks > 0) {
      if (!autotune_enabled() || sc->n_etasks + sc->n_chunks < kTuneMinItems) {
        ABG_TRY(run(kVarTma));
        return ran ? ABG_OK : run(kVarWarp);
      }
      const TuneKey key{sc->n_tasks, sc->n_etasks, sc->n_chunks, nchunk, (int)sizeof(TIn)};
      std::lock_guard<std::mutex> lock(g_tune_mu);
      const auto it = g_tune.find(key);
      if (it != g_tune.end()) return run(it->second);
      cudaEvent_t e0, e1;
      ABG_CUDA(cudaEventCreate(&e0));
      ABG_CUDA(cudaEventCreate(&e1));
      int best = kVarWarp;
      float best_ms = INFINITY;
      int st = ABG_OK;
      for (int vid : {kVarTma, kVarWarp, kVarRows}) {
        if ((st = run(vid)) != ABG_OK) break;  // warm-up run (and: does the variant apply?)
        if (!ran) continue;
        cudaEventRecord(e0, s);
        if ((st = run(vid)) != ABG_OK) break;
        cudaEventRecord(e1, s);
        float ms = 0.f;
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) !=
                                                           cudaSuccess) {
          st = ABG_EDEVICE;
          set_error("SpMM autotuner: timing failed");
          break;
        }
        if (ms < best_ms) {
          best_ms = ms;
          best = vid;
        }
      }
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      if (st != ABG_OK) return st;
      if (g_tune.size() >= kTuneCap) g_tune.clear();
      g_tune[key] = best;
      g_tuned.fetch_add(1);
      return run(best);  // the output of the chosen variant (the same bits as any other)
    }
  }
  return run(kVarRows);
}

template <class TIn>
static int dispatch_spmm(const abg_graph::Schedule* sc, const int32_t* rows, int64_t n_rows,
                         const int64_t* ptr, const int32_t* col, const float* val, const TIn* B,
                         int64_t ldb, int64_t b_rows, float* C, int64_t ldc, int nchunk,
                         const EpiParams& ep, float* part, int64_t ldp, int* wait_err,
                         cudaStream_t s) {
  Shape sh = shape_for(nchunk);
#define ABG_SPMM_CASE(g, v)                                                                     \
  if (sh.G == g && sh.V == v)                                                                   \
    return run_spmm<g, v, TIn>(sc, rows, n_rows, ptr, col, val, B, ldb, b_rows, C, ldc, nchunk, \
                               ep, part, ldp, wait_err, s);
  ABG_SPMM_CASE(4, 1)
  ABG_SPMM_CASE(8, 1)
  ABG_SPMM_CASE(16, 1)
  ABG_SPMM_CASE(32, 1)
  ABG_SPMM_CASE(32, 2)
  ABG_SPMM_CASE(32, 4)
  ABG_SPMM_CASE(32, 8)
#undef ABG_SPMM_CASE
  set_error("internal: no SpMM shape");
  return ABG_EINVAL;
}

static int run_scale_rows(int64_t n_rows, float* C, int64_t ldc, int nchunk, const EpiParams& ep,
                          cudaStream_t s) {
  Shape sh = shape_for(nchunk);
#define ABG_SCALE_CASE(g, v) \
  if (sh.G == g && sh.V == v) { k_scale_rows<g, v><<<blocks_for(n_rows, g), 256, 0, s>>>(n_rows, C, ldc, nchunk, ep); ::abg::note_launch(); }
  ABG_SCALE_CASE(4, 1)
  ABG_SCALE_CASE(8, 1)
  ABG_SCALE_CASE(16, 1)
  ABG_SCALE_CASE(32, 1)
  ABG_SCALE_CASE(32, 2)
  ABG_SCALE_CASE(32, 4)
  ABG_SCALE_CASE(32, 8)
#undef ABG_SCALE_CASE
  ABG_LAUNCH_CHECK();
  return ABG_OK;
}

int propagate(const abg_graph* g, const float* x_f32, const __nv_bfloat16* x_bf16, int64_t ldx,
              int d, double alpha, int gamma, float* zhat, int64_t ldz, cudaStream_t s,
              bool bf16_rounds) {
  ABG_CHECK(d >= 1 && d <= kMaxD, "propagate: need 1 <= d <= %d", kMaxD);
  ABG_CHECK(gamma >= 0, "propagate: gamma < 0");
  ABG_CHECK(alpha >= 0.0 && alpha < 1.0, "propagate: need 0 <= alpha < 1");
  ABG_CHECK((x_f32 != nullptr) != (x_bf16 != nullptr), "propagate: exactly one attribute matrix");
  ABG_CHECK(ldx >= d && ldz >= d && ldz % 4 == 0 && ldx % 4 == 0,
            "propagate: leading dimensions must be >= d and multiples of 4");
  const int nchunk = (d + 3) / 4;
  EpiParams ep_restart{1, 1.f, (float)(1.0 - alpha), (float)alpha,
                       x_f32 ? (const void*)x_f32 : (const void*)x_bf16, x_bf16 != nullptr, ldx, d};
  if (gamma == 0) {
    EpiParams ep = ep_restart;
    ep.mode = 2;
    return run_scale_rows(g->n_u, zhat, ldz, nchunk, ep, s);
  }
  Scratch scr(s);
  const int64_t ldw = round_up(d, 4);   // FP32 rows (and the heavy-row partials)
  const int64_t ldh = round_up(d, 8);   // BF16 rows (16-byte aligned)
  float* W = nullptr;
  __nv_bfloat16 *Wb = nullptr, *Zb = nullptr;
  if (bf16_rounds) {  // W and the intermediate Z stored in BF16, accumulated in FP32
    ABG_TRY(scr.get(&Wb, (size_t)g->n_v * ldh));
    if (gamma > 1) ABG_TRY(scr.get(&Zb, (size_t)g->n_u * ldh));
  } else {
    ABG_TRY(scr.get(&W, (size_t)g->n_v * ldw));
  }
  int64_t nparts = std::max<int64_t>(1, std::max(g->sched_u.n_chunks, g->sched_v.n_chunks));
  float* part;
  ABG_TRY(scr.get(&part, (size_t)nparts * ldw));
  float* Wout = bf16_rounds ? reinterpret_cast<float*>(Wb) : W;
  const int64_t ldwo = bf16_rounds ? ldh : ldw;
  for (int it = 0; it < gamma; ++it) {
    // W = L^T Z   (Z_0 = (1-a) X gathered straight from the attributes)
    EpiParams ev{0, it == 0 ? (float)(1.0 - alpha) : 1.f, 0.f, 0.f, nullptr, 0, 0, d,
                 bf16_rounds ? 1 : 0};
    if (it == 0 && x_bf16)
      ABG_TRY(dispatch_spmm<__nv_bfloat16>(&g->sched_v, nullptr, 0, g->v_ptr, g->v_col, g->v_val,
                                           x_bf16, ldx, g->n_u, Wout, ldwo, nchunk, ev, part, ldw,
                                           g->wait_err, s));
    else if (it == 0)
      ABG_TRY(dispatch_spmm<float>(&g->sched_v, nullptr, 0, g->v_ptr, g->v_col, g->v_val, x_f32,
                                   ldx, g->n_u, Wout, ldwo, nchunk, ev, part, ldw, g->wait_err, s));
    else if (bf16_rounds)
      ABG_TRY(dispatch_spmm<__nv_bfloat16>(&g->sched_v, nullptr, 0, g->v_ptr, g->v_col, g->v_val,
                                           Zb, ldh, g->n_u, Wout, ldwo, nchunk, ev, part, ldw,
                                           g->wait_err, s));
    else
      ABG_TRY(dispatch_spmm<float>(&g->sched_v, nullptr, 0, g->v_ptr, g->v_col, g->v_val, zhat,
                                   ldz, g->n_u, Wout, ldwo, nchunk, ev, part, ldw, g->wait_err, s));
    // Z = (1-a) X + a L W   (+ Eq. 2 on the last round, always written in FP32)
    const bool last = it == gamma - 1;
    EpiParams eu = ep_restart;
    eu.mode = last ? 2 : 1;
    eu.out_bf16 = bf16_rounds && !last;
    float* Zout = eu.out_bf16 ? reinterpret_cast<float*>(Zb) : zhat;
    const int64_t ldzo = eu.out_bf16 ? ldh : ldz;
    if (bf16_rounds)
      ABG_TRY(dispatch_spmm<__nv_bfloat16>(&g->sched_u, nullptr, 0, g->u_ptr, g->u_col, g->u_val,
                                           Wb, ldh, g->n_v, Zout, ldzo, nchunk, eu, part, ldw,
                                           g->wait_err, s));
    else
      ABG_TRY(dispatch_spmm<float>(&g->sched_u, nullptr, 0, g->u_ptr, g->u_col, g->u_val, W, ldw,
                                   g->n_v, Zout, ldzo, nchunk, eu, part, ldw, g->wait_err, s));
  }
  return ABG_OK;
}

int check_wait_flag(const abg_graph* g, cudaStream_t s) {
  int flag = 0, tc = 0;
  ABG_CUDA(cudaMemcpyAsync(&flag, g->wait_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  ABG_TRY(tc_wait_flag(s, &tc));  // synchronises s
  if (flag == 0 && tc == 0) return ABG_OK;
  if (flag) {
    ABG_CUDA(cudaMemsetAsync(g->wait_err, 0, sizeof(int), s));
    ABG_CUDA(cudaStreamSynchronize(s));
  }
  set_error("a bounded wait in the %s pipeline ran out; its results are invalid",
            flag ? "SpMM gather" : "tensor-core GEMM");
  return ABG_EDEVICE;
}

int spmm_plain(const int64_t* ptr, const int32_t* col, const float* val, int64_t rows,
               const float* B, int64_t ldb, int n, float* C, int64_t ldc, cudaStream_t s) {
  ABG_CHECK(n >= 1 && n <= kMaxD, "spmm: width out of range");
  EpiParams ep{0, 1.f, 0.f, 0.f, nullptr, 0, 0, n};
  return dispatch_spmm<float>(nullptr, nullptr, rows, ptr, col, val, B, ldb, 0, C, ldc,
                              (n + 3) / 4, ep, nullptr, 0, nullptr, s);
}

__global__ void k_csr_to_dense(const int64_t* __restrict__ ptr, const int32_t* __restrict__ col,
                               const float* __restrict__ val, int64_t rows,
                               float* __restrict__ dense, int64_t ld) {
  int64_t r = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  if (r >= rows) return;
  for (int64_t j = ptr[r] + (threadIdx.x & 31); j < ptr[r + 1]; j += 32)
    atomicAdd(dense + r * ld + col[j], val[j]);  // duplicates add up, as in a sparse sum
}

int csr_to_dense(const int64_t* ptr, const int32_t* col, const float* val, int64_t rows, int cols,
                 float* dense, int64_t ld, cudaStream_t s) {
  ABG_CUDA(cudaMemsetAsync(dense, 0, sizeof(float) * ld * rows, s));
  k_csr_to_dense<<<ceil_div(rows, 8), 256, 0, s>>>(ptr, col, val, rows, dense, ld); ::abg::note_launch();
  ABG_LAUNCH_CHECK();
  return ABG_OK;
}

__global__ void k_bf16_to_f32(const __nv_bfloat16* __restrict__ x, int64_t ldx, int64_t rows,
                              int cols, float* __restrict__ out, int64_t ldo) {
  int64_t total = rows * (int64_t)cols;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    int64_t r = t / cols;
    int c = (int)(t - r * cols);
    out[r * ldo + c] = __bfloat162float(x[r * ldx + c]);
  }
}

int bf16_to_f32(const __nv_bfloat16* x, int64_t ldx, int64_t rows, int cols, float* out,
                int64_t ldo, cudaStream_t s) {
  k_bf16_to_f32<<<num_sms() * 8, 256, 0, s>>>(x, ldx, rows, cols, out, ldo); ::abg::note_launch();
  ABG_LAUNCH_CHECK();
  return ABG_OK;
}

__global__ void k_f32_to_bf16(const float* __restrict__ x, int64_t ldx, int64_t rows, int cols,
                              __nv_bfloat16* __restrict__ out, int64_t ldo) {
  int64_t total = rows * (int64_t)cols;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    int64_t r = t / cols;
    int c = (int)(t - r * cols);
    out[r * ldo + c] = __float2bfloat16_rn(x[r * ldx + c]);
  }
}

int f32_to_bf16(const float* x, int64_t ldx, int64_t rows, int cols, __nv_bfloat16* out,
                int64_t ldo, cudaStream_t s) {
  k_f32_to_bf16<<<num_sms() * 8, 256, 0, s>>>(x, ldx, rows, cols, out, ldo); ::abg::note_launch();
  ABG_LAUNCH_CHECK();
  return ABG_OK;
}

}  // namespace abg

extern "C" ABG_API int64_t abg_spmm_tuned_shapes(void) { return abg::g_tuned.load(); }
