// Algorithm 1 propagation: gamma rounds of the two chained sparse products
//   W = L_U^T Z            (CSC rows = V nodes)
//   Z = (1-a) X + a L_U W  (CSR rows = U nodes, restart fused in the epilogue)
// followed by the row normalisation of Eq. 2 fused into the last round.
//
// Kernel shape: a group of G lanes owns one output row; each lane owns V
// float4 column chunks of that row, so one gathered input row is read with
// G*V coalesced 16-byte loads. The group loads up to G (index, value) pairs
// cooperatively, broadcasts them with shuffles and keeps 8 gathers in flight.
// Light rows run in decreasing-degree order; rows with more than kHeavyRow
// edges are split into kHeavyChunk-edge chunks whose partial sums go to a
// scratch buffer and are added back in chunk order, so results do not depend
// on scheduling (no floating-point atomics).
#include "internal.cuh"

namespace abg {

struct EpiParams {
  int mode;          // 0: C = scale*acc   1: restart   2: restart + Eq. 2 normalisation
  float scale;       // mode 0
  float c_x, c_p;    // modes 1/2: C = c_x * X + c_p * acc
  const void* x;     // restart attributes (float or bf16), row stride ldx
  int x_bf16;
  int64_t ldx;
  int d;             // row width: components at or beyond d are treated as 0 and written as 0
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

template <int G, int V>
__device__ __forceinline__ void epilogue_store(int64_t row, const float4 (&acc_in)[V], float* C,
                                               int64_t ldc, int nchunk, int lig, unsigned mask,
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
      int ch = lig + G * v;
      float4 xv = make_float4(0.f, 0.f, 0.f, 0.f);
      if (ch < nchunk) {
        if (ep.x_bf16)
          xv = ld_bf16x4(reinterpret_cast<const __nv_bfloat16*>(ep.x) + row * ep.ldx + 4 * ch);
        else
          xv = ld_nc_f4(reinterpret_cast<const float*>(ep.x) + row * ep.ldx + 4 * ch);
        xv = mask_tail(xv, ch, ep.d);
      }
      float4 z;
      z.x = fmaf(ep.c_p, acc[v].x, ep.c_x * xv.x);
      z.y = fmaf(ep.c_p, acc[v].y, ep.c_x * xv.y);
      z.z = fmaf(ep.c_p, acc[v].z, ep.c_x * xv.z);
      z.w = fmaf(ep.c_p, acc[v].w, ep.c_x * xv.w);
      out[v] = z;
      ss += z.x * z.x + z.y * z.y + z.z * z.z + z.w * z.w;
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
    if (ch < nchunk) st_f4(C + row * ldc + 4 * ch, out[v]);
  }
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
  for (int64_t c = heavy_chunk0[grp]; c < heavy_chunk0[grp + 1]; ++c) {
#pragma unroll
    for (int v = 0; v < V; ++v) {
      int ch = lig + G * v;
      if (ch < nchunk) {
        float4 p = ld_f4(part + c * ldp + 4 * ch);
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

template <int G, int V, class TIn>
static int run_spmm(const abg_graph::Schedule* sc, const int32_t* rows, int64_t n_rows,
                    const int64_t* ptr, const int32_t* col, const float* val, const TIn* B,
                    int64_t ldb, float* C, int64_t ldc, int nchunk, const EpiParams& ep,
                    float* part, int64_t ldp, cudaStream_t s) {
  if (n_rows > 0) {
    k_spmm_rows<G, V, TIn><<<blocks_for(n_rows, G), 256, 0, s>>>(rows, n_rows, ptr, col, val, B,
                                                                 ldb, C, ldc, nchunk, ep); ::abg::note_launch();
  }
  if (sc && sc->n_chunks > 0) {
    k_spmm_chunks<G, V, TIn><<<blocks_for(sc->n_chunks, G), 256, 0, s>>>(
        sc->chunk_begin, sc->chunk_row_slot, sc->heavy_row, sc->n_chunks, ptr, col, val, B, ldb,
        part, ldp, nchunk); ::abg::note_launch();
    k_spmm_reduce<G, V><<<blocks_for(sc->n_heavy, G), 256, 0, s>>>(
        sc->heavy_row, sc->heavy_chunk0, sc->n_heavy, part, ldp, C, ldc, nchunk, ep); ::abg::note_launch();
  }
  ABG_LAUNCH_CHECK();
  return ABG_OK;
}

template <class TIn>
static int dispatch_spmm(const abg_graph::Schedule* sc, const int32_t* rows, int64_t n_rows,
                         const int64_t* ptr, const int32_t* col, const float* val, const TIn* B,
                         int64_t ldb, float* C, int64_t ldc, int nchunk, const EpiParams& ep,
                         float* part, int64_t ldp, cudaStream_t s) {
  Shape sh = shape_for(nchunk);
#define ABG_SPMM_CASE(g, v)                                                                      \
  if (sh.G == g && sh.V == v)                                                                    \
    return run_spmm<g, v, TIn>(sc, rows, n_rows, ptr, col, val, B, ldb, C, ldc, nchunk, ep, part, \
                               ldp, s);
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
              int d, double alpha, int gamma, float* zhat, int64_t ldz, cudaStream_t s) {
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
  const int64_t ldw = round_up(d, 4);
  float* W;
  ABG_TRY(scr.get(&W, (size_t)g->n_v * ldw));
  int64_t nparts = std::max<int64_t>(1, std::max(g->sched_u.n_chunks, g->sched_v.n_chunks));
  float* part;
  ABG_TRY(scr.get(&part, (size_t)nparts * ldw));
  for (int it = 0; it < gamma; ++it) {
    // W = L^T Z   (Z_0 = (1-a) X gathered straight from the attributes)
    if (it == 0) {
      EpiParams ep{0, (float)(1.0 - alpha), 0.f, 0.f, nullptr, 0, 0, d};
      if (x_bf16)
        ABG_TRY(dispatch_spmm<__nv_bfloat16>(&g->sched_v, g->sched_v.light, g->sched_v.n_light,
                                             g->v_ptr, g->v_col, g->v_val, x_bf16, ldx, W, ldw,
                                             nchunk, ep, part, ldw, s));
      else
        ABG_TRY(dispatch_spmm<float>(&g->sched_v, g->sched_v.light, g->sched_v.n_light, g->v_ptr,
                                     g->v_col, g->v_val, x_f32, ldx, W, ldw, nchunk, ep, part,
                                     ldw, s));
    } else {
      EpiParams ep{0, 1.f, 0.f, 0.f, nullptr, 0, 0, d};
      ABG_TRY(dispatch_spmm<float>(&g->sched_v, g->sched_v.light, g->sched_v.n_light, g->v_ptr,
                                   g->v_col, g->v_val, zhat, ldz, W, ldw, nchunk, ep, part, ldw,
                                   s));
    }
    // Z = (1-a) X + a L W   (+ Eq. 2 on the last round)
    EpiParams ep = ep_restart;
    ep.mode = (it == gamma - 1) ? 2 : 1;
    ABG_TRY(dispatch_spmm<float>(&g->sched_u, g->sched_u.light, g->sched_u.n_light, g->u_ptr,
                                 g->u_col, g->u_val, W, ldw, zhat, ldz, nchunk, ep, part, ldw, s));
  }
  return ABG_OK;
}

int spmm_plain(const int64_t* ptr, const int32_t* col, const float* val, int64_t rows,
               const float* B, int64_t ldb, int n, float* C, int64_t ldc, cudaStream_t s) {
  ABG_CHECK(n >= 1 && n <= kMaxD, "spmm: width out of range");
  EpiParams ep{0, 1.f, 0.f, 0.f, nullptr, 0, 0, n};
  return dispatch_spmm<float>(nullptr, nullptr, rows, ptr, col, val, B, ldb, C, ldc, (n + 3) / 4,
                              ep, nullptr, 0, s);
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

}  // namespace abg
