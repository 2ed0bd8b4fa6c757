// Tall-skinny products C = A B_s on the 5th-generation tensor cores
// (tcgen05.mma kind::tf32, accumulator in tensor memory).
//
// A (rows x K, fp32, row-major) is the tall operand, B_s (K x N per segment)
// the small one. One CTA computes a 128-row tile (one UMMA M) for the tile's
// segment, streaming K in 32-column blocks (one 128-byte swizzle row) through
// a ring of shared-memory stages:
//   warp 0      TMA producer: A block, B_hi and B_lo blocks (128B swizzle)
//   warp 1      allocates tensor memory; one thread issues the MMAs
//   warps 2..5  split the A block in place into tf32 hi and lo parts
//   warps 6..9  epilogue (tcgen05.ld of their 32-lane quarter of TMEM)
// The kernel is persistent (one CTA per SM walks its tiles) with two TMEM
// accumulators, so a tile's MMAs overlap the previous tile's epilogue.
// Three-term split (the usual 3xTF32 scheme): x = hi + lo with
// hi = rna_tf32(x), lo = rna_tf32(x - hi), and A B ~ hi(A) hi(B) + lo(A) hi(B)
// + hi(A) lo(B); both parts are exact tf32 values, so the operand precision is
// about 2^-21 relative, with fp32 accumulation. B_hi / B_lo are prepared once
// per call by a small kernel (transposed to K-major, zero outside K_s x N_s).
// Every mbarrier wait is bounded; a wait that runs out sets a device flag
// (read by tc_wait_flag) and the CTA still frees its tensor memory.
//
// BF16 variants (tcgen05.mma kind::f16, fp32 accumulation) serve products whose
// tall operand is stored in BF16 (the random-feature matrix R when BF16
// contractions are selected): k_tc_nn16 takes the A tile from TMA as is (no
// split warps) with B rounded to BF16 once and kept in shared memory;
// k_tc_tn16 reads the A rows as MN-major operand tiles straight from TMA and
// only rounds the fp32 B rows to BF16 (no transpose).
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "batch.cuh"
#include "internal.cuh"
#include "tma.cuh"

namespace abg {

namespace {

constexpr int kTcM = 128;        // rows per tile = UMMA M
constexpr int kTcBK = 32;        // K per stage (fp32: one 128-byte swizzle row)
constexpr int kTcThreads = 320;  // 10 warps
constexpr uint32_t kTcABytes = kTcM * kTcBK * 4;  // 16 KiB

__device__ int g_tc_wait_err = 0;

struct TcArgs {
  int nkb;       // K blocks
  int Np;        // UMMA N (multiple of 16, <= 256)
  int N, K;      // largest N_s, K_s
  const int* segN;
  const int* segK;
  const int* tile_seg;
  const int64_t* tile_row0;
  const int* tile_rows;
  float* C;
  int64_t ldc;
  int epi;
  const float* aux;
  int64_t ldaux;
  const float* aux2;
  int64_t ldaux2;
  const float* sign;
  int64_t sign_seg;
  int32_t* labels;
  float* margin;
  int first;
  int* changes;
  unsigned* minbits;
  int stages;
  uint32_t stage_bytes;
  uint32_t b_bytes;
  uint32_t tmem_cols;
  int b_resident;  // BF16 kernel: all K blocks of B stay in shared memory (one segment)
  int aux_vec;     // aux / aux2 rows start on 16 bytes (the Phi rule loads them 4 at a time)
  int* wait_err;   // device flag of the solve (or the process-wide one): a wait ran out
  // random features (Eq. 13): C[i][n] = out_scale sin(in_scale acc), C[i][N + n] = ... cos,
  // and per-tile FP64 column sums of both halves into colsum[tile][2N]
  int sincos;
  float in_scale, out_scale;
  double* colsum;
};

// x rounded to tf32 (10 explicit mantissa bits), to nearest with ties away from zero, as an
// fp32 bit pattern with the low 13 bits zero: half a tf32 ulp (bit 12) is added to the
// magnitude bits and the rest truncated (a carry moves into the exponent as it should).
// Integer add and mask run at full rate, unlike the conversion instruction.
__device__ __forceinline__ float rna_tf32(float x) {
  return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row atoms 1024 bytes apart
__device__ __forceinline__ uint64_t sw128_desc(uint32_t addr) {
  uint64_t d = (uint64_t)((addr >> 4) & 0x3FFFu);  // start address
  d |= (uint64_t)1 << 16;                          // leading byte offset (unused when swizzled)
  d |= (uint64_t)(1024 >> 4) << 32;                // stride byte offset: next 8-row atom
  d |= (uint64_t)1 << 46;                          // descriptor version
  d |= (uint64_t)2 << 61;                          // layout: 128-byte swizzle
  return d;
}

// instruction descriptor: D f32, A/B tf32, both K-major, M = 128, N = n
__host__ __device__ constexpr uint32_t tf32_idesc(int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(kTcM >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

// the same MMA with A (128 lanes x 8 tf32 columns) read from tensor memory
__device__ __forceinline__ void mma_tf32_ta(uint32_t tmem_d, uint32_t tmem_a, uint64_t b,
                                            uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n\t}" ::"r"(tmem_d),
      "r"(tmem_a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

// instruction descriptor: D f32, A/B bf16, M = 128, N = n; a_mn / b_mn: operand is MN-major
__host__ __device__ constexpr uint32_t bf16_idesc(int n, bool a_mn, bool b_mn) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((a_mn ? 1u : 0u) << 15) |
         ((b_mn ? 1u : 0u) << 16) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kTcM >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

// shared-memory matrix descriptor, MN-major with 128-byte swizzle: each K row holds 64 bf16
// of the MN dimension in 128 bytes, 8 K rows form a 1024-byte atom (the next 8 K rows 1024
// bytes on), and the next 64 MN elements start lbo bytes on
__device__ __forceinline__ uint64_t sw128_mn_desc(uint32_t addr, uint32_t lbo) {
  uint64_t d = (uint64_t)((addr >> 4) & 0x3FFFu);  // start address
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;     // leading byte offset: next 64 MN elements
  d |= (uint64_t)(1024 >> 4) << 32;                // stride byte offset: next 8 K rows
  d |= (uint64_t)1 << 46;                          // descriptor version
  d |= (uint64_t)2 << 61;                          // layout: 128-byte swizzle
  return d;
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// 32 consecutive fp32 columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, "
      "%30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// B_hi / B_lo (segment s rows s*Np .. s*Np + Np, K-major, Kp columns) from B_s (K x N row-major)
__global__ void k_tc_prep_b(const float* __restrict__ B, int64_t ldb, int64_t b_seg,
                            const int* __restrict__ segK, int K, const int* __restrict__ segN, int N,
                            int Np, int Kp, float* __restrict__ bhi, float* __restrict__ blo) {
  const int sg = blockIdx.y;
  const int Ks = segK ? segK[sg] : K;
  const int Ns = segN ? segN[sg] : N;
  const float* Bs = B + sg * b_seg;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)Np * Kp;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int n = (int)(e / Kp), k = (int)(e % Kp);
    float h = 0.f, l = 0.f;
    if (n < Ns && k < Ks) {
      const float x = Bs[(int64_t)k * ldb + n];
      h = rna_tf32(x);
      l = rna_tf32(x - h);
    }
    const int64_t o = ((int64_t)sg * Np + n) * Kp + k;
    bhi[o] = h;
    blo[o] = l;
  }
}

// 16 / 32 consecutive 32-bit columns of this thread's TMEM lane from registers (complete after
// tmem_wait_st)
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15, %16};" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
      "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]),
      "r"(r[15])
      : "memory");
}
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
      "%28, %29, %30, %31, %32};" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
      "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]),
      "r"(r[15]), "r"(r[16]), "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]),
      "r"(r[22]), "r"(r[23]), "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]),
      "r"(r[29]), "r"(r[30]), "r"(r[31])
      : "memory");
}
__device__ __forceinline__ void tmem_wait_st() {
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// 32 consecutive fp32 columns of this thread's TMEM lane, without waiting: the registers are
// valid only after tmem_wait_ld()
__device__ __forceinline__ void tmem_ld32_async(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, "
      "%30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// One arrival per warp once all its lanes are done (their shared-memory writes fenced to the
// async proxy, or their tensor-memory loads fenced): a barrier sized in warps then sees 32x
// fewer arrivals than one sized in threads, which serialise on the barrier's word.
__device__ __forceinline__ void warp_arrive(uint32_t bar) {
  __syncwarp();
  if ((threadIdx.x & 31) == 0) mbar_arrive(bar);
}

struct Best {
  float v;
  int i;
  float s;
};
// columns arrive in increasing order: a tie keeps the lower index (and sets the margin to 0);
// selects instead of branches, so the lanes of a warp never diverge
__device__ __forceinline__ void push_best(Best& b, float v, int i) {
  const bool gt = v > b.v;
  b.s = gt ? b.v : fmaxf(b.s, v);
  b.i = gt ? i : b.i;
  b.v = gt ? v : b.v;
}

// per-tile epilogue of one accumulator row (this thread's TMEM lane)
template <bool ARGMAX>
__device__ __forceinline__ void tc_epilogue_row(const TcArgs& p, uint32_t tacc, int quad, int lane,
                                                int sg, int64_t row0, int nrows, int Ns) {
  const int r = quad * 32 + lane;
  const int64_t gm = row0 + r;
  const bool valid = r < nrows;
  Best b{-INFINITY, 0x7fffffff, -INFINITY};
  int old_label = -1;  // read before the TMEM loads so the two latencies overlap
  if constexpr (ARGMAX) {
    if (valid && !p.first) old_label = p.labels[gm];
    // the scores of the row (Np <= 128 columns), 64 columns per TMEM wait
    const uint32_t ta = tacc + ((uint32_t)(quad * 32) << 16);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (64 * h >= p.Np) break;  // uniform over the warp
      uint32_t r[2][32];
      tmem_ld32_async(ta + 64 * h, r[0]);
      if (p.Np > 64 * h + 32) tmem_ld32_async(ta + 64 * h + 32, r[1]);
      tmem_wait_ld();
      if (valid) {
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const int col = 64 * h + 32 * c + j;
            if (col < Ns) push_best(b, __uint_as_float(r[c][j]), col);
          }
      }
    }
  }
  for (int c0 = 0; c0 < p.Np && !ARGMAX; c0 += 32) {
    float v[32];
    tmem_ld32(tacc + ((uint32_t)(quad * 32) << 16) + (uint32_t)c0, v);
    if (!valid) continue;
    if (p.epi == (int)Epi::PhiUpdate) {
      // Phi rule (Eq. 17): this row's P and Phi values of the chunk are all requested before
      // any is used (16 at a time, 16-byte loads where four columns are in range), so their
      // memory latencies overlap instead of following one another
      const float* prow = p.aux + gm * p.ldaux + c0;
      const float* qrow = p.aux2 + gm * p.ldaux2 + c0;
#pragma unroll
      for (int h = 0; h < 32; h += 16) {
        float pv[16], ph[16];
#pragma unroll
        for (int j = 0; j < 16; j += 4) {
          const int gn = c0 + h + j;
          if (p.aux_vec && gn + 3 < Ns) {
            const float4 a = *reinterpret_cast<const float4*>(prow + h + j);
            const float4 b = *reinterpret_cast<const float4*>(qrow + h + j);
            pv[j] = a.x, pv[j + 1] = a.y, pv[j + 2] = a.z, pv[j + 3] = a.w;
            ph[j] = b.x, ph[j + 1] = b.y, ph[j + 2] = b.z, ph[j + 3] = b.w;
          } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              pv[j + q] = gn + q < Ns ? prow[h + j + q] : 0.f;
              ph[j + q] = gn + q < Ns ? qrow[h + j + q] : 0.f;
            }
          }
        }
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const float x = v[h + j];
          if (c0 + h + j < Ns) v[h + j] = x > 0.f ? ph[j] * sqrtf(fmaxf(pv[j], 0.f) / x) : 0.f;
        }
      }
    } else {
      // the other epilogues read nothing per element but the sign vector
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const int gn = c0 + j;
        float x = v[j];
        if (gn < Ns) {
          switch (p.epi) {
            case (int)Epi::Relu: x = fmaxf(x, 0.f); break;
            case (int)Epi::SignRelu: x = fmaxf(p.sign[sg * p.sign_seg + gn] * x, 0.f); break;
            case (int)Epi::Sign: x = p.sign[sg * p.sign_seg + gn] * x; break;
            default: break;
          }
        }
        v[j] = x;
      }
    }
    {
      float* crow = p.C + gm * p.ldc;
      // 16-byte stores where four columns are in range (ldc is a multiple of 4)
#pragma unroll
      for (int j = 0; j < 32; j += 4) {
        const int gn = c0 + j;
        if (gn + 3 < Ns) {
          *reinterpret_cast<float4*>(crow + gn) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
        } else {
#pragma unroll
          for (int q = 0; q < 4; ++q)
            if (gn + q < Ns) crow[gn + q] = v[j + q];
        }
      }
    }
  }
  if constexpr (ARGMAX) {
    int changed = 0;
    float mg = INFINITY;
    if (valid) {
      mg = Ns > 1 ? b.v - b.s : INFINITY;
      if (!p.first && old_label != b.i) changed = 1;
      p.labels[gm] = b.i;
      if (p.margin) p.margin[gm] = mg;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      changed += __shfl_xor_sync(0xffffffffu, changed, o);
      mg = fminf(mg, __shfl_xor_sync(0xffffffffu, mg, o));
    }
    if (lane == 0) {
      if (changed) atomicAdd(p.changes + sg, changed);
      if (mg < INFINITY) atomicMin(p.minbits + sg, __float_as_uint(fmaxf(mg, 0.f)));
    }
  }
}

// Reduce-scatter over the warp: afterwards v[0] of lane l holds the sum over all 32 lanes of
// their v[l] (31 shuffles; the additions run in a fixed order).
__device__ __forceinline__ void warp_colsum32(float (&v)[32], int lane) {
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int j = 0; j < o; ++j) {
      const float send = up ? v[j] : v[j + o];
      const float keep = up ? v[j + o] : v[j];
      v[j] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
}

// Random-feature epilogue of one tile (Eq. 13): this thread's row of sin / cos values, and the
// tile's column sums (each warp sums its 32 rows per column in FP32, the four warps' sums are
// added in FP64 in warp order). cs: shared scratch of 4 x 2 Np floats.
__device__ void tc_epilogue_sincos(const TcArgs& p, uint32_t tacc, int quad, int lane, int64_t tile,
                                   int64_t row0, int nrows, float* cs) {
  const int r = quad * 32 + lane;
  const int64_t gm = row0 + r;
  const bool valid = r < nrows;
  const int N = p.N;
  float* crow = p.C + gm * p.ldc;
  for (int c0 = 0; c0 < p.Np; c0 += 32) {
    float v[32];
    tmem_ld32(tacc + ((uint32_t)(quad * 32) << 16) + (uint32_t)c0, v);
    float sn[32], cn[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      sn[j] = 0.f;
      cn[j] = 0.f;
      if (valid && c0 + j < N) {
        float sv, cv;
        sincosf(p.in_scale * v[j], &sv, &cv);
        sn[j] = sv * p.out_scale;
        cn[j] = cv * p.out_scale;
      }
    }
    if (valid) {
      // 16-byte stores where four columns are in range; the cos half starts at column N,
      // so its stores are 16-byte aligned only when N is a multiple of 4
      const bool cos_vec = (N & 3) == 0;
#pragma unroll
      for (int j = 0; j < 32; j += 4) {
        const int gn = c0 + j;
        if (gn + 3 < N) {
          *reinterpret_cast<float4*>(crow + gn) = make_float4(sn[j], sn[j + 1], sn[j + 2], sn[j + 3]);
          if (cos_vec) {
            *reinterpret_cast<float4*>(crow + N + gn) =
                make_float4(cn[j], cn[j + 1], cn[j + 2], cn[j + 3]);
          } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) crow[N + gn + q] = cn[j + q];
          }
        } else {
#pragma unroll
          for (int q = 0; q < 4; ++q)
            if (gn + q < N) {
              crow[gn + q] = sn[j + q];
              crow[N + gn + q] = cn[j + q];
            }
        }
      }
    }
    warp_colsum32(sn, lane);
    warp_colsum32(cn, lane);
    if (c0 + lane < p.Np) {  // the last 32-column load may reach past Np (a multiple of 16)
      cs[quad * 2 * p.Np + c0 + lane] = sn[0];
      cs[quad * 2 * p.Np + p.Np + c0 + lane] = cn[0];
    }
  }
  asm volatile("bar.sync 1, 128;" ::: "memory");  // the four epilogue warps
  for (int c = r; c < 2 * N; c += 128) {
    const int pos = c < N ? c : p.Np + (c - N);
    double sum = 0.0;
#pragma unroll
    for (int q = 0; q < 4; ++q) sum += (double)cs[q * 2 * p.Np + pos];
    p.colsum[tile * 2 * N + c] = sum;
  }
  asm volatile("bar.sync 1, 128;" ::: "memory");  // cs free for the next tile
}

// Persistent: CTA c takes tiles c, c + gridDim.x, ...; the stage ring runs across tile
// boundaries and the accumulator alternates between two TMEM buffers, so the MMAs of a
// tile overlap the epilogue of the previous one.
//   warp 0: TMA producer      warp 1: TMEM owner + MMA issuer
//   warps 2-5: tf32 split     warps 6-9: epilogue (TMEM lane quarter = warp % 4)
// MODE 0: C = acc with the elementwise epilogues; 1: NCI argmax; 2: random features (sin/cos
// and column sums). SPLITW warps split A; EPIG groups of four epilogue warps take the tiles of
// alternate accumulator buffers (group g: buffer g), so a slow epilogue keeps up with the MMAs.
// ATM (N <= 128): the split warps write A's hi and lo parts into tensor memory (one 64-column
// slot per stage after the two 128-column accumulators) and the MMAs read A from there, so
// shared memory carries A once (TMA in, split warps out) instead of three more times (the
// split's two writes and the MMAs' reads of hi and lo).
template <int MODE, int SPLITW, int EPIG, bool ATM>
__global__ void __launch_bounds__(32 * (2 + SPLITW + 4 * EPIG), 1)
    k_tc_nn(const __grid_constant__ CUtensorMap amap, const __grid_constant__ CUtensorMap bhi_map,
            const __grid_constant__ CUtensorMap blo_map, const TcArgs p, int64_t n_tiles) {
  constexpr bool ARGMAX = MODE == 1;
  constexpr int kSplitT = 32 * SPLITW;  // split threads
  static_assert(EPIG == 1 || EPIG == 2, "one or two epilogue groups");
  static_assert(MODE != 2 || EPIG == 1, "the sin/cos epilogue's column sums use one group");
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  __shared__ uint32_t tmem_slot;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int S = p.stages;
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + (size_t)S * p.stage_bytes);
  const uint32_t full0 = smem_addr(bars), split0 = full0 + 8 * S, empty0 = full0 + 16 * S,
                 tfull0 = full0 + 24 * S, tempty0 = tfull0 + 16;
  if (threadIdx.x == 0) {
    for (int i = 0; i < S; ++i) {
      mbar_init(full0 + 8 * i, 1);
      mbar_init(split0 + 8 * i, SPLITW);  // one arrival per split warp
      mbar_init(empty0 + 8 * i, 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(tfull0 + 8 * i, 1);
      mbar_init(tempty0 + 8 * i, 4);  // one arrival per epilogue warp
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(&tmem_slot)),
                 "r"(p.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  const uint32_t acc_cols = ATM ? 128u : p.tmem_cols / 2;  // columns of one accumulator buffer
  const uint32_t a_tm0 = tmem + 2 * acc_cols;                // ATM: A slot of stage s at + 64 s
  const uint32_t boff = (ATM ? 1u : 2u) * kTcABytes;         // B_hi within a stage
  // after a wait has run out anywhere, later CTAs skip their work instead of waiting again
  bool bad = *reinterpret_cast<volatile int*>(p.wait_err) != 0;

  if (warp == 0) {
    if (lane == 0) {  // producer
      int s = 0;
      uint32_t ph = 0;
      int64_t n = 0;  // stages issued so far
      for (int64_t tile = blockIdx.x; tile < n_tiles && !bad; tile += gridDim.x) {
        const int sg = p.tile_seg[tile];
        const int row0 = (int)p.tile_row0[tile];
        for (int kb = 0; kb < p.nkb; ++kb, ++n) {
          if (n >= S && !mbar_wait_bounded(empty0 + 8 * s, ph ^ 1u)) {
            bad = true;
            break;
          }
          const uint32_t st = smem_addr(smem + (size_t)s * p.stage_bytes);
          mbar_expect_tx(full0 + 8 * s, kTcABytes + 2 * p.b_bytes);
          tma_load_2d(st, &amap, kb * kTcBK, row0, full0 + 8 * s);
          tma_load_2d(st + boff, &bhi_map, kb * kTcBK, sg * p.Np, full0 + 8 * s);
          tma_load_2d(st + boff + p.b_bytes, &blo_map, kb * kTcBK, sg * p.Np, full0 + 8 * s);
          if (++s == S) {
            s = 0;
            ph ^= 1u;
          }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {  // MMA issuer
      const uint32_t idesc = tf32_idesc(p.Np);
      int s = 0;
      uint32_t ph = 0;
      int it = 0;
      for (int64_t tile = blockIdx.x; tile < n_tiles && !bad; tile += gridDim.x, ++it) {
        const int bsel = it & 1;
        if (it >= 2 && !mbar_wait_bounded(tempty0 + 8 * bsel, ((it >> 1) - 1) & 1)) {
          bad = true;
          break;
        }
        tc_fence_after();
        const uint32_t tacc = tmem + (uint32_t)bsel * acc_cols;
        for (int kb = 0; kb < p.nkb; ++kb) {
          if (!mbar_wait_bounded(full0 + 8 * s, ph) || !mbar_wait_bounded(split0 + 8 * s, ph)) {
            bad = true;
            break;
          }
          tc_fence_after();
          const uint32_t st = smem_addr(smem + (size_t)s * p.stage_bytes);
          const uint32_t b_hi = st + boff, b_lo = b_hi + p.b_bytes;
          if constexpr (ATM) {
            const uint32_t ta = a_tm0 + 64u * (uint32_t)s;  // hi: columns 0..31, lo: 32..63
#pragma unroll
            for (int j = 0; j < kTcBK / 8; ++j) {  // UMMA K = 8 tf32 = 8 TMEM columns
              const uint32_t off = 32u * j;
              mma_tf32_ta(tacc, ta + 8u * j, sw128_desc(b_hi + off), idesc, (kb | j) != 0);
              mma_tf32_ta(tacc, ta + 32u + 8u * j, sw128_desc(b_hi + off), idesc, 1u);
              mma_tf32_ta(tacc, ta + 8u * j, sw128_desc(b_lo + off), idesc, 1u);
            }
          } else {
            const uint32_t a_hi = st, a_lo = st + kTcABytes;
#pragma unroll
            for (int j = 0; j < kTcBK / 8; ++j) {  // UMMA K = 8 tf32 = 32 bytes
              const uint32_t off = 32u * j;
              mma_tf32(tacc, sw128_desc(a_hi + off), sw128_desc(b_hi + off), idesc,
                       (kb | j) != 0);
              mma_tf32(tacc, sw128_desc(a_lo + off), sw128_desc(b_hi + off), idesc, 1u);
              mma_tf32(tacc, sw128_desc(a_hi + off), sw128_desc(b_lo + off), idesc, 1u);
            }
          }
          mma_commit(empty0 + 8 * s);  // the stage is free once these MMAs have read it
          if (++s == S) {
            s = 0;
            ph ^= 1u;
          }
        }
        if (bad) break;
        mma_commit(tfull0 + 8 * bsel);  // accumulator complete
      }
    }
  } else if (warp < 2 + SPLITW) {
    // split each A block into tf32 hi (in place) and lo parts; zero columns >= K_s
    const int t = threadIdx.x - 64;
    int s = 0;
    uint32_t ph = 0;
    for (int64_t tile = blockIdx.x; tile < n_tiles && !bad; tile += gridDim.x) {
      const int sg = p.tile_seg[tile];
      const int Ks = p.segK ? p.segK[sg] : p.K;
      for (int kb = 0; kb < p.nkb; ++kb) {
        const bool ok = mbar_wait_bounded(full0 + 8 * s, ph);
        if (__any_sync(0xffffffffu, !ok)) {  // the whole warp leaves together
          bad = true;
          break;
        }
        if constexpr (ATM) {
          // this thread's tile row (its TMEM lane) and its share of the stage's 8 chunks; the
          // 128-byte swizzle puts logical chunk j of row r at physical chunk j ^ (r & 7), so
          // eight lanes in a row read eight different chunks
          constexpr int kCh = SPLITW >= 8 ? 4 : 8;
          const int quad = warp & 3, r = 32 * quad + lane;
          const int j0 = SPLITW >= 8 ? ((warp - 2) >> 2) * kCh : 0;
          const unsigned char* arow = smem + (size_t)s * p.stage_bytes + (size_t)r * 128;
          uint32_t hv[4 * kCh], lv[4 * kCh];
#pragma unroll
          for (int c = 0; c < kCh; ++c) {
            const int j = j0 + c;
            const float4 v = *reinterpret_cast<const float4*>(arow + ((j ^ (r & 7)) * 16));
            const int k0 = kb * kTcBK + 4 * j;
            const float x[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const float h = k0 + e < Ks ? rna_tf32(x[e]) : 0.f;
              const float l = k0 + e < Ks ? rna_tf32(x[e] - h) : 0.f;
              hv[4 * c + e] = __float_as_uint(h);
              lv[4 * c + e] = __float_as_uint(l);
            }
          }
          const uint32_t ta = a_tm0 + ((uint32_t)(32 * quad) << 16) + 64u * (uint32_t)s +
                              (uint32_t)(4 * j0);
          if constexpr (kCh == 4) {
            tmem_st16(ta, hv);
            tmem_st16(ta + 32u, lv);
          } else {
            tmem_st32(ta, hv);
            tmem_st32(ta + 32u, lv);
          }
          tmem_wait_st();
          tc_fence_before();  // the MMAs read these columns after the barrier
          warp_arrive(split0 + 8 * s);
          if (++s == S) {
            s = 0;
            ph ^= 1u;
          }
          continue;
        }
        float4* a = reinterpret_cast<float4*>(smem + (size_t)s * p.stage_bytes);
        float4* alo = a + kTcABytes / 16;
#pragma unroll 4
        for (int q = t; q < (int)(kTcABytes / 16); q += kSplitT) {
          const int r = q >> 3;
          const int lc = (q & 7) ^ (r & 7);  // logical 16-byte chunk under the 128-byte swizzle
          const int k0 = kb * kTcBK + lc * 4;
          const float4 v = a[q];
          float4 h, l;
          h.x = k0 < Ks ? rna_tf32(v.x) : 0.f;
          h.y = k0 + 1 < Ks ? rna_tf32(v.y) : 0.f;
          h.z = k0 + 2 < Ks ? rna_tf32(v.z) : 0.f;
          h.w = k0 + 3 < Ks ? rna_tf32(v.w) : 0.f;
          l.x = k0 < Ks ? rna_tf32(v.x - h.x) : 0.f;
          l.y = k0 + 1 < Ks ? rna_tf32(v.y - h.y) : 0.f;
          l.z = k0 + 2 < Ks ? rna_tf32(v.z - h.z) : 0.f;
          l.w = k0 + 3 < Ks ? rna_tf32(v.w - h.w) : 0.f;
          a[q] = h;
          alo[q] = l;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // visible to the MMAs
        warp_arrive(split0 + 8 * s);
        if (++s == S) {
          s = 0;
          ph ^= 1u;
        }
      }
    }
  } else {
    // epilogue: group g = (warp - 2 - SPLITW) / 4 takes the tiles it == g (mod EPIG)
    const int quad = warp & 3;
    const int grp = (warp - 2 - SPLITW) >> 2;
    int it = grp;
    for (int64_t tile = blockIdx.x + (int64_t)grp * gridDim.x; tile < n_tiles;
         tile += (int64_t)EPIG * gridDim.x, it += EPIG) {
      const int bsel = it & 1;
      bad = bad || !mbar_wait_bounded(tfull0 + 8 * bsel, (it >> 1) & 1);
      bad = __any_sync(0xffffffffu, bad);
      if (bad) break;
      tc_fence_after();
      const int sg = p.tile_seg[tile];
      const int Ns = p.segN ? p.segN[sg] : p.N;
      if constexpr (MODE == 2) {
        tc_epilogue_sincos(p, tmem + (uint32_t)bsel * acc_cols, quad, lane, tile,
                           p.tile_row0[tile], p.tile_rows[tile],
                           reinterpret_cast<float*>(smem + (size_t)S * p.stage_bytes +
                                                    round_up(8 * (3 * S + 4), 16)));
      } else {
        tc_epilogue_row<ARGMAX>(p, tmem + (uint32_t)bsel * acc_cols, quad, lane, sg,
                                p.tile_row0[tile], p.tile_rows[tile], Ns);
      }
      tc_fence_before();
      warp_arrive(tempty0 + 8 * bsel);  // this buffer may take the next accumulator
    }
  }
  if (bad) atomicExch(p.wait_err, 1);
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(p.tmem_cols)
                 : "memory");
  }
}

// ---------------------------------------------------------------------------
// TN: partial[c] (K x N, fp32) = A[rows of chunk c]^T B[rows of chunk c], the
// reduction running over the tall rows. Both operands need the row index as the
// UMMA K dimension, so the split warps also transpose: each 32-row block of A
// and B arrives row-major (TMA, no swizzle) and is written as K-major 128-byte
// swizzled tf32 hi / lo tiles (A: up to two 128-row M blocks covering K <= 256;
// B: Np rows). Persistent over the chunks of the row space; the chunk partials
// are then summed in FP64 in chunk order (reduce_pieces), as for the SIMT kernel.
//   warp 0: TMA producer (raw A, B rows)   warp 1: TMEM owner + MMA issuer
//   warps 2-5: transpose + split           warps 6-9: epilogue (partials to global)
// ---------------------------------------------------------------------------
struct TnArgs {
  int K, N;          // largest K_s (columns of A), N_s (columns of B)
  int Np;            // UMMA N
  int mblk;          // 128-row M blocks covering K
  int ka_box, nb_box;  // raw tile widths (multiples of 4)
  const int* segK;
  const int* segN;
  const int* chunk_seg;
  const int64_t* chunk_row0;
  const int* chunk_rows;
  float* part;       // [chunk][K][N]
  int stages;
  uint32_t raw_bytes, raw_a_bytes;  // one raw stage, its A part
  uint32_t op_bytes;                // one operand set (A hi, A lo, B hi, B lo)
  int nops;                         // operand sets (2: split of block b+1 overlaps MMAs of b)
  uint32_t tmem_cols;
  int* wait_err;                    // as in TcArgs
};

constexpr int kTnRows = 32;  // rows per block = UMMA K extent of one operand set
#ifndef ABG_TN_NOPS
#define ABG_TN_NOPS 2
#endif

__global__ void __launch_bounds__(kTcThreads, 1)
    k_tc_tn(const __grid_constant__ CUtensorMap amap, const __grid_constant__ CUtensorMap bmap,
            const TnArgs p, int64_t n_chunks) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  __shared__ uint32_t tmem_slot;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int S = p.stages;
  const int NO = p.nops;
  unsigned char* ops = smem;                                   // operand sets (1024-aligned)
  unsigned char* raw = smem + (size_t)NO * p.op_bytes;         // raw stages
  uint64_t* bars = reinterpret_cast<uint64_t*>(raw + (size_t)S * p.raw_bytes);
  const uint32_t rfull0 = smem_addr(bars), rempty0 = rfull0 + 8 * S, opfull0 = rfull0 + 16 * S,
                 opempty0 = opfull0 + 8 * NO, tfull = opempty0 + 8 * NO, tempty = tfull + 8;
  const uint32_t a_hi_bytes = (uint32_t)p.mblk * kTcM * 128, b_hi_bytes = (uint32_t)p.Np * 128;
  if (threadIdx.x == 0) {
    for (int i = 0; i < S; ++i) {
      mbar_init(rfull0 + 8 * i, 1);
      mbar_init(rempty0 + 8 * i, 4);  // one arrival per transposing warp
    }
    for (int i = 0; i < NO; ++i) {
      mbar_init(opfull0 + 8 * i, 4);
      mbar_init(opempty0 + 8 * i, 1);
    }
    mbar_init(tfull, 1);
    mbar_init(tempty, 4);  // one arrival per epilogue warp
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(&tmem_slot)),
                 "r"(p.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  bool bad = *reinterpret_cast<volatile int*>(p.wait_err) != 0;

  if (warp == 0) {
    if (lane == 0) {  // producer
      int s = 0;
      uint32_t ph = 0;
      int64_t n = 0;
      for (int64_t c = blockIdx.x; c < n_chunks && !bad; c += gridDim.x) {
        const int64_t r0 = p.chunk_row0[c];
        const int nb = (p.chunk_rows[c] + kTnRows - 1) / kTnRows;
        for (int b = 0; b < nb; ++b, ++n) {
          if (n >= S && !mbar_wait_bounded(rempty0 + 8 * s, ph ^ 1u)) {
            bad = true;
            break;
          }
          const uint32_t st = smem_addr(raw + (size_t)s * p.raw_bytes);
          mbar_expect_tx(rfull0 + 8 * s, p.raw_bytes);
          tma_load_2d(st, &amap, 0, (int)(r0 + b * kTnRows), rfull0 + 8 * s);
          tma_load_2d(st + p.raw_a_bytes, &bmap, 0, (int)(r0 + b * kTnRows), rfull0 + 8 * s);
          if (++s == S) {
            s = 0;
            ph ^= 1u;
          }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {  // MMA issuer
      const uint32_t idesc = tf32_idesc(p.Np);
      int os = 0;  // operand set of the next block, and its phase
      uint32_t op_ph = 0;
      int it = 0;
      for (int64_t c = blockIdx.x; c < n_chunks && !bad; c += gridDim.x, ++it) {
        if (it >= 1 && !mbar_wait_bounded(tempty, (it - 1) & 1)) {  // partial read out
          bad = true;
          break;
        }
        tc_fence_after();
        const int nb = (p.chunk_rows[c] + kTnRows - 1) / kTnRows;
        for (int b = 0; b < nb; ++b) {
          if (!mbar_wait_bounded(opfull0 + 8 * os, op_ph)) {
            bad = true;
            break;
          }
          tc_fence_after();
          const uint32_t ob = smem_addr(ops + (size_t)os * p.op_bytes);
          const uint32_t a_hi = ob, a_lo = ob + a_hi_bytes, b_hi = ob + 2 * a_hi_bytes,
                         b_lo = b_hi + b_hi_bytes;
          for (int mb = 0; mb < p.mblk; ++mb) {
            const uint32_t dcol = tmem + (uint32_t)(mb * p.Np);
            const uint32_t ao = (uint32_t)mb * kTcM * 128;
#pragma unroll
            for (int j = 0; j < kTnRows / 8; ++j) {
              const uint32_t off = 32u * j;
              mma_tf32(dcol, sw128_desc(a_hi + ao + off), sw128_desc(b_hi + off), idesc,
                       (b | j) != 0);
              mma_tf32(dcol, sw128_desc(a_lo + ao + off), sw128_desc(b_hi + off), idesc, 1u);
              mma_tf32(dcol, sw128_desc(a_hi + ao + off), sw128_desc(b_lo + off), idesc, 1u);
            }
          }
          mma_commit(opempty0 + 8 * os);  // the operand set may be rewritten
          if (++os == NO) {
            os = 0;
            op_ph ^= 1u;
          }
        }
        if (bad) break;
        mma_commit(tfull);
      }
    }
  } else if (warp < 6) {
    // transpose + split: A_raw[m][ka] -> A_op[ka][m] (K-major, 128B swizzle), same for B
    const int t = threadIdx.x - 64;
    const uint32_t a_rows = (uint32_t)p.mblk * kTcM;
    int s = 0, os = 0;
    uint32_t ph = 0, op_ph = 0;
    int64_t n = 0;
    for (int64_t c = blockIdx.x; c < n_chunks && !bad; c += gridDim.x) {
      const int sg = p.chunk_seg[c];
      const int Ks = p.segK ? p.segK[sg] : p.K;
      const int Ns = p.segN ? p.segN[sg] : p.N;
      const int rows = p.chunk_rows[c];
      const int nb = (rows + kTnRows - 1) / kTnRows;
      for (int b = 0; b < nb; ++b, ++n) {
        const bool ok = mbar_wait_bounded(rfull0 + 8 * s, ph) &&
                        (n < NO || mbar_wait_bounded(opempty0 + 8 * os, op_ph ^ 1u));
        if (__any_sync(0xffffffffu, !ok)) {  // the whole warp leaves together
          bad = true;
          break;
        }
        const float* ra = reinterpret_cast<const float*>(raw + (size_t)s * p.raw_bytes);
        const float* rb = reinterpret_cast<const float*>(raw + (size_t)s * p.raw_bytes +
                                                         p.raw_a_bytes);
        const int mvalid = rows - b * kTnRows;  // rows of this block inside the chunk
        // The source block is 32 rows x ld floats (row-major); operand row rr holds source
        // column rr over the 32 rows (K-major, 128-byte swizzle). Each unit is a 4 x 4 block:
        // four float4 row reads, a transpose in registers, four float4 operand writes per part.
        // A warp covers 32 consecutive columns x 16 rows, so the reads touch four 128-byte row
        // segments and the writes eight distinct 16-byte bank groups: both take the minimum
        // four wavefronts (the per-element column reads they replace conflicted 8 ways).
        auto emit = [&](const float* src, int ld, int lim, uint32_t rows_out, unsigned char* hi,
                        unsigned char* lo) {
          const uint32_t ncol4 = rows_out / 4;                 // 4-column groups (rows_out % 4 == 0)
          const uint32_t nunits = ((ncol4 + 7) / 8) * 64;      // 8 column groups x 8 row groups
          for (uint32_t u = t; u < nunits; u += 128) {
            const uint32_t g = u >> 5, l = u & 31;
            const uint32_t c4 = 8 * (g >> 1) + (l & 7);        // column group
            const int k4 = (int)(4 * (g & 1) + (l >> 3));      // row group (4 source rows)
            if (c4 >= ncol4) continue;
            const int c0 = (int)(4 * c4), m0 = 4 * k4;
            float4 v[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const int m = m0 + e;
              v[e] = (c0 < ld && m < mvalid) ? *reinterpret_cast<const float4*>(src + m * ld + c0)
                                             : make_float4(0.f, 0.f, 0.f, 0.f);
            }
            const float cm[4] = {c0 < lim ? 1.f : 0.f, c0 + 1 < lim ? 1.f : 0.f,
                                 c0 + 2 < lim ? 1.f : 0.f, c0 + 3 < lim ? 1.f : 0.f};
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              // column c0 + j over rows m0..m0+3 (columns at or beyond lim are zero)
              float x[4];
#pragma unroll
              for (int e = 0; e < 4; ++e) {
                const float4 r = v[e];
                const float val = j == 0 ? r.x : (j == 1 ? r.y : (j == 2 ? r.z : r.w));
                x[e] = cm[j] != 0.f ? val : 0.f;
              }
              float4 h, lw;
              h.x = rna_tf32(x[0]);
              h.y = rna_tf32(x[1]);
              h.z = rna_tf32(x[2]);
              h.w = rna_tf32(x[3]);
              lw.x = rna_tf32(x[0] - h.x);
              lw.y = rna_tf32(x[1] - h.y);
              lw.z = rna_tf32(x[2] - h.z);
              lw.w = rna_tf32(x[3] - h.w);
              const int rr = c0 + j, blk = rr >> 7, rl = rr & 127;
              const uint32_t off = (uint32_t)blk * kTcM * 128 + (uint32_t)rl * 128 +
                                   (uint32_t)((k4 ^ (rl & 7)) * 16);
              *reinterpret_cast<float4*>(hi + off) = h;
              *reinterpret_cast<float4*>(lo + off) = lw;
            }
          }
        };
        unsigned char* o = ops + (size_t)os * p.op_bytes;
        emit(ra, p.ka_box, Ks, a_rows, o, o + a_hi_bytes);
        emit(rb, p.nb_box, Ns, (uint32_t)p.Np, o + 2 * a_hi_bytes, o + 2 * a_hi_bytes + b_hi_bytes);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // visible to the MMAs
        warp_arrive(rempty0 + 8 * s);
        warp_arrive(opfull0 + 8 * os);
        if (++os == NO) {
          os = 0;
          op_ph ^= 1u;
        }
        if (++s == S) {
          s = 0;
          ph ^= 1u;
        }
      }
    }
  } else {
    // epilogue: M block rows -> partial rows (K index), N columns
    const int quad = warp & 3;
    int it = 0;
    for (int64_t c = blockIdx.x; c < n_chunks; c += gridDim.x, ++it) {
      bad = bad || !mbar_wait_bounded(tfull, it & 1);
      bad = __any_sync(0xffffffffu, bad);
      if (bad) break;
      tc_fence_after();
      float* pc = p.part + c * (int64_t)p.K * p.N;
      for (int mb = 0; mb < p.mblk; ++mb) {
        const int ka = mb * kTcM + quad * 32 + lane;
        for (int c0 = 0; c0 < p.Np; c0 += 32) {
          float v[32];
          tmem_ld32(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(mb * p.Np + c0), v);
          if (ka >= p.K) continue;
          float* prow = pc + (int64_t)ka * p.N;
#pragma unroll
          for (int j = 0; j < 32; ++j)
            if (c0 + j < p.N) prow[c0 + j] = v[j];
        }
      }
      tc_fence_before();
      warp_arrive(tempty);
    }
  }
  if (bad) atomicExch(p.wait_err, 1);
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(p.tmem_cols)
                 : "memory");
  }
}

// ---------------------------------------------------------------------------
// TN with per-thread staging: each transposing thread copies its own 4 x 4 blocks of A and B
// for the next row block into a private slot of shared memory with cp.async (16-byte copies,
// zero-filled outside the block), and transposes + splits the current block from the other
// slot into the operand set. An mbarrier arrival has release semantics and would wait for
// loads still in flight into registers; cp.async copies are outside that ordering, so the
// next block's copies stay in flight across the hand-off to the MMAs. Two operand sets when
// they fit (K <= 128), else one. Two TMEM accumulators alternate between chunks, so the
// partial of one chunk drains while the next accumulates.
//   warp 0: TMEM owner + MMA issuer   warps 1..TW: copy, transpose, split
//   warps TW+1..TW+4: epilogue (chunk partials to global, FP32)
// ---------------------------------------------------------------------------
constexpr int kTn2Units = 3;  // 4 x 4 blocks per transposing thread and row block

struct Tn2Args {
  const float* A;
  int64_t lda;
  const float* B;
  int64_t ldb;
  int K, N, Np, mblk;
  const int* segK;
  const int* segN;
  const int* chunk_seg;
  const int64_t* chunk_row0;
  const int* chunk_rows;
  float* part;     // [chunk][K][N]
  int nops;
  uint32_t op_bytes;
  uint32_t stage_bytes;  // one staging slot: transposing threads x units x 64 bytes
  int syrk;              // A == B (a Gram matrix): B's operand is the first Np rows of A's
  int swap;              // K > 128: B's 128 operand rows are the MMA's M, A's 256 its N
  uint32_t acc_cols;     // TMEM columns of one accumulator (>= mblk * Np)
  uint32_t tmem_cols;
  int* wait_err;
};

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, uint32_t src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src),
               "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// 13 warps put four on one SM sub-partition, whose 16K registers allow 128 a thread
template <int TW>
__global__ void __maxnreg__(128) k_tc_tn2(const Tn2Args p, int64_t n_chunks) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  __shared__ uint32_t tmem_slot;
  constexpr int kT = 32 * TW;  // transposing threads
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int NO = p.nops;
  unsigned char* ops = smem;
  unsigned char* stage = smem + (size_t)NO * p.op_bytes;  // two staging slots
  uint64_t* bars = reinterpret_cast<uint64_t*>(stage + 2 * (size_t)p.stage_bytes);
  const uint32_t opfull0 = smem_addr(bars), opempty0 = opfull0 + 8 * NO,
                 tfull0 = opempty0 + 8 * NO, tempty0 = tfull0 + 16, drain = tempty0 + 16;
  const uint32_t a_hi_bytes = (uint32_t)p.mblk * kTcM * 128,
                 b_hi_bytes = (uint32_t)(p.swap ? kTcM : p.Np) * 128;
  if (threadIdx.x == 0) {
    for (int i = 0; i < NO; ++i) {
      mbar_init(opfull0 + 8 * i, TW);  // one arrival per transposing warp
      mbar_init(opempty0 + 8 * i, 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(tfull0 + 8 * i, 1);
      mbar_init(tempty0 + 8 * i, 4);  // one arrival per epilogue warp
    }
    mbar_init(drain, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(&tmem_slot)),
                 "r"(p.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  bool bad = *reinterpret_cast<volatile int*>(p.wait_err) != 0;

  if (warp == 0) {
    if (lane == 0) {  // MMA issuer
      const uint32_t idesc = tf32_idesc(p.swap ? p.mblk * kTcM : p.Np);
      int os = 0;
      uint32_t op_ph = 0;
      int it = 0;
      bool issued = false;
      for (int64_t c = blockIdx.x; c < n_chunks && !bad; c += gridDim.x, ++it) {
        const int abuf = it & 1;
        if (it >= 2 && !mbar_wait_bounded(tempty0 + 8 * abuf, ((it >> 1) - 1) & 1)) {
          bad = true;
          break;
        }
        tc_fence_after();
        const uint32_t acc = tmem + (uint32_t)abuf * p.acc_cols;
        const int nb = (p.chunk_rows[c] + kTnRows - 1) / kTnRows;
        for (int b = 0; b < nb; ++b) {
          if (!mbar_wait_bounded(opfull0 + 8 * os, op_ph)) {
            bad = true;
            break;
          }
          tc_fence_after();
          const uint32_t ob = smem_addr(ops + (size_t)os * p.op_bytes);
          const uint32_t a_hi = ob, a_lo = ob + a_hi_bytes,
                         b_hi = p.syrk ? a_hi : ob + 2 * a_hi_bytes,
                         b_lo = p.syrk ? a_lo : b_hi + b_hi_bytes;
          if (p.swap) {
            // D^T (B's columns x A's 256 columns) in one MMA per term and K step
#pragma unroll
            for (int j = 0; j < kTnRows / 8; ++j) {
              const uint32_t off = 32u * j;
              mma_tf32(acc, sw128_desc(b_hi + off), sw128_desc(a_hi + off), idesc, (b | j) != 0);
              mma_tf32(acc, sw128_desc(b_hi + off), sw128_desc(a_lo + off), idesc, 1u);
              mma_tf32(acc, sw128_desc(b_lo + off), sw128_desc(a_hi + off), idesc, 1u);
            }
          } else {
            for (int mb = 0; mb < p.mblk; ++mb) {
              const uint32_t dcol = acc + (uint32_t)(mb * p.Np);
              const uint32_t ao = (uint32_t)mb * kTcM * 128;
#pragma unroll
              for (int j = 0; j < kTnRows / 8; ++j) {
                const uint32_t off = 32u * j;
                mma_tf32(dcol, sw128_desc(a_hi + ao + off), sw128_desc(b_hi + off), idesc,
                         (b | j) != 0);
                mma_tf32(dcol, sw128_desc(a_lo + ao + off), sw128_desc(b_hi + off), idesc, 1u);
                mma_tf32(dcol, sw128_desc(a_hi + ao + off), sw128_desc(b_lo + off), idesc, 1u);
              }
            }
          }
          issued = true;
          mma_commit(opempty0 + 8 * os);  // the operand set may be rewritten
          if (++os == NO) {
            os = 0;
            op_ph ^= 1u;
          }
        }
        if (bad) break;
        mma_commit(tfull0 + 8 * abuf);  // this chunk's partial is complete
      }
      // every MMA issued has finished before the CTA may free its tensor memory
      if (issued) {
        mma_commit(drain);
        if (!mbar_wait_bounded(drain, 0)) bad = true;
      }
    }
  } else if (warp <= TW) {
    const int t = threadIdx.x - 32;
    const uint32_t a_rows = (uint32_t)p.mblk * kTcM;
    int os = 0;
    uint32_t op_ph = 0;
    int64_t n = 0;
    auto store4 = [&](const float4 (&v)[4], int c0, int k4, int lim, unsigned char* hi,
                      unsigned char* lo) {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        float x[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const float4 r = v[e];
          const float val = j == 0 ? r.x : (j == 1 ? r.y : (j == 2 ? r.z : r.w));
          x[e] = c0 + j < lim ? val : 0.f;
        }
        float4 h, lw;
        h.x = rna_tf32(x[0]);
        h.y = rna_tf32(x[1]);
        h.z = rna_tf32(x[2]);
        h.w = rna_tf32(x[3]);
        lw.x = rna_tf32(x[0] - h.x);
        lw.y = rna_tf32(x[1] - h.y);
        lw.z = rna_tf32(x[2] - h.z);
        lw.w = rna_tf32(x[3] - h.w);
        const int rr = c0 + j, blk = rr >> 7, rl = rr & 127;
        const uint32_t off = (uint32_t)blk * kTcM * 128 + (uint32_t)rl * 128 +
                             (uint32_t)((k4 ^ (rl & 7)) * 16);
        *reinterpret_cast<float4*>(hi + off) = h;
        *reinterpret_cast<float4*>(lo + off) = lw;
      }
    };
    // units: (column group c4, row group k4); a warp covers 4 column groups x all 8 row
    // groups, lane l taking row group l & 7. A 16-byte shared store is served eight lanes at
    // a time, and those eight then hold the same column and eight row groups: eight
    // different 16-byte chunks of the 128-byte swizzle row, no bank conflict.
    // A thread's units are the same for every block; which block they read changes.
    const uint32_t na4 = a_rows / 4, nb4 = (uint32_t)p.Np / 4;
    const uint32_t ua = ((na4 + 3) / 4) * 32, ub = p.syrk ? 0u : ((nb4 + 3) / 4) * 32;
    constexpr int kMaxU = kTn2Units;  // units per thread (A and B together), checked at launch
    int uc0[kMaxU], uk4[kMaxU], uwhich[kMaxU];
#pragma unroll
    for (int q = 0; q < kMaxU; ++q) {
      const uint32_t u = (uint32_t)t + (uint32_t)q * kT;
      uwhich[q] = -1;
      uc0[q] = 0;
      uk4[q] = 0;
      if (u < ua + ub) {
        const bool isA = u < ua;
        const uint32_t uu = isA ? u : u - ua;
        const uint32_t g = uu >> 5, l = uu & 31;
        const uint32_t c4 = 4 * g + (l >> 3);
        if (c4 < (isA ? na4 : nb4)) {
          uwhich[q] = isA ? 0 : 1;
          uc0[q] = (int)(4 * c4);
          uk4[q] = (int)(l & 7);
        }
      }
    }
    auto nblocks = [&](int64_t c) { return (p.chunk_rows[c] + kTnRows - 1) / kTnRows; };
    // this thread's 16-byte pieces of block b of chunk c into staging slot sl: unit q, row e
    // at ((q * 4 + e) * kT + t) * 16, zero-filled outside the block's rows or the width
    const uint32_t stage0 = smem_addr(stage);
    auto issue = [&](int sl, int64_t c, int b) {
      const int sg = p.chunk_seg[c];
      const int mvalid = p.chunk_rows[c] - b * kTnRows;
      const int64_t row0 = p.chunk_row0[c] + (int64_t)b * kTnRows;
      const int Ks = p.segK ? p.segK[sg] : p.K;
      const int Ns = p.segN ? p.segN[sg] : p.N;
#pragma unroll
      for (int q = 0; q < kMaxU; ++q) {
        if (uwhich[q] < 0) continue;
        const bool isA = uwhich[q] == 0;
        const float* src = isA ? p.A + row0 * p.lda : p.B + row0 * p.ldb;
        const int64_t ld = isA ? p.lda : p.ldb;
        const int lim = isA ? Ks : Ns;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int m = 4 * uk4[q] + e;
          const bool ok = uc0[q] < lim && m < mvalid;
          const uint32_t dst = stage0 + (uint32_t)sl * p.stage_bytes +
                               (uint32_t)(((q * 4 + e) * kT + t) * 16);
          cp_async16(dst, ok ? (const void*)(src + (int64_t)m * ld + uc0[q]) : (const void*)p.A,
                     ok ? 16u : 0u);
        }
      }
    };
    int64_t c = blockIdx.x;
    int b = 0, sl = 0;
    if (c < n_chunks) issue(0, c, 0);
    cp_async_commit();
    while (c < n_chunks && !bad) {
      int64_t c2 = c;
      int b2 = b;
      if (++b2 >= nblocks(c2)) {
        c2 += gridDim.x;
        b2 = 0;
      }
      if (c2 < n_chunks) issue(sl ^ 1, c2, b2);
      cp_async_commit();
      cp_async_wait<1>();  // this block's copies have landed (the next block's may not)
      const bool ok = n < NO || mbar_wait_bounded(opempty0 + 8 * os, op_ph ^ 1u);
      if (__any_sync(0xffffffffu, !ok)) {  // the whole warp leaves together
        bad = true;
        break;
      }
      const int sg = p.chunk_seg[c];
      const int Ks = p.segK ? p.segK[sg] : p.K;
      const int Ns = p.segN ? p.segN[sg] : p.N;
      unsigned char* o = ops + (size_t)os * p.op_bytes;
      const float4* st = reinterpret_cast<const float4*>(stage + (size_t)sl * p.stage_bytes);
#pragma unroll
      for (int q = 0; q < kMaxU; ++q) {
        if (uwhich[q] < 0) continue;
        float4 v[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) v[e] = st[(q * 4 + e) * kT + t];
        if (uwhich[q] == 0)
          store4(v, uc0[q], uk4[q], Ks, o, o + a_hi_bytes);
        else
          store4(v, uc0[q], uk4[q], Ns, o + 2 * a_hi_bytes, o + 2 * a_hi_bytes + b_hi_bytes);
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // visible to the MMAs
      warp_arrive(opfull0 + 8 * os);
      if (++os == NO) {
        os = 0;
        op_ph ^= 1u;
      }
      ++n;
      c = c2;
      b = b2;
      sl ^= 1;
    }
    cp_async_wait<0>();  // no copy in flight when the CTA leaves
  } else {
    // epilogue: accumulator rows (the K index) -> partial rows, N columns
    const int quad = warp & 3;
    int it = 0;
    for (int64_t c = blockIdx.x; c < n_chunks; c += gridDim.x, ++it) {
      const int abuf = it & 1;
      bad = bad || !mbar_wait_bounded(tfull0 + 8 * abuf, (it >> 1) & 1);
      bad = __any_sync(0xffffffffu, bad);
      if (bad) break;
      tc_fence_after();
      float* pc = p.part + c * (int64_t)p.K * p.N;
      if (p.swap) {
        // this lane's accumulator row is B's column n; its columns are A's columns ka
        const int n = quad * 32 + lane;
        for (int c0 = 0; c0 < p.mblk * kTcM; c0 += 32) {
          float v[32];
          tmem_ld32(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(abuf * p.acc_cols + c0),
                    v);
          if (n >= p.N) continue;
#pragma unroll
          for (int j = 0; j < 32; ++j)
            if (c0 + j < p.K) pc[(int64_t)(c0 + j) * p.N + n] = v[j];
        }
      } else {
        for (int mb = 0; mb < p.mblk; ++mb) {
          const int ka = mb * kTcM + quad * 32 + lane;
          for (int c0 = 0; c0 < p.Np; c0 += 32) {
            float v[32];
            tmem_ld32(tmem + ((uint32_t)(quad * 32) << 16) +
                          (uint32_t)(abuf * p.acc_cols + mb * p.Np + c0), v);
            if (ka >= p.K) continue;
            float* prow = pc + (int64_t)ka * p.N;
#pragma unroll
            for (int j = 0; j < 32; ++j)
              if (c0 + j < p.N) prow[c0 + j] = v[j];
          }
        }
      }
      tc_fence_before();
      warp_arrive(tempty0 + 8 * abuf);
    }
  }
  if (bad) atomicExch(p.wait_err, 1);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(p.tmem_cols)
                 : "memory");
  }
}

// ---------------------------------------------------------------------------
// BF16 NN: C = A16 B_s with A16 (rows x K, bf16, row-major) and B_s rounded to bf16 once.
// K moves in 64-column blocks (one 128-byte swizzle row of bf16), four UMMA K = 16 steps
// each. With one segment all of B stays in shared memory; otherwise each stage carries its
// B block. No split warps: the A tile goes from TMA to the MMAs untouched.
//   warp 0: TMA producer   warp 1: TMEM owner + MMA issuer   warps 2-5: epilogue
// ---------------------------------------------------------------------------
constexpr int kBK16 = 64;                              // bf16 K per stage
constexpr uint32_t kA16Bytes = kTcM * kBK16 * 2;       // 16 KiB
constexpr int kNn16Threads = 192;

// B16 (segment s rows s*Np .. s*Np + Np, K-major bf16, Kp columns) from B_s (K x N fp32)
__global__ void k_tc_prep_b16(const float* __restrict__ B, int64_t ldb, int64_t b_seg,
                              const int* __restrict__ segK, int K, const int* __restrict__ segN,
                              int N, int Np, int Kp, __nv_bfloat16* __restrict__ out) {
  const int sg = blockIdx.y;
  const int Ks = segK ? segK[sg] : K;
  const int Ns = segN ? segN[sg] : N;
  const float* Bs = B + sg * b_seg;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)Np * Kp;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int n = (int)(e / Kp), k = (int)(e % Kp);
    const float x = (n < Ns && k < Ks) ? Bs[(int64_t)k * ldb + n] : 0.f;
    out[((int64_t)sg * Np + n) * Kp + k] = __float2bfloat16_rn(x);
  }
}

__global__ void __launch_bounds__(kNn16Threads, 1)
    k_tc_nn16(const __grid_constant__ CUtensorMap amap, const __grid_constant__ CUtensorMap bmap,
              const TcArgs p, int64_t n_tiles) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  __shared__ uint32_t tmem_slot;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int S = p.stages;
  const uint32_t bres_bytes = p.b_resident ? (uint32_t)p.nkb * p.b_bytes : 0u;
  unsigned char* bres = smem;
  unsigned char* stg = smem + bres_bytes;
  uint64_t* bars = reinterpret_cast<uint64_t*>(stg + (size_t)S * p.stage_bytes);
  const uint32_t full0 = smem_addr(bars), empty0 = full0 + 8 * S, bfull = full0 + 16 * S,
                 tfull0 = bfull + 8, tempty0 = tfull0 + 16;
  if (threadIdx.x == 0) {
    for (int i = 0; i < S; ++i) {
      mbar_init(full0 + 8 * i, 1);
      mbar_init(empty0 + 8 * i, 1);
    }
    mbar_init(bfull, 1);
    for (int i = 0; i < 2; ++i) {
      mbar_init(tfull0 + 8 * i, 1);
      mbar_init(tempty0 + 8 * i, 128);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(&tmem_slot)),
                 "r"(p.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  const uint32_t acc_cols = p.tmem_cols / 2;
  bool bad = *reinterpret_cast<volatile int*>(p.wait_err) != 0;

  if (warp == 0) {
    if (lane == 0 && !bad) {  // producer
      if (p.b_resident) {     // every K block of B, once
        mbar_expect_tx(bfull, bres_bytes);
        for (int kb = 0; kb < p.nkb; ++kb)
          tma_load_2d(smem_addr(bres + (size_t)kb * p.b_bytes), &bmap, kb * kBK16, 0, bfull);
      }
      const uint32_t tx = kA16Bytes + (p.b_resident ? 0u : p.b_bytes);
      int s = 0;
      uint32_t ph = 0;
      int64_t n = 0;
      for (int64_t tile = blockIdx.x; tile < n_tiles && !bad; tile += gridDim.x) {
        const int sg = p.tile_seg[tile];
        const int row0 = (int)p.tile_row0[tile];
        for (int kb = 0; kb < p.nkb; ++kb, ++n) {
          if (n >= S && !mbar_wait_bounded(empty0 + 8 * s, ph ^ 1u)) {
            bad = true;
            break;
          }
          const uint32_t st = smem_addr(stg + (size_t)s * p.stage_bytes);
          mbar_expect_tx(full0 + 8 * s, tx);
          tma_load_2d(st, &amap, kb * kBK16, row0, full0 + 8 * s);
          if (!p.b_resident)
            tma_load_2d(st + kA16Bytes, &bmap, kb * kBK16, sg * p.Np, full0 + 8 * s);
          if (++s == S) {
            s = 0;
            ph ^= 1u;
          }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0 && !bad) {  // MMA issuer
      const uint32_t idesc = bf16_idesc(p.Np, false, false);
      if (p.b_resident && !mbar_wait_bounded(bfull, 0)) bad = true;
      tc_fence_after();
      int s = 0;
      uint32_t ph = 0;
      int it = 0;
      for (int64_t tile = blockIdx.x; tile < n_tiles && !bad; tile += gridDim.x, ++it) {
        const int bsel = it & 1;
        if (it >= 2 && !mbar_wait_bounded(tempty0 + 8 * bsel, ((it >> 1) - 1) & 1)) {
          bad = true;
          break;
        }
        tc_fence_after();
        const uint32_t tacc = tmem + (uint32_t)bsel * acc_cols;
        for (int kb = 0; kb < p.nkb; ++kb) {
          if (!mbar_wait_bounded(full0 + 8 * s, ph)) {
            bad = true;
            break;
          }
          tc_fence_after();
          const uint32_t a = smem_addr(stg + (size_t)s * p.stage_bytes);
          const uint32_t b = p.b_resident ? smem_addr(bres + (size_t)kb * p.b_bytes)
                                          : a + kA16Bytes;
#pragma unroll
          for (int j = 0; j < kBK16 / 16; ++j) {  // UMMA K = 16 bf16 = 32 bytes
            const uint32_t off = 32u * j;
            mma_bf16(tacc, sw128_desc(a + off), sw128_desc(b + off), idesc, (kb | j) != 0);
          }
          mma_commit(empty0 + 8 * s);
          if (++s == S) {
            s = 0;
            ph ^= 1u;
          }
        }
        if (bad) break;
        mma_commit(tfull0 + 8 * bsel);
      }
    }
  } else {
    // epilogue: warps 2-5 own TMEM lane quarters 2, 3, 0, 1
    const int quad = warp & 3;
    int it = 0;
    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++it) {
      const int bsel = it & 1;
      bad = bad || !mbar_wait_bounded(tfull0 + 8 * bsel, (it >> 1) & 1);
      bad = __any_sync(0xffffffffu, bad);
      if (bad) break;
      tc_fence_after();
      const int sg = p.tile_seg[tile];
      const int Ns = p.segN ? p.segN[sg] : p.N;
      tc_epilogue_row<false>(p, tmem + (uint32_t)bsel * acc_cols, quad, lane, sg,
                             p.tile_row0[tile], p.tile_rows[tile], Ns);
      tc_fence_before();
      mbar_arrive(tempty0 + 8 * bsel);
    }
  }
  if (bad) atomicExch(p.wait_err, 1);
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(p.tmem_cols)
                 : "memory");
  }
}

// ---------------------------------------------------------------------------
// BF16 TN: partial[c] (K x N) = A16[rows of chunk c]^T B[rows of chunk c]. The reduction
// index (rows) is UMMA K for both operands, and both are stored with their M / N index
// contiguous, so both go to the MMAs as MN-major tiles: A16 arrives from TMA in 64-row x
// 64-column boxes (128-byte swizzle) and is used in place; the converter warps round each
// 64-row block of the fp32 B rows to bf16 into the same MN-major layout (zeros for rows
// past the chunk and columns past N_s). A raw stage is free once the MMAs have read its A
// boxes (commit) and the converters its B rows (128 arrivals).
//   warp 0: TMA producer   warp 1: TMEM owner + MMA issuer
//   warps 2-5: B converters   warps 6-9: epilogue (partials to global)
// ---------------------------------------------------------------------------
constexpr int kTn16Rows = 64;                          // rows per block (4 UMMA K steps)
constexpr uint32_t kMnBox = kTn16Rows * 128;           // one 64 x 64 bf16 box: 8 KiB

__global__ void __launch_bounds__(kTcThreads, 1)
    k_tc_tn16(const __grid_constant__ CUtensorMap amap, const __grid_constant__ CUtensorMap bmap,
              const TnArgs p, int64_t n_chunks) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  __shared__ uint32_t tmem_slot;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int S = p.stages;
  const int NO = p.nops;
  unsigned char* ops = smem;                                   // converted B sets
  unsigned char* raw = smem + (size_t)NO * p.op_bytes;         // A boxes + raw B rows
  uint64_t* bars = reinterpret_cast<uint64_t*>(raw + (size_t)S * p.raw_bytes);
  const uint32_t rfull0 = smem_addr(bars), rempty0 = rfull0 + 8 * S, opfull0 = rfull0 + 16 * S,
                 opempty0 = opfull0 + 8 * NO, tfull = opempty0 + 8 * NO, tempty = tfull + 8;
  // 64-column boxes of A that hold columns < K (the rest of the 128 * mblk operand rows only
  // feed accumulator rows >= K, which the epilogue drops)
  const int nbox_a = (p.K + 63) / 64;
  const int nch_b = (p.Np + 63) / 64;             // 64-column chunks of the B operand
  const uint32_t tx = (uint32_t)nbox_a * kMnBox + (uint32_t)kTn16Rows * p.nb_box * 4;
  if (threadIdx.x == 0) {
    for (int i = 0; i < S; ++i) {
      mbar_init(rfull0 + 8 * i, 1);
      mbar_init(rempty0 + 8 * i, 129);  // MMA commit + 128 converter threads
    }
    for (int i = 0; i < NO; ++i) {
      mbar_init(opfull0 + 8 * i, 128);
      mbar_init(opempty0 + 8 * i, 1);
    }
    mbar_init(tfull, 1);
    mbar_init(tempty, 128);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(&tmem_slot)),
                 "r"(p.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  bool bad = *reinterpret_cast<volatile int*>(p.wait_err) != 0;

  if (warp == 0) {
    if (lane == 0) {  // producer
      int s = 0;
      uint32_t ph = 0;
      int64_t n = 0;
      for (int64_t c = blockIdx.x; c < n_chunks && !bad; c += gridDim.x) {
        const int64_t r0 = p.chunk_row0[c];
        const int nb = (p.chunk_rows[c] + kTn16Rows - 1) / kTn16Rows;
        for (int b = 0; b < nb; ++b, ++n) {
          if (n >= S && !mbar_wait_bounded(rempty0 + 8 * s, ph ^ 1u)) {
            bad = true;
            break;
          }
          const uint32_t st = smem_addr(raw + (size_t)s * p.raw_bytes);
          const int y = (int)(r0 + b * kTn16Rows);
          mbar_expect_tx(rfull0 + 8 * s, tx);
          for (int q = 0; q < nbox_a; ++q)
            tma_load_2d(st + (uint32_t)q * kMnBox, &amap, q * 64, y, rfull0 + 8 * s);
          tma_load_2d(st + p.raw_a_bytes, &bmap, 0, y, rfull0 + 8 * s);
          if (++s == S) {
            s = 0;
            ph ^= 1u;
          }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {  // MMA issuer
      const uint32_t idesc = bf16_idesc(p.Np, true, true);
      int s = 0, os = 0;
      uint32_t ph = 0, op_ph = 0;
      int it = 0;
      for (int64_t c = blockIdx.x; c < n_chunks && !bad; c += gridDim.x, ++it) {
        if (it >= 1 && !mbar_wait_bounded(tempty, (it - 1) & 1)) {
          bad = true;
          break;
        }
        tc_fence_after();
        const int nb = (p.chunk_rows[c] + kTn16Rows - 1) / kTn16Rows;
        for (int b = 0; b < nb; ++b) {
          if (!mbar_wait_bounded(rfull0 + 8 * s, ph) ||
              !mbar_wait_bounded(opfull0 + 8 * os, op_ph)) {
            bad = true;
            break;
          }
          tc_fence_after();
          const uint32_t a0 = smem_addr(raw + (size_t)s * p.raw_bytes);
          const uint32_t b0 = smem_addr(ops + (size_t)os * p.op_bytes);
          for (int mb = 0; mb < p.mblk; ++mb) {
            const uint32_t dcol = tmem + (uint32_t)(mb * p.Np);
            const uint32_t am = a0 + (uint32_t)mb * 2 * kMnBox;
#pragma unroll
            for (int j = 0; j < kTn16Rows / 16; ++j) {  // 16 rows = two 8-row groups
              const uint32_t off = 2048u * j;
              mma_bf16(dcol, sw128_mn_desc(am + off, kMnBox), sw128_mn_desc(b0 + off, kMnBox),
                       idesc, (b | j) != 0);
            }
          }
          mma_commit(rempty0 + 8 * s);   // A boxes read
          mma_commit(opempty0 + 8 * os);  // B set read
          if (++s == S) {
            s = 0;
            ph ^= 1u;
          }
          if (++os == NO) {
            os = 0;
            op_ph ^= 1u;
          }
        }
        if (bad) break;
        mma_commit(tfull);
      }
    }
  } else if (warp < 6) {
    // B rows (fp32, nb_box wide) -> bf16 MN-major 128-byte swizzled chunks of 64 columns
    const int t = threadIdx.x - 64;
    int s = 0, os = 0;
    uint32_t ph = 0, op_ph = 0;
    int64_t n = 0;
    for (int64_t c = blockIdx.x; c < n_chunks && !bad; c += gridDim.x) {
      const int sg = p.chunk_seg[c];
      const int Ns = p.segN ? p.segN[sg] : p.N;
      const int rows = p.chunk_rows[c];
      const int nb = (rows + kTn16Rows - 1) / kTn16Rows;
      for (int b = 0; b < nb; ++b, ++n) {
        if (!mbar_wait_bounded(rfull0 + 8 * s, ph) ||
            (n >= NO && !mbar_wait_bounded(opempty0 + 8 * os, op_ph ^ 1u))) {
          bad = true;
          break;
        }
        const float* rb = reinterpret_cast<const float*>(raw + (size_t)s * p.raw_bytes +
                                                         p.raw_a_bytes);
        const int mvalid = rows - b * kTn16Rows;
        unsigned char* o = ops + (size_t)os * p.op_bytes;
        const int units = kTn16Rows * nch_b * 8;  // 16-byte units of the operand
        for (int q = t; q < units; q += 128) {
          const int row = q / (nch_b * 8), cu = q % (nch_b * 8);
          const int ch = cu >> 3, u = cu & 7;
          const int n0 = ch * 64 + u * 8;
          float v[8];
          if (row < mvalid && n0 + 7 < Ns) {
            const float4 x0 = *reinterpret_cast<const float4*>(rb + row * p.nb_box + n0);
            const float4 x1 = *reinterpret_cast<const float4*>(rb + row * p.nb_box + n0 + 4);
            v[0] = x0.x; v[1] = x0.y; v[2] = x0.z; v[3] = x0.w;
            v[4] = x1.x; v[5] = x1.y; v[6] = x1.z; v[7] = x1.w;
          } else {
#pragma unroll
            for (int e = 0; e < 8; ++e)
              v[e] = (row < mvalid && n0 + e < Ns) ? rb[row * p.nb_box + n0 + e] : 0.f;
          }
          uint4 w;
          __nv_bfloat162 h;
          h = __floats2bfloat162_rn(v[0], v[1]);
          w.x = *reinterpret_cast<const uint32_t*>(&h);
          h = __floats2bfloat162_rn(v[2], v[3]);
          w.y = *reinterpret_cast<const uint32_t*>(&h);
          h = __floats2bfloat162_rn(v[4], v[5]);
          w.z = *reinterpret_cast<const uint32_t*>(&h);
          h = __floats2bfloat162_rn(v[6], v[7]);
          w.w = *reinterpret_cast<const uint32_t*>(&h);
          *reinterpret_cast<uint4*>(o + (uint32_t)ch * kMnBox + (uint32_t)row * 128 +
                                    (uint32_t)((u ^ (row & 7)) * 16)) = w;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // visible to the MMAs
        mbar_arrive(rempty0 + 8 * s);
        mbar_arrive(opfull0 + 8 * os);
        if (++os == NO) {
          os = 0;
          op_ph ^= 1u;
        }
        if (++s == S) {
          s = 0;
          ph ^= 1u;
        }
      }
    }
  } else {
    // epilogue: M block rows -> partial rows (K index), N columns
    const int quad = warp & 3;
    int it = 0;
    for (int64_t c = blockIdx.x; c < n_chunks; c += gridDim.x, ++it) {
      bad = bad || !mbar_wait_bounded(tfull, it & 1);
      bad = __any_sync(0xffffffffu, bad);
      if (bad) break;
      tc_fence_after();
      float* pc = p.part + c * (int64_t)p.K * p.N;
      for (int mb = 0; mb < p.mblk; ++mb) {
        const int ka = mb * kTcM + quad * 32 + lane;
        for (int c0 = 0; c0 < p.Np; c0 += 32) {
          float v[32];
          tmem_ld32(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(mb * p.Np + c0), v);
          if (ka >= p.K) continue;
          float* prow = pc + (int64_t)ka * p.N;
#pragma unroll
          for (int j = 0; j < 32; ++j)
            if (c0 + j < p.N) prow[c0 + j] = v[j];
        }
      }
      tc_fence_before();
      mbar_arrive(tempty);
    }
  }
  if (bad) atomicExch(p.wait_err, 1);
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(p.tmem_cols)
                 : "memory");
  }
}

bool tc_disabled() {
  const char* e = std::getenv("ABG_TENSOR_CORES");
  return e && e[0] == '0';
}

}  // namespace

namespace {
// The flag of the solve running on this thread (TcFlagScope), else the process-wide one.
thread_local int* t_tc_flag = nullptr;
std::mutex g_flag_mu;
int* g_flag_addr[64] = {};

int process_flag(int** out) {
  int dev = 0;
  ABG_CUDA(cudaGetDevice(&dev));
  ABG_CHECK(dev >= 0 && dev < 64, "device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_flag_mu);
  if (!g_flag_addr[dev]) {
    void* a = nullptr;
    ABG_CUDA(cudaGetSymbolAddress(&a, g_tc_wait_err));
    g_flag_addr[dev] = static_cast<int*>(a);
  }
  *out = g_flag_addr[dev];
  return ABG_OK;
}

int current_flag(int** out) {
  if (t_tc_flag) {
    *out = t_tc_flag;
    return ABG_OK;
  }
  return process_flag(out);
}
}  // namespace

TcFlagScope::TcFlagScope(int* flag) : prev(t_tc_flag) { t_tc_flag = flag; }
TcFlagScope::~TcFlagScope() { t_tc_flag = prev; }

int tc_wait_flag(cudaStream_t s, int* flag) {
  *flag = 0;
  int* f = nullptr;
  ABG_TRY(current_flag(&f));
  ABG_CUDA(cudaMemcpyAsync(flag, f, sizeof(int), cudaMemcpyDeviceToHost, s));
  ABG_CUDA(cudaStreamSynchronize(s));
  if (*flag) {
    ABG_CUDA(cudaMemsetAsync(f, 0, sizeof(int), s));
    ABG_CUDA(cudaStreamSynchronize(s));
  }
  return ABG_OK;
}

// ABG_TC_A_TMEM=0 keeps A in shared memory (the layout before A moved to tensor memory)
static bool a_tmem_off() {
  static const bool off = [] {
    const char* e = std::getenv("ABG_TC_A_TMEM");
    return e && e[0] == '0';
  }();
  return off;
}

int tc_gemm_nn(const RowSpace& rs, const NN& a, cudaStream_t s, bool* used) {
  static_assert(kTile == kTcM, "row-space tiles must match the UMMA M");
  *used = false;
  if (a.ldc % 4 != 0 || reinterpret_cast<uintptr_t>(a.C) % 16 != 0) return ABG_OK;
  if (tc_disabled() || a.N > 256 || rs.n_tiles == 0) return ABG_OK;
  if (a.sincos && (a.segN || a.argmax || a.ldc < 2 * a.N)) return ABG_OK;
  if (a.lda % 4 != 0 || reinterpret_cast<uintptr_t>(a.A) % 16 != 0 || rs.rows > INT32_MAX)
    return ABG_OK;
  const auto enc = tensor_map_encoder();
  if (!enc) return ABG_OK;
  const int nseg = rs.nseg;
  const int Np = (int)round_up(a.N, 16);
  const int nkb = (int)ceil_div(a.K, kTcBK);
  const int Kp = nkb * kTcBK;
  if ((int64_t)nseg * Np > INT32_MAX) return ABG_OK;
  Scratch scr(s);
  float *bhi, *blo;
  ABG_TRY(scr.get(&bhi, (size_t)nseg * Np * Kp));
  ABG_TRY(scr.get(&blo, (size_t)nseg * Np * Kp));
  {
    const int64_t work = (int64_t)Np * Kp;
    dim3 g((unsigned)std::min<int64_t>(ceil_div(work, 256), 256), (unsigned)nseg);
    k_tc_prep_b<<<g, 256, 0, s>>>(a.B, a.ldb, a.b_seg, a.segK, a.K, a.segN, a.N, Np, Kp, bhi, blo);
    note_launch();
    ABG_LAUNCH_CHECK();
  }
  CUtensorMap amap, hmap, lmap;
  {
    const cuuint64_t dims[2] = {(cuuint64_t)a.K, (cuuint64_t)rs.rows};
    const cuuint64_t strides[1] = {(cuuint64_t)a.lda * 4};
    const cuuint32_t box[2] = {(cuuint32_t)kTcBK, (cuuint32_t)kTcM};
    const cuuint32_t es[2] = {1, 1};
    if (enc(&amap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(a.A), dims, strides, box,
            es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return ABG_OK;
  }
  {
    const cuuint64_t dims[2] = {(cuuint64_t)Kp, (cuuint64_t)nseg * Np};
    const cuuint64_t strides[1] = {(cuuint64_t)Kp * 4};
    const cuuint32_t box[2] = {(cuuint32_t)kTcBK, (cuuint32_t)Np};
    const cuuint32_t es[2] = {1, 1};
    if (enc(&hmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, bhi, dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS ||
        enc(&lmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, blo, dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return ABG_OK;
  }
  TcArgs p{};
  ABG_TRY(current_flag(&p.wait_err));
  p.nkb = nkb;
  p.Np = Np;
  p.N = a.N;
  p.K = a.K;
  p.segN = a.segN;
  p.segK = a.segK;
  p.tile_seg = rs.tile_seg;
  p.tile_row0 = rs.tile_row0;
  p.tile_rows = rs.tile_rows;
  p.C = a.C;
  p.ldc = a.ldc;
  p.epi = (int)a.epi;
  p.aux = a.aux;
  p.ldaux = a.ldaux;
  p.aux2 = a.aux2;
  p.ldaux2 = a.ldaux2;
  p.aux_vec = a.ldaux % 4 == 0 && a.ldaux2 % 4 == 0 &&
              reinterpret_cast<uintptr_t>(a.aux) % 16 == 0 &&
              reinterpret_cast<uintptr_t>(a.aux2) % 16 == 0;
  p.sign = a.sign;
  p.sign_seg = a.sign_seg;
  p.labels = a.labels;
  p.margin = a.margin;
  p.first = a.first;
  p.changes = a.changes;
  p.minbits = a.minbits;
  p.sincos = a.sincos ? 1 : 0;
  p.in_scale = a.in_scale;
  p.out_scale = a.out_scale;
  p.colsum = a.colsum_part;
  // A in tensor memory when two 128-column accumulators leave room for the A slots
  const bool atm = Np <= 128 && !a_tmem_off();
  p.b_bytes = (uint32_t)Np * kTcBK * 4;
  p.stage_bytes = (atm ? 1 : 2) * kTcABytes + 2 * p.b_bytes;  // multiple of 1024
  p.stages = (int)std::max<int64_t>(2, std::min<int64_t>(4, (200 * 1024) / p.stage_bytes));
  if (atm) {
    p.tmem_cols = 512;  // accumulators at 0 and 128, A slots of 64 columns from 256
  } else {
    p.tmem_cols = 64;  // two accumulator buffers of a power of two >= 32 columns each
    while ((int)p.tmem_cols < 2 * Np) p.tmem_cols *= 2;
  }
  // stages, alignment slack, barriers, and for the sin/cos epilogue its column-sum scratch
  const size_t smem = (size_t)p.stages * p.stage_bytes + 1024 +
                      round_up(8 * (3 * p.stages + 4), 16) +
                      (a.sincos ? sizeof(float) * 8 * (size_t)Np : 0);
  if (smem > 227 * 1024) return ABG_OK;
  // warp layouts: the argmax epilogue is the slow part of the NCI scores (two epilogue
  // groups); the plain products are bound by the tf32 split (eight split warps); the sin/cos
  // epilogue's registers leave room for the base layout only
  const unsigned grid = (unsigned)std::min<int64_t>(rs.n_tiles, num_sms());
  auto launch = [&](auto kern, int warps) -> int {
    ABG_TRY(raise_smem_limit((const void*)kern, smem));
    kern<<<grid, 32 * warps, smem, s>>>(amap, hmap, lmap, p, rs.n_tiles);
    return ABG_OK;
  };
  if (a.argmax) {
    ABG_TRY(atm ? launch(k_tc_nn<1, 4, 2, true>, 14) : launch(k_tc_nn<1, 4, 2, false>, 14));
  } else if (a.sincos) {
    ABG_TRY(atm ? launch(k_tc_nn<2, 4, 1, true>, 10) : launch(k_tc_nn<2, 4, 1, false>, 10));
  } else {
    ABG_TRY(atm ? launch(k_tc_nn<0, 8, 1, true>, 14) : launch(k_tc_nn<0, 8, 1, false>, 14));
  }
  note_launch();
  note_tc_launch();
  ABG_LAUNCH_CHECK();
  *used = true;
  return ABG_OK;
}

// ABG_TC_TN_SWAP=0 keeps the two 128-row M blocks for K > 128
static bool swap_off() {
  static const bool off = [] {
    const char* e = std::getenv("ABG_TC_TN_SWAP");
    return e && e[0] == '0';
  }();
  return off;
}

// k_tc_tn2 for N <= 128 when two operand sets fit; false in *used otherwise
static int tc_gemm_tn2(const RowSpace& rs, const TN& a, float* part, cudaStream_t s, bool* used) {
  constexpr int TW = 8;
  *used = false;
  Tn2Args p{};
  p.K = a.K;
  p.N = a.N;
  p.Np = (int)round_up(a.N, 16);
  p.mblk = (int)ceil_div(a.K, kTcM);
  if (p.Np > 128 || p.mblk > 2) return ABG_OK;
  // a Gram matrix (A == B, K == N <= 128): B's operand is the first Np rows of A's, so B is
  // neither staged nor transposed
  p.syrk = a.A == a.B && a.K == a.N && a.lda == a.ldb && a.segK == a.segN && p.mblk == 1;
  // units per transposing thread: A (mblk 128 / 4 column groups) and B (Np / 4), x 8 row
  // groups, in warps of 4 column groups (k_tc_tn2 holds at most kTn2Units per thread)
  const int64_t units =
      ceil_div(p.mblk * kTcM / 4, 4) * 32 + (p.syrk ? 0 : ceil_div(p.Np / 4, 4) * 32);
  if (units > kTn2Units * 32 * TW) return ABG_OK;
  const int U = (int)ceil_div(units, 32 * TW);  // units per transposing thread
  p.stage_bytes = 32u * TW * (uint32_t)U * 64u;
  ABG_TRY(current_flag(&p.wait_err));
  p.A = a.A;
  p.lda = a.lda;
  p.B = a.B;
  p.ldb = a.ldb;
  p.segK = a.segK;
  p.segN = a.segN;
  p.chunk_seg = rs.chunk_seg;
  p.chunk_row0 = rs.chunk_row0;
  p.chunk_rows = rs.chunk_rows;
  p.part = part;
  // K > 128: one MMA per term covers both 128-column halves of A when B (<= 128 columns, its
  // operand padded to 128 rows) takes the MMA's M and A's 256 columns its N
  p.swap = p.mblk == 2 && !p.syrk && !swap_off();
  p.op_bytes = 2u * p.mblk * kTcM * 128 +
               (p.syrk ? 0u : 2u * (uint32_t)(p.swap ? kTcM : p.Np) * 128);
  p.acc_cols = 32;
  while ((int)p.acc_cols < (p.swap ? p.mblk * kTcM : p.mblk * p.Np)) p.acc_cols *= 2;
  p.tmem_cols = 2 * p.acc_cols;
  if (p.tmem_cols > 512) return ABG_OK;
  size_t smem = 0;
  for (p.nops = 2; p.nops >= 1; --p.nops) {
    smem = 1024 + (size_t)p.nops * p.op_bytes + 2 * (size_t)p.stage_bytes + 8 * (2 * p.nops + 5);
    if (smem <= 220 * 1024) break;
  }
  if (p.nops < 1) return ABG_OK;
  ABG_TRY(raise_smem_limit((const void*)k_tc_tn2<TW>, smem));
  const unsigned grid = (unsigned)std::min<int64_t>(rs.n_chunks, num_sms());
  k_tc_tn2<TW><<<grid, 32 * (TW + 5), smem, s>>>(p, rs.n_chunks);
  note_launch();
  note_tc_launch();
  ABG_LAUNCH_CHECK();
  *used = true;
  return ABG_OK;
}

int tc_gemm_tn(const RowSpace& rs, const TN& a, float* part, cudaStream_t s, bool* used) {
  *used = false;
  if (tc_disabled() || a.K > 256 || a.N > 256 || rs.n_chunks == 0) return ABG_OK;
  if (a.lda % 4 != 0 || a.ldb % 4 != 0 || reinterpret_cast<uintptr_t>(a.A) % 16 != 0 ||
      reinterpret_cast<uintptr_t>(a.B) % 16 != 0 || rs.rows > INT32_MAX)
    return ABG_OK;
  ABG_TRY(tc_gemm_tn2(rs, a, part, s, used));
  if (*used) return ABG_OK;
  const auto enc = tensor_map_encoder();
  if (!enc) return ABG_OK;
  TnArgs p{};
  ABG_TRY(current_flag(&p.wait_err));
  p.K = a.K;
  p.N = a.N;
  p.Np = (int)round_up(a.N, 16);
  p.mblk = (int)ceil_div(a.K, kTcM);
  p.ka_box = (int)round_up(a.K, 4);
  p.nb_box = (int)round_up(a.N, 4);
  p.segK = a.segK;
  p.segN = a.segN;
  p.chunk_seg = rs.chunk_seg;
  p.chunk_row0 = rs.chunk_row0;
  p.chunk_rows = rs.chunk_rows;
  p.part = part;
  p.raw_a_bytes = (uint32_t)round_up((int64_t)kTnRows * p.ka_box * 4, 128);
  p.raw_bytes = p.raw_a_bytes + (uint32_t)round_up((int64_t)kTnRows * p.nb_box * 4, 128);
  p.op_bytes = 2u * p.mblk * kTcM * 128 + 2u * p.Np * 128;
  p.tmem_cols = 32;
  while ((int)p.tmem_cols < p.mblk * p.Np) p.tmem_cols *= 2;
  if (p.tmem_cols > 512) return ABG_OK;
  size_t smem = 0;
  bool fits = false;
  for (p.nops = ABG_TN_NOPS; p.nops >= 1 && !fits; --p.nops) {
    for (p.stages = 4; p.stages >= 2; --p.stages) {
      smem = 1024 + (size_t)p.nops * p.op_bytes + (size_t)p.stages * p.raw_bytes +
             8 * (2 * p.stages + 2 * p.nops + 2);
      if (smem <= 220 * 1024) {
        fits = true;
        break;
      }
    }
    if (fits) break;
  }
  if (!fits) return ABG_OK;
  CUtensorMap amap, bmap;
  {
    const cuuint64_t dims[2] = {(cuuint64_t)a.K, (cuuint64_t)rs.rows};
    const cuuint64_t strides[1] = {(cuuint64_t)a.lda * 4};
    const cuuint32_t box[2] = {(cuuint32_t)p.ka_box, (cuuint32_t)kTnRows};
    const cuuint32_t es[2] = {1, 1};
    if (enc(&amap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(a.A), dims, strides, box,
            es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return ABG_OK;
  }
  {
    const cuuint64_t dims[2] = {(cuuint64_t)a.N, (cuuint64_t)rs.rows};
    const cuuint64_t strides[1] = {(cuuint64_t)a.ldb * 4};
    const cuuint32_t box[2] = {(cuuint32_t)p.nb_box, (cuuint32_t)kTnRows};
    const cuuint32_t es[2] = {1, 1};
    if (enc(&bmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(a.B), dims, strides, box,
            es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return ABG_OK;
  }
  ABG_TRY(raise_smem_limit((const void*)k_tc_tn, smem));
  const unsigned grid = (unsigned)std::min<int64_t>(rs.n_chunks, num_sms());
  k_tc_tn<<<grid, kTcThreads, smem, s>>>(amap, bmap, p, rs.n_chunks);
  note_launch();
  note_tc_launch();
  ABG_LAUNCH_CHECK();
  *used = true;
  return ABG_OK;
}

int tc_gemm_nn16(const RowSpace& rs, const NN& a, cudaStream_t s, bool* used) {
  *used = false;
  if (!a.A16 || a.segK || a.argmax || a.sincos || tc_disabled()) return ABG_OK;
  if (a.ldc % 4 != 0 || reinterpret_cast<uintptr_t>(a.C) % 16 != 0) return ABG_OK;
  if (a.N > 256 || rs.n_tiles == 0 || rs.rows > INT32_MAX) return ABG_OK;
  if (a.lda16 % 8 != 0 || reinterpret_cast<uintptr_t>(a.A16) % 16 != 0) return ABG_OK;
  const auto enc = tensor_map_encoder();
  if (!enc) return ABG_OK;
  const int nseg = rs.nseg;
  const int Np = (int)round_up(a.N, 16);
  const int nkb = (int)ceil_div(a.K, kBK16);
  const int Kp = nkb * kBK16;
  if ((int64_t)nseg * Np > INT32_MAX) return ABG_OK;
  Scratch scr(s);
  __nv_bfloat16* b16;
  ABG_TRY(scr.get(&b16, (size_t)nseg * Np * Kp));
  {
    const int64_t work = (int64_t)Np * Kp;
    dim3 g((unsigned)std::min<int64_t>(ceil_div(work, 256), 256), (unsigned)nseg);
    k_tc_prep_b16<<<g, 256, 0, s>>>(a.B, a.ldb, a.b_seg, nullptr, a.K, a.segN, a.N, Np, Kp, b16);
    note_launch();
    ABG_LAUNCH_CHECK();
  }
  CUtensorMap amap, bmap;
  const cuuint32_t es[2] = {1, 1};
  {
    const cuuint64_t dims[2] = {(cuuint64_t)a.K, (cuuint64_t)rs.rows};
    const cuuint64_t strides[1] = {(cuuint64_t)a.lda16 * 2};
    const cuuint32_t box[2] = {(cuuint32_t)kBK16, (cuuint32_t)kTcM};
    if (enc(&amap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16*>(a.A16), dims,
            strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return ABG_OK;
  }
  {
    const cuuint64_t dims[2] = {(cuuint64_t)Kp, (cuuint64_t)nseg * Np};
    const cuuint64_t strides[1] = {(cuuint64_t)Kp * 2};
    const cuuint32_t box[2] = {(cuuint32_t)kBK16, (cuuint32_t)Np};
    if (enc(&bmap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, b16, dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return ABG_OK;
  }
  TcArgs p{};
  ABG_TRY(current_flag(&p.wait_err));
  p.nkb = nkb;
  p.Np = Np;
  p.N = a.N;
  p.K = a.K;
  p.segN = a.segN;
  p.tile_seg = rs.tile_seg;
  p.tile_row0 = rs.tile_row0;
  p.tile_rows = rs.tile_rows;
  p.C = a.C;
  p.ldc = a.ldc;
  p.epi = (int)a.epi;
  p.aux = a.aux;
  p.ldaux = a.ldaux;
  p.aux2 = a.aux2;
  p.ldaux2 = a.ldaux2;
  p.aux_vec = a.ldaux % 4 == 0 && a.ldaux2 % 4 == 0 &&
              reinterpret_cast<uintptr_t>(a.aux) % 16 == 0 &&
              reinterpret_cast<uintptr_t>(a.aux2) % 16 == 0;
  p.sign = a.sign;
  p.sign_seg = a.sign_seg;
  p.b_bytes = (uint32_t)Np * 128;  // one 64-wide K block of B
  const size_t cap = 220 * 1024 - 1024 - 8 * (2 * 8 + 5);
  p.b_resident = nseg == 1 && (size_t)nkb * p.b_bytes + 2 * kA16Bytes <= cap;
  p.stage_bytes = kA16Bytes + (p.b_resident ? 0u : p.b_bytes);
  const size_t bres = p.b_resident ? (size_t)nkb * p.b_bytes : 0;
  p.stages = (int)std::min<size_t>(8, (cap - bres) / p.stage_bytes);
  if (p.stages < 2) return ABG_OK;
  p.tmem_cols = 64;
  while ((int)p.tmem_cols < 2 * Np) p.tmem_cols *= 2;
  const size_t smem = bres + (size_t)p.stages * p.stage_bytes + 1024 + 8 * (2 * p.stages + 5);
  ABG_TRY(raise_smem_limit((const void*)k_tc_nn16, smem));
  const unsigned grid = (unsigned)std::min<int64_t>(rs.n_tiles, num_sms());
  k_tc_nn16<<<grid, kNn16Threads, smem, s>>>(amap, bmap, p, rs.n_tiles);
  note_launch();
  note_tc_launch();
  ABG_LAUNCH_CHECK();
  *used = true;
  return ABG_OK;
}

int tc_gemm_tn16(const RowSpace& rs, const TN& a, float* part, cudaStream_t s, bool* used) {
  *used = false;
  if (!a.A16 || a.segK || tc_disabled() || a.K > 256 || a.N > 256 || rs.n_chunks == 0)
    return ABG_OK;
  if (a.lda16 % 8 != 0 || a.ldb % 4 != 0 || reinterpret_cast<uintptr_t>(a.A16) % 16 != 0 ||
      reinterpret_cast<uintptr_t>(a.B) % 16 != 0 || rs.rows > INT32_MAX)
    return ABG_OK;
  const auto enc = tensor_map_encoder();
  if (!enc) return ABG_OK;
  TnArgs p{};
  ABG_TRY(current_flag(&p.wait_err));
  p.K = a.K;
  p.N = a.N;
  p.Np = (int)round_up(a.N, 16);
  p.mblk = (int)ceil_div(a.K, kTcM);
  p.nb_box = (int)round_up(a.N, 4);
  p.segN = a.segN;
  p.chunk_seg = rs.chunk_seg;
  p.chunk_row0 = rs.chunk_row0;
  p.chunk_rows = rs.chunk_rows;
  p.part = part;
  p.raw_a_bytes = 2u * p.mblk * kMnBox;
  p.raw_bytes = (uint32_t)round_up((int64_t)p.raw_a_bytes + (int64_t)kTn16Rows * p.nb_box * 4, 1024);
  p.op_bytes = (uint32_t)ceil_div(p.Np, 64) * kMnBox;
  p.tmem_cols = 32;
  while ((int)p.tmem_cols < p.mblk * p.Np) p.tmem_cols *= 2;
  if (p.tmem_cols > 512) return ABG_OK;
  size_t smem = 0;
  bool fits = false;
  for (p.nops = 2; p.nops >= 1 && !fits; --p.nops) {
    for (p.stages = 4; p.stages >= 2; --p.stages) {
      smem = 1024 + (size_t)p.nops * p.op_bytes + (size_t)p.stages * p.raw_bytes +
             8 * (2 * p.stages + 2 * p.nops + 2);
      if (smem <= 220 * 1024) {
        fits = true;
        break;
      }
    }
    if (fits) break;
  }
  if (!fits) return ABG_OK;
  CUtensorMap amap, bmap;
  const cuuint32_t es[2] = {1, 1};
  {
    const cuuint64_t dims[2] = {(cuuint64_t)a.K, (cuuint64_t)rs.rows};
    const cuuint64_t strides[1] = {(cuuint64_t)a.lda16 * 2};
    const cuuint32_t box[2] = {64, (cuuint32_t)kTn16Rows};
    if (enc(&amap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16*>(a.A16), dims,
            strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return ABG_OK;
  }
  {
    const cuuint64_t dims[2] = {(cuuint64_t)a.N, (cuuint64_t)rs.rows};
    const cuuint64_t strides[1] = {(cuuint64_t)a.ldb * 4};
    const cuuint32_t box[2] = {(cuuint32_t)p.nb_box, (cuuint32_t)kTn16Rows};
    if (enc(&bmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(a.B), dims, strides, box,
            es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return ABG_OK;
  }
  ABG_TRY(raise_smem_limit((const void*)k_tc_tn16, smem));
  const unsigned grid = (unsigned)std::min<int64_t>(rs.n_chunks, num_sms());
  k_tc_tn16<<<grid, kTcThreads, smem, s>>>(amap, bmap, p, rs.n_chunks);
  note_launch();
  note_tc_launch();
  ABG_LAUNCH_CHECK();
  *used = true;
  return ABG_OK;
}

}  // namespace abg
