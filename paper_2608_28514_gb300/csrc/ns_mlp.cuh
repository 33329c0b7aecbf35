// ns_mlp.cuh -- the emulator-style likelihood of the benchmark suite:
// log L = -1/2 sum_k ((MLP(theta)_k - data_k) / sigma_k)^2 with a SiLU MLP
// (the stand-in for the neural-network emulator of section 5).
//
// Two evaluators of a batch of candidate points:
//  * BF16 on the 5th-generation tensor cores (tcgen05): per layer, the
//    weights W [out][in] are the A operand (M = 128 output features per
//    tile, K-major), the batch of candidates the B operand (N <= kMlpNbMax
//    points, K-major), the FP32 accumulators live in tensor memory.  Weight
//    tiles are packed once, on the host, into the exact 128-byte-swizzled
//    shared-memory image of one 128 x 64 BF16 tile (16 KB) and streamed by
//    the TMA engine (cp.async.bulk) through a ring of shared-memory stages;
//    one thread issues the MMAs; four warps read the accumulators back
//    (tcgen05.ld), add the bias, apply SiLU and write BF16 activations
//    straight into the next layer's swizzled B operand.  The last layer's
//    epilogue forms the chi^2 per candidate.
//  * FP32 on the CUDA cores (the FP32 path and the re-evaluation of points
//    near the threshold).
//
// Every wait on an mbarrier is bounded; on a timeout the block sets an error
// flag, drains its own copies, frees its tensor memory and returns.
#pragma once

#include <cuda_bf16.h>

#include "ns_device.cuh"

namespace nsd {

constexpr int kMlpMaxLayers = 8;
constexpr int kMlpNbMax = 128;    // candidates per call, at most (the MMA's N)
constexpr int kMlpStagesMax = 4;  // weight tiles in flight, at most
constexpr int kMlpTileBytes = 128 * 128;  // 128 rows x 64 BF16 (128 bytes)
constexpr int kMlpMaxK = 512;     // widest padded layer input
constexpr unsigned kMlpWaitCap = 1u << 22;

// Offsets into the packed image (host-built, device-resident):
//   tiles  : BF16 swizzled weight tiles, layer by layer, M-tile by M-tile,
//            K-block by K-block (16 KB each);
//   f32    : per layer bias (padded out), then data and 1/sigma of the last
//            layer (padded out), then the FP32 weights transposed, [in][out]
//            (as BF16 bit patterns, two per float slot, when every weight is
//            a BF16 value: the FP32 arithmetic then reads half the bytes).
struct MlpDesc {
  int n_layers, d;
  int in[kMlpMaxLayers], out[kMlpMaxLayers];        // true widths
  int kpad[kMlpMaxLayers], mpad[kMlpMaxLayers];      // in padded to 64, out padded to 128
  int tile0[kMlpMaxLayers];                          // index of the layer's first tile
  long long bias0[kMlpMaxLayers];                    // float offset of the layer's bias
  long long w32_0[kMlpMaxLayers];                    // float offset of the layer's FP32 weights
  long long data0, isig0;                            // float offsets (last layer, padded)
  int n_tiles;
  int w_bf16;  // the FP32 master weights are all BF16 values: stored as BF16 (exact), read as FP32
  long long tile_bytes, f32_floats;
  float lo[kMaxDim], span[kMaxDim];
};

// ---------------------------------------------------------------------------
// PTX wrappers (sm_100+)
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n.reg .pred p;\n"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      "selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: false if the barrier did not flip within kMlpWaitCap tries.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
  for (unsigned i = 0; i < kMlpWaitCap; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(unsigned* slot, unsigned ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(slot)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(unsigned taddr, unsigned ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(ncols) : "memory");
}

// D[tmem] (+)= A[smem] * B[smem]^T, kind::f16 (BF16 in, FP32 accumulate).
__device__ __forceinline__ void umma_bf16(unsigned d_tmem, uint64_t adesc, uint64_t bdesc, unsigned idesc,
                                          unsigned accumulate) {
  asm volatile(
      "{\n.reg .pred p;\n"
      "setp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                   smem_u32(bar))
               : "memory");
}

// 32 lanes x 32 bits, 16 consecutive columns per thread.
__device__ __forceinline__ void tmem_ld16(unsigned taddr, float (&v)[16]) {
  unsigned r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle; rows of 128
// bytes, 8-row atoms 1024 bytes apart (stride byte offset), descriptor
// version 1 (bits 46-47), layout type 2 = SWIZZLE_128B (bits 61-63).
__device__ __forceinline__ uint64_t sdesc_sw128(unsigned saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// Instruction descriptor, kind::f16: D FP32 (bits 4-5 = 1), A and B BF16
// (bits 7-9 = 1, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 in
// bits 17-22, M >> 4 in bits 24-28.
__host__ __device__ constexpr unsigned idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(N >> 3) << 17) | ((unsigned)(M >> 4) << 24);
}

// Byte offset of element (row r, k) of a 128-byte-swizzled K-major tile
// whose rows hold 64 BF16 (1024-byte aligned base).
__host__ __device__ __forceinline__ unsigned sw128_offset(int r, int k) {
  const unsigned byte = (unsigned)k * 2u;
  return (unsigned)r * 128u + ((((byte >> 4) ^ (unsigned)(r & 7)) & 7u) << 4) + (byte & 15u);
}

__device__ __forceinline__ float silu(float z) { return z / (1.f + expf(-z)); }

// SiLU of the BF16 path's epilogues: exp and divide on the special-function
// unit (relative error near FP32 rounding, far below the BF16 rounding of
// the stored activation).
__device__ __forceinline__ float silu_fast(float z) { return __fdividef(z, 1.f + __expf(-z)); }

// Shared memory of the BF16 evaluator (offsets from a 1024-aligned base):
// STAGES weight tiles, the B operand for up to NBMAX candidates, chi^2
// partials.  The streaming of weight tiles from L2 is throughput-bound, not
// latency-bound, so a few stages suffice.
// P = 3: the FP32-accurate variant (activations as three BF16 planes).
template <int NBMAX, int STAGES, int P = 1>
struct MlpSmem {
  static_assert(NBMAX % 16 == 0 && NBMAX <= kMlpNbMax && STAGES >= 2 && STAGES <= kMlpStagesMax, "");
  static_assert(P >= 1 && P <= 3, "");
  static constexpr int kStageOff = 0;
  static constexpr int kActOff = kStageOff + STAGES * kMlpTileBytes;  // [P][kpad/64][NBMAX][128 B]
  static constexpr int kPlaneBytes = (kMlpMaxK / 64) * NBMAX * 128;
  static constexpr int kActBytes = P * kPlaneBytes;
  static constexpr int kChiOff = kActOff + kActBytes;                 // [4][NBMAX] floats
  static constexpr int kBytes = kChiOff + 4 * NBMAX * 4;
};

// a = hi + mid + lo exactly, each a BF16 value (8 significand bits each;
// the remainders a - hi and (a - hi) - mid are exact in FP32).
__device__ __forceinline__ void split3_bf16(float a, __nv_bfloat16& hi, __nv_bfloat16& mid, __nv_bfloat16& lo) {
  hi = __float2bfloat16_rn(a);
  const float r1 = a - __bfloat162float(hi);
  mid = __float2bfloat16_rn(r1);
  lo = __float2bfloat16_rn(r1 - __bfloat162float(mid));
}

// The value v of one operand element as P BF16 planes at dst, dst +
// plane_bytes, dst + 2 plane_bytes: P = 1 rounds it to BF16; P = 2 keeps 16
// significand bits (hi + lo, lo the BF16 rounding of the exact remainder,
// relative error at most 2^-17); P = 3 keeps all of it (hi + mid + lo).
template <int P>
__device__ __forceinline__ void store_planes(char* dst, int plane_bytes, float v) {
  if constexpr (P == 1) {
    *reinterpret_cast<__nv_bfloat16*>(dst) = __float2bfloat16_rn(v);
  } else if constexpr (P == 2) {
    const __nv_bfloat16 hi = __float2bfloat16_rn(v);
    *reinterpret_cast<__nv_bfloat16*>(dst) = hi;
    *reinterpret_cast<__nv_bfloat16*>(dst + plane_bytes) = __float2bfloat16_rn(v - __bfloat162float(hi));
  } else {
    __nv_bfloat16 h0, h1, h2;
    split3_bf16(v, h0, h1, h2);
    *reinterpret_cast<__nv_bfloat16*>(dst) = h0;
    *reinterpret_cast<__nv_bfloat16*>(dst + plane_bytes) = h1;
    *reinterpret_cast<__nv_bfloat16*>(dst + 2 * plane_bytes) = h2;
  }
}

// Warp roles of the BF16 evaluator: warps 0-7 read the accumulators back
// (warp w owns tensor-memory lanes 32(w%4)..32(w%4)+31 and every other
// 16-column chunk, starting at chunk w/4), warp 8 streams the weight tiles,
// warp 9 issues the MMAs.  The block needs at least kMlpThreads threads.
constexpr int kMlpEpiWarps = 8;
constexpr int kMlpProducerWarp = 8;
constexpr int kMlpMmaWarp = 9;
constexpr int kMlpThreads = 320;
// tensor memory: two halves of 256 columns; an output-layer group of M-tiles
// fills one half while the epilogue drains the other
constexpr int kMlpHalfCols = 256;

// Per-block state of the BF16 evaluator that outlives one call: the tensor
// memory, the mbarriers of the weight-tile ring and of the two accumulator
// halves, and the running counters their phases follow.  Static shared
// memory, set up once per block (mlp_ctx_init) and released before the
// block exits (mlp_ctx_free).  An error (a wait that gave up) is sticky.
struct MlpCtx {
  uint64_t full[kMlpStagesMax], empty[kMlpStagesMax];
  uint64_t acc_full[2], acc_free[2], drain;
  // evaluation split over a thread-block cluster (ns_mlp_cluster.cuh): the
  // peers' slices of a layer's input have landed (one local arrive with the
  // expected bytes); every peer has finished a layer's MMAs (one remote
  // arrive per peer)
  uint64_t act_ready, peer_free;
  unsigned tmem;
  unsigned item;      // weight tiles consumed so far
  unsigned uses[2];   // groups that have used each accumulator half
  unsigned xu;        // act_ready phases waited for (cluster split)
  unsigned xu_armed;  // act_ready phases armed
  unsigned pu;        // peer_free phases waited for
  unsigned err;
};

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void epi_bar_sync() {
  asm volatile("bar.sync 1, %0;\n" ::"n"(kMlpEpiWarps * 32) : "memory");
}
__device__ __forceinline__ unsigned ctx_err(const MlpCtx* c) { return *reinterpret_cast<const volatile unsigned*>(&c->err); }
__device__ __forceinline__ void ctx_set_err(MlpCtx* c) { *reinterpret_cast<volatile unsigned*>(&c->err) = 1u; }

// Called by every thread of the block.
inline __device__ void mlp_ctx_init(MlpCtx* c) {
  const int tid = threadIdx.x;
  if ((tid >> 5) == 0) tmem_alloc(&c->tmem, 512);
  if (tid == 0) {
    for (int s = 0; s < kMlpStagesMax; ++s) {
      mbar_init(&c->full[s], 1);
      mbar_init(&c->empty[s], 1);
    }
    for (int h = 0; h < 2; ++h) {
      mbar_init(&c->acc_full[h], 1);
      mbar_init(&c->acc_free[h], kMlpEpiWarps * 32);
    }
    mbar_init(&c->drain, 1);
    unsigned ncta;
    asm volatile("mov.u32 %0, %%cluster_nctarank;\n" : "=r"(ncta));
    mbar_init(&c->act_ready, 1);
    mbar_init(&c->peer_free, ncta > 1 ? ncta - 1 : 1);
    mbar_fence_init();
    c->item = 0u;
    c->uses[0] = c->uses[1] = 0u;
    c->xu = c->xu_armed = c->pu = 0u;
    c->err = 0u;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
}
inline __device__ void mlp_ctx_free(MlpCtx* c) {
  tc_fence_before();
  __syncthreads();
  if ((threadIdx.x >> 5) == 0) tmem_dealloc(c->tmem, 512);
  __syncthreads();
}

// 1024-byte aligned start (in the shared window) of a region beginning at p.
__device__ __forceinline__ char* align1024_shared(char* p) {
  const unsigned a = smem_u32(p);
  return p + ((1024u - (a & 1023u)) & 1023u);
}

// Sum over the warp of 16 values per lane: lane L returns the total of
// column (L >> 1) & 15 (butterfly reduce-scatter, 16 shuffles).
__device__ __forceinline__ float warp_sum16(const float (&s)[16], int lane) {
  float a[8], b[4], c[2];
  const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4, b1 = lane & 2;
#pragma unroll
  for (int j = 0; j < 8; ++j) a[j] = (b4 ? s[j + 8] : s[j]) + __shfl_xor_sync(kFull, b4 ? s[j] : s[j + 8], 16);
#pragma unroll
  for (int j = 0; j < 4; ++j) b[j] = (b3 ? a[j + 4] : a[j]) + __shfl_xor_sync(kFull, b3 ? a[j] : a[j + 4], 8);
#pragma unroll
  for (int j = 0; j < 2; ++j) c[j] = (b2 ? b[j + 2] : b[j]) + __shfl_xor_sync(kFull, b2 ? b[j] : b[j + 2], 4);
  float d = (b1 ? c[1] : c[0]) + __shfl_xor_sync(kFull, b1 ? c[0] : c[1], 2);
  return d + __shfl_xor_sync(kFull, d, 1);
}

// How a layer's M-tiles are grouped on the accumulator halves for a call
// with N candidates.  Hidden layers: one group of all M-tiles from column 0
// (the next layer's input is written in place, so the layer's MMAs must all
// be done first; MT x N <= 512).  Output layer: groups of 256 / N M-tiles,
// alternating halves.
struct MlpGroup {
  int g0, g1, h0, nh;
};
__device__ __forceinline__ MlpGroup mlp_group(int MT, bool last, int gi, int N) {
  MlpGroup G;
  if (!last) {
    G.g0 = 0;
    G.g1 = MT;
    G.h0 = 0;
    G.nh = (MT * N > kMlpHalfCols) ? 2 : 1;
  } else {
    const int per = kMlpHalfCols / N;
    G.g0 = gi * per;
    G.g1 = min(MT, G.g0 + per);
    G.h0 = gi & 1;
    G.nh = 1;
  }
  return G;
}
__device__ __forceinline__ int mlp_n_groups(int MT, bool last, int N) {
  const int per = kMlpHalfCols / N;
  return last ? (MT + per - 1) / per : 1;
}

// Evaluates the batch x [n][d] (unit cube, 1 <= n <= NBMAX) with the BF16
// tensor-core path into out[n] (log L); the MMAs run with N = n rounded up
// to 16.  With `rows` non-null, candidate r is row rows[r] of x and its
// log L goes to out[rows[r]] (a gather/scatter by index list).
// P = 3 evaluates in FP32 accuracy on the same tensor cores, for networks
// whose weights are BF16 values: every activation (and the input) is split
// exactly into three BF16 planes, each weight tile multiplies all three
// (products of two BF16 values are exact in FP32, the accumulation is FP32),
// and the epilogues run in FP32 (accurate SiLU; the output residual as
// (y + bias - data) / sigma).  It differs from the CUDA-core FP32 evaluator
// only in the order of the FP32 sums.  Called by every thread of a block of at least kMlpThreads threads,
// with the block's context `ctx` (mlp_ctx_init).  `sm` is 1024-byte aligned
// and holds MlpSmem<NBMAX, STAGES>::kBytes.  Returns false (for every
// thread) if a wait gave up, now or before.
template <int NBMAX, int STAGES, int P = 1>
inline __device__ bool mlp_eval_bf16(const MlpDesc& M, const uint8_t* __restrict__ tiles,
                                     const float* __restrict__ f32, const float* x, int x_stride, int n,
                                     float* out, char* sm, MlpCtx* ctx, const int* rows = nullptr) {
  using L = MlpSmem<NBMAX, STAGES, P>;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  char* stages = sm + L::kStageOff;
  char* act = sm + L::kActOff;
  float* chi = reinterpret_cast<float*>(sm + L::kChiOff);
  constexpr unsigned S = STAGES;
  if (ctx_err(ctx)) return false;  // uniform: nothing writes it between calls
  const int N = (n + 15) & ~15;
  const unsigned item0 = ctx->item, use0 = ctx->uses[0], use1 = ctx->uses[1];
  const unsigned tmem = ctx->tmem;
  const int last = M.n_layers - 1;

  // layer-0 input: theta = lo + span x in BF16, rows = candidates, K = d (pad 0)
  const int kb0 = M.kpad[0] / 64;
  for (int q = tid; q < kb0 * N * 64; q += blockDim.x) {
    const int kb = q / (N * 64), rem = q % (N * 64), r = rem / 64, k = rem % 64;
    const int i = kb * 64 + k;
    float v = 0.f;
    if (r < n && i < M.d) v = fmaf(M.span[i], x[(size_t)(rows ? rows[r] : r) * x_stride + i], M.lo[i]);
    char* dst = act + kb * NBMAX * 128 + sw128_offset(r, k);
    store_planes<P>(dst, L::kPlaneBytes, v);
  }
  for (int q = tid; q < 4 * NBMAX; q += blockDim.x) chi[q] = 0.f;
  fence_proxy_async();
  __syncthreads();

  if (warp == kMlpProducerWarp) {
    // weight tiles in consumption order = image order
    if (lane == 0) {
      const unsigned end = item0 + (unsigned)M.n_tiles;
      unsigned it = item0;
      bool err = false;
      for (; it < end; ++it) {
        const unsigned s = it % S;
        if (ctx_err(ctx) || (it >= S && !mbar_wait(&ctx->empty[s], ((it / S) - 1) & 1))) {
          err = true;
          break;
        }
        mbar_expect_tx(&ctx->full[s], kMlpTileBytes);
        bulk_g2s(stages + s * kMlpTileBytes, tiles + (size_t)(it - item0) * kMlpTileBytes, kMlpTileBytes,
                 &ctx->full[s]);
      }
      if (err) {
        ctx_set_err(ctx);
        // every copy issued lands before the block moves on (only the last S can be outstanding)
        for (unsigned j = (it - item0 > S) ? it - S : item0; j < it; ++j) mbar_wait(&ctx->full[j % S], (j / S) & 1);
      }
    }
    __syncwarp();
  } else if (warp == kMlpMmaWarp) {
    if (lane == 0) {
      const unsigned idesc = idesc_bf16(128, N);
      unsigned it = item0, uses[2] = {use0, use1};
      bool err = false;
      for (int l = 0; l <= last && !err; ++l) {
        const int KB = M.kpad[l] / 64, MT = M.mpad[l] / 128;
        const int ng = mlp_n_groups(MT, l == last, N);
        for (int gi = 0; gi < ng && !err; ++gi) {
          const MlpGroup G = mlp_group(MT, l == last, gi, N);
          // the previous user of each half has been drained; at a layer's
          // first group, of both halves (that epilogue also wrote this layer's input)
          for (int h = 0; h < 2 && !err; ++h) {
            const bool need = (gi == 0) || (h >= G.h0 && h < G.h0 + G.nh);
            if (need && uses[h] > 0 && !mbar_wait(&ctx->acc_free[h], (uses[h] - 1) & 1)) err = true;
          }
          if (err || ctx_err(ctx)) {
            err = true;
            break;
          }
          tc_fence_after();
          const unsigned col0 = (unsigned)G.h0 * kMlpHalfCols;
          for (int t = G.g0; t < G.g1 && !err; ++t) {
            for (int kb = 0; kb < KB; ++kb, ++it) {
              const unsigned s = it % S;
              if (!mbar_wait(&ctx->full[s], (it / S) & 1)) {
                err = true;
                break;
              }
              tc_fence_after();
              const unsigned d_tmem = tmem + col0 + (unsigned)((t - G.g0) * N);
              const unsigned a0 = smem_u32(stages + s * kMlpTileBytes);
#pragma unroll
              for (int pl = 0; pl < P; ++pl) {
                const unsigned b0 = smem_u32(act + pl * L::kPlaneBytes + kb * NBMAX * 128);
#pragma unroll
                for (int k = 0; k < 4; ++k)
                  umma_bf16(d_tmem, sdesc_sw128(a0 + 32 * k), sdesc_sw128(b0 + 32 * k), idesc,
                            (kb > 0 || k > 0 || pl > 0) ? 1u : 0u);
              }
              umma_commit(&ctx->empty[s]);
            }
          }
          if (err) break;
          for (int h = G.h0; h < G.h0 + G.nh; ++h) {
            umma_commit(&ctx->acc_full[h]);
            ++uses[h];
          }
        }
      }
      if (err) {
        ctx_set_err(ctx);
        umma_commit(&ctx->drain);  // the MMAs already issued finish before the block moves on
        mbar_wait(&ctx->drain, 0);
      } else {
        ctx->item = it;
        ctx->uses[0] = uses[0];
        ctx->uses[1] = uses[1];
      }
    }
    __syncwarp();
  } else if (warp < kMlpEpiWarps) {
    const int q = warp & 3, ch = warp >> 2;  // lane quadrant, chunk parity
    const unsigned lane_base = (unsigned)(q * 32) << 16;
    const int n_chunks = N / 16;
    unsigned uses[2] = {use0, use1};
    bool err = false;
    for (int l = 0; l <= last && !err; ++l) {
      const int MT = M.mpad[l] / 128;
      const bool is_last = (l == last);
      const int ng = mlp_n_groups(MT, is_last, N);
      for (int gi = 0; gi < ng && !err; ++gi) {
        const MlpGroup G = mlp_group(MT, is_last, gi, N);
        for (int h = G.h0; h < G.h0 + G.nh; ++h) {
          bool ok = true;
          if (lane == 0) ok = mbar_wait(&ctx->acc_full[h], uses[h] & 1);
          if (!__shfl_sync(kFull, ok ? 1 : 0, 0)) err = true;
        }
        if (err) break;
        tc_fence_after();
        const unsigned col0 = (unsigned)G.h0 * kMlpHalfCols;
        if (!is_last) {
          // bias + SiLU, BF16 straight into the next layer's swizzled B operand
          for (int t = G.g0; t < G.g1; ++t) {
            const int f = t * 128 + q * 32 + lane;
            const float bias = f32[M.bias0[l] + f];
            const int kb = f >> 6, k = f & 63;
            char* dst = act + kb * NBMAX * 128;
            for (int i = ch; i < n_chunks; i += 2) {
              const int c0 = i * 16;
              float v[16];
              tmem_ld16(tmem + lane_base + col0 + (unsigned)((t - G.g0) * N + c0), v);
              // BF16 path: SiLU on the special-function unit; the wider paths: accurate SiLU
#pragma unroll
              for (int c = 0; c < 16; ++c)
                store_planes<P>(dst + sw128_offset(c0 + c, k), L::kPlaneBytes,
                                (P == 1) ? silu_fast(v[c] + bias) : silu(v[c] + bias));
            }
          }
          fence_proxy_async();
        } else {
          // chi^2: per candidate column, one tile of 128 features at a time,
          // added in tile order (so a candidate's value does not depend on
          // its batch: the grouping of tiles follows N)
          for (int i = ch; i < n_chunks; i += 2) {
            const int c0 = i * 16;
            for (int t = G.g0; t < G.g1; ++t) {
              const int f = t * 128 + q * 32 + lane;
              const float is = f32[M.isig0 + f];
              const float bias = f32[M.bias0[l] + f], dk = f32[M.data0 + f];
              const float cb = (bias - dk) * is;
              float v[16], sacc[16];
              tmem_ld16(tmem + lane_base + col0 + (unsigned)((t - G.g0) * N + c0), v);
#pragma unroll
              for (int c = 0; c < 16; ++c) {
                const float r = (P == 1) ? fmaf(v[c], is, cb) : ((v[c] + bias) - dk) * is;
                sacc[c] = r * r;
              }
              const float tot = warp_sum16(sacc, lane);
              if ((lane & 1) == 0) chi[q * NBMAX + c0 + ((lane >> 1) & 15)] += tot;
            }
          }
        }
        tc_fence_before();
        for (int h = G.h0; h < G.h0 + G.nh; ++h) {
          mbar_arrive(&ctx->acc_free[h]);
          ++uses[h];
        }
      }
    }
    if (err) ctx_set_err(ctx);
    epi_bar_sync();
    for (int r = tid; r < n; r += kMlpEpiWarps * 32)
      out[rows ? rows[r] : r] = -0.5f * (chi[r] + chi[NBMAX + r] + chi[2 * NBMAX + r] + chi[3 * NBMAX + r]);
  }
  __syncthreads();
  return ctx_err(ctx) == 0u;
}

// FP32 CUDA-core evaluator: the same function in FP32 (weights = the FP32
// masters, stored transposed [in][out] so that a warp's weight loads are
// coalesced).  One pass evaluates up to NB candidates: thread t owns the
// output features t and t + blockDim.x of each chunk of 2 blockDim.x
// features and keeps their NB accumulators in registers; the activations
// sit transposed in shared memory ([feature][candidate], row stride NB + 4)
// so that one 16-byte broadcast load feeds 4 candidates.  Weights are
// fetched one block of kMlpF32Ku inputs ahead.  act: mlp_f32_act_bytes(NB).
constexpr int kMlpF32Nb = 8;        // candidates per pass of the re-evaluation
constexpr int kMlpF32NbWide = 32;   // candidates per pass of the FP32 path
constexpr int kMlpF32Ku = 4;
__host__ __device__ constexpr int mlp_f32_stride(int nb) { return nb + 4; }
__host__ __device__ constexpr size_t mlp_f32_act_bytes(int nb) {
  return sizeof(float) * 2 * (size_t)kMlpMaxK * (size_t)mlp_f32_stride(nb);
}

template <int NB, bool W16>
__device__ __noinline__ void mlp_eval_f32_w(const MlpDesc& M, const float* __restrict__ f32, const float* x,
                                            int x_stride, int n, float* out, float* act, const int* rows) {
  static_assert(NB % 4 == 0, "NB must be a multiple of 4");
  constexpr int S = mlp_f32_stride(NB);
  constexpr int KU = kMlpF32Ku;
  const int tid = threadIdx.x, B = blockDim.x;
  float* a0 = act;
  float* a1 = act + kMlpMaxK * S;
  for (int q = tid; q < M.d * NB; q += B) {
    const int i = q / NB, r = q - i * NB;
    a0[i * S + r] = (r < n) ? fmaf(M.span[i], x[(size_t)(rows ? rows[r] : r) * x_stride + i], M.lo[i]) : 0.f;
  }
  __syncthreads();
  float part[NB];
#pragma unroll
  for (int r = 0; r < NB; ++r) part[r] = 0.f;
  for (int l = 0; l < M.n_layers; ++l) {
    const int nin = M.in[l], nout = M.out[l];
    const bool last = (l == M.n_layers - 1);
    const float* WT = f32 + M.w32_0[l];
    const uint16_t* WT16 = reinterpret_cast<const uint16_t*>(WT);
    auto wld = [&](size_t idx) -> float {
      if constexpr (W16) return __uint_as_float((uint32_t)WT16[idx] << 16);
      else return WT[idx];
    };
    const float* bias = f32 + M.bias0[l];
    for (int o0 = 0; o0 < nout; o0 += 2 * B) {
      const int oa = o0 + tid, ob = oa + B;
      const bool va = oa < nout, vb = ob < nout;
      const int ca = va ? oa : 0, cb = vb ? ob : 0;  // clamped: every load stays in the layer
      float acc_a[NB], acc_b[NB];
      {
        const float ba = bias[ca], bb = bias[cb];
#pragma unroll
        for (int r = 0; r < NB; ++r) {
          acc_a[r] = ba;
          acc_b[r] = bb;
        }
      }
      float wa[KU], wb[KU];
#pragma unroll
      for (int u = 0; u < KU; ++u) {
        wa[u] = (u < nin) ? wld((size_t)u * nout + ca) : 0.f;
        wb[u] = (u < nin) ? wld((size_t)u * nout + cb) : 0.f;
      }
      for (int i0 = 0; i0 < nin; i0 += KU) {
        float na[KU], nb[KU];
#pragma unroll
        for (int u = 0; u < KU; ++u) {
          const int i = i0 + KU + u;
          na[u] = (i < nin) ? wld((size_t)i * nout + ca) : 0.f;
          nb[u] = (i < nin) ? wld((size_t)i * nout + cb) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < KU; ++u) {
          if (i0 + u < nin) {
            const float4* ar = reinterpret_cast<const float4*>(a0 + (i0 + u) * S);
#pragma unroll
            for (int q = 0; q < NB / 4; ++q) {
              const float4 v = ar[q];
              acc_a[4 * q + 0] = fmaf(wa[u], v.x, acc_a[4 * q + 0]);
              acc_a[4 * q + 1] = fmaf(wa[u], v.y, acc_a[4 * q + 1]);
              acc_a[4 * q + 2] = fmaf(wa[u], v.z, acc_a[4 * q + 2]);
              acc_a[4 * q + 3] = fmaf(wa[u], v.w, acc_a[4 * q + 3]);
              acc_b[4 * q + 0] = fmaf(wb[u], v.x, acc_b[4 * q + 0]);
              acc_b[4 * q + 1] = fmaf(wb[u], v.y, acc_b[4 * q + 1]);
              acc_b[4 * q + 2] = fmaf(wb[u], v.z, acc_b[4 * q + 2]);
              acc_b[4 * q + 3] = fmaf(wb[u], v.w, acc_b[4 * q + 3]);
            }
          }
        }
#pragma unroll
        for (int u = 0; u < KU; ++u) {
          wa[u] = na[u];
          wb[u] = nb[u];
        }
      }
      if (!last) {  // 16-byte stores: four candidates of one feature each
        if (va) {
#pragma unroll
          for (int r = 0; r < NB; r += 4)
            *reinterpret_cast<float4*>(a1 + oa * S + r) =
                make_float4(silu(acc_a[r]), silu(acc_a[r + 1]), silu(acc_a[r + 2]), silu(acc_a[r + 3]));
        }
        if (vb) {
#pragma unroll
          for (int r = 0; r < NB; r += 4)
            *reinterpret_cast<float4*>(a1 + ob * S + r) =
                make_float4(silu(acc_b[r]), silu(acc_b[r + 1]), silu(acc_b[r + 2]), silu(acc_b[r + 3]));
        }
      } else {
        if (va) {
          const float dk = f32[M.data0 + oa], is = f32[M.isig0 + oa];
#pragma unroll
          for (int r = 0; r < NB; ++r) {
            const float rr = (acc_a[r] - dk) * is;
            part[r] = fmaf(rr, rr, part[r]);
          }
        }
        if (vb) {
          const float dk = f32[M.data0 + ob], is = f32[M.isig0 + ob];
#pragma unroll
          for (int r = 0; r < NB; ++r) {
            const float rr = (acc_b[r] - dk) * is;
            part[r] = fmaf(rr, rr, part[r]);
          }
        }
      }
    }
    __syncthreads();
    if (!last) {
      float* tmp = a0;
      a0 = a1;
      a1 = tmp;
    }
  }
  // chi^2: block sum of part[r] per candidate in a fixed order (warp
  // partials staged in the free activation buffer)
  float* red = a1;  // [NB][32]
  const int lane = tid & 31, wid = tid >> 5, nw = B >> 5;
#pragma unroll
  for (int r = 0; r < NB; ++r) {
    float s = part[r];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(kFull, s, o);
    if (lane == 0) red[r * 32 + wid] = s;
  }
  __syncthreads();
  for (int r = tid; r < n; r += B) {
    float s = 0.f;
    for (int w = 0; w < nw; ++w) s += red[r * 32 + w];
    out[rows ? rows[r] : r] = -0.5f * s;
  }
  __syncthreads();
}

// The FP32 evaluator for the image's weight storage.  With `rows`
// non-null, candidate r is row rows[r] of x and its log L goes to
// out[rows[r]].
template <int NB>
__device__ __forceinline__ void mlp_eval_f32(const MlpDesc& M, const float* __restrict__ f32, const float* x,
                                             int x_stride, int n, float* out, float* act,
                                             const int* rows = nullptr) {
  if (M.w_bf16) mlp_eval_f32_w<NB, true>(M, f32, x, x_stride, n, out, act, rows);
  else mlp_eval_f32_w<NB, false>(M, f32, x, x_stride, n, out, act, rows);
}

}  // namespace nsd
