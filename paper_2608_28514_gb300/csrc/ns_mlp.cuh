// ns_mlp.cuh -- the emulator-style likelihood of the benchmark suite:
// log L = -1/2 sum_k ((MLP(theta)_k - data_k) / sigma_k)^2 with a SiLU MLP
// (the stand-in for the neural-network emulator of section 5).
//
// Two evaluators of a batch of candidate points:
//  * BF16 on the 5th-generation tensor cores (tcgen05): per layer, the
//    weights W [out][in] are the A operand (M = 128 output features per
//    tile, K-major), the batch of candidates the B operand (N = kMlpNb
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
constexpr int kMlpNb = 64;        // candidates per block (the MMA's N)
constexpr int kMlpStages = 6;     // weight tiles in flight
constexpr int kMlpTileBytes = 128 * 128;  // 128 rows x 64 BF16 (128 bytes)
constexpr int kMlpMaxK = 512;     // widest padded layer input
constexpr unsigned kMlpWaitCap = 1u << 22;

// Offsets into the packed image (host-built, device-resident):
//   tiles  : BF16 swizzled weight tiles, layer by layer, M-tile by M-tile,
//            K-block by K-block (16 KB each);
//   f32    : per layer bias (padded out), then data and 1/sigma of the last
//            layer (padded out), then FP32 weights [out][in] row-major.
struct MlpDesc {
  int n_layers, d;
  int in[kMlpMaxLayers], out[kMlpMaxLayers];        // true widths
  int kpad[kMlpMaxLayers], mpad[kMlpMaxLayers];      // in padded to 64, out padded to 128
  int tile0[kMlpMaxLayers];                          // index of the layer's first tile
  long long bias0[kMlpMaxLayers];                    // float offset of the layer's bias
  long long w32_0[kMlpMaxLayers];                    // float offset of the layer's FP32 weights
  long long data0, isig0;                            // float offsets (last layer, padded)
  int n_tiles;
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

// Shared memory of the BF16 evaluator (offsets from a 1024-aligned base).
struct MlpSmem {
  static constexpr int kStageOff = 0;
  static constexpr int kActOff = kStageOff + kMlpStages * kMlpTileBytes;      // [kpad/64][kMlpNb][128 B]
  static constexpr int kActBytes = (kMlpMaxK / 64) * kMlpNb * 128;
  static constexpr int kChiOff = kActOff + kActBytes;                         // [4][kMlpNb] floats
  static constexpr int kBarOff = kChiOff + 4 * kMlpNb * 4;                    // mbarriers
  static constexpr int kMiscOff = kBarOff + 8 * (2 * kMlpStages + 2);
  static constexpr int kBytes = kMiscOff + 64;
};

// Tensor memory of the BF16 evaluator: 512 columns, allocated once per block
// (allocating again after the permit is relinquished is not allowed) and
// freed once before the block exits.  Called by every thread; returns the
// base address.
inline __device__ unsigned mlp_tmem_alloc(unsigned* slot) {
  if ((threadIdx.x >> 5) == 0) tmem_alloc(slot, 512);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  return *slot;
}
inline __device__ void mlp_tmem_free(unsigned tmem) {
  tc_fence_before();
  __syncthreads();
  if ((threadIdx.x >> 5) == 0) tmem_dealloc(tmem, 512);
  __syncthreads();
}

// 1024-byte aligned start (in the shared window) of a region beginning at p.
__device__ __forceinline__ char* align1024_shared(char* p) {
  const unsigned a = smem_u32(p);
  return p + ((1024u - (a & 1023u)) & 1023u);
}

// Evaluates the batch x [n][d] (unit cube, n <= kMlpNb) with the BF16
// tensor-core path into out[n] (log L), using the block's tensor memory
// `tmem` (mlp_tmem_alloc).  Must be called by every thread of the block (at
// least 128 threads: warps 0-3 read the accumulators back).  `sm` is 1024-byte aligned and holds
// MlpSmem::kBytes.  Returns false (for every thread) on a wait timeout.
inline __device__ bool mlp_eval_bf16(const MlpDesc& M, const uint8_t* __restrict__ tiles,
                                     const float* __restrict__ f32, const float* x, int x_stride, int n,
                                     float* out, char* sm, unsigned tmem) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  char* stages = sm + MlpSmem::kStageOff;
  char* act = sm + MlpSmem::kActOff;
  float* chi = reinterpret_cast<float*>(sm + MlpSmem::kChiOff);
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + MlpSmem::kBarOff);
  uint64_t* empty = full + kMlpStages;
  uint64_t* done = empty + kMlpStages;
  unsigned* misc = reinterpret_cast<unsigned*>(sm + MlpSmem::kMiscOff);  // [1] error flag
  const unsigned NB = kMlpNb;
  const unsigned idesc = idesc_bf16(128, kMlpNb);

  if (tid == 0) {
    for (int s = 0; s < kMlpStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(done, 1);
    mbar_fence_init();
    misc[1] = 0u;
  }
  // layer-0 input: theta = lo + span x in BF16, rows = candidates, K = d (pad 0)
  const int kb0 = M.kpad[0] / 64;
  for (int q = tid; q < kb0 * kMlpNb * 64; q += blockDim.x) {
    const int kb = q / (kMlpNb * 64), rem = q % (kMlpNb * 64), r = rem / 64, k = rem % 64;
    const int i = kb * 64 + k;
    float v = 0.f;
    if (r < n && i < M.d) v = fmaf(M.span[i], x[(size_t)r * x_stride + i], M.lo[i]);
    *reinterpret_cast<__nv_bfloat16*>(act + kb * kMlpNb * 128 + sw128_offset(r, k)) = __float2bfloat16_rn(v);
  }
  for (int q = tid; q < 4 * kMlpNb; q += blockDim.x) chi[q] = 0.f;
  fence_proxy_async();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();

  unsigned item = 0;      // weight tiles consumed so far (stage ring position)
  unsigned done_phase = 0;
  bool ok = true;
  for (int l = 0; l < M.n_layers && ok; ++l) {
    const int KB = M.kpad[l] / 64, MT = M.mpad[l] / 128;
    const bool last = (l == M.n_layers - 1);
    const int group = 512 / kMlpNb;  // M-tiles whose accumulators fit in tensor memory at once
    for (int g0 = 0; g0 < MT && ok; g0 += group) {
      const int g1 = min(MT, g0 + group);
      const int n_items = (g1 - g0) * KB;
      if (tid == 0) {
        // one thread streams the weight tiles (TMA bulk copies, kMlpStages in
        // flight) and issues the MMAs; a stage is refilled once the MMAs of
        // the tile before the current one have completed, so the tensor pipe
        // always has queued work
        const uint8_t* src0 = tiles + (size_t)(M.tile0[l] + g0 * KB) * kMlpTileBytes;
        int issued = 0, consumed = 0;
        bool err = false;
        for (; issued < n_items && issued < kMlpStages; ++issued) {
          const unsigned it = item + issued, s = it % kMlpStages;
          if (it >= kMlpStages && !mbar_wait(&empty[s], ((it / kMlpStages) - 1) & 1)) {
            err = true;
            break;
          }
          mbar_expect_tx(&full[s], kMlpTileBytes);
          bulk_g2s(stages + s * kMlpTileBytes, src0 + (size_t)issued * kMlpTileBytes, kMlpTileBytes, &full[s]);
        }
        for (int i = 0; i < n_items && !err; ++i) {
          const unsigned it = item + i, s = it % kMlpStages;
          if (!mbar_wait(&full[s], (it / kMlpStages) & 1)) {
            err = true;
            break;
          }
          consumed = i + 1;
          tc_fence_after();
          const int t = g0 + i / KB, kb = i % KB;
          const unsigned d_tmem = tmem + (unsigned)((t - g0) * kMlpNb);
          const unsigned a0 = smem_u32(stages + s * kMlpTileBytes);
          const unsigned b0 = smem_u32(act + kb * kMlpNb * 128);
#pragma unroll
          for (int k = 0; k < 4; ++k)
            umma_bf16(d_tmem, sdesc_sw128(a0 + 32 * k), sdesc_sw128(b0 + 32 * k), idesc,
                      (kb > 0 || k > 0) ? 1u : 0u);
          umma_commit(&empty[s]);
          const int j = i - 1 + kMlpStages;  // next tile, into the stage of tile i-1
          if (i >= 1 && j < n_items && j >= issued) {
            const unsigned itj = item + j, sj = itj % kMlpStages;
            if (!mbar_wait(&empty[sj], ((itj / kMlpStages) - 1) & 1)) {
              err = true;
              break;
            }
            mbar_expect_tx(&full[sj], kMlpTileBytes);
            bulk_g2s(stages + sj * kMlpTileBytes, src0 + (size_t)j * kMlpTileBytes, kMlpTileBytes, &full[sj]);
            issued = j + 1;
          }
        }
        umma_commit(done);
        if (err) {
          // drain: every copy this thread issued lands before the block moves on
          for (int i = consumed; i < issued; ++i) {
            const unsigned it = item + i;
            mbar_wait(&full[it % kMlpStages], (it / kMlpStages) & 1);
          }
          misc[1] = 1u;
        }
      }
      item += n_items;
      __syncthreads();
      if (misc[1] != 0u) {
        ok = false;
        break;
      }
      // all threads wait for the group's MMAs
      if (!mbar_wait(done, done_phase)) {
        misc[1] = 1u;
      }
      done_phase ^= 1u;
      __syncthreads();
      if (misc[1] != 0u) {
        ok = false;
        break;
      }
      tc_fence_after();
      // epilogue: warp w reads lanes 32w..32w+31 (output features) of each M-tile
      for (int t = g0; t < g1 && warp < 4; ++t) {
        const int f = t * 128 + warp * 32 + lane;
        for (int c0 = 0; c0 < kMlpNb; c0 += 16) {
          float v[16];
          tmem_ld16(tmem + ((unsigned)(warp * 32) << 16) + (unsigned)((t - g0) * kMlpNb + c0), v);
          if (!last) {
            const float bias = f32[M.bias0[l] + f];
            const int kb = f / 64, k = f % 64;
            char* dst = act + kb * kMlpNb * 128;
#pragma unroll
            for (int c = 0; c < 16; ++c) {
              const float h = silu(v[c] + bias);
              *reinterpret_cast<__nv_bfloat16*>(dst + sw128_offset(c0 + c, k)) = __float2bfloat16_rn(h);
            }
          } else {
            const float bias = f32[M.bias0[l] + f];
            const float dk = f32[M.data0 + f], is = f32[M.isig0 + f];
            float r2[16];
#pragma unroll
            for (int c = 0; c < 16; ++c) {
              const float r = (v[c] + bias - dk) * is;
              r2[c] = r * r;
            }
            // sum over the warp's 32 features for each of the 16 columns
#pragma unroll
            for (int c = 0; c < 16; ++c) {
              float s = r2[c];
#pragma unroll
              for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
              r2[c] = s;
            }
            if (lane < 16) {
              float s = r2[0];
#pragma unroll
              for (int c = 1; c < 16; ++c)
                if (lane == c) s = r2[c];
              chi[warp * kMlpNb + c0 + lane] += s;
            }
          }
        }
      }
      // the next layer's MMAs read the new activations: make them visible
      fence_proxy_async();
      tc_fence_before();
      __syncthreads();
      tc_fence_after();
    }
  }
  if (ok) {
    for (int r = tid; r < n; r += blockDim.x)
      out[r] = -0.5f * (chi[r] + chi[kMlpNb + r] + chi[2 * kMlpNb + r] + chi[3 * kMlpNb + r]);
  }
  tc_fence_before();
  __syncthreads();
  return ok;
}

// FP32 CUDA-core evaluator: the same function in FP32 (weights = the FP32
// masters).  Each block evaluates up to kMlpF32Nb candidates; act: shared
// FP32 [2][kMlpF32Nb][kMlpMaxK].
constexpr int kMlpF32Nb = 8;
inline __device__ void mlp_eval_f32(const MlpDesc& M, const float* __restrict__ f32, const float* x, int x_stride,
                                    int n, float* out, float* act) {
  const int tid = threadIdx.x, B = blockDim.x;
  float* a0 = act;
  float* a1 = act + kMlpF32Nb * kMlpMaxK;
  for (int q = tid; q < kMlpF32Nb * kMlpMaxK; q += B) {
    const int r = q / kMlpMaxK, i = q % kMlpMaxK;
    a0[q] = (r < n && i < M.d) ? fmaf(M.span[i], x[(size_t)r * x_stride + i], M.lo[i]) : 0.f;
  }
  __syncthreads();
  float part[kMlpF32Nb];
#pragma unroll
  for (int r = 0; r < kMlpF32Nb; ++r) part[r] = 0.f;
  for (int l = 0; l < M.n_layers; ++l) {
    const int nin = M.in[l], nout = M.out[l];
    const bool last = (l == M.n_layers - 1);
    const float* W = f32 + M.w32_0[l];
    const float* bias = f32 + M.bias0[l];
    for (int o = tid; o < nout; o += B) {
      float acc[kMlpF32Nb];
#pragma unroll
      for (int r = 0; r < kMlpF32Nb; ++r) acc[r] = bias[o];
      const float* wr = W + (size_t)o * nin;
      for (int i = 0; i < nin; ++i) {
        const float w = wr[i];
#pragma unroll
        for (int r = 0; r < kMlpF32Nb; ++r) acc[r] = fmaf(w, a0[r * kMlpMaxK + i], acc[r]);
      }
      if (!last) {
#pragma unroll
        for (int r = 0; r < kMlpF32Nb; ++r) a1[r * kMlpMaxK + o] = silu(acc[r]);
      } else {
        const float dk = f32[M.data0 + o], is = f32[M.isig0 + o];
#pragma unroll
        for (int r = 0; r < kMlpF32Nb; ++r) {
          const float rr = (acc[r] - dk) * is;
          part[r] = fmaf(rr, rr, part[r]);
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
  // chi^2: block sum of part[r] per candidate, fixed order
  __shared__ float red[kMlpF32Nb][32];
  const int lane = tid & 31, wid = tid >> 5, nw = B >> 5;
#pragma unroll
  for (int r = 0; r < kMlpF32Nb; ++r) {
    float s = part[r];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(kFull, s, o);
    if (lane == 0) red[r][wid] = s;
  }
  __syncthreads();
  if (tid < n) {
    float s = 0.f;
    for (int w = 0; w < nw; ++w) s += red[tid][w];
    out[tid] = -0.5f * s;
  }
  __syncthreads();
}

}  // namespace nsd
