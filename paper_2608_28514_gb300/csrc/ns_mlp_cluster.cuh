// ns_mlp_cluster.cuh -- the tensor-core evaluator of the MLP likelihood split
// over the C CTAs (C = 2 or 4) of a thread-block cluster, so that one
// batch of candidates -- one nested-sampling run's round -- is evaluated by
// C SMs at once.
//
// CTA r of the cluster owns the 128-row output tiles t with t % C == r of
// every layer: it streams only those weight tiles (a C-th of the image, by
// its own TMA bulk copies: the slices are disjoint, nothing is multicast),
// issues their MMAs into its own tensor memory and runs their epilogues.  A
// hidden layer's epilogue writes the CTA's 128-feature slice of the next
// layer's input (two 64-wide K-blocks of the swizzled B operand) in place
// in its own shared memory and then copies it, with shared::cta ->
// shared::cluster bulk copies, into the same place of every other CTA; the
// receiving CTA's MMA warp waits on an mbarrier that counts those bytes.
// Before a CTA writes a slice into a peer, the peer has finished the MMAs
// that read the previous layer's input there (each CTA announces the end of
// a layer's MMAs with a remote mbarrier arrive on every peer).  The output
// layer's epilogue forms each CTA's partial chi^2 per candidate over its own
// tiles; the partials are gathered in CTA 0's shared memory and summed there
// in rank order.
//
// Every wait is bounded (kMlpWaitCap tries); a wait that gives up sets the
// CTA's sticky error, which CTA 0 collects.
#pragma once

#include "ns_mlp.cuh"

namespace nsd {

constexpr int kMlpClusterMax = 4;

// ---------------------------------------------------------------------------
// Cluster PTX wrappers (sm_90+)
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned cl_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;\n" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned cl_size() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;\n" : "=r"(r));
  return r;
}
// Every thread of every CTA of the cluster; release / acquire at cluster scope.
__device__ __forceinline__ void cl_sync() {
  asm volatile("barrier.cluster.arrive.release;\n" ::: "memory");
  asm volatile("barrier.cluster.wait.acquire;\n" ::: "memory");
}
// The shared::cluster address of shared::cta address `sa` in CTA `rank`.
__device__ __forceinline__ unsigned cl_map(unsigned sa, unsigned rank) {
  unsigned r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;\n" : "=r"(r) : "r"(sa), "r"(rank));
  return r;
}
__device__ __forceinline__ float cl_ld_f32(unsigned ca) {
  float v;
  asm volatile("ld.shared::cluster.f32 %0, [%1];\n" : "=f"(v) : "r"(ca) : "memory");
  return v;
}
__device__ __forceinline__ int cl_ld_s32(unsigned ca) {
  int v;
  asm volatile("ld.shared::cluster.s32 %0, [%1];\n" : "=r"(v) : "r"(ca) : "memory");
  return v;
}
__device__ __forceinline__ void cl_st_f32(unsigned ca, float v) {
  asm volatile("st.shared::cluster.f32 [%0], %1;\n" ::"r"(ca), "f"(v) : "memory");
}
__device__ __forceinline__ void cl_st_s32(unsigned ca, int v) {
  asm volatile("st.shared::cluster.s32 [%0], %1;\n" ::"r"(ca), "r"(v) : "memory");
}
// Arrive (release, cluster scope) on the mbarrier at cluster address ca.
__device__ __forceinline__ void cl_mbar_arrive(unsigned ca) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];\n" ::"r"(ca) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait_cl(uint64_t* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n.reg .pred p;\n"
      "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
      "selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait with cluster-scope acquire: false if the phase did not flip.
__device__ __forceinline__ bool mbar_wait_cl(uint64_t* bar, unsigned parity) {
  for (unsigned i = 0; i < kMlpWaitCap; ++i)
    if (mbar_try_wait_cl(bar, parity)) return true;
  return false;
}
// Bulk copy of `bytes` (multiple of 16) from this CTA's shared memory to
// cluster address dst_ca; completes `bytes` of transactions on the
// mbarrier at cluster address mbar_ca (in the destination CTA).
__device__ __forceinline__ void bulk_s2cl(unsigned dst_ca, const void* src, unsigned bytes, unsigned mbar_ca) {
  asm volatile(
      "cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst_ca),
      "r"(smem_u32(src)), "r"(bytes), "r"(mbar_ca)
      : "memory");
}

// CTA 0's mailbox (static shared memory at the same address in every CTA of
// the cluster): the command of the next evaluation (kind and batch size; the
// run kernel's followers read it), each CTA's error flag and partial chi^2
// per candidate.
struct ClusterMail {
  int op, n;
  int err[kMlpClusterMax];
  float chi[kMlpClusterMax][kMlpNbMax];
};
enum { kClOpExit = 0, kClOpBf16 = 1, kClOpX2 = 2, kClOpFp32 = 3 };  // the op is the planes of the pass

// Where the candidates' unit-cube coordinates come from: global memory (g:
// every CTA builds the layer-0 operand itself), or rows of CTA 0's shared
// memory (s, through the index list rows when not null; valid in CTA 0
// only): CTA 0 builds the layer-0 operand and copies it into the other CTAs.
struct XIn {
  const float* g;
  const float* s;
  const int* rows;
  int stride;
};

// The MLP's tile rows divide among C CTAs: every layer's 128-row tile count
// is a multiple of C.
__host__ __device__ inline bool mlp_cluster_fits(const MlpDesc& M, int C) {
  if (C < 1 || C > kMlpClusterMax) return false;
  for (int l = 0; l < M.n_layers; ++l)
    if ((M.mpad[l] / 128) % C != 0) return false;
  return true;
}

// One CTA's share of the evaluation of n (1 <= n <= NBMAX) candidates by a
// cluster of C CTAs (this CTA is `rank`).  Called by every thread of a block
// of at least kMlpThreads threads, with the block's context (mlp_ctx_init;
// its act_ready / peer_free barriers) and `sm` as for mlp_eval_bf16.  On
// return (before any cluster barrier), this CTA's partial chi^2 of candidate
// r is in CTA 0's mail->chi[rank][r] and its error flag in mail->err[rank];
// the caller synchronises the cluster and CTA 0 sums the partials.  P = 3
// is the FP32-accurate three-plane variant.  Returns false if a wait gave
// up (now or before).
template <int NBMAX, int STAGES, int P = 1>
inline __device__ bool mlp_eval_bf16_cl(const MlpDesc& M, const uint8_t* __restrict__ tiles,
                                        const float* __restrict__ f32, const XIn& X, int n, char* sm, MlpCtx* ctx,
                                        ClusterMail* mail, unsigned C, unsigned rank) {
  using L = MlpSmem<NBMAX, STAGES, P>;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  char* stages = sm + L::kStageOff;
  char* act = sm + L::kActOff;
  float* chi = reinterpret_cast<float*>(sm + L::kChiOff);
  constexpr unsigned S = STAGES;
  const int N = (n + 15) & ~15;
  const unsigned item0 = ctx->item, use0 = ctx->uses[0], use1 = ctx->uses[1], xu0 = ctx->xu, pu0 = ctx->pu;
  const unsigned tmem = ctx->tmem;
  const int last = M.n_layers - 1;
  const bool failed = ctx_err(ctx) != 0u;  // uniform: nothing writes it between calls
  const int kb0 = M.kpad[0] / 64;
  // layer-0 operand copied in from CTA 0 (its bytes complete an act_ready phase here)
  const bool recv0 = (X.g == nullptr) && rank > 0;
  const unsigned bytes0 = (unsigned)kb0 * (unsigned)P * (unsigned)N * 128u;

  if (!failed && !recv0) {
    // layer-0 input: theta = lo + span x in BF16, rows = candidates, K = d (pad 0)
    for (int q = tid; q < kb0 * N * 64; q += blockDim.x) {
      const int kb = q / (N * 64), rem = q % (N * 64), r = rem / 64, k = rem % 64;
      const int i = kb * 64 + k;
      float v = 0.f;
      if (r < n && i < M.d) {
        const float xv = X.g ? X.g[(size_t)r * X.stride + i] : X.s[(size_t)(X.rows ? X.rows[r] : r) * X.stride + i];
        v = fmaf(M.span[i], xv, M.lo[i]);
      }
      char* dst = act + kb * NBMAX * 128 + sw128_offset(r, k);
      store_planes<P>(dst, L::kPlaneBytes, v);
    }
    fence_proxy_async();
  }
  if (!failed) {
    for (int q = tid; q < 4 * NBMAX; q += blockDim.x) chi[q] = 0.f;
    if (tid == 0 && recv0) {
      mbar_expect_tx(&ctx->act_ready, bytes0);
      ctx->xu_armed = xu0 + 1u;
    }
  }
  __syncthreads();
  if (!failed && X.g == nullptr && rank == 0 && tid == 0) {
    // the layer-0 operand into every other CTA (the previous pass's reads of
    // those K-blocks ended before the cluster barrier that opened this one)
    const unsigned rdy = smem_u32(&ctx->act_ready);
    for (int kb = 0; kb < kb0; ++kb)
      for (int pl = 0; pl < P; ++pl) {
        const char* src = act + pl * L::kPlaneBytes + kb * NBMAX * 128;
        for (unsigned p = 1; p < C; ++p) bulk_s2cl(cl_map(smem_u32(src), p), src, (unsigned)N * 128u, cl_map(rdy, p));
      }
  }

  if (failed) {
    // nothing to do; the peers' waits on this CTA give up and report
  } else if (warp == kMlpProducerWarp) {
    // this CTA's weight tiles, in consumption order (layer, own M-tile, K-block)
    if (lane == 0) {
      unsigned it = item0;
      bool err = false;
      for (int l = 0; l <= last && !err; ++l) {
        const int KB = M.kpad[l] / 64, MT = M.mpad[l] / 128;
        for (int t = (int)rank; t < MT && !err; t += (int)C)
          for (int kb = 0; kb < KB; ++kb, ++it) {
            const unsigned s = it % S;
            if (ctx_err(ctx) || (it >= S && !mbar_wait(&ctx->empty[s], ((it / S) - 1) & 1))) {
              err = true;
              break;
            }
            mbar_expect_tx(&ctx->full[s], kMlpTileBytes);
            bulk_g2s(stages + s * kMlpTileBytes, tiles + (size_t)(M.tile0[l] + t * KB + kb) * kMlpTileBytes,
                     kMlpTileBytes, &ctx->full[s]);
          }
      }
      if (err) {
        ctx_set_err(ctx);
        for (unsigned j = (it - item0 > S) ? it - S : item0; j < it; ++j) mbar_wait(&ctx->full[j % S], (j / S) & 1);
      }
    }
    __syncwarp();
  } else if (warp == kMlpMmaWarp) {
    if (lane == 0) {
      const unsigned idesc = idesc_bf16(128, N);
      unsigned it = item0, uses[2] = {use0, use1}, xu = xu0;
      bool err = false;
      for (int l = 0; l <= last && !err; ++l) {
        const int KB = M.kpad[l] / 64, own = (M.mpad[l] / 128) / (int)C;
        const int ng = mlp_n_groups(own, l == last, N);
        for (int gi = 0; gi < ng && !err; ++gi) {
          const MlpGroup G = mlp_group(own, l == last, gi, N);
          for (int h = 0; h < 2 && !err; ++h) {
            const bool need = (gi == 0) || (h >= G.h0 && h < G.h0 + G.nh);
            if (need && uses[h] > 0 && !mbar_wait(&ctx->acc_free[h], (uses[h] - 1) & 1)) err = true;
          }
          // the layer's input slices of the other CTAs have landed (layer 0:
          // the operand CTA 0 copied in)
          if (!err && gi == 0 && (l > 0 || recv0)) {
            if (!mbar_wait_cl(&ctx->act_ready, xu & 1)) err = true;
            ++xu;
          }
          if (err || ctx_err(ctx)) {
            err = true;
            break;
          }
          tc_fence_after();
          const unsigned col0 = (unsigned)G.h0 * kMlpHalfCols;
          for (int j = G.g0; j < G.g1 && !err; ++j) {
            for (int kb = 0; kb < KB; ++kb, ++it) {
              const unsigned s = it % S;
              if (!mbar_wait(&ctx->full[s], (it / S) & 1)) {
                err = true;
                break;
              }
              tc_fence_after();
              const unsigned d_tmem = tmem + col0 + (unsigned)((j - G.g0) * N);
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
        umma_commit(&ctx->drain);
        mbar_wait(&ctx->drain, 0);
      } else {
        ctx->item = it;
        ctx->uses[0] = uses[0];
        ctx->uses[1] = uses[1];
        ctx->xu = xu;
      }
    }
    __syncwarp();
  } else if (warp < kMlpEpiWarps) {
    // Every epilogue warp passes the same named barriers whatever happens
    // (a failed wait only sets epi_err), so an error cannot leave a barrier
    // short of arrivals.  After an error this CTA stops announcing its MMAs
    // to the peers, so no peer starts a copy into it any more.
    const int q = warp & 3, ch = warp >> 2;  // lane quadrant, chunk parity
    const unsigned lane_base = (unsigned)(q * 32) << 16;
    const int n_chunks = N / 16;
    unsigned uses[2] = {use0, use1}, pu = pu0, xa = xu0 + (recv0 ? 1u : 0u);
    __shared__ int epi_err;
    if (tid == 0) epi_err = 0;
    epi_bar_sync();
    for (int l = 0; l <= last; ++l) {
      const int own = (M.mpad[l] / 128) / (int)C;
      const bool is_last = (l == last);
      const int ng = mlp_n_groups(own, is_last, N);
      for (int gi = 0; gi < ng; ++gi) {
        const MlpGroup G = mlp_group(own, is_last, gi, N);
        bool ok = true;
        for (int h = G.h0; h < G.h0 + G.nh; ++h) {
          bool okh = true;
          if (lane == 0 && ok && !*reinterpret_cast<volatile int*>(&epi_err))
            okh = mbar_wait(&ctx->acc_full[h], uses[h] & 1);
          ok = ok && __shfl_sync(kFull, okh ? 1 : 0, 0);
        }
        if (!ok && lane == 0) epi_err = 1;
        tc_fence_after();
        const unsigned col0 = (unsigned)G.h0 * kMlpHalfCols;
        if (!is_last) {
          // this CTA's MMAs of layer l are done: the peers may write the next
          // layer's input into it; wait until every peer's are done, so that
          // this CTA may overwrite its own slice (the source of its last
          // copies) and write into the peers
          epi_bar_sync();
          if (tid == 0) {
            bool fine = !*reinterpret_cast<volatile int*>(&epi_err);
            if (fine) {
              const unsigned pf = smem_u32(&ctx->peer_free);
              for (unsigned p = 1; p < C; ++p) cl_mbar_arrive(cl_map(pf, (rank + p) % C));
              fine = mbar_wait_cl(&ctx->peer_free, pu & 1);
            }
            if (!fine) epi_err = 1;
          }
          epi_bar_sync();
          if (!*reinterpret_cast<volatile int*>(&epi_err)) {
            // bias + SiLU, BF16 straight into the next layer's swizzled B operand
            for (int j = G.g0; j < G.g1; ++j) {
              const int t = (int)rank + j * (int)C;
              const int f = t * 128 + q * 32 + lane;
              const float bias = f32[M.bias0[l] + f];
              const int kb = f >> 6, k = f & 63;
              char* dst = act + kb * NBMAX * 128;
              for (int i = ch; i < n_chunks; i += 2) {
                const int c0 = i * 16;
                float v[16];
                tmem_ld16(tmem + lane_base + col0 + (unsigned)((j - G.g0) * N + c0), v);
                // BF16 path: SiLU on the special-function unit; the wider paths: accurate SiLU
#pragma unroll
                for (int c = 0; c < 16; ++c)
                  store_planes<P>(dst + sw128_offset(c0 + c, k), L::kPlaneBytes,
                                  (P == 1) ? silu_fast(v[c] + bias) : silu(v[c] + bias));
              }
            }
          }
          fence_proxy_async();
        } else if (ok) {
          // chi^2: per candidate column, one of this CTA's output tiles at a
          // time, added in tile order (batch-independent, as on one CTA)
          for (int i = ch; i < n_chunks; i += 2) {
            const int c0 = i * 16;
            for (int j = G.g0; j < G.g1; ++j) {
              const int t = (int)rank + j * (int)C;
              const int f = t * 128 + q * 32 + lane;
              const float is = f32[M.isig0 + f];
              const float bias = f32[M.bias0[l] + f], dk = f32[M.data0 + f];
              const float cb = (bias - dk) * is;
              float v[16], sacc[16];
              tmem_ld16(tmem + lane_base + col0 + (unsigned)((j - G.g0) * N + c0), v);
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
      if (!is_last) {
        // this CTA's slice of the next layer's input into every peer, and the
        // bytes this CTA expects from the peers
        epi_bar_sync();
        if (tid == 0 && !*reinterpret_cast<volatile int*>(&epi_err)) {
          const unsigned bytes = (unsigned)N * 128u;
          const unsigned rdy = smem_u32(&ctx->act_ready);
          for (int j = 0; j < own; ++j) {
            const int t = (int)rank + j * (int)C;
            for (int kb = 2 * t; kb < 2 * t + 2; ++kb)
              for (int pl = 0; pl < P; ++pl) {
                const char* src = act + pl * L::kPlaneBytes + kb * NBMAX * 128;
                for (unsigned p = 1; p < C; ++p) {
                  const unsigned dst_rank = (rank + p) % C;
                  bulk_s2cl(cl_map(smem_u32(src), dst_rank), src, bytes, cl_map(rdy, dst_rank));
                }
              }
          }
          mbar_expect_tx(&ctx->act_ready, (C - 1u) * (unsigned)own * 2u * (unsigned)P * bytes);
          ctx->xu_armed = xa + 1u;
        }
        ++pu;
        ++xa;
      }
    }
    epi_bar_sync();
    const bool bad = *reinterpret_cast<volatile int*>(&epi_err) != 0;
    if (bad && tid == 0) ctx_set_err(ctx);
    // this CTA's partial chi^2 per candidate into CTA 0's mailbox
    const unsigned mchi = smem_u32(&mail->chi[rank][0]);
    for (int r = tid; r < n; r += kMlpEpiWarps * 32)
      cl_st_f32(cl_map(mchi + 4u * (unsigned)r, 0),
                chi[r] + chi[NBMAX + r] + chi[2 * NBMAX + r] + chi[3 * NBMAX + r]);
    if (tid == 0 && !bad) ctx->pu = pu;
  }
  __syncthreads();
  const bool ok = ctx_err(ctx) == 0u;
  if (tid == 0) cl_st_s32(cl_map(smem_u32(&mail->err[rank]), 0), ok ? 0 : 1);
  return ok;
}

// CTA 0 after the cluster barrier that follows mlp_eval_bf16_cl: log L of
// candidate r = -1/2 the sum of the C partials in rank order, into
// out[rows ? rows[r] : r].  Every thread of the block; false if any CTA
// reported an error.
inline __device__ bool mlp_cl_collect(const ClusterMail* mail, unsigned C, int n, float* out, const int* rows) {
  for (int r = threadIdx.x; r < n; r += blockDim.x) {
    float s = 0.f;
    for (unsigned q = 0; q < C; ++q) s += mail->chi[q][r];
    out[rows ? rows[r] : r] = -0.5f * s;
  }
  int bad = 0;
  for (unsigned q = 0; q < C; ++q) bad |= mail->err[q];
  __syncthreads();
  return bad == 0;
}

// Before a cluster CTA leaves its last cluster barrier: after an error, wait
// (bounded) until the last layer-input exchange it armed has landed, so that
// no peer's copy is still on its way into its shared memory.  (Phases of an
// mbarrier complete in order, so at most the last one can be open.)  Every
// thread of the block.
inline __device__ void mlp_cl_drain(MlpCtx* ctx) {
  if (threadIdx.x == 0 && ctx_err(ctx) && ctx->xu_armed > ctx->xu)
    mbar_wait_cl(&ctx->act_ready, (ctx->xu_armed - 1u) & 1u);
  __syncthreads();
}

}  // namespace nsd
