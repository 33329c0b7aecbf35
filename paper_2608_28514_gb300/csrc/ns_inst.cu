// ns_inst.cu -- instantiates the per-dimension kernels for one register
// class (compiled once per class with -DNS_DMAX=<class>, so the classes
// build in parallel).
#include "ns_run.cuh"

#ifndef NS_DMAX
#error "compile with -DNS_DMAX=<register class>"
#endif

namespace nsd {

#define NS_CAT2(a, b) a##b
#define NS_CAT(a, b) NS_CAT2(a, b)

cudaError_t NS_CAT(launch_run_, NS_DMAX)(const RunDesc* runs, const int* ids, int n, int block, size_t smem,
                                         int chunk, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(k_run<NS_DMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_run<NS_DMAX><<<n, block, smem, s>>>(runs, ids, chunk);
  return cudaGetLastError();
}

cudaError_t NS_CAT(occupancy_run_, NS_DMAX)(int block, size_t smem, int* blocks_per_sm) {
  cudaError_t e = cudaFuncSetAttribute(k_run<NS_DMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_run<NS_DMAX>, block, smem);
}

cudaError_t NS_CAT(launch_loglike_, NS_DMAX)(const LikParams& P, int n, const float* x, float* out,
                                             cudaStream_t s) {
  k_loglike<NS_DMAX><<<(n + 127) / 128, 128, 0, s>>>(P, n, x, out);
  return cudaGetLastError();
}

cudaError_t NS_CAT(launch_slice_, NS_DMAX)(const LikParams& P, const SliceCfg& SC, int m, int n_pad,
                                           int correction, const float* live_x, const float* live_l,
                                           const int* seed_slot, const float* W, const float* chol, const int* cid,
                                           float* new_x, float* new_l, float* hist_l, float* hist_x, int* hist_len,
                                           long long* evals, int* flags, float* dir_scratch, int warp,
                                           cudaStream_t s) {
  if (warp) {  // four walkers (warps) per block
    k_slice_warp<NS_DMAX><<<(m + 3) / 4, 128, 0, s>>>(P, SC, m, n_pad, correction, live_x, live_l, seed_slot, W, chol,
                                                      cid, new_x, new_l, hist_l, hist_x, hist_len, evals, flags,
                                                      dir_scratch);
    return cudaGetLastError();
  }
  k_slice<NS_DMAX><<<(m + 127) / 128, 128, sizeof(float) * 128 * dir_row(NS_DMAX), s>>>(P, SC, m, n_pad, correction, live_x, live_l, seed_slot, W, chol,
                                                   cid, new_x, new_l, hist_l, hist_x, hist_len, evals, flags,
                                                   dir_scratch);
  return cudaGetLastError();
}

#if NS_DMAX == 32
// MLP runs (any d <= 32) use the widest class with the lock-step walkers.
// cluster > 1: each run is a cluster of that many CTAs (blocks r*cluster ..
// r*cluster + cluster - 1), which share its tensor-core evaluations.
cudaError_t launch_run_mlp(const RunDesc* runs, const int* ids, int n, int block, size_t smem, int chunk, int cluster,
                           cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(k_run<32, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (cluster <= 1) {
    k_run<32, true><<<n, block, smem, s>>>(runs, ids, chunk);
    return cudaGetLastError();
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(n * cluster), 1, 1);
  cfg.blockDim = dim3((unsigned)block, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_run<32, true>, runs, ids, chunk);
}
#endif

}  // namespace nsd
