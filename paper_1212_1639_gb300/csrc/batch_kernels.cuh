// Definitions of the launchers declared in batch_launch.h; included by the
// per-precision translation units, which instantiate them.
#pragma once
#include <cstring>

#include "batch_launch.h"

namespace pfk {

template <class R>
using BatchKernel = void (*)(BatchArgs<R>);

template <class R, int POS>
BatchKernel<R> batch_kernel_p(int nt, int cl) {
  switch (cl) {
    case 2: return k_batch_cycle<R, POS, 256, 2>;
    case 4: return k_batch_cycle<R, POS, 256, 4>;
    case 8: return k_batch_cycle<R, POS, 256, 8>;
    default: return nt == 512 ? k_batch_cycle<R, POS, 512, 1> : k_batch_cycle<R, POS, 256, 1>;
  }
}

template <class R>
BatchKernel<R> batch_kernel(int pos, int nt, int cl) {
  return pos == POS_SYSTEMATIC ? batch_kernel_p<R, POS_SYSTEMATIC>(nt, cl)
                               : batch_kernel_p<R, POS_MULTINOMIAL>(nt, cl);
}

inline void cluster_config(cudaLaunchConfig_t* cfg, cudaLaunchAttribute* attr, unsigned grid,
                           int nt, int cl, cudaStream_t s) {
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->gridDim = dim3(grid, 1, 1);
  cfg->blockDim = dim3((unsigned)nt, 1, 1);
  cfg->dynamicSmemBytes = 0;
  cfg->stream = s;
  attr->id = cudaLaunchAttributeClusterDimension;
  attr->val.clusterDim.x = (unsigned)cl;
  attr->val.clusterDim.y = 1;
  attr->val.clusterDim.z = 1;
  cfg->attrs = attr;
  cfg->numAttrs = 1;
}

template <class R>
cudaError_t batch_cycle_launch(int pos, int nt, int cl, unsigned grid, const BatchArgs<R>& a,
                               cudaStream_t s) {
  BatchKernel<R> kern = batch_kernel<R>(pos, nt, cl);
  if (cl == 1) {
    kern<<<grid, nt, 0, s>>>(a);
    return cudaGetLastError();
  }
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  cluster_config(&cfg, attr, grid, nt, cl, s);
  return cudaLaunchKernelEx(&cfg, kern, a);
}

template <class R>
unsigned batch_cycle_resident(int pos, int nt, int cl, int sms) {
  BatchKernel<R> kern = batch_kernel<R>(pos, nt, cl);
  if (cl == 1) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, nt, 0) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    return (unsigned)(per_sm * sms);
  }
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  cluster_config(&cfg, attr, (unsigned)(cl * sms), nt, cl, nullptr);
  int nclusters = 0;
  if (cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return (unsigned)(nclusters * cl);
}

template <class R>
cudaError_t batch_init_launch(unsigned grid, const BatchArgs<R>& a, cudaStream_t s) {
  k_batch_init<R><<<grid, BB, 0, s>>>(a);
  return cudaGetLastError();
}

template <class R>
cudaError_t batch_prepare() {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, k_batch_init<R>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, k_batch_estimate<R>);
  return e;
}

template <class R>
cudaError_t batch_estimate_launch(unsigned grid, const BatchArgs<R>& a, cudaStream_t s) {
  k_batch_estimate<R><<<grid, BB, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace pfk
