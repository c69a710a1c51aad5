// The batched-filter kernels for binary32 state, and their launchers.
#include "batch_kernels.cuh"

namespace pfk {

template cudaError_t batch_cycle_launch<float>(int, int, int, unsigned, const BatchArgs<float>&,
                                            cudaStream_t);
template unsigned batch_cycle_resident<float>(int, int, int, int);
template cudaError_t batch_init_launch<float>(unsigned, const BatchArgs<float>&, cudaStream_t);
template cudaError_t batch_prepare<float>();
template cudaError_t batch_estimate_launch<float>(unsigned, const BatchArgs<float>&, cudaStream_t);

}  // namespace pfk
