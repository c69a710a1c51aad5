// The batched-filter kernels for binary64 state, and their launchers.
#include "batch_kernels.cuh"

namespace pfk {

template cudaError_t batch_cycle_launch<double>(int, int, int, unsigned, const BatchArgs<double>&,
                                            cudaStream_t);
template unsigned batch_cycle_resident<double>(int, int, int, int);
template cudaError_t batch_init_launch<double>(unsigned, const BatchArgs<double>&, cudaStream_t);
template cudaError_t batch_prepare<double>();
template cudaError_t batch_estimate_launch<double>(unsigned, const BatchArgs<double>&, cudaStream_t);

}  // namespace pfk
