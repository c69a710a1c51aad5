// Launchers of the batched-filter kernels (batch.cuh).  The kernels are
// instantiated in their own translation units, one per state precision
// (batch_f32.cu, batch_f64.cu), which define these functions; the host code
// in api.cu only calls them.
#pragma once
#include <cuda_runtime.h>

#include "batch.cuh"

namespace pfk {

// The cycle kernel for resampling positions `pos`, nt threads per CTA and
// clusters of cl CTAs (1: no clusters), on `grid` CTAs.
template <class R>
cudaError_t batch_cycle_launch(int pos, int nt, int cl, unsigned grid, const BatchArgs<R>& a,
                               cudaStream_t s);

// CTAs of that kernel resident at once on `sms` SMs (clusters: the most
// clusters that fit x cl); 0 if the shape does not fit.
template <class R>
unsigned batch_cycle_resident(int pos, int nt, int cl, int sms);

template <class R>
cudaError_t batch_init_launch(unsigned grid, const BatchArgs<R>& a, cudaStream_t s);

// Load the init and summary kernels now (module loading is otherwise lazy,
// at the first launch).
template <class R>
cudaError_t batch_prepare();

template <class R>
cudaError_t batch_estimate_launch(unsigned grid, const BatchArgs<R>& a, cudaStream_t s);

}  // namespace pfk
