// Batched FP32 sweep for problems with 16 lanes per walker, and the dispatch of a batched
// segment to the kernel of its lane count.
#include "sweep_batch.cuh"

namespace sail {

cudaError_t launch_sweep_batch(const BatchProblem *d_probs, const BatchItem *d_items, int n_items, int *d_counter,
                               size_t smem, int warps, int lanes, cudaStream_t st) {
    if (n_items <= 0) return cudaSuccess;
    return lanes == 8 ? launch_sweep_batch8(d_probs, d_items, n_items, d_counter, smem, warps, st)
                      : launch_batch_g<16>(d_probs, d_items, n_items, d_counter, smem, warps, st);
}

}  // namespace sail
