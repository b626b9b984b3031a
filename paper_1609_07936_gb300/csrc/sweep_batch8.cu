// Batched FP32 sweep for problems with 8 lanes per walker.
#include "sweep_batch.cuh"

namespace sail {

cudaError_t launch_sweep_batch8(const BatchProblem *d_probs, const BatchItem *d_items, int n_items, int *d_counter,
                                size_t smem, int warps, int mode, cudaStream_t st) {
    switch (mode) {
        case kWalk: return launch_batch_g<8, kWalk>(d_probs, d_items, n_items, d_counter, smem, warps, st);
        case kHastings: return launch_batch_g<8, kHastings>(d_probs, d_items, n_items, d_counter, smem, warps, st);
        default: return launch_batch_g<8, kPlain>(d_probs, d_items, n_items, d_counter, smem, warps, st);
    }
}

}  // namespace sail
