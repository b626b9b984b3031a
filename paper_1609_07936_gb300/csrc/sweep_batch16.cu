// Batched FP32 sweep for problems with 16 lanes per walker, and the dispatch of a batched
// launch to the kernel of its lane count and move-loop variant.
#include "sweep_batch.cuh"

namespace sail {

int sweep_mode(const DevProblem &P) { return P.walk_len > 0 ? kWalk : (P.hastings ? kHastings : kPlain); }

cudaError_t launch_sweep_batch(const BatchProblem *d_probs, const BatchItem *d_items, int n_items, int *d_counter,
                               size_t smem, int warps, int lanes, int mode, cudaStream_t st) {
    if (n_items <= 0) return cudaSuccess;
    if (lanes == 8) return launch_sweep_batch8(d_probs, d_items, n_items, d_counter, smem, warps, mode, st);
    switch (mode) {
        case kWalk: return launch_batch_g<16, kWalk>(d_probs, d_items, n_items, d_counter, smem, warps, st);
        case kHastings: return launch_batch_g<16, kHastings>(d_probs, d_items, n_items, d_counter, smem, warps, st);
        default: return launch_batch_g<16, kPlain>(d_probs, d_items, n_items, d_counter, smem, warps, st);
    }
}

}  // namespace sail
