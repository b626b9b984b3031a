// Batched FP32 sweep: many inversions in one persistent launch per lane count and move-loop
// variant (the move loop of sweep_group.cuh; the plain loop reads each move's spectrum values
// one move ahead, since the batch's spectra stay in global memory).  A launch holds the loops of every chunk count in
// one body; the one-move-at-a-time loop (run_group) fits that body's registers without spills,
// the look-ahead loop does not, so the batch keeps the former.  sweep_batch8.cu and sweep_batch16.cu
// instantiate it for 8 and 16 lanes per walker.
#pragma once
#include "sweep_group.cuh"

namespace sail {

namespace {

template <int G, int MODE>
__device__ __forceinline__ void run_group_c(const BatchProblem &BP, int grp, const float *sm) {
    switch (BP.P.n_tau_pad / 32) {
        case 1: run_group<G, 1, false, MODE, MODE == kPlain>(BP.P, BP.S, BP.n0, BP.n1, grp, sm, nullptr, 0); break;
        case 2: run_group<G, 2, false, MODE, MODE == kPlain>(BP.P, BP.S, BP.n0, BP.n1, grp, sm, nullptr, 0); break;
        case 3: run_group<G, 3, false, MODE, MODE == kPlain>(BP.P, BP.S, BP.n0, BP.n1, grp, sm, nullptr, 0); break;
        case 4: run_group<G, 4, false, MODE, MODE == kPlain>(BP.P, BP.S, BP.n0, BP.n1, grp, sm, nullptr, 0); break;
        case 5: run_group<G, 5, false, MODE, MODE == kPlain>(BP.P, BP.S, BP.n0, BP.n1, grp, sm, nullptr, 0); break;
        case 6: run_group<G, 6, false, MODE, MODE == kPlain>(BP.P, BP.S, BP.n0, BP.n1, grp, sm, nullptr, 0); break;
        case 7: run_group<G, 7, false, MODE, MODE == kPlain>(BP.P, BP.S, BP.n0, BP.n1, grp, sm, nullptr, 0); break;
        case 8: run_group<G, 8, false, MODE, MODE == kPlain>(BP.P, BP.S, BP.n0, BP.n1, grp, sm, nullptr, 0); break;
        default:
            if constexpr (G == 16) {
                switch (BP.P.n_tau_pad / 32) {
                    case 9: run_group<16, 9, false, MODE, MODE == kPlain>(BP.P, BP.S, BP.n0, BP.n1, grp, sm, nullptr, 0); break;
                    case 10: run_group<16, 10, false, MODE, MODE == kPlain>(BP.P, BP.S, BP.n0, BP.n1, grp, sm, nullptr, 0); break;
                    case 11: run_group<16, 11, false, MODE, MODE == kPlain>(BP.P, BP.S, BP.n0, BP.n1, grp, sm, nullptr, 0); break;
                    case 12: run_group<16, 12, false, MODE, MODE == kPlain>(BP.P, BP.S, BP.n0, BP.n1, grp, sm, nullptr, 0); break;
                    case 13: run_group<16, 13, false, MODE, MODE == kPlain>(BP.P, BP.S, BP.n0, BP.n1, grp, sm, nullptr, 0); break;
                    case 14: run_group<16, 14, false, MODE, MODE == kPlain>(BP.P, BP.S, BP.n0, BP.n1, grp, sm, nullptr, 0); break;
                    case 15: run_group<16, 15, false, MODE, MODE == kPlain>(BP.P, BP.S, BP.n0, BP.n1, grp, sm, nullptr, 0); break;
                    case 16: run_group<16, 16, false, MODE, MODE == kPlain>(BP.P, BP.S, BP.n0, BP.n1, grp, sm, nullptr, 0); break;
                    default: break;
                }
            }
            break;
    }
}

// Many inversions in one persistent launch: blocks take (problem, group range) items from a
// queue, load the item's problem tables when the problem changes, and run one walker group per
// warp.  One launch serves the problems of one lane count G (its register budget differs);
// the per-walker arithmetic is that of sweep_fp32_kernel, so a walker's trajectory does not
// depend on which block, or which other problems, share the launch.
template <int G, int MODE>
__global__ void __launch_bounds__(sweep_threads<G, G == 8 ? 8 : 16>()) sweep_batch_kernel(const BatchProblem *probs,
                                                                        const BatchItem *items, int n_items,
                                                                        int *counter) {
    extern __shared__ float4 smem4[];
    float *sm = reinterpret_cast<float *>(smem4);
    __shared__ int s_item, s_loaded;
    if (threadIdx.x == 0) s_loaded = -1;
    const int warp = threadIdx.x >> 5;
    for (;;) {
        __syncthreads();                       // the previous item is finished with the tables
        if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= n_items) break;
        const BatchItem I = items[it];
        const BatchProblem &BP = probs[I.prob];
        if (I.prob != s_loaded) {
            load_tables_g<G == 8>(BP.P, sm);
            __syncthreads();
            if (threadIdx.x == 0) s_loaded = I.prob;
        }
        __syncthreads();
        const int grp = I.grp_lo + warp;
        if (grp >= I.grp_hi || BP.n0 >= BP.n1) continue;
        run_group_c<G, MODE>(BP, grp, sm);
    }
}

template <int G, int MODE>
cudaError_t launch_batch_g(const BatchProblem *d_probs, const BatchItem *d_items, int n_items, int *d_counter,
                           size_t smem, int warps, cudaStream_t st) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    constexpr int kMaxWarps = sweep_threads<G, G == 8 ? 8 : 16>() / 32;
    if (warps > kMaxWarps) warps = kMaxWarps;
    cudaError_t e = cudaFuncSetAttribute(sweep_batch_kernel<G, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(d_counter, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    // persistent: as many blocks as fit on the SMs at once
    int per_sm = 1;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sweep_batch_kernel<G, MODE>, warps * 32, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int blocks = n_items < sms * per_sm ? n_items : sms * per_sm;
    sweep_batch_kernel<G, MODE><<<blocks, warps * 32, smem, st>>>(d_probs, d_items, n_items, d_counter);
    return cudaGetLastError();
}

}  // namespace

}  // namespace sail
