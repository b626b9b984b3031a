// FP32 production sweep whose Metropolis decisions near the acceptance threshold are taken
// again from Delta chi2 in FP64 (the move loop of sweep_group.cuh in its kGuard variant); its
// own translation unit so the kernels compile in parallel with the others.
#include "sweep_group.cuh"

namespace sail {

cudaError_t launch_sweep_guard(const DevProblem &P, const DevState &S, int n0, int n1, cudaStream_t st) {
    return launch_sweep_w<kGuard>(P, S, n0, n1, st);
}

}  // namespace sail
