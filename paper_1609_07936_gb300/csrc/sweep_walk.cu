// FP32 production sweep with the index walk of Sec. 2.3 choosing a move's bins (the move loop
// of sweep_group.cuh in its kWalk variant); its own translation unit so the kernels compile in
// parallel with the others.
#include "sweep_group.cuh"

namespace sail {

cudaError_t launch_sweep_walk(const DevProblem &P, const DevState &S, int n0, int n1, cudaStream_t st) {
    return launch_sweep_w<kWalk>(P, S, n0, n1, st);
}

}  // namespace sail
