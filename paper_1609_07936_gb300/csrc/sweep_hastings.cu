// FP32 production sweep with the Metropolis-Hastings acceptance (the move loop of
// sweep_group.cuh in its kHastings variant); its own translation unit so the kernels compile
// in parallel with the others.
#include "sweep_group.cuh"

namespace sail {

cudaError_t launch_sweep_hastings(const DevProblem &P, const DevState &S, int n0, int n1, cudaStream_t st) {
    return launch_sweep_w<kHastings>(P, S, n0, n1, st);
}

}  // namespace sail
