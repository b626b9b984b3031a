// The shared-bin FP32 sweep for groups of 4 walkers (sweep_shared.cuh).
#include "sweep_shared.cuh"

namespace sail {

cudaError_t launch_sweep_shared4(const DevProblem &P, const DevState &S, int n0, int n1, cudaStream_t st) {
    return P.hastings ? launch_shared_w<4, kHastings>(P, S, n0, n1, st) : launch_shared_w<4, kPlain>(P, S, n0, n1, st);
}

}  // namespace sail
