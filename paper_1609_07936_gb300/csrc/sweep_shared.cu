// Dispatch of the shared-bin FP32 sweep by group size (sweep_shared.cuh; one translation unit
// per group size).
#include "sail_internal.cuh"

namespace sail {

cudaError_t launch_sweep_shared8(const DevProblem &P, const DevState &S, int n0, int n1, cudaStream_t st);
cudaError_t launch_sweep_shared4(const DevProblem &P, const DevState &S, int n0, int n1, cudaStream_t st);
cudaError_t launch_sweep_shared2(const DevProblem &P, const DevState &S, int n0, int n1, cudaStream_t st);

cudaError_t launch_sweep_shared(const DevProblem &P, const DevState &S, int n0, int n1, cudaStream_t st) {
    switch (P.shared_bins) {
        case 8: return launch_sweep_shared8(P, S, n0, n1, st);
        case 4: return launch_sweep_shared4(P, S, n0, n1, st);
        case 2: return launch_sweep_shared2(P, S, n0, n1, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace sail
