// Device helpers of the Metropolis move shared by the FP64 and FP32 sweeps.
#pragma once
#include <cmath>

namespace sail {

// Eq. (amplitude-acceptance-adjustment): y = 1 if the acceptance a >= p, else (a/p)^m, with a
// the fraction of moves the walker accepted in its previous sweep and a floor y_min.  An
// integer m is applied by repeated multiplication.  Evaluated once per walker and sweep.
__device__ __forceinline__ double amplitude(int accepted_prev, int n_omega, double y_p, double y_m,
                                            double y_min) {
    const double acc = (double)accepted_prev / (double)n_omega;
    double y;
    if (acc >= y_p) {
        y = 1.0;
    } else {
        const double q = acc / y_p;
        if (y_m == floor(y_m) && y_m >= 1.0 && y_m <= 16.0) {
            y = q;
            for (int k = 1; k < (int)y_m; ++k) y = y * q;
        } else {
            y = pow(q, y_m);
        }
    }
    return y < y_min ? y_min : y;
}

}  // namespace sail
