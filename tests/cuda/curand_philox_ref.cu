// Test-only: runs the Philox4x32-10 of the cuRAND device header over a list of counters,
// an implementation independent of both the oracle and libsail.
#include <cstdint>
#include <curand_kernel.h>

__global__ void ref_kernel(int n, const uint32_t *ctr, uint64_t seed, uint32_t *out) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const uint4 c = make_uint4(ctr[4 * q], ctr[4 * q + 1], ctr[4 * q + 2], ctr[4 * q + 3]);
    const uint4 r = curand_Philox4x32_10(c, make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
    out[4 * q] = r.x;
    out[4 * q + 1] = r.y;
    out[4 * q + 2] = r.z;
    out[4 * q + 3] = r.w;
}

extern "C" int curand_philox_ref(int n, const uint32_t *d_ctr, uint64_t seed, uint32_t *d_out) {
    if (n <= 0) return 0;
    ref_kernel<<<(n + 255) / 256, 256>>>(n, d_ctr, seed, d_out);
    if (cudaGetLastError() != cudaSuccess) return -1;
    return cudaDeviceSynchronize() == cudaSuccess ? 0 : -1;
}
