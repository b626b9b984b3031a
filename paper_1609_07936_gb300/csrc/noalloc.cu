// sail_residue_noalloc: the residue chi2 of given spectra, computed without any device
// memory from the caller beyond its inputs and outputs.
//
// Every other entry point of this library works inside a workspace the caller allocates.
// Some callers cannot allocate device memory for it: a plug-in loaded into a host program
// whose allocator owns the whole device memory budget, or a service loop that must not pay
// for cudaMalloc / cudaFree (cudaFree waits for the whole device).  For them this entry
// point keeps its only scratch, the weighted kernel table and data, in the fixed array
// below, which each GPU that loads the library holds until the process exits.
//
// Compiled with -fmad=false like the other FP64 kernels: the residual sums run over j
// ascending and chi2 over i ascending, so the result equals the residual recomputation of
// a handle up to the last bits of the device exp in the kernel table.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <mutex>

#include "../../include/sail.h"
#include "sail_internal.cuh"

namespace sail {

// Scratch: the FP64 kernel table [n_omega][n_tau_pad] followed by Fhat [n_tau_pad].
constexpr size_t kNoAllocTable = size_t(1) << 20;  // doubles: n_omega * n_tau_pad <= 1,048,576
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocTable + kMaxTau];

namespace {

constexpr double kPi = 3.14159265358979323846;

// K_ij / sigma_i of Eq. (correlation-model) for all (j, i < n_tau_pad), zero past n_tau.
__global__ void noalloc_table_kernel(double *scratch, const double *tau, const double *F, const double *sigma,
                                     int n_tau, const double *omega, int n_omega, int pad) {
    const double dw = (omega[n_omega - 1] - omega[0]) / (double)(n_omega - 1);
    double *K = scratch;
    double *Fh = scratch + (size_t)n_omega * pad;
    const size_t total = (size_t)n_omega * pad;
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x) {
        const int j = (int)(q / pad), i = (int)(q % pad);
        double v = 0.0;
        if (i < n_tau) {
            double Kij;
            if (tau[i] == 0.0) Kij = dw / (2.0 * kPi);
            else Kij = exp(-(double)j * dw * tau[i]) * (-expm1(-dw * tau[i])) / (2.0 * kPi * tau[i]);
            v = Kij / sigma[i];
        }
        K[q] = v;
        if (j == 0) Fh[i] = i < n_tau ? F[i] / sigma[i] : 0.0;
    }
}

// One block per spectrum: R_i = Fhat_i - sum_j Khat_ij a_j, chi2 = sum_i R_i^2.
__global__ void __launch_bounds__(128) noalloc_residue_kernel(const double *scratch, int n_tau, int n_omega, int pad,
                                                              const double *a, double *chi2, double *R) {
    __shared__ double Rs[kMaxTau];
    const int w = blockIdx.x;
    const double *K = scratch;
    const double *Fh = scratch + (size_t)n_omega * pad;
    const double *aw = a + (size_t)w * n_omega;
    for (int i = threadIdx.x; i < n_tau; i += blockDim.x) {
        double model = 0.0;
        for (int j = 0; j < n_omega; ++j) model = model + K[(size_t)j * pad + i] * aw[j];
        const double r = Fh[i] - model;
        Rs[i] = r;
        if (R) R[(size_t)w * n_tau + i] = r;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double c2 = 0.0;
        for (int i = 0; i < n_tau; ++i) c2 = c2 + Rs[i] * Rs[i];
        chi2[w] = c2;
    }
}

std::mutex g_mu;
constexpr int kMaxDevices = 64;
void *g_scratch_addr[kMaxDevices];  // device address of the scratch array, per device

}  // namespace

}  // namespace sail

using namespace sail;

extern "C" int sail_residue_noalloc(const double *d_tau, const double *d_F, const double *d_sigma, int n_tau,
                                    const double *d_omega, int n_omega, const double *d_a, int n_spectra,
                                    double *d_chi2, double *d_R, void *stream) {
    if (!d_tau || !d_F || !d_sigma || !d_omega || !d_a || !d_chi2)
        return set_error(SAIL_EINVAL, "sail_residue_noalloc: NULL array argument");
    if (n_tau < 1 || n_tau > kMaxTau || n_omega < 2 || n_spectra < 0)
        return set_error(SAIL_EINVAL, "sail_residue_noalloc: needs 1 <= n_tau <= 512, n_omega >= 2, n_spectra >= 0");
    const int pad = (n_tau + 31) / 32 * 32;
    if ((size_t)n_omega * (size_t)pad > kNoAllocTable)
        return set_error(SAIL_EINVAL, "sail_residue_noalloc: n_omega * (n_tau rounded up to 32) = %zu exceeds the "
                                      "fixed scratch of %zu table entries",
                         (size_t)n_omega * (size_t)pad, kNoAllocTable);
    if (n_spectra == 0) return SAIL_OK;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return set_error(SAIL_ECUDA, "sail_residue_noalloc: no current CUDA device");
    void *scratch = nullptr;
    {
        // First call on a device: look up the array's device address with that device current.
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_scratch_addr[dev]) {
            const cudaError_t e = cudaGetSymbolAddress(&g_scratch_addr[dev], g_noalloc_scratch);
            if (e != cudaSuccess) {
                g_scratch_addr[dev] = nullptr;
                return set_error(SAIL_ECUDA, "sail_residue_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
            }
        }
        scratch = g_scratch_addr[dev];
    }
    cudaStream_t st = (cudaStream_t)stream;
    const size_t total = (size_t)n_omega * pad;
    const int blocks = (int)std::min<size_t>((total + 255) / 256, 4096);
    noalloc_table_kernel<<<blocks, 256, 0, st>>>((double *)scratch, d_tau, d_F, d_sigma, n_tau, d_omega, n_omega,
                                                  pad);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(SAIL_ECUDA, "sail_residue_noalloc: %s", cudaGetErrorString(e));
    noalloc_residue_kernel<<<n_spectra, 128, 0, st>>>((const double *)scratch, n_tau, n_omega, pad, d_a, d_chi2,
                                                      d_R);
    e = cudaGetLastError();
    if (e != cudaSuccess) return set_error(SAIL_ECUDA, "sail_residue_noalloc: %s", cudaGetErrorString(e));
    return SAIL_OK;
}
