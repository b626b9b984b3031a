// Residual recomputation for FP32 state: R = Fhat - Khat b over all walkers, chi2 = sum R^2.
//
// A dense contraction (walkers x bins) . (bins x tau) run as a tiled FP32-FMA GEMM: a block
// owns 16 walkers and every tau point; bins are taken 32 at a time through shared memory;
// each thread accumulates its products for one chunk of bins in FP32 and adds the chunk to an
// FP64 accumulator (chunks of 16 bins when n_tau_pad > 256), so the residual carries FP32
// products with FP64 summation across the whole bin range: the rounding left in
// F/sigma ~ 1e4-1e5 minus a model of the same size stays far below 1.  chi2 is summed in
// FP64 from the FP64 residual.  Before it, for FP32 state only,
// the spectra can be put back on both sum rules (restore_kernel in exact64.cu).
// resync_fp64_kernel is the same contraction in FP64 throughout.
#include <cstdint>

#include "sail_internal.cuh"

namespace sail {

namespace {

constexpr int kWalkersPerBlock = 16;
constexpr int kTauGroups = 16;        // threads per walker

template <int TI>  // tau values per thread: n_tau_pad = 16 * TI
__global__ void __launch_bounds__(kWalkersPerBlock * kTauGroups) resync_fp32_kernel(DevProblem P, DevState S) {
    constexpr int PAD = kTauGroups * TI;
    constexpr int kChunk = TI <= 16 ? 32 : 16;   // bins per shared-memory chunk (<= 32 KB of columns)
    __shared__ float sK[kChunk][PAD];
    __shared__ float sB[kWalkersPerBlock][kChunk + 1];
    const int tid = threadIdx.x;
    const int wl = tid / kTauGroups, g = tid % kTauGroups;
    const int w0 = blockIdx.x * kWalkersPerBlock;
    const int w = w0 + wl;
    const int NO = P.n_omega;
    double acc64[TI];
    float acc32[TI];
#pragma unroll
    for (int k = 0; k < TI; ++k) acc64[k] = 0.0;
    for (int j0 = 0; j0 < NO; j0 += kChunk) {
        const int nj = min(kChunk, NO - j0);
        __syncthreads();
        // kernel columns j0..j0+nj-1, each n_tau_pad floats (zero rows past the last bin)
        for (int q = tid; q < kChunk * PAD / 4; q += blockDim.x) {
            const int jj = q / (PAD / 4), c4 = q % (PAD / 4);
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (jj < nj) v = reinterpret_cast<const float4 *>(P.Khat32 + (size_t)(j0 + jj) * PAD)[c4];
            reinterpret_cast<float4 *>(&sK[jj][0])[c4] = v;
        }
        for (int q = tid; q < kWalkersPerBlock * kChunk; q += blockDim.x) {
            const int ww = q / kChunk, jj = q % kChunk;
            const int wg = w0 + ww;
            sB[ww][jj] = (wg < P.n_walkers && jj < nj) ? S.b32[(size_t)wg * NO + j0 + jj] : 0.0f;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < TI; ++k) acc32[k] = 0.0f;
#pragma unroll 8
        for (int jj = 0; jj < kChunk; ++jj) {
            const float bv = sB[wl][jj];
#pragma unroll
            for (int k = 0; k < TI; ++k) acc32[k] = fmaf(bv, sK[jj][g + kTauGroups * k], acc32[k]);
        }
#pragma unroll
        for (int k = 0; k < TI; ++k) acc64[k] += (double)acc32[k];
    }
    double c2 = 0.0;
    if (w < P.n_walkers) {
#pragma unroll
        for (int k = 0; k < TI; ++k) {
            const int i = g + kTauGroups * k;
            const double r = i < P.n_tau ? P.Fhat64[i] - acc64[k] : 0.0;
            S.R32[(size_t)w * PAD + i] = (float)r;
            c2 += r * r;
        }
    }
    // the 16 threads of a walker are 16 consecutive lanes
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) c2 += __shfl_xor_sync(0xFFFFFFFFu, c2, o);
    if (w < P.n_walkers && g == 0) S.chi2[w] = c2;
}

// The plain FP64 recomputation of the same contraction (the comparison path for the tensor-core
// and FP32 forms): the FP32 spectra and the FP64 kernel columns multiplied and summed in FP64
// throughout.  Bins are taken 8 at a time through shared memory (8 x n_tau_pad doubles).
template <int TI>
__global__ void __launch_bounds__(kWalkersPerBlock * kTauGroups) resync_fp64_kernel(DevProblem P, DevState S) {
    constexpr int PAD = kTauGroups * TI;
    constexpr int kChunk = 8;
    __shared__ double sK[kChunk][PAD];
    __shared__ double sB[kWalkersPerBlock][kChunk + 1];
    const int tid = threadIdx.x;
    const int wl = tid / kTauGroups, g = tid % kTauGroups;
    const int w0 = blockIdx.x * kWalkersPerBlock;
    const int w = w0 + wl;
    const int NO = P.n_omega;
    double acc[TI];
#pragma unroll
    for (int k = 0; k < TI; ++k) acc[k] = 0.0;
    for (int j0 = 0; j0 < NO; j0 += kChunk) {
        const int nj = min(kChunk, NO - j0);
        __syncthreads();
        for (int q = tid; q < kChunk * PAD / 2; q += blockDim.x) {
            const int jj = q / (PAD / 2), c2 = q % (PAD / 2);
            double2 v = make_double2(0.0, 0.0);
            if (jj < nj) v = reinterpret_cast<const double2 *>(P.Khat64 + (size_t)(j0 + jj) * PAD)[c2];
            reinterpret_cast<double2 *>(&sK[jj][0])[c2] = v;
        }
        for (int q = tid; q < kWalkersPerBlock * kChunk; q += blockDim.x) {
            const int ww = q / kChunk, jj = q % kChunk;
            const int wg = w0 + ww;
            sB[ww][jj] = (wg < P.n_walkers && jj < nj) ? (double)S.b32[(size_t)wg * NO + j0 + jj] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int jj = 0; jj < kChunk; ++jj) {
            const double bv = sB[wl][jj];
#pragma unroll
            for (int k = 0; k < TI; ++k) acc[k] = fma(bv, sK[jj][g + kTauGroups * k], acc[k]);
        }
    }
    double c2 = 0.0;
    if (w < P.n_walkers) {
#pragma unroll
        for (int k = 0; k < TI; ++k) {
            const int i = g + kTauGroups * k;
            const double r = i < P.n_tau ? P.Fhat64[i] - acc[k] : 0.0;
            S.R32[(size_t)w * PAD + i] = (float)r;
            c2 += r * r;
        }
    }
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) c2 += __shfl_xor_sync(0xFFFFFFFFu, c2, o);
    if (w < P.n_walkers && g == 0) S.chi2[w] = c2;
}

template <int TI>
cudaError_t launch_ti64(const DevProblem &P, const DevState &S, cudaStream_t st) {
    const int blocks = (P.n_walkers + kWalkersPerBlock - 1) / kWalkersPerBlock;
    resync_fp64_kernel<TI><<<blocks, kWalkersPerBlock * kTauGroups, 0, st>>>(P, S);
    return cudaGetLastError();
}

template <int TI>
cudaError_t launch_ti(const DevProblem &P, const DevState &S, cudaStream_t st) {
    const int blocks = (P.n_walkers + kWalkersPerBlock - 1) / kWalkersPerBlock;
    resync_fp32_kernel<TI><<<blocks, kWalkersPerBlock * kTauGroups, 0, st>>>(P, S);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_resync_fp64(const DevProblem &P, const DevState &S, cudaStream_t st) {
    switch (P.n_tau_pad / 32) {
        case 1: return launch_ti64<2>(P, S, st);
        case 2: return launch_ti64<4>(P, S, st);
        case 3: return launch_ti64<6>(P, S, st);
        case 4: return launch_ti64<8>(P, S, st);
        case 5: return launch_ti64<10>(P, S, st);
        case 6: return launch_ti64<12>(P, S, st);
        case 7: return launch_ti64<14>(P, S, st);
        case 8: return launch_ti64<16>(P, S, st);
        case 9: return launch_ti64<18>(P, S, st);
        case 10: return launch_ti64<20>(P, S, st);
        case 11: return launch_ti64<22>(P, S, st);
        case 12: return launch_ti64<24>(P, S, st);
        case 13: return launch_ti64<26>(P, S, st);
        case 14: return launch_ti64<28>(P, S, st);
        case 15: return launch_ti64<30>(P, S, st);
        case 16: return launch_ti64<32>(P, S, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_resync_fp32(const DevProblem &P, const DevState &S, cudaStream_t st) {
    switch (P.n_tau_pad / 32) {   // n_tau_pad = 32 m, so TI = 2 m
        case 1: return launch_ti<2>(P, S, st);
        case 2: return launch_ti<4>(P, S, st);
        case 3: return launch_ti<6>(P, S, st);
        case 4: return launch_ti<8>(P, S, st);
        case 5: return launch_ti<10>(P, S, st);
        case 6: return launch_ti<12>(P, S, st);
        case 7: return launch_ti<14>(P, S, st);
        case 8: return launch_ti<16>(P, S, st);
        case 9: return launch_ti<18>(P, S, st);
        case 10: return launch_ti<20>(P, S, st);
        case 11: return launch_ti<22>(P, S, st);
        case 12: return launch_ti<24>(P, S, st);
        case 13: return launch_ti<26>(P, S, st);
        case 14: return launch_ti<28>(P, S, st);
        case 15: return launch_ti<30>(P, S, st);
        case 16: return launch_ti<32>(P, S, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace sail
