// FP32 production sweep (Sec. 2.2 moves, Eq. probability-density acceptance) and the
// proposal probe.
//
// One warp per walker; lane l holds R_i and M_i = Fhat_i - R_i for i = l + 32 c in
// registers.  A walker's spectrum is stored as a = g b: an accepted move multiplies the
// common scale g by r (kept as an unevaluated pair of floats, so its error stays ~1e-14
// over a whole resync interval) and writes only b_p and b_s, so a move touches two bins
// of the spectrum and two columns of the kernel table, as Sec. 2.2 notes.  Random words
// for 32 consecutive moves are drawn at once, one Philox call per lane, and broadcast by
// shuffle.  Delta chi2 = sum_i d_i (2 R_i + d_i) is reduced by an xor butterfly.  The
// scale is folded back into b when the kernel ends, so residual recomputation sees a = b.
#include <cmath>
#include <cstdint>

#include "moves.cuh"
#include "philox.cuh"
#include "sail_internal.cuh"

namespace sail {

namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// (hi, lo) <- (hi, lo) * r with the product's rounding error carried in lo.
__device__ __forceinline__ void pair_scale(float &hi, float &lo, float r) {
    const float p = hi * r;
    const float e = fmaf(hi, r, -p);
    const float l = fmaf(lo, r, e);
    const float s = p + l;
    lo = l - (s - p);
    hi = s;
}

template <int C>
__global__ void __launch_bounds__(128) sweep_fp32_kernel(DevProblem P, DevState S, int n0, int n1) {
    const int lane = threadIdx.x & 31;
    const int w = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (w >= P.n_walkers) return;
    const int NO = P.n_omega, PAD = P.n_tau_pad;
    const float *__restrict__ K = P.Khat32;
    const float *__restrict__ beta = P.beta32;
    float *b = S.b32 + (size_t)w * NO;

    float R[C], M[C];
#pragma unroll
    for (int c = 0; c < C; ++c) {
        R[c] = S.R32[(size_t)w * PAD + lane + 32 * c];
        M[c] = P.Fhat32[lane + 32 * c] - R[c];
    }
    float ghi = S.g2[2 * w], glo = S.g2[2 * w + 1];
    double chi2 = S.chi2[w];
    int accp = S.acc_prev[w];
    unsigned long long h = S.hash[w], nacc = 0, npos = 0;
    const uint2 key = philox_key(P.seed);
    const double dmove = P.move_scale > 0.0 ? P.move_scale : 1.0 / NO;
    const float dwf = (float)P.dw;

    for (int n = n0; n < n1; ++n) {
        const float invT = (float)(1.0 / P.Tsweep[n]);
        const float yd = (float)(amplitude(accp, NO, P.y_p, P.y_m, P.y_min) * dmove);
        int acc = 0, pos = 0;
        float dchi = 0.0f;
        uint4 batch = make_uint4(0u, 0u, 0u, 0u);
        for (int mv = 0; mv < NO; ++mv) {
            const int src = mv & 31;
            if (src == 0) batch = philox4x32_10(make_uint4((uint32_t)(mv + lane), (uint32_t)n, (uint32_t)w, 0u), key);
            const uint32_t w0 = __shfl_sync(kFull, batch.x, src);
            const uint32_t w1 = __shfl_sync(kFull, batch.y, src);
            const uint32_t w2 = __shfl_sync(kFull, batch.z, src);
            const uint32_t w3 = __shfl_sync(kFull, batch.w, src);
            int p, s;
            move_bins(w0, w1, NO, p, s);
            const float eps = yd * (2.0f * unit32(w2) - 1.0f);
            const float u = unit32(w3);
            const float r = 1.0f - eps;
            const float gap = (float)(p - s) * dwf;      // x_p - x_s
            const float dp = eps * beta[s] / gap;
            const float ds = -eps * beta[p] / gap;
            const float ap = fmaf(r, ghi * b[p], dp);
            const float as = fmaf(r, ghi * b[s], ds);
            unsigned code;
            if (ap < 0.0f || as < 0.0f) {
                code = 2;
                ++pos;
            } else {
                const float *Kp = K + (size_t)p * PAD + lane;
                const float *Ks = K + (size_t)s * PAD + lane;
                float d[C];
                float part = 0.0f;
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    d[c] = fmaf(-ds, __ldg(Ks + 32 * c), fmaf(-dp, __ldg(Kp + 32 * c), eps * M[c]));
                    part = fmaf(d[c], fmaf(2.0f, R[c], d[c]), part);
                }
                const float D = warp_sum(part);
                if (D <= 0.0f || u < __expf(-D * invT)) {
#pragma unroll
                    for (int c = 0; c < C; ++c) {
                        R[c] += d[c];
                        M[c] -= d[c];
                    }
                    pair_scale(ghi, glo, r);
                    if (lane == 0) {
                        b[p] = ap / ghi;
                        b[s] = as / ghi;
                    }
                    __syncwarp();
                    dchi += D;
                    ++acc;
                    code = 1;
                } else {
                    code = 0;
                }
            }
            h = (h ^ code) * kFnvPrime;
        }
        chi2 += (double)dchi;
        accp = acc;
        nacc += acc;
        npos += pos;
        if (S.acc_trace && lane == 0) S.acc_trace[(size_t)n * P.n_walkers + w] = acc;
    }
    // fold the common scale into the stored spectrum
    for (int j = lane; j < NO; j += 32) {
        const float v = b[j];
        b[j] = fmaf(glo, v, ghi * v);
    }
#pragma unroll
    for (int c = 0; c < C; ++c) S.R32[(size_t)w * PAD + lane + 32 * c] = R[c];
    if (lane == 0) {
        S.g2[2 * w] = 1.0f;
        S.g2[2 * w + 1] = 0.0f;
        S.chi2[w] = chi2;
        S.acc_prev[w] = accp;
        S.hash[w] = h;
        S.n_acc[w] += nacc;
        S.n_pos[w] += npos;
    }
}

template <int C>
cudaError_t launch_c(const DevProblem &P, const DevState &S, int n0, int n1, cudaStream_t st) {
    const int threads = 128;
    const int blocks = (P.n_walkers * 32 + threads - 1) / threads;
    sweep_fp32_kernel<C><<<blocks, threads, 0, st>>>(P, S, n0, n1);
    return cudaGetLastError();
}

// The proposal probe: one warp per proposal, the handle's own move arithmetic on the
// stored state, no state change.
__global__ void probe_kernel(DevProblem P, DevState S, int precision, int n, const int *walker,
                             const int *pp, const int *ss, const double *epsv, double *delta, int *ok) {
    const int lane = threadIdx.x & 31;
    const int q = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (q >= n) return;
    const int w = walker[q], p = pp[q], s = ss[q];
    const int NO = P.n_omega, PAD = P.n_tau_pad;
    if (precision == 0) {
        const double eps = epsv[q], r = 1.0 - eps;
        const double *a = S.a64 + (size_t)w * NO;
        const double xp = P.x64[p], xs = P.x64[s];
        const double dp = eps * (P.B - P.A * xs) / (xp - xs);
        const double ds = eps * (P.B - P.A * xp) / (xs - xp);
        const double ap = r * a[p] + dp, as = r * a[s] + ds;
        if (ap < 0.0 || as < 0.0) {
            if (lane == 0) { ok[q] = 0; delta[q] = 0.0; }
            return;
        }
        double part = 0.0;
        for (int i = lane; i < P.n_tau; i += 32) {
            const double R = S.R64[(size_t)w * PAD + i];
            const double d = eps * (P.Fhat64[i] - R) - dp * P.Khat64[(size_t)p * PAD + i] - ds * P.Khat64[(size_t)s * PAD + i];
            part += d * (2.0 * R + d);
        }
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(kFull, part, o);
        if (lane == 0) { ok[q] = 1; delta[q] = part; }
        return;
    }
    const float eps = (float)epsv[q], r = 1.0f - eps;
    const float ghi = S.g2[2 * w];
    const float *b = S.b32 + (size_t)w * NO;
    const float gap = (float)(p - s) * (float)P.dw;
    const float dp = eps * P.beta32[s] / gap;
    const float ds = -eps * P.beta32[p] / gap;
    const float ap = fmaf(r, ghi * b[p], dp), as = fmaf(r, ghi * b[s], ds);
    if (ap < 0.0f || as < 0.0f) {
        if (lane == 0) { ok[q] = 0; delta[q] = 0.0; }
        return;
    }
    float part = 0.0f;
    for (int i = lane; i < PAD; i += 32) {
        const float R = S.R32[(size_t)w * PAD + i];
        const float M = P.Fhat32[i] - R;
        const float d = fmaf(-ds, P.Khat32[(size_t)s * PAD + i], fmaf(-dp, P.Khat32[(size_t)p * PAD + i], eps * M));
        part = fmaf(d, fmaf(2.0f, R, d), part);
    }
    part = warp_sum(part);
    if (lane == 0) { ok[q] = 1; delta[q] = (double)part; }
}

// Every resident thread reads the buffer reps times with 16-byte loads (grid-stride).
__global__ void read_probe_kernel(const uint4 *__restrict__ buf, size_t n16, int reps,
                                  unsigned long long *sink) {
    uint32_t acc = 0;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (int r = 0; r < reps; ++r) {
        for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < n16; q += stride) {
            const uint4 v = __ldcg(buf + q);
            acc ^= v.x ^ v.y ^ v.z ^ v.w;
        }
    }
    if (acc == 0x9E3779B9u) sink[0] = acc;  // keeps the loads; practically never taken
}

}  // namespace

cudaError_t launch_read_probe(const void *buf, size_t bytes, int reps, void *sink, cudaStream_t st) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    read_probe_kernel<<<sms * 4, 512, 0, st>>>((const uint4 *)buf, bytes / 16, reps, (unsigned long long *)sink);
    return cudaGetLastError();
}

cudaError_t launch_sweep_fp32(const DevProblem &P, const DevState &S, int n0, int n1, cudaStream_t st) {
    switch (P.n_tau_pad / 32) {
        case 1: return launch_c<1>(P, S, n0, n1, st);
        case 2: return launch_c<2>(P, S, n0, n1, st);
        case 3: return launch_c<3>(P, S, n0, n1, st);
        case 4: return launch_c<4>(P, S, n0, n1, st);
        case 5: return launch_c<5>(P, S, n0, n1, st);
        case 6: return launch_c<6>(P, S, n0, n1, st);
        case 7: return launch_c<7>(P, S, n0, n1, st);
        case 8: return launch_c<8>(P, S, n0, n1, st);
        case 9: return launch_c<9>(P, S, n0, n1, st);
        case 10: return launch_c<10>(P, S, n0, n1, st);
        case 11: return launch_c<11>(P, S, n0, n1, st);
        case 12: return launch_c<12>(P, S, n0, n1, st);
        case 13: return launch_c<13>(P, S, n0, n1, st);
        case 14: return launch_c<14>(P, S, n0, n1, st);
        case 15: return launch_c<15>(P, S, n0, n1, st);
        case 16: return launch_c<16>(P, S, n0, n1, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_probe(const DevProblem &P, const DevState &S, int precision, int n, const int *walker,
                         const int *p, const int *s, const double *eps, double *delta, int *ok, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const int threads = 128;
    probe_kernel<<<(n * 32 + threads - 1) / threads, threads, 0, st>>>(P, S, precision, n, walker, p, s, eps,
                                                                      delta, ok);
    return cudaGetLastError();
}

}  // namespace sail
