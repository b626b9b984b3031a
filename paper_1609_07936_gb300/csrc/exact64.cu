// FP64 kernels whose every operation is rounded on its own (this file is compiled with
// -fmad=false): the validation sweep, the residual recomputation, the branching solve and
// imprint, the stochastic average and the state initialisation.  Sums run in the order the
// method's definition states them (j ascending for a model value, i ascending for chi2,
// walkers ascending for an average), so these kernels reproduce a plain sequential FP64
// evaluation of the same formulas bit for bit, up to the library exp of the Metropolis test.
#include <cfloat>
#include <cmath>
#include <cstdint>

#include "moves.cuh"
#include "philox.cuh"
#include <cuda_bf16.h>

#include "sail_internal.cuh"

namespace sail {

namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;

// ------------------------------------------------------------------ state set-up
__global__ void init_state_kernel(DevProblem P, DevState S, int precision, const double *a0,
                                  const double *R0, double chi2_0) {
    const int w = blockIdx.x;
    if (w >= P.n_walkers) return;
    for (int j = threadIdx.x; j < P.n_omega; j += blockDim.x) {
        if (precision == 0) S.a64[(size_t)w * P.n_omega + j] = a0[j];
        else S.b32[(size_t)w * P.n_omega + j] = (float)a0[j];
    }
    for (int i = threadIdx.x; i < P.n_tau_pad; i += blockDim.x) {
        const double r = i < P.n_tau ? R0[i] : 0.0;
        if (precision == 0) S.R64[(size_t)w * P.n_tau_pad + i] = r;
        else S.R32[(size_t)w * P.n_tau_pad + i] = (float)r;
    }
    if (threadIdx.x == 0) {
        S.chi2[w] = chi2_0;
        S.acc_prev[w] = P.n_omega;
        S.hash[w] = kFnvOffset;
        S.n_acc[w] = 0;
        S.n_pos[w] = 0;
        if (precision != 0) {
            S.g2[2 * w] = 1.0f;
            S.g2[2 * w + 1] = 0.0f;
        }
    }
}

// ------------------------------------------------------------------ validation sweep
// One warp per walker.  Lane l holds R_i for i = l + 32 c.  Every move is Sec. 2.2:
//   eps = 1 - r, delta_p = eps (B - A x_s) / (x_p - x_s), delta_s = eps (B - A x_p) / (x_s - x_p),
//   a_p' = r a_p + delta_p, a_s' = r a_s + delta_s (rejected if either is negative),
//   d_i = eps (Fhat_i - R_i) - delta_p Khat_ip - delta_s Khat_is,
//   Delta chi2 = sum_i d_i (2 R_i + d_i), summed over i ascending,
// accepted with probability min(1, exp(-Delta chi2 / T)) (Eq. probability-density); an
// accepted move rescales every bin by r, writes a_p', a_s' and adds d to R.
// Bins of a move (Sec. 2.3) in the oracle's order: p from word w0, then its index walk of
// L = P.walk_len steps (step t: Philox counter (mv, n, w, 1 + t), proposal word x, acceptance
// word y; move when u a_p <= a_j); s from word w1 on the bins other than the final p, then its
// walk (words z, w; proposals on the bins other than p).  Each walk is skipped with
// probability walk_rho (words x, y of counter (mv, n, w, 2 + L)).
__device__ void walk_bins64(const DevProblem &P, const double *a, uint32_t w0, uint32_t w1, int mv, int n, int w,
                            uint2 key, int &p_out, int &s_out) {
    const int NO = P.n_omega, L = P.walk_len;
    int p = (int)(((uint64_t)w0 * (uint64_t)NO) >> 32);
    bool walk_p = false, walk_s = false;
    if (L > 0) {
        const uint4 mix = philox4x32_10(make_uint4((uint32_t)mv, (uint32_t)n, (uint32_t)w, (uint32_t)(2 + L)), key);
        walk_p = !(unit64(mix.x) < P.walk_rho);
        walk_s = !(unit64(mix.y) < P.walk_rho);
    }
    for (int t = 1; t <= L && walk_p; ++t) {
        const uint4 r = philox4x32_10(make_uint4((uint32_t)mv, (uint32_t)n, (uint32_t)w, (uint32_t)(1 + t)), key);
        const int j = (int)(((uint64_t)r.x * (uint64_t)NO) >> 32);
        if (unit64(r.y) * a[p] <= a[j]) p = j;
    }
    int s = (int)(((uint64_t)w1 * (uint64_t)(NO - 1)) >> 32);
    s += (s >= p);
    for (int t = 1; t <= L && walk_s; ++t) {
        const uint4 r = philox4x32_10(make_uint4((uint32_t)mv, (uint32_t)n, (uint32_t)w, (uint32_t)(1 + t)), key);
        int j = (int)(((uint64_t)r.z * (uint64_t)(NO - 1)) >> 32);
        j += (j >= p);
        if (unit64(r.w) * a[s] <= a[j]) s = j;
    }
    p_out = p;
    s_out = s;
}

template <int C>
__global__ void __launch_bounds__(128) sweep_fp64_kernel(DevProblem P, DevState S, int n0, int n1) {
    const int lane = threadIdx.x & 31;
    const int w = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (w >= P.n_walkers) return;
    const int NT = P.n_tau, NO = P.n_omega, PAD = P.n_tau_pad;
    double *a = S.a64 + (size_t)w * NO;
    double R[C], Fh[C];
#pragma unroll
    for (int c = 0; c < C; ++c) {
        R[c] = S.R64[(size_t)w * PAD + lane + 32 * c];
        Fh[c] = P.Fhat64[lane + 32 * c];
    }
    double chi2 = S.chi2[w];
    int accp = S.acc_prev[w];
    unsigned long long h = S.hash[w], nacc = 0, npos = 0;
    const uint2 key = philox_key(P.seed);
    const double dmove = P.move_scale > 0.0 ? P.move_scale : 1.0 / NO;
    const int wg = w + P.walker_base;   // the walker's index in the whole population

    for (int n = n0; n < n1; ++n) {
        const double T = P.Tsweep[n];
        const double y = amplitude(accp, NO, P.y_p, P.y_m, P.y_min);
        int acc = 0;
        for (int mv = 0; mv < NO; ++mv) {
            const uint4 rnd = philox4x32_10(make_uint4((uint32_t)mv, (uint32_t)n, (uint32_t)wg, 0u), key);
            // shared bins: the group's first walker's words 0 and 1 (its own counter)
            uint2 bw = make_uint2(rnd.x, rnd.y);
            if (P.shared_bins > 1 && wg % P.shared_bins != 0) {
                const uint4 g = philox4x32_10(
                    make_uint4((uint32_t)mv, (uint32_t)n, (uint32_t)(wg - wg % P.shared_bins), 0u), key);
                bw = make_uint2(g.x, g.y);
            }
            int p, s;
            walk_bins64(P, a, bw.x, bw.y, mv, n, wg, key, p, s);
            const double eps = (y * dmove) * (2.0 * unit64(rnd.z) - 1.0);
            const double u = unit64(rnd.w);
            const double r = 1.0 - eps;
            const double xp = P.x64[p], xs = P.x64[s];
            const double dp = eps * (P.B - P.A * xs) / (xp - xs);
            const double ds = eps * (P.B - P.A * xp) / (xs - xp);
            const double ap = r * a[p] + dp;
            const double as = r * a[s] + ds;
            unsigned code;
            if (ap < 0.0 || as < 0.0) {
                code = 2;
                ++npos;
            } else {
                const double *Kp = P.Khat64 + (size_t)p * PAD;
                const double *Ks = P.Khat64 + (size_t)s * PAD;
                double d[C], t[C];
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    const int i = lane + 32 * c;
                    const double M = Fh[c] - R[c];
                    d[c] = eps * M - dp * Kp[i] - ds * Ks[i];
                    t[c] = d[c] * (2.0 * R[c] + d[c]);
                }
                double D = 0.0;
#pragma unroll
                for (int c = 0; c < C; ++c) {
                    for (int l = 0; l < 32; ++l) {
                        const double v = __shfl_sync(kFull, t[c], l);
                        if (32 * c + l < NT) D = D + v;
                    }
                }
                bool accept;
                if (!P.hastings) {
                    accept = D <= 0.0 || u < exp(-D / T);
                } else {
                    // Metropolis-Hastings with the move's Jacobian r^(N-4), the reverse amplitude
                    // -eps/r proposable only when |eps/r| < y d (the oracle's or_accept)
                    accept = fabs(eps / r) < y * dmove && u < exp(-D / T + (double)(NO - 4) * log(r));
                }
                if (accept) {
                    for (int j = lane; j < NO; j += 32) a[j] = r * a[j];
                    __syncwarp();
                    if (lane == 0) {
                        a[p] = ap;
                        a[s] = as;
                    }
                    __syncwarp();
#pragma unroll
                    for (int c = 0; c < C; ++c) R[c] = R[c] + d[c];
                    chi2 = chi2 + D;
                    ++acc;
                    code = 1;
                } else {
                    code = 0;
                }
            }
            h = (h ^ code) * kFnvPrime;
        }
        accp = acc;
        nacc += acc;
        if (S.acc_trace && lane == 0) S.acc_trace[(size_t)n * P.n_walkers + w] = acc;
    }
#pragma unroll
    for (int c = 0; c < C; ++c) S.R64[(size_t)w * PAD + lane + 32 * c] = R[c];
    if (lane == 0) {
        S.chi2[w] = chi2;
        S.acc_prev[w] = accp;
        S.hash[w] = h;
        S.n_acc[w] += nacc;
        S.n_pos[w] += npos;
    }
}

// ------------------------------------------------------------------ residual recomputation
// R_i = Fhat_i - sum_j Khat_ij a_j with j ascending, chi2 = sum_i R_i^2 with i ascending.
// One block per walker.  FP32 state enters as (double) b_j; the sweep kernel folds its
// common scale into b before this runs.
//
// FP32 state only: rounding in the moves lets sum a and sum a x wander by ~1e-6 of A and B
// over a resync interval (exact arithmetic keeps them fixed, Sec. 2.2), so before the residual
// is formed each walker is put back on both sum rules with the
// affine reweighting b_j <- b_j kappa (1 + lambda (x_j - c)): c = B'/A', kappa = A / A',
// lambda = (B/A - c) / var', where A' = sum b, B' = sum b x and var' = sum b x^2 / A' - c^2 are
// the walker's current moments (lambda = 0 if the tilt could make a factor negative).  One
// warp per walker, one pass for the moments: FP32 per bin, in the offset t_j = x_j - x_mid =
// (j - (N-1)/2) dw from the grid's midpoint (uniform bins), with compensated per-lane sums and
// FP64 across lanes; the factor is applied in FP32, the state's own precision (FP64 runs at a
// small fraction of the FP32 rate on this GPU).
__device__ __forceinline__ void kahan_add(float &s, float &comp, float v) {
    const float y = v - comp;
    const float t = s + y;
    comp = (t - s) - y;
    s = t;
}

// The three BF16 pieces (each the round-to-nearest BF16 of what is left) of 8 consecutive
// spectrum values for the tensor-copy recomputation, stored as three 16-byte rows at
// [piece][walker][bin] of At (v past the last bin is 0).
__device__ __forceinline__ void put_pieces8(unsigned short *At, size_t plane, size_t at, const float (&v)[8]) {
    uint32_t w1[4], w2[4], w3[4];
#pragma unroll
    for (int e = 0; e < 8; e += 2) {
        uint32_t p1[2], p2[2], p3[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const __nv_bfloat16 b1 = __float2bfloat16_rn(v[e + h]);
            const float r = v[e + h] - __bfloat162float(b1);
            const __nv_bfloat16 b2 = __float2bfloat16_rn(r);
            const __nv_bfloat16 b3 = __float2bfloat16_rn(r - __bfloat162float(b2));
            p1[h] = __bfloat16_as_ushort(b1);
            p2[h] = __bfloat16_as_ushort(b2);
            p3[h] = __bfloat16_as_ushort(b3);
        }
        w1[e / 2] = p1[0] | (p1[1] << 16);
        w2[e / 2] = p2[0] | (p2[1] << 16);
        w3[e / 2] = p3[0] | (p3[1] << 16);
    }
    *reinterpret_cast<uint4 *>(At + at) = make_uint4(w1[0], w1[1], w1[2], w1[3]);
    *reinterpret_cast<uint4 *>(At + plane + at) = make_uint4(w2[0], w2[1], w2[2], w2[3]);
    *reinterpret_cast<uint4 *>(At + 2 * plane + at) = make_uint4(w3[0], w3[1], w3[2], w3[3]);
}

// At (optional): also write the restored spectra's BF16 pieces for the tensor-copy
// recomputation, rows of nop bins, planes of `plane` elements (the padding stays zero).
__global__ void __launch_bounds__(256) restore_kernel(DevProblem P, DevState S, unsigned short *At, int nop,
                                                      size_t plane) {
    const int w = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (w >= P.n_walkers) return;
    float *b = S.b32 + (size_t)w * P.n_omega;
    const float dw = (float)P.dw, half = 0.5f * (float)(P.n_omega - 1);
    float a0 = 0.f, c0 = 0.f, a1 = 0.f, c1 = 0.f, a2 = 0.f, c2 = 0.f;
    for (int j = lane; j < P.n_omega; j += 32) {
        const float v = b[j], xj = ((float)j - half) * dw;
        kahan_add(a0, c0, v);
        kahan_add(a1, c1, v * xj);
        kahan_add(a2, c2, v * xj * xj);
    }
    double s0 = (double)a0 - (double)c0, s1 = (double)a1 - (double)c1, s2 = (double)a2 - (double)c2;
    for (int o = 16; o > 0; o >>= 1) {
        s0 += __shfl_xor_sync(0xFFFFFFFFu, s0, o);
        s1 += __shfl_xor_sync(0xFFFFFFFFu, s1, o);
        s2 += __shfl_xor_sync(0xFFFFFFFFu, s2, o);
    }
    if (s0 > 0.0) {
        const double xmid = 0.5 * (P.x64[0] + P.x64[P.n_omega - 1]);
        const double c = s1 / s0;                               // centre, as an offset from xmid
        const double var = s2 / s0 - c * c;
        const double kappa = P.A / s0;
        double lambda = var > 0.0 ? (P.B / P.A - xmid - c) / var : 0.0;
        if (!(fabs(lambda * (P.n_omega - 1) * P.dw) < 0.5)) lambda = 0.0;
        const float kf = (float)kappa, lk = (float)(kappa * lambda), cf = (float)c;
        for (int j = lane; j < P.n_omega; j += 32) {
            const float xj = ((float)j - half) * dw;
            b[j] = b[j] * fmaf(lk, xj - cf, kf);
        }
    }
    if (!At) return;
    // the pieces of the restored spectrum, 8 bins a lane (16-byte stores)
    __syncwarp();
    const size_t row = (size_t)w * nop;
    for (int j0 = 8 * lane; j0 < P.n_omega; j0 += 256) {
        float v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = j0 + e < P.n_omega ? b[j0 + e] : 0.0f;
        put_pieces8(At, plane, row + j0, v);
    }
}

__global__ void __launch_bounds__(128) resync_kernel(DevProblem P, DevState S, int precision) {
    __shared__ double Rs[kMaxTau];
    const int w = blockIdx.x;
    const int NO = P.n_omega, PAD = P.n_tau_pad;
    for (int i = threadIdx.x; i < PAD; i += blockDim.x) {
        double r = 0.0;
        if (i < P.n_tau) {
            double model = 0.0;
            if (precision == 0) {
                const double *a = S.a64 + (size_t)w * NO;
                for (int j = 0; j < NO; ++j) model = model + P.Khat64[(size_t)j * PAD + i] * a[j];
            } else {
                const float *b = S.b32 + (size_t)w * NO;
                for (int j = 0; j < NO; ++j) model = model + P.Khat64[(size_t)j * PAD + i] * (double)b[j];
            }
            r = P.Fhat64[i] - model;
        }
        Rs[i] = r;
        if (precision == 0) S.R64[(size_t)w * PAD + i] = r;
        else S.R32[(size_t)w * PAD + i] = (float)r;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double c2 = 0.0;
        for (int i = 0; i < P.n_tau; ++i) c2 = c2 + Rs[i] * Rs[i];
        S.chi2[w] = c2;
    }
}

// ------------------------------------------------------------------ branching (Sec. 2.5)
// Walker l has weight w_l = exp[-Delta (z_l - P_r)], z_l = (chi2_l - min) / (mean - min), and
// multiplier m_l = floor(w_l + xi_l).  Writing Theta = exp(Delta P_r) and E_l = exp(-Delta z_l),
// m_l = floor(Theta E_l + xi_l), which steps up by one at each "break point"
// Delta z_l + ln(k - xi_l) = ln Theta, k = 1, 2, ...  P_r is fixed by sum m = N: ln Theta lies
// between the N-th and (N+1)-th smallest break points of all walkers, found by bisection on
// ln Theta until the count is exactly N.  Z(Delta) = #{m_l = 0}; Delta doubles from 1 until
// Z >= round(f N), then bisects, stopping at the first Delta with Z = round(f N).
struct SolveShared {
    double red_d[32];
    int red_i[32];
    double bcast_d;
    int bcast_i;
    double theta;
    double cmin, spread;
    int scan[kSolveThreads / 32];
};

__device__ double block_sum_d(double v, SolveShared &sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) sh.red_d[warp] = v;
    __syncthreads();
    if (warp == 0) {
        v = lane < (int)(blockDim.x >> 5) ? sh.red_d[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
        if (lane == 0) sh.bcast_d = v;
    }
    __syncthreads();
    return sh.bcast_d;
}

__device__ int block_sum_i(int v, SolveShared &sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) sh.red_i[warp] = v;
    __syncthreads();
    if (warp == 0) {
        v = lane < (int)(blockDim.x >> 5) ? sh.red_i[lane] : 0;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
        if (lane == 0) sh.bcast_i = v;
    }
    __syncthreads();
    return sh.bcast_i;
}

// Exclusive prefix sum over the block in thread order; returns this thread's offset and
// writes the total to *total.
__device__ int block_scan_excl(int v, int *total, SolveShared &sh) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int incl = v;
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += t;
    }
    __syncthreads();
    if (lane == 31) sh.scan[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const int nw = (int)(blockDim.x >> 5);
        int x = lane < nw ? sh.scan[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(kFull, x, o);
            if (lane >= o) x += t;
        }
        if (lane < nw) sh.scan[lane] = x;  // inclusive over warps
    }
    __syncthreads();
    const int warp_off = warp > 0 ? sh.scan[warp - 1] : 0;
    *total = sh.scan[(blockDim.x >> 5) - 1];
    return warp_off + incl - v;
}

// Multipliers at one Delta; returns Z.  Walker l = threadIdx.x + kSolveThreads * q, q < PT.
template <int PT>
__device__ int multipliers_at(int N, const double *z, const double *xi, double Delta, int *m,
                              SolveShared &sh) {
    const int tid = threadIdx.x;
    double E[PT];
    double sE = 0.0;
#pragma unroll
    for (int q = 0; q < PT; ++q) {
        const int l = tid + kSolveThreads * q;
        E[q] = l < N ? exp(-Delta * z[q]) : 0.0;
        sE += E[q];
    }
    sE = block_sum_d(sE, sh);
    auto count_at = [&](double lnTheta, bool store) -> int {
        if (tid < 32) {
            const double Th = exp(lnTheta);
            if (tid == 0) sh.theta = Th;
        }
        __syncthreads();
        const double Th = sh.theta;
        int c = 0;
#pragma unroll
        for (int q = 0; q < PT; ++q) {
            const int l = tid + kSolveThreads * q;
            int mq = 0;
            if (l < N) {
                const double v = floor(Th * E[q] + xi[q]);
                mq = v >= (double)N ? N : (int)v;
            }
            if (store) m[q] = mq;
            c += mq;
        }
        return block_sum_i(c, sh);
    };
    // Sum m is close to Theta * sum E; bracket ln Theta around ln(N / sum E).
    const double guess = log((double)N / sE);
    double lo = guess - 0.25, hi = guess + 0.25;
    int clo = count_at(lo, false), chi = count_at(hi, false);
    for (int it = 0; it < 200 && clo >= N; ++it) { lo -= (hi - lo); clo = count_at(lo, false); }
    for (int it = 0; it < 200 && chi < N; ++it) { hi += (hi - lo); chi = count_at(hi, false); }
    bool hit = false;
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (!(mid > lo && mid < hi)) break;
        const int c = count_at(mid, true);
        if (c == N) { hit = true; break; }
        if (c < N) lo = mid; else hi = mid;
    }
    if (!hit) {
        // Break points tied at ln Theta: take the upper end and drop the surplus copies
        // from the highest walker indices whose count rises across the final bracket.
        int c = count_at(hi, true);
        int mlo[PT];
        {
            if (tid < 32) { const double Th = exp(lo); if (tid == 0) sh.theta = Th; }
            __syncthreads();
            const double Th = sh.theta;
#pragma unroll
            for (int q = 0; q < PT; ++q) {
                const int l = tid + kSolveThreads * q;
                const double v = l < N ? floor(Th * E[q] + xi[q]) : 0.0;
                mlo[q] = v >= (double)N ? N : (int)v;
            }
            __syncthreads();
        }
        for (int q = PT - 1; q >= 0 && c > N; --q) {
            for (int t = kSolveThreads - 1; t >= 0 && c > N; --t) {
                // serial over walkers in descending index order; thread t owns walker l
                if (tid == t) {
                    const int l = t + kSolveThreads * q;
                    int take = 0;
                    if (l < N) {
                        const int extra = m[q] - mlo[q];
                        take = extra < (c - N) ? extra : (c - N);
                        m[q] -= take;
                    }
                    sh.bcast_i = take;
                }
                __syncthreads();
                c -= sh.bcast_i;
                __syncthreads();
            }
        }
    }
    int zc = 0;
#pragma unroll
    for (int q = 0; q < PT; ++q) {
        const int l = tid + kSolveThreads * q;
        zc += (l < N && m[q] == 0);
    }
    return block_sum_i(zc, sh);
}

// The Delta search runs as speculative rounds over many blocks: every trial Delta the
// sequential search could visit next is evaluated at once, one block (one SM) per trial, and
// a one-thread control kernel replays the sequential search over the results.  Round 0 holds
// the doubling trials 2^k, k = 0..64; each later round a depth-7 tree of bisection midpoints.
// The replay takes exactly the steps, trial values and early exit of the sequential search,
// so the chosen Delta and multipliers are the same; one SM per trial brings 127 SMs' FP64
// units to bear on what is otherwise a long chain on one SM.
constexpr int kTreeDepth = 7;
constexpr int kMaxCand = (1 << kTreeDepth) - 1;   // 127 >= the 65 doubling trials

struct SolveCtl {
    double lo, hi, Delta;
    int Zhi, Zt, done, it, n_cand;
};

template <int PT>
__device__ void load_zxi(const BranchScratch &B, int N, double *z, double *xi) {
#pragma unroll
    for (int q = 0; q < PT; ++q) {
        const int l = threadIdx.x + kSolveThreads * q;
        z[q] = l < N ? B.z[l] : 0.0;
        xi[q] = l < N ? B.xi[l] : 0.5;
    }
}

__global__ void __launch_bounds__(kSolveThreads) branch_prep_kernel(DevProblem P, DevState S, BranchScratch B,
                                                                    int block_index, double fraction) {
    __shared__ double s_cmin, s_spread;
    extern __shared__ double s_chi2[];           // the walkers' chi2, staged for the ordered sum
    const int N = P.n_walkers, tid = threadIdx.x;
    SolveCtl *ctl = reinterpret_cast<SolveCtl *>(B.ctl);
    int Zt = (int)floor(fraction * N + 0.5);
    if (Zt > N - 1) Zt = N - 1;
    for (int l = tid; l < N; l += blockDim.x) s_chi2[l] = S.chi2[l];
    __syncthreads();
    if (tid == 0) {
        double cmin = s_chi2[0], csum = 0.0;
        for (int l = 0; l < N; ++l) {
            if (s_chi2[l] < cmin) cmin = s_chi2[l];
            csum += s_chi2[l];
        }
        s_cmin = cmin;
        s_spread = csum / N - cmin;
        ctl->Zt = Zt;
        ctl->done = Zt <= 0;
        ctl->it = 0;
        ctl->lo = 0.0;
        ctl->hi = 1.0;
        ctl->Delta = 0.0;
        ctl->n_cand = 65;
    }
    if (tid < 65) B.cand[tid] = ldexp(1.0, tid);
    __syncthreads();
    const double cmin = s_cmin, spread = s_spread;
    const uint2 key = philox_key(P.seed);
    for (int l = tid; l < N; l += blockDim.x) {
        B.z[l] = spread > 0.0 ? (s_chi2[l] - cmin) / spread : 0.0;
        B.xi[l] = unit64(philox4x32_10(make_uint4((uint32_t)(l + P.walker_base), (uint32_t)block_index, 0u, 1u), key).x);
    }
}

template <int PT>
__global__ void __launch_bounds__(kSolveThreads) branch_eval_kernel(int N, BranchScratch B) {
    __shared__ SolveShared sh;
    const SolveCtl *ctl = reinterpret_cast<const SolveCtl *>(B.ctl);
    if (ctl->done || (int)blockIdx.x >= ctl->n_cand) return;   // uniform per block
    double z[PT], xi[PT];
    int m[PT];
    load_zxi<PT>(B, N, z, xi);
    const int Z = multipliers_at<PT>(N, z, xi, B.cand[blockIdx.x], m, sh);
    if (threadIdx.x == 0) B.cand_Z[blockIdx.x] = Z;
}

// Writes the 127 midpoints of a depth-7 bisection tree over (lo, hi) in heap order: node n
// (1-based) holds the interval reached by the outcomes on its path; its children 2n and 2n+1
// are the intervals after "Z > target" (hi <- mid) and "Z < target" (lo <- mid).
__device__ void build_tree(double lo, double hi, double *cand) {
    double nlo[kMaxCand + 1], nhi[kMaxCand + 1];
    nlo[1] = lo;
    nhi[1] = hi;
    for (int n = 1; n <= kMaxCand; ++n) {
        const double mid = 0.5 * (nlo[n] + nhi[n]);
        cand[n - 1] = mid;
        if (2 * n <= kMaxCand) {
            nlo[2 * n] = nlo[n];
            nhi[2 * n] = mid;
            nlo[2 * n + 1] = mid;
            nhi[2 * n + 1] = nhi[n];
        }
    }
}

__global__ void branch_control_kernel(BranchScratch B, int round) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    SolveCtl *ctl = reinterpret_cast<SolveCtl *>(B.ctl);
    if (ctl->done) return;
    const int Zt = ctl->Zt;
    if (round == 0) {
        // doubling: hi = 1, 2, 4, ... while Z(hi) < target, at most 64 doublings
        double lo = 0.0, hi = 1.0;
        int k = 0, Zhi = B.cand_Z[0];
        while (k < 64 && Zhi < Zt) {
            lo = hi;
            hi = 2.0 * hi;
            ++k;
            Zhi = B.cand_Z[k];
        }
        ctl->lo = lo;
        ctl->hi = hi;
        ctl->Zhi = Zhi;
        if (Zhi == Zt) {
            ctl->done = 1;
            ctl->Delta = hi;
            return;
        }
    } else {
        double lo = ctl->lo, hi = ctl->hi;
        int n = 1;
        for (int d = 0; d < kTreeDepth; ++d) {
            if (ctl->it >= 64) { ctl->done = 1; ctl->Delta = hi; return; }
            const double mid = B.cand[n - 1];
            if (mid <= lo || mid >= hi) { ctl->done = 1; ctl->Delta = hi; return; }
            const int Zm = B.cand_Z[n - 1];
            ctl->it += 1;
            if (Zm == Zt) { ctl->done = 1; ctl->Delta = mid; return; }
            if (Zm < Zt) { lo = mid; n = 2 * n + 1; }
            else { hi = mid; n = 2 * n; }
        }
        ctl->lo = lo;
        ctl->hi = hi;
    }
    if (ctl->it >= 64) { ctl->done = 1; ctl->Delta = ctl->hi; return; }
    build_tree(ctl->lo, ctl->hi, B.cand);
    ctl->n_cand = kMaxCand;
}

// Final multipliers at the chosen Delta and the imprint pairing: zero-multiplier walkers
// ascending, matched with surplus copies (walker l listed m_l - 1 times) ascending.
template <int PT>
__global__ void __launch_bounds__(kSolveThreads) branch_final_kernel(int N, BranchScratch B, int event) {
    __shared__ SolveShared sh;
    const SolveCtl *ctl = reinterpret_cast<const SolveCtl *>(B.ctl);
    const int tid = threadIdx.x;
    int m[PT];
    double Delta = 0.0;
    if (ctl->Zt <= 0) {
#pragma unroll
        for (int q = 0; q < PT; ++q) m[q] = 1;
    } else {
        double z[PT], xi[PT];
        load_zxi<PT>(B, N, z, xi);
        Delta = ctl->done ? ctl->Delta : ctl->hi;
        multipliers_at<PT>(N, z, xi, Delta, m, sh);
    }
    int zero_base = 0, copy_base = 0;
#pragma unroll
    for (int q = 0; q < PT; ++q) {
        const int l = tid + kSolveThreads * q;
        const bool valid = l < N;
        const int isz = valid && m[q] == 0;
        const int surplus = valid && m[q] > 1 ? m[q] - 1 : 0;
        int tz, tc;
        const int zo = block_scan_excl(isz, &tz, sh);
        const int co = block_scan_excl(surplus, &tc, sh);
        if (valid) {
            B.m[l] = m[q];
            if (isz) B.zero_l[zero_base + zo] = l;
            for (int k = 0; k < surplus; ++k) B.donor_l[copy_base + co + k] = l;
            if (B.m_trace) B.m_trace[(size_t)event * N + l] = m[q];
        }
        zero_base += tz;
        copy_base += tc;
    }
    if (tid == 0) {
        B.n_pairs[0] = zero_base < copy_base ? zero_base : copy_base;
        B.delta[0] = Delta;
        if (B.delta_trace) B.delta_trace[event] = Delta;
    }
}

template <int PT>
cudaError_t launch_solve(const DevProblem &P, const DevState &S, const BranchScratch &B, int block_index,
                         double fraction, int event, cudaStream_t st, int *launches) {
    const int N = P.n_walkers;
    const size_t staged = (size_t)N * sizeof(double);   // <= 128 KiB (16384 walkers)
    cudaError_t e0 = cudaFuncSetAttribute(branch_prep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)staged);
    if (e0 != cudaSuccess) return e0;
    branch_prep_kernel<<<1, kSolveThreads, staged, st>>>(P, S, B, block_index, fraction);
    branch_eval_kernel<PT><<<kMaxCand, kSolveThreads, 0, st>>>(N, B);
    branch_control_kernel<<<1, 32, 0, st>>>(B, 0);
    *launches += 3;
    for (int r = 1; r <= (64 + kTreeDepth - 1) / kTreeDepth; ++r) {
        branch_eval_kernel<PT><<<kMaxCand, kSolveThreads, 0, st>>>(N, B);
        branch_control_kernel<<<1, 32, 0, st>>>(B, r);
        *launches += 2;
    }
    branch_final_kernel<PT><<<1, kSolveThreads, 0, st>>>(N, B, event);
    *launches += 1;
    return cudaGetLastError();
}

// Imprinting (Sec. 2.5): a^(l1) <- t a^(l2) + (1 - t) a^(l1); the residual mixes the same way
// by linearity and chi2 of l1 is summed again.  One block per pair; no donor is imprinted.
__global__ void __launch_bounds__(128) imprint_kernel(DevProblem P, DevState S, BranchScratch B,
                                                      int precision, double t) {
    __shared__ double Rs[kMaxTau];
    const int q = blockIdx.x;
    if (q >= B.n_pairs[0]) return;
    const int l1 = B.zero_l[q], l2 = B.donor_l[q];
    const double omt = 1.0 - t;
    const int NO = P.n_omega, PAD = P.n_tau_pad;
    if (precision == 0) {
        double *a1 = S.a64 + (size_t)l1 * NO;
        const double *a2 = S.a64 + (size_t)l2 * NO;
        for (int j = threadIdx.x; j < NO; j += blockDim.x) a1[j] = t * a2[j] + omt * a1[j];
        for (int i = threadIdx.x; i < PAD; i += blockDim.x) {
            const double r = t * S.R64[(size_t)l2 * PAD + i] + omt * S.R64[(size_t)l1 * PAD + i];
            S.R64[(size_t)l1 * PAD + i] = r;
            Rs[i] = r;
        }
    } else {
        float *b1 = S.b32 + (size_t)l1 * NO;
        const float *b2 = S.b32 + (size_t)l2 * NO;
        const float tf = (float)t, omtf = (float)omt;
        for (int j = threadIdx.x; j < NO; j += blockDim.x) b1[j] = tf * b2[j] + omtf * b1[j];
        for (int i = threadIdx.x; i < PAD; i += blockDim.x) {
            const double r = t * (double)S.R32[(size_t)l2 * PAD + i] + omt * (double)S.R32[(size_t)l1 * PAD + i];
            S.R32[(size_t)l1 * PAD + i] = (float)r;
            Rs[i] = (double)(float)r;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double c2 = 0.0;
        for (int i = 0; i < P.n_tau; ++i) c2 = c2 + Rs[i] * Rs[i];
        S.chi2[l1] = c2;
    }
}

// Walker rows for another handle of the population: spectrum and residual of idx[q] in FP64.
__global__ void walker_rows_kernel(DevProblem P, DevState S, int precision, const int *idx, double *a_rows,
                                   double *R_rows) {
    const int q = blockIdx.x, l = idx[q];
    const int NO = P.n_omega, NT = P.n_tau, PAD = P.n_tau_pad;
    for (int j = threadIdx.x; j < NO; j += blockDim.x)
        a_rows[(size_t)q * NO + j] = precision == 0 ? S.a64[(size_t)l * NO + j] : (double)S.b32[(size_t)l * NO + j];
    for (int i = threadIdx.x; i < NT; i += blockDim.x)
        R_rows[(size_t)q * NT + i] = precision == 0 ? S.R64[(size_t)l * PAD + i] : (double)S.R32[(size_t)l * PAD + i];
}

// Imprinting from donor rows (Sec. 2.5), the arithmetic of imprint_kernel with the donor's
// values read from rows in this device's memory: walker idx[q] <- t row q + (1 - t) itself.
__global__ void __launch_bounds__(128) imprint_rows_kernel(DevProblem P, DevState S, int precision, const int *idx,
                                                           const double *a_rows, const double *R_rows, double t) {
    __shared__ double Rs[kMaxTau];
    const int q = blockIdx.x, l1 = idx[q];
    const double omt = 1.0 - t;
    const int NO = P.n_omega, NT = P.n_tau, PAD = P.n_tau_pad;
    const double *a2 = a_rows + (size_t)q * NO, *R2 = R_rows + (size_t)q * NT;
    if (precision == 0) {
        double *a1 = S.a64 + (size_t)l1 * NO;
        for (int j = threadIdx.x; j < NO; j += blockDim.x) a1[j] = t * a2[j] + omt * a1[j];
        for (int i = threadIdx.x; i < PAD; i += blockDim.x) {
            const double r = t * (i < NT ? R2[i] : 0.0) + omt * S.R64[(size_t)l1 * PAD + i];
            S.R64[(size_t)l1 * PAD + i] = r;
            Rs[i] = r;
        }
    } else {
        float *b1 = S.b32 + (size_t)l1 * NO;
        const float tf = (float)t, omtf = (float)omt;
        for (int j = threadIdx.x; j < NO; j += blockDim.x) b1[j] = tf * (float)a2[j] + omtf * b1[j];
        for (int i = threadIdx.x; i < PAD; i += blockDim.x) {
            const double r = t * (i < NT ? R2[i] : 0.0) + omt * (double)S.R32[(size_t)l1 * PAD + i];
            S.R32[(size_t)l1 * PAD + i] = (float)r;
            Rs[i] = (double)(float)r;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double c2 = 0.0;
        for (int i = 0; i < NT; ++i) c2 = c2 + Rs[i] * Rs[i];
        S.chi2[l1] = c2;
    }
}

// ------------------------------------------------------------------ statistics
__global__ void block_stats_kernel(DevProblem P, DevState S, BlockCounters *out) {
    double cmin = DBL_MAX, csum = 0.0;
    unsigned long long acc = 0, pos = 0;
    for (int w = threadIdx.x; w < P.n_walkers; w += blockDim.x) {
        const double c = S.chi2[w];
        cmin = c < cmin ? c : cmin;
        csum += c;
        acc += S.n_acc[w];
        pos += S.n_pos[w];
    }
    for (int o = 16; o > 0; o >>= 1) {
        const double c = __shfl_xor_sync(kFull, cmin, o);
        cmin = c < cmin ? c : cmin;
        csum += __shfl_xor_sync(kFull, csum, o);
        acc += __shfl_xor_sync(kFull, acc, o);
        pos += __shfl_xor_sync(kFull, pos, o);
    }
    __shared__ double smin[32], ssum[32];
    __shared__ unsigned long long sacc[32], spos[32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) { smin[warp] = cmin; ssum[warp] = csum; sacc[warp] = acc; spos[warp] = pos; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < (int)(blockDim.x >> 5); ++k) {
            cmin = smin[k] < cmin ? smin[k] : cmin;
            csum += ssum[k];
            acc += sacc[k];
            pos += spos[k];
        }
        out->chi2_min = cmin;
        out->chi2_sum = csum;
        out->acc = acc;
        out->pos = pos;
    }
}

// ------------------------------------------------------------------ stochastic average
// Walkers with chi2 <= factor * min chi2; mean over them (walkers ascending) and the standard
// error sqrt(sum (a - mean)^2 / (n - 1)) / sqrt(n) per bin (Sec. 1).
__global__ void average_select_kernel(DevProblem P, DevState S, double factor, int *n_used,
                                      double *cut_out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double cmin = S.chi2[0];
    for (int w = 1; w < P.n_walkers; ++w) if (S.chi2[w] < cmin) cmin = S.chi2[w];
    const double cut = factor * cmin;
    int used = 0;
    for (int w = 0; w < P.n_walkers; ++w) used += (S.chi2[w] <= cut);
    *n_used = used;
    *cut_out = cut;
}

__global__ void average_bins_kernel(DevProblem P, DevState S, int precision, const int *n_used,
                                    const double *cut_in, double *mean, double *err) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= P.n_omega) return;
    const double cut = *cut_in;
    const int used = *n_used;
    auto at = [&](int w) -> double {
        if (precision == 0) return S.a64[(size_t)w * P.n_omega + j];
        return (double)S.b32[(size_t)w * P.n_omega + j];
    };
    double m = 0.0;
    for (int w = 0; w < P.n_walkers; ++w) if (S.chi2[w] <= cut) m += at(w);
    m /= used;
    double e = 0.0;
    if (used > 1) {
        for (int w = 0; w < P.n_walkers; ++w) {
            if (!(S.chi2[w] <= cut)) continue;
            const double v = at(w) - m;
            e += v * v;
        }
        e = sqrt(e / (used - 1)) / sqrt((double)used);
    }
    mean[j] = m;
    if (err) err[j] = e;
}

__global__ void __launch_bounds__(128) residual_of_kernel(DevProblem P, const double *a, double *R,
                                                          double *chi2) {
    __shared__ double Rs[kMaxTau];
    for (int i = threadIdx.x; i < P.n_tau_pad; i += blockDim.x) {
        double r = 0.0;
        if (i < P.n_tau) {
            double model = 0.0;
            for (int j = 0; j < P.n_omega; ++j) model = model + P.Khat64[(size_t)j * P.n_tau_pad + i] * a[j];
            r = P.Fhat64[i] - model;
        }
        Rs[i] = r;
        if (R) R[i] = r;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double c2 = 0.0;
        for (int i = 0; i < P.n_tau; ++i) c2 = c2 + Rs[i] * Rs[i];
        *chi2 = c2;
    }
}

__global__ void philox_kernel(int n, const uint32_t *ctr, uint64_t seed, uint32_t *out) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const uint4 c = make_uint4(ctr[4 * q], ctr[4 * q + 1], ctr[4 * q + 2], ctr[4 * q + 3]);
    const uint4 r = philox4x32_10(c, philox_key(seed));
    out[4 * q] = r.x;
    out[4 * q + 1] = r.y;
    out[4 * q + 2] = r.z;
    out[4 * q + 3] = r.w;
}

template <int C>
cudaError_t launch_sweep64_c(const DevProblem &P, const DevState &S, int n0, int n1, cudaStream_t st) {
    const int threads = 128;
    const int blocks = (P.n_walkers * 32 + threads - 1) / threads;
    sweep_fp64_kernel<C><<<blocks, threads, 0, st>>>(P, S, n0, n1);
    return cudaGetLastError();
}


// Smoothing of one spectrum (Sec. smoothing), in the oracle's order of operations: the
// three-point stencil of strength s from the old values, ends (1 - s) a_0 + s a_1 and
// (1 - s) a_{N-1} + s a_{N-2}; then sums in bin order and the tilt a_j (1 + beta (x_j - m)),
// m = B'/A', beta = (B - B') / sum_j a_j (x_j - m)^2, which restores sum_j a_j x_j = B and
// keeps sum_j a_j (skipped when |beta| max_j |x_j - m| >= 1/2).  FP64 arithmetic; E is the
// element type of the state.
template <typename E>
__device__ void smooth_one(E *a, int N, const double *x, double B, double s) {
    const double c = 1.0 - 2.0 * s, e = 1.0 - s;
    double prev = (double)a[0];
    a[0] = (E)(e * (double)a[0] + s * (double)a[1]);
    for (int j = 1; j < N - 1; ++j) {
        const double cur = (double)a[j];
        a[j] = (E)(s * prev + c * cur + s * (double)a[j + 1]);
        prev = cur;
    }
    a[N - 1] = (E)(e * (double)a[N - 1] + s * prev);
    double A1 = 0.0, B1 = 0.0;
    for (int j = 0; j < N; ++j) {
        const double v = (double)a[j];
        A1 += v;
        B1 += v * x[j];
    }
    if (!(A1 > 0.0)) return;
    const double m = B1 / A1;
    double V = 0.0;
    for (int j = 0; j < N; ++j) {
        const double d = x[j] - m;
        V += (double)a[j] * d * d;
    }
    double beta = V > 0.0 ? (B - B1) / V : 0.0;
    const double span = fabs(x[0] - m) > fabs(x[N - 1] - m) ? fabs(x[0] - m) : fabs(x[N - 1] - m);
    if (!(fabs(beta) * span < 0.5)) beta = 0.0;
    for (int j = 0; j < N; ++j) a[j] = (E)((double)a[j] * (1.0 + beta * (x[j] - m)));
}

// Puts each FP64 spectrum back on both sum rules in the oracle's order (or_restore): sums in
// bin order, then a_j kappa (1 + lambda (x_j - c)).  One thread per walker.
__global__ void __launch_bounds__(128) restore_seq_kernel(DevProblem P, DevState S) {
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= P.n_walkers) return;
    const int N = P.n_omega;
    double *a = S.a64 + (size_t)w * N;
    const double *x = P.x64;
    double A1 = 0.0, B1 = 0.0;
    for (int j = 0; j < N; ++j) {
        A1 += a[j];
        B1 += a[j] * x[j];
    }
    if (!(A1 > 0.0)) return;
    const double c = B1 / A1;
    double V = 0.0;
    for (int j = 0; j < N; ++j) {
        const double d = x[j] - c;
        V += a[j] * d * d;
    }
    const double kappa = P.A / A1;
    double lambda = V > 0.0 ? (P.B / P.A - c) * A1 / V : 0.0;
    if (!(fabs(lambda * (x[N - 1] - x[0])) < 0.5)) lambda = 0.0;
    for (int j = 0; j < N; ++j) a[j] = a[j] * (kappa * (1.0 + lambda * (x[j] - c)));
}

__global__ void __launch_bounds__(128) smooth_kernel(DevProblem P, DevState S, int precision, double s) {
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= P.n_walkers) return;
    if (precision == 0)
        smooth_one(S.a64 + (size_t)w * P.n_omega, P.n_omega, P.x64, P.B, s);
    else
        smooth_one(S.b32 + (size_t)w * P.n_omega, P.n_omega, P.x64, P.B, s);
}

}  // namespace

// ------------------------------------------------------------------ launchers
cudaError_t launch_init_state(const DevProblem &P, const DevState &S, int precision, const double *a0,
                              const double *R0, double chi2_0, cudaStream_t st) {
    init_state_kernel<<<P.n_walkers, 128, 0, st>>>(P, S, precision, a0, R0, chi2_0);
    return cudaGetLastError();
}

cudaError_t launch_sweep_fp64(const DevProblem &P, const DevState &S, int n0, int n1, cudaStream_t st) {
    switch (P.n_tau_pad / 32) {
        case 1: return launch_sweep64_c<1>(P, S, n0, n1, st);
        case 2: return launch_sweep64_c<2>(P, S, n0, n1, st);
        case 3: return launch_sweep64_c<3>(P, S, n0, n1, st);
        case 4: return launch_sweep64_c<4>(P, S, n0, n1, st);
        case 5: return launch_sweep64_c<5>(P, S, n0, n1, st);
        case 6: return launch_sweep64_c<6>(P, S, n0, n1, st);
        case 7: return launch_sweep64_c<7>(P, S, n0, n1, st);
        case 8: return launch_sweep64_c<8>(P, S, n0, n1, st);
        case 9: return launch_sweep64_c<9>(P, S, n0, n1, st);
        case 10: return launch_sweep64_c<10>(P, S, n0, n1, st);
        case 11: return launch_sweep64_c<11>(P, S, n0, n1, st);
        case 12: return launch_sweep64_c<12>(P, S, n0, n1, st);
        case 13: return launch_sweep64_c<13>(P, S, n0, n1, st);
        case 14: return launch_sweep64_c<14>(P, S, n0, n1, st);
        case 15: return launch_sweep64_c<15>(P, S, n0, n1, st);
        case 16: return launch_sweep64_c<16>(P, S, n0, n1, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_resync(const DevProblem &P, const DevState &S, int precision, int restore, int kind,
                          int *status, cudaStream_t st, int *launches) {
    if (precision == 0) {
        if (P.hastings && restore) {
            // the Hastings chain drifts off the sum rules by rounding: put it back first
            restore_seq_kernel<<<(P.n_walkers + 127) / 128, 128, 0, st>>>(P, S);
            *launches += 1;
        }
        resync_kernel<<<P.n_walkers, 128, 0, st>>>(P, S, precision);
        *launches += 1;
        return cudaGetLastError();
    }
    if (kind == 2 && !P.tma) return cudaErrorInvalidValue;
    if (restore) {
        // with the tensor-copy recomputation the restoration also writes the BF16 pieces
        unsigned short *At = kind == 2 ? (unsigned short *)P.tma->At : nullptr;
        const int nop = kind == 2 ? P.tma->nop : 0;
        const size_t plane = kind == 2 ? (size_t)P.tma->n_blocks_walkers * 128 * nop : 0;
        restore_kernel<<<(P.n_walkers * 32 + 255) / 256, 256, 0, st>>>(P, S, At, nop, plane);
        *launches += 1;
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (kind == 3) {                  // FP64 GEMM
        *launches += 1;
        return launch_resync_fp64(P, S, st);
    }
    if (kind == 2) {                  // (pieces of the spectra), tensor-copy GEMM, chi2 pass
        *launches += restore ? 2 : 3;
        return launch_resync_tma(P, S, *P.tma, status, !restore, st);
    }
    *launches += kind == 1 ? 2 : 1;   // tensor-core GEMM + chi2 pass, or the FP32 GEMM
    return kind == 1 ? launch_resync_tc(P, S, status, false, st) : launch_resync_fp32(P, S, st);
}

cudaError_t launch_branch(const DevProblem &P, const DevState &S, const BranchScratch &B, int precision,
                          int block_index, double fraction, double imprint_t, int event, cudaStream_t st,
                          int *launches) {
    cudaError_t e;
    if (P.n_walkers <= kSolveThreads * 4) e = launch_solve<4>(P, S, B, block_index, fraction, event, st, launches);
    else if (P.n_walkers <= kSolveThreads * 8) e = launch_solve<8>(P, S, B, block_index, fraction, event, st, launches);
    else e = launch_solve<16>(P, S, B, block_index, fraction, event, st, launches);
    if (e != cudaSuccess) return e;
    imprint_kernel<<<P.n_walkers, 128, 0, st>>>(P, S, B, precision, imprint_t);
    *launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_branch_solve(const DevProblem &P, const DevState &S, const BranchScratch &B, int block_index,
                                double fraction, cudaStream_t st, int *launches) {
    if (P.n_walkers <= kSolveThreads * 4) return launch_solve<4>(P, S, B, block_index, fraction, 0, st, launches);
    if (P.n_walkers <= kSolveThreads * 8) return launch_solve<8>(P, S, B, block_index, fraction, 0, st, launches);
    return launch_solve<16>(P, S, B, block_index, fraction, 0, st, launches);
}

cudaError_t launch_walker_rows(const DevProblem &P, const DevState &S, int precision, int n, const int *idx,
                               double *a_rows, double *R_rows, cudaStream_t st) {
    walker_rows_kernel<<<n, 128, 0, st>>>(P, S, precision, idx, a_rows, R_rows);
    return cudaGetLastError();
}

cudaError_t launch_imprint_rows(const DevProblem &P, const DevState &S, int precision, int n, const int *idx,
                                const double *a_rows, const double *R_rows, double t, cudaStream_t st) {
    imprint_rows_kernel<<<n, 128, 0, st>>>(P, S, precision, idx, a_rows, R_rows, t);
    return cudaGetLastError();
}

cudaError_t launch_smooth(const DevProblem &P, const DevState &S, int precision, double s, cudaStream_t st) {
    smooth_kernel<<<(P.n_walkers + 127) / 128, 128, 0, st>>>(P, S, precision, s);
    return cudaGetLastError();
}

cudaError_t launch_block_stats(const DevProblem &P, const DevState &S, BlockCounters *out, cudaStream_t st) {
    block_stats_kernel<<<1, 1024, 0, st>>>(P, S, out);
    return cudaGetLastError();
}

cudaError_t launch_average(const DevProblem &P, const DevState &S, int precision, double factor, double *mean,
                           double *err, int *n_used, double *cut, double *R_mean, double *chi2_mean,
                           cudaStream_t st, int *launches) {
    average_select_kernel<<<1, 32, 0, st>>>(P, S, factor, n_used, cut);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    average_bins_kernel<<<(P.n_omega + 127) / 128, 128, 0, st>>>(P, S, precision, n_used, cut, mean, err);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    residual_of_kernel<<<1, 128, 0, st>>>(P, mean, R_mean, chi2_mean);
    *launches += 3;
    return cudaGetLastError();
}

cudaError_t launch_philox(int n, const uint32_t *ctr, uint64_t seed, uint32_t *out, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    philox_kernel<<<(n + 255) / 256, 256, 0, st>>>(n, ctr, seed, out);
    return cudaGetLastError();
}

}  // namespace sail
