// FP32 production sweep (Sec. 2.2 moves, Eq. probability-density acceptance) and the
// proposal probe.
//
// Kernel columns from two small tables.  Eq. (efficient-correlation-model) writes the bin
// kernel as c_i q_i^j with q_i = e^{-dw tau_i}; so with j = 32 h + l,
//     Khat_ij = Khat_{i,32h} * q_i^l = Qhi[h][i] * Qlo[l][i],
// and the two tables ((N_omega/32 + 32) rows of n_tau_pad floats, 57 KB at 200 x 1000) sit in
// shared memory.  A move reads its two columns from there: no L2 traffic, no L2 latency.
//
// Walker layout.  One persistent block per SM; 16 lanes per walker (two walkers per warp),
// lane l of a half-warp holding R_i and M_i = Fhat_i - R_i for i = 32 c + 2 l, 32 c + 2 l + 1.
// The move's scalar work (random words, bins, amplitudes, positivity, Metropolis) is shared by
// the two walkers of a warp.  Random words for 16 consecutive moves are drawn at once, one
// Philox call per lane, and broadcast by shuffle within the half-warp.  Delta chi2 =
// sum_i d_i (2 R_i + d_i) is reduced by an xor butterfly over the half-warp.
//
// Spectrum.  a = g b: an accepted move multiplies the common scale g by r (an unevaluated
// pair of floats, error ~1e-14 over a launch) and writes only b_p and b_s.  When the block's
// spectra fit in shared memory next to the tables they are staged there for the launch.  The
// scale is folded back into b when the launch ends, so residual recomputation sees a = b.
#include <cmath>
#include <cstdint>

#include "moves.cuh"
#include "philox.cuh"
#include "sail_internal.cuh"

namespace sail {

namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kThreads = 512;          // at most 16 warps (32 walkers) per round

__device__ __forceinline__ float half_sum(float v) {
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
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

// The FP32 move amplitudes of Eqs. (update-delta-p/s): rgap[k] = 1 / (k dw).
__device__ __forceinline__ void deltas(float eps, int p, int s, const float *beta, const float *rgap,
                                       float &dp, float &ds) {
    const int k = p - s;
    const float inv_gap = k > 0 ? rgap[k] : -rgap[-k];   // 1 / (x_p - x_s)
    dp = (eps * beta[s]) * inv_gap;
    ds = -(eps * beta[p]) * inv_gap;
}

struct SweepGeom {
    int pairs_total;      // ceil(n_walkers / 2)
    int pairs_per_cta;
    int warps;            // warps per block
    int rounds;           // pairs handled one after another by each warp
    int stage_b;          // spectra staged in shared memory
};

// Loads a problem's kernel factor tables, beta and the reciprocal gaps into shared memory.
__device__ void load_tables(const DevProblem &P, float *sm) {
    const int NO = P.n_omega, PAD = P.n_tau_pad, NH = (NO + 31) >> 5;
    float *sQhi = sm;
    float *sQlo = sQhi + (size_t)NH * PAD;
    float *sBeta = sQlo + (size_t)32 * PAD;
    float *sRgap = sBeta + NO;
    const float4 *g4 = reinterpret_cast<const float4 *>(P.Qhi32);
    float4 *s4 = reinterpret_cast<float4 *>(sQhi);
    for (int q = threadIdx.x; q < NH * PAD / 4; q += blockDim.x) s4[q] = g4[q];
    g4 = reinterpret_cast<const float4 *>(P.Qlo32);
    s4 = reinterpret_cast<float4 *>(sQlo);
    for (int q = threadIdx.x; q < 32 * PAD / 4; q += blockDim.x) s4[q] = g4[q];
    for (int q = threadIdx.x; q < NO; q += blockDim.x) {
        sBeta[q] = P.beta32[q];
        sRgap[q] = P.rgap32[q];
    }
}

// Packed pairs of floats: Blackwell executes mul/fma.rn.f32x2 as one instruction for two
// independent round-to-nearest operations, so each element pair of the move costs half the
// instructions of two scalar streams and rounds exactly as they would.
typedef unsigned long long f2;
__device__ __forceinline__ f2 pk(float a, float b) {
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ float2 up(f2 v) {
    float2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
    return r;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b) {
    f2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {
    f2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f2 add2(f2 a, f2 b) {
    f2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 lds2(const float *p) { return *reinterpret_cast<const f2 *>(p); }

// Sweeps [n0, n1) for the two walkers 2 pair, 2 pair + 1 of one problem on one warp (half-warp
// per walker).  sm holds the problem's tables; b_stage, if not null, the staged spectra of
// walkers walker_lo.. .  Every 16 moves each lane of a half-warp draws the random words of one
// move and works out that move's bins, amplitude eps, acceptance uniform u and delta_p,
// delta_s (Eqs. update-delta-p/s); the move loop then takes them by shuffle.
template <int C2>
__device__ void run_pair(const DevProblem &P, const DevState &S, int n0, int n1, int pair, const float *sm,
                         float *b_stage, int walker_lo) {
    const int NO = P.n_omega, PAD = P.n_tau_pad, NH = (NO + 31) >> 5;
    const float *sQhi = sm;
    const float *sQlo = sQhi + (size_t)NH * PAD;
    const float *sBeta = sQlo + (size_t)32 * PAD;
    const float *sRgap = sBeta + NO;
    const int lane = threadIdx.x & 31, hl = lane & 15, half = lane >> 4;
    const uint2 key = philox_key(P.seed);
    const double dmove = P.move_scale > 0.0 ? P.move_scale : 1.0 / NO;

    const int w = 2 * pair + half;
    const bool active = w < P.n_walkers;
    const int wr = active ? w : 2 * pair;             // a valid walker to read from
    float *b = b_stage ? b_stage + (size_t)(wr - walker_lo) * NO : S.b32 + (size_t)wr * NO;

    f2 R[C2], M[C2];
#pragma unroll
    for (int c = 0; c < C2; ++c) {
        const float2 r2 = *reinterpret_cast<const float2 *>(S.R32 + (size_t)wr * PAD + 32 * c + 2 * hl);
        const float2 f2v = *reinterpret_cast<const float2 *>(P.Fhat32 + 32 * c + 2 * hl);
        R[c] = pk(r2.x, r2.y);
        M[c] = pk(f2v.x - r2.x, f2v.y - r2.y);
    }
    float ghi = S.g2[2 * wr], glo = S.g2[2 * wr + 1];
    double chi2 = S.chi2[wr];
    int accp = S.acc_prev[wr];
    unsigned long long nacc = 0, npos = 0;
    const f2 two = pk(2.0f, 2.0f), minus_one = pk(-1.0f, -1.0f);

    for (int n = n0; n < n1; ++n) {
        const float invT = (float)(1.0 / P.Tsweep[n]);
        const float yd = (float)(amplitude(accp, NO, P.y_p, P.y_m, P.y_min) * dmove);
        int acc = 0, pos = 0;
        float dchi = 0.0f;
        int my_ps = 0;
        float my_eps = 0.0f, my_u = 0.0f, my_dp = 0.0f, my_ds = 0.0f;
        for (int mv = 0; mv < NO; ++mv) {
            const int src = mv & 15;
            if (src == 0) {
                const uint4 rnd = philox4x32_10(make_uint4((uint32_t)(mv + hl), (uint32_t)n, (uint32_t)wr, 0u), key);
                int p, s;
                move_bins(rnd.x, rnd.y, NO, p, s);
                my_ps = p | (s << 16);
                my_eps = yd * (2.0f * unit32(rnd.z) - 1.0f);
                my_u = unit32(rnd.w);
                deltas(my_eps, p, s, sBeta, sRgap, my_dp, my_ds);
            }
            const int ps = __shfl_sync(kFull, my_ps, src, 16);
            const float eps = __shfl_sync(kFull, my_eps, src, 16);
            const float u = __shfl_sync(kFull, my_u, src, 16);
            const float dp = __shfl_sync(kFull, my_dp, src, 16);
            const float ds = __shfl_sync(kFull, my_ds, src, 16);
            const int p = ps & 0xFFFF, s = ps >> 16;
            const float r = 1.0f - eps;
            const float ap = fmaf(r, ghi * b[p], dp);
            const float as = fmaf(r, ghi * b[s], ds);
            const bool ok = active && ap >= 0.0f && as >= 0.0f;
            pos += (active && !ok);
            if (__any_sync(kFull, ok)) {
                const float *qhp = sQhi + (p >> 5) * PAD + 2 * hl;
                const float *qlp = sQlo + (p & 31) * PAD + 2 * hl;
                const float *qhs = sQhi + (s >> 5) * PAD + 2 * hl;
                const float *qls = sQlo + (s & 31) * PAD + 2 * hl;
                const f2 e2 = pk(eps, eps), mdp = pk(-dp, -dp), mds = pk(-ds, -ds);
                f2 d[C2];
                f2 part = pk(0.0f, 0.0f);
#pragma unroll
                for (int c = 0; c < C2; ++c) {
                    const f2 Kp = mul2(lds2(qhp + 32 * c), lds2(qlp + 32 * c));
                    const f2 Ks = mul2(lds2(qhs + 32 * c), lds2(qls + 32 * c));
                    d[c] = fma2(mds, Ks, fma2(mdp, Kp, mul2(e2, M[c])));
                    part = fma2(d[c], fma2(two, R[c], d[c]), part);
                }
                const float2 pp = up(part);
                const float D = half_sum(pp.x + pp.y);
                if (ok && (D <= 0.0f || u < __expf(-D * invT))) {
#pragma unroll
                    for (int c = 0; c < C2; ++c) {
                        R[c] = add2(R[c], d[c]);
                        M[c] = fma2(minus_one, d[c], M[c]);
                    }
                    pair_scale(ghi, glo, r);
                    if (hl == 0) {
                        const float inv_g = 1.0f / ghi;
                        b[p] = ap * inv_g;
                        b[s] = as * inv_g;
                    }
                    dchi += D;
                    ++acc;
                }
            }
            __syncwarp();
        }
        chi2 += (double)dchi;
        accp = acc;
        nacc += acc;
        npos += pos;
        if (active && S.acc_trace && hl == 0) S.acc_trace[(size_t)n * P.n_walkers + w] = acc;
    }
    if (!active) return;
    // fold the common scale into the spectrum and write the walker back
    float *bg = S.b32 + (size_t)w * NO;
    for (int j = hl; j < NO; j += 16) {
        const float v = b[j];
        bg[j] = fmaf(glo, v, ghi * v);
    }
#pragma unroll
    for (int c = 0; c < C2; ++c)
        *reinterpret_cast<float2 *>(S.R32 + (size_t)w * PAD + 32 * c + 2 * hl) = up(R[c]);
    if (hl == 0) {
        S.g2[2 * w] = 1.0f;
        S.g2[2 * w + 1] = 0.0f;
        S.chi2[w] = chi2;
        S.acc_prev[w] = accp;
        S.n_acc[w] += nacc;
        S.n_pos[w] += npos;
    }
}

template <int C2>
__global__ void __launch_bounds__(kThreads) sweep_fp32_kernel(DevProblem P, DevState S, int n0, int n1,
                                                              SweepGeom G) {
    extern __shared__ float4 smem4[];
    float *sm = reinterpret_cast<float *>(smem4);
    const int NO = P.n_omega, PAD = P.n_tau_pad, NH = (NO + 31) >> 5;
    float *sB = sm + (size_t)(NH + 32) * PAD + 2 * NO;   // staged spectra [2 * pairs_per_cta][NO]
    load_tables(P, sm);
    const int pair_lo = blockIdx.x * G.pairs_per_cta;
    const int pair_hi = min(pair_lo + G.pairs_per_cta, G.pairs_total);
    const int walker_lo = 2 * pair_lo;
    const int walker_hi = min(2 * pair_hi, P.n_walkers);
    if (G.stage_b) {
        const size_t n = (size_t)(walker_hi - walker_lo) * NO;
        const float *src = S.b32 + (size_t)walker_lo * NO;
        for (size_t q = threadIdx.x; q < n; q += blockDim.x) sB[q] = src[q];
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5;
    for (int round = 0; round < G.rounds; ++round) {
        const int pair = pair_lo + round * G.warps + warp;
        if (pair >= pair_hi) break;                       // uniform across the warp
        run_pair<C2>(P, S, n0, n1, pair, sm, G.stage_b ? sB : nullptr, walker_lo);
    }
}

// Many inversions in one persistent launch: blocks take (problem, pair range) items from a
// queue, load the item's problem tables when the problem changes, and run one pair per warp.
// The per-walker arithmetic is that of sweep_fp32_kernel, so a walker's trajectory does not
// depend on which block, or which other problems, share the launch.
__global__ void __launch_bounds__(kThreads) sweep_batch_kernel(const BatchProblem *probs, const BatchItem *items,
                                                               int n_items, int *counter) {
    extern __shared__ float4 smem4[];
    float *sm = reinterpret_cast<float *>(smem4);
    __shared__ int s_item, s_loaded;
    if (threadIdx.x == 0) s_loaded = -1;
    const int warp = threadIdx.x >> 5;
    for (;;) {
        __syncthreads();                       // the previous item is finished with the tables
        if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= n_items) break;
        const BatchItem I = items[it];
        const BatchProblem &BP = probs[I.prob];
        if (I.prob != s_loaded) {
            load_tables(BP.P, sm);
            __syncthreads();
            if (threadIdx.x == 0) s_loaded = I.prob;
        }
        __syncthreads();
        const int pair = I.pair_lo + warp;
        if (pair >= I.pair_hi || BP.n0 >= BP.n1) continue;
        switch (BP.P.n_tau_pad / 32) {
            case 1: run_pair<1>(BP.P, BP.S, BP.n0, BP.n1, pair, sm, nullptr, 0); break;
            case 2: run_pair<2>(BP.P, BP.S, BP.n0, BP.n1, pair, sm, nullptr, 0); break;
            case 3: run_pair<3>(BP.P, BP.S, BP.n0, BP.n1, pair, sm, nullptr, 0); break;
            case 4: run_pair<4>(BP.P, BP.S, BP.n0, BP.n1, pair, sm, nullptr, 0); break;
            case 5: run_pair<5>(BP.P, BP.S, BP.n0, BP.n1, pair, sm, nullptr, 0); break;
            case 6: run_pair<6>(BP.P, BP.S, BP.n0, BP.n1, pair, sm, nullptr, 0); break;
            case 7: run_pair<7>(BP.P, BP.S, BP.n0, BP.n1, pair, sm, nullptr, 0); break;
            case 8: run_pair<8>(BP.P, BP.S, BP.n0, BP.n1, pair, sm, nullptr, 0); break;
            case 9: run_pair<9>(BP.P, BP.S, BP.n0, BP.n1, pair, sm, nullptr, 0); break;
            case 10: run_pair<10>(BP.P, BP.S, BP.n0, BP.n1, pair, sm, nullptr, 0); break;
            case 11: run_pair<11>(BP.P, BP.S, BP.n0, BP.n1, pair, sm, nullptr, 0); break;
            case 12: run_pair<12>(BP.P, BP.S, BP.n0, BP.n1, pair, sm, nullptr, 0); break;
            case 13: run_pair<13>(BP.P, BP.S, BP.n0, BP.n1, pair, sm, nullptr, 0); break;
            case 14: run_pair<14>(BP.P, BP.S, BP.n0, BP.n1, pair, sm, nullptr, 0); break;
            case 15: run_pair<15>(BP.P, BP.S, BP.n0, BP.n1, pair, sm, nullptr, 0); break;
            case 16: run_pair<16>(BP.P, BP.S, BP.n0, BP.n1, pair, sm, nullptr, 0); break;
            default: break;
        }
    }
}

size_t table_bytes(const DevProblem &P) {
    const size_t NH = (size_t)(P.n_omega + 31) / 32;
    return (NH + 32) * (size_t)P.n_tau_pad * 4 + 2 * (size_t)P.n_omega * 4;
}

template <int C2>
cudaError_t launch_c(const DevProblem &P, const DevState &S, int n0, int n1, cudaStream_t st) {
    int dev = 0, sms = 0, smem_max = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    SweepGeom G;
    G.pairs_total = (P.n_walkers + 1) / 2;
    const int ctas = G.pairs_total < sms ? G.pairs_total : sms;
    G.pairs_per_cta = (G.pairs_total + ctas - 1) / ctas;
    const int max_warps = kThreads / 32;
    G.rounds = (G.pairs_per_cta + max_warps - 1) / max_warps;
    G.warps = (G.pairs_per_cta + G.rounds - 1) / G.rounds;
    const size_t tb = table_bytes(P);
    const size_t staged = (size_t)2 * G.pairs_per_cta * P.n_omega * 4;
    if (tb > (size_t)smem_max) return cudaErrorInvalidValue;
    G.stage_b = tb + staged <= (size_t)smem_max;
    const size_t smem = tb + (G.stage_b ? staged : 0);
    cudaError_t e = cudaFuncSetAttribute(sweep_fp32_kernel<C2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int n_ctas = (G.pairs_total + G.pairs_per_cta - 1) / G.pairs_per_cta;
    sweep_fp32_kernel<C2><<<n_ctas, G.warps * 32, smem, st>>>(P, S, n0, n1, G);
    return cudaGetLastError();
}

// The proposal probe: one warp per proposal, the FP32 arithmetic of the sweep (or FP64 for a
// validation handle) on the stored state, no state change.
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
    float dp, ds;
    deltas(eps, p, s, P.beta32, P.rgap32, dp, ds);
    const float ap = fmaf(r, ghi * b[p], dp), as = fmaf(r, ghi * b[s], ds);
    if (ap < 0.0f || as < 0.0f) {
        if (lane == 0) { ok[q] = 0; delta[q] = 0.0; }
        return;
    }
    float part = 0.0f;
    for (int i = lane; i < PAD; i += 32) {
        const float R = S.R32[(size_t)w * PAD + i];
        const float M = P.Fhat32[i] - R;
        const float Kp = P.Qhi32[(p >> 5) * PAD + i] * P.Qlo32[(p & 31) * PAD + i];
        const float Ks = P.Qhi32[(s >> 5) * PAD + i] * P.Qlo32[(s & 31) * PAD + i];
        const float d = fmaf(-ds, Ks, fmaf(-dp, Kp, eps * M));
        part = fmaf(d, fmaf(2.0f, R, d), part);
    }
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(kFull, part, o);
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

// Shared-memory read bandwidth: each thread reads 16-byte words of a 32 KiB block-local
// buffer, a warp's 32 lanes on 512 consecutive bytes (no bank conflicts), reps times; the
// loads are volatile so none is merged or hoisted.
__global__ void __launch_bounds__(1024) smem_probe_kernel(int reps, unsigned long long *sink) {
    __shared__ uint4 buf[2048];
    for (int q = threadIdx.x; q < 2048; q += blockDim.x) buf[q] = make_uint4(q, q * 3u, q * 5u, q * 7u);
    __syncthreads();
    uint32_t acc = 0;
    int idx = threadIdx.x;
    const uint32_t base = (uint32_t)__cvta_generic_to_shared(buf);
#pragma unroll 8
    for (int r = 0; r < reps; ++r) {
        uint32_t x, y, z, w;
        asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                     : "=r"(x), "=r"(y), "=r"(z), "=r"(w)
                     : "r"(base + 16u * (uint32_t)idx));
        acc ^= x ^ y ^ z ^ w;
        idx = (idx + 1056) & 2047;   // next 512-byte row for the warp, shifted by 32 words
    }
    if (acc == 0x9E3779B9u) sink[0] = acc;  // keeps the loads; practically never taken
}

}  // namespace

cudaError_t launch_smem_probe(int reps, void *sink, cudaStream_t st, double *bytes) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int blocks = 2 * sms;
    smem_probe_kernel<<<blocks, 1024, 0, st>>>(reps, (unsigned long long *)sink);
    *bytes = (double)blocks * 1024.0 * (double)reps * 16.0;
    return cudaGetLastError();
}

size_t sweep_fp32_table_bytes(const DevProblem &P) { return table_bytes(P); }

cudaError_t launch_sweep_batch(const BatchProblem *d_probs, const BatchItem *d_items, int n_items, int *d_counter,
                               size_t smem, int warps, cudaStream_t st) {
    if (n_items <= 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = cudaFuncSetAttribute(sweep_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(d_counter, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    // one block per SM, or two when two blocks' tables fit in one SM's shared memory
    int per_sm = 1;
    int smem_sm = 0;
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    if (2 * (smem + 2048) <= (size_t)smem_sm && warps <= 8) per_sm = 2;
    const int blocks = n_items < sms * per_sm ? n_items : sms * per_sm;
    sweep_batch_kernel<<<blocks, warps * 32, smem, st>>>(d_probs, d_items, n_items, d_counter);
    return cudaGetLastError();
}

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
