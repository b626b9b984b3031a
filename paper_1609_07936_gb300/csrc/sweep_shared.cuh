// The FP32 sweep with shared bins: the W walkers of a warp (W = 2, 4 or 8) propose, at every
// move, the bins drawn by the group's first walker, each with its own amplitude and
// acceptance draw (a walker's bins stay uniform and independent of its spectrum, so its chain
// is the method's chain).
//
// With shared bins the bins' part of the residual change is common to the group: from the
// move amplitudes of Eqs. (update-delta-p/s), delta_p = eps c_s and delta_s = -eps c_p with
// c_j = beta_j / (x_p - x_s), so
//     d_i = eps M_i - delta_p Khat_ip - delta_s Khat_is = eps (M_i + Kc_i),
//     Kc_i = c_p Khat_is - c_s Khat_ip,
// and with M_i = Fhat_i - R_i a walker's change is d_i = eps t_i, t_i = G_i - R_i,
// G_i = Fhat_i + Kc_i.  Then
//     delta chi2 = sum_i d_i (2 R_i + d_i) = 2 eps (G.R - |R|^2) + eps^2 (|G|^2 - 2 G.R + |R|^2),
// where |R|^2 is the walker's residue chi2, which it tracks anyway, and |G|^2 belongs to the
// move.  The warp forms G and |G|^2 once per move (the columns from the factor tables,
// Eq. efficient-correlation-model); a walker pays one fused multiply-add per element for G.R
// and, when it accepts, R <- R + eps (G - R).
//
// Layout.  The warp's 32 lanes split the tau points (lane l holds i = l + 32 k, k < C) and each
// lane holds the residuals of all W walkers there, packed in walker pairs for f32x2
// arithmetic.  Lane l does the scalar work of walker l mod W (its spectrum, scale, counters);
// the 32 / W lanes of a walker do it alike, one of them writes.  delta chi2 of the W walkers is
// reduced by a transposing butterfly (each step halves the walkers a lane keeps) and two plain
// steps.  Each lane draws the random words of one walker for one of 32 / W consecutive moves;
// the next move's G is formed while the current move is reduced and tested.
//
// sweep_shared8.cu, sweep_shared4.cu and sweep_shared2.cu instantiate it for groups of 8, 4
// and 2 walkers (one translation unit each, compiled in parallel); sweep_shared.cu dispatches.
#pragma once
#include <cmath>
#include <cstdint>

#include "sweep_group.cuh"

namespace sail {

namespace {

__device__ __forceinline__ float lds_f32(uint32_t a) {
    float v;
    asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(a));
    return v;
}

// One walker's words for one move: the bins it would draw itself (the group's first walker's
// serve the group), its amplitude and its threshold -T ln u (with the Hastings Jacobian and
// the reverse move's feasibility folded in).
struct SharedDraw {
    int ps;
    float eps, thr;
};

template <int MODE>
__device__ __forceinline__ SharedDraw shared_draw(int mv, int n, int walker, uint2 key, int NO, float yd, float T) {
    const uint4 rnd = philox4x32_10(make_uint4((uint32_t)mv, (uint32_t)n, (uint32_t)walker, 0u), key);
    SharedDraw m;
    int p, s;
    move_bins(rnd.x, rnd.y, NO, p, s);
    m.ps = p | (s << 16);
    m.eps = yd * (2.0f * unit32(rnd.z) - 1.0f);
    m.thr = -logf(unit32(rnd.w)) * T;
    if constexpr (MODE == kHastings) {
        const float r = 1.0f - m.eps;
        m.thr = fabsf(m.eps / r) < yd ? m.thr + T * (float)(NO - 4) * log1pf(-m.eps) : -INFINITY;
    }
    return m;
}

// G_i = Fhat_i + c_p Khat_is - c_s Khat_ip for the lane's elements, duplicated in both halves
// of a pair, for the move with bins ps; also returns c_p, c_s and |G|^2 over all tau (every
// lane of the warp calls).
template <int C>
__device__ __forceinline__ void form_g(f2 (&G)[C], const float (&Fh)[C], int ps, uint32_t qhi, uint32_t qlo,
                                       int PAD, const float *beta, const float *rgap, float &cp, float &cs,
                                       float &gg) {
    const int p = ps & 0xFFFF, s = ps >> 16;
    const int k = p - s;
    const float ig = k > 0 ? rgap[k] : -rgap[-k];           // 1 / (x_p - x_s)
    cp = beta[p] * ig;
    cs = beta[s] * ig;
    const uint32_t hp = qhi + 4u * (uint32_t)((p >> 5) * PAD), lp = qlo + 4u * (uint32_t)((p & 31) * PAD);
    const uint32_t hs = qhi + 4u * (uint32_t)((s >> 5) * PAD), ls = qlo + 4u * (uint32_t)((s & 31) * PAD);
#pragma unroll
    for (int c = 0; c < C; ++c) {
        const float kp = lds_f32(hp + 128u * c) * lds_f32(lp + 128u * c);
        const float ks = lds_f32(hs + 128u * c) * lds_f32(ls + 128u * c);
        const float g = Fh[c] + fmaf(cp, ks, -(cs * kp));
        G[c] = pk(g, g);
        gg = c == 0 ? g * g : fmaf(g, g, gg);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) gg += __shfl_xor_sync(kFull, gg, o);
}

template <int W, int C, bool STAGED, int MODE>
__device__ __forceinline__ void run_shared(const DevProblem &P, const DevState &S, int n0, int n1, int grp,
                                           const float *sm, float *b_stage, int walker_lo) {
    constexpr int Q = W / 2;           // walker pairs
    constexpr int LW = W == 8 ? 3 : (W == 4 ? 2 : 1);  // log2 W
    constexpr int MPD = 32 / W;        // moves one draw round covers
    const int NO = P.n_omega, PAD = P.n_tau_pad, NH = (NO + 31) >> 5;
    const float *sQhi = sm;
    const float *sQlo = sQhi + (size_t)NH * PAD;
    const float *sBeta = sQlo + (size_t)32 * PAD;
    const float *sRgap = sBeta + NO;
    const int lane = threadIdx.x & 31, v = lane & (W - 1), q = lane >> LW;
    const uint32_t qhi = (uint32_t)__cvta_generic_to_shared(sQhi) + 4u * lane;
    const uint32_t qlo = (uint32_t)__cvta_generic_to_shared(sQlo) + 4u * lane;
    const uint2 key = philox_key(P.seed);
    const double dmove = P.move_scale > 0.0 ? P.move_scale : 1.0 / NO;

    const int g0 = W * grp;            // the group's first walker
    const int w = g0 + v;              // the walker of this lane's scalar work
    const bool active = w < P.n_walkers;
    const int wr = active ? w : g0;    // a valid walker to read from
    float *b = STAGED ? b_stage + (size_t)(wr - walker_lo) * NO : S.b32 + (size_t)wr * NO;
    const uint32_t bsh = STAGED ? (uint32_t)__cvta_generic_to_shared(b) : 0u;
    auto bget = [&](int j) -> float {
        if constexpr (STAGED) return lds_f32(bsh + 4u * (uint32_t)j);
        else return b[j];
    };
    auto bset = [&](int j, float val) {
        if constexpr (STAGED)
            asm volatile("st.shared.f32 [%0], %1;" ::"r"(bsh + 4u * (uint32_t)j), "f"(val) : "memory");
        else
            b[j] = val;
    };

    // residual elements of all W walkers (pairs), Fhat of the lane's elements
    f2 R[C][Q];
    float Fh[C];
#pragma unroll
    for (int c = 0; c < C; ++c) {
        const int i = lane + 32 * c;
        Fh[c] = P.Fhat32[i];
#pragma unroll
        for (int j = 0; j < Q; ++j) {
            const int wa = min(g0 + 2 * j, P.n_walkers - 1), wb = min(g0 + 2 * j + 1, P.n_walkers - 1);
            R[c][j] = pk(S.R32[(size_t)wa * PAD + i], S.R32[(size_t)wb * PAD + i]);
        }
    }
    float ghi = S.g2[2 * wr], glo = S.g2[2 * wr + 1];
    double chi2 = S.chi2[wr];
    float chi2f = (float)chi2;         // |R|^2 of the walker, as the moves change it
    int accp = S.acc_prev[wr];
    unsigned nacc = 0, npos = 0;
    const f2 minus_one = pk(-1.0f, -1.0f);

    for (int n = n0; n < n1; ++n) {
        const float T = (float)P.Tsweep[n];
        const float yd = (float)(amplitude(accp, NO, P.y_p, P.y_m, P.y_min) * dmove);
        int acc = 0, pos = 0;
        float dchi = 0.0f;
        // lane (v, q) holds walker v's words of move mv0 + q of the current round, and of the
        // next round
        SharedDraw cur = shared_draw<MODE>(q, n, w + P.walker_base, key, NO, yd, T);
        SharedDraw nxt = cur;
        if (MPD < NO) nxt = shared_draw<MODE>(MPD + q, n, w + P.walker_base, key, NO, yd, T);
        f2 Ga[C], Gb[C];
        float cpa, csa, gga, cpb = 0.0f, csb = 0.0f, ggb = 0.0f;
        const int ps0 = __shfl_sync(kFull, cur.ps, 0);
        form_g<C>(Ga, Fh, ps0, qhi, qlo, PAD, sBeta, sRgap, cpa, csa, gga);
        // this lane's walker's b at the current move's bins, read one move ahead (see below)
        float bpc = bget(ps0 & 0xFFFF), bsc = bget(ps0 >> 16);
        // one move; the loop runs two per iteration with G and Gn exchanging roles
        auto move = [&](const int mv, f2 (&G)[C], f2 (&Gn)[C], float &cp, float &cs, float &gg, float &cpn,
                        float &csn, float &ggn) {
            const int m = mv & (MPD - 1);
            if (m == 0 && mv > 0) {
                cur = nxt;
                if (mv + MPD < NO) nxt = shared_draw<MODE>(mv + MPD + q, n, w + P.walker_base, key, NO, yd, T);
            }
            // this move: the shared bins, every walker's amplitude, this lane's walker's threshold
            const int ps = __shfl_sync(kFull, cur.ps, W * m);
            f2 e2[Q];
#pragma unroll
            for (int j = 0; j < Q; ++j)
                e2[j] = pk(__shfl_sync(kFull, cur.eps, 2 * j + W * m), __shfl_sync(kFull, cur.eps, 2 * j + 1 + W * m));
            const float eps = __shfl_sync(kFull, cur.eps, v + W * m);
            const float thr = __shfl_sync(kFull, cur.thr, v + W * m);
            // the next move's bins (after the sweep's last move: this move's again, unused) and
            // this lane's walker's b values there, read now so that their latency overlaps this
            // move (measured at 512 tau x 2048 bins x 16384 walkers, groups of 4, spectra in
            // global memory: +10%); if this move is accepted and writes one of those bins, the
            // written value replaces the one read (the value a read after the write returns)
            const int nps_cur = __shfl_sync(kFull, cur.ps, (W * (m + 1)) & 31);
            const int nps_nxt = __shfl_sync(kFull, nxt.ps, 0);
            const int nps = mv + 1 >= NO ? ps : (m + 1 < MPD ? nps_cur : nps_nxt);
            float bpn = bget(nps & 0xFFFF), bsn = bget(nps >> 16);
            // every walker's G.R
            f2 acc2[Q];
#pragma unroll
            for (int j = 0; j < Q; ++j) acc2[j] = 0ull;
#pragma unroll
            for (int c = 0; c < C; ++c)
#pragma unroll
                for (int j = 0; j < Q; ++j) acc2[j] = fma2(G[c], R[c][j], acc2[j]);
            // the next move's G, while this one is reduced and tested
            form_g<C>(Gn, Fh, nps, qhi, qlo, PAD, sBeta, sRgap, cpn, csn, ggn);
            // transposing butterfly: after the step with mask 2^b a lane keeps the walkers whose
            // bit b equals its own; the last steps add up the lanes of each walker
            float s[W];
#pragma unroll
            for (int j = 0; j < Q; ++j) {
                const float2 a = up(acc2[j]);
                s[2 * j] = a.x;
                s[2 * j + 1] = a.y;
            }
#pragma unroll
            for (int bit = LW - 1; bit >= 0; --bit) {
                const int half = 1 << bit;
                const bool hi = (lane >> bit) & 1;
#pragma unroll
                for (int j = 0; j < half; ++j) {
                    const float keep = hi ? s[half + j] : s[j];
                    const float send = hi ? s[j] : s[half + j];
                    s[j] = keep + __shfl_xor_sync(kFull, send, half);
                }
            }
            float GR = s[0];
#pragma unroll
            for (int o = W; o < 32; o <<= 1) GR += __shfl_xor_sync(kFull, GR, o);
            // this lane's walker: delta chi2 = eps (2 (G.R - |R|^2) + eps (|G|^2 - 2 G.R + |R|^2))
            const float D = eps * fmaf(eps, (gg - 2.0f * GR) + chi2f, 2.0f * (GR - chi2f));
            // this lane's walker: positivity (Eq. probability-density) and the Metropolis test
            const int p = ps & 0xFFFF, sb = ps >> 16;
            const float r = 1.0f - eps;
            const float ap = fmaf(r, ghi * bpc, eps * cs);
            const float as = fmaf(r, ghi * bsc, -(eps * cp));
            const bool ok = active && ap >= 0.0f && as >= 0.0f;
            pos += (active && !ok);
            const bool accepted = ok && (MODE == kHastings ? D < thr : (D <= 0.0f || D < thr));
            const unsigned amask = __ballot_sync(kFull, accepted) & ((1u << W) - 1u);
            if (accepted) {
                pair_scale(ghi, glo, r);
                const float inv_g = 1.0f / ghi;
                const float bp_new = ap * inv_g, bs_new = as * inv_g;
                if (q == 0) {
                    bset(p, bp_new);
                    bset(sb, bs_new);
                }
                const int pn = nps & 0xFFFF, sn = nps >> 16;
                bpn = pn == p ? bp_new : (pn == sb ? bs_new : bpn);
                bsn = sn == p ? bp_new : (sn == sb ? bs_new : bsn);
                dchi += D;
                chi2f += D;
                ++acc;
            }
            // accepted walkers: R <- R + eps (G - R)
#pragma unroll
            for (int j = 0; j < Q; ++j) {
                if (amask & (3u << (2 * j))) {
                    const float2 e = up(e2[j]);
                    const f2 ea = pk((amask >> (2 * j)) & 1u ? e.x : 0.0f, (amask >> (2 * j + 1)) & 1u ? e.y : 0.0f);
#pragma unroll
                    for (int c = 0; c < C; ++c) R[c][j] = fma2(ea, fma2(minus_one, R[c][j], G[c]), R[c][j]);
                }
            }
            __syncwarp();
            bpc = bpn;
            bsc = bsn;
        };
        for (int mv = 0; mv + 1 < NO; mv += 2) {
            move(mv, Ga, Gb, cpa, csa, gga, cpb, csb, ggb);
            move(mv + 1, Gb, Ga, cpb, csb, ggb, cpa, csa, gga);
        }
        if (NO & 1) move(NO - 1, Ga, Gb, cpa, csa, gga, cpb, csb, ggb);
        chi2 += (double)dchi;
        accp = acc;
        nacc += acc;
        npos += pos;
        if (active && S.acc_trace && q == 0) S.acc_trace[(size_t)n * P.n_walkers + w] = acc;
    }
    // fold the common scale into the spectrum and write the walkers back
    if (active) {
        float *bg = S.b32 + (size_t)w * NO;
        for (int j = q; j < NO; j += MPD) {
            const float val = b[j];
            bg[j] = fmaf(glo, val, ghi * val);
        }
    }
#pragma unroll
    for (int c = 0; c < C; ++c)
#pragma unroll
        for (int j = 0; j < Q; ++j) {
            const float2 r2 = up(R[c][j]);
            const int i = lane + 32 * c;
            if (g0 + 2 * j < P.n_walkers) S.R32[(size_t)(g0 + 2 * j) * PAD + i] = r2.x;
            if (g0 + 2 * j + 1 < P.n_walkers) S.R32[(size_t)(g0 + 2 * j + 1) * PAD + i] = r2.y;
        }
    if (active && q == 0) {
        S.g2[2 * w] = 1.0f;
        S.g2[2 * w + 1] = 0.0f;
        S.chi2[w] = chi2;
        S.acc_prev[w] = accp;
        S.n_acc[w] += nacc;
        S.n_pos[w] += npos;
    }
}

// Threads a block: 16 warps for groups of 2 or 4 up to 8 chunks (128 registers a thread), else 8
// (the widest variants take up to 254); with more walker groups than that per SM the warps run
// in rounds.
template <int W, int C>
constexpr int shared_threads() { return W <= 4 && C <= 8 ? 512 : 256; }

template <int W, int C, int MODE>
__global__ void __launch_bounds__(shared_threads<W, C>()) sweep_shared_kernel(DevProblem P, DevState S, int n0, int n1,
                                                                        SweepGeom Gm) {
    extern __shared__ float4 smem4[];
    float *sm = reinterpret_cast<float *>(smem4);
    const int NO = P.n_omega, PAD = P.n_tau_pad, NH = (NO + 31) >> 5;
    float *sB = sm + (size_t)(NH + 32) * PAD + 2 * NO;   // staged spectra [W * groups_per_cta][NO]
    load_tables(P, sm);
    const int grp_lo = blockIdx.x * Gm.groups_per_cta;
    const int grp_hi = min(grp_lo + Gm.groups_per_cta, Gm.groups_total);
    const int walker_lo = W * grp_lo;
    const int walker_hi = min(W * grp_hi, P.n_walkers);
    if (Gm.stage_b) {
        const size_t n = (size_t)(walker_hi - walker_lo) * NO;
        const float *src = S.b32 + (size_t)walker_lo * NO;
        for (size_t k = threadIdx.x; k < n; k += blockDim.x) sB[k] = src[k];
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5;
    for (int round = 0; round < Gm.rounds; ++round) {
        const int grp = grp_lo + round * Gm.warps + warp;
        if (grp >= grp_hi) break;                         // uniform across the warp
        if (Gm.stage_b)
            run_shared<W, C, true, MODE>(P, S, n0, n1, grp, sm, sB, walker_lo);
        else
            run_shared<W, C, false, MODE>(P, S, n0, n1, grp, sm, nullptr, walker_lo);
    }
}

template <int W, int C, int MODE>
cudaError_t launch_shared_c(const DevProblem &P, const DevState &S, int n0, int n1, cudaStream_t st) {
    int dev = 0, sms = 0, smem_max = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    SweepGeom Gm;
    Gm.groups_total = (P.n_walkers + W - 1) / W;
    const int ctas = Gm.groups_total < sms ? Gm.groups_total : sms;
    Gm.groups_per_cta = (Gm.groups_total + ctas - 1) / ctas;
    constexpr int max_warps = shared_threads<W, C>() / 32;
    Gm.rounds = (Gm.groups_per_cta + max_warps - 1) / max_warps;
    Gm.warps = (Gm.groups_per_cta + Gm.rounds - 1) / Gm.rounds;
    const size_t tb = table_bytes(P);
    const size_t staged = (size_t)W * Gm.groups_per_cta * P.n_omega * 4;
    if (tb > (size_t)smem_max) return cudaErrorInvalidValue;
    Gm.stage_b = tb + staged <= (size_t)smem_max;
    const size_t smem = tb + (Gm.stage_b ? staged : 0);
    cudaError_t e = cudaFuncSetAttribute(sweep_shared_kernel<W, C, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    const int n_ctas = (Gm.groups_total + Gm.groups_per_cta - 1) / Gm.groups_per_cta;
    sweep_shared_kernel<W, C, MODE><<<n_ctas, Gm.warps * 32, smem, st>>>(P, S, n0, n1, Gm);
    return cudaGetLastError();
}

// The sweep for groups of W walkers at the problem's chunk count (up to 8 chunks for W = 8,
// 16 otherwise: the register budget).
template <int W, int MODE>
cudaError_t launch_shared_w(const DevProblem &P, const DevState &S, int n0, int n1, cudaStream_t st) {
    const int C = P.n_tau_pad / 32;
    switch (C) {
        case 1: return launch_shared_c<W, 1, MODE>(P, S, n0, n1, st);
        case 2: return launch_shared_c<W, 2, MODE>(P, S, n0, n1, st);
        case 3: return launch_shared_c<W, 3, MODE>(P, S, n0, n1, st);
        case 4: return launch_shared_c<W, 4, MODE>(P, S, n0, n1, st);
        case 5: return launch_shared_c<W, 5, MODE>(P, S, n0, n1, st);
        case 6: return launch_shared_c<W, 6, MODE>(P, S, n0, n1, st);
        case 7: return launch_shared_c<W, 7, MODE>(P, S, n0, n1, st);
        case 8: return launch_shared_c<W, 8, MODE>(P, S, n0, n1, st);
        default: break;
    }
    if constexpr (W <= 4) {
        switch (C) {
            case 9: return launch_shared_c<W, 9, MODE>(P, S, n0, n1, st);
            case 10: return launch_shared_c<W, 10, MODE>(P, S, n0, n1, st);
            case 11: return launch_shared_c<W, 11, MODE>(P, S, n0, n1, st);
            case 12: return launch_shared_c<W, 12, MODE>(P, S, n0, n1, st);
            case 13: return launch_shared_c<W, 13, MODE>(P, S, n0, n1, st);
            case 14: return launch_shared_c<W, 14, MODE>(P, S, n0, n1, st);
            case 15: return launch_shared_c<W, 15, MODE>(P, S, n0, n1, st);
            case 16: return launch_shared_c<W, 16, MODE>(P, S, n0, n1, st);
            default: break;
        }
    }
    return cudaErrorInvalidValue;
}

}  // namespace

}  // namespace sail
