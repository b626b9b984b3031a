// The FP32 production sweep (Sec. 2.2 moves, Eq. probability-density acceptance): the device
// code shared by the sweep translation units (sweep_fp32.cu: single-problem kernels and
// probes; sweep_walk.cu and sweep_hastings.cu: the kernels with an index walk and with the
// Hastings acceptance; sweep_batch8.cu and sweep_batch16.cu: batched kernels).  Two move loops:
// run_group takes one move at a time; run_group_ahead looks ahead over drawn proposals and
// spends the kernel columns on feasible moves only (the same draws and decisions; on a uniform
// tau grid with 8 lanes per walker the one-move loop forms its columns from the quad-compact
// tables, whose FP32 values differ from the full rows' in the last bits).
//
// Kernel columns from two small tables.  Eq. (efficient-correlation-model) writes the bin
// kernel as c_i q_i^j with q_i = e^{-dw tau_i}; so with j = 32 h + l,
//     Khat_ij = Khat_{i,32h} * q_i^l = Qhi[h][i] * Qlo[l][i],
// and the two tables ((N_omega/32 + 32) rows of n_tau_pad floats, 57 KB at 200 x 1000) sit in
// shared memory.  A move reads its two columns from there: no L2 traffic, no L2 latency.
//
// Walker layout.  One persistent block per SM; G lanes per walker (G = 8: four walkers a warp,
// for n_tau <= 256; G = 16: two), lane l of a walker's group holding R_i and M_i = Fhat_i - R_i
// for its 32 / G consecutive i of every 32-tau chunk.  Each lane of a group draws the random
// words of one move at a time (one Philox call per move: G consecutive moves, or one window of
// proposals, per round) and works out that move's scalars; the move loop takes them by shuffle
// within the group.  Delta chi2 =
// sum_i d_i (2 R_i + d_i) is reduced by an xor butterfly over the group.
//
// Spectrum.  a = g b: an accepted move multiplies the common scale g by r (an unevaluated
// pair of floats, error ~1e-14 over a launch) and writes only b_p and b_s.  When the block's
// spectra fit in shared memory next to the tables they are staged there for the launch.  The
// scale is folded back into b when the launch ends, so residual recomputation sees a = b.
#pragma once
#include <cmath>
#include <cstdint>

#include "moves.cuh"
#include "philox.cuh"
#include "sail_internal.cuh"

namespace sail {

namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kThreads = 512;          // at most 16 warps per round

// Move-loop variants, compiled separately so the plain loop carries no code of the others.
constexpr int kPlain = 0;              // uniform bins, Metropolis test (the paper's)
constexpr int kWalk = 1;               // bins from the index walk (Sec. 2.3)
constexpr int kHastings = 2;           // uniform bins, Metropolis-Hastings test with the Jacobian
constexpr int kGuard = 3;              // uniform bins, Metropolis test, decisions near the threshold
                                       // taken again in FP64

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
    int groups_total;     // walker groups (one warp each): ceil(n_walkers / walkers per warp)
    int groups_per_cta;
    int warps;            // warps per block
    int rounds;           // groups handled one after another by each warp
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

// Shared-memory layout of the sweep tables (float offsets).
//
// Full rows (16 lanes per walker, the look-ahead loop and the shared-bin kernels): the factor
// rows Qhi [NH][PAD] and Qlo [32][PAD].
//
// Quad-compact (the one-move loop with 8 lanes per walker, uniform tau grid, tau_i = tau_0 +
// i dtau).  Lane l of a walker
// holds the four consecutive points i0 + e (e < 4, i0 = 32 c + 4 l) of every chunk c, and along
// a uniform grid e^{-j dw tau_{i0+e}} = e^{-j dw tau_i0} X_j^e with X_j = e^{-j dw dtau}; so
//     Khat_{i0+e,j} = Qhi[j/32][i0] Qlo[j%32][i0] * X_j^e * rho_{i0+e},
// rho_i the ratio of Khat_{i,0} to Khat_{i0,0} (Eq. efficient-correlation-model applied along
// tau as well as omega).  A move then reads one factor value of each of its four rows per lane
// and chunk (4 bytes, not 16), the per-bin powers (1, X, X^2, X^3) once per column, and the lane's
// -rho quad once per chunk.  The compact rows keep the quad starts only (k = 8 c + l, pitch a
// multiple of 32 floats) and come in four copies, copy s offset by 8 s banks, so that the four
// walkers of a warp (walker s of the warp reads copy s) read four random rows in one
// conflict-free shared-memory access.  Measured: the one-move loop, which loads columns for
// every proposal, gains (uneven batch +8%, to-target anneals +2.5%); the look-ahead loop, which
// loads them for feasible moves only and waits on its chain rather than on shared memory, loses
// 2% to the extra instructions per chunk, and keeps the full rows.
struct TabLayout {
    int hi, lo, rho, x4, beta, rgap, total;
    int pitch;            // floats per row
    int cs_hi, cs_lo;     // floats per copy (quad-compact)
};
__host__ __device__ __forceinline__ TabLayout tab_layout(bool compact, int NO, int PAD) {
    const int NH = (NO + 31) >> 5;
    TabLayout T{};
    if (compact) {
        T.pitch = (8 * (PAD / 32) + 31) / 32 * 32;
        T.cs_hi = NH * T.pitch + 8;
        T.cs_lo = 32 * T.pitch + 8;
        T.hi = 0;
        T.lo = 4 * T.cs_hi;
        T.rho = T.lo + 4 * T.cs_lo;
        T.x4 = T.rho + PAD;
        T.beta = T.x4 + 4 * NO;
    } else {
        T.pitch = PAD;
        T.hi = 0;
        T.lo = NH * PAD;
        T.rho = T.x4 = 0;
        T.beta = T.lo + 32 * PAD;
    }
    T.rgap = T.beta + NO;
    T.total = T.rgap + NO;
    return T;
}

// Loads a problem's tables in the full-row or the quad-compact layout.
template <bool CT>
__device__ void load_tables_g(const DevProblem &P, float *sm) {
    if constexpr (!CT) {
        load_tables(P, sm);
    } else {
        const int NO = P.n_omega, PAD = P.n_tau_pad, NH = (NO + 31) >> 5;
        const TabLayout T = tab_layout(true, NO, PAD);
        const int used = 8 * (PAD / 32);           // quad starts per row
        for (int q = threadIdx.x; q < 4 * NH * T.pitch; q += blockDim.x) {
            const int cp = q / (NH * T.pitch), r = q % (NH * T.pitch), h = r / T.pitch, k = r % T.pitch;
            sm[T.hi + cp * T.cs_hi + r] = k < used ? P.Qhi32[(size_t)h * PAD + 4 * k] : 0.0f;
        }
        for (int q = threadIdx.x; q < 4 * 32 * T.pitch; q += blockDim.x) {
            const int cp = q / (32 * T.pitch), r = q % (32 * T.pitch), l = r / T.pitch, k = r % T.pitch;
            sm[T.lo + cp * T.cs_lo + r] = k < used ? P.Qlo32[(size_t)l * PAD + 4 * k] : 0.0f;
        }
        for (int q = threadIdx.x; q < PAD; q += blockDim.x) sm[T.rho + q] = P.mrho32[q];
        const float4 *x4 = reinterpret_cast<const float4 *>(P.x4_32);
        float4 *s4 = reinterpret_cast<float4 *>(sm + T.x4);
        for (int q = threadIdx.x; q < NO; q += blockDim.x) {
            s4[q] = x4[q];
            sm[T.beta + q] = P.beta32[q];
            sm[T.rgap + q] = P.rgap32[q];
        }
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

// One chunk of the four factor rows a move needs (Qhi and Qlo rows of bins p and s): a lane's
// E-float piece of each (shared-window addresses).
__device__ __forceinline__ void ld_chunk(uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, f2 (&v0)[1],
                                         f2 (&v1)[1], f2 (&v2)[1], f2 (&v3)[1]) {
    asm volatile("ld.shared.u64 %0, [%4];\n\tld.shared.u64 %1, [%5];\n\t"
                 "ld.shared.u64 %2, [%6];\n\tld.shared.u64 %3, [%7];"
                 : "=l"(v0[0]), "=l"(v1[0]), "=l"(v2[0]), "=l"(v3[0])
                 : "r"(a0), "r"(a1), "r"(a2), "r"(a3));
}
__device__ __forceinline__ void ld_chunk(uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3, f2 (&v0)[2],
                                         f2 (&v1)[2], f2 (&v2)[2], f2 (&v3)[2]) {
    asm volatile("ld.shared.v2.u64 {%0, %1}, [%8];\n\tld.shared.v2.u64 {%2, %3}, [%9];\n\t"
                 "ld.shared.v2.u64 {%4, %5}, [%10];\n\tld.shared.v2.u64 {%6, %7}, [%11];"
                 : "=l"(v0[0]), "=l"(v0[1]), "=l"(v1[0]), "=l"(v1[1]), "=l"(v2[0]), "=l"(v2[1]), "=l"(v3[0]),
                   "=l"(v3[1])
                 : "r"(a0), "r"(a1), "r"(a2), "r"(a3));
}

template <int G>
__device__ __forceinline__ float group_sum(float v) {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// The random words of one move (Philox counter (move, sweep, walker, 0)): bins p, s packed in
// one word, amplitude eps, Metropolis threshold -T ln u (u < exp(-D / T) <=> D < -T ln u) and
// delta_p, delta_s (Eqs. update-delta-p/s).
struct MoveDraw {
    int ps;
    float eps, thr, dp, ds;
};

// With an index walk (kWalk) the draw keeps p's start and s's start index on the other n - 1
// bins (not yet shifted past p) and leaves delta_p, delta_s to the move (the walk sets p, s).
//
// With the Hastings acceptance the threshold takes the move's Jacobian: D < -T ln u +
// T (N - 4) ln r, and a move whose reverse amplitude -eps/r cannot be proposed
// (|eps/r| >= y d) gets -infinity.
template <int MODE>
__device__ __forceinline__ MoveDraw draw_move(int mv, int n, int walker, uint2 key, int NO, float yd, float T,
                                              const float *beta, const float *rgap) {
    constexpr bool WALK = MODE == kWalk;
    const uint4 rnd = philox4x32_10(make_uint4((uint32_t)mv, (uint32_t)n, (uint32_t)walker, 0u), key);
    MoveDraw m;
    m.eps = yd * (2.0f * unit32(rnd.z) - 1.0f);
    m.thr = -logf(unit32(rnd.w)) * T;
    if constexpr (MODE == kHastings) {
        const float r = 1.0f - m.eps;
        m.thr = fabsf(m.eps / r) < yd ? m.thr + T * (float)(NO - 4) * log1pf(-m.eps) : -INFINITY;
    }
    if constexpr (WALK) {
        m.ps = (int)(((uint64_t)rnd.x * (uint64_t)NO) >> 32) | ((int)(((uint64_t)rnd.y * (uint64_t)(NO - 1)) >> 32) << 16);
        m.dp = m.ds = 0.0f;
    } else {
        int p, s;
        move_bins(rnd.x, rnd.y, NO, p, s);
        m.ps = p | (s << 16);
        deltas(m.eps, p, s, beta, rgap, m.dp, m.ds);
    }
    return m;
}

__device__ __forceinline__ MoveDraw take_move(const MoveDraw &mine, int src, int width) {
    MoveDraw m;
    m.ps = __shfl_sync(kFull, mine.ps, src, width);
    m.eps = __shfl_sync(kFull, mine.eps, src, width);
    m.thr = __shfl_sync(kFull, mine.thr, src, width);
    m.dp = __shfl_sync(kFull, mine.dp, src, width);
    m.ds = __shfl_sync(kFull, mine.ds, src, width);
    return m;
}

// Shared-window addresses of a lane's piece of chunk 0 of the four factor rows of a move.
struct RowAddr {
    uint32_t hp, lp, hs, ls;
};
__device__ __forceinline__ RowAddr row_addr(int ps, uint32_t qhi, uint32_t qlo, int PAD) {
    const int p = ps & 0xFFFF, s = ps >> 16;
    RowAddr a;
    a.hp = qhi + 4u * (uint32_t)((p >> 5) * PAD);
    a.lp = qlo + 4u * (uint32_t)((p & 31) * PAD);
    a.hs = qhi + 4u * (uint32_t)((s >> 5) * PAD);
    a.ls = qlo + 4u * (uint32_t)((s & 31) * PAD);
    return a;
}

// A lane's view of the sweep tables (shared-window addresses): its piece of chunk 0 of row 0
// of the hi and lo tables (quad-compact, CT: in its walker's copy), its -rho quad of chunk 0
// and the per-bin powers (CT), and the row pitch in floats.
struct ColTab {
    uint32_t hi, lo, rho, x4;
    int pitch;
};
template <int G, bool CT>
__device__ __forceinline__ ColTab col_tab(const TabLayout &T, const float *sm, int gl, int sub) {
    static_assert(!CT || G == 8, "the quad-compact tables serve 8 lanes per walker");
    const uint32_t base = (uint32_t)__cvta_generic_to_shared(sm);
    ColTab t;
    t.pitch = T.pitch;
    if constexpr (CT) {
        t.hi = base + 4u * (uint32_t)(T.hi + sub * T.cs_hi + gl);
        t.lo = base + 4u * (uint32_t)(T.lo + sub * T.cs_lo + gl);
        t.rho = base + 4u * (uint32_t)(T.rho + 4 * gl);
        t.x4 = base + 4u * (uint32_t)T.x4;
    } else {
        t.hi = base + 4u * (uint32_t)(T.hi + (32 / G) * gl);
        t.lo = base + 4u * (uint32_t)(T.lo + (32 / G) * gl);
        t.rho = t.x4 = 0u;
    }
    return t;
}

__device__ __forceinline__ float lds1(uint32_t a) {
    float v;
    asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ float4 lds4(uint32_t a) {
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a));
    return v;
}

// dpart = -delta_p Khat_p - delta_s Khat_s over the lane's elements.  Full rows: each column
// element the product of its two factor rows (Eq. efficient-correlation-model).  Quad-compact
// (CT): per chunk u = delta_p Qhi Qlo at the lane's quad start of p (v likewise for s), then
// element e of the quad is -rho_e (u X_p^e + v X_s^e).
template <int G, int C>
__device__ __forceinline__ void columns(f2 (&dpart)[C][32 / G / 2], uint32_t qhi, uint32_t qlo, int PAD,
                                        const MoveDraw &m) {
    constexpr int H = 32 / G / 2;
    const RowAddr a = row_addr(m.ps, qhi, qlo, PAD);
    const f2 mdp = pk(-m.dp, -m.dp), mds = pk(-m.ds, -m.ds);
#pragma unroll
    for (int c = 0; c < C; ++c) {
        f2 hp[H], lp[H], hs[H], ls[H];
        ld_chunk(a.hp + 128u * c, a.lp + 128u * c, a.hs + 128u * c, a.ls + 128u * c, hp, lp, hs, ls);
#pragma unroll
        for (int h = 0; h < H; ++h) dpart[c][h] = fma2(mds, mul2(hs[h], ls[h]), mul2(mdp, mul2(hp[h], lp[h])));
    }
}
template <int G, int C, bool CT>
__device__ __forceinline__ void columns_tab(f2 (&dpart)[C][32 / G / 2], const ColTab &t, const MoveDraw &m) {
    if constexpr (CT) {
        const int p = m.ps & 0xFFFF, s = m.ps >> 16;
        const uint32_t hp = t.hi + 4u * (uint32_t)((p >> 5) * t.pitch), lp = t.lo + 4u * (uint32_t)((p & 31) * t.pitch);
        const uint32_t hs = t.hi + 4u * (uint32_t)((s >> 5) * t.pitch), ls = t.lo + 4u * (uint32_t)((s & 31) * t.pitch);
        const float4 xp = lds4(t.x4 + 16u * (uint32_t)p), xs = lds4(t.x4 + 16u * (uint32_t)s);
        const f2 xp01 = pk(xp.x, xp.y), xp23 = pk(xp.z, xp.w), xs01 = pk(xs.x, xs.y), xs23 = pk(xs.z, xs.w);
        const f2 dps = pk(m.dp, m.ds);
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const float vhp = lds1(hp + 32u * c), vlp = lds1(lp + 32u * c);
            const float vhs = lds1(hs + 32u * c), vls = lds1(ls + 32u * c);
            const float4 mr = lds4(t.rho + 128u * c);
            const float2 uv = up(mul2(mul2(pk(vhp, vhs), pk(vlp, vls)), dps));
            const f2 u2 = pk(uv.x, uv.x), v2 = pk(uv.y, uv.y);
            dpart[c][0] = mul2(pk(mr.x, mr.y), fma2(v2, xs01, mul2(u2, xp01)));
            dpart[c][1] = mul2(pk(mr.z, mr.w), fma2(v2, xs23, mul2(u2, xp23)));
        }
    } else {
        columns<G, C>(dpart, t.hi, t.lo, t.pitch, m);
    }
}

// A lane's part of delta chi2 = sum_i d_i (2 R_i + d_i), two interleaved accumulators.
template <int C, int H>
__device__ __forceinline__ float delta_sum(const f2 (&d)[C][H], const f2 (&R)[C][H], f2 two) {
    f2 part0 = 0ull, part1 = 0ull;
#pragma unroll
    for (int c = 0; c < C; ++c)
#pragma unroll
        for (int h = 0; h < H; ++h) {
            if ((c * H + h) & 1)
                part1 = fma2(d[c][h], fma2(two, R[c][h], d[c][h]), part1);
            else
                part0 = fma2(d[c][h], fma2(two, R[c][h], d[c][h]), part0);
        }
    const float2 pp = up(add2(part0, part1));
    return pp.x + pp.y;
}

// The same sum with the magnitude of its terms, S = sum_i |d_i| |2 R_i + d_i| (the lane's parts):
// the Delta chi2 part is formed by the same operations as delta_sum, so it rounds the same.
__device__ __forceinline__ f2 abs2(f2 v) {
    f2 r;
    asm("and.b64 %0, %1, 0x7FFFFFFF7FFFFFFF;" : "=l"(r) : "l"(v));
    return r;
}
template <int C, int H>
__device__ __forceinline__ void delta_sum_mag(const f2 (&d)[C][H], const f2 (&R)[C][H], f2 two, float &D, float &S) {
    f2 part0 = 0ull, part1 = 0ull, mag = 0ull;
#pragma unroll
    for (int c = 0; c < C; ++c)
#pragma unroll
        for (int h = 0; h < H; ++h) {
            const f2 t = fma2(two, R[c][h], d[c][h]);
            if ((c * H + h) & 1)
                part1 = fma2(d[c][h], t, part1);
            else
                part0 = fma2(d[c][h], t, part0);
            mag = fma2(abs2(d[c][h]), abs2(t), mag);
        }
    const float2 pp = up(add2(part0, part1)), mm = up(mag);
    D = pp.x + pp.y;
    S = mm.x + mm.y;
}

// Delta chi2 of move m in FP64 on the walker's FP32 state (Sec. 2.2): the lane's elements of
// sum_i d_i (2 R_i + d_i), d_i = eps M_i - delta_p Khat_ip - delta_s Khat_is, each kernel column
// element the FP64 product of its FP32 factors (full rows: the two factor rows, exact;
// quad-compact: the two quad-start factors, X^e and rho_e), summed in FP64 over the walker's G
// lanes.  Every lane of the warp calls it (the butterfly is warp-wide).
template <int G, int C, bool CT>
__device__ __forceinline__ double delta_chi2_fp64(const f2 (&R)[C][32 / G / 2], const f2 (&M)[C][32 / G / 2],
                                                  const ColTab &t, const MoveDraw &m) {
    constexpr int H = 32 / G / 2;
    const double eps = (double)m.eps, dp = (double)m.dp, ds = (double)m.ds;
    double part = 0.0;
    if constexpr (CT) {
        const int p = m.ps & 0xFFFF, s = m.ps >> 16;
        const uint32_t hp = t.hi + 4u * (uint32_t)((p >> 5) * t.pitch), lp = t.lo + 4u * (uint32_t)((p & 31) * t.pitch);
        const uint32_t hs = t.hi + 4u * (uint32_t)((s >> 5) * t.pitch), ls = t.lo + 4u * (uint32_t)((s & 31) * t.pitch);
        const float4 xp4 = lds4(t.x4 + 16u * (uint32_t)p), xs4 = lds4(t.x4 + 16u * (uint32_t)s);
        const double xp[4] = {xp4.x, xp4.y, xp4.z, xp4.w}, xs[4] = {xs4.x, xs4.y, xs4.z, xs4.w};
#pragma unroll
        for (int c = 0; c < C; ++c) {
            const double bp = (double)lds1(hp + 32u * c) * (double)lds1(lp + 32u * c);
            const double bs = (double)lds1(hs + 32u * c) * (double)lds1(ls + 32u * c);
            const float4 mr4 = lds4(t.rho + 128u * c);
            const double rho[4] = {-(double)mr4.x, -(double)mr4.y, -(double)mr4.z, -(double)mr4.w};
#pragma unroll
            for (int h = 0; h < H; ++h) {
                const float2 r = up(R[c][h]), mm = up(M[c][h]);
                const int e = 2 * h;
                const double d0 = eps * (double)mm.x - dp * (bp * xp[e] * rho[e]) - ds * (bs * xs[e] * rho[e]);
                const double d1 = eps * (double)mm.y - dp * (bp * xp[e + 1] * rho[e + 1]) - ds * (bs * xs[e + 1] * rho[e + 1]);
                part += d0 * (2.0 * (double)r.x + d0);
                part += d1 * (2.0 * (double)r.y + d1);
            }
        }
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) part += __shfl_xor_sync(kFull, part, o, G);
        return part;
    }
    const RowAddr a = row_addr(m.ps, t.hi, t.lo, t.pitch);
#pragma unroll
    for (int c = 0; c < C; ++c) {
        f2 hp[H], lp[H], hs[H], ls[H];
        ld_chunk(a.hp + 128u * c, a.lp + 128u * c, a.hs + 128u * c, a.ls + 128u * c, hp, lp, hs, ls);
#pragma unroll
        for (int h = 0; h < H; ++h) {
            const float2 Hp = up(hp[h]), Lp = up(lp[h]), Hs = up(hs[h]), Ls = up(ls[h]);
            const float2 r = up(R[c][h]), mm = up(M[c][h]);
            const double kp0 = (double)Hp.x * (double)Lp.x, ks0 = (double)Hs.x * (double)Ls.x;
            const double kp1 = (double)Hp.y * (double)Lp.y, ks1 = (double)Hs.y * (double)Ls.y;
            const double d0 = eps * (double)mm.x - dp * kp0 - ds * ks0;
            const double d1 = eps * (double)mm.y - dp * kp1 - ds * ks1;
            part += d0 * (2.0 * (double)r.x + d0);
            part += d1 * (2.0 * (double)r.y + d1);
        }
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) part += __shfl_xor_sync(kFull, part, o, G);
    return part;
}

// The Metropolis decision of a feasible move with the FP64 guard (kGuard): the FP32 decision
// stands unless its Delta chi2 D lies within 1e-5 S of the threshold or of 0 (or every decision
// is to be checked, fp64_accept = 2); then Delta chi2 is evaluated in FP64 on the same state and
// decides, and D takes its value.  n_re and n_flip count the decisions taken again and those
// that changed.  Warp-uniform entry (every lane calls it).
template <int G, int C, bool CT>
__device__ __forceinline__ bool guarded_accept(bool live, float &D, float S, float thr, int mode,
                                               const f2 (&R)[C][32 / G / 2], const f2 (&M)[C][32 / G / 2],
                                               const ColTab &tab, const MoveDraw &m,
                                               unsigned &n_re, unsigned &n_flip) {
    bool acc = live && (D <= 0.0f || D < thr);
    const float band = 1e-5f * S;
    const bool near = live && (mode == 2 || fabsf(D - thr) <= band || fabsf(D) <= band);
    if (__any_sync(kFull, near)) {
        const double D64 = delta_chi2_fp64<G, C, CT>(R, M, tab, m);
        if (near) {
            const bool acc64 = D64 <= 0.0 || D64 < (double)thr;
            n_re += 1;
            n_flip += acc64 != acc;
            acc = acc64;
            D = (float)D64;
        }
    }
    return acc;
}

// Sweeps [n0, n1) for the 32 / G walkers of group grp of one problem on one warp, G lanes per
// walker.  Lane l of a walker's G lanes holds R_i and M_i = Fhat_i - R_i for
// i = 32 c + E l .. 32 c + E l + E - 1 (E = 32 / G floats of every 32-tau chunk c) and reads the
// same E-float pieces of the kernel factor rows, so the G lanes of one walker cover a chunk
// with one 128-byte shared-memory access.  sm holds the problem's tables; b_stage, if not null,
// the staged spectra of walkers walker_lo.. .
//
// Every G moves each lane draws the random words of one move; the move loop takes them by
// shuffle.  The loop is software-pipelined: while move k's delta chi2 is reduced and tested,
// the warp already loads move k+1's kernel columns and forms the part of its residual change
// that does not depend on move k, dpart = -delta_p Khat_p - delta_s Khat_s; when move k+1 is
// evaluated, d = eps M + dpart (for n_tau > 256 the columns are loaded when the move is
// evaluated: the pipeline's registers do not fit).  Columns are loaded for every walker, also
// those whose move then fails the positivity test: with few warps per SM the sweep is bound by
// the latency of each warp's instruction stream more than by shared-memory bandwidth.
//
// BA (uniform bins only): each move's b_p, b_s are read one move ahead, during the move before
// it, and patched if that move wrote one of those bins.  The batched kernel's plain loop, whose
// spectra stay in global memory, takes this (measured +6% on uneven batches); the
// single-problem kernel reads b when the move is evaluated (the early read measured 0.5% slower
// with staged spectra and 6% slower at 512 tau, where the columns are not pipelined).
template <int G, int C, bool STAGED, int MODE, bool BA = false>
__device__ __forceinline__ void run_group(const DevProblem &P, const DevState &S, int n0, int n1, int grp,
                                          const float *sm,
                          float *b_stage, int walker_lo) {
    constexpr int E = 32 / G;          // floats of a 32-tau chunk per lane
    constexpr int H = E / 2;           // float pairs of a chunk per lane
    constexpr int WPW = 32 / G;        // walkers per warp
    // the pipelined loop holds four arrays of C H float pairs (R, M, d and the next move's
    // dpart); past 8 chunks that outgrows the registers, and the columns of a move are loaded
    // when it is evaluated
    constexpr bool WALK = MODE == kWalk;
    constexpr bool PIPE = C <= 8 && !WALK;
    constexpr bool BAHEAD = BA && !WALK;   // b read one move ahead (above)
    const int NO = P.n_omega, PAD = P.n_tau_pad;
    constexpr bool CT = G == 8;       // quad-compact tables with 8 lanes per walker
    const TabLayout TL = tab_layout(CT, NO, PAD);
    const float *sBeta = sm + TL.beta;
    const float *sRgap = sm + TL.rgap;
    const int lane = threadIdx.x & 31, gl = lane & (G - 1), sub = lane / G;
    const ColTab tab = col_tab<G, CT>(TL, sm, gl, sub);
    const uint2 key = philox_key(P.seed);
    const double dmove = P.move_scale > 0.0 ? P.move_scale : 1.0 / NO;
    const float rho = (float)P.walk_rho;

    const int w = WPW * grp + sub;
    const bool active = w < P.n_walkers;
    const int wr = active ? w : WPW * grp;            // a valid walker to read from
    float *b = STAGED ? b_stage + (size_t)(wr - walker_lo) * NO : S.b32 + (size_t)wr * NO;
    // the walker's spectrum b: shared memory when staged, else global memory
    const uint32_t bsh = STAGED ? (uint32_t)__cvta_generic_to_shared(b) : 0u;
    auto bget = [&](int j) -> float {
        if constexpr (STAGED) {
            float v;
            asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(bsh + 4u * (uint32_t)j));
            return v;
        } else {
            return b[j];
        }
    };
    auto bset = [&](int j, float v) {
        if constexpr (STAGED)
            asm volatile("st.shared.f32 [%0], %1;" ::"r"(bsh + 4u * (uint32_t)j), "f"(v) : "memory");
        else
            b[j] = v;
    };

    f2 R[C][H], M[C][H];
#pragma unroll
    for (int c = 0; c < C; ++c) {
#pragma unroll
        for (int h = 0; h < H; ++h) {
            const int i = 32 * c + E * gl + 2 * h;
            const float2 r2 = *reinterpret_cast<const float2 *>(S.R32 + (size_t)wr * PAD + i);
            const float2 f2v = *reinterpret_cast<const float2 *>(P.Fhat32 + i);
            R[c][h] = pk(r2.x, r2.y);
            M[c][h] = pk(f2v.x - r2.x, f2v.y - r2.y);
        }
    }
    float ghi = S.g2[2 * wr], glo = S.g2[2 * wr + 1];
    double chi2 = S.chi2[wr];
    int accp = S.acc_prev[wr];
    unsigned long long nacc = 0, npos = 0;
    unsigned n_re = 0, n_flip = 0;     // kGuard: decisions taken again in FP64, and changed
    const f2 two = pk(2.0f, 2.0f), minus_one = pk(-1.0f, -1.0f);

    for (int n = n0; n < n1; ++n) {
        const float T = (float)P.Tsweep[n];
        const float yd = (float)(amplitude(accp, NO, P.y_p, P.y_m, P.y_min) * dmove);
        int acc = 0, pos = 0;
        float dchi = 0.0f;
        MoveDraw mine = draw_move<MODE>(gl, n, wr + P.walker_base, key, NO, yd, T, sBeta, sRgap);
        MoveDraw cur = take_move(mine, 0, G);
        f2 dcur[PIPE ? C : 1][H];
        if constexpr (PIPE) columns_tab<G, C, CT>(dcur, tab, cur);
        // b at the current move's bins, read one move ahead (BAHEAD, see below)
        float bpc = 0.0f, bsc = 0.0f;
        if constexpr (BAHEAD) {
            bpc = bget(cur.ps & 0xFFFF);
            bsc = bget(cur.ps >> 16);
        }
        for (int mv = 0; mv < NO; ++mv) {
            if constexpr (WALK) {
                // the index walk (Sec. 2.3) on the spectrum as it is now: lane t of the group
                // draws step t + 1's words (counter (mv, n, w, 2 + t)), lane L the admixture's
                const int L = P.walk_len;
                const uint4 wr4 = philox4x32_10(make_uint4((uint32_t)mv, (uint32_t)n, (uint32_t)(wr + P.walker_base), 2u + gl), key);
                const bool walk_p = !(unit32(__shfl_sync(kFull, wr4.x, L, G)) < rho);
                const bool walk_s = !(unit32(__shfl_sync(kFull, wr4.y, L, G)) < rho);
                int wp = cur.ps & 0xFFFF;
                float bp = bget(wp);
                for (int t = 0; t < L; ++t) {
                    const uint32_t xj = __shfl_sync(kFull, wr4.x, t, G), xu = __shfl_sync(kFull, wr4.y, t, G);
                    const int j = (int)(((uint64_t)xj * (uint64_t)NO) >> 32);
                    const float bj = bget(j);
                    if (walk_p && unit32(xu) * bp <= bj) {
                        wp = j;
                        bp = bj;
                    }
                }
                int ws = cur.ps >> 16;
                ws += (ws >= wp);
                float bs = bget(ws);
                for (int t = 0; t < L; ++t) {
                    const uint32_t xj = __shfl_sync(kFull, wr4.z, t, G), xu = __shfl_sync(kFull, wr4.w, t, G);
                    int j = (int)(((uint64_t)xj * (uint64_t)(NO - 1)) >> 32);
                    j += (j >= wp);
                    const float bj = bget(j);
                    if (walk_s && unit32(xu) * bs <= bj) {
                        ws = j;
                        bs = bj;
                    }
                }
                cur.ps = wp | (ws << 16);
                deltas(cur.eps, wp, ws, sBeta, sRgap, cur.dp, cur.ds);
            }
            // BAHEAD: move k+1's words (they do not depend on move k's outcome) and its b
            // values, read now so that their latency overlaps move k; if move k is accepted
            // and writes one of those bins, the written value replaces the one read (the value
            // a read after the write returns).  nxt's bins are valid indices also past the
            // sweep's last move.
            MoveDraw nxt;
            float bpn = 0.0f, bsn = 0.0f;
            if constexpr (BAHEAD) {
                nxt = take_move(mine, (mv + 1) & (G - 1), G);
                bpn = bget(nxt.ps & 0xFFFF);
                bsn = bget(nxt.ps >> 16);
            }
            // move k: positivity (Eq. probability-density) on the spectrum as it is now
            const int p = cur.ps & 0xFFFF, s = cur.ps >> 16;
            const float r = 1.0f - cur.eps;
            float bp, bs;
            if constexpr (BAHEAD) {
                bp = bpc;
                bs = bsc;
            } else {
                bp = bget(p);
                bs = bget(s);
            }
            const float ap = fmaf(r, ghi * bp, cur.dp);
            const float as = fmaf(r, ghi * bs, cur.ds);
            const bool ok = active && ap >= 0.0f && as >= 0.0f;
            pos += (active && !ok);
            // move k: residual change d = eps M + dpart
            const f2 e2 = pk(cur.eps, cur.eps);
            f2 d[C][H];
            if constexpr (PIPE) {
#pragma unroll
                for (int c = 0; c < C; ++c)
#pragma unroll
                    for (int h = 0; h < H; ++h) d[c][h] = fma2(e2, M[c][h], dcur[c][h]);
            } else {
                columns_tab<G, C, CT>(d, tab, cur);
#pragma unroll
                for (int c = 0; c < C; ++c)
#pragma unroll
                    for (int h = 0; h < H; ++h) d[c][h] = fma2(e2, M[c][h], d[c][h]);
            }
            // move k+1: its words (unless taken above) and (pipelined) its columns, into dcur,
            // now free; neither depends on move k's outcome
            if constexpr (!BAHEAD) nxt = take_move(mine, (mv + 1) & (G - 1), G);
            if constexpr (PIPE) columns_tab<G, C, CT>(dcur, tab, nxt);
            // move k: delta chi2 = sum d (2 R + d) and the Metropolis test
            float D;
            bool acc_k;
            if constexpr (MODE == kGuard) {
                float Dp, Sp;
                delta_sum_mag<C, H>(d, R, two, Dp, Sp);
                D = group_sum<G>(Dp);
                acc_k = guarded_accept<G, C, CT>(ok, D, group_sum<G>(Sp), cur.thr, P.fp64_accept, R, M, tab, cur,
                                             n_re, n_flip);
            } else {
                D = group_sum<G>(delta_sum<C, H>(d, R, two));
                // the Hastings threshold may be negative: then D <= 0 does not pass by itself
                acc_k = ok && (MODE == kHastings ? D < cur.thr : (D <= 0.0f || D < cur.thr));
            }
            if (acc_k) {
#pragma unroll
                for (int c = 0; c < C; ++c) {
#pragma unroll
                    for (int h = 0; h < H; ++h) {
                        R[c][h] = add2(R[c][h], d[c][h]);
                        M[c][h] = fma2(minus_one, d[c][h], M[c][h]);
                    }
                }
                pair_scale(ghi, glo, r);
                if constexpr (BAHEAD) {
                    const float inv_g = 1.0f / ghi;
                    const float bp_new = ap * inv_g, bs_new = as * inv_g;
                    if (gl == 0) {
                        bset(p, bp_new);
                        bset(s, bs_new);
                    }
                    const int pn = nxt.ps & 0xFFFF, sn = nxt.ps >> 16;
                    bpn = pn == p ? bp_new : (pn == s ? bs_new : bpn);
                    bsn = sn == p ? bp_new : (sn == s ? bs_new : bsn);
                } else if (gl == 0) {
                    const float inv_g = 1.0f / ghi;
                    bset(p, ap * inv_g);
                    bset(s, as * inv_g);
                }
                dchi += D;
                ++acc;
            }
            __syncwarp();
            cur = nxt;
            if constexpr (BAHEAD) {
                bpc = bpn;
                bsc = bsn;
            }
            // the next batch of G moves, one per lane, before its first move is taken
            if (((mv + 2) & (G - 1)) == 0 && mv + 2 < NO)
                mine = draw_move<MODE>(mv + 2 + gl, n, wr + P.walker_base, key, NO, yd, T, sBeta, sRgap);
        }
        chi2 += (double)dchi;
        accp = acc;
        nacc += acc;
        npos += pos;
        if (active && S.acc_trace && gl == 0) S.acc_trace[(size_t)n * P.n_walkers + w] = acc;
    }
    if (!active) return;
    // fold the common scale into the spectrum and write the walker back
    float *bg = S.b32 + (size_t)w * NO;
    for (int j = gl; j < NO; j += G) {
        const float v = b[j];
        bg[j] = fmaf(glo, v, ghi * v);
    }
#pragma unroll
    for (int c = 0; c < C; ++c)
#pragma unroll
        for (int h = 0; h < H; ++h)
            *reinterpret_cast<float2 *>(S.R32 + (size_t)w * PAD + 32 * c + E * gl + 2 * h) = up(R[c][h]);
    if (gl == 0) {
        S.g2[2 * w] = 1.0f;
        S.g2[2 * w + 1] = 0.0f;
        S.chi2[w] = chi2;
        S.acc_prev[w] = accp;
        S.n_acc[w] += nacc;
        S.n_pos[w] += npos;
        if constexpr (MODE == kGuard) {
            if (n_re) atomicAdd(&S.guard[0], (unsigned long long)n_re);
            if (n_flip) atomicAdd(&S.guard[1], (unsigned long long)n_flip);
        }
    }
}

// The look-ahead move loop, for uniform bins (the plain and the Hastings variants).
//
// A proposal that would make an amplitude negative, or (Hastings) whose reverse move cannot be
// proposed, is rejected before its kernel columns matter: about 40% of the moves at paper
// scale.  A move's bins, amplitude and threshold do not depend on the spectrum; its
// feasibility does, through b_p, b_s and the scale g only.  So each walker keeps its next 2G
// proposals drawn (lane l of its group holds proposals wb + l, window A, and wb + G + l,
// window B), tests all of them at once against the spectrum, takes the first feasible one by a
// ballot, counts the infeasible ones before it as rejected moves, and spends columns, reduction
// and Metropolis test on feasible moves only.  The chain is the sequential one move for move:
// the same draws, decisions and arithmetic, in the same order.
//
// The walkers of a warp run through their sweeps independently (each has its own move index
// and sweep); the warp loops until all have finished.  Pipelining: while move k's delta chi2 is
// reduced, the later proposals' feasibility is evaluated for both outcomes of move k and the
// columns of the first proposal feasible if move k is rejected are loaded; after the test the
// outcome picks the flags, and if they name another move (acceptance changed a feasibility,
// rarely), its columns are loaded then.
template <int G, int C, bool STAGED, int MODE>
__device__ __forceinline__ void run_group_ahead(const DevProblem &P, const DevState &S, int n0, int n1, int grp,
                                                const float *sm, float *b_stage, int walker_lo) {
    static_assert(MODE != kWalk, "the index walk chooses its bins from the spectrum: run_group");
    constexpr int E = 32 / G;          // floats of a 32-tau chunk per lane
    constexpr int H = E / 2;           // float pairs of a chunk per lane
    constexpr int WPW = 32 / G;        // walkers per warp
    constexpr bool PIPE = C <= 8;      // registers for the prefetched columns (see run_group)
    // full factor rows (see TabLayout)
    const int NO = P.n_omega, PAD = P.n_tau_pad, NH = (NO + 31) >> 5;
    const float *sQhi = sm;
    const float *sQlo = sQhi + (size_t)NH * PAD;
    const float *sBeta = sQlo + (size_t)32 * PAD;
    const float *sRgap = sBeta + NO;
    const int lane = threadIdx.x & 31, gl = lane & (G - 1), sub = lane / G;
    const uint32_t qhi = (uint32_t)__cvta_generic_to_shared(sQhi) + 4u * E * gl;
    const uint32_t qlo = (uint32_t)__cvta_generic_to_shared(sQlo) + 4u * E * gl;
    const uint2 key = philox_key(P.seed);
    const double dmove = P.move_scale > 0.0 ? P.move_scale : 1.0 / NO;

    const int w = WPW * grp + sub;
    const bool active = w < P.n_walkers;
    const int wr = active ? w : WPW * grp;            // a valid walker to read from
    float *b = STAGED ? b_stage + (size_t)(wr - walker_lo) * NO : S.b32 + (size_t)wr * NO;
    const uint32_t bsh = STAGED ? (uint32_t)__cvta_generic_to_shared(b) : 0u;
    auto bget = [&](int j) -> float {
        if constexpr (STAGED) {
            float v;
            asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(bsh + 4u * (uint32_t)j));
            return v;
        } else {
            return b[j];
        }
    };
    auto bset = [&](int j, float v) {
        if constexpr (STAGED)
            asm volatile("st.shared.f32 [%0], %1;" ::"r"(bsh + 4u * (uint32_t)j), "f"(v) : "memory");
        else
            b[j] = v;
    };

    f2 R[C][H], M[C][H];
#pragma unroll
    for (int c = 0; c < C; ++c) {
#pragma unroll
        for (int h = 0; h < H; ++h) {
            const int i = 32 * c + E * gl + 2 * h;
            const float2 r2 = *reinterpret_cast<const float2 *>(S.R32 + (size_t)wr * PAD + i);
            const float2 f2v = *reinterpret_cast<const float2 *>(P.Fhat32 + i);
            R[c][h] = pk(r2.x, r2.y);
            M[c][h] = pk(f2v.x - r2.x, f2v.y - r2.y);
        }
    }
    float ghi = S.g2[2 * wr], glo = S.g2[2 * wr + 1];
    double chi2 = S.chi2[wr];
    int accp = S.acc_prev[wr];
    unsigned nacc = 0, npos = 0;       // this launch's accepted and positivity-rejected moves
    unsigned n_re = 0, n_flip = 0;     // kGuard: decisions taken again in FP64, and changed
    const f2 two = pk(2.0f, 2.0f), minus_one = pk(-1.0f, -1.0f);

    // the walker's sweep (the same in all G lanes of its group)
    int n = n0;
    bool done = !active || n0 >= n1;
    float T = 0.0f, yd = 0.0f, dchi = 0.0f;
    int acc = 0, pos = 0;
    int wb = 0;                        // window A = proposals [wb, wb + G), B = [wb + G, wb + 2G)
    int lo = 0;                        // the first proposal not yet consumed
    MoveDraw pa, pb;                   // this lane's proposals wb + gl and wb + G + gl
    pa.ps = pb.ps = 1 << 16;           // valid bins for walkers that draw nothing
    pa.eps = pb.eps = pa.thr = pb.thr = pa.dp = pb.dp = pa.ds = pb.ds = 0.0f;
    auto start_sweep = [&]() {
        T = (float)P.Tsweep[n];
        yd = (float)(amplitude(accp, NO, P.y_p, P.y_m, P.y_min) * dmove);
        acc = pos = 0;
        dchi = 0.0f;
        wb = lo = 0;
        pa = draw_move<MODE>(gl, n, wr + P.walker_base, key, NO, yd, T, sBeta, sRgap);
        pb = draw_move<MODE>(G + gl, n, wr + P.walker_base, key, NO, yd, T, sBeta, sRgap);
    };
    // slide the windows by G once the current move lies in window B
    auto slide = [&]() {
        pa = pb;
        wb += G;
        pb = draw_move<MODE>(wb + G + gl, n, wr + P.walker_base, key, NO, yd, T, sBeta, sRgap);
    };
    if (!done) start_sweep();

    const int base = sub * G;
    const uint32_t lowG = G == 32 ? kFull : (1u << G) - 1u;
    // bit t of the result: proposal wb + t of this lane's walker (A's lanes, then B's)
    auto group_bits = [&](bool in_a, bool in_b) -> uint32_t {
        const uint32_t ba = (__ballot_sync(kFull, in_a) >> base) & lowG;
        const uint32_t bb = (__ballot_sync(kFull, in_b) >> base) & lowG;
        return ba | (bb << G);
    };
    auto below = [](int t) -> uint32_t { return t >= 32 ? kFull : (1u << t) - 1u; };
    // positivity rejections among the proposals from lo up to bit t (t < 0: all the windows');
    // a plain move is infeasible only by positivity, so there the count is the skipped span
    auto count_pos = [&](uint32_t pfm, int t) -> int {
        if constexpr (MODE == kHastings) return __popc(pfm & below(t < 0 ? 2 * G : t));
        else return max(0, min(wb + (t < 0 ? 2 * G : t), NO) - lo);
    };
    // proposal wb + t, from the lane that holds it (t >= 0; every lane calls)
    auto take_bit = [&](int t) -> MoveDraw { return take_move(t < G ? pa : pb, t & (G - 1), G); };
    // feasibility of proposal q (number idx) on the spectrum as it is now
    auto feasible_now = [&](const MoveDraw &q, int idx, bool live, bool &ok, bool &pf) {
        const bool valid = live && idx >= lo && idx < NO;
        const int qp = q.ps & 0xFFFF, qs = q.ps >> 16;
        const float rq = 1.0f - q.eps;
        const float ap = fmaf(rq, ghi * bget(qp), q.dp), as = fmaf(rq, ghi * bget(qs), q.ds);
        const bool posok = ap >= 0.0f && as >= 0.0f;
        const bool hok = MODE != kHastings || q.thr > -INFINITY;
        ok = valid && posok && hok;
        pf = valid && !posok;
    };

    MoveDraw cur = pa;                 // the move evaluated next: feasible, proposal number icur
    int icur = 0;
    bool need = !done;                 // the walker has no current move: search from lo
    bool load = false;                 // cur's columns are still to be loaded
    f2 dcur[PIPE ? C : 1][H];
    for (;;) {
        // ---- walkers without a current move search their windows (a sweep's start, or no
        // feasible proposal left in the windows), sliding them and ending sweeps as needed
        while (__any_sync(kFull, need)) {
            bool oa, fa, ob, fb;
            feasible_now(pa, wb + gl, need, oa, fa);
            feasible_now(pb, wb + G + gl, need, ob, fb);
            const uint32_t okm = group_bits(oa, ob);
            const uint32_t pfm = MODE == kHastings ? group_bits(fa, fb) : 0u;
            const int t = __ffs(okm) - 1;
            const MoveDraw found = take_bit(t < 0 ? 0 : t);
            if (need) {
                pos += count_pos(pfm, t);
                if (t >= 0) {
                    cur = found;
                    icur = wb + t;
                    lo = icur + 1;
                    need = false;
                    load = true;
                    if (t >= G) slide();
                } else if (wb + 2 * G >= NO) {
                    // the sweep is over
                    chi2 += (double)dchi;
                    accp = acc;
                    nacc += acc;
                    npos += pos;
                    if (S.acc_trace && gl == 0) S.acc_trace[(size_t)n * P.n_walkers + w] = acc;
                    if (++n >= n1) {
                        done = true;
                        need = false;
                    } else {
                        start_sweep();
                    }
                } else {
                    wb += 2 * G;
                    lo = wb;
                    pa = draw_move<MODE>(wb + gl, n, wr + P.walker_base, key, NO, yd, T, sBeta, sRgap);
                    pb = draw_move<MODE>(wb + G + gl, n, wr + P.walker_base, key, NO, yd, T, sBeta, sRgap);
                }
            }
        }
        if (!__any_sync(kFull, !done)) break;
        const bool live = !done;
        if constexpr (PIPE) {
            if (load) columns<G, C>(dcur, qhi, qlo, PAD, cur);
            load = false;
        }
        // move icur: the amplitudes it would set, and d = eps M + dpart
        const int p = cur.ps & 0xFFFF, s = cur.ps >> 16;
        const float r = 1.0f - cur.eps;
        const float ap = fmaf(r, ghi * bget(p), cur.dp);
        const float as = fmaf(r, ghi * bget(s), cur.ds);
        const f2 e2 = pk(cur.eps, cur.eps);
        f2 d[C][H];
        if constexpr (PIPE) {
#pragma unroll
            for (int c = 0; c < C; ++c)
#pragma unroll
                for (int h = 0; h < H; ++h) d[c][h] = fma2(e2, M[c][h], dcur[c][h]);
        } else {
            columns<G, C>(d, qhi, qlo, PAD, cur);
#pragma unroll
            for (int c = 0; c < C; ++c)
#pragma unroll
                for (int h = 0; h < H; ++h) d[c][h] = fma2(e2, M[c][h], d[c][h]);
        }
        // the spectrum if the move is accepted: scale g r, b_p and b_s as the update writes them
        float gah = ghi, gal = glo;
        pair_scale(gah, gal, r);
        const float inv_g = 1.0f / gah;
        const float bpn = ap * inv_g, bsn = as * inv_g;
        // the later proposals' feasibility for either outcome of this move
        bool rA, fA, aA, gA, rB, fB, aB, gB;
        auto feasible_both = [&](const MoveDraw &q, int idx, bool &okr, bool &pfr, bool &oka, bool &pfa) {
            const bool valid = live && idx >= lo && idx < NO;
            const int qp = q.ps & 0xFFFF, qs = q.ps >> 16;
            const float rq = 1.0f - q.eps;
            const float vp = bget(qp), vs = bget(qs);
            const float vpa = qp == p ? bpn : (qp == s ? bsn : vp);
            const float vsa = qs == p ? bpn : (qs == s ? bsn : vs);
            const bool posr = fmaf(rq, ghi * vp, q.dp) >= 0.0f && fmaf(rq, ghi * vs, q.ds) >= 0.0f;
            const bool posa = fmaf(rq, gah * vpa, q.dp) >= 0.0f && fmaf(rq, gah * vsa, q.ds) >= 0.0f;
            const bool hok = MODE != kHastings || q.thr > -INFINITY;
            okr = valid && posr && hok;
            pfr = valid && !posr;
            oka = valid && posa && hok;
            pfa = valid && !posa;
        };
        feasible_both(pa, wb + gl, rA, fA, aA, gA);
        feasible_both(pb, wb + G + gl, rB, fB, aB, gB);
        const uint32_t okr = group_bits(rA, rB), oka = group_bits(aA, aB);
        uint32_t pfr = 0, pfa = 0;
        if constexpr (MODE == kHastings) {
            pfr = group_bits(fA, fB);
            pfa = group_bits(gA, gB);
        }
        const int tr = __ffs(okr) - 1;
        if constexpr (PIPE) columns<G, C>(dcur, qhi, qlo, PAD, take_bit(tr < 0 ? 0 : tr));
        // move icur: delta chi2 = sum d (2 R + d) and the Metropolis test (the Hastings
        // threshold may be negative: then D <= 0 does not pass by itself)
        float D;
        bool accepted;
        if constexpr (MODE == kGuard) {
            float Dp, Sp;
            delta_sum_mag<C, H>(d, R, two, Dp, Sp);
            D = group_sum<G>(Dp);
            accepted = guarded_accept<G, C, false>(live, D, group_sum<G>(Sp), cur.thr, P.fp64_accept, R, M,
                                                   ColTab{qhi, qlo, 0u, 0u, PAD}, cur,
                                            n_re, n_flip);
        } else {
            D = group_sum<G>(delta_sum<C, H>(d, R, two));
            accepted = live && (MODE == kHastings ? D < cur.thr : (D <= 0.0f || D < cur.thr));
        }
        if (accepted) {
#pragma unroll
            for (int c = 0; c < C; ++c) {
#pragma unroll
                for (int h = 0; h < H; ++h) {
                    R[c][h] = add2(R[c][h], d[c][h]);
                    M[c][h] = fma2(minus_one, d[c][h], M[c][h]);
                }
            }
            ghi = gah;
            glo = gal;
            if (gl == 0) {
                bset(p, bpn);
                bset(s, bsn);
            }
            dchi += D;
            ++acc;
        }
        __syncwarp();
        // the next move: the first feasible proposal for the outcome
        const uint32_t okm = accepted ? oka : okr, pfm = accepted ? pfa : pfr;
        const int t = __ffs(okm) - 1;
        const MoveDraw nxt = take_bit(t < 0 ? 0 : t);
        if (live) {
            pos += count_pos(pfm, t);
            if (t < 0) {
                need = true;
                lo = wb + 2 * G;
            } else {
                icur = wb + t;
                lo = icur + 1;
                cur = nxt;
                load = t != tr;        // not the prefetched move: its columns are loaded first
                if (t >= G) slide();
            }
        }
    }
    if (!active) return;
    // fold the common scale into the spectrum and write the walker back
    float *bg = S.b32 + (size_t)w * NO;
    for (int j = gl; j < NO; j += G) {
        const float v = b[j];
        bg[j] = fmaf(glo, v, ghi * v);
    }
#pragma unroll
    for (int c = 0; c < C; ++c)
#pragma unroll
        for (int h = 0; h < H; ++h)
            *reinterpret_cast<float2 *>(S.R32 + (size_t)w * PAD + 32 * c + E * gl + 2 * h) = up(R[c][h]);
    if (gl == 0) {
        S.g2[2 * w] = 1.0f;
        S.g2[2 * w + 1] = 0.0f;
        S.chi2[w] = chi2;
        S.acc_prev[w] = accp;
        S.n_acc[w] += nacc;
        S.n_pos[w] += npos;
        if constexpr (MODE == kGuard) {
            if (n_re) atomicAdd(&S.guard[0], (unsigned long long)n_re);
            if (n_flip) atomicAdd(&S.guard[1], (unsigned long long)n_flip);
        }
    }
}

// The move loop of a variant: the index walk's bins depend on the spectrum, so it proposes
// and evaluates one move at a time; the uniform-bin variants may look ahead (AHEAD) where the
// next move's columns can be prefetched (up to 8 chunks).  Past that the look-ahead's search
// would stand in front of every column load, and the one-move loop is faster (measured at
// 512 tau: 3.69e9 against 2.16e9 walker-moves/s).
template <int G, int C, bool STAGED, int MODE, bool AHEAD>
__device__ __forceinline__ void run_walkers(const DevProblem &P, const DevState &S, int n0, int n1, int grp,
                                            const float *sm, float *b_stage, int walker_lo) {
    if constexpr (MODE == kWalk || C > 8 || !AHEAD)
        run_group<G, C, STAGED, MODE>(P, S, n0, n1, grp, sm, b_stage, walker_lo);
    else
        run_group_ahead<G, C, STAGED, MODE>(P, S, n0, n1, grp, sm, b_stage, walker_lo);
}

// Threads per block of the sweep kernels: 16 warps with 16 lanes per walker and up to 4
// chunks, or 9 (the first count without prefetched columns): 128 registers a thread; 12 warps
// otherwise (168 registers: the residual arrays grow with the chunks); 8 warps with 8 lanes per
// walker (whose 4 walkers a warp hold twice the residual elements per lane).
// The guarded variant past 8 chunks gets 8 warps (255 registers a thread) for its FP64 check.
template <int G, int C, int MODE = kPlain>
constexpr int sweep_threads() {
    return G == 8 ? 256 : (MODE == kGuard && C > 8) ? 256 : ((C <= 4 || C == 9) ? kThreads : 384);
}

// The table layout a kernel variant loads: quad-compact where its 8-lane walkers run the
// one-move loop (see TabLayout).
template <int G, int C, int MODE, bool AHEAD>
__host__ __device__ constexpr bool sweep_compact() {
    return G == 8 && !(MODE != kWalk && C <= 8 && AHEAD);
}

template <int G, int C, int MODE, bool AHEAD>
__global__ void __launch_bounds__(sweep_threads<G, C, MODE>()) sweep_fp32_kernel(DevProblem P, DevState S, int n0, int n1,
                                                              SweepGeom Gm) {
    extern __shared__ float4 smem4[];
    float *sm = reinterpret_cast<float *>(smem4);
    constexpr int WPW = 32 / G;
    const int NO = P.n_omega, PAD = P.n_tau_pad, NH = (NO + 31) >> 5;
    constexpr bool CT = sweep_compact<G, C, MODE, AHEAD>();
    // staged spectra [WPW * groups_per_cta][NO], after the tables
    float *sB = CT ? sm + tab_layout(true, NO, PAD).total : sm + (size_t)(NH + 32) * PAD + 2 * NO;
    load_tables_g<CT>(P, sm);
    const int grp_lo = blockIdx.x * Gm.groups_per_cta;
    const int grp_hi = min(grp_lo + Gm.groups_per_cta, Gm.groups_total);
    const int walker_lo = WPW * grp_lo;
    const int walker_hi = min(WPW * grp_hi, P.n_walkers);
    if (Gm.stage_b) {
        const size_t n = (size_t)(walker_hi - walker_lo) * NO;
        const float *src = S.b32 + (size_t)walker_lo * NO;
        for (size_t q = threadIdx.x; q < n; q += blockDim.x) sB[q] = src[q];
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5;
    for (int round = 0; round < Gm.rounds; ++round) {
        const int grp = grp_lo + round * Gm.warps + warp;
        if (grp >= grp_hi) break;                         // uniform across the warp
        if (Gm.stage_b)
            run_walkers<G, C, true, MODE, AHEAD>(P, S, n0, n1, grp, sm, sB, walker_lo);
        else
            run_walkers<G, C, false, MODE, AHEAD>(P, S, n0, n1, grp, sm, nullptr, walker_lo);
    }
}

// Bytes of the full-row tables and of the tables of either layout.
size_t table_bytes(const DevProblem &P) {
    const size_t NH = (size_t)(P.n_omega + 31) / 32;
    return (NH + 32) * (size_t)P.n_tau_pad * 4 + 2 * (size_t)P.n_omega * 4;
}
size_t table_bytes_g(bool compact, const DevProblem &P) {
    return (size_t)tab_layout(compact, P.n_omega, P.n_tau_pad).total * 4;
}

template <int G, int C, int MODE, bool AHEAD>
cudaError_t launch_c(const DevProblem &P, const DevState &S, int n0, int n1, cudaStream_t st) {
    int dev = 0, sms = 0, smem_max = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    constexpr int WPW = 32 / G;
    SweepGeom Gm;
    Gm.groups_total = (P.n_walkers + WPW - 1) / WPW;
    const int ctas = Gm.groups_total < sms ? Gm.groups_total : sms;
    Gm.groups_per_cta = (Gm.groups_total + ctas - 1) / ctas;
    const int max_warps = sweep_threads<G, C, MODE>() / 32;
    Gm.rounds = (Gm.groups_per_cta + max_warps - 1) / max_warps;
    Gm.warps = (Gm.groups_per_cta + Gm.rounds - 1) / Gm.rounds;
    const size_t tb = table_bytes_g(sweep_compact<G, C, MODE, AHEAD>(), P);
    const size_t staged = (size_t)WPW * Gm.groups_per_cta * P.n_omega * 4;
    if (tb > (size_t)smem_max) return cudaErrorInvalidValue;
    Gm.stage_b = tb + staged <= (size_t)smem_max;
    const size_t smem = tb + (Gm.stage_b ? staged : 0);
    cudaError_t e = cudaFuncSetAttribute(sweep_fp32_kernel<G, C, MODE, AHEAD>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    const int n_ctas = (Gm.groups_total + Gm.groups_per_cta - 1) / Gm.groups_per_cta;
    sweep_fp32_kernel<G, C, MODE, AHEAD><<<n_ctas, Gm.warps * 32, smem, st>>>(P, S, n0, n1, Gm);
    return cudaGetLastError();
}

// Up to 8 chunks the plain and Hastings variants come in both move loops (P.ahead chooses).
template <int G, int C, int MODE>
cudaError_t launch_pick(const DevProblem &P, const DevState &S, int n0, int n1, cudaStream_t st) {
    if constexpr (MODE != kWalk && C <= 8)
        if (P.ahead) return launch_c<G, C, MODE, true>(P, S, n0, n1, st);
    return launch_c<G, C, MODE, false>(P, S, n0, n1, st);
}

template <int MODE>
cudaError_t launch_sweep_w(const DevProblem &P, const DevState &S, int n0, int n1, cudaStream_t st) {
    if (P.lanes == 8) {
        switch (P.n_tau_pad / 32) {
            case 1: return launch_pick<8, 1, MODE>(P, S, n0, n1, st);
            case 2: return launch_pick<8, 2, MODE>(P, S, n0, n1, st);
            case 3: return launch_pick<8, 3, MODE>(P, S, n0, n1, st);
            case 4: return launch_pick<8, 4, MODE>(P, S, n0, n1, st);
            case 5: return launch_pick<8, 5, MODE>(P, S, n0, n1, st);
            case 6: return launch_pick<8, 6, MODE>(P, S, n0, n1, st);
            case 7: return launch_pick<8, 7, MODE>(P, S, n0, n1, st);
            case 8: return launch_pick<8, 8, MODE>(P, S, n0, n1, st);
            default: return cudaErrorInvalidValue;
        }
    }
    switch (P.n_tau_pad / 32) {
        case 1: return launch_pick<16, 1, MODE>(P, S, n0, n1, st);
        case 2: return launch_pick<16, 2, MODE>(P, S, n0, n1, st);
        case 3: return launch_pick<16, 3, MODE>(P, S, n0, n1, st);
        case 4: return launch_pick<16, 4, MODE>(P, S, n0, n1, st);
        case 5: return launch_pick<16, 5, MODE>(P, S, n0, n1, st);
        case 6: return launch_pick<16, 6, MODE>(P, S, n0, n1, st);
        case 7: return launch_pick<16, 7, MODE>(P, S, n0, n1, st);
        case 8: return launch_pick<16, 8, MODE>(P, S, n0, n1, st);
        case 9: return launch_pick<16, 9, MODE>(P, S, n0, n1, st);
        case 10: return launch_pick<16, 10, MODE>(P, S, n0, n1, st);
        case 11: return launch_pick<16, 11, MODE>(P, S, n0, n1, st);
        case 12: return launch_pick<16, 12, MODE>(P, S, n0, n1, st);
        case 13: return launch_pick<16, 13, MODE>(P, S, n0, n1, st);
        case 14: return launch_pick<16, 14, MODE>(P, S, n0, n1, st);
        case 15: return launch_pick<16, 15, MODE>(P, S, n0, n1, st);
        case 16: return launch_pick<16, 16, MODE>(P, S, n0, n1, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

}  // namespace sail
