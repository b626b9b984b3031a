// Residual recomputation on the tensor cores, BF16 with three pieces per operand and six
// products (resync kind 2): R = Fhat - Khat b for FP32 state, as a pipelined tcgen05 GEMM fed
// by the Tensor Memory Accelerator.
//
// Operands.  Each FP32 value x is split into three BF16 pieces, x = x1 + x2 + x3 (each the
// round-to-nearest BF16 of what is left), and the products kept are x1 y1 (main accumulator)
// and x1 y2 + x2 y1 + x1 y3 + x2 y2 + x3 y1 (correction accumulator); the dropped terms are
// ~2^-24 of a product.  The pieces are written once per recomputation (spectra, an elementwise
// pass) or once per handle (kernel table) as plain row-major BF16 arrays [piece][row][bin],
// rows of 64-bin multiples.  A tile of 64 bins (128 bytes per row) moves to shared memory as
// one 3D tensor copy (cp.async.bulk.tensor) with the 128-byte swizzle, which is the K-major
// operand layout the MMA reads with a SWIZZLE_128B descriptor (8-row groups 1024 bytes apart;
// the K steps of 16 bins advance the start address by 32 bytes inside the swizzle atom).
//
// Block: 128 walkers (the MMA's M) x N tau columns (N = 128, 96, 64 or 32, the widest
// dividing the padded tau count), 18 warps with fixed roles:
//   warp 0: one thread issues the tensor copies of stage s (3 spectra tiles, 3 kernel tiles)
//           once the MMAs have released it (mbarrier empty[s]) and arms full[s] with the byte
//           count;
//   warp 1: one thread waits full[s], issues the stage's 24 MMAs (four K steps of 16 bins,
//           six products each), commits them to empty[s] and the main accumulator buffer to
//           accfull[b], and starts the next stage in the other buffer once the epilogue has
//           drained it (accempty[b]);
//   warps 2-17: drain the main accumulator of each 64-bin period with tcgen05.ld and add it to
//           per-thread float pairs (packed Fast2Sum, round to nearest), four warps per 32-lane
//           quarter of tensor memory (each a quarter of the columns); after the last period add
//           the correction accumulator once, then write R.
// A thread keeps a float pair for each of its N / 4 columns in registers (96 a thread: the
// most that 576 threads can launch with).
// The tensor core's FP32 accumulator rounds toward zero in its internal sums; restarting the
// main chain every 64 bins (four MMAs) keeps that bias near 2^-22 of a product, and the periods
// are summed in float pairs.  The correction products are about 2^-8 of the main ones, so their
// one accumulator runs over all bins (the bias, ~2^-24 per addition of a sum 2^-8 of the model,
// stays near 1e-7 of the model at 2048 bins): the epilogue drains half the columns per period
// (measured 0.448 -> 0.440 ms per call at 512 x 2048 x 16384, the same maximum error).  Tensor
// memory holds two buffers of N main columns and one region of N correction columns, so the
// MMAs of one period overlap the draining of the previous one; shared memory
// holds two (N > 64) or three stages of 64 bins.  Every wait is bounded: on time-out a thread
// sets the status word and the block's abort flag, the roles leave their loops, the copy thread
// waits (bounded) for the copies it issued, the MMA thread for its MMAs, and tensor memory is
// freed before the block returns.
//
// Measured limit (512 tau x 2048 bins x 16384 walkers, N = 128): the MMA rate.  Alone, this
// MMA shape runs at 64 cycles (4096 multiply-adds a cycle per SM), also with the six-product
// pattern, random data, concurrent bulk copies into other shared memory and concurrent
// tensor-memory loads (67); in this kernel it took about 160 cycles with a TwoSum epilogue.
// Timing-only copies show where the rest goes: without the epilogue's arithmetic the MMAs take
// 116 cycles, without the tensor copies 151, without both 105; the epilogue's floating-point
// work, running on the same SM, slows the tensor pipe more than anything else.
#include <cstdint>

#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include "sail_internal.cuh"

namespace sail {

namespace {

constexpr int kM = 128;                      // walkers per block (MMA M)
constexpr int kKT = 64;                      // bins per stage (one 128-byte swizzle atom of BF16)
constexpr int kPeriodTiles = 1;              // stages per accumulation period (64 bins)
constexpr int kEpiWarps = 16;
constexpr int kThreads = 32 * (2 + kEpiWarps);
constexpr uint32_t kTileA = kM * kKT * 2;    // bytes of one piece of the spectra tile (16 KB)
constexpr uint32_t kSBO = 1024;              // 8 rows x 128 bytes: one swizzle pattern
constexpr long long kSpin = 1ll << 26;

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory descriptor of a K-major operand in the 128-byte swizzle: start address, leading
// offset (unused with this swizzle: 1), stride between 8-row groups, descriptor version 1,
// layout type 2 (SWIZZLE_128B).
__device__ __forceinline__ uint64_t desc(uint32_t addr) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) | ((uint64_t)((kSBO >> 4) & 0x3FFFu) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}

__device__ __forceinline__ bool try_wait(uint32_t mbar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait on an mbarrier phase (also gives up when the block aborts); false on give-up.
__device__ bool wait(uint32_t mbar, uint32_t parity, volatile int *abort) {
    for (long long it = 0; it < kSpin; ++it) {
        if (try_wait(mbar, parity)) return true;
        if ((it & 1023) == 1023 && *abort) return false;
    }
    return false;
}

__device__ __forceinline__ void arrive(uint32_t mbar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mbar) : "memory");
}

__device__ __forceinline__ void arrive_tx(uint32_t mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
}

// One 3D tensor copy global -> shared (bins x, rows y, piece z), completing on mbar.
__device__ __forceinline__ void tma_3d(uint32_t dst, const CUtensorMap *map, int x, int y, int z, uint32_t mbar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(z), "r"(mbar)
        : "memory");
}

__device__ __forceinline__ void tmem_ld4(uint32_t taddr, uint32_t v[4]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3])
                 : "r"(taddr));
}

// (hi, lo) += m + c for a period's main partial m and correction partial c (all terms are
// non-negative), two columns at a time in packed FP32 pairs (add/sub.rn.f32x2: two independent
// round-to-nearest operations per instruction, the rounding of the scalar form): Fast2Sum of m
// into hi, its rounding error and c added to lo.  The error term is exact when hi >= m (the
// kernel decays with the bin's frequency, so the running sum soon dominates a period's
// partial); otherwise it is off by at most a rounding of the running sum.  Five packed
// additions per two columns and period instead of TwoSum's seven scalar ones: the epilogue's
// arithmetic runs beside the MMAs on the same SM and slows them (measured at 512 x 2048 x
// 16384: 0.505 ms per recomputation with TwoSum, 0.466 with scalar Fast2Sum, 0.454 packed; the
// same maximum error; 0.448 with a single thread polling each period's barrier).
typedef unsigned long long f2;
__device__ __forceinline__ f2 pk(uint32_t a, uint32_t b) {
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "r"(a), "r"(b));
    return r;
}
__device__ __forceinline__ f2 add2(f2 a, f2 b) {
    f2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 sub2(f2 a, f2 b) {
    f2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ void fast_two_sum_add1(f2 &hi, f2 &lo, f2 m) {
    const f2 s = add2(hi, m);
    lo = add2(lo, sub2(m, sub2(s, hi)));
    hi = s;
}
__device__ __forceinline__ void fast_two_sum_add2(f2 &hi, f2 &lo, f2 m, f2 c) {
    const f2 s = add2(hi, m);
    lo = add2(lo, add2(sub2(m, sub2(s, hi)), c));
    hi = s;
}

// The three BF16 pieces of 8 consecutive values as three 16-byte core-matrix rows.
__device__ __forceinline__ void split8(const float (&v)[8], uint4 &r1, uint4 &r2, uint4 &r3) {
    uint32_t w1[4], w2[4], w3[4];
#pragma unroll
    for (int e = 0; e < 8; e += 2) {
        uint32_t p1[2], p2[2], p3[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const float x = v[e + h];
            const __nv_bfloat16 b1 = __float2bfloat16_rn(x);
            const float r = x - __bfloat162float(b1);
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
    r1 = make_uint4(w1[0], w1[1], w1[2], w1[3]);
    r2 = make_uint4(w2[0], w2[1], w2[2], w2[3]);
    r3 = make_uint4(w3[0], w3[1], w3[2], w3[3]);
}

// The three BF16 pieces of the spectra, [piece][walker row][bin] with rows of NOP bins
// (n_omega rounded up to 64) and W_pad rows (n_walkers rounded up to 128), zero past the last
// walker or bin: thread t splits 8 consecutive bins of one row (coalesced loads and stores).
__global__ void presplit_spectra_kernel(DevProblem P, DevState S, uint4 *At, int n_rows, int nop) {
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int per_row = nop / 8;
    if (t >= (size_t)n_rows * per_row) return;
    const int w = (int)(t / per_row), j0 = (int)(t % per_row) * 8;
    float v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e)
        v[e] = (w < P.n_walkers && j0 + e < P.n_omega) ? S.b32[(size_t)w * P.n_omega + j0 + e] : 0.0f;
    uint4 r1, r2, r3;
    split8(v, r1, r2, r3);
    const size_t plane = (size_t)n_rows * nop / 8;             // uint4 per piece
    At[t] = r1;
    At[plane + t] = r2;
    At[2 * plane + t] = r3;
}

// The three BF16 pieces of the kernel table, [piece][tau row][bin] (once per handle).
__global__ void presplit_kernel_table(DevProblem P, uint4 *Bt, int nop) {
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int per_row = nop / 8;
    if (t >= (size_t)P.n_tau_pad * per_row) return;
    const int i = (int)(t / per_row), j0 = (int)(t % per_row) * 8;
    float v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e)
        v[e] = (i < P.n_tau && j0 + e < P.n_omega) ? P.Khat32[(size_t)(j0 + e) * P.n_tau_pad + i] : 0.0f;
    uint4 r1, r2, r3;
    split8(v, r1, r2, r3);
    const size_t plane = (size_t)P.n_tau_pad * nop / 8;
    Bt[t] = r1;
    Bt[plane + t] = r2;
    Bt[2 * plane + t] = r3;
}

template <int N>
struct TmaCfg {
    static constexpr uint32_t kTileB = N * kKT * 2;
    static constexpr uint32_t kStage = 3 * (kTileA + kTileB);
    static constexpr int kStages = N <= 64 ? 3 : 2;                // 3 x 72 KB at N = 64, 2 x 96 KB at 128
    static constexpr uint32_t kCols = 4 * N <= 256 ? 256 : 512;   // two buffers of (main, corr)
    static constexpr int kPart = N / 4;                            // columns per epilogue thread
    static constexpr int kBars = 2 * kStages + 5;                 // full, empty, accfull, accempty, done
    static constexpr size_t kSmem = (size_t)kStages * kStage + 8 * kBars + 16 + 1024;
};

template <int N>
__global__ void __maxnreg__(96)
    resync_tma_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, DevProblem P,
                      DevState S, int n_kt, int *status) {
    using C = TmaCfg<N>;
    static_assert(N % 32 == 0 && N >= 32 && N <= 128, "tau columns per block");
    extern __shared__ unsigned char smem_raw[];
    unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + (size_t)C::kStages * C::kStage);
    // bar[0, S) full, bar[S, 2S) empty, bar[2S, 2S + 2) accfull, bar[2S + 2, 2S + 4) accempty,
    // bar[2S + 4] done (S stages); then the tensor-memory address and the abort flag
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bar + C::kBars);
    volatile int *abort = reinterpret_cast<volatile int *>(tmem_slot + 1);
    volatile int *epi_ok = abort + 1;                  // [2]: epilogue verdict per accumulator buffer
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nb = blockIdx.x, wb = blockIdx.y;
    const uint32_t sbase = smem_u32(smem), bbase = smem_u32(bar);
    auto full = [&](int s) { return bbase + 8u * (uint32_t)s; };
    auto empty = [&](int s) { return bbase + 8u * (uint32_t)(C::kStages + s); };
    auto accfull = [&](int b) { return bbase + 8u * (uint32_t)(2 * C::kStages + b); };
    auto accempty = [&](int b) { return bbase + 8u * (uint32_t)(2 * C::kStages + 2 + b); };
    const uint32_t done_bar = bbase + 8u * (uint32_t)(2 * C::kStages + 4);
    auto tileA = [&](int s, int q) { return sbase + (uint32_t)s * C::kStage + (uint32_t)q * kTileA; };
    auto tileB = [&](int s, int q) { return sbase + (uint32_t)s * C::kStage + 3u * kTileA + (uint32_t)q * C::kTileB; };

    if (tid == 0) {
        for (int s = 0; s < C::kStages; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(full(s)));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(empty(s)));
        }
        for (int b = 0; b < 2; ++b) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(accfull(b)));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(accempty(b)), "r"(kEpiWarps));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(done_bar));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        *abort = 0;
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(C::kCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tmem_slot;
    const int n_periods = (n_kt + kPeriodTiles - 1) / kPeriodTiles;

    if (warp == 0) {
        if (lane == 0) {
            // ---- tensor copies
            int issued = 0;
            for (int kt = 0; kt < n_kt && !*abort; ++kt) {
                const int s = kt % C::kStages, u = kt / C::kStages;
                if (u > 0 && !wait(empty(s), (uint32_t)((u - 1) & 1), abort)) {
                    atomicExch(status, 1);
                    *abort = 1;
                    break;
                }
                arrive_tx(full(s), C::kStage);
                for (int q = 0; q < 3; ++q) {
                    tma_3d(tileA(s, q), &tmA, kt * kKT, wb * kM, q, full(s));
                    tma_3d(tileB(s, q), &tmB, kt * kKT, nb * N, q, full(s));
                }
                issued = kt + 1;
            }
            if (*abort) {
                // copies still landing in shared memory: wait (bounded) for the stages issued
                for (int kt = issued > C::kStages ? issued - C::kStages : 0; kt < issued; ++kt) {
                    const long long lim = kSpin;
                    for (long long it = 0; it < lim; ++it)
                        if (try_wait(full(kt % C::kStages), (uint32_t)((kt / C::kStages) & 1))) break;
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---- MMAs.  A descriptor is linear in its start address (bits 0-13 hold it in
            // 16-byte units), so each operand's descriptor is one base plus a constant offset.
            const uint32_t idesc = idesc_bf16(kM, N);
            const uint64_t dA = desc(tileA(0, 0)), dB = desc(tileB(0, 0));
            constexpr uint64_t kTa = kTileA >> 4, kTb = C::kTileB >> 4, kKs = 32u >> 4;
            int kt = 0;
            for (int d = 0; d < n_periods && !*abort; ++d) {
                const int b = d & 1, u = d >> 1;
                if (u > 0 && !wait(accempty(b), (uint32_t)((u - 1) & 1), abort)) {
                    atomicExch(status, 1);
                    *abort = 1;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint32_t dmain = tmem + (uint32_t)(b * N), dcorr = tmem + (uint32_t)(2 * N);
                for (int t = 0; t < kPeriodTiles && kt < n_kt; ++t, ++kt) {
                    const int s = kt % C::kStages;
                    if (!wait(full(s), (uint32_t)((kt / C::kStages) & 1), abort)) {
                        atomicExch(status, 1);
                        *abort = 1;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;");
                    const uint64_t sa = dA + (uint64_t)((uint32_t)s * (C::kStage >> 4)),
                                   sb = dB + (uint64_t)((uint32_t)s * (C::kStage >> 4));
#pragma unroll
                    for (int ks = 0; ks < kKT / 16; ++ks) {   // 16 bins = 32 bytes of the swizzle atom
                        const uint64_t a0 = sa + ks * kKs, a1 = a0 + kTa, a2 = a0 + 2 * kTa;
                        const uint64_t b0 = sb + ks * kKs, b1 = b0 + kTb, b2 = b0 + 2 * kTb;
                        const uint32_t acc = (t > 0 || ks > 0) ? 1u : 0u;
                        const uint32_t acc_c = (d > 0 || t > 0 || ks > 0) ? 1u : 0u;
                        mma_bf16(dmain, a0, b0, idesc, acc);
                        mma_bf16(dcorr, a0, b1, idesc, acc_c);
                        mma_bf16(dcorr, a1, b0, idesc, 1u);
                        mma_bf16(dcorr, a0, b2, idesc, 1u);
                        mma_bf16(dcorr, a1, b1, idesc, 1u);
                        mma_bf16(dcorr, a2, b0, idesc, 1u);
                    }
                    commit(empty(s));
                }
                if (*abort) break;
                commit(accfull(b));
            }
            // every MMA issued has completed before the tensor memory is freed
            commit(done_bar);
            for (long long it = 0; it < kSpin; ++it)
                if (try_wait(done_bar, 0u)) break;
        }
    } else {
        // ---- epilogue: warps 2..17; a warp may read tensor-memory lanes 32 (warp % 4) .. +31,
        // and the four warps of each such quarter take a quarter of the columns each
        const int quarter = warp & 3, part = (warp - 2) >> 2;
        const uint32_t lane_base = (uint32_t)(32 * quarter) << 16;
        f2 hi2[C::kPart / 2], lo2[C::kPart / 2];
#pragma unroll
        for (int c = 0; c < C::kPart / 2; ++c) {
            hi2[c] = 0ull;
            lo2[c] = 0ull;
        }
        for (int d = 0; d < n_periods; ++d) {
            const int b = d & 1;
            // one thread polls the period's barrier and posts the verdict in epi_ok[b]; the 16
            // epilogue warps meet at named barrier 1 (each converged for the .sync.aligned
            // tensor-memory loads), so all leave the loop at the same period (the flag of a
            // buffer is rewritten only after every warp has passed the next period's barrier)
            if (warp == 2 && lane == 0) {
                const bool ok = wait(accfull(b), (uint32_t)((d >> 1) & 1), abort);
                if (!ok) {
                    atomicExch(status, 1);
                    *abort = 1;
                }
                epi_ok[b] = ok ? 1 : 0;
            }
            asm volatile("bar.sync 1, %0;" ::"r"(32 * kEpiWarps) : "memory");
            if (!epi_ok[b]) break;
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t col0 = (uint32_t)(b * N + part * C::kPart);
#pragma unroll
            for (int c = 0; c < C::kPart; c += 8) {
                uint32_t v0[4], v1[4];
                tmem_ld4(tmem + lane_base + col0 + (uint32_t)c, v0);
                tmem_ld4(tmem + lane_base + col0 + (uint32_t)(c + 4), v1);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                fast_two_sum_add1(hi2[c / 2], lo2[c / 2], pk(v0[0], v0[1]));
                fast_two_sum_add1(hi2[c / 2 + 1], lo2[c / 2 + 1], pk(v0[2], v0[3]));
                fast_two_sum_add1(hi2[c / 2 + 2], lo2[c / 2 + 2], pk(v1[0], v1[1]));
                fast_two_sum_add1(hi2[c / 2 + 3], lo2[c / 2 + 3], pk(v1[2], v1[3]));
            }
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncwarp();
            if (lane == 0) arrive(accempty(b));
        }
        if (!*abort) {
            // the correction accumulator, complete with the last period's commit, added once
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t colc = (uint32_t)(2 * N + part * C::kPart);
#pragma unroll
            for (int c = 0; c < C::kPart; c += 8) {
                uint32_t v0[4], v1[4];
                tmem_ld4(tmem + lane_base + colc + (uint32_t)c, v0);
                tmem_ld4(tmem + lane_base + colc + (uint32_t)(c + 4), v1);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                lo2[c / 2] = add2(lo2[c / 2], pk(v0[0], v0[1]));
                lo2[c / 2 + 1] = add2(lo2[c / 2 + 1], pk(v0[2], v0[3]));
                lo2[c / 2 + 2] = add2(lo2[c / 2 + 2], pk(v1[0], v1[1]));
                lo2[c / 2 + 3] = add2(lo2[c / 2 + 3], pk(v1[2], v1[3]));
            }
            const int w = wb * kM + 32 * quarter + lane;
            if (w < P.n_walkers) {
                float *Rw = S.R32 + (size_t)w * P.n_tau_pad + nb * N + part * C::kPart;
                const double *Fw = P.Fhat64 + nb * N + part * C::kPart;
                const int i0 = nb * N + part * C::kPart;
#pragma unroll
                for (int c = 0; c < C::kPart; ++c) {
                    float h, l;
                    if (c & 1)
                        asm("mov.b64 {_, %0}, %2;\n\tmov.b64 {_, %1}, %3;" : "=f"(h), "=f"(l) : "l"(hi2[c / 2]), "l"(lo2[c / 2]));
                    else
                        asm("mov.b64 {%0, _}, %2;\n\tmov.b64 {%1, _}, %3;" : "=f"(h), "=f"(l) : "l"(hi2[c / 2]), "l"(lo2[c / 2]));
                    const double r = i0 + c < P.n_tau ? Fw[c] - ((double)h + (double)l) : 0.0;
                    Rw[c] = (float)r;
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(C::kCols));
}

// chi2 = sum_i R_i^2 (FP64) from the stored residual; one warp per walker.
__global__ void tma_chi2_kernel(DevProblem P, DevState S) {
    const int w = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (w >= P.n_walkers) return;
    double c2 = 0.0;
    for (int i = lane; i < P.n_tau; i += 32) {
        const double r = (double)S.R32[(size_t)w * P.n_tau_pad + i];
        c2 += r * r;
    }
    for (int o = 16; o > 0; o >>= 1) c2 += __shfl_xor_sync(0xFFFFFFFFu, c2, o);
    if (lane == 0) S.chi2[w] = c2;
}

template <int N>
cudaError_t launch_n(const DevProblem &P, const DevState &S, const TmaPlan &T, int *status, cudaStream_t st) {
    using C = TmaCfg<N>;
    cudaError_t e = cudaFuncSetAttribute(resync_tma_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::kSmem);
    if (e != cudaSuccess) return e;
    const dim3 grid(T.n_blocks_tau, T.n_blocks_walkers);
    resync_tma_kernel<N><<<grid, kThreads, C::kSmem, st>>>(T.map_a, T.map_b, P, S, T.n_kt, status);
    return cudaGetLastError();
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

// A [3][rows][nop] BF16 array as a 3D tensor copied in boxes of 64 bins x box_rows rows x one
// piece, with the 128-byte swizzle (the operand layout of the MMA's SWIZZLE_128B descriptors).
bool encode_pieces(CUtensorMap *map, void *base, size_t rows, int nop, uint32_t box_rows) {
    PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)nop, (cuuint64_t)rows, 3};
    const cuuint64_t strides[2] = {(cuuint64_t)nop * 2, (cuuint64_t)nop * 2 * rows};
    const cuuint32_t box[3] = {(cuuint32_t)kKT, box_rows, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
           CUDA_SUCCESS;
}

int bins_padded(int n_omega) { return (n_omega + kKT - 1) / kKT * kKT; }
int walkers_padded(int n_walkers) { return (n_walkers + kM - 1) / kM * kM; }

}  // namespace

int tma_tau_block(int n_tau_pad) {
    for (int nc = 128; nc >= 32; nc -= 32)
        if (n_tau_pad % nc == 0) return nc;
    return 0;
}

size_t tma_spectra_bytes(int n_walkers, int n_omega) {
    return (size_t)3 * walkers_padded(n_walkers) * bins_padded(n_omega) * 2;
}

size_t tma_table_bytes(int n_tau_pad, int n_omega) { return (size_t)3 * n_tau_pad * bins_padded(n_omega) * 2; }

cudaError_t tma_plan_init(TmaPlan &T, const DevProblem &P, void *At, void *Bt, cudaStream_t st) {
    T.n = tma_tau_block(P.n_tau_pad);
    if (T.n == 0) return cudaErrorInvalidValue;
    const int nop = bins_padded(P.n_omega);
    T.nop = nop;
    T.n_kt = nop / kKT;
    T.n_blocks_tau = P.n_tau_pad / T.n;
    T.n_blocks_walkers = walkers_padded(P.n_walkers) / kM;
    T.At = At;
    T.Bt = Bt;
    if (((uintptr_t)At & 127) || ((uintptr_t)Bt & 127)) return cudaErrorInvalidValue;
    if (!encode_pieces(&T.map_a, At, (size_t)walkers_padded(P.n_walkers), nop, kM) ||
        !encode_pieces(&T.map_b, Bt, (size_t)P.n_tau_pad, nop, (uint32_t)T.n))
        return cudaErrorInvalidValue;
    const size_t threads = (size_t)P.n_tau_pad * nop / 8;
    presplit_kernel_table<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(P, (uint4 *)Bt, nop);
    // the spectra pieces' padding (rows past the last walker, bins past the last bin) stays zero:
    // the sum-rule restoration writes only the walkers' bins
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return cudaMemsetAsync(At, 0, tma_spectra_bytes(P.n_walkers, P.n_omega), st);
}

cudaError_t launch_resync_tma(const DevProblem &P, const DevState &S, const TmaPlan &T, int *status, bool presplit,
                              cudaStream_t st) {
    cudaError_t e = cudaSuccess;
    if (presplit) {
        const int nop = T.nop, rows = T.n_blocks_walkers * kM;
        const size_t threads = (size_t)rows * nop / 8;
        presplit_spectra_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(P, S, (uint4 *)T.At, rows, nop);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    switch (T.n) {
        case 128: e = launch_n<128>(P, S, T, status, st); break;
        case 96: e = launch_n<96>(P, S, T, status, st); break;
        case 64: e = launch_n<64>(P, S, T, status, st); break;
        case 32: e = launch_n<32>(P, S, T, status, st); break;
        default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    tma_chi2_kernel<<<(P.n_walkers * 32 + 255) / 256, 256, 0, st>>>(P, S);
    return cudaGetLastError();
}

}  // namespace sail
