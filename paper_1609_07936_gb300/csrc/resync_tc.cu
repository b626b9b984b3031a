// Residual recomputation on the 5th-generation tensor cores: R = Fhat - Khat b for FP32 state.
//
// The contraction (walkers x bins) . (bins x tau) runs as tcgen05.mma kind::tf32 with a
// three-term split of both operands: x = x_hi + x_lo with x_hi the value cut to TF32 (10
// mantissa bits) and x_lo the exact FP32 remainder, and
//     Khat b ~ K_hi b_hi + (K_hi b_lo + K_lo b_hi)
// (the dropped K_lo b_lo term is ~2^-20 of a product, random in sign), so each product keeps
// about 21 bits.
//
// Accumulation.  The tensor core's FP32 accumulator rounds toward zero in its internal sums,
// so a long chain of MMAs into one accumulator drifts low by ~2^-24 per MMA (measured: 3e-5
// relative over 1000 bins).  Here the main term and the two small terms go to separate
// tensor-memory accumulators that restart with every 32-bin tile (4 MMAs of K = 8 each); after
// each tile every thread drains its columns with tcgen05.ld and adds them to an unevaluated
// float pair (TwoSum, round to nearest), so the bias is that of 4 MMAs per tile and the sum
// over tiles carries ~2^-44 relative error.
//
// The library launches this kernel for the TF32 form (resync kind 1); the BF16 form (kind 2)
// runs as the tensor-copy pipeline of resync_tma.cu.  The template's BF16 operand format:
// each operand is split into three BF16 pieces,
// x = x1 + x2 + x3 (each the round-to-nearest BF16 of what is left), and the products kept are
// x1 y1 (main accumulator) and x1 y2 + x2 y1 + x1 y3 + x2 y2 + x3 y1 (correction accumulator);
// the dropped terms are ~2^-24 of a product.  kind::f16 with BF16 A and B (both operands of
// one MMA the same type), K = 16 per MMA.
//
// Block: 128 walkers (the MMA's M) x NC tau columns (NC <= 128, a multiple of 16; n_tau_pad
// is split over gridDim.y blocks), 16 warps: warp w reads tensor-memory lanes
// 32 (w % 4) .. +31 (its walkers) and columns (w / 4) NC/4 .. +NC/4.  Bins are taken 32 at a
// time: the block writes the split spectra tile and the split kernel tile into shared memory in
// the canonical K-major layout without swizzle (core matrices of 8 rows x 16 bytes; the next
// core matrix along K 128 bytes on, the next 8-row group 1024 bytes on), thread 0 issues the
// tile's 12 MMAs and commits them to an mbarrier, and the block waits on it before draining
// and reusing the tiles.  Every wait is bounded: on time-out the block sets the status word,
// stops issuing, frees its tensor memory and returns.  chi2 is summed from the stored
// residual by resync_chi2_kernel.
#include <cstdint>

#include <cuda_bf16.h>

#include "sail_internal.cuh"

namespace sail {

namespace {

constexpr int kM = 128;            // walkers per block (MMA M)
constexpr int kKT = 32;            // bins per shared-memory tile
constexpr int kThreads = 512;      // 16 warps
constexpr uint32_t kLBO = 128;     // bytes between core matrices along K
constexpr uint32_t kCorrCol = 128; // tensor-memory column of the correction accumulator

// Operand format of a resync variant: element bytes, pieces per operand, and the byte stride
// between 8-row groups of a [rows x 32] K-major tile (its core matrices of 8 rows x 16 bytes
// laid side by side along K).
template <bool BF16>
struct Fmt {
    static constexpr int kElem = BF16 ? 2 : 4;
    static constexpr int kPieces = BF16 ? 3 : 2;
    static constexpr int kPerCore = 16 / kElem;             // elements of a core-matrix row
    static constexpr uint32_t kSBO = (kKT / kPerCore) * 128;  // 512 (BF16) or 1024 (TF32)
    static constexpr int kSteps = kKT * kElem / 32;          // MMAs of K = 32 bytes per tile
};
constexpr uint32_t kCols = 256;    // tensor-memory columns allocated per block
constexpr long long kSpinLimit = 1ll << 26;

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Byte offset of element (row r, k) of a [rows x 32] K-major tile in the canonical layout.
template <bool BF16>
__device__ __forceinline__ uint32_t tile_off(int r, int k) {
    using F = Fmt<BF16>;
    return (uint32_t)(((r >> 3) * (kKT / F::kPerCore) + k / F::kPerCore) * 128 + (r & 7) * 16 +
                      (k % F::kPerCore) * F::kElem);
}

// Shared-memory matrix descriptor: start address, leading (K) and stride (M/N) byte
// offsets, descriptor version 1, no swizzle.
template <bool BF16>
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((kLBO >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((Fmt<BF16>::kSBO >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor: D FP32; A and B TF32 (kind::tf32) or BF16 (kind::f16); both
// K-major; N and M.
template <bool BF16>
__host__ __device__ constexpr uint32_t instr_desc(int M, int N) {
    return (1u << 4) | ((BF16 ? 1u : 2u) << 7) | ((BF16 ? 1u : 2u) << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

template <bool BF16>
__device__ __forceinline__ void mma(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    if constexpr (BF16)
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
            "l"(a), "l"(b), "r"(idesc), "r"(acc));
    else
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
            "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

// Writes one core-matrix row (kPerCore consecutive K elements, 16 bytes) of every piece of the
// values v at byte offset off of the tiles t[0..kPieces): the TF32 high part and the remainder,
// or three BF16 pieces, each the round-to-nearest BF16 of what is left.
template <bool BF16>
__device__ __forceinline__ void put_row(unsigned char *const *t, uint32_t off, const float *v) {
    if constexpr (BF16) {
        uint32_t w1[4], w2[4], w3[4];
#pragma unroll
        for (int e = 0; e < 8; e += 2) {
            __nv_bfloat16 p1[2], p2[2], p3[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const float x = v[e + h];
                p1[h] = __float2bfloat16_rn(x);
                const float r1 = x - __bfloat162float(p1[h]);
                p2[h] = __float2bfloat16_rn(r1);
                p3[h] = __float2bfloat16_rn(r1 - __bfloat162float(p2[h]));
            }
            w1[e / 2] = (uint32_t)__bfloat16_as_ushort(p1[0]) | ((uint32_t)__bfloat16_as_ushort(p1[1]) << 16);
            w2[e / 2] = (uint32_t)__bfloat16_as_ushort(p2[0]) | ((uint32_t)__bfloat16_as_ushort(p2[1]) << 16);
            w3[e / 2] = (uint32_t)__bfloat16_as_ushort(p3[0]) | ((uint32_t)__bfloat16_as_ushort(p3[1]) << 16);
        }
        *reinterpret_cast<uint4 *>(t[0] + off) = make_uint4(w1[0], w1[1], w1[2], w1[3]);
        *reinterpret_cast<uint4 *>(t[1] + off) = make_uint4(w2[0], w2[1], w2[2], w2[3]);
        *reinterpret_cast<uint4 *>(t[2] + off) = make_uint4(w3[0], w3[1], w3[2], w3[3]);
    } else {
        float hi[4], lo[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            hi[e] = __uint_as_float(__float_as_uint(v[e]) & 0xFFFFE000u);
            lo[e] = v[e] - hi[e];
        }
        *reinterpret_cast<float4 *>(t[0] + off) = make_float4(hi[0], hi[1], hi[2], hi[3]);
        *reinterpret_cast<float4 *>(t[1] + off) = make_float4(lo[0], lo[1], lo[2], lo[3]);
    }
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t mbar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait on an mbarrier phase; false on time-out.
__device__ bool mbar_wait(uint32_t mbar, uint32_t parity, long long limit) {
    for (long long it = 0; it < limit; ++it)
        if (mbar_try_wait(mbar, parity)) return true;
    return false;
}

__device__ __forceinline__ void tmem_ld4(uint32_t taddr, uint32_t v[4]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3])
        : "r"(taddr));
}

// (hi, lo) <- (hi, lo) + x: x added to hi without loss, the rounding error carried in lo.
__device__ __forceinline__ void two_sum_add(float &hi, float &lo, float x) {
    const float s = hi + x;
    const float bb = s - hi;
    const float err = (hi - (s - bb)) + (x - bb);
    hi = s;
    lo += err;
}

template <int NC, bool BF16>   // tau columns per block (a multiple of 16, <= 128); operand format
__global__ void __launch_bounds__(kThreads) resync_tc_kernel(DevProblem P, DevState S, int *status) {
    using F = Fmt<BF16>;
    constexpr int CS = NC / 4;                    // columns per thread, a multiple of 4
    constexpr int kATile = kM * kKT * F::kElem;   // bytes of one piece of the spectra tile
    constexpr int kBTile = NC * kKT * F::kElem;   // bytes of one piece of the kernel tile
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *sA[F::kPieces], *sB[F::kPieces];
#pragma unroll
    for (int q = 0; q < F::kPieces; ++q) {
        sA[q] = smem + q * kATile;
        sB[q] = smem + F::kPieces * kATile + q * kBTile;
    }
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem + F::kPieces * (kATile + kBTile));
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(mbar + 1);
    int *abort_flag = reinterpret_cast<int *>(tmem_slot + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int quarter = warp & 3, slice = warp >> 2;
    const int w0 = blockIdx.x * kM;
    const int i0 = blockIdx.y * NC;              // first tau column of this block
    const int NO = P.n_omega, NOP = P.n_omega_pad, PAD = P.n_tau_pad;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        *abort_flag = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tmem_slot;
    const uint32_t mbar_a = smem_u32(mbar);
    const uint32_t idesc = instr_desc<BF16>(kM, NC);
    // wait_test: the first tile's MMAs and commit are withheld, so its wait runs out (test hook
    // for the time-out path; nothing is in flight when the block gives up)
    const long long spin = P.wait_test ? 1024 : kSpinLimit;

    float acc_hi[CS], acc_lo[CS];
#pragma unroll
    for (int c = 0; c < CS; ++c) {
        acc_hi[c] = 0.0f;
        acc_lo[c] = 0.0f;
    }
    uint32_t phase = 0;
    const int n_tiles = NOP / kKT;
    for (int t = 0; t < n_tiles; ++t) {
        const int j0 = t * kKT;
        // spectra tile: 128 walkers x 32 bins, split into pieces.  A thread writes whole
        // core-matrix rows (16 bytes of every piece); consecutive threads take consecutive
        // walkers, so a warp's stores fill 128-byte core matrices without bank conflicts.
        constexpr int PC = F::kPerCore, RC = kKT / PC;   // row chunks per tile row
        for (int q = tid; q < kM * RC; q += kThreads) {
            const int r = q % kM, kc = q / kM;
            const int w = w0 + r, jb = j0 + kc * PC;
            float v[PC];
#pragma unroll
            for (int e = 0; e < PC; ++e)
                v[e] = (w < P.n_walkers && jb + e < NO) ? S.b32[(size_t)w * NO + jb + e] : 0.0f;
            put_row<BF16>(sA, tile_off<BF16>(r, kc * PC), v);
        }
        // kernel tile: NC tau rows x 32 bins (TF32: the precomputed split tables; BF16: the
        // FP32 table split here), written the same way
        for (int q = tid; q < NC * RC; q += kThreads) {
            const int r = q % NC, kc = q / NC;
            const uint32_t off = tile_off<BF16>(r, kc * PC);
            if constexpr (BF16) {
                float v[PC];
#pragma unroll
                for (int e = 0; e < PC; ++e) {
                    const int j = j0 + kc * PC + e;
                    v[e] = j < NO ? P.Khat32[(size_t)j * PAD + i0 + r] : 0.0f;
                }
                put_row<BF16>(sB, off, v);
            } else {
                const size_t g = (size_t)(i0 + r) * NOP + j0 + kc * PC;   // 16-byte aligned: NOP % 32 == 0
                *reinterpret_cast<float4 *>(sB[0] + off) = *reinterpret_cast<const float4 *>(P.Khi32 + g);
                *reinterpret_cast<float4 *>(sB[1] + off) = *reinterpret_cast<const float4 *>(P.Klo32 + g);
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (*abort_flag) break;
        if (tid == 0 && !(P.wait_test && t == 0)) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            for (int ks = 0; ks < F::kSteps; ++ks) {
                const uint32_t koff = (uint32_t)ks * 2 * kLBO;   // 32 bytes of K = two core matrices
                uint64_t a[F::kPieces], b[F::kPieces];
#pragma unroll
                for (int q = 0; q < F::kPieces; ++q) {
                    a[q] = smem_desc<BF16>(smem_u32(sA[q]) + koff);
                    b[q] = smem_desc<BF16>(smem_u32(sB[q]) + koff);
                }
                const uint32_t first = ks > 0 ? 1u : 0u;
                mma<BF16>(tmem, a[0], b[0], idesc, first);                // main term
                mma<BF16>(tmem + kCorrCol, a[0], b[1], idesc, first);     // corrections
                mma<BF16>(tmem + kCorrCol, a[1], b[0], idesc, 1u);
                if constexpr (BF16) {
                    mma<BF16>(tmem + kCorrCol, a[0], b[2], idesc, 1u);
                    mma<BF16>(tmem + kCorrCol, a[1], b[1], idesc, 1u);
                    mma<BF16>(tmem + kCorrCol, a[2], b[0], idesc, 1u);
                }
            }
            mma_commit(mbar_a);
        }
        // all threads wait until the MMAs have read the tiles and written the accumulators
        if (!mbar_wait(mbar_a, phase, spin)) {
            if (tid == 0) atomicExch(status, 1);
            *abort_flag = 1;   // benign race: every writer stores 1
        }
        phase ^= 1u;
        __syncthreads();
        if (*abort_flag) {
            // give the MMAs in flight one more bounded wait before the tensor memory is freed
            if (tid == 0) mbar_wait(mbar_a, phase ^ 1u, spin);
            __syncthreads();
            break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        // drain this tile's partial sums into the float pairs
        const uint32_t lane_base = (uint32_t)(32 * quarter) << 16;
#pragma unroll
        for (int c = 0; c < CS; c += 4) {
            uint32_t vm[4], vc[4];
            tmem_ld4(tmem + lane_base + (uint32_t)(slice * CS + c), vm);
            tmem_ld4(tmem + lane_base + kCorrCol + (uint32_t)(slice * CS + c), vc);
#pragma unroll
            for (int e = 0; e < 4; ++e)
                two_sum_add(acc_hi[c + e], acc_lo[c + e], __uint_as_float(vm[e]) + __uint_as_float(vc[e]));
        }
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();   // accumulators drained before the next tile's MMAs overwrite them
    }
    if (!*abort_flag) {
        const int w = w0 + 32 * quarter + lane;
        if (w < P.n_walkers) {
#pragma unroll
            for (int c = 0; c < CS; ++c) {
                const int i = i0 + slice * CS + c;
                const double model = (double)acc_hi[c] + (double)acc_lo[c];
                const double r = i < P.n_tau ? P.Fhat64[i] - model : 0.0;
                S.R32[(size_t)w * PAD + i] = (float)r;
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols));
}

// chi2 = sum_i R_i^2 (FP64) from the stored residual; one warp per walker.
__global__ void resync_chi2_kernel(DevProblem P, DevState S) {
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

template <bool BF16>
size_t tc_smem_bytes(int nc) {
    using F = Fmt<BF16>;
    return (size_t)F::kPieces * ((size_t)kM * kKT + (size_t)nc * kKT) * F::kElem + 64;
}

template <int NC, bool BF16>
cudaError_t launch_nc(const DevProblem &P, const DevState &S, int *status, cudaStream_t st) {
    const size_t smem = tc_smem_bytes<BF16>(NC);
    cudaError_t e =
        cudaFuncSetAttribute(resync_tc_kernel<NC, BF16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const dim3 grid((P.n_walkers + kM - 1) / kM, P.n_tau_pad / NC);
    resync_tc_kernel<NC, BF16><<<grid, kThreads, smem, st>>>(P, S, status);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    resync_chi2_kernel<<<(P.n_walkers * 32 + 255) / 256, 256, 0, st>>>(P, S);
    return cudaGetLastError();
}

template <bool BF16>
cudaError_t launch_tc(const DevProblem &P, const DevState &S, int *status, cudaStream_t st) {
    const int pad = P.n_tau_pad;
    for (int nc = 128; nc >= 16; nc -= 16) {
        if (pad % nc) continue;
        if (P.tc_cols > 0 && nc != P.tc_cols) continue;
        switch (nc) {
            case 128: return launch_nc<128, BF16>(P, S, status, st);
            case 112: return launch_nc<112, BF16>(P, S, status, st);
            case 96: return launch_nc<96, BF16>(P, S, status, st);
            case 80: return launch_nc<80, BF16>(P, S, status, st);
            case 64: return launch_nc<64, BF16>(P, S, status, st);
            case 48: return launch_nc<48, BF16>(P, S, status, st);
            case 32: return launch_nc<32, BF16>(P, S, status, st);
            case 16: return launch_nc<16, BF16>(P, S, status, st);
            default: break;
        }
    }
    return cudaErrorInvalidValue;
}

}  // namespace

// Columns per block: P.tc_cols if set (a multiple of 16 dividing n_tau_pad, <= 128), else
// the widest such width.  Every width gives the same result bit for bit: each column's sum
// runs over the same tiles in the same order.
cudaError_t launch_resync_tc(const DevProblem &P, const DevState &S, int *status, bool bf16, cudaStream_t st) {
    // the BF16 x6 recomputation runs as the tensor-copy pipeline of resync_tma.cu
    if (bf16) return cudaErrorInvalidValue;
    return launch_tc<false>(P, S, status, st);
}

}  // namespace sail
