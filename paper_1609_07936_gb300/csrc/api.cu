// Host side of libsail: argument checks, the FP64 tables of Sec. 2.1-2.2, the start spectrum,
// the workspace layout and the block loop of Sec. 3 (sweeps -> residual recomputation ->
// imprinted branching -> statistics).  Compiled with -ffp-contract=off: host arithmetic
// rounds every product and sum on its own.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/sail.h"
#include "sail_internal.cuh"

using namespace sail;

namespace {

thread_local std::string g_err;

int fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

}  // namespace

int sail::set_error(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

namespace {

int cuda_fail(cudaError_t e, const char *what) {
    return fail(SAIL_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define SAIL_CUDA(call, what)                      \
    do {                                           \
        cudaError_t e_ = (call);                   \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

constexpr double kPi = 3.14159265358979323846;
// largest weighted model term (max Khat_ij * A) and weighted datum an FP32 state accepts: their
// squares summed over 512 tau points stay below 1e33, far inside FP32's range
constexpr double kFp32TermMax = 1e15;

size_t align_up(size_t v) { return (v + 255) & ~size_t(255); }

struct Layout {
    size_t Khat64, Khat32, Fhat64, Fhat32, x64, beta32, rgap32, Qhi32, Qlo32, x4_32, mrho32, Khi32, Klo32, Tsweep, a0, R0;
    size_t status;
    size_t a64, b32, g2, R64, R32, chi2, acc_prev, hash, n_acc, n_pos, guard;
    size_t acc_trace, m_trace, delta_trace;
    size_t m, zero_l, donor_l, n_pairs, delta, counters, bz, bxi, cand, cand_Z, ctl;
    size_t mean, err, R_mean, chi2_mean, n_used, cut;
    size_t pr_walker, pr_p, pr_s, pr_eps, pr_delta, pr_ok;
    size_t tma_a, tma_b;     // pre-tiled BF16 pieces of the spectra and the kernel table (resync kind 2)
    size_t chi2_all;         // chi2 of the whole population (sail_branch_solve)
    size_t total;
    int max_events;
};

Layout make_layout(int n_tau, int n_omega, const sail_params &p) {
    Layout L{};
    const size_t W = (size_t)p.n_walkers, NO = (size_t)n_omega;
    const size_t PAD = (size_t)((n_tau + 31) / 32 * 32);
    size_t off = 0;
    auto take = [&](size_t bytes) { const size_t at = off; off = align_up(off + (bytes ? bytes : 1)); return at; };
    L.Khat64 = take(NO * PAD * 8);
    L.Khat32 = take(NO * PAD * 4);
    L.Fhat64 = take(PAD * 8);
    L.Fhat32 = take(PAD * 4);
    L.x64 = take(NO * 8);
    L.beta32 = take(NO * 4);
    L.rgap32 = take(NO * 4);
    L.Qhi32 = take((NO + 31) / 32 * PAD * 4);
    L.Qlo32 = take(32 * PAD * 4);
    const size_t NOP = (NO + 31) / 32 * 32;
    L.Khi32 = take(PAD * NOP * 4);
    L.Klo32 = take(PAD * NOP * 4);
    L.status = take(4);
    L.Tsweep = take((size_t)p.n_sweeps * 8);
    L.a0 = take(NO * 8);
    L.R0 = take(PAD * 8);
    if (p.precision == SAIL_PREC_FP64) {
        L.a64 = take(W * NO * 8);
        L.R64 = take(W * PAD * 8);
    } else {
        L.b32 = take(W * NO * 4);
        L.g2 = take(W * 2 * 4);
        L.R32 = take(W * PAD * 4);
    }
    if (p.precision == SAIL_PREC_FP32 && p.resync_kind == 2) {
        L.tma_a = take(tma_spectra_bytes(p.n_walkers, n_omega));
        L.tma_b = take(tma_table_bytes((int)PAD, n_omega));
    }
    L.chi2 = take(W * 8);
    L.acc_prev = take(W * 4);
    L.hash = take(W * 8);
    L.n_acc = take(W * 8);
    L.n_pos = take(W * 8);
    L.guard = take(16);
    L.max_events = p.n_sweeps / (p.sweeps_per_block > 0 ? p.sweeps_per_block : 1) + 1;
    if (p.trace) {
        L.acc_trace = take((size_t)p.n_sweeps * W * 4);
        L.m_trace = take((size_t)L.max_events * W * 4);
        L.delta_trace = take((size_t)L.max_events * 8);
    }
    // branching scratch: this handle's walkers, or the whole population of a shard
    const size_t WB = std::max(W, (size_t)p.walker_total);
    L.m = take(WB * 4);
    L.zero_l = take(WB * 4);
    L.donor_l = take(WB * 4);
    L.n_pairs = take(4);
    L.delta = take(8);
    L.bz = take(WB * 8);
    L.bxi = take(WB * 8);
    L.chi2_all = take(WB * 8);
    L.cand = take(128 * 8);
    L.cand_Z = take(128 * 4);
    L.ctl = take(64);
    L.counters = take(sizeof(BlockCounters));
    L.mean = take(NO * 8);
    L.err = take(NO * 8);
    L.R_mean = take(PAD * 8);
    L.chi2_mean = take(8);
    L.n_used = take(4);
    L.cut = take(8);
    L.pr_walker = take((size_t)kProbeMax * 4);
    L.pr_p = take((size_t)kProbeMax * 4);
    L.pr_s = take((size_t)kProbeMax * 4);
    L.pr_eps = take((size_t)kProbeMax * 8);
    L.pr_delta = take((size_t)kProbeMax * 8);
    L.pr_ok = take((size_t)kProbeMax * 4);
    L.x4_32 = take(NO * 16);
    L.mrho32 = take(PAD * 4);
    L.total = off;
    return L;
}

int check_params(int n_tau, int n_omega, const sail_params *p) {
    if (!p) return fail(SAIL_EINVAL, "params is NULL");
    if (n_tau < 1 || n_tau > kMaxTau) return fail(SAIL_EINVAL, "n_tau must be in [1, %d]", kMaxTau);
    if (n_omega < 2 || n_omega > (1 << 20)) return fail(SAIL_EINVAL, "n_omega must be in [2, 2^20]");
    if (p->n_walkers < 1 || p->n_walkers > kMaxWalkers)
        return fail(SAIL_EINVAL, "n_walkers must be in [1, %d]", kMaxWalkers);
    if (p->precision != SAIL_PREC_FP64 && p->precision != SAIL_PREC_FP32)
        return fail(SAIL_EINVAL, "unknown precision %d", p->precision);
    if (p->n_sweeps < 1 || p->sweeps_per_block < 1 || p->resync_every < 1)
        return fail(SAIL_EINVAL, "n_sweeps, sweeps_per_block and resync_every must be >= 1");
    if (!(p->T_start > 0) || !(p->T_end > 0) || !std::isfinite(p->T_start) || !std::isfinite(p->T_end))
        return fail(SAIL_EINVAL, "temperatures must be finite and > 0");
    if (!(p->T_end_abs >= 0) || !std::isfinite(p->T_end_abs)) return fail(SAIL_EINVAL, "T_end_abs must be finite, >= 0");
    if (!(p->T_start_abs >= 0) || !std::isfinite(p->T_start_abs))
        return fail(SAIL_EINVAL, "T_start_abs must be finite, >= 0");
    if (p->walker_offset < 0 || p->walker_total < 0 || p->walker_total > kMaxWalkers ||
        (p->walker_total > 0 && p->walker_offset + p->n_walkers > p->walker_total))
        return fail(SAIL_EINVAL, "a shard needs 0 <= walker_offset, offset + n_walkers <= walker_total <= %d",
                    kMaxWalkers);
    if (p->shared_bins > 1 && p->walker_offset % p->shared_bins != 0)
        return fail(SAIL_EINVAL, "walker_offset must be a multiple of shared_bins");
    if (!(p->branch_fraction >= 0 && p->branch_fraction < 1)) return fail(SAIL_EINVAL, "branch_fraction must be in [0, 1)");
    if (!(p->imprint_t >= 0 && p->imprint_t <= 1)) return fail(SAIL_EINVAL, "imprint_t must be in [0, 1]");
    if (!(p->y_p > 0 && p->y_p <= 1) || !(p->y_m >= 1) || !(p->y_min > 0 && p->y_min <= 1))
        return fail(SAIL_EINVAL, "amplitude heuristic needs 0 < p <= 1, m >= 1, 0 < y_min <= 1");
    if (!(p->move_scale < 1) || std::isnan(p->move_scale)) return fail(SAIL_EINVAL, "move_scale must be < 1");
    if (!std::isfinite(p->B)) return fail(SAIL_EINVAL, "B must be given (Sec. 2.2)");
    if (!(p->avg_chi2_factor >= 1)) return fail(SAIL_EINVAL, "avg_chi2_factor must be >= 1");
    if (p->resync_kind < 0 || p->resync_kind > 3) return fail(SAIL_EINVAL, "resync_kind must be 0, 1, 2 or 3");
    if (p->sweep_lanes != 0 && p->sweep_lanes != 8 && p->sweep_lanes != 16)
        return fail(SAIL_EINVAL, "sweep_lanes must be 0, 8 or 16");
    if (p->sweep_lanes == 8 && n_tau > 256) return fail(SAIL_EINVAL, "sweep_lanes = 8 needs n_tau <= 256");
    if (p->schedule_kind != SAIL_SCHEDULE_GEOMETRIC && p->schedule_kind != SAIL_SCHEDULE_SELF_COOLING)
        return fail(SAIL_EINVAL, "unknown schedule_kind %d", p->schedule_kind);
    if (p->adaptive_branching != 0 && p->adaptive_branching != 1) return fail(SAIL_EINVAL, "adaptive_branching must be 0 or 1");
    if (!std::isfinite(p->cool_begin) || !std::isfinite(p->freeze_begin))
        return fail(SAIL_EINVAL, "cool_begin and freeze_begin must be finite");
    if (!(p->smooth_s >= 0.0 && p->smooth_s < 0.5)) return fail(SAIL_EINVAL, "smooth_s must be in [0, 0.5)");
    if (p->index_walk_len < 0 || p->index_walk_len > 7) return fail(SAIL_EINVAL, "index_walk_len must be in [0, 7]");
    if (!(p->walk_uniform >= 0.0 && p->walk_uniform <= 1.0)) return fail(SAIL_EINVAL, "walk_uniform must be in [0, 1]");
    if (p->hastings != 0 && p->hastings != 1) return fail(SAIL_EINVAL, "hastings must be 0 or 1");
    if (p->hastings && p->index_walk_len > 0)
        return fail(SAIL_EINVAL, "hastings needs uniform bins (index_walk_len = 0): the walk's bin choice "
                                 "depends on the state, and its ratio is not part of the correction");
    if (p->shared_bins != 0 && p->shared_bins != 1 && p->shared_bins != 2 && p->shared_bins != 4 &&
        p->shared_bins != 8)
        return fail(SAIL_EINVAL, "shared_bins must be 0, 1, 2, 4 or 8");
    if (p->shared_bins > 1 && p->index_walk_len > 0)
        return fail(SAIL_EINVAL, "shared_bins needs uniform bins (index_walk_len = 0): a walk depends on "
                                 "each walker's spectrum");
    if (p->shared_bins > 1 && p->precision == SAIL_PREC_FP32 && n_tau > 32 * (p->shared_bins == 8 ? 8 : 16))
        return fail(SAIL_EINVAL, "shared_bins = %d needs n_tau <= %d in FP32", p->shared_bins,
                    p->shared_bins == 8 ? 256 : 512);
    if (p->sweep_loop < 0 || p->sweep_loop > 2) return fail(SAIL_EINVAL, "sweep_loop must be 0, 1 or 2");
    if (p->fp64_accept < 0 || p->fp64_accept > 2) return fail(SAIL_EINVAL, "fp64_accept must be 0, 1 or 2");
    if (p->fp64_accept && (p->precision != SAIL_PREC_FP32 || p->index_walk_len > 0 || p->hastings || p->shared_bins > 1))
        return fail(SAIL_EINVAL, "fp64_accept needs FP32 precision, uniform bins, the Metropolis test and own bins");
    if (p->n_walkers > 1 && p->branching && p->n_walkers > kMaxWalkers)
        return fail(SAIL_EINVAL, "branching supports at most %d walkers", kMaxWalkers);
    return SAIL_OK;
}

}  // namespace

struct sail_ctx {
    sail_params prm;
    int n_tau, n_omega, pad;
    double dw, A, B, lambda0, chi2_0;
    cudaStream_t stream;
    char *ws;
    size_t ws_bytes;
    Layout L;
    DevProblem P;
    DevState S;
    BranchScratch Bs;
    std::vector<double> T;   // temperature table (host copy)
    int sweeps_done, blocks_done, events;
    long long launches, moves;
    unsigned long long acc_seen, pos_seen;
    // protocol against the sawtooth instability (self-cooling, adaptive branching)
    unsigned long long acc_before;  // accepted moves of all walkers before the current block
    double acc_ref;          // acceptance of the first block (< 0 until known)
    double T_freeze;         // smallest residue when the freeze-out began (< 0 until then)
    std::vector<double> chi2_host;
    TmaPlan tma;             // resync kind 2: tensor maps of the pre-tiled operands
    int *status;             // device status word: nonzero after a timed-out device wait
    bool ahead_auto;         // FP32 sweep_loop 0 with enough walkers: the loop follows the rejections
    double pos_frac_last = -1.0;   // positivity-rejected share of the last block's proposals
    bool converged;          // chi2 of the averaged spectrum reached target_chi2
    double chi2_of_mean;
    // optional per-kernel timing: event pairs recorded around launches, read at block ends
    struct Timed { cudaEvent_t a, b; int kind; };
    std::vector<Timed> timed;
    int n_timed;
    double ms[3];
    long long n_kind[3];
};

namespace {

enum { kSweep = 0, kResync = 1, kBranch = 2 };

// Positivity-rejected share of a block's proposals from which the automatic move loop takes the
// look-ahead loop for the next block (measured on the paper-scale problem: look-ahead +12% at
// 40% rejections, one move at a time 6% faster at 22-27%).
constexpr double kAheadMinPos = 0.30;

// The move loop of the next block: the automatic choice follows the last block's positivity
// rejections (see sail_anneal); explicit choices and walker counts below the threshold keep the
// create-time choice.
int sweep_ahead_next(const sail_ctx *h) {
    if (h->ahead_auto && h->pos_frac_last >= 0.0) return h->pos_frac_last >= kAheadMinPos ? 1 : 0;
    return h->P.ahead;
}

// A named NVTX range around the host calls that enqueue one phase of the schedule (sweep,
// residual recomputation, branching, batched sweep segment): a profiler attached to the process
// shows the phases on the host timeline next to their kernels; without one it costs a branch.
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range &) = delete;
    Range &operator=(const Range &) = delete;
};

int timed_begin(sail_ctx *h) {
    if (!h->prm.timing) return -1;
    if (h->n_timed == (int)h->timed.size()) {
        sail_ctx::Timed t{};
        if (cudaEventCreate(&t.a) != cudaSuccess || cudaEventCreate(&t.b) != cudaSuccess) return -1;
        h->timed.push_back(t);
    }
    const int k = h->n_timed++;
    cudaEventRecord(h->timed[k].a, h->stream);
    return k;
}

void timed_end(sail_ctx *h, int k, int kind) {
    if (k < 0) return;
    cudaEventRecord(h->timed[k].b, h->stream);
    h->timed[k].kind = kind;
}

// after a stream synchronisation: fold the recorded pairs into the totals
void timed_collect(sail_ctx *h) {
    for (int k = 0; k < h->n_timed; ++k) {
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, h->timed[k].a, h->timed[k].b) == cudaSuccess) {
            h->ms[h->timed[k].kind] += ms;
            h->n_kind[h->timed[k].kind] += 1;
        }
    }
    h->n_timed = 0;
}

}  // namespace

extern "C" {

void sail_default_params(sail_params *p) {
    if (!p) return;
    std::memset(p, 0, sizeof *p);
    p->n_walkers = 1024;
    p->precision = SAIL_PREC_FP32;
    p->n_sweeps = 20000;
    p->sweeps_per_block = 100;
    p->resync_every = 50;
    p->branching = 1;
    p->T_start = 10.0;
    p->T_end = 1e-9;
    p->branch_fraction = 0.25;
    p->imprint_t = 0.1;
    p->move_scale = 0.0;
    p->y_p = 1.0;
    p->y_m = 2.0;
    p->y_min = 1e-4;
    p->A = NAN;
    p->B = NAN;
    p->avg_chi2_factor = 1.5;
    p->target_chi2 = 0.0;
    p->seed = 0;
    p->trace = 0;
    p->schedule_kind = SAIL_SCHEDULE_GEOMETRIC;
    p->adaptive_branching = 0;
    p->cool_begin = 0.1;
    p->freeze_begin = 0.5;
    p->smooth_s = 0.0;
}

const char *sail_last_error(void) { return g_err.c_str(); }

int sail_workspace_size(int n_tau, int n_omega, const sail_params *p, size_t *bytes) {
    if (!bytes) return fail(SAIL_EINVAL, "bytes is NULL");
    if (!p) return fail(SAIL_EINVAL, "params is NULL");
    sail_params q = *p;
    if (!std::isfinite(q.B)) q.B = 0.0;  // size does not depend on B
    const int rc = check_params(n_tau, n_omega, &q);
    if (rc) return rc;
    *bytes = make_layout(n_tau, n_omega, *p).total;
    return SAIL_OK;
}

int sail_create(sail_t *out, const double *tau, const double *F, const double *sigma, int n_tau,
                const double *omega, int n_omega, const sail_params *p, void *d_workspace, size_t ws_bytes,
                void *stream) {
    if (!out || !tau || !F || !sigma || !omega) return fail(SAIL_EINVAL, "NULL array argument");
    *out = nullptr;
    int rc = check_params(n_tau, n_omega, p);
    if (rc) return rc;
    if (!d_workspace) return fail(SAIL_EINVAL, "workspace is NULL");
    if (((uintptr_t)d_workspace & 255) != 0) return fail(SAIL_EINVAL, "workspace must be 256-byte aligned");
    const Layout L = make_layout(n_tau, n_omega, *p);
    if (ws_bytes < L.total) return fail(SAIL_ENOMEM, "workspace has %zu bytes, needs %zu", ws_bytes, L.total);

    // ---- grid and data (Sec. 2.1): equal bins of width dw starting at 0, centres x_j
    const double dw = (omega[n_omega - 1] - omega[0]) / (double)(n_omega - 1);
    if (!(dw > 0)) return fail(SAIL_EINVAL, "omega must increase");
    for (int j = 0; j < n_omega; ++j)
        if (!(std::fabs(omega[j] - (j + 0.5) * dw) <= 1e-9 * dw * (j + 1)))
            return fail(SAIL_EINVAL, "omega[%d] is not the centre of bin %d of equal bins from 0", j, j);
    for (int i = 0; i < n_tau; ++i) {
        if (!(tau[i] >= 0) || !std::isfinite(tau[i])) return fail(SAIL_EINVAL, "tau[%d] must be finite and >= 0", i);
        if (!(sigma[i] > 0) || !std::isfinite(sigma[i])) return fail(SAIL_EINVAL, "sigma[%d] must be finite and > 0", i);
        if (!std::isfinite(F[i])) return fail(SAIL_EINVAL, "F[%d] is not finite", i);
    }
    // a uniform tau grid (tau_i = tau_0 + i dtau, dtau >= 0) lets the 8-lane sweep form its
    // kernel columns from one factor value per four tau points (Eq. efficient-correlation-model
    // along tau); a decreasing grid is not taken (its powers e^{-j dw e dtau} would grow with j)
    const double dtau = n_tau > 1 ? (tau[n_tau - 1] - tau[0]) / (double)(n_tau - 1) : 0.0;
    bool uniform_tau = dtau >= 0.0;
    for (int i = 0; i < n_tau; ++i)
        if (!(std::fabs(tau[i] - (tau[0] + (double)i * dtau)) <= 1e-12 * std::max(1.0, std::fabs(tau[n_tau - 1]))))
            uniform_tau = false;
    if (p->precision == SAIL_PREC_FP32 && p->sweep_lanes == 8 && !uniform_tau)
        return fail(SAIL_EINVAL, "sweep_lanes = 8 needs a uniform tau grid (tau_i = tau_0 + i dtau)");
    double A = p->A;
    const double B = p->B;
    if (std::isnan(A)) {
        // Sec. 2.2: F(0) = c_0 A with c_0 = dw / 2 pi
        int i0 = -1;
        for (int i = 0; i < n_tau; ++i) if (tau[i] == 0.0) { i0 = i; break; }
        if (i0 < 0) return fail(SAIL_EINVAL, "A = NaN needs a point at tau = 0");
        A = F[i0] / (dw / (2.0 * kPi));
    }
    if (!(A > 0) || !std::isfinite(A)) return fail(SAIL_EINVAL, "A must be finite and > 0");
    const double x0 = omega[0], xN = omega[n_omega - 1];
    if (!(B / A > x0 && B / A < xN))
        return fail(SAIL_EINVAL, "B/A = %g lies outside the bin centres (%g, %g)", B / A, x0, xN);

    const int PAD = (n_tau + 31) / 32 * 32;
    const size_t NO = (size_t)n_omega;
    // lanes per walker of the FP32 sweep: 8 (the quad-compact column tables) on a uniform tau
    // grid of at most 256 points whose tables fit in shared memory, else 16
    int lanes = p->sweep_lanes;
    if (p->precision == SAIL_PREC_FP32) {
        DevProblem probe{};
        probe.n_omega = n_omega;
        probe.n_tau_pad = PAD;
        int dev = 0, smem_max = 0;
        const bool got = cudaGetDevice(&dev) == cudaSuccess &&
                         cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) == cudaSuccess;
        if (lanes == 0) {
            probe.lanes = 8;
            lanes = (PAD <= 256 && uniform_tau && (!got || sweep_fp32_table_bytes(probe) <= (size_t)smem_max)) ? 8 : 16;
        }
        probe.lanes = lanes;
        if (got && sweep_fp32_table_bytes(probe) > (size_t)smem_max)
            return fail(SAIL_EINVAL, "FP32 sweep tables need %zu bytes of shared memory, the device has %d",
                        sweep_fp32_table_bytes(probe), smem_max);
    }
    if (lanes == 0) lanes = PAD <= 256 && uniform_tau ? 8 : 16;
    // ---- weighted bin-integrated kernel, Eq. (correlation-model): column-major [j][i]
    std::vector<double> K64(NO * PAD, 0.0), F64(PAD, 0.0);
    std::vector<float> K32(NO * PAD, 0.0f), F32(PAD, 0.0f), beta(NO);
    for (int i = 0; i < n_tau; ++i) {
        for (int j = 0; j < n_omega; ++j) {
            double Kij;
            if (tau[i] == 0.0) Kij = dw / (2.0 * kPi);
            else Kij = std::exp(-(double)j * dw * tau[i]) * (-std::expm1(-dw * tau[i])) / (2.0 * kPi * tau[i]);
            K64[(size_t)j * PAD + i] = Kij / sigma[i];
            K32[(size_t)j * PAD + i] = (float)(Kij / sigma[i]);
        }
        F64[i] = F[i] / sigma[i];
        F32[i] = (float)F64[i];
    }
    for (int j = 0; j < n_omega; ++j) beta[j] = (float)(B - A * omega[j]);
    if (p->precision == SAIL_PREC_FP32) {
        // FP32 state: a single term Khat_ij a_j of the model is at most max Khat * A, and a move's
        // residual change and its square summed over tau must stay inside FP32's range (3.4e38)
        double kmax = 0.0, fmax = 0.0;
        for (size_t q = 0; q < NO * PAD; ++q) kmax = std::max(kmax, K64[q]);
        for (int i = 0; i < n_tau; ++i) fmax = std::max(fmax, std::fabs(F64[i]));
        if (!(kmax * A <= kFp32TermMax) || !(fmax <= kFp32TermMax))
            return fail(SAIL_EINVAL, "weighted data too large for FP32 state: max Khat * A = %g, max |F / sigma| = %g "
                                     "(limit %g; sigma too small for the kernel's range, use FP64)",
                        kmax * A, fmax, kFp32TermMax);
    }
    // FP32 sweep tables: Khat_{i,32h+l} = Khat_{i,32h} q_i^l (Eq. efficient-correlation-model)
    const int NH = (n_omega + 31) / 32;
    std::vector<float> Qhi((size_t)NH * PAD, 0.0f), Qlo((size_t)32 * PAD, 0.0f), rgap(NO, 0.0f);
    for (int h = 0; h < NH; ++h)
        for (int i = 0; i < n_tau; ++i) Qhi[(size_t)h * PAD + i] = (float)K64[(size_t)(32 * h) * PAD + i];
    for (int l = 0; l < 32; ++l)
        for (int i = 0; i < n_tau; ++i) Qlo[(size_t)l * PAD + i] = (float)std::exp(-(double)l * dw * tau[i]);
    for (int k = 1; k < n_omega; ++k) rgap[k] = (float)(1.0 / ((double)k * dw));
    // uniform tau: Khat_{i0+e,j} = Khat_{i0,j} rho_{i0+e} X_j^e with i0 a multiple of 4,
    // X_j = e^{-j dw dtau} and rho_i = Khat_{i,0} / Khat_{i0,0} (the bin integral's factor over
    // sigma); the tables hold X_j^e in FP64 rounded once, and -rho
    std::vector<float> x4(NO * 4, 0.0f), mrho(PAD, 0.0f);
    if (uniform_tau) {
        for (int j = 0; j < n_omega; ++j)
            for (int e = 0; e < 4; ++e) x4[(size_t)j * 4 + e] = (float)std::exp(-(double)j * dw * (double)e * dtau);
        for (int i = 0; i < n_tau; ++i) mrho[i] = (float)(-(K64[i] / K64[i & ~3]));
    }
    // tensor-core resync tables, K-major [i][j]: Khi = Khat cut to TF32, Klo = the remainder
    const int NOP = (n_omega + 31) / 32 * 32;
    std::vector<float> Khi((size_t)PAD * NOP, 0.0f), Klo((size_t)PAD * NOP, 0.0f);
    for (int i = 0; i < n_tau; ++i)
        for (int j = 0; j < n_omega; ++j) {
            const double k64 = K64[(size_t)j * PAD + i];
            uint32_t bits;
            const float f = (float)k64;
            std::memcpy(&bits, &f, 4);
            bits &= 0xFFFFE000u;
            float hi;
            std::memcpy(&hi, &bits, 4);
            Khi[(size_t)i * NOP + j] = hi;
            Klo[(size_t)i * NOP + j] = (float)(k64 - (double)hi);
        }

    // ---- start spectrum: largest entropy with sum a = A and sum a x = B, a_j ~ exp(-lambda x_j)
    const double target = B / A, xc = 0.5 * (x0 + xN), span = xN - x0;
    double lo = -700.0 / span, hi = 700.0 / span;
    for (int it = 0; it < 400; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        double s0 = 0.0, s1 = 0.0;
        for (int j = 0; j < n_omega; ++j) {
            const double wgt = std::exp(-mid * (omega[j] - xc));
            s0 += wgt;
            s1 += wgt * omega[j];
        }
        if (s1 / s0 > target) lo = mid; else hi = mid;
    }
    const double lambda = 0.5 * (lo + hi);
    std::vector<double> a0(NO);
    double s0 = 0.0;
    for (int j = 0; j < n_omega; ++j) { a0[j] = std::exp(-lambda * (omega[j] - xc)); s0 += a0[j]; }
    for (int j = 0; j < n_omega; ++j) a0[j] = A * a0[j] / s0;
    // residual and residue of the start spectrum (unit of T and chi2, Sec. 3)
    std::vector<double> R0(PAD, 0.0);
    double chi2_0 = 0.0;
    for (int i = 0; i < n_tau; ++i) {
        double model = 0.0;
        for (int j = 0; j < n_omega; ++j) model += K64[(size_t)j * PAD + i] * a0[j];
        R0[i] = F64[i] - model;
        chi2_0 += R0[i] * R0[i];
    }
    // temperature of every sweep: the geometric schedule in units of chi2_0, or block 0 of the
    // self-cooling one at chi2_0 (later blocks are set as the anneal reaches them)
    std::vector<double> T(p->n_sweeps);
    const double T_end_rel = p->T_end_abs > 0 ? p->T_end_abs / chi2_0 : p->T_end;
    const double T_start_rel = p->T_start_abs > 0 ? p->T_start_abs / chi2_0 : p->T_start;
    for (int n = 0; n < p->n_sweeps; ++n) {
        if (p->schedule_kind == SAIL_SCHEDULE_SELF_COOLING) {
            T[n] = n < p->sweeps_per_block ? chi2_0 : NAN;
            continue;
        }
        const double t = p->n_sweeps > 1 ? (double)n / (double)(p->n_sweeps - 1) : 0.0;
        T[n] = chi2_0 * (T_start_rel * std::pow(T_end_rel / T_start_rel, t));
    }

    sail_ctx *h = new sail_ctx();
    h->prm = *p;
    h->prm.A = A;
    h->n_tau = n_tau;
    h->n_omega = n_omega;
    h->pad = PAD;
    h->dw = dw;
    h->A = A;
    h->B = B;
    h->lambda0 = lambda;
    h->chi2_0 = chi2_0;
    h->stream = (cudaStream_t)stream;
    h->ws = (char *)d_workspace;
    h->ws_bytes = ws_bytes;
    h->L = L;
    h->T = T;
    h->acc_before = 0;
    h->acc_ref = -1.0;
    h->T_freeze = -1.0;
    char *ws = h->ws;
    DevProblem &P = h->P;
    P.n_tau = n_tau;
    P.n_omega = n_omega;
    P.n_walkers = p->n_walkers;
    P.n_tau_pad = PAD;
    P.n_sweeps = p->n_sweeps;
    P.A = A;
    P.B = B;
    P.dw = dw;
    P.move_scale = p->move_scale;
    P.y_p = p->y_p;
    P.y_m = p->y_m;
    P.y_min = p->y_min;
    P.seed = p->seed;
    P.Khat64 = (const double *)(ws + L.Khat64);
    P.Khat32 = (const float *)(ws + L.Khat32);
    P.Fhat64 = (const double *)(ws + L.Fhat64);
    P.Fhat32 = (const float *)(ws + L.Fhat32);
    P.x64 = (const double *)(ws + L.x64);
    P.beta32 = (const float *)(ws + L.beta32);
    P.rgap32 = (const float *)(ws + L.rgap32);
    P.Qhi32 = (const float *)(ws + L.Qhi32);
    P.Qlo32 = (const float *)(ws + L.Qlo32);
    P.x4_32 = (const float *)(ws + L.x4_32);
    P.mrho32 = (const float *)(ws + L.mrho32);
    P.Khi32 = (const float *)(ws + L.Khi32);
    P.Klo32 = (const float *)(ws + L.Klo32);
    P.n_omega_pad = NOP;
    P.wait_test = p->wait_test;
    P.lanes = lanes;
    P.walk_len = p->index_walk_len;
    P.walk_rho = p->walk_uniform;
    P.hastings = p->hastings;
    P.shared_bins = p->shared_bins > 1 ? p->shared_bins : 0;
    P.walker_base = p->walker_offset;
    P.fp64_accept = p->fp64_accept;
    {
        // the look-ahead loop pays where several warps share each scheduler (4096 walkers on
        // 152 SMs: +12%); with few walkers per SM its longer chain per move costs more (1500:
        // -14%)
        int dev = 0, sms = 1;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        P.ahead = p->sweep_loop == 2 ? 1 : p->sweep_loop == 1 ? 0 : (p->n_walkers >= 16 * sms ? 1 : 0);
        h->ahead_auto = p->sweep_loop == 0 && P.ahead == 1;
    }
    h->status = (int *)(ws + L.status);
    P.Tsweep = (const double *)(ws + L.Tsweep);
    DevState &S = h->S;
    S.a64 = p->precision == SAIL_PREC_FP64 ? (double *)(ws + L.a64) : nullptr;
    S.R64 = p->precision == SAIL_PREC_FP64 ? (double *)(ws + L.R64) : nullptr;
    S.b32 = p->precision == SAIL_PREC_FP32 ? (float *)(ws + L.b32) : nullptr;
    S.g2 = p->precision == SAIL_PREC_FP32 ? (float *)(ws + L.g2) : nullptr;
    S.R32 = p->precision == SAIL_PREC_FP32 ? (float *)(ws + L.R32) : nullptr;
    S.chi2 = (double *)(ws + L.chi2);
    S.acc_prev = (int *)(ws + L.acc_prev);
    S.hash = (unsigned long long *)(ws + L.hash);
    S.n_acc = (unsigned long long *)(ws + L.n_acc);
    S.n_pos = (unsigned long long *)(ws + L.n_pos);
    S.guard = (unsigned long long *)(ws + L.guard);
    S.acc_trace = p->trace ? (int *)(ws + L.acc_trace) : nullptr;
    BranchScratch &Bs = h->Bs;
    Bs.m = (int *)(ws + L.m);
    Bs.zero_l = (int *)(ws + L.zero_l);
    Bs.donor_l = (int *)(ws + L.donor_l);
    Bs.n_pairs = (int *)(ws + L.n_pairs);
    Bs.delta = (double *)(ws + L.delta);
    Bs.m_trace = p->trace ? (int *)(ws + L.m_trace) : nullptr;
    Bs.delta_trace = p->trace ? (double *)(ws + L.delta_trace) : nullptr;
    Bs.z = (double *)(ws + L.bz);
    Bs.xi = (double *)(ws + L.bxi);
    Bs.cand = (double *)(ws + L.cand);
    Bs.cand_Z = (int *)(ws + L.cand_Z);
    Bs.ctl = (void *)(ws + L.ctl);

    cudaStream_t st = h->stream;
    auto up = [&](size_t off, const void *src, size_t bytes) {
        return cudaMemcpyAsync(ws + off, src, bytes, cudaMemcpyHostToDevice, st);
    };
    cudaError_t e = cudaSuccess;
    std::vector<double> x(omega, omega + n_omega);
    if (e == cudaSuccess) e = up(L.Khat64, K64.data(), K64.size() * 8);
    if (e == cudaSuccess) e = up(L.Khat32, K32.data(), K32.size() * 4);
    if (e == cudaSuccess) e = up(L.Fhat64, F64.data(), F64.size() * 8);
    if (e == cudaSuccess) e = up(L.Fhat32, F32.data(), F32.size() * 4);
    if (e == cudaSuccess) e = up(L.x64, x.data(), NO * 8);
    if (e == cudaSuccess) e = up(L.beta32, beta.data(), NO * 4);
    if (e == cudaSuccess) e = up(L.rgap32, rgap.data(), NO * 4);
    if (e == cudaSuccess) e = up(L.Qhi32, Qhi.data(), Qhi.size() * 4);
    if (e == cudaSuccess) e = up(L.Qlo32, Qlo.data(), Qlo.size() * 4);
    if (e == cudaSuccess) e = up(L.x4_32, x4.data(), x4.size() * 4);
    if (e == cudaSuccess) e = up(L.mrho32, mrho.data(), mrho.size() * 4);
    if (e == cudaSuccess) e = up(L.Khi32, Khi.data(), Khi.size() * 4);
    if (e == cudaSuccess) e = up(L.Klo32, Klo.data(), Klo.size() * 4);
    if (e == cudaSuccess) e = cudaMemsetAsync(ws + L.status, 0, 4, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(ws + L.guard, 0, 16, st);
    if (e == cudaSuccess) e = up(L.Tsweep, T.data(), T.size() * 8);
    if (e == cudaSuccess) e = up(L.a0, a0.data(), NO * 8);
    if (e == cudaSuccess) e = up(L.R0, R0.data(), PAD * 8);
    if (e == cudaSuccess && p->trace)
        e = cudaMemsetAsync(ws + L.acc_trace, 0, (size_t)p->n_sweeps * p->n_walkers * 4, st);
    P.tma = nullptr;
    if (e == cudaSuccess && p->precision == SAIL_PREC_FP32 && p->resync_kind == 2) {
        e = tma_plan_init(h->tma, P, ws + L.tma_a, ws + L.tma_b, st);
        P.tma = &h->tma;
    }
    if (e == cudaSuccess)
        e = launch_init_state(P, S, p->precision, (const double *)(ws + L.a0), (const double *)(ws + L.R0), chi2_0, st);
    h->launches = 1;
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        delete h;
        return cuda_fail(e, "sail_create");
    }
    *out = h;
    return SAIL_OK;
}

int sail_destroy(sail_t h) {
    if (!h) return fail(SAIL_EINVAL, "NULL handle");
    cudaStreamSynchronize(h->stream);
    for (auto &t : h->timed) {
        cudaEventDestroy(t.a);
        cudaEventDestroy(t.b);
    }
    delete h;
    return SAIL_OK;
}

int sail_get_info(sail_t h, sail_info *info) {
    if (!h || !info) return fail(SAIL_EINVAL, "NULL argument");
    std::memset(info, 0, sizeof *info);
    info->n_tau = h->n_tau;
    info->n_omega = h->n_omega;
    info->n_walkers = h->prm.n_walkers;
    info->n_tau_pad = h->pad;
    info->precision = h->prm.precision;
    info->sweeps_done = h->sweeps_done;
    info->blocks_done = h->blocks_done;
    info->n_sweeps = h->prm.n_sweeps;
    info->chi2_0 = h->chi2_0;
    info->d_omega = h->dw;
    info->A = h->A;
    info->B = h->B;
    info->lambda0 = h->lambda0;
    info->kernel_launches = h->launches;
    info->workspace_bytes = h->L.total;
    info->sweep_ms = h->ms[kSweep];
    info->resync_ms = h->ms[kResync];
    info->branch_ms = h->ms[kBranch];
    info->sweep_launches = h->n_kind[kSweep];
    info->resync_launches = h->n_kind[kResync];
    info->branch_launches = h->n_kind[kBranch];
    info->moves = h->moves;
    info->sweep_lanes = h->prm.precision == SAIL_PREC_FP32 ? h->P.lanes : 0;
    info->sweep_ahead = h->prm.precision == SAIL_PREC_FP32 ? sweep_ahead_next(h) : 0;
    if (h->prm.fp64_accept) {
        unsigned long long g[2] = {0, 0};
        SAIL_CUDA(cudaMemcpyAsync(g, h->ws + h->L.guard, 16, cudaMemcpyDeviceToHost, h->stream), "D2H");
        SAIL_CUDA(cudaStreamSynchronize(h->stream), "info sync");
        info->fp64_rechecks = (long long)g[0];
        info->fp64_flips = (long long)g[1];
    }
    return SAIL_OK;
}

namespace {

int average_to_host(sail_t h, double *mean, double *err, int *n_used, double *chi2_mean) {
    char *ws = h->ws;
    int l = 0;
    cudaError_t e = launch_average(h->P, h->S, h->prm.precision, h->prm.avg_chi2_factor,
                                   (double *)(ws + h->L.mean), (double *)(ws + h->L.err), (int *)(ws + h->L.n_used),
                                   (double *)(ws + h->L.cut), (double *)(ws + h->L.R_mean),
                                   (double *)(ws + h->L.chi2_mean), h->stream, &l);
    h->launches += l;
    if (e != cudaSuccess) return cuda_fail(e, "average");
    const size_t NO = (size_t)h->n_omega;
    if (mean) SAIL_CUDA(cudaMemcpyAsync(mean, ws + h->L.mean, NO * 8, cudaMemcpyDeviceToHost, h->stream), "average D2H");
    if (err) SAIL_CUDA(cudaMemcpyAsync(err, ws + h->L.err, NO * 8, cudaMemcpyDeviceToHost, h->stream), "average D2H");
    int nu = 0;
    double c2 = 0;
    SAIL_CUDA(cudaMemcpyAsync(&nu, ws + h->L.n_used, 4, cudaMemcpyDeviceToHost, h->stream), "average D2H");
    SAIL_CUDA(cudaMemcpyAsync(&c2, ws + h->L.chi2_mean, 8, cudaMemcpyDeviceToHost, h->stream), "average D2H");
    SAIL_CUDA(cudaStreamSynchronize(h->stream), "average sync");
    if (n_used) *n_used = nu;
    if (chi2_mean) *chi2_mean = c2;
    return SAIL_OK;
}

}  // namespace

}  // extern "C"

namespace {

// ---- one block of the schedule (Sec. 3), in steps shared by single and batched annealing ----
struct BlockPending {
    int n_begin, block_end;
    bool branched;
    BlockCounters bc;
    int dev_status;
    double delta;
    int zeros;
};

bool handle_active(const sail_ctx *h) { return h->sweeps_done < h->prm.n_sweeps && !h->converged; }

int block_end_of(const sail_ctx *h) {
    const int k = h->prm.sweeps_per_block;
    return std::min((h->sweeps_done / k + 1) * k, h->prm.n_sweeps);
}

int next_resync(const sail_ctx *h, int n, int block_end) {
    return std::min((n / h->prm.resync_every + 1) * h->prm.resync_every, block_end);
}

// residual recomputation after sweeps [n, next) ran
int segment_done(sail_ctx *h, int n, int next) {
    const sail_params &p = h->prm;
    Range range("sail.resync");
    const int tk = timed_begin(h);
    int l = 0;
    const cudaError_t e = launch_resync(h->P, h->S, p.precision, 1, p.resync_kind, h->status, h->stream, &l);
    timed_end(h, tk, kResync);
    if (e != cudaSuccess) return cuda_fail(e, "resync launch");
    h->launches += l;
    h->moves += (long long)(next - n) * p.n_walkers * h->n_omega;
    return SAIL_OK;
}

// branching and statistics at the block end; the read-backs are queued, not waited for
// Self-cooling schedule (Sec. self-cooling): T of block b >= 1 from block b-1's mean residue
// cbar and smallest residue cmin (sail_params.schedule_kind documents the phases).
double self_cooling_T(int b, int n_blocks, int b_cool, int b_freeze, double cbar, double cmin, double T_final,
                      double *T_freeze) {
    if (b < b_cool) return cbar;
    if (b < b_freeze) {
        const double x = (double)(b - b_cool + 1) / (double)(b_freeze - b_cool);
        return std::pow(cbar, 1.0 - x) * std::pow(cmin, x);
    }
    if (*T_freeze < 0.0) *T_freeze = cmin;
    if (!(*T_freeze > T_final)) return *T_freeze;
    const double y = (double)(b - b_freeze + 1) / (double)(n_blocks - b_freeze);
    return *T_freeze * std::pow(T_final / *T_freeze, y);
}

void cooling_blocks(int n_blocks, double cool_begin, double freeze_begin, int *b_cool, int *b_freeze) {
    int bc = (int)std::floor(cool_begin * (double)n_blocks + 0.5);
    int bf = (int)std::floor(freeze_begin * (double)n_blocks + 0.5);
    bc = std::min(std::max(bc, 0), n_blocks);
    bf = std::min(std::max(bf, bc), n_blocks);
    *b_cool = bc;
    *b_freeze = bf;
}

int block_tail(sail_ctx *h, BlockPending &b) {
    const sail_params &p = h->prm;
    const int k = p.sweeps_per_block;
    cudaStream_t st = h->stream;
    h->sweeps_done = b.block_end;
    b.delta = 0.0;
    b.zeros = 0;
    b.dev_status = 0;
    const bool full = (b.block_end % k) == 0;
    b.branched = p.branching && p.n_walkers > 1 && full;
    // the protocol against the sawtooth instability: the finished block's acceptance and
    // residue statistics (after its residual recomputation, before branching)
    const bool cooling = p.schedule_kind == SAIL_SCHEDULE_SELF_COOLING;
    double scale = 1.0, cbar = 0.0, cmin = 0.0;
    if (full && (cooling || p.adaptive_branching)) {
        BlockCounters bc{};
        cudaError_t e = launch_block_stats(h->P, h->S, (BlockCounters *)(h->ws + h->L.counters), st);
        h->launches += 1;
        if (e != cudaSuccess) return cuda_fail(e, "stats launch");
        SAIL_CUDA(cudaMemcpyAsync(&bc, h->ws + h->L.counters, sizeof bc, cudaMemcpyDeviceToHost, st), "stats D2H");
        if (cooling) {
            h->chi2_host.resize(p.n_walkers);
            SAIL_CUDA(cudaMemcpyAsync(h->chi2_host.data(), h->S.chi2, (size_t)p.n_walkers * 8, cudaMemcpyDeviceToHost, st),
                      "chi2 D2H");
        }
        SAIL_CUDA(cudaStreamSynchronize(st), "block statistics");
        const double acc = (double)(bc.acc - h->acc_before) / ((double)k * (double)p.n_walkers * (double)h->n_omega);
        h->acc_before = bc.acc;
        if (p.adaptive_branching) {
            if (h->acc_ref < 0.0) h->acc_ref = acc;
            scale = (h->acc_ref > 0.0 && acc < h->acc_ref) ? acc / h->acc_ref : 1.0;
        }
        if (cooling) {
            cmin = h->chi2_host[0];
            for (int w = 0; w < p.n_walkers; ++w) {
                cbar += h->chi2_host[w];
                if (h->chi2_host[w] < cmin) cmin = h->chi2_host[w];
            }
            cbar /= (double)p.n_walkers;
        }
    }
    if (b.branched) {
        Range range("sail.branch");
        int l = 0;
        const int tk = timed_begin(h);
        const cudaError_t e = launch_branch(h->P, h->S, h->Bs, p.precision, b.block_end / k - 1,
                                            p.branch_fraction * scale, p.imprint_t * scale, h->events, st, &l);
        timed_end(h, tk, kBranch);
        h->launches += l;
        if (e != cudaSuccess) return cuda_fail(e, "branch launch");
        h->events += 1;
    }
    if (full && p.smooth_s > 0.0) {
        // smoothing (Sec. smoothing), then every walker's residual and chi2 anew
        Range range("sail.smooth");
        int l = 0;
        const int tk = timed_begin(h);
        cudaError_t e = launch_smooth(h->P, h->S, p.precision, p.smooth_s, st);
        if (e == cudaSuccess)
            e = launch_resync(h->P, h->S, p.precision, p.precision == SAIL_PREC_FP32 ? 1 : 0, p.resync_kind, h->status,
                              st, &l);
        timed_end(h, tk, kBranch);
        h->launches += 1 + l;
        if (e != cudaSuccess) return cuda_fail(e, "smoothing launch");
    }
    if (full && cooling && b.block_end < p.n_sweeps) {
        const int n_blocks = (p.n_sweeps + k - 1) / k;
        int bcool = 0, bfreeze = 0;
        cooling_blocks(n_blocks, p.cool_begin, p.freeze_begin, &bcool, &bfreeze);
        const double T_final = p.T_end_abs > 0 ? p.T_end_abs : p.T_end * h->chi2_0;
        const double Tn = self_cooling_T(b.block_end / k, n_blocks, bcool, bfreeze, cbar, cmin, T_final, &h->T_freeze);
        const int q1 = std::min(b.block_end + k, p.n_sweeps);
        for (int q = b.block_end; q < q1; ++q) h->T[q] = Tn;
        SAIL_CUDA(cudaMemcpyAsync(h->ws + h->L.Tsweep + (size_t)b.block_end * 8, h->T.data() + b.block_end,
                                  (size_t)(q1 - b.block_end) * 8, cudaMemcpyHostToDevice, st), "temperature H2D");
    }
    const cudaError_t e = launch_block_stats(h->P, h->S, (BlockCounters *)(h->ws + h->L.counters), st);
    h->launches += 1;
    if (e != cudaSuccess) return cuda_fail(e, "stats launch");
    SAIL_CUDA(cudaMemcpyAsync(&b.bc, h->ws + h->L.counters, sizeof b.bc, cudaMemcpyDeviceToHost, st), "stats D2H");
    SAIL_CUDA(cudaMemcpyAsync(&b.dev_status, h->status, 4, cudaMemcpyDeviceToHost, st), "stats D2H");
    if (b.branched) {
        SAIL_CUDA(cudaMemcpyAsync(&b.delta, h->ws + h->L.delta, 8, cudaMemcpyDeviceToHost, st), "stats D2H");
        SAIL_CUDA(cudaMemcpyAsync(&b.zeros, h->ws + h->L.n_pairs, 4, cudaMemcpyDeviceToHost, st), "stats D2H");
    }
    return SAIL_OK;
}

// after the stream synchronisation: statistics, counters, target check
int block_finish(sail_ctx *h, const BlockPending &b, sail_block_stats *out) {
    const sail_params &p = h->prm;
    timed_collect(h);
    if (b.dev_status) return fail(SAIL_ETIMEOUT, "a device-side wait timed out (status %d)", b.dev_status);
    if (out) {
        sail_block_stats &s = *out;
        std::memset(&s, 0, sizeof s);
        const double proposed = (double)(b.block_end - b.n_begin) * p.n_walkers * h->n_omega;
        s.block = h->blocks_done;
        s.sweep_end = b.block_end;
        s.T = h->T[b.block_end - 1];
        s.chi2_min = b.bc.chi2_min;
        s.chi2_mean = b.bc.chi2_sum / p.n_walkers;
        s.acceptance = (double)(b.bc.acc - h->acc_seen) / proposed;
        s.positivity_rejected = (double)(b.bc.pos - h->pos_seen) / proposed;
        s.branch_delta = b.delta;
        s.branch_zeros = b.zeros;
    }
    {
        const double proposed = (double)(b.block_end - b.n_begin) * p.n_walkers * h->n_omega;
        h->pos_frac_last = (double)(b.bc.pos - h->pos_seen) / proposed;
    }
    h->acc_seen = b.bc.acc;
    h->pos_seen = b.bc.pos;
    h->blocks_done += 1;
    if (p.target_chi2 > 0) {
        double c2 = 0;
        const int rc = average_to_host(h, nullptr, nullptr, nullptr, &c2);
        if (rc) return rc;
        h->chi2_of_mean = c2;
        h->converged = c2 <= p.target_chi2;
    }
    return SAIL_OK;
}

}  // namespace

extern "C" {

int sail_anneal(sail_t h, int max_blocks, sail_block_stats *stats, int *n_done) {
    if (!h) return fail(SAIL_EINVAL, "NULL handle");
    if (max_blocks < 0) return fail(SAIL_EINVAL, "max_blocks < 0");
    const sail_params &p = h->prm;
    int done = 0;
    cudaStream_t st = h->stream;
    while (done < max_blocks && handle_active(h)) {
        // automatic move loop: the look-ahead loop pays for its proposal bookkeeping by
        // skipping positivity-rejected moves, so it runs while the last block rejected at least
        // kAheadMinPos of its proposals (both loops draw the same proposals and take the same
        // decisions)
        h->P.ahead = sweep_ahead_next(h);
        BlockPending b{};
        b.n_begin = h->sweeps_done;
        b.block_end = block_end_of(h);
        for (int n = b.n_begin; n < b.block_end;) {
            const int next = next_resync(h, n, b.block_end);
            const int tk = timed_begin(h);
            cudaError_t e;
            {
                Range range("sail.sweep");
                e = p.precision == SAIL_PREC_FP64 ? launch_sweep_fp64(h->P, h->S, n, next, st)
                                                  : launch_sweep_fp32(h->P, h->S, n, next, st);
            }
            timed_end(h, tk, kSweep);
            h->launches += 1;
            if (e != cudaSuccess) return cuda_fail(e, "sweep launch");
            const int rc = segment_done(h, n, next);
            if (rc) return rc;
            n = next;
        }
        int rc = block_tail(h, b);
        if (rc) return rc;
        SAIL_CUDA(cudaStreamSynchronize(st), "block sync");
        rc = block_finish(h, b, stats ? &stats[done] : nullptr);
        if (rc) return rc;
        done += 1;
    }
    if (n_done) *n_done = done;
    if (p.target_chi2 > 0 && !h->converged && h->sweeps_done >= p.n_sweeps) return SAIL_NOT_CONVERGED;
    return SAIL_OK;
}

int sail_average(sail_t h, double *S_mean, double *S_err, int *n_used, double *chi2_of_mean) {
    if (!h || !S_mean) return fail(SAIL_EINVAL, "NULL argument");
    return average_to_host(h, S_mean, S_err, n_used, chi2_of_mean);
}

int sail_get_state(sail_t h, double *a, double *R, double *chi2, int *acc_prev, uint64_t *hash) {
    if (!h) return fail(SAIL_EINVAL, "NULL handle");
    const size_t W = (size_t)h->prm.n_walkers, NO = (size_t)h->n_omega, PAD = (size_t)h->pad;
    cudaStream_t st = h->stream;
    char *ws = h->ws;
    const bool f64 = h->prm.precision == SAIL_PREC_FP64;
    std::vector<float> fbuf;
    std::vector<double> rbuf;
    if (a) {
        if (f64) SAIL_CUDA(cudaMemcpyAsync(a, ws + h->L.a64, W * NO * 8, cudaMemcpyDeviceToHost, st), "D2H");
        else { fbuf.resize(W * NO); SAIL_CUDA(cudaMemcpyAsync(fbuf.data(), ws + h->L.b32, W * NO * 4, cudaMemcpyDeviceToHost, st), "D2H"); }
    }
    std::vector<float> rf;
    if (R) {
        if (f64) { rbuf.resize(W * PAD); SAIL_CUDA(cudaMemcpyAsync(rbuf.data(), ws + h->L.R64, W * PAD * 8, cudaMemcpyDeviceToHost, st), "D2H"); }
        else { rf.resize(W * PAD); SAIL_CUDA(cudaMemcpyAsync(rf.data(), ws + h->L.R32, W * PAD * 4, cudaMemcpyDeviceToHost, st), "D2H"); }
    }
    if (chi2) SAIL_CUDA(cudaMemcpyAsync(chi2, ws + h->L.chi2, W * 8, cudaMemcpyDeviceToHost, st), "D2H");
    if (acc_prev) SAIL_CUDA(cudaMemcpyAsync(acc_prev, ws + h->L.acc_prev, W * 4, cudaMemcpyDeviceToHost, st), "D2H");
    if (hash) SAIL_CUDA(cudaMemcpyAsync(hash, ws + h->L.hash, W * 8, cudaMemcpyDeviceToHost, st), "D2H");
    SAIL_CUDA(cudaStreamSynchronize(st), "get_state sync");
    if (a && !f64) for (size_t q = 0; q < W * NO; ++q) a[q] = (double)fbuf[q];
    if (R) {
        for (size_t w = 0; w < W; ++w)
            for (int i = 0; i < h->n_tau; ++i)
                R[w * h->n_tau + i] = f64 ? rbuf[w * PAD + i] : (double)rf[w * PAD + i];
    }
    return SAIL_OK;
}

int sail_set_state(sail_t h, const double *a, const int *acc_prev) {
    if (!h || !a) return fail(SAIL_EINVAL, "NULL argument");
    const size_t W = (size_t)h->prm.n_walkers, NO = (size_t)h->n_omega;
    cudaStream_t st = h->stream;
    char *ws = h->ws;
    std::vector<float> fbuf, g;
    if (h->prm.precision == SAIL_PREC_FP64) {
        SAIL_CUDA(cudaMemcpyAsync(ws + h->L.a64, a, W * NO * 8, cudaMemcpyHostToDevice, st), "H2D");
    } else {
        fbuf.resize(W * NO);
        for (size_t q = 0; q < W * NO; ++q) fbuf[q] = (float)a[q];
        g.resize(2 * W);
        for (size_t w = 0; w < W; ++w) { g[2 * w] = 1.0f; g[2 * w + 1] = 0.0f; }
        SAIL_CUDA(cudaMemcpyAsync(ws + h->L.b32, fbuf.data(), W * NO * 4, cudaMemcpyHostToDevice, st), "H2D");
        SAIL_CUDA(cudaMemcpyAsync(ws + h->L.g2, g.data(), W * 2 * 4, cudaMemcpyHostToDevice, st), "H2D");
    }
    if (acc_prev) SAIL_CUDA(cudaMemcpyAsync(ws + h->L.acc_prev, acc_prev, W * 4, cudaMemcpyHostToDevice, st), "H2D");
    int l = 0;
    SAIL_CUDA(launch_resync(h->P, h->S, h->prm.precision, 0, h->prm.resync_kind, h->status, st, &l), "resync launch");
    h->launches += l;
    SAIL_CUDA(cudaStreamSynchronize(st), "set_state sync");
    return SAIL_OK;
}

int sail_get_trace(sail_t h, int *acc, int *m, double *delta, int *n_events) {
    if (!h) return fail(SAIL_EINVAL, "NULL handle");
    if (!h->prm.trace) return fail(SAIL_ESTATE, "handle was created without trace");
    const size_t W = (size_t)h->prm.n_walkers;
    cudaStream_t st = h->stream;
    if (acc && h->sweeps_done > 0)
        SAIL_CUDA(cudaMemcpyAsync(acc, h->ws + h->L.acc_trace, (size_t)h->sweeps_done * W * 4, cudaMemcpyDeviceToHost, st), "D2H");
    if (m && h->events > 0)
        SAIL_CUDA(cudaMemcpyAsync(m, h->ws + h->L.m_trace, (size_t)h->events * W * 4, cudaMemcpyDeviceToHost, st), "D2H");
    if (delta && h->events > 0)
        SAIL_CUDA(cudaMemcpyAsync(delta, h->ws + h->L.delta_trace, (size_t)h->events * 8, cudaMemcpyDeviceToHost, st), "D2H");
    SAIL_CUDA(cudaStreamSynchronize(st), "trace sync");
    if (n_events) *n_events = h->events;
    return SAIL_OK;
}

namespace {

// Checkpoint layout: a header, the host-side schedule state, then device regions in a fixed
// order (each region's bytes as the workspace holds them).
struct CkptHeader {
    char magic[8];
    int version, n_tau, n_omega, n_walkers, precision, n_sweeps, sweeps_per_block, resync_every, trace;
    int schedule_kind, branching;
    uint64_t seed;
    int sweeps_done, blocks_done, events, converged;
    long long moves;
    unsigned long long acc_seen, pos_seen, acc_before;
    double acc_ref, T_freeze, chi2_of_mean;
};

struct CkptRegion {
    size_t off, bytes;
};

std::vector<CkptRegion> ckpt_regions(const sail_ctx *h) {
    const size_t W = (size_t)h->prm.n_walkers, NO = (size_t)h->n_omega, PAD = (size_t)h->pad;
    const Layout &L = h->L;
    std::vector<CkptRegion> r;
    if (h->prm.precision == SAIL_PREC_FP64) {
        r.push_back({L.a64, W * NO * 8});
        r.push_back({L.R64, W * PAD * 8});
    } else {
        r.push_back({L.b32, W * NO * 4});
        r.push_back({L.g2, W * 2 * 4});
        r.push_back({L.R32, W * PAD * 4});
    }
    r.push_back({L.chi2, W * 8});
    r.push_back({L.acc_prev, W * 4});
    r.push_back({L.hash, W * 8});
    r.push_back({L.n_acc, W * 8});
    r.push_back({L.n_pos, W * 8});
    r.push_back({L.guard, 16});
    r.push_back({L.Tsweep, (size_t)h->prm.n_sweeps * 8});
    if (h->prm.trace) {
        r.push_back({L.acc_trace, (size_t)h->prm.n_sweeps * W * 4});
        r.push_back({L.m_trace, (size_t)L.max_events * W * 4});
        r.push_back({L.delta_trace, (size_t)L.max_events * 8});
    }
    return r;
}

size_t ckpt_bytes(const sail_ctx *h) {
    size_t n = sizeof(CkptHeader) + (size_t)h->prm.n_sweeps * 8;   // header and the host T table
    for (const CkptRegion &r : ckpt_regions(h)) n += r.bytes;
    return n;
}

CkptHeader ckpt_header(const sail_ctx *h) {
    CkptHeader c{};
    std::memcpy(c.magic, "SAILCKPT", 8);
    c.version = 1;
    c.n_tau = h->n_tau;
    c.n_omega = h->n_omega;
    c.n_walkers = h->prm.n_walkers;
    c.precision = h->prm.precision;
    c.n_sweeps = h->prm.n_sweeps;
    c.sweeps_per_block = h->prm.sweeps_per_block;
    c.resync_every = h->prm.resync_every;
    c.trace = h->prm.trace;
    c.schedule_kind = h->prm.schedule_kind;
    c.branching = h->prm.branching;
    c.seed = h->prm.seed;
    c.sweeps_done = h->sweeps_done;
    c.blocks_done = h->blocks_done;
    c.events = h->events;
    c.converged = h->converged ? 1 : 0;
    c.moves = h->moves;
    c.acc_seen = h->acc_seen;
    c.pos_seen = h->pos_seen;
    c.acc_before = h->acc_before;
    c.acc_ref = h->acc_ref;
    c.T_freeze = h->T_freeze;
    c.chi2_of_mean = h->chi2_of_mean;
    return c;
}

}  // namespace

int sail_branch_solve(sail_t h, int n_total, const double *chi2_all, int block, double fraction, int *m,
                      double *delta, int *zero_l, int *donor_l, int *n_pairs) {
    if (!h || !chi2_all || !m || !delta || !zero_l || !donor_l || !n_pairs) return fail(SAIL_EINVAL, "NULL argument");
    const int cap = std::max(h->prm.n_walkers, h->prm.walker_total);
    if (n_total < 2 || n_total > cap) return fail(SAIL_EINVAL, "n_total must be in [2, %d] (walker_total)", cap);
    if (block < 0) return fail(SAIL_EINVAL, "block must be >= 0");
    if (!(fraction >= 0.0 && fraction < 1.0)) return fail(SAIL_EINVAL, "fraction must be in [0, 1)");
    for (int l = 0; l < n_total; ++l)
        if (!std::isfinite(chi2_all[l]) || chi2_all[l] < 0) return fail(SAIL_EINVAL, "chi2_all[%d] is not a residue", l);
    cudaStream_t st = h->stream;
    double *d_chi2 = (double *)(h->ws + h->L.chi2_all);
    SAIL_CUDA(cudaMemcpyAsync(d_chi2, chi2_all, (size_t)n_total * 8, cudaMemcpyHostToDevice, st), "solve H2D");
    DevProblem P = h->P;
    P.n_walkers = n_total;
    P.walker_base = 0;
    DevState S = h->S;
    S.chi2 = d_chi2;
    BranchScratch B = h->Bs;
    B.m_trace = nullptr;
    B.delta_trace = nullptr;
    int l = 0;
    SAIL_CUDA(launch_branch_solve(P, S, B, block, fraction, st, &l), "solve launch");
    h->launches += l;
    int np = 0;
    SAIL_CUDA(cudaMemcpyAsync(m, B.m, (size_t)n_total * 4, cudaMemcpyDeviceToHost, st), "solve D2H");
    SAIL_CUDA(cudaMemcpyAsync(delta, B.delta, 8, cudaMemcpyDeviceToHost, st), "solve D2H");
    SAIL_CUDA(cudaMemcpyAsync(&np, B.n_pairs, 4, cudaMemcpyDeviceToHost, st), "solve D2H");
    SAIL_CUDA(cudaStreamSynchronize(st), "solve sync");
    if (np > 0) {
        SAIL_CUDA(cudaMemcpyAsync(zero_l, B.zero_l, (size_t)np * 4, cudaMemcpyDeviceToHost, st), "solve D2H");
        SAIL_CUDA(cudaMemcpyAsync(donor_l, B.donor_l, (size_t)np * 4, cudaMemcpyDeviceToHost, st), "solve D2H");
        SAIL_CUDA(cudaStreamSynchronize(st), "solve sync");
    }
    *n_pairs = np;
    return SAIL_OK;
}

namespace {

int rows_index(sail_t h, int n, const int *idx, int **d_idx) {
    if (n < 0 || n > kProbeMax) return fail(SAIL_EINVAL, "n must be in [0, %d]", kProbeMax);
    for (int q = 0; q < n; ++q)
        if (idx[q] < 0 || idx[q] >= h->prm.n_walkers) return fail(SAIL_EINVAL, "idx[%d] = %d is not a walker", q, idx[q]);
    *d_idx = (int *)(h->ws + h->L.pr_walker);
    SAIL_CUDA(cudaMemcpyAsync(*d_idx, idx, (size_t)n * 4, cudaMemcpyHostToDevice, h->stream), "rows H2D");
    return SAIL_OK;
}

}  // namespace

int sail_walker_rows(sail_t h, int n, const int *idx, double *d_a_rows, double *d_R_rows) {
    if (!h || (n > 0 && (!idx || !d_a_rows || !d_R_rows))) return fail(SAIL_EINVAL, "NULL argument");
    if (n == 0) return SAIL_OK;
    int *d_idx = nullptr;
    const int rc = rows_index(h, n, idx, &d_idx);
    if (rc) return rc;
    SAIL_CUDA(launch_walker_rows(h->P, h->S, h->prm.precision, n, d_idx, d_a_rows, d_R_rows, h->stream), "rows launch");
    h->launches += 1;
    SAIL_CUDA(cudaStreamSynchronize(h->stream), "rows sync");
    return SAIL_OK;
}

int sail_imprint_rows(sail_t h, int n, const int *idx, const double *d_a_rows, const double *d_R_rows, double t) {
    if (!h || (n > 0 && (!idx || !d_a_rows || !d_R_rows))) return fail(SAIL_EINVAL, "NULL argument");
    if (!(t >= 0.0 && t <= 1.0)) return fail(SAIL_EINVAL, "t must be in [0, 1]");
    if (n == 0) return SAIL_OK;
    for (int q = 0; q < n; ++q)
        for (int r = 0; r < q; ++r)
            if (idx[r] == idx[q]) return fail(SAIL_EINVAL, "walker %d imprinted twice", idx[q]);
    int *d_idx = nullptr;
    const int rc = rows_index(h, n, idx, &d_idx);
    if (rc) return rc;
    SAIL_CUDA(launch_imprint_rows(h->P, h->S, h->prm.precision, n, d_idx, d_a_rows, d_R_rows, t, h->stream),
              "imprint launch");
    h->launches += 1;
    SAIL_CUDA(cudaStreamSynchronize(h->stream), "imprint sync");
    return SAIL_OK;
}

int sail_checkpoint_size(sail_t h, size_t *bytes) {
    if (!h || !bytes) return fail(SAIL_EINVAL, "NULL argument");
    *bytes = ckpt_bytes(h);
    return SAIL_OK;
}

int sail_checkpoint(sail_t h, void *buf, size_t bytes) {
    if (!h || !buf) return fail(SAIL_EINVAL, "NULL argument");
    if (bytes < ckpt_bytes(h)) return fail(SAIL_EINVAL, "checkpoint buffer has %zu bytes, needs %zu", bytes, ckpt_bytes(h));
    char *out = (char *)buf;
    const CkptHeader c = ckpt_header(h);
    std::memcpy(out, &c, sizeof c);
    out += sizeof c;
    std::memcpy(out, h->T.data(), (size_t)h->prm.n_sweeps * 8);
    out += (size_t)h->prm.n_sweeps * 8;
    for (const CkptRegion &r : ckpt_regions(h)) {
        SAIL_CUDA(cudaMemcpyAsync(out, h->ws + r.off, r.bytes, cudaMemcpyDeviceToHost, h->stream), "checkpoint D2H");
        out += r.bytes;
    }
    SAIL_CUDA(cudaStreamSynchronize(h->stream), "checkpoint sync");
    return SAIL_OK;
}

int sail_restore(sail_t h, const void *buf, size_t bytes) {
    if (!h || !buf) return fail(SAIL_EINVAL, "NULL argument");
    if (bytes < sizeof(CkptHeader)) return fail(SAIL_EINVAL, "checkpoint too short");
    CkptHeader c;
    std::memcpy(&c, buf, sizeof c);
    const CkptHeader mine = ckpt_header(h);
    if (std::memcmp(c.magic, "SAILCKPT", 8) != 0 || c.version != 1) return fail(SAIL_EINVAL, "not a checkpoint");
    if (c.n_tau != mine.n_tau || c.n_omega != mine.n_omega || c.n_walkers != mine.n_walkers ||
        c.precision != mine.precision || c.n_sweeps != mine.n_sweeps || c.sweeps_per_block != mine.sweeps_per_block ||
        c.resync_every != mine.resync_every || c.trace != mine.trace || c.schedule_kind != mine.schedule_kind ||
        c.branching != mine.branching || c.seed != mine.seed)
        return fail(SAIL_EINVAL, "checkpoint of a different problem or schedule");
    if (bytes < ckpt_bytes(h)) return fail(SAIL_EINVAL, "checkpoint has %zu bytes, needs %zu", bytes, ckpt_bytes(h));
    if (c.sweeps_done < 0 || c.sweeps_done > c.n_sweeps || c.events < 0 || c.events > h->L.max_events)
        return fail(SAIL_EINVAL, "checkpoint position out of range");
    const char *in = (const char *)buf + sizeof c;
    std::memcpy(h->T.data(), in, (size_t)h->prm.n_sweeps * 8);
    in += (size_t)h->prm.n_sweeps * 8;
    for (const CkptRegion &r : ckpt_regions(h)) {
        SAIL_CUDA(cudaMemcpyAsync(h->ws + r.off, in, r.bytes, cudaMemcpyHostToDevice, h->stream), "restore H2D");
        in += r.bytes;
    }
    SAIL_CUDA(cudaStreamSynchronize(h->stream), "restore sync");
    h->sweeps_done = c.sweeps_done;
    h->blocks_done = c.blocks_done;
    h->events = c.events;
    h->converged = c.converged != 0;
    h->moves = c.moves;
    h->acc_seen = c.acc_seen;
    h->pos_seen = c.pos_seen;
    h->acc_before = c.acc_before;
    h->acc_ref = c.acc_ref;
    h->T_freeze = c.T_freeze;
    h->chi2_of_mean = c.chi2_of_mean;
    return SAIL_OK;
}

int sail_delta_probe(sail_t h, int n, const int *walker, const int *p, const int *s, const double *eps,
                     double *delta, int *ok) {
    if (!h) return fail(SAIL_EINVAL, "NULL handle");
    if (n < 0 || n > kProbeMax) return fail(SAIL_EINVAL, "n must be in [0, %d]", kProbeMax);
    if (n == 0) return SAIL_OK;
    if (!walker || !p || !s || !eps || !delta || !ok) return fail(SAIL_EINVAL, "NULL array argument");
    for (int q = 0; q < n; ++q) {
        if (walker[q] < 0 || walker[q] >= h->prm.n_walkers || p[q] < 0 || p[q] >= h->n_omega || s[q] < 0 ||
            s[q] >= h->n_omega || p[q] == s[q] || !(std::fabs(eps[q]) < 1.0))
            return fail(SAIL_EINVAL, "proposal %d out of range", q);
    }
    cudaStream_t st = h->stream;
    char *ws = h->ws;
    SAIL_CUDA(cudaMemcpyAsync(ws + h->L.pr_walker, walker, (size_t)n * 4, cudaMemcpyHostToDevice, st), "H2D");
    SAIL_CUDA(cudaMemcpyAsync(ws + h->L.pr_p, p, (size_t)n * 4, cudaMemcpyHostToDevice, st), "H2D");
    SAIL_CUDA(cudaMemcpyAsync(ws + h->L.pr_s, s, (size_t)n * 4, cudaMemcpyHostToDevice, st), "H2D");
    SAIL_CUDA(cudaMemcpyAsync(ws + h->L.pr_eps, eps, (size_t)n * 8, cudaMemcpyHostToDevice, st), "H2D");
    SAIL_CUDA(launch_probe(h->P, h->S, h->prm.precision, n, (const int *)(ws + h->L.pr_walker),
                           (const int *)(ws + h->L.pr_p), (const int *)(ws + h->L.pr_s),
                           (const double *)(ws + h->L.pr_eps), (double *)(ws + h->L.pr_delta),
                           (int *)(ws + h->L.pr_ok), st),
              "probe launch");
    h->launches += 1;
    SAIL_CUDA(cudaMemcpyAsync(delta, ws + h->L.pr_delta, (size_t)n * 8, cudaMemcpyDeviceToHost, st), "D2H");
    SAIL_CUDA(cudaMemcpyAsync(ok, ws + h->L.pr_ok, (size_t)n * 4, cudaMemcpyDeviceToHost, st), "D2H");
    SAIL_CUDA(cudaStreamSynchronize(st), "probe sync");
    return SAIL_OK;
}

int sail_probe_read_bandwidth(const void *d_buf, size_t bytes, int reps, void *d_sink, void *stream) {
    if (!d_buf || !d_sink || reps < 1 || bytes < 16 || (bytes & 15) || ((uintptr_t)d_buf & 15))
        return fail(SAIL_EINVAL, "read probe needs a 16-byte aligned buffer of 16k bytes and reps >= 1");
    SAIL_CUDA(launch_read_probe(d_buf, bytes, reps, d_sink, (cudaStream_t)stream), "read probe launch");
    return SAIL_OK;
}

int sail_probe_smem_bandwidth(int reps, void *d_sink, void *stream, double *bytes_read) {
    if (!d_sink || !bytes_read || reps < 1) return fail(SAIL_EINVAL, "smem probe needs a sink, a byte count and reps >= 1");
    SAIL_CUDA(launch_smem_probe(reps, d_sink, (cudaStream_t)stream, bytes_read), "smem probe launch");
    return SAIL_OK;
}

int sail_philox(int n, const uint32_t *d_ctr, uint64_t seed, uint32_t *d_out, void *stream) {
    if (n < 0 || (n > 0 && (!d_ctr || !d_out))) return fail(SAIL_EINVAL, "bad arguments");
    SAIL_CUDA(launch_philox(n, d_ctr, seed, d_out, (cudaStream_t)stream), "philox launch");
    return SAIL_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- batches
namespace {

constexpr int kTuneCandidates[3] = {16, 8, 4};   // walker groups per queue item (= warps per block)

}  // namespace

struct sail_batch_ctx {
    std::vector<sail_t> h;
    cudaStream_t stream;
    char *ws;
    size_t ws_bytes;
    BatchProblem *d_probs;
    BatchItem *d_items;
    int *d_counter;
    size_t max_items;
    // a batched sweep segment launches one kernel per class of problems: lanes per walker
    // (16 or 8) times move-loop variant (plain, walk, Hastings); class = 3 * (lanes == 8) + mode
    static constexpr int kClasses = 6;
    size_t smem[kClasses];     // shared memory of each class's kernel: its problems' largest tables
    cudaStream_t aux[kClasses - 1];   // further streams: the classes' kernels run side by side
    cudaEvent_t fork, join[kClasses - 1];
    int autotune;
    int item_pairs;            // chosen mapping
    int tune_next;             // next candidate to try (autotune), or 3 when done
    double tune_ns[3];         // device ns per walker-move of each candidate
    double last_ns;
    long long sweep_launches, last_seg_moves;
    cudaEvent_t ev0, ev1;
    // tensor-core tile width tuning per n_tau_pad class: candidates, trial times
    struct TcTune { int pad; int cand[8]; int n_cand; int next; double ns[8]; int chosen; };
    std::vector<TcTune> tc;
};

namespace {

size_t batch_header_bytes(int n, const sail_problem *probs) {
    size_t items = 0;
    for (int k = 0; k < n; ++k) items += (size_t)(probs[k].params.n_walkers + 1) / 2;
    return align_up((size_t)n * sizeof(BatchProblem)) + align_up(items * sizeof(BatchItem)) + 256;
}

int check_batch(int n, const sail_problem *probs) {
    if (n < 1 || !probs) return fail(SAIL_EINVAL, "a batch needs n >= 1 problems");
    for (int k = 0; k < n; ++k) {
        const sail_params &p = probs[k].params;
        if (p.precision != SAIL_PREC_FP32) return fail(SAIL_EINVAL, "problem %d: batches run FP32 precision", k);
        if (p.shared_bins > 1) return fail(SAIL_EINVAL, "problem %d: batches do not run shared bins", k);
        if (p.fp64_accept) return fail(SAIL_EINVAL, "problem %d: batches do not run fp64_accept", k);
        if (p.sweeps_per_block != probs[0].params.sweeps_per_block || p.resync_every != probs[0].params.resync_every)
            return fail(SAIL_EINVAL, "problem %d: sweeps_per_block and resync_every must match problem 0", k);
        const int rc = check_params(probs[k].n_tau, probs[k].n_omega, &p);
        if (rc) return rc;
    }
    return SAIL_OK;
}

int batch_class(const DevProblem &P) { return 3 * (P.lanes == 8 ? 1 : 0) + sweep_mode(P); }

void batch_streams_create(sail_batch_ctx *b) {
    cudaEventCreate(&b->ev0);
    cudaEventCreate(&b->ev1);
    cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    for (int c = 0; c < sail_batch_ctx::kClasses - 1; ++c) {
        cudaEventCreateWithFlags(&b->join[c], cudaEventDisableTiming);
        cudaStreamCreateWithFlags(&b->aux[c], cudaStreamNonBlocking);
    }
}

void batch_streams_destroy(sail_batch_ctx *b) {
    cudaEventDestroy(b->ev0);
    cudaEventDestroy(b->ev1);
    cudaEventDestroy(b->fork);
    for (int c = 0; c < sail_batch_ctx::kClasses - 1; ++c) {
        cudaEventDestroy(b->join[c]);
        cudaStreamDestroy(b->aux[c]);
    }
}

// One batched sweep segment: the items of class c are count[c] consecutive items from the
// start of the class's range in the item list (classes in order); the first non-empty class
// runs on the batch stream, the others on further streams forked from and joined back into
// it.  d_counter[c] is class c's queue.
cudaError_t batch_sweep_segment(sail_batch_ctx *b, const int *count) {
    cudaStream_t st = b->stream;
    cudaError_t e = cudaSuccess;
    int used = 0;
    for (int c = 0; c < sail_batch_ctx::kClasses; ++c) used += count[c] > 0;
    if (used > 1) {
        if ((e = cudaEventRecord(b->fork, st)) != cudaSuccess) return e;
        for (int c = 0; c < used - 1; ++c)
            if ((e = cudaStreamWaitEvent(b->aux[c], b->fork, 0)) != cudaSuccess) return e;
    }
    int offset = 0, k = 0;
    for (int c = 0; c < sail_batch_ctx::kClasses; ++c) {
        if (count[c] == 0) continue;
        cudaStream_t sc = k == 0 ? st : b->aux[k - 1];
        e = launch_sweep_batch(b->d_probs, b->d_items + offset, count[c], b->d_counter + c, b->smem[c], b->item_pairs,
                               c >= 3 ? 8 : 16, c % 3, sc);
        if (e != cudaSuccess) return e;
        offset += count[c];
        ++k;
    }
    for (int c = 0; c < used - 1; ++c) {
        if ((e = cudaEventRecord(b->join[c], b->aux[c])) != cudaSuccess) return e;
        if ((e = cudaStreamWaitEvent(st, b->join[c], 0)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace

extern "C" {

int sail_batch_workspace_size(int n, const sail_problem *probs, size_t *bytes) {
    if (!bytes) return fail(SAIL_EINVAL, "bytes is NULL");
    int rc = check_batch(n, probs);
    if (rc) return rc;
    size_t total = batch_header_bytes(n, probs);
    for (int k = 0; k < n; ++k) {
        size_t b = 0;
        rc = sail_workspace_size(probs[k].n_tau, probs[k].n_omega, &probs[k].params, &b);
        if (rc) return rc;
        total += align_up(b);
    }
    *bytes = total;
    return SAIL_OK;
}

int sail_batch_create(sail_batch_t *out, int n, const sail_problem *probs, int autotune, void *d_workspace,
                      size_t ws_bytes, void *stream) {
    if (!out) return fail(SAIL_EINVAL, "out is NULL");
    *out = nullptr;
    size_t need = 0;
    int rc = sail_batch_workspace_size(n, probs, &need);
    if (rc) return rc;
    if (!d_workspace || ((uintptr_t)d_workspace & 255)) return fail(SAIL_EINVAL, "workspace must be 256-byte aligned");
    if (ws_bytes < need) return fail(SAIL_ENOMEM, "batch workspace has %zu bytes, needs %zu", ws_bytes, need);
    sail_batch_ctx *b = new sail_batch_ctx();
    b->stream = (cudaStream_t)stream;
    b->ws = (char *)d_workspace;
    b->ws_bytes = ws_bytes;
    size_t off = 0;
    b->d_probs = (BatchProblem *)(b->ws + off);
    off += align_up((size_t)n * sizeof(BatchProblem));
    b->d_items = (BatchItem *)(b->ws + off);
    b->max_items = 0;
    for (int k = 0; k < n; ++k) b->max_items += (size_t)(probs[k].params.n_walkers + 1) / 2;
    off += align_up(b->max_items * sizeof(BatchItem));
    b->d_counter = (int *)(b->ws + off);
    off += 256;
    for (size_t &m : b->smem) m = 0;
    for (int k = 0; k < n; ++k) {
        size_t sub = 0;
        sail_workspace_size(probs[k].n_tau, probs[k].n_omega, &probs[k].params, &sub);
        sail_t h = nullptr;
        const sail_problem &q = probs[k];
        rc = sail_create(&h, q.tau, q.F, q.sigma, q.n_tau, q.omega, q.n_omega, &q.params, b->ws + off, sub, stream);
        if (rc) {
            for (sail_t x : b->h) sail_destroy(x);
            delete b;
            return rc;
        }
        b->h.push_back(h);
        size_t &sm = b->smem[batch_class(h->P)];
        sm = std::max(sm, sweep_fp32_table_bytes(h->P));
        off += align_up(sub);
    }
    b->autotune = autotune;
    b->item_pairs = kTuneCandidates[0];
    b->tune_next = autotune ? 0 : 3;
    b->last_ns = 0.0;
    batch_streams_create(b);
    if (autotune) {
        for (sail_t h : b->h) {
            const int pad = h->pad;
            bool seen = false;
            for (auto &t : b->tc) seen = seen || t.pad == pad;
            if (seen) continue;
            sail_batch_ctx::TcTune t{};
            t.pad = pad;
            for (int nc = 128; nc >= 16 && t.n_cand < 3; nc -= 16)
                if (pad % nc == 0) t.cand[t.n_cand++] = nc;
            t.next = 0;
            t.chosen = 0;
            b->tc.push_back(t);
        }
    }
    *out = b;
    return SAIL_OK;
}

int sail_batch_destroy(sail_batch_t b) {
    if (!b) return fail(SAIL_EINVAL, "NULL batch");
    cudaStreamSynchronize(b->stream);
    for (sail_t h : b->h) sail_destroy(h);
    batch_streams_destroy(b);
    delete b;
    return SAIL_OK;
}

int sail_batch_handle(sail_batch_t b, int k, sail_t *h) {
    if (!b || !h || k < 0 || k >= (int)b->h.size()) return fail(SAIL_EINVAL, "bad batch index");
    *h = b->h[k];
    return SAIL_OK;
}

int sail_batch_tuning(sail_batch_t b, int *item_pairs, double *ns_per_move, long long *sweep_launches) {
    if (!b) return fail(SAIL_EINVAL, "NULL batch");
    if (item_pairs) *item_pairs = b->item_pairs;
    if (ns_per_move) *ns_per_move = b->last_ns;
    if (sweep_launches) *sweep_launches = b->sweep_launches;
    return SAIL_OK;
}

}  // extern "C"

namespace {

// Runs up to max_blocks blocks for every live problem of b (empty slots are skipped).
int batch_run_blocks(sail_batch_ctx *b, int max_blocks, int *n_done) {
    const int N = (int)b->h.size();
    cudaStream_t st = b->stream;
    std::vector<BlockPending> pend(N);
    std::vector<int> cur(N), active(N);
    std::vector<BatchProblem> hp(N);
    std::vector<BatchItem> items, cls_items[sail_batch_ctx::kClasses];
    int done = 0;
    while (done < max_blocks) {
        bool any = false;
        for (int k = 0; k < N; ++k) {
            active[k] = b->h[k] != nullptr && handle_active(b->h[k]);
            if (!active[k]) continue;
            any = true;
            pend[k] = BlockPending{};
            pend[k].n_begin = b->h[k]->sweeps_done;
            pend[k].block_end = block_end_of(b->h[k]);
            cur[k] = pend[k].n_begin;
        }
        if (!any) break;
        for (;;) {
            // one segment: every problem with sweeps left in this block advances to its next resync
            for (auto &v : cls_items) v.clear();
            long long seg_moves = 0;
            for (int k = 0; k < N; ++k) {
                sail_ctx *h = b->h[k];
                hp[k].n0 = hp[k].n1 = 0;
                if (!active[k] || cur[k] >= pend[k].block_end) continue;
                hp[k].P = h->P;
                hp[k].S = h->S;
                hp[k].n0 = cur[k];
                hp[k].n1 = next_resync(h, cur[k], pend[k].block_end);
                seg_moves += (long long)(hp[k].n1 - hp[k].n0) * h->prm.n_walkers * h->n_omega;
                const int wpw = sweep_walkers_per_warp(h->P);
                const int groups = (h->prm.n_walkers + wpw - 1) / wpw;
                // walker groups per item = warps per block (at most 8 with 8 lanes per walker, 12
                // with 16)
                const int per = std::min(b->item_pairs, h->P.lanes == 8 ? 8 : 12);
                std::vector<BatchItem> &dst = cls_items[batch_class(h->P)];
                for (int lo = 0; lo < groups; lo += per) dst.push_back(BatchItem{k, lo, std::min(lo + per, groups)});
            }
            int count[sail_batch_ctx::kClasses];
            items.clear();
            for (int c = 0; c < sail_batch_ctx::kClasses; ++c) {
                count[c] = (int)cls_items[c].size();
                items.insert(items.end(), cls_items[c].begin(), cls_items[c].end());
            }
            if (items.empty()) break;
            SAIL_CUDA(cudaMemcpyAsync(b->d_probs, hp.data(), (size_t)N * sizeof(BatchProblem), cudaMemcpyHostToDevice, st),
                      "batch H2D");
            SAIL_CUDA(cudaMemcpyAsync(b->d_items, items.data(), items.size() * sizeof(BatchItem),
                                      cudaMemcpyHostToDevice, st), "batch H2D");
            cudaEventRecord(b->ev0, st);
            cudaError_t e;
            {
                Range range("sail.batch_sweep");
                e = batch_sweep_segment(b, count);
            }
            cudaEventRecord(b->ev1, st);
            if (e != cudaSuccess) return cuda_fail(e, "batched sweep launch");
            for (int k = 0; k < N; ++k) {
                if (hp[k].n1 <= hp[k].n0) continue;
                sail_ctx *h = b->h[k];
                // tensor-core tile width: try the candidates of this n_tau_pad class in turn
                cudaEvent_t t0 = nullptr, t1 = nullptr;
                sail_batch_ctx::TcTune *tt = nullptr;
                for (auto &t : b->tc)
                    if (t.pad == h->pad) tt = &t;
                if (tt && h->prm.resync_kind == 1) {
                    if (tt->next < tt->n_cand) {
                        h->P.tc_cols = tt->cand[tt->next];
                        cudaEventCreate(&t0);
                        cudaEventCreate(&t1);
                        cudaEventRecord(t0, st);
                    } else {
                        h->P.tc_cols = tt->chosen;
                    }
                }
                const int rc = segment_done(h, hp[k].n0, hp[k].n1);
                if (t0) {
                    cudaEventRecord(t1, st);
                    cudaEventSynchronize(t1);
                    float ms = 0.0f;
                    cudaEventElapsedTime(&ms, t0, t1);
                    const double per = ms * 1e6 / ((double)h->prm.n_walkers * h->n_omega * h->pad);
                    tt->ns[tt->next] = per;
                    tt->next += 1;
                    if (tt->next == tt->n_cand) {
                        int best = 0;
                        for (int c = 1; c < tt->n_cand; ++c)
                            if (tt->ns[c] < tt->ns[best]) best = c;
                        tt->chosen = tt->cand[best];
                    }
                    cudaEventDestroy(t0);
                    cudaEventDestroy(t1);
                }
                if (rc) return rc;
                cur[k] = hp[k].n1;
            }
            for (int c = 0; c < sail_batch_ctx::kClasses; ++c) b->sweep_launches += count[c] > 0;
            b->last_seg_moves = seg_moves;
            // walker-to-block mapping: time this launch, try the next candidate, keep the fastest
            if (b->tune_next < 3) {
                SAIL_CUDA(cudaEventSynchronize(b->ev1), "batch timing");
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, b->ev0, b->ev1);
                b->last_ns = seg_moves > 0 ? ms * 1e6 / (double)seg_moves : 0.0;
                b->tune_ns[b->tune_next] = b->last_ns;
                b->tune_next += 1;
                if (b->tune_next < 3) {
                    b->item_pairs = kTuneCandidates[b->tune_next];
                } else {
                    int best = 0;
                    for (int c = 1; c < 3; ++c)
                        if (b->tune_ns[c] < b->tune_ns[best]) best = c;
                    b->item_pairs = kTuneCandidates[best];
                }
            }
        }
        for (int k = 0; k < N; ++k) {
            if (!active[k]) continue;
            const int rc = block_tail(b->h[k], pend[k]);
            if (rc) return rc;
        }
        SAIL_CUDA(cudaStreamSynchronize(st), "batch block sync");
        if (b->tune_next >= 3 && b->last_seg_moves > 0) {
            float ms = 0.0f;
            if (cudaEventElapsedTime(&ms, b->ev0, b->ev1) == cudaSuccess)
                b->last_ns = ms * 1e6 / (double)b->last_seg_moves;
        }
        for (int k = 0; k < N; ++k) {
            if (!active[k]) continue;
            const int rc = block_finish(b->h[k], pend[k], nullptr);
            if (rc) return rc;
        }
        done += 1;
    }
    if (n_done) *n_done = done;
    return SAIL_OK;
}

}  // namespace

extern "C" {

int sail_batch_anneal(sail_batch_t b, int max_blocks, int *n_done) {
    if (!b) return fail(SAIL_EINVAL, "NULL batch");
    if (max_blocks < 0) return fail(SAIL_EINVAL, "max_blocks < 0");
    return batch_run_blocks(b, max_blocks, n_done);
}

}  // extern "C"

// ---------------------------------------------------------------- serving
// Continuous batching: requests wait in a FIFO; at every step the head of the queue is
// admitted while its workspace fits a free region of the server's device buffer (first fit;
// the buffer size is the admission cap) and a slot is free, one block runs for every resident
// problem through the batched sweep, and problems that reached their target chi2 or the end
// of their schedule leave, their averaged spectrum kept on the host.  A step admits only
// requests submitted before it began, so a request that arrives while a block runs joins at
// the next block boundary.  Steps are driven either by the caller (sail_server_step) or by a
// worker thread of the server (sail_server_start): submission, polling and results take a
// mutex that the block itself does not hold, so they never wait for a block to finish.
struct sail_server_ctx {
    sail_batch_ctx batch;              // slots: batch.h[k] == nullptr when free
    std::vector<size_t> slot_off, slot_size;
    std::vector<int> slot_id;
    struct Region { size_t off, size; };
    std::vector<Region> free_regions;  // sorted by offset, coalesced
    size_t data_begin;
    int sweeps_per_block, resync_every;
    long long max_pairs, resident_pairs;
    struct Request {
        int id;
        std::vector<double> tau, F, sigma, omega;
        sail_params params;
        size_t bytes;
    };
    std::deque<Request> queue;
    struct Result {
        sail_request_info info;
        std::vector<double> mean, err;
        std::vector<int> acc_trace, m_trace;
        std::vector<double> delta_trace;
        int n_omega, trace_sweeps, trace_events;
    };
    std::vector<Result> results;
    // concurrency: mu guards queue, results, completions and the counters below; step_mu makes
    // steps one at a time (the slots, regions and the batch belong to the step that holds it)
    std::mutex mu, step_mu;
    std::condition_variable cv;
    std::thread worker;
    bool worker_on = false, stop = false;
    std::deque<int> completions;       // ids retired by the worker and not yet polled
    int worker_rc = SAIL_OK;
    std::string worker_err;
    long long steps_started = 0;
    int n_resident = 0;
    int device = 0;
    std::chrono::steady_clock::time_point t0;
};

namespace {

double server_clock(const sail_server_ctx *s) {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - s->t0).count();
}

bool region_take(sail_server_ctx *s, size_t bytes, size_t *off) {
    for (size_t r = 0; r < s->free_regions.size(); ++r) {
        auto &R = s->free_regions[r];
        if (R.size >= bytes) {
            *off = R.off;
            R.off += bytes;
            R.size -= bytes;
            if (R.size == 0) s->free_regions.erase(s->free_regions.begin() + (long)r);
            return true;
        }
    }
    return false;
}

void region_give(sail_server_ctx *s, size_t off, size_t bytes) {
    auto &F = s->free_regions;
    size_t r = 0;
    while (r < F.size() && F[r].off < off) ++r;
    F.insert(F.begin() + (long)r, sail_server_ctx::Region{off, bytes});
    // coalesce with the neighbours
    if (r + 1 < F.size() && F[r].off + F[r].size == F[r + 1].off) {
        F[r].size += F[r + 1].size;
        F.erase(F.begin() + (long)r + 1);
    }
    if (r > 0 && F[r - 1].off + F[r - 1].size == F[r].off) {
        F[r - 1].size += F[r].size;
        F.erase(F.begin() + (long)r);
    }
}

// One admission / block / retirement round; the caller holds step_mu.  Retired ids go to
// completed[] (up to max_completed) and, when to_poll, to the poll queue.
int server_step(sail_server_t s, int *completed, int max_completed, int *n_completed, bool to_poll) {
    sail_batch_ctx &b = s->batch;
    const int slots = (int)b.h.size();
    long long k;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        k = ++s->steps_started;
    }
    // admission: the head of the queue while it fits (FIFO order), requests submitted before
    // this step began only
    for (;;) {
        sail_server_ctx::Request r;
        int slot = -1;
        size_t off = 0;
        {
            std::lock_guard<std::mutex> lk(s->mu);
            if (s->queue.empty()) break;
            const sail_server_ctx::Request &f = s->queue.front();
            if (s->results[f.id].info.submit_step >= k) break;
            for (int q = 0; q < slots && slot < 0; ++q)
                if (!b.h[q]) slot = q;
            const long long pairs = (f.params.n_walkers + 1) / 2;
            if (slot < 0 || s->resident_pairs + pairs > s->max_pairs || !region_take(s, f.bytes, &off)) break;
            r = std::move(s->queue.front());
            s->queue.pop_front();
        }
        sail_t h = nullptr;
        const int rc = sail_create(&h, r.tau.data(), r.F.data(), r.sigma.data(), (int)r.tau.size(), r.omega.data(),
                                   (int)r.omega.size(), &r.params, b.ws + off, r.bytes, b.stream);
        if (rc) {
            region_give(s, off, r.bytes);
            std::lock_guard<std::mutex> lk(s->mu);
            auto &res = s->results[r.id].info;
            res.state = rc;
            res.done_step = k;
            res.t_done = server_clock(s);
            if (to_poll) s->completions.push_back(r.id);
            return rc;
        }
        b.h[slot] = h;
        size_t &sm = b.smem[batch_class(h->P)];
        sm = std::max(sm, sweep_fp32_table_bytes(h->P));
        s->slot_off[slot] = off;
        s->slot_size[slot] = r.bytes;
        s->slot_id[slot] = r.id;
        s->resident_pairs += (r.params.n_walkers + 1) / 2;
        std::lock_guard<std::mutex> lk(s->mu);
        auto &res = s->results[r.id].info;
        res.state = 1;
        res.admit_step = k;
        res.t_admit = server_clock(s);
        s->n_resident += 1;
    }
    int active = 0;
    for (int q = 0; q < slots; ++q) active += b.h[q] != nullptr;
    if (active > 0) {
        const int rc = batch_run_blocks(&b, 1, nullptr);
        if (rc) return rc;
    }
    // retirement
    int nc = 0;
    for (int q = 0; q < slots; ++q) {
        sail_ctx *h = b.h[q];
        if (!h || handle_active(h)) continue;
        const int id = s->slot_id[q];
        std::vector<double> mean(h->n_omega, 0.0), err(h->n_omega, 0.0);
        int n_used = 0;
        double c2 = 0.0;
        int rc = average_to_host(h, mean.data(), err.data(), &n_used, &c2);
        if (rc) return rc;
        std::vector<int> acc, m;
        std::vector<double> dl;
        int n_ev = 0;
        if (h->prm.trace) {
            acc.resize((size_t)h->sweeps_done * h->prm.n_walkers);
            m.resize((size_t)h->events * h->prm.n_walkers);
            dl.resize((size_t)h->events);
            rc = sail_get_trace(h, acc.data(), m.data(), dl.data(), &n_ev);
            if (rc) return rc;
        }
        {
            std::lock_guard<std::mutex> lk(s->mu);
            auto &res = s->results[id];
            res.mean = std::move(mean);
            res.err = std::move(err);
            res.acc_trace = std::move(acc);
            res.m_trace = std::move(m);
            res.delta_trace = std::move(dl);
            res.trace_sweeps = h->prm.trace ? h->sweeps_done : 0;
            res.trace_events = n_ev;
            res.info.n_used = n_used;
            res.info.chi2_of_mean = c2;
            res.info.converged = h->converged ? 1 : 0;
            res.info.sweeps = h->sweeps_done;
            res.info.done_step = k;
            res.info.t_done = server_clock(s);
            res.info.state = 2;
            s->n_resident -= 1;
            if (to_poll) s->completions.push_back(id);
        }
        if (completed && nc < max_completed) completed[nc] = id;
        ++nc;
        s->resident_pairs -= (h->prm.n_walkers + 1) / 2;
        sail_destroy(h);
        b.h[q] = nullptr;
        region_give(s, s->slot_off[q], s->slot_size[q]);
        s->slot_id[q] = -1;
    }
    // the sweeps each resident request has run so far (request information between steps)
    {
        std::lock_guard<std::mutex> lk(s->mu);
        for (int q = 0; q < slots; ++q)
            if (b.h[q]) s->results[s->slot_id[q]].info.sweeps = b.h[q]->sweeps_done;
    }
    if (n_completed) *n_completed = nc;
    return SAIL_OK;
}

void server_counts(sail_server_t s, int *n_active, int *n_queued) {
    if (n_active) *n_active = s->n_resident;
    if (n_queued) *n_queued = (int)s->queue.size();
}

void server_worker(sail_server_t s) {
    cudaSetDevice(s->device);
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv.wait(lk, [s] { return s->stop || !s->queue.empty() || s->n_resident > 0; });
            if (s->stop) return;
        }
        int rc;
        {
            std::lock_guard<std::mutex> lk(s->step_mu);
            rc = server_step(s, nullptr, 0, nullptr, true);
        }
        if (rc) {
            std::lock_guard<std::mutex> lk(s->mu);
            s->worker_rc = rc;
            s->worker_err = g_err;
            return;
        }
    }
}

void server_stop_worker(sail_server_t s) {
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (!s->worker_on) return;
        s->stop = true;
    }
    s->cv.notify_all();
    s->worker.join();
    std::lock_guard<std::mutex> lk(s->mu);
    s->worker_on = false;
    s->stop = false;
}

}  // namespace

extern "C" {

int sail_server_create(sail_server_t *out, int max_resident, long long max_walkers, int sweeps_per_block,
                       int resync_every, void *d_workspace, size_t ws_bytes, void *stream) {
    if (!out) return fail(SAIL_EINVAL, "out is NULL");
    *out = nullptr;
    if (max_resident < 1 || max_walkers < 2 || sweeps_per_block < 1 || resync_every < 1)
        return fail(SAIL_EINVAL, "server needs max_resident >= 1, max_walkers >= 2 and positive periods");
    if (!d_workspace || ((uintptr_t)d_workspace & 255)) return fail(SAIL_EINVAL, "workspace must be 256-byte aligned");
    const long long max_pairs = max_walkers / 2 + max_resident;
    const size_t header = align_up((size_t)max_resident * sizeof(BatchProblem)) +
                          align_up((size_t)max_pairs * sizeof(BatchItem)) + 256;
    if (ws_bytes <= header) return fail(SAIL_ENOMEM, "server workspace smaller than its %zu-byte header", header);
    sail_server_ctx *s = new sail_server_ctx();
    sail_batch_ctx &b = s->batch;
    b.stream = (cudaStream_t)stream;
    b.ws = (char *)d_workspace;
    b.ws_bytes = ws_bytes;
    b.d_probs = (BatchProblem *)b.ws;
    b.d_items = (BatchItem *)(b.ws + align_up((size_t)max_resident * sizeof(BatchProblem)));
    b.d_counter = (int *)(b.ws + header - 256);
    b.max_items = (size_t)max_pairs;
    b.h.assign(max_resident, nullptr);
    b.autotune = 1;
    b.item_pairs = kTuneCandidates[0];
    b.tune_next = 0;
    for (size_t &m : b.smem) m = 0;
    batch_streams_create(&b);
    s->slot_off.assign(max_resident, 0);
    s->slot_size.assign(max_resident, 0);
    s->slot_id.assign(max_resident, -1);
    s->data_begin = header;
    s->free_regions.push_back(sail_server_ctx::Region{header, ws_bytes - header});
    s->sweeps_per_block = sweeps_per_block;
    s->resync_every = resync_every;
    s->max_pairs = max_walkers / 2;
    s->resident_pairs = 0;
    cudaGetDevice(&s->device);
    s->t0 = std::chrono::steady_clock::now();
    *out = s;
    return SAIL_OK;
}

int sail_server_submit(sail_server_t s, const sail_problem *req, int *id) {
    if (!s || !req || !id) return fail(SAIL_EINVAL, "NULL argument");
    const sail_params &p = req->params;
    if (p.precision != SAIL_PREC_FP32) return fail(SAIL_EINVAL, "served inversions run FP32 precision");
    if (p.shared_bins > 1) return fail(SAIL_EINVAL, "served inversions do not run shared bins");
    if (p.fp64_accept) return fail(SAIL_EINVAL, "served inversions do not run fp64_accept");
    if (p.sweeps_per_block != s->sweeps_per_block || p.resync_every != s->resync_every)
        return fail(SAIL_EINVAL, "request periods differ from the server's");
    size_t bytes = 0;
    int rc = sail_workspace_size(req->n_tau, req->n_omega, &p, &bytes);
    if (rc) return rc;
    if ((p.n_walkers + 1) / 2 > s->max_pairs) return fail(SAIL_EINVAL, "request has more walkers than the server holds");
    if (align_up(bytes) > s->batch.ws_bytes - s->data_begin) return fail(SAIL_ENOMEM, "request larger than the server");
    sail_server_ctx::Request r;
    r.tau.assign(req->tau, req->tau + req->n_tau);
    r.F.assign(req->F, req->F + req->n_tau);
    r.sigma.assign(req->sigma, req->sigma + req->n_tau);
    r.omega.assign(req->omega, req->omega + req->n_omega);
    r.params = p;
    r.bytes = align_up(bytes);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        r.id = (int)s->results.size();
        *id = r.id;
        sail_server_ctx::Result res{};
        res.n_omega = req->n_omega;
        res.info.state = 0;
        res.info.submit_step = s->steps_started;
        res.info.admit_step = -1;
        res.info.done_step = -1;
        res.info.t_submit = server_clock(s);
        res.info.t_admit = -1.0;
        res.info.t_done = -1.0;
        s->results.push_back(std::move(res));
        s->queue.push_back(std::move(r));
    }
    s->cv.notify_one();
    return SAIL_OK;
}

int sail_server_step(sail_server_t s, int *completed, int max_completed, int *n_completed, int *n_active,
                     int *n_queued) {
    if (!s) return fail(SAIL_EINVAL, "NULL server");
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->worker_on) return fail(SAIL_ESTATE, "the server's worker thread drives the steps");
    }
    int rc;
    {
        std::lock_guard<std::mutex> lk(s->step_mu);
        rc = server_step(s, completed, max_completed, n_completed, false);
    }
    std::lock_guard<std::mutex> lk(s->mu);
    server_counts(s, n_active, n_queued);
    return rc;
}

int sail_server_start(sail_server_t s) {
    if (!s) return fail(SAIL_EINVAL, "NULL server");
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->worker_on) return fail(SAIL_ESTATE, "the worker thread is already running");
    if (s->worker_rc) return fail(s->worker_rc, "the worker thread stopped on an error: %s", s->worker_err.c_str());
    cudaGetDevice(&s->device);
    s->stop = false;
    s->worker_on = true;
    s->worker = std::thread(server_worker, s);
    return SAIL_OK;
}

int sail_server_poll(sail_server_t s, int *completed, int max_completed, int *n_completed, int *n_active,
                     int *n_queued) {
    if (!s) return fail(SAIL_EINVAL, "NULL server");
    if (max_completed < 0 || (max_completed > 0 && !completed)) return fail(SAIL_EINVAL, "bad completion buffer");
    std::lock_guard<std::mutex> lk(s->mu);
    int nc = 0;
    while (nc < max_completed && !s->completions.empty()) {
        completed[nc++] = s->completions.front();
        s->completions.pop_front();
    }
    if (n_completed) *n_completed = nc;
    server_counts(s, n_active, n_queued);
    if (s->worker_rc) return fail(s->worker_rc, "the worker thread stopped on an error: %s", s->worker_err.c_str());
    return SAIL_OK;
}

int sail_server_stop(sail_server_t s) {
    if (!s) return fail(SAIL_EINVAL, "NULL server");
    server_stop_worker(s);
    return SAIL_OK;
}

int sail_server_result(sail_server_t s, int id, double *S_mean, double *S_err, double *chi2_of_mean, int *converged,
                       int *sweeps_done) {
    if (!s) return fail(SAIL_EINVAL, "NULL server");
    std::lock_guard<std::mutex> lk(s->mu);
    if (id < 0 || id >= (int)s->results.size()) return fail(SAIL_EINVAL, "unknown request id");
    const auto &r = s->results[id];
    if (r.info.state < 0) return fail(r.info.state, "request %d failed at admission", id);
    if (r.info.state != 2) return fail(SAIL_ESTATE, "request %d has not completed", id);
    if (S_mean) std::memcpy(S_mean, r.mean.data(), r.mean.size() * 8);
    if (S_err) std::memcpy(S_err, r.err.data(), r.err.size() * 8);
    if (chi2_of_mean) *chi2_of_mean = r.info.chi2_of_mean;
    if (converged) *converged = r.info.converged;
    if (sweeps_done) *sweeps_done = r.info.sweeps;
    return SAIL_OK;
}

int sail_server_request_info(sail_server_t s, int id, sail_request_info *info) {
    if (!s || !info) return fail(SAIL_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    if (id < 0 || id >= (int)s->results.size()) return fail(SAIL_EINVAL, "unknown request id");
    *info = s->results[id].info;
    return SAIL_OK;
}

int sail_server_trace(sail_server_t s, int id, int *acc, int *m, double *delta, int *n_sweeps, int *n_events) {
    if (!s) return fail(SAIL_EINVAL, "NULL server");
    std::lock_guard<std::mutex> lk(s->mu);
    if (id < 0 || id >= (int)s->results.size()) return fail(SAIL_EINVAL, "unknown request id");
    const auto &r = s->results[id];
    if (r.info.state != 2) return fail(SAIL_ESTATE, "request %d has not completed", id);
    if (n_sweeps) *n_sweeps = r.trace_sweeps;
    if (n_events) *n_events = r.trace_events;
    if (acc && !r.acc_trace.empty()) std::memcpy(acc, r.acc_trace.data(), r.acc_trace.size() * 4);
    if (m && !r.m_trace.empty()) std::memcpy(m, r.m_trace.data(), r.m_trace.size() * 4);
    if (delta && !r.delta_trace.empty()) std::memcpy(delta, r.delta_trace.data(), r.delta_trace.size() * 8);
    return SAIL_OK;
}

int sail_server_destroy(sail_server_t s) {
    if (!s) return fail(SAIL_EINVAL, "NULL server");
    server_stop_worker(s);
    cudaStreamSynchronize(s->batch.stream);
    for (sail_t h : s->batch.h)
        if (h) sail_destroy(h);
    batch_streams_destroy(&s->batch);
    delete s;
    return SAIL_OK;
}

}  // extern "C"
