// Internal declarations shared by the kernels and the host side of libsail.
// Layouts in device memory (all arrays 256-byte aligned inside the caller's workspace):
//   Khat64 / Khat32  [n_omega][n_tau_pad]  column j of K_ij / sigma_i, zero past n_tau
//   Fhat64 / Fhat32  [n_tau_pad]           F_i / sigma_i, zero past n_tau
//   x64              [n_omega]             bin centres
//   beta32           [n_omega]             B - A x_j
//   rgap32           [n_omega]             1 / (k dw), k = 0..n_omega-1 (k = 0 unused)
//   Qhi32            [ceil(n_omega/32)][n_tau_pad]  Khat_{i,32h}
//   Qlo32            [32][n_tau_pad]        q_i^l = e^{-l dw tau_i}; Khat_{i,32h+l} = Qhi[h][i] Qlo[l][i]
//   x4_32            [n_omega][4]           (1, X_j, X_j^2, X_j^3), X_j = e^{-j dw dtau} (uniform tau only)
//   mrho32           [n_tau_pad]            -Khat_{i,0} / Khat_{4 floor(i/4),0}, zero past n_tau (uniform tau)
//   Tsweep           [n_sweeps]            absolute temperature of each sweep
//   a64  (FP64)      [n_walkers][n_omega]  spectra
//   b32  (FP32)      [n_walkers][n_omega]  spectra / common scale g
//   g2   (FP32)      [n_walkers][2]        common scale as an unevaluated float pair (hi, lo)
//   R64 / R32        [n_walkers][n_tau_pad] residuals, zero past n_tau
#pragma once
#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

namespace sail {

constexpr int kMaxChunks = 16;        // residual chunks of 32 per lane: n_tau <= 512
constexpr int kMaxTau = 32 * kMaxChunks;
constexpr int kProbeMax = 65536;      // proposals per sail_delta_probe call
constexpr int kSolveThreads = 1024;   // branching solve: one block
constexpr int kSolvePerThread = 16;   // walkers per solve thread: n_walkers <= 16384
constexpr int kMaxWalkers = kSolveThreads * kSolvePerThread;
constexpr unsigned long long kFnvOffset = 0xCBF29CE484222325ull;
constexpr unsigned long long kFnvPrime = 0x100000001B3ull;

// The tensor-copy (TMA) residual recomputation of a handle: the tensor maps of its pre-tiled
// spectra and kernel-table buffers (resync_tma.cu) and the block shape.
struct TmaPlan {
    CUtensorMap map_a, map_b;
    void *At, *Bt;
    int n, n_kt, n_blocks_tau, n_blocks_walkers;
    int nop;               // bins of a row of the piece arrays (n_omega rounded up to 64)
};

struct DevProblem {
    int n_tau, n_omega, n_walkers, n_tau_pad, n_sweeps;
    double A, B, dw;
    double move_scale, y_p, y_m, y_min;
    uint64_t seed;
    const double *Khat64;
    const float *Khat32;
    const double *Fhat64;
    const float *Fhat32;
    const double *x64;
    const float *beta32;
    const float *rgap32;
    const float *Qhi32;
    const float *Qlo32;
    const float *Khi32;    // [n_tau_pad][n_omega_pad] Khat cut to TF32 (K-major, tensor-core resync)
    const float *Klo32;    // [n_tau_pad][n_omega_pad] Khat - Khi
    int n_omega_pad;       // n_omega rounded up to 32
    int tc_cols;           // tau columns per tensor-core resync block (0: the widest that fits)
    int wait_test;         // test hook: the tensor-core resync withholds its first commit
    int lanes;             // FP32 sweep: lanes per walker (8: 4 walkers per warp, n_tau <= 256 on a uniform
                           // tau grid, columns from quad-compact tables; 16: 2, full factor rows)
    int walk_len;          // steps of the index walk (0: uniform bins)
    int hastings;          // Metropolis-Hastings acceptance with the move's Jacobian
    double walk_rho;       // probability that an index skips its walk
    int shared_bins;       // W > 1: walkers in groups of W propose their first walker's bins
    int ahead;             // FP32, up to 8 chunks: the look-ahead move loop (else one move at a time)
    const double *Tsweep;
    const TmaPlan *tma;    // host pointer (launchers only): the BF16 tensor-copy recomputation, or null
    int walker_base;       // population index of walker 0: the walker word of every random counter
    int fp64_accept;       // FP32: 1 = decisions near the threshold taken again in FP64, 2 = all of them
    const float *x4_32;    // uniform tau grid: per-bin powers of X_j (8-lane sweep's columns)
    const float *mrho32;   // uniform tau grid: minus the ratio of Khat_{i,0} to its quad's first
};

struct DevState {
    double *a64;
    float *b32;
    float *g2;
    double *R64;
    float *R32;
    double *chi2;
    int *acc_prev;
    unsigned long long *hash;
    unsigned long long *n_acc;
    unsigned long long *n_pos;
    int *acc_trace;        // [n_sweeps][n_walkers] or null
    unsigned long long *guard;   // [2]: decisions taken again in FP64, and how many of them changed
};

struct BranchScratch {
    int *m;                // [n_walkers] multipliers
    int *zero_l;           // [n_walkers] imprinted walkers, ascending
    int *donor_l;          // [n_walkers] donor of each imprinted walker
    int *n_pairs;          // [1]
    double *delta;         // [1] Delta of the solve
    int *m_trace;          // [max_events][n_walkers] or null
    double *delta_trace;   // [max_events] or null
    double *z;             // [n_walkers] normalised chi2 of the solve
    double *xi;            // [n_walkers] branching draws
    double *cand;          // [128] trial Deltas of one speculative round
    int *cand_Z;           // [128] zero counts at the trials
    void *ctl;             // search state (64 bytes)
};

struct BlockCounters {     // device-side block statistics, read back once per block
    double chi2_min, chi2_sum;
    unsigned long long acc, pos;
};

// ---- launchers (return cudaGetLastError() of the launch) ----
cudaError_t launch_init_state(const DevProblem &P, const DevState &S, int precision,
                              const double *a0, const double *R0, double chi2_0, cudaStream_t st);
cudaError_t launch_sweep_fp64(const DevProblem &P, const DevState &S, int sweep_begin,
                              int sweep_end, cudaStream_t st);
cudaError_t launch_sweep_fp32(const DevProblem &P, const DevState &S, int sweep_begin,
                              int sweep_end, cudaStream_t st);
// The FP32 sweep of a problem with an index walk (P.walk_len > 0); launch_sweep_fp32 calls it.
cudaError_t launch_sweep_walk(const DevProblem &P, const DevState &S, int sweep_begin, int sweep_end,
                              cudaStream_t st);
// The FP32 sweep of a problem with shared bins (P.shared_bins = 2, 4 or 8), plain or Hastings.
cudaError_t launch_sweep_shared(const DevProblem &P, const DevState &S, int sweep_begin, int sweep_end,
                                cudaStream_t st);
// The FP32 sweep whose decisions near the acceptance threshold are taken again in FP64
// (P.fp64_accept, uniform bins, Metropolis test).
cudaError_t launch_sweep_guard(const DevProblem &P, const DevState &S, int sweep_begin, int sweep_end,
                               cudaStream_t st);
// The FP32 sweep with the Metropolis-Hastings acceptance (P.hastings, uniform bins).
cudaError_t launch_sweep_hastings(const DevProblem &P, const DevState &S, int sweep_begin, int sweep_end,
                                  cudaStream_t st);
// FP64 state: sequential FP64 recomputation, after (restore != 0 and the Hastings acceptance)
// putting the spectra back on the sum rules in bin order.  FP32 state: optional sum-rule
// restoration (restore != 0), then the tiled GEMM of resync_fp32.cu or the tensor cores.
cudaError_t launch_resync(const DevProblem &P, const DevState &S, int precision, int restore, int kind,
                          int *status, cudaStream_t st, int *launches);
cudaError_t launch_resync_fp64(const DevProblem &P, const DevState &S, cudaStream_t st);
cudaError_t launch_resync_fp32(const DevProblem &P, const DevState &S, cudaStream_t st);
// Tensor-core (tcgen05) residual recomputation for FP32 state, TF32 with a three-term split or
// (bf16) BF16 with three pieces and six products; status[0] <- 1 on a timed-out wait.
cudaError_t launch_resync_tc(const DevProblem &P, const DevState &S, int *status, bool bf16, cudaStream_t st);
// The BF16 x6 recomputation as a pipelined GEMM fed by tensor copies (resync_tma.cu): tau
// columns per block for a padded tau count, workspace bytes of the pre-tiled spectra and
// kernel table, the plan (tensor maps; pre-tiles the kernel table on st) and the launch
// (splits the spectra unless presplit is false because the sum-rule restoration wrote the
// pieces, GEMM, chi2); status[0] <- 1 on a timed-out wait.
int tma_tau_block(int n_tau_pad);
size_t tma_spectra_bytes(int n_walkers, int n_omega);
size_t tma_table_bytes(int n_tau_pad, int n_omega);
cudaError_t tma_plan_init(TmaPlan &T, const DevProblem &P, void *At, void *Bt, cudaStream_t st);
cudaError_t launch_resync_tma(const DevProblem &P, const DevState &S, const TmaPlan &T, int *status, bool presplit,
                              cudaStream_t st);
cudaError_t launch_branch(const DevProblem &P, const DevState &S, const BranchScratch &B,
                          int precision, int block_index, double fraction, double imprint_t,
                          int event, cudaStream_t st, int *launches);
// The branching solve alone (multipliers, Delta, imprint pairs into B) over P.n_walkers chi2
// values in S.chi2, draws keyed by population index (P.walker_base + l); no imprint, no trace.
cudaError_t launch_branch_solve(const DevProblem &P, const DevState &S, const BranchScratch &B, int block_index,
                                double fraction, cudaStream_t st, int *launches);
// Rows of walkers idx[0..n) (device array) in FP64, and imprinting of walkers idx from donor rows.
cudaError_t launch_walker_rows(const DevProblem &P, const DevState &S, int precision, int n, const int *idx,
                               double *a_rows, double *R_rows, cudaStream_t st);
cudaError_t launch_imprint_rows(const DevProblem &P, const DevState &S, int precision, int n, const int *idx,
                                const double *a_rows, const double *R_rows, double t, cudaStream_t st);
// Smoothing (Sec. smoothing) of every walker's spectrum with strength s and the tilt that
// restores the second sum rule; one thread per walker, sums in bin order (FP64 arithmetic for
// either state precision).  The residuals are stale afterwards.
cudaError_t launch_smooth(const DevProblem &P, const DevState &S, int precision, double s, cudaStream_t st);
cudaError_t launch_block_stats(const DevProblem &P, const DevState &S, BlockCounters *out,
                               cudaStream_t st);
cudaError_t launch_average(const DevProblem &P, const DevState &S, int precision, double factor,
                           double *mean, double *err, int *n_used, double *cut, double *R_mean,
                           double *chi2_mean, cudaStream_t st, int *launches);
cudaError_t launch_probe(const DevProblem &P, const DevState &S, int precision, int n,
                         const int *walker, const int *p, const int *s, const double *eps,
                         double *delta, int *ok, cudaStream_t st);
cudaError_t launch_philox(int n, const uint32_t *ctr, uint64_t seed, uint32_t *out, cudaStream_t st);
// Shared memory the FP32 sweep needs for its kernel tables (must fit one block).
size_t sweep_fp32_table_bytes(const DevProblem &P);
// Walkers one warp of the FP32 sweep runs (32 / P.lanes); batched launches count items in these
// groups.
int sweep_walkers_per_warp(const DevProblem &P);

// One problem of a batched sweep launch: sweeps [n0, n1) (n0 == n1: nothing this launch).
struct BatchProblem {
    DevProblem P;
    DevState S;
    int n0, n1;
};
struct BatchItem {      // walker groups [grp_lo, grp_hi) of problem prob, one group per warp
    int prob, grp_lo, grp_hi;
};
// Move-loop variant of a problem's FP32 sweep: 0 plain, 1 index walk, 2 Metropolis-Hastings.
int sweep_mode(const DevProblem &P);
// Persistent FP32 sweep over many problems whose DevProblem.lanes all equal `lanes` and whose
// sweep_mode all equal `mode`: blocks of `warps` warps (at most 8 when lanes = 8, 12 when 16)
// take items from the queue.
cudaError_t launch_sweep_batch(const BatchProblem *d_probs, const BatchItem *d_items, int n_items, int *d_counter,
                               size_t smem, int warps, int lanes, int mode, cudaStream_t st);
cudaError_t launch_sweep_batch8(const BatchProblem *d_probs, const BatchItem *d_items, int n_items, int *d_counter,
                                size_t smem, int warps, int mode, cudaStream_t st);
cudaError_t launch_read_probe(const void *buf, size_t bytes, int reps, void *sink, cudaStream_t st);
cudaError_t launch_smem_probe(int reps, void *sink, cudaStream_t st, double *bytes);

// Records the message sail_last_error() returns on this thread; returns code.
int set_error(int code, const char *fmt, ...);

}  // namespace sail
