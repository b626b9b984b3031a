/*
 * sail.h - C ABI of the GB300 library for SAIL, the simulated-annealing
 * inversion of the Laplace transform (Lutsyshyn & Astrakharchik,
 * arXiv:1609.07936).
 *
 * One handle holds one inversion: the data F(tau_i) with noise sigma_i on a
 * tau grid, a histogram spectral model on n_omega equal bins of [0, w_max]
 * (Sec. 2.1, Eq. spectral-model), and a population of n_walkers Markov
 * walkers annealed by sum-rule-preserving Metropolis moves (Sec. 2.2), with
 * a periodic full recomputation of the residual and imprinted branching of
 * the population after every block of sweeps (Sec. 2.5).
 *
 * Memory: the library never allocates device memory.  The caller passes one
 * device buffer ("workspace", at least sail_workspace_size() bytes, 256-byte
 * aligned) and a CUDA stream; every kernel of the handle runs on that stream
 * and all device state lives in the workspace until sail_destroy().  Host
 * arrays passed in are read during the call only; host arrays passed out are
 * written before the call returns.  Calls on one handle must not overlap.
 *
 * Errors: functions return SAIL_OK (0), a positive status (SAIL_NOT_CONVERGED)
 * or a negative error code; sail_last_error() gives a message for the calling
 * thread.  No function aborts or exits the process.
 */
#ifndef SAIL_H
#define SAIL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SAIL_OK 0
#define SAIL_NOT_CONVERGED 1   /* target chi2 not reached; results are still valid */
#define SAIL_EINVAL (-1)       /* invalid argument (grid, data, parameters, handle) */
#define SAIL_ENOMEM (-2)       /* workspace smaller than sail_workspace_size() */
#define SAIL_ECUDA (-3)        /* a CUDA runtime call or kernel launch failed */
#define SAIL_ESTATE (-4)       /* call not valid in the handle's current state */
#define SAIL_ETIMEOUT (-5)     /* a bounded device-side wait gave up (results of that call invalid) */

/* Arithmetic of the Metropolis moves. */
#define SAIL_PREC_FP64 0   /* validation path: FP64 state, explicit rescale of every bin, sums in the
                              oracle's order, no fused multiply-add */
#define SAIL_PREC_FP32 1   /* production path: FP32 state and residual, lazy common scale,
                              FP64 residual recomputation and chi2; sail_create refuses data whose
                              weighted terms could leave FP32's range (max_ij K_ij/sigma_i * A or
                              max_i |F_i|/sigma_i above 1e15) with SAIL_EINVAL */

/* Temperature schedules. */
#define SAIL_SCHEDULE_GEOMETRIC 0
#define SAIL_SCHEDULE_SELF_COOLING 1

typedef struct sail_ctx *sail_t;

/* Run parameters.  sail_default_params() fills the paper's choices (Sec. 3):
 * T_start = 10 in units of the start residue, k = 100 sweeps per block,
 * branching of a quarter of the walkers with imprint strength 0.1, amplitude
 * heuristic p = 1, m = 2. */
typedef struct sail_params {
    int n_walkers;          /* population size N_w (>= 1) */
    int precision;          /* SAIL_PREC_FP64 or SAIL_PREC_FP32 */
    int n_sweeps;           /* length of the temperature schedule, in sweeps of n_omega moves */
    int sweeps_per_block;   /* k: branching after every k sweeps (Sec. 3) */
    int resync_every;       /* full residual recomputation period, in sweeps */
    int branching;          /* 1: imprinted branching at every block end (Sec. 2.5) */
    double T_start, T_end;  /* geometric schedule, in units of the start residue chi2_0 (Sec. 3) */
    double T_end_abs;       /* > 0: the schedule ends at this absolute temperature instead of
                               T_end chi2_0 (reach the noise level, chi2 ~ n_tau, whatever chi2_0) */
    double branch_fraction; /* fraction of walkers given a zero multiplier (1/4) */
    double imprint_t;       /* imprint strength t (0.1) */
    double move_scale;      /* d: 1 - r is uniform on (-y d, y d); <= 0 selects 1 / n_omega */
    double y_p, y_m, y_min; /* Eq. (amplitude-acceptance-adjustment) p, m, and a floor for y */
    double A, B;            /* sum constants of Sec. 2.2; A = NaN takes F(0) / c_0 (needs tau_0 = 0) */
    double avg_chi2_factor; /* average walkers with chi2 <= factor * min chi2 (1.5) */
    double target_chi2;     /* > 0: sail_anneal stops once chi2 of the averaged spectrum <= target */
    uint64_t seed;          /* key of the Philox4x32-10 stream */
    int trace;              /* 1: record every walker's accepted-move count per sweep and the
                               branching multipliers (validation; enlarges the workspace) */
    int timing;             /* 1: time every kernel with CUDA events on the handle's stream;
                               totals appear in sail_info */
    int resync_kind;        /* FP32 state: 0 = FP32-FMA GEMM with FP64 chunk sums, 1 = tensor
                               cores (tcgen05 TF32, three-term split), 2 = tensor cores
                               (tcgen05 BF16, three pieces per operand and six products),
                               3 = FP64-FMA GEMM (FP64 products and sums throughout: the plain
                               FP64 recomputation the mixed-precision forms are compared with) */
    int wait_test;          /* test hook, 0 in use: 1 makes the tensor-core resync withhold its
                               first commit so its bounded wait runs out (sail_anneal then
                               returns SAIL_ETIMEOUT) */
    int sweep_lanes;        /* FP32 moves: GPU lanes per walker, 0 = choose (8 when n_tau <= 256
                               on a uniform tau grid, tau_i = tau_0 + i dtau, else 16), 8 (n_tau
                               <= 256 on a uniform grid only: sail_create returns SAIL_EINVAL
                               otherwise; its one-move loop forms the kernel columns from
                               tables of every fourth tau point) or 16.  The choice sets the
                               order of the FP32 delta-chi2 sum, so trajectories depend on it */
    /* The paper's protocol against the sawtooth instability (Sec. self-cooling, Sec. 2.5,
     * Sec. smoothing).  All three act at the end of every full block of k sweeps, in this
     * order: block statistics (acceptance; mean and smallest residue after the block's
     * residual recomputation), branching, smoothing, next block's temperature. */
    int schedule_kind;      /* SAIL_SCHEDULE_GEOMETRIC (T_start -> T_end) or SAIL_SCHEDULE_SELF_COOLING:
                               T constant per block; block 0 at chi2_0; block b >= 1 from
                               block b-1's mean residue cbar and smallest residue cmin:
                               boiling (b < b_cool) T = cbar; cooling (b < b_freeze)
                               T = cbar^(1-x) cmin^x, x = (b - b_cool + 1) / (b_freeze - b_cool);
                               freeze-out T = T_F (T_fin / T_F)^y, y = (b - b_freeze + 1) /
                               (n_blocks - b_freeze), T_F = cmin at its start, T_fin the end
                               temperature (T_end_abs, else T_end chi2_0; T held at T_F if
                               T_F <= T_fin); T_start is not used */
    int adaptive_branching; /* 1: branching fraction and imprint strength times
                               min(1, block acceptance / first block's acceptance) */
    double cool_begin;      /* self-cooling: b_cool = round(cool_begin n_blocks) (0.1) */
    double freeze_begin;    /* self-cooling: b_freeze = round(freeze_begin n_blocks) (0.5) */
    double smooth_s;        /* 0 <= s < 0.5: three-point smoothing of every spectrum after branching,
                               s a_{j-1} + (1-2s) a_j + s a_{j+1} (ends (1-s) a_0 + s a_1), then the
                               tilt a_j (1 + beta (x_j - m)) restoring the second sum rule, then a
                               full residual recomputation; 0 = off (the paper's runs use 1e-2) */
    int index_walk_len;     /* L in [0, 7]: steps of the index walk choosing p and s (Sec. 2.3);
                               0 = p uniform, s uniform on the other bins.  L > 0: each index
                               walks from that start, proposing a uniform bin j' and moving
                               when u a_j <= a_j' (stationary law a_j / A); s walks on the bins
                               other than the final p.  Words: step t from Philox counter
                               (move, sweep, walker, 1 + t), admixture from (.., 2 + L) */
    int hastings;           /* 1: Metropolis-Hastings acceptance for exact detailed balance of the
                               move (a, eps) -> (r a + delta, -eps/r): accept when |eps/r| < y d
                               (the reverse move can be proposed) and u < exp(-D/T) r^(n_omega-4),
                               r^(n_omega-4) the move's Jacobian on the sum-rule manifold; the
                               spectra are put back on the sum rules at every residual
                               recomputation; needs index_walk_len = 0.  0: the paper's
                               Metropolis test */
    double walk_uniform;    /* probability that an index skips its walk (uniform admixture) */
    int shared_bins;        /* W: 0 or 1 = every walker draws its own bins (the paper's move);
                               2, 4 or 8 = the walkers w with equal w / W all propose, at each
                               move, the bins of their group's first walker W (w / W) (words 0
                               and 1 of its move counter), each keeping its own amplitude and
                               acceptance draw (words 2 and 3 of its own counter).  Every
                               walker's chain is still the method's chain (its bins stay uniform
                               and independent of its spectrum); the walkers of a group become
                               correlated.  The FP32 sweep then forms the bins' part of the
                               residual change once per group.  Needs index_walk_len = 0; FP32
                               needs n_tau <= 256 for W = 8 (512 for W = 2 and 4); not
                               accepted by the batch and the server */
    int sweep_loop;         /* FP32 move loop for n_tau <= 256 (uniform bins, own bins): 1 = one move
                               at a time; 2 = look-ahead (each walker keeps its next 16 proposals
                               drawn and spends columns and reduction on feasible ones only; the
                               same draws and decisions, and with 8 lanes per walker on a uniform
                               tau grid the one-move loop's column values differ from the
                               look-ahead's in the last bits); 0 = choose: look-ahead when the problem has
                               at least 16 walkers per SM (measured faster there, slower with fewer)
                               and the last block rejected at least 30% of its proposals for
                               positivity (measured +12% at 40%, -6% at 22-27%) */
    double T_start_abs;     /* > 0: the geometric schedule starts at this absolute temperature
                               instead of T_start chi2_0 (skip the boiling far above the data's
                               scale, whatever chi2_0 is); 0 = T_start */
    /* A shard of a larger population (one inversion's walkers split over several handles, e.g.
     * one per GPU; see sail_branch_solve).  walker_offset is the population index of this
     * handle's walker 0: every random counter uses offset + w as its walker word, so a shard
     * draws exactly what the whole population would for those walkers (a multiple of
     * shared_bins when bins are shared).  walker_total (0: n_walkers) sizes the branching
     * scratch for sail_branch_solve over the whole population (at most 16384 walkers).  A
     * shard runs with branching = 0: the population branches through sail_branch_solve,
     * sail_walker_rows and sail_imprint_rows. */
    int walker_offset;
    int walker_total;
    /* FP64 acceptance near the threshold (FP32 precision, uniform bins, the Metropolis test of
     * Sec. 2.2): 1 = a decision whose FP32 Delta chi2 lies within 1e-5 S of the acceptance
     * threshold -T ln u (or of 0), S = sum_i |d_i| (2 |R_i| + |d_i|) the magnitude of its
     * terms, is taken again from Delta chi2 evaluated in FP64 on the same FP32-stored state
     * (each kernel column as the exact FP64 product of its two FP32 factors, one rounding at
     * the end); 2 = every feasible move's decision so (a test mode); 0 = off.  Counted in
     * sail_info.fp64_rechecks and fp64_flips.  Not with index_walk_len > 0, hastings,
     * shared_bins, batches or the server (EINVAL). */
    int fp64_accept;
} sail_params;

/* Per-block statistics (the paper prints T, residue and acceptance per block, Sec. 4). */
typedef struct sail_block_stats {
    int block;              /* block index */
    int sweep_end;          /* sweeps completed after this block */
    double T;               /* absolute temperature of the block's last sweep */
    double chi2_min, chi2_mean;
    double acceptance;      /* accepted / proposed moves in the block */
    double positivity_rejected; /* proposals rejected because a bin would go negative / proposed */
    double branch_delta;    /* Delta of the branching solve (0 without branching) */
    int branch_zeros;       /* walkers imprinted */
    int reserved;
} sail_block_stats;

typedef struct sail_info {
    int n_tau, n_omega, n_walkers, n_tau_pad, precision;
    int sweeps_done, blocks_done, n_sweeps;
    double chi2_0;          /* residue of the start spectrum (unit of T) */
    double d_omega, A, B;
    double lambda0;         /* tilt of the start spectrum a_j ~ exp(-lambda0 x_j) */
    long long kernel_launches; /* kernels this handle has launched so far */
    size_t workspace_bytes;
    /* with timing = 1: device time in ms and launch counts of the sweep kernel, the
     * residual recomputation and the branching kernels */
    double sweep_ms, resync_ms, branch_ms;
    long long sweep_launches, resync_launches, branch_launches;
    long long moves;           /* walker-moves proposed so far */
    int sweep_lanes;           /* FP32 sweep: GPU lanes per walker in use (0 for FP64) */
    int sweep_ahead;           /* FP32 sweep: 1 if the next block runs the look-ahead move loop */
    long long fp64_rechecks;   /* fp64_accept: decisions taken again in FP64 so far */
    long long fp64_flips;      /* ... of which the FP64 decision differed from the FP32 one */
} sail_info;

/* Fills *p with the defaults listed above (n_walkers 1024, FP32, 20000 sweeps,
 * resync every 50 sweeps, T 10 -> 1e-9, seed 0). */
void sail_default_params(sail_params *p);

/* Bytes of device workspace a handle with these sizes needs (Sec. 2.1-2.5 state:
 * kernel tables, per-walker spectra, residuals, chi2, counters, branching scratch). */
int sail_workspace_size(int n_tau, int n_omega, const sail_params *p, size_t *bytes);

/*
 * Creates a handle (Sec. 2.1-2.2).
 *   tau[n_tau]      >= 0, any order; F[n_tau] data; sigma[n_tau] > 0 noise (chi2 is
 *                   sum_i ((F_i - model_i) / sigma_i)^2, Eq. residue weighted by sigma)
 *   omega[n_omega]  bin centres x_j = (j + 1/2) dw of equal bins starting at 0
 *   p               parameters (copied); p->B must be finite and x_0 < B/A < x_{n-1}
 *   d_workspace     device buffer of ws_bytes >= sail_workspace_size(), 256-byte aligned
 *   stream          cudaStream_t (NULL = legacy default stream)
 * Builds the weighted bin-integrated kernel table K_ij / sigma_i (Eq. correlation-model),
 * the maximum-entropy start spectrum with the two sum rules, its residue chi2_0 and
 * the temperature table, copies them to the workspace and starts every walker there.
 * Synchronises the stream before returning.
 */
int sail_create(sail_t *out, const double *tau, const double *F, const double *sigma, int n_tau,
                const double *omega, int n_omega, const sail_params *p, void *d_workspace,
                size_t ws_bytes, void *stream);

/*
 * Runs up to max_blocks blocks of the schedule (Sec. 3): each block is
 * sweeps_per_block sweeps of n_omega Metropolis moves per walker (Sec. 2.2, Eq.
 * probability-density), with the residual recomputed every resync_every sweeps and
 * at the block end, then imprinted branching (Sec. 2.5).  stats[max_blocks] (may be
 * NULL) receives one record per block run; *n_done (may be NULL) the number run.
 * Returns SAIL_OK, or SAIL_NOT_CONVERGED when target_chi2 > 0 and the schedule ended
 * without reaching it.  One stream synchronisation per block.
 */
int sail_anneal(sail_t h, int max_blocks, sail_block_stats *stats, int *n_done);

/*
 * Stochastic average (Sec. 1): mean and standard error (sample std / sqrt(n)) per bin
 * over the walkers with chi2 <= avg_chi2_factor * min chi2, and the chi2 of the mean
 * spectrum.  S_mean, S_err: host arrays of n_omega (S_err may be NULL).  Branching
 * correlates walkers, so the error is a lower bound.
 */
int sail_average(sail_t h, double *S_mean, double *S_err, int *n_used, double *chi2_of_mean);

int sail_get_info(sail_t h, sail_info *info);

/*
 * Copies walker state to host arrays (any may be NULL): a[n_walkers * n_omega] spectra
 * (the common scale folded in), R[n_walkers * n_tau] residuals F/sigma - K a / sigma,
 * chi2[n_walkers], acc_prev[n_walkers] (accepted moves in the last sweep),
 * hash[n_walkers] (FNV-1a of every move's outcome: 0 rejected, 1 accepted, 2 negative).
 */
int sail_get_state(sail_t h, double *a, double *R, double *chi2, int *acc_prev, uint64_t *hash);

/*
 * Replaces the spectra (a[n_walkers * n_omega], required) and optionally acc_prev;
 * the residuals and chi2 are recomputed from them.  Sum rules are not enforced.
 */
int sail_set_state(sail_t h, const double *a, const int *acc_prev);

/*
 * Branching of a population split over several handles (Sec. 2.5, the same solve as
 * sail_anneal's).  sail_branch_solve runs the multiplier solve on the device of handle h for
 * the n_total chi2 values chi2_all (host array, the whole population in index order; draws
 * xi_l from Philox counter (l, block, 0, 1)): multipliers m[n_total], Delta, and the imprint
 * pairs zero_l[k] <- donor_l[k] (population indices, k < *n_pairs; host arrays of n_total).
 * Every handle of the population computes the same result from the same chi2.  h needs
 * walker_total >= n_total.
 * sail_walker_rows copies walkers idx[0..n) (this handle's indices) into device arrays
 * a_rows[n][n_omega] and R_rows[n][n_tau] in FP64 (exact for either state precision), e.g. to
 * send donors to the GPU that holds their receivers; sail_imprint_rows imprints this handle's
 * walkers idx[0..n) with donor rows in this GPU's memory, a <- t a_donor + (1 - t) a and
 * R likewise, in the arithmetic sail_anneal's imprint uses, and sums their chi2 anew.
 * n <= 65536; idx is a host array.
 */
int sail_branch_solve(sail_t h, int n_total, const double *chi2_all, int block, double fraction, int *m,
                      double *delta, int *zero_l, int *donor_l, int *n_pairs);
int sail_walker_rows(sail_t h, int n, const int *idx, double *d_a_rows, double *d_R_rows);
int sail_imprint_rows(sail_t h, int n, const int *idx, const double *d_a_rows, const double *d_R_rows, double t);

/*
 * Checkpoint and resume mid-schedule.  sail_checkpoint writes into a caller's host buffer of
 * sail_checkpoint_size() bytes everything the rest of the schedule depends on: the walkers'
 * spectra (and FP32 common scales), residuals exactly as stored, chi2, last-sweep acceptance,
 * move hashes and counters, the trace so far (trace = 1), the sweep and block position, the
 * temperature table (self-cooling fills it block by block) and the adaptive-branching and
 * freeze-out state.  Counter-based random numbers (keyed by walker, sweep and move) need no
 * generator state.  sail_restore loads such a buffer into a handle created from the same data
 * and parameters (SAIL_EINVAL if the sizes, precision, schedule or seed differ): its next
 * sail_anneal continues exactly where the checkpointed handle stopped, so an interrupted and
 * resumed run ends bit for bit like the uninterrupted one.  Taken between sail_anneal calls.
 */
int sail_checkpoint_size(sail_t h, size_t *bytes);
int sail_checkpoint(sail_t h, void *buf, size_t bytes);
int sail_restore(sail_t h, const void *buf, size_t bytes);

/*
 * Trace of a handle created with trace = 1: acc[sweeps_done * n_walkers] accepted
 * moves per sweep and walker; m[n_events * n_walkers] branching multipliers and
 * delta[n_events] (each may be NULL; n_events = number of branchings so far).
 */
int sail_get_trace(sail_t h, int *acc, int *m, double *delta, int *n_events);

/*
 * Evaluates n proposals on the current walker states with the handle's move
 * arithmetic (Sec. 2.2) without changing them: walker[q], bins p[q] != s[q],
 * eps[q] = 1 - r.  Writes ok[q] (0: a bin would go negative, 1: valid) and, for
 * valid moves, delta[q] = the change of chi2.  Host arrays; 0 <= n <= 65536.
 */
int sail_delta_probe(sail_t h, int n, const int *walker, const int *p, const int *s,
                     const double *eps, double *delta, int *ok);

/* Device Philox4x32-10 (Salmon et al., SC'11) over n counters: d_ctr[4n] -> d_out[4n]
 * (device pointers), key = seed.  The generator every kernel draws from. */
int sail_philox(int n, const uint32_t *d_ctr, uint64_t seed, uint32_t *d_out, void *stream);

/* Measurement utility for the roofline (no counterpart in the paper): every SM reads
 * d_buf[0 .. bytes) reps times with 16-byte loads and writes a checksum to d_sink[0..7]
 * (device pointers; d_buf 16-byte aligned, bytes a multiple of 16).  Timed by the caller
 * on its stream, it gives the read bandwidth of L2 (a buffer far smaller than L2) or of
 * HBM (a buffer far larger). */
int sail_probe_read_bandwidth(const void *d_buf, size_t bytes, int reps, void *d_sink, void *stream);

/* Measurement utility for the roofline (no counterpart in the paper): two blocks per SM read
 * a 32 KiB shared-memory buffer with conflict-free 16-byte loads, reps loads per thread; the
 * number of bytes read goes to *bytes_read (host).  Timed by the caller on its stream, it
 * gives the shared-memory read bandwidth the FP32 sweep's kernel tables are read at.
 * d_sink: 8 bytes of device memory. */
int sail_probe_smem_bandwidth(int reps, void *d_sink, void *stream, double *bytes_read);

/*
 * Residue chi2 = sum_i ((F_i - sum_j K_ij a_j) / sigma_i)^2 of n_spectra histogram spectra,
 * for callers that cannot allocate device memory.  The paper has no counterpart: this is a
 * variant of the residual recomputation that sail_anneal and sail_set_state run inside a
 * handle's workspace.  Every other entry point needs that caller-allocated workspace; a
 * plug-in inside a program whose allocator owns the whole device memory, or a service loop
 * that must not pay for cudaMalloc / cudaFree, cannot provide one.  This one allocates
 * nothing: its only scratch (the weighted kernel table and data) lives in a fixed array of
 * 8 MiB + 4 KiB that every GPU loading the library holds until the process exits.
 *   d_tau, d_F, d_sigma [n_tau], d_omega [n_omega] (bin centres from 0, as in sail_create),
 *   d_a [n_spectra * n_omega]: device inputs.  d_chi2 [n_spectra] and, if not NULL,
 *   d_R [n_spectra * n_tau] (residuals F/sigma - K a/sigma): device outputs.
 * Limits: 1 <= n_tau <= 512 and n_omega * (n_tau rounded up to 32) <= 1,048,576; larger
 * sizes return SAIL_EINVAL with a message.  The grid is not checked.  Kernels run on
 * stream; the call returns without synchronising.
 * The first call on each device looks up the scratch array's device address with that
 * device current, so make that first call before any stream capture.  All calls share the
 * one array, which keeps the last call's contents: calls whose kernels overlap on the GPU
 * (other streams, other threads) race and must be serialised by the caller.
 */
int sail_residue_noalloc(const double *d_tau, const double *d_F, const double *d_sigma, int n_tau,
                         const double *d_omega, int n_omega, const double *d_a, int n_spectra,
                         double *d_chi2, double *d_R, void *stream);

/* ---------------------------------------------------------------- batches
 * Many independent inversions (each a k-vector or data set of its own, Sec. 2.1) annealed
 * together: every block, one persistent sweep launch covers the walkers of all problems
 * (blocks of the GPU take (problem, walker range) items from a queue), then each problem's
 * residual recomputation, branching and statistics run as for a single handle.  A problem's
 * results do not depend on the other problems in the batch: its random numbers are keyed by
 * its own seed and walker indices, and every step of its arithmetic is per walker or per
 * problem.  All problems use FP32 precision and share sweeps_per_block and resync_every. */
typedef struct sail_batch_ctx *sail_batch_t;

typedef struct sail_problem {
    const double *tau, *F, *sigma; /* host arrays of n_tau, as in sail_create */
    int n_tau;
    const double *omega;           /* host array of n_omega bin centres */
    int n_omega;
    sail_params params;            /* precision SAIL_PREC_FP32 */
} sail_problem;

/* Workspace bytes for a batch of n problems (their handles' workspaces plus the queue). */
int sail_batch_workspace_size(int n, const sail_problem *probs, size_t *bytes);

/* Creates every problem's handle inside d_workspace (ws_bytes >= sail_batch_workspace_size)
 * on stream.  autotune = 1 lets the first sweep launches and residual recomputations try the
 * candidate walker-to-block mappings (items of 4, 8 or 16 walker pairs per block) and
 * tensor-core tile widths, timing each with CUDA events, and keep the fastest; results do
 * not depend on either choice. */
int sail_batch_create(sail_batch_t *out, int n, const sail_problem *probs, int autotune, void *d_workspace,
                      size_t ws_bytes, void *stream);

/* Runs up to max_blocks blocks for every problem with sweeps left (and, with a target, not
 * yet converged); *n_done: blocks run. */
int sail_batch_anneal(sail_batch_t b, int max_blocks, int *n_done);

/* The handle of problem k for sail_average, sail_get_state, sail_get_info ... (owned by the
 * batch: do not destroy it, do not anneal it on its own). */
int sail_batch_handle(sail_batch_t b, int k, sail_t *h);

/* The autotuner's choice of walker pairs per block item, the device time per walker-move of
 * the last batched sweep launch (ns, 0 before any), and the batched sweep launches so far
 * (each problem's own kernel count is in its sail_info). */
int sail_batch_tuning(sail_batch_t b, int *item_pairs, double *ns_per_move, long long *sweep_launches);

int sail_batch_destroy(sail_batch_t b);

/* ---------------------------------------------------------------- serving
 * Continuous batching of inversion requests (no counterpart in the paper, which inverts one
 * data set at a time; the requests are the independent k-vectors of Sec. 2.1).  Requests queue
 * in submission order; each step admits the head of the queue while a slot is free, the
 * resident walkers stay within max_walkers and the request's workspace fits a free region of
 * d_workspace (first fit: the buffer size is the HBM admission cap), runs one block for every
 * resident problem through the batched sweep, and retires problems that reached their
 * target_chi2 (checked each block on the averaged spectrum) or their last sweep, keeping the
 * averaged spectrum on the host.  A step admits only requests submitted before it began, so a
 * request submitted while a block runs is admitted at the next block boundary.  A request's
 * result does not depend on which others share the device (see the batch above).
 *
 * Steps are driven either by the caller (sail_server_step, blocking for one block) or by the
 * server's own worker thread (sail_server_start ... sail_server_stop, completions collected
 * with sail_server_poll).  Submission, polling, results and request information may be called
 * from any thread at any time, also while a block runs; they never wait for the block. */
typedef struct sail_server_ctx *sail_server_t;

/* Life of one request, times in seconds on the server's steady clock (0 at creation), steps
 * counted from 1 (a request submitted after step k began has submit_step = k). */
typedef struct sail_request_info {
    int state;              /* 0 queued, 1 resident, 2 completed, < 0 the error that refused it */
    int converged;          /* completed: the target chi2 was reached */
    int sweeps;             /* sweeps run (resident: as of the last finished step) */
    int n_used;             /* completed: walkers in the average */
    long long submit_step;  /* steps begun when the request was submitted */
    long long admit_step;   /* the step that admitted it (-1 while queued) */
    long long done_step;    /* the step that retired it (-1 before) */
    double t_submit, t_admit, t_done;   /* -1 until reached */
    double chi2_of_mean;    /* completed: chi2 of the averaged spectrum */
} sail_request_info;

int sail_server_create(sail_server_t *out, int max_resident, long long max_walkers, int sweeps_per_block,
                       int resync_every, void *d_workspace, size_t ws_bytes, void *stream);
/* Copies the request (host arrays and parameters; FP32, the server's periods); *id for its
 * result.  Thread-safe; wakes the worker thread if it runs. */
int sail_server_submit(sail_server_t s, const sail_problem *req, int *id);
/* Admission, one block, retirement, on the calling thread.  completed[max_completed] receives
 * the ids retired in this step (*n_completed of them); *n_active / *n_queued: resident and
 * waiting requests after it.  SAIL_ESTATE while the worker thread runs. */
int sail_server_step(sail_server_t s, int *completed, int max_completed, int *n_completed, int *n_active,
                     int *n_queued);
/* Starts the worker thread, which runs steps on the device current at this call while any
 * request is queued or resident and sleeps otherwise.  SAIL_ESTATE if it already runs. */
int sail_server_start(sail_server_t s);
/* Ids retired by the worker since the last poll (up to max_completed, oldest first), and the
 * resident / queued counts now.  Returns the worker's error (and stays in it) if a step failed. */
int sail_server_poll(sail_server_t s, int *completed, int max_completed, int *n_completed, int *n_active,
                     int *n_queued);
/* Stops the worker thread after the step it is running, if any. */
int sail_server_stop(sail_server_t s);
/* Result of a completed request: averaged spectrum and its standard error (host arrays of
 * n_omega, may be NULL), chi2 of the average, whether the target was reached, sweeps run. */
int sail_server_result(sail_server_t s, int id, double *S_mean, double *S_err, double *chi2_of_mean, int *converged,
                       int *sweeps_done);
int sail_server_request_info(sail_server_t s, int id, sail_request_info *info);
/* Per-sweep accepted counts [n_sweeps][n_walkers], branching multipliers [n_events][n_walkers]
 * and Deltas [n_events] of a completed request created with params.trace = 1, laid out as
 * sail_get_trace's (n_sweeps = 0 without trace); any array may be NULL to query the counts. */
int sail_server_trace(sail_server_t s, int id, int *acc, int *m, double *delta, int *n_sweeps, int *n_events);
/* Stops the worker thread, then frees the server and its resident requests. */
int sail_server_destroy(sail_server_t s);

/* Frees the host side of the handle; the workspace stays the caller's. */
int sail_destroy(sail_t h);

/* Message of the last error on this thread ("" if none). */
const char *sail_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SAIL_H */
