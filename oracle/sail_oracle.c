/*
 * Plain FP64 CPU oracle for SAIL: simulated annealing of a population of
 * histogram spectra against Laplace-transform data (Lutsyshyn & Astrakharchik,
 * arXiv:1609.07936).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no code
 * with the CUDA library: it is the method written out step by step in the
 * paper's order and notation, slow and obvious, so that a reader can check it
 * against the paper by eye.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC (every product and
 * sum is rounded on its own, as written).
 *
 * Notation (Sec. 2.1-2.2): bins j = 0..N_omega-1 of width dw, bin j = [j dw, (j+1) dw),
 * centre x_j = (j + 1/2) dw; data points i = 0..N_tau-1.  Weighted quantities
 * Khat_ij = K_ij / sigma_i and Fhat_i = F_i / sigma_i; residual
 * R_i = Fhat_i - sum_j Khat_ij a_j; residue chi2 = sum_i R_i^2.
 *
 * Readings of points the paper leaves open:
 *   - chi2 is weighted by the noise sigma_i (Eq. residue is the case sigma = 1);
 *   - the start spectrum is the maximum-entropy histogram with the two sum
 *     rules, a_j proportional to exp(-lambda x_j);
 *   - the move amplitude eps = 1 - r is uniform on (-y d, y d);
 *   - p is uniform on the bins and s uniform on the other bins (zero-length
 *     index walk, Sec. 2.3); an index walk of L > 0 steps is an independence
 *     walk with law a_j / A, s walking on the bins other than p (or_move_bins);
 *   - optionally the walkers share their bins in groups of W (bin_words): the
 *     group's first walker's bin draw serves the whole group;
 *   - an optional Hastings acceptance with the move's Jacobian r^(N_omega-4)
 *     (or_accept), for exact detailed balance, with the spectra put back on the
 *     sum rules at every residual recomputation (or_restore);
 *   - the branching weight is w = exp[-Delta (chi2 - P_r)] (the printed
 *     formula applies the weight to P(chi2), read as chi2);
 *   - random numbers come from Philox4x32-10 (Salmon et al., SC'11), counter
 *     (move, sweep, walker, 0) for a move and (walker, block, 0, 1) for the
 *     branching draw xi, key = the 64-bit seed;
 *   - self-cooling (Sec. self-cooling): T constant per block; boil at the
 *     population's mean residue, a geometric ramp to its smallest residue, then
 *     a freeze-out lowering T by a constant proportion per block to the
 *     schedule's end temperature (or_self_cooling);
 *   - adaptive branching (Sec. 2.5): fraction and imprint strength times
 *     min(1, acceptance / first block's acceptance);
 *   - smoothing (Sec. smoothing) after branching, its second-sum-rule
 *     renormalisation a multiplicative linear tilt (or_smooth), followed by a
 *     full residual recomputation.
 *
 * Parity status: every function below is pinned by the CPU tests except the
 * Philox stream, whose CPU pins are statistical and whose value pin is the
 * GPU test against the cuRAND header's Philox4x32-10.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_PI 3.14159265358979323846

/* ------------------------------------------------------------------ Philox
 * Philox4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3", SC'11).  One round multiplies words 0 and 2
 * by the two round constants, keeps the 64-bit products' halves, and mixes in
 * words 1 and 3 and the round key; the key is bumped by the two Weyl
 * constants between rounds. */
static void philox_round(uint32_t x[4], const uint32_t k[2]) {
    uint64_t p0 = (uint64_t)0xD2511F53u * x[0];
    uint64_t p1 = (uint64_t)0xCD9E8D57u * x[2];
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t y0 = hi1 ^ x[1] ^ k[0];
    uint32_t y1 = lo1;
    uint32_t y2 = hi0 ^ x[3] ^ k[1];
    uint32_t y3 = lo0;
    x[0] = y0; x[1] = y1; x[2] = y2; x[3] = y3;
}

void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t x[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k[2] = {key[0], key[1]};
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k[0] += 0x9E3779B9u; k[1] += 0xBB67AE85u; }
        philox_round(x, k);
    }
    out[0] = x[0]; out[1] = x[1]; out[2] = x[2]; out[3] = x[3];
}

static void draw(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t out[4]) {
    uint32_t ctr[4] = {c0, c1, c2, c3};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    or_philox4x32_10(ctr, key, out);
}

/* A 32-bit word to a uniform on (0, 1): (w + 1/2) / 2^32, exact in FP64. */
static double unit(uint32_t w) { return ((double)w + 0.5) * 2.3283064365386963e-10; }

/* ---------------------------------------------------------- the model
 * Eq. (correlation-model): bin j contributes
 * K_ij = (1/2pi) int_{j dw}^{(j+1) dw} e^{-w tau_i} dw
 *      = e^{-j dw tau_i} (1 - e^{-dw tau_i}) / (2 pi tau_i),  and dw / 2pi at tau = 0
 * (Eq. efficient-correlation-model and c-coefficients for tau_i = i dtau).
 * Returns 0, or -1 if the grid is not a set of equal bins starting at 0. */
int or_tables(int n_tau, int n_omega, const double *tau, const double *F, const double *sigma,
              const double *x, double *Khat, double *Fhat, double *dw_out) {
    if (n_tau < 1 || n_omega < 2) return -1;
    double dw = (x[n_omega - 1] - x[0]) / (double)(n_omega - 1);
    if (!(dw > 0)) return -1;
    for (int j = 0; j < n_omega; ++j)
        if (fabs(x[j] - (j + 0.5) * dw) > 1e-9 * dw * (j + 1)) return -1;
    for (int i = 0; i < n_tau; ++i) {
        if (!(tau[i] >= 0) || !(sigma[i] > 0) || !isfinite(F[i])) return -1;
        for (int j = 0; j < n_omega; ++j) {
            double K;
            if (tau[i] == 0.0) K = dw / (2.0 * OR_PI);
            else K = exp(-(double)j * dw * tau[i]) * (-expm1(-dw * tau[i])) / (2.0 * OR_PI * tau[i]);
            Khat[(size_t)i * n_omega + j] = K / sigma[i];
        }
        Fhat[i] = F[i] / sigma[i];
    }
    *dw_out = dw;
    return 0;
}

/* Residual R_i = Fhat_i - sum_j Khat_ij a_j (plain sums over j ascending);
 * returns chi2 = sum_i R_i^2 (Eq. residue, weighted). */
double or_residual(int n_tau, int n_omega, const double *Khat, const double *Fhat,
                   const double *a, double *R) {
    double chi2 = 0.0;
    for (int i = 0; i < n_tau; ++i) {
        double model = 0.0;
        for (int j = 0; j < n_omega; ++j) model += Khat[(size_t)i * n_omega + j] * a[j];
        double r = Fhat[i] - model;
        if (R) R[i] = r;
        chi2 += r * r;
    }
    return chi2;
}

/* Start spectrum: the histogram of largest entropy whose sums are the two
 * constants of Sec. 2.2, sum_j a_j = A and sum_j a_j x_j = B, i.e.
 * a_j = A e^{-lambda x_j} / sum_k e^{-lambda x_k} with lambda found by
 * bisection (the tilted mean falls as lambda grows).  lambda = 0 is the flat
 * histogram.  Returns -1 unless x_0 < B/A < x_{N-1}. */
int or_initial_spectrum(int n_omega, const double *x, double A, double B, double *a, double *lambda_out) {
    if (!(A > 0)) return -1;
    double target = B / A;
    if (!(target > x[0] && target < x[n_omega - 1])) return -1;
    double xc = 0.5 * (x[0] + x[n_omega - 1]);
    double span = x[n_omega - 1] - x[0];
    double lo = -700.0 / span, hi = 700.0 / span;
    for (int it = 0; it < 400; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        double s0 = 0.0, s1 = 0.0;
        for (int j = 0; j < n_omega; ++j) {
            double w = exp(-mid * (x[j] - xc));
            s0 += w;
            s1 += w * x[j];
        }
        if (s1 / s0 > target) lo = mid; else hi = mid;
    }
    double lambda = 0.5 * (lo + hi);
    double s0 = 0.0;
    for (int j = 0; j < n_omega; ++j) { a[j] = exp(-lambda * (x[j] - xc)); s0 += a[j]; }
    for (int j = 0; j < n_omega; ++j) a[j] = A * a[j] / s0;
    if (lambda_out) *lambda_out = lambda;
    return 0;
}

/* ------------------------------------------------------------ one move
 * Sec. 2.2, Eqs. (update-scheme-p/s/j) and (update-delta-p/s):
 *   a_p' = r a_p + delta_p,  a_s' = r a_s + delta_s,  a_j' = r a_j otherwise,
 *   delta_p (x_p - x_s) = (B - A x_s)(1 - r),  delta_s (x_s - x_p) = (B - A x_p)(1 - r),
 * where x_p - x_s = w_p - w_s (bin left edges differ as the centres do).
 * The model becomes F' = r F + delta_p K_p + delta_s K_s, so in weighted form
 *   d_i = eps M_i - delta_p Khat_ip - delta_s Khat_is,  M_i = Fhat_i - R_i,  eps = 1 - r,
 *   R' = R + d,  Delta chi2 = sum_i [(R_i + d_i)^2 - R_i^2] = sum_i d_i (2 R_i + d_i).
 * Returns 1 if the move keeps a >= 0 (then *delta, ap, as and d are set),
 * 0 if it is rejected by the positivity factor of Eq. (probability-density). */
int or_propose(int n_tau, int n_omega, const double *Khat, const double *Fhat, const double *x,
               double A, double B, const double *a, const double *R, int p, int s, double eps,
               double *delta, double *ap, double *as, double *d) {
    double r = 1.0 - eps;
    double dp = eps * (B - A * x[s]) / (x[p] - x[s]);
    double ds = eps * (B - A * x[p]) / (x[s] - x[p]);
    double new_p = r * a[p] + dp;
    double new_s = r * a[s] + ds;
    if (new_p < 0.0 || new_s < 0.0) return 0;
    double D = 0.0;
    for (int i = 0; i < n_tau; ++i) {
        double M = Fhat[i] - R[i];
        double di = eps * M - dp * Khat[(size_t)i * n_omega + p] - ds * Khat[(size_t)i * n_omega + s];
        d[i] = di;
        D += di * (2.0 * R[i] + di);
    }
    *delta = D;
    *ap = new_p;
    *as = new_s;
    return 1;
}

/* Amplitude factor of Eq. (amplitude-acceptance-adjustment): y = 1 if the
 * acceptance rate acc >= p, else (acc / p)^m, here with acc the fraction of
 * the walker's moves accepted in its previous sweep and a floor y_min.  An
 * integer m is applied by repeated multiplication. */
double or_amplitude(int accepted_prev, int n_omega, double y_p, double y_m, double y_min) {
    double acc = (double)accepted_prev / (double)n_omega;
    double y;
    if (acc >= y_p) y = 1.0;
    else {
        double q = acc / y_p;
        if (y_m == floor(y_m) && y_m >= 1.0 && y_m <= 16.0) {
            y = q;
            for (int k = 1; k < (int)y_m; ++k) y = y * q;
        } else {
            y = pow(q, y_m);
        }
    }
    if (y < y_min) y = y_min;
    return y;
}

/* --------------------------------------------------------- branching
 * Sec. 2.5.  Walker l gets weight w_l = exp[-Delta (z_l - P_r)] and multiplier
 * m_l = floor(w_l + xi_l).  With z normalised as (chi2 - min) / (mean - min)
 * the scale of Delta is O(1).  m_l >= k exactly when
 * Delta z_l + ln(k - xi_l) <= Delta P_r, so choosing P_r such that sum m = N
 * means: m_l = the number of walker l's "break points" b_lk = Delta z_l + ln(k - xi_l),
 * k = 1, 2, ..., among the N smallest break points of all walkers (ties go to the
 * lower walker index).  Z(Delta) = #{l : m_l = 0}; Delta is the value at which
 * Z equals the target round(f N): found by doubling from 1 and then bisecting,
 * stopping at the first trial with Z = target (else the upper end after 64 halvings).
 *
 * The N smallest break points are taken with a binary min-heap seeded with
 * every walker's k = 1 point: each pop of (l, k) adds one to m_l and pushes (l, k+1). */
typedef struct { double b; int l; int k; } or_bp;

static int bp_less(const or_bp *u, const or_bp *v) {
    if (u->b != v->b) return u->b < v->b;
    if (u->l != v->l) return u->l < v->l;
    return u->k < v->k;
}

static void heap_down(or_bp *h, int n, int i) {
    for (;;) {
        int c = 2 * i + 1;
        if (c >= n) return;
        if (c + 1 < n && bp_less(&h[c + 1], &h[c])) c = c + 1;
        if (!bp_less(&h[c], &h[i])) return;
        or_bp t = h[c]; h[c] = h[i]; h[i] = t;
        i = c;
    }
}

/* m_l for a given Delta; returns Z, the number of walkers with m_l = 0. */
int or_multipliers_at(int n, const double *z, const double *xi, double Delta, int *m, or_bp *heap) {
    for (int l = 0; l < n; ++l) {
        m[l] = 0;
        heap[l].b = Delta * z[l] + log(1.0 - xi[l]);
        heap[l].l = l;
        heap[l].k = 1;
    }
    for (int i = n / 2 - 1; i >= 0; --i) heap_down(heap, n, i);
    for (int taken = 0; taken < n; ++taken) {
        or_bp top = heap[0];
        m[top.l] += 1;
        heap[0].k = top.k + 1;
        heap[0].b = Delta * z[top.l] + log((double)(top.k + 1) - xi[top.l]);
        heap_down(heap, n, 0);
    }
    int Z = 0;
    for (int l = 0; l < n; ++l) Z += (m[l] == 0);
    return Z;
}

/* Full branching solve.  Writes m (sum m = n) and returns Delta. */
double or_branch_multipliers(int n, const double *chi2, const double *xi, double fraction, int *m) {
    int Zt = (int)floor(fraction * n + 0.5);
    if (Zt > n - 1) Zt = n - 1;
    if (Zt <= 0) { for (int l = 0; l < n; ++l) m[l] = 1; return 0.0; }
    double cmin = chi2[0], csum = 0.0;
    for (int l = 0; l < n; ++l) { if (chi2[l] < cmin) cmin = chi2[l]; csum += chi2[l]; }
    double spread = csum / n - cmin;
    double *z = (double *)malloc(sizeof(double) * n);
    or_bp *heap = (or_bp *)malloc(sizeof(or_bp) * n);
    for (int l = 0; l < n; ++l) z[l] = spread > 0.0 ? (chi2[l] - cmin) / spread : 0.0;

    double lo = 0.0, hi = 1.0;
    int Zhi = or_multipliers_at(n, z, xi, hi, m, heap);
    for (int it = 0; it < 64 && Zhi < Zt; ++it) {
        lo = hi;
        hi = 2.0 * hi;
        Zhi = or_multipliers_at(n, z, xi, hi, m, heap);
    }
    if (Zhi != Zt) {
        for (int it = 0; it < 64; ++it) {
            double mid = 0.5 * (lo + hi);
            if (mid <= lo || mid >= hi) break;
            int Zm = or_multipliers_at(n, z, xi, mid, m, heap);
            if (Zm == Zt) { hi = mid; Zhi = Zm; break; }
            if (Zm < Zt) lo = mid; else { hi = mid; Zhi = Zm; }
        }
    }
    or_multipliers_at(n, z, xi, hi, m, heap);
    free(z);
    free(heap);
    return hi;
}

/* Pairing for imprinting: the walkers with m = 0 in ascending index order are
 * matched with the surplus copies (walker l listed m_l - 1 times) in ascending
 * index order.  Returns the number of pairs. */
int or_pairs(int n, const int *m, int *zero_l, int *donor_l) {
    int nz = 0, nd = 0;
    for (int l = 0; l < n; ++l) if (m[l] == 0) zero_l[nz++] = l;
    for (int l = 0; l < n; ++l) for (int c = 1; c < m[l]; ++c) donor_l[nd++] = l;
    return nz < nd ? nz : nd;
}

/* --------------------------------------------------------- the anneal */
typedef struct {
    int n_sweeps;          /* length of the whole schedule */
    int sweeps_per_block;  /* k: a block is k sweeps, each followed by branching */
    int resync_every;      /* full residual recomputation period, in sweeps */
    int branching;         /* 0 / 1 */
    double T_start, T_end; /* in units of the start residue chi2_0 (Sec. 3) */
    double branch_fraction;
    double imprint_t;
    double move_scale;     /* d: eps is uniform on (-y d, y d) */
    double y_p, y_m, y_min;
    uint64_t seed;
    int schedule_kind;     /* 0: geometric T_start -> T_end; 1: self-cooling (Sec. self-cooling) */
    int adaptive;          /* 1: branching fraction and imprint strength follow the acceptance (Sec. 2.5) */
    double cool_begin;     /* self-cooling: fraction of the blocks boiled before the ramp */
    double freeze_begin;   /* self-cooling: fraction of the blocks after which the freeze-out starts */
    double smooth_s;       /* smoothing strength s (Sec. smoothing); 0: no smoothing */
    int walk_len;          /* L: steps of the index walk (Sec. 2.3); 0: uniform bins */
    double walk_uniform;   /* rho: probability that an index skips its walk (uniform admixture) */
    int hastings;          /* 1: Metropolis-Hastings acceptance with the move's Jacobian */
    int shared_bins;       /* W > 1: walkers w with equal w / W propose the bins of walker W (w / W) */
    int walker_base;       /* index in the whole population of this run's walker 0: the walker word of
                              every move counter is walker_base + w (a shard of a population split
                              over several runs draws exactly the words the whole run would) */
} or_params;

/* What the anneal carries from block to block besides the walkers. */
typedef struct {
    double *T;             /* [n_sweeps] absolute temperature of every sweep */
    double T_final;        /* self-cooling: temperature the freeze-out ends at, T_end chi2_0 */
    double acc_ref;        /* acceptance of the first block (adaptive branching); < 0 until known */
    double T_freeze;       /* self-cooling: chi2_min when the freeze-out began; < 0 until then */
    int64_t acc_before;    /* accepted moves of all walkers before the current block */
} or_state;

/* T for sweep n: geometric from T_start to T_end over the schedule, times chi2_0. */
double or_temperature(const or_params *prm, int n, double chi2_0) {
    double t = prm->n_sweeps > 1 ? (double)n / (double)(prm->n_sweeps - 1) : 0.0;
    return chi2_0 * (prm->T_start * pow(prm->T_end / prm->T_start, t));
}

/* Self-cooling, Sec. self-cooling.  Reading: the schedule is cut into n_blocks
 * blocks of k sweeps; T is constant within a block.  Block 0 runs at the start
 * residue chi2_0 (the population's mean residue then).  Block b >= 1 takes the
 * mean residue cbar and the smallest residue cmin of the population at the end
 * of block b - 1 (after its residual recomputation, before branching):
 *   boiling,    b < b_cool:            T = cbar;
 *   cooling,    b_cool <= b < b_freeze: T = cbar^(1 - x) cmin^x,
 *               x = (b - b_cool + 1) / (b_freeze - b_cool), reaching cmin;
 *   freeze-out, b >= b_freeze:         T = T_F (T_final / T_F)^y,
 *               y = (b - b_freeze + 1) / (n_blocks - b_freeze): from below
 *               T_F = cmin at the first freeze-out block, lowered by the same
 *               proportion every block, to the schedule's end temperature
 *               T_final at the last block (held at T_F if T_F <= T_final). */
void or_cooling_blocks(int n_blocks, double cool_begin, double freeze_begin, int *b_cool, int *b_freeze) {
    int bc = (int)floor(cool_begin * (double)n_blocks + 0.5);
    int bf = (int)floor(freeze_begin * (double)n_blocks + 0.5);
    if (bc < 0) bc = 0;
    if (bc > n_blocks) bc = n_blocks;
    if (bf < bc) bf = bc;
    if (bf > n_blocks) bf = n_blocks;
    *b_cool = bc;
    *b_freeze = bf;
}

double or_self_cooling(int b, int n_blocks, int b_cool, int b_freeze, double cbar, double cmin, double T_final,
                       double *T_freeze) {
    if (b < b_cool) return cbar;
    if (b < b_freeze) {
        double x = (double)(b - b_cool + 1) / (double)(b_freeze - b_cool);
        return pow(cbar, 1.0 - x) * pow(cmin, x);
    }
    if (*T_freeze < 0.0) *T_freeze = cmin;
    if (!(*T_freeze > T_final)) return *T_freeze;
    double y = (double)(b - b_freeze + 1) / (double)(n_blocks - b_freeze);
    return *T_freeze * pow(T_final / *T_freeze, y);
}

/* Fills the temperature table: the whole geometric schedule, or block 0 of the
 * self-cooling one (the other blocks are set as the anneal reaches them). */
void or_init_temperatures(const or_params *prm, double chi2_0, double *T) {
    for (int n = 0; n < prm->n_sweeps; ++n) {
        if (prm->schedule_kind == 1)
            T[n] = n < prm->sweeps_per_block ? chi2_0 : NAN;
        else
            T[n] = or_temperature(prm, n, chi2_0);
    }
}

/* Adaptive branching, Sec. 2.5: the branching fraction and the imprint strength
 * are reduced as the acceptance drops.  Reading: both are multiplied by
 * min(1, acc / acc_ref), acc the block's acceptance rate and acc_ref that of the
 * first block. */
double or_adaptive_scale(double acc, double acc_ref) {
    return (acc_ref > 0.0 && acc < acc_ref) ? acc / acc_ref : 1.0;
}

/* Smoothing, Sec. smoothing: three-point stencil of strength s,
 *   a_j <- s a_{j-1} + (1 - 2s) a_j + s a_{j+1}  (0 < j < N-1),
 *   a_0 <- (1 - s) a_0 + s a_1,   a_{N-1} <- (1 - s) a_{N-1} + s a_{N-2},
 * all from the old values.  It keeps sum_j a_j; the second sum rule moves by
 * s dw (a_0 - a_{N-1}).  Renormalisation (reading): the tilt
 * a_j <- a_j (1 + beta (x_j - m)), m = B'/A', beta = (B - B') / sum_j a_j (x_j - m)^2,
 * which keeps sum_j a_j and restores sum_j a_j x_j = B (skipped when the tilt
 * could make a factor negative: |beta| max_j |x_j - m| >= 1/2). */
void or_smooth(int n_omega, const double *x, double B, double s, double *a) {
    int N = n_omega;
    double c = 1.0 - 2.0 * s, e = 1.0 - s;
    double prev = a[0];
    a[0] = e * a[0] + s * a[1];
    for (int j = 1; j < N - 1; ++j) {
        double cur = a[j];
        a[j] = s * prev + c * cur + s * a[j + 1];
        prev = cur;
    }
    a[N - 1] = e * a[N - 1] + s * prev;
    double A1 = 0.0, B1 = 0.0;
    for (int j = 0; j < N; ++j) {
        A1 += a[j];
        B1 += a[j] * x[j];
    }
    if (!(A1 > 0.0)) return;
    double m = B1 / A1, V = 0.0;
    for (int j = 0; j < N; ++j) {
        double d = x[j] - m;
        V += a[j] * d * d;
    }
    double beta = V > 0.0 ? (B - B1) / V : 0.0;
    double span = fabs(x[0] - m) > fabs(x[N - 1] - m) ? fabs(x[0] - m) : fabs(x[N - 1] - m);
    if (!(fabs(beta) * span < 0.5)) beta = 0.0;
    for (int j = 0; j < N; ++j) a[j] = a[j] * (1.0 + beta * (x[j] - m));
}

static uint64_t fnv_step(uint64_t h, unsigned code) {
    h ^= (uint64_t)code;
    h *= 0x100000001B3ull;
    return h;
}

/* Bin choice of a move, Sec. 2.3 (selection of update frequencies).  With a
 * zero-length walk p is uniform on the bins and s uniform on the others.
 * Reading for L > 0: each index takes L steps of an independence walk whose
 * stationary law is a_j / A: from the current bin j, propose j' uniform and move
 * there when u a_j <= a_j' (probability min(1, a_j'/a_j)).  p walks first from
 * its uniform start; s then starts uniform on the bins other than the final p
 * and walks with proposals drawn on those bins.  Each index skips its walk with
 * probability rho (the uniform admixture).  Words: starts from words 0 and 1 of
 * the move's counter (mv, n, w, 0); step t = 1..L from counter (mv, n, w, 1 + t)
 * as (proposal of p, acceptance of p, proposal of s, acceptance of s); the two
 * admixture uniforms from words 0 and 1 of counter (mv, n, w, 2 + L). */
void or_move_bins(const or_params *prm, int n_omega, const double *a, uint32_t w0, uint32_t w1, int mv, int n, int w,
                  int *p_out, int *s_out) {
    int L = prm->walk_len;
    int p = (int)(((uint64_t)w0 * (uint64_t)n_omega) >> 32);
    int walk_p = 0, walk_s = 0;
    if (L > 0) {
        uint32_t mix[4];
        draw(prm->seed, (uint32_t)mv, (uint32_t)n, (uint32_t)w, (uint32_t)(2 + L), mix);
        walk_p = !(unit(mix[0]) < prm->walk_uniform);
        walk_s = !(unit(mix[1]) < prm->walk_uniform);
    }
    for (int t = 1; t <= L && walk_p; ++t) {
        uint32_t r[4];
        draw(prm->seed, (uint32_t)mv, (uint32_t)n, (uint32_t)w, (uint32_t)(1 + t), r);
        int j = (int)(((uint64_t)r[0] * (uint64_t)n_omega) >> 32);
        if (unit(r[1]) * a[p] <= a[j]) p = j;
    }
    int s = (int)(((uint64_t)w1 * (uint64_t)(n_omega - 1)) >> 32);
    if (s >= p) s += 1;
    for (int t = 1; t <= L && walk_s; ++t) {
        uint32_t r[4];
        draw(prm->seed, (uint32_t)mv, (uint32_t)n, (uint32_t)w, (uint32_t)(1 + t), r);
        int j = (int)(((uint64_t)r[2] * (uint64_t)(n_omega - 1)) >> 32);
        if (j >= p) j += 1;
        if (unit(r[3]) * a[s] <= a[j]) s = j;
    }
    *p_out = p;
    *s_out = s;
}

/* Acceptance of a move that passed the positivity test.  Plain: the Metropolis
 * test for density exp(-chi2 / T), Eq. (probability-density): D <= 0 or
 * u < exp(-D / T).  Hastings (reading of the move's detailed balance; the paper
 * claims ergodicity only): the move (a, eps) -> (r a + delta(eps), -eps / r),
 * r = 1 - eps, is its own inverse; on the (N_omega - 2)-dimensional manifold of
 * the two sum rules its Jacobian is r^(N_omega - 2) times |d eps'/d eps| = r^-2.
 * The reverse move needs |eps / r| < y d to be proposable; then accept when
 * u < exp(-D / T) r^(N_omega - 4). */
int or_accept(const or_params *prm, int n_omega, double yd, double eps, double D, double T, double u) {
    if (!prm->hastings) return D <= 0.0 || u < exp(-D / T);
    double r = 1.0 - eps;
    if (!(fabs(eps / r) < yd)) return 0;
    return u < exp(-D / T + (double)(n_omega - 4) * log(r));
}

/* Puts a spectrum back on both sum rules: a_j <- a_j kappa (1 + lambda (x_j - c)),
 * c = B'/A', kappa = A / A', lambda = (B/A - c) A' / sum_j a_j (x_j - c)^2 (sums in bin
 * order; lambda = 0 when the tilt could turn a factor negative).  In exact arithmetic
 * a no-op.  The Hastings chain needs it: a move maps the sum errors e to r e, and its
 * accepted moves have r > 1 on average, so rounding errors grow geometrically without it. */
void or_restore(int n_omega, const double *x, double A, double B, double *a) {
    int N = n_omega;
    double A1 = 0.0, B1 = 0.0;
    for (int j = 0; j < N; ++j) {
        A1 += a[j];
        B1 += a[j] * x[j];
    }
    if (!(A1 > 0.0)) return;
    double c = B1 / A1, V = 0.0;
    for (int j = 0; j < N; ++j) {
        double d = x[j] - c;
        V += a[j] * d * d;
    }
    double kappa = A / A1;
    double lambda = V > 0.0 ? (B / A - c) * A1 / V : 0.0;
    if (!(fabs(lambda * (x[N - 1] - x[0])) < 0.5)) lambda = 0.0;
    for (int j = 0; j < N; ++j) a[j] = a[j] * (kappa * (1.0 + lambda * (x[j] - c)));
}

/* Shared bins (a reading of the move beyond the paper, which draws every walker's
 * indices on its own): with W > 1 the walkers w with equal w / W all propose, at
 * move mv of sweep n, the bins that the group's first walker g = W (w / W) draws
 * from words 0 and 1 of its own counter (mv, n, g, 0); each walker keeps words 2
 * and 3 of its own counter for its amplitude and its acceptance draw.  A walker's
 * bins stay uniform and independent of its spectrum, so each walker's chain is the
 * paper's chain; only the walkers of a group become correlated.  With W <= 1 every
 * walker uses its own words 0 and 1 (the paper's move). */
static void bin_words(const or_params *prm, int mv, int n, int w, const uint32_t own[4], uint32_t *w0, uint32_t *w1) {
    if (prm->shared_bins > 1) {
        uint32_t g[4];
        draw(prm->seed, (uint32_t)mv, (uint32_t)n, (uint32_t)(w - w % prm->shared_bins), 0u, g);
        *w0 = g[0];
        *w1 = g[1];
    } else {
        *w0 = own[0];
        *w1 = own[1];
    }
}

/* One sweep (N_omega proposals) of walker w at sweep index n. */
static void sweep_walker(int n_tau, int n_omega, const double *Khat, const double *Fhat,
                         const double *x, double A, double B, const or_params *prm, double T,
                         int n, int w, double *a, double *R, double *chi2, int *acc_prev,
                         uint64_t *hash, int64_t *n_acc, int64_t *n_pos, double *d) {
    double y = or_amplitude(*acc_prev, n_omega, prm->y_p, prm->y_m, prm->y_min);
    double dmove = prm->move_scale > 0.0 ? prm->move_scale : 1.0 / n_omega;
    int accepted = 0;
    const int wg = w + prm->walker_base;   /* the walker's index in the whole population */
    for (int mv = 0; mv < n_omega; ++mv) {
        uint32_t rnd[4];
        draw(prm->seed, (uint32_t)mv, (uint32_t)n, (uint32_t)wg, 0u, rnd);
        uint32_t w0, w1;
        bin_words(prm, mv, n, wg, rnd, &w0, &w1);
        int p, s;
        or_move_bins(prm, n_omega, a, w0, w1, mv, n, wg, &p, &s);
        double eps = (y * dmove) * (2.0 * unit(rnd[2]) - 1.0);
        double u = unit(rnd[3]);
        double D, ap, as;
        unsigned code;
        if (!or_propose(n_tau, n_omega, Khat, Fhat, x, A, B, a, R, p, s, eps, &D, &ap, &as, d)) {
            code = 2;
            *n_pos += 1;
        } else if (or_accept(prm, n_omega, y * dmove, eps, D, T, u)) {
            double r = 1.0 - eps;
            for (int j = 0; j < n_omega; ++j) a[j] = r * a[j];
            a[p] = ap;
            a[s] = as;
            for (int i = 0; i < n_tau; ++i) R[i] = R[i] + d[i];
            *chi2 = *chi2 + D;
            accepted += 1;
            code = 1;
        } else {
            code = 0;
        }
        *hash = fnv_step(*hash, code);
    }
    *acc_prev = accepted;
    *n_acc += accepted;
}

/* Imprinting, Sec. 2.5: a^(l1) <- t a^(l2) + (1 - t) a^(l1); by linearity the residual
 * mixes the same way, and chi2 of l1 is summed again from the mixed residual.  Returns it. */
double or_imprint(int n_omega, int n_tau, double t, double *a1, double *R1, const double *a2, const double *R2) {
    double omt = 1.0 - t;
    for (int j = 0; j < n_omega; ++j) a1[j] = t * a2[j] + omt * a1[j];
    double c2 = 0.0;
    for (int i = 0; i < n_tau; ++i) {
        R1[i] = t * R2[i] + omt * R1[i];
        c2 += R1[i] * R1[i];
    }
    return c2;
}

/* Runs sweeps [sweep_begin, sweep_end) of the schedule on all walkers.
 * After sweep n the residuals are recomputed from scratch when (n+1) is a
 * multiple of resync_every or of sweeps_per_block, or n is the last sweep; at
 * each block end ((n+1) a multiple of sweeps_per_block) the population is
 * branched with imprinting if enabled.  acc_trace, if given, receives the
 * accepted-move count of every walker in every sweep run ([sweep][walker]);
 * m_trace, if given, the multipliers of every branching ([event][walker]). */
int or_anneal(int n_tau, int n_omega, int n_walkers, const double *Khat, const double *Fhat,
              const double *x, double A, double B, const or_params *prm, or_state *st,
              double *a, double *R, double *chi2, int *acc_prev, uint64_t *hash,
              int64_t *n_acc, int64_t *n_pos, int sweep_begin, int sweep_end,
              int *acc_trace, int *m_trace, double *delta_trace) {
    int events = 0;
    for (int n = sweep_begin; n < sweep_end; ++n) {
        double T = st->T[n];
#pragma omp parallel for schedule(static)
        for (int w = 0; w < n_walkers; ++w) {
            double *d = (double *)malloc(sizeof(double) * (n_tau > 0 ? n_tau : 1));
            sweep_walker(n_tau, n_omega, Khat, Fhat, x, A, B, prm, T, n, w,
                         a + (size_t)w * n_omega, R + (size_t)w * n_tau, chi2 + w,
                         acc_prev + w, hash + w, n_acc + w, n_pos + w, d);
            free(d);
        }
        if (acc_trace)
            for (int w = 0; w < n_walkers; ++w)
                acc_trace[(size_t)(n - sweep_begin) * n_walkers + w] = acc_prev[w];
        int k = prm->sweeps_per_block;
        int block_end = ((n + 1) % k) == 0;
        if (((n + 1) % prm->resync_every) == 0 || block_end || n + 1 == prm->n_sweeps) {
#pragma omp parallel for schedule(static)
            for (int w = 0; w < n_walkers; ++w) {
                if (prm->hastings) or_restore(n_omega, x, A, B, a + (size_t)w * n_omega);
                chi2[w] = or_residual(n_tau, n_omega, Khat, Fhat, a + (size_t)w * n_omega,
                                      R + (size_t)w * n_tau);
            }
        }
        /* End of block b: its acceptance and residue statistics (after the
         * recomputation above, before branching), then branching (Sec. 2.5),
         * smoothing (Sec. smoothing) and the next block's temperature
         * (Sec. self-cooling). */
        double scale = 1.0, cbar = 0.0, cmin = chi2[0];
        if (block_end && (prm->schedule_kind == 1 || prm->adaptive)) {
            int64_t acc_total = 0;
            for (int w = 0; w < n_walkers; ++w) acc_total += n_acc[w];
            double acc = (double)(acc_total - st->acc_before) / ((double)k * (double)n_walkers * (double)n_omega);
            st->acc_before = acc_total;
            if (prm->adaptive) {
                if (st->acc_ref < 0.0) st->acc_ref = acc;
                scale = or_adaptive_scale(acc, st->acc_ref);
            }
            for (int w = 0; w < n_walkers; ++w) {
                cbar += chi2[w];
                if (chi2[w] < cmin) cmin = chi2[w];
            }
            cbar /= (double)n_walkers;
        }
        if (block_end && prm->branching && n_walkers > 1) {
            int b = (n + 1) / k - 1;
            double *xi = (double *)malloc(sizeof(double) * n_walkers);
            int *m = (int *)malloc(sizeof(int) * n_walkers);
            int *zl = (int *)malloc(sizeof(int) * n_walkers);
            int *dl = (int *)malloc(sizeof(int) * n_walkers);
            for (int l = 0; l < n_walkers; ++l) {
                uint32_t rnd[4];
                draw(prm->seed, (uint32_t)l, (uint32_t)b, 0u, 1u, rnd);
                xi[l] = unit(rnd[0]);
            }
            double Delta = or_branch_multipliers(n_walkers, chi2, xi, prm->branch_fraction * scale, m);
            int np = or_pairs(n_walkers, m, zl, dl);
            double t = prm->imprint_t * scale;
            for (int q = 0; q < np; ++q)
                chi2[zl[q]] = or_imprint(n_omega, n_tau, t, a + (size_t)zl[q] * n_omega, R + (size_t)zl[q] * n_tau,
                                         a + (size_t)dl[q] * n_omega, R + (size_t)dl[q] * n_tau);
            if (m_trace) memcpy(m_trace + (size_t)events * n_walkers, m, sizeof(int) * n_walkers);
            if (delta_trace) delta_trace[events] = Delta;
            events += 1;
            free(xi); free(m); free(zl); free(dl);
        }
        if (block_end && prm->smooth_s > 0.0) {
#pragma omp parallel for schedule(static)
            for (int w = 0; w < n_walkers; ++w) {
                or_smooth(n_omega, x, B, prm->smooth_s, a + (size_t)w * n_omega);
                chi2[w] = or_residual(n_tau, n_omega, Khat, Fhat, a + (size_t)w * n_omega,
                                      R + (size_t)w * n_tau);
            }
        }
        if (block_end && prm->schedule_kind == 1 && n + 1 < prm->n_sweeps) {
            int n_blocks = (prm->n_sweeps + k - 1) / k, bc, bf;
            or_cooling_blocks(n_blocks, prm->cool_begin, prm->freeze_begin, &bc, &bf);
            int b_next = (n + 1) / k;
            double Tn = or_self_cooling(b_next, n_blocks, bc, bf, cbar, cmin, st->T_final, &st->T_freeze);
            for (int q = n + 1; q < n + 1 + k && q < prm->n_sweeps; ++q) st->T[q] = Tn;
        }
    }
    return events;
}

/* Stochastic average, Sec. 1: mean over walkers whose chi2 <= factor * min chi2,
 * with the standard error of the mean (sample std / sqrt(n)) per bin. */
int or_average(int n_walkers, int n_omega, const double *a, const double *chi2, double factor,
               double *mean, double *err) {
    double cmin = chi2[0];
    for (int w = 1; w < n_walkers; ++w) if (chi2[w] < cmin) cmin = chi2[w];
    double cut = factor * cmin;
    int used = 0;
    for (int j = 0; j < n_omega; ++j) { mean[j] = 0.0; err[j] = 0.0; }
    for (int w = 0; w < n_walkers; ++w) {
        if (!(chi2[w] <= cut)) continue;
        used += 1;
        for (int j = 0; j < n_omega; ++j) mean[j] += a[(size_t)w * n_omega + j];
    }
    for (int j = 0; j < n_omega; ++j) mean[j] /= used;
    if (used > 1) {
        for (int w = 0; w < n_walkers; ++w) {
            if (!(chi2[w] <= cut)) continue;
            for (int j = 0; j < n_omega; ++j) {
                double e = a[(size_t)w * n_omega + j] - mean[j];
                err[j] += e * e;
            }
        }
        for (int j = 0; j < n_omega; ++j) err[j] = sqrt(err[j] / (used - 1)) / sqrt((double)used);
    }
    return used;
}
