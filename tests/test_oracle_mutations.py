"""Planted mistakes: each mutated copy of the oracle source (compiled here, never committed)
must fail at least one pin, so a plausible slip in the oracle cannot pass unnoticed."""
import ctypes
import os
import subprocess
import tempfile

import numpy as np
import pytest

import oracle as O

SRC = os.path.join(os.path.dirname(O.__file__), "sail_oracle.c")

MUTATIONS = {
    # delta_s with the wrong sign of the gap
    "delta_s_sign": ("double ds = eps * (B - A * x[p]) / (x[s] - x[p]);",
                     "double ds = eps * (B - A * x[p]) / (x[p] - x[s]);"),
    # Delta chi2 without the d^2 term
    "drop_d2": ("D += di * (2.0 * R[i] + di);", "D += di * (2.0 * R[i]);"),
    # kernel without the 1/tau factor
    "kernel_tau": ("/ (2.0 * OR_PI * tau[i]);", "/ (2.0 * OR_PI);"),
    # a Philox multiplier swapped for the other one
    "philox_const": ("uint64_t p0 = (uint64_t)0xD2511F53u * x[0];", "uint64_t p0 = (uint64_t)0xCD9E8D57u * x[0];"),
    # break points ln(k + xi) instead of ln(k - xi)
    "branch_sign": ("heap[0].b = Delta * z[top.l] + log((double)(top.k + 1) - xi[top.l]);",
                    "heap[0].b = Delta * z[top.l] + log((double)(top.k + 1) + xi[top.l]);"),
    # adaptive branching that forgets to scale the imprint strength
    "imprint_unscaled": ("double t = prm->imprint_t * scale;",
                         "double t = prm->imprint_t;"),
    # smoothing stencil with the end weight in the interior
    "stencil_weight": ("double c = 1.0 - 2.0 * s, e = 1.0 - s;", "double c = 1.0 - s, e = 1.0 - s;"),
    # self-cooling ramp running from the minimum to the mean
    "cooling_reversed": ("return pow(cbar, 1.0 - x) * pow(cmin, x);", "return pow(cbar, x) * pow(cmin, 1.0 - x);"),
    # smoothing renormalisation tilting the wrong way
    "renorm_sign": ("double beta = V > 0.0 ? (B - B1) / V : 0.0;", "double beta = V > 0.0 ? (B1 - B) / V : 0.0;"),
    # index walk accepting by the inverse ratio (law a_j^-1 instead of a_j)
    "walk_ratio": ("if (unit(r[1]) * a[p] <= a[j]) p = j;", "if (unit(r[1]) * a[j] <= a[p]) p = j;"),
    # s walk whose proposals may land on p
    "walk_skip": ("        if (j >= p) j += 1;\n        if (unit(r[3])", "        if (unit(r[3])"),
    # Hastings factor with the manifold's Jacobian alone (no d eps'/d eps)
    "hastings_exponent": ("(double)(n_omega - 4) * log(r)", "(double)(n_omega - 2) * log(r)"),
    # Hastings acceptance without the reverse move's feasibility
    "hastings_reverse": ("    if (!(fabs(eps / r) < yd)) return 0;\n", ""),
    # shared bins drawn from the group's index instead of its first walker's counter
    "shared_group_index": ("(uint32_t)(w - w % prm->shared_bins)", "(uint32_t)(w / prm->shared_bins)"),
    # shared bins ignored (every walker its own bins)
    "shared_ignored": ("    if (prm->shared_bins > 1) {", "    if (prm->shared_bins > 1 << 30) {"),
    # Metropolis test for exp(+chi2 / T)
    "metropolis_sign": ("return D <= 0.0 || u < exp(-D / T);", "return D <= 0.0 || u < exp(D / T);"),
    # accepted move that forgets to rescale the other bins by r
    "rescale_dropped": ("for (int j = 0; j < n_omega; ++j) a[j] = r * a[j];", ""),
    # residual updated with the wrong sign of d
    "residual_sign": ("R[i] = R[i] + d[i];", "R[i] = R[i] - d[i];"),
    # amplitude heuristic with one power of the acceptance too many
    "amplitude_power": ("for (int k = 1; k < (int)y_m; ++k) y = y * q;", "for (int k = 1; k <= (int)y_m; ++k) y = y * q;"),
    # start-spectrum bisection moving the wrong end
    "start_bisection": ("if (s1 / s0 > target) lo = mid; else hi = mid;", "if (s1 / s0 > target) hi = mid; else lo = mid;"),
    # geometric schedule running from T_end up to T_start
    "schedule_inverted": ("pow(prm->T_end / prm->T_start, t)", "pow(prm->T_start / prm->T_end, t)"),
    # amplitude and acceptance draws taken from each other's word
    "words_swapped": ("double eps = (y * dmove) * (2.0 * unit(rnd[2]) - 1.0);\n        double u = unit(rnd[3]);",
                      "double eps = (y * dmove) * (2.0 * unit(rnd[3]) - 1.0);\n        double u = unit(rnd[2]);"),
    # the bins' word mapped by the other rounding (ceiling instead of floor of w N / 2^32)
    "bin_rounding": ("int p = (int)(((uint64_t)w0 * (uint64_t)n_omega) >> 32);",
                     "int p = (int)((((uint64_t)w0 * (uint64_t)n_omega) + 0xFFFFFFFFull) >> 32) % n_omega;"),
    # sum-rule restoration tilting the wrong way
    "restore_tilt_sign": ("double lambda = V > 0.0 ? (B / A - c) * A1 / V : 0.0;",
                          "double lambda = V > 0.0 ? (c - B / A) * A1 / V : 0.0;"),
    # sum-rule restoration without its guard against negative factors
    "restore_unguarded": ("    if (!(fabs(lambda * (x[N - 1] - x[0])) < 0.5)) lambda = 0.0;\n", ""),
    # average that drops walkers exactly at the chi2 cut
    "average_cut": ("if (!(chi2[w] <= cut)) continue;\n        used += 1;", "if (!(chi2[w] < cut)) continue;\n        used += 1;"),
}


def _build(name):
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert old in src, name
    td = tempfile.mkdtemp()
    c = os.path.join(td, "m.c")
    open(c, "w").write(src.replace(old, new))
    so = os.path.join(td, "m.so")
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-shared", "-fPIC", "-o", so, c, "-lm"])
    return so


def _with_lib(so):
    """Re-type a mutated library with the oracle's own signatures."""
    saved = O._lib
    O._lib = None
    O._LIB_saved = O._LIB
    O._LIB = so
    orig_build = O.build
    O.build = lambda force=False: so
    try:
        return O.lib()
    finally:
        O.build = orig_build
        O._LIB = O._LIB_saved
        O._lib = saved


def _pins_pass(L):
    saved = O._lib
    O._lib = L
    try:
        from tests import test_oracle_model as M, test_oracle_moves as V, test_oracle_branching as B
        from tests import test_oracle_protocol as Q
        from tests import test_oracle_walk as Wk
        from tests import test_oracle_hastings as Hs
        from tests import test_oracle_shared as Sh
        from tests import test_oracle_restore as Rs
        from tests import test_oracle_sweep_definition as Sd
        checks = [M.test_kernel_is_the_bin_integral, M.test_philox_inverts_to_its_counter,
                  V.test_delta_formulas_keep_both_sums, V.test_delta_chi2_matches_brute_force,
                  lambda: B.test_multipliers_match_enumeration(0),
                  Q.test_smoothing_worked_example, Q.test_smoothing_keeps_both_sum_rules,
                  Q.test_self_cooling_phases, Q.test_adaptive_branching_scales_fraction_and_imprint,
                  lambda: Wk.test_walk_law_matches_the_matrix_power(3, 0.0),
                  lambda: Hs.test_jacobian_is_r_to_the_n_minus_4(0.07),
                  Hs.test_hastings_chain_samples_the_uniform_polytope,
                  lambda: Sh.test_first_walkers_follow_their_own_bins(4),
                  V.test_zero_temperature_never_raises_chi2, V.test_sweeps_keep_invariants_and_bookkeeping,
                  V.test_amplitude_heuristic, V.test_temperature_schedule_is_geometric,
                  lambda: M.test_start_spectrum_sum_rules_and_max_entropy(0.15),
                  B.test_average_over_good_walkers,
                  Rs.test_hand_worked_example, Rs.test_tilt_skipped_when_a_factor_could_turn_negative,
                  Sd.test_oracle_sweeps_are_the_definition]
        for c in checks:
            try:
                c()
            except AssertionError:
                return False
        return True
    finally:
        O._lib = saved


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name):
    L = _with_lib(_build(name))
    assert not _pins_pass(L), f"mutation {name} passed every pin"


def test_unmutated_oracle_passes_the_same_checks():
    assert _pins_pass(O.lib())
