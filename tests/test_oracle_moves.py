"""Pins for the oracle's Metropolis sweep: sum rules, positivity, chi2 bookkeeping,
degenerate cases of the move, the temperature schedule and the amplitude heuristic."""
import numpy as np
import pytest

import oracle as O
from workloads import make_problem, Peak, tiny_double_lorentz


def _small_problem(n_tau=6, n_omega=10, W=4.0, seed=0):
    tau = 0.5 * np.arange(n_tau, dtype=np.float64)
    return make_problem("small", tau, n_omega, W, [Peak("lorentz", 1.5, 0.4, 1.0)], 1e-3, seed, 4)


def test_delta_formulas_keep_both_sums():
    """Eqs. (update-delta-p/s): with r = 1 - eps the move keeps sum a and sum a x."""
    P = tiny_double_lorentz()
    K, Fh, dw = O.tables(P.tau, P.F, P.sigma, P.omega)
    a, _ = O.initial_spectrum(P.omega, P.A, P.B)
    R, _ = O.residual(K, Fh, a)
    rng = np.random.default_rng(0)
    for _ in range(200):
        p, s = rng.choice(P.n_omega, 2, replace=False)
        eps = rng.uniform(-0.02, 0.02)
        ok, D, ap, as_, d = O.propose(K, Fh, P.omega, P.A, P.B, a, R, p, s, eps)
        if not ok:
            continue
        b = (1 - eps) * a
        b[p], b[s] = ap, as_
        assert abs(b.sum() - P.A) <= 1e-13 * P.A
        assert abs(b @ P.omega - P.B) <= 1e-13 * P.B


def test_delta_chi2_matches_brute_force():
    """Delta chi2 and d from the O(N_tau) update equal recomputation from scratch."""
    P = _small_problem()
    K, Fh, dw = O.tables(P.tau, P.F, P.sigma, P.omega)
    rng = np.random.default_rng(1)
    for trial in range(300):
        a = rng.uniform(0.0, 2.0, P.n_omega)
        A, B = a.sum(), a @ P.omega
        R, chi2 = O.residual(K, Fh, a)
        p, s = rng.choice(P.n_omega, 2, replace=False)
        eps = rng.uniform(-0.3, 0.3)
        ok, D, ap, as_, d = O.propose(K, Fh, P.omega, A, B, a, R, p, s, eps)
        b = (1 - eps) * a
        dp = eps * (B - A * P.omega[s]) / (P.omega[p] - P.omega[s])
        ds = eps * (B - A * P.omega[p]) / (P.omega[s] - P.omega[p])
        b[p] += dp
        b[s] += ds
        assert ok == (b[p] >= 0 and b[s] >= 0)
        if not ok:
            continue
        R2, chi2b = O.residual(K, Fh, b)
        scale = np.sum(np.abs(d * (2 * R + d))) + 1e-300
        assert abs(D - (chi2b - chi2)) <= 1e-11 * max(scale, chi2)
        np.testing.assert_allclose(R + d, R2, rtol=1e-11, atol=1e-11 * np.abs(R).max())


def test_special_frequency_suppresses_the_other_bin():
    """Eq. (special-frequency): if x_s = B/A then delta_p = 0 and a_p just rescales."""
    omega = (np.arange(8) + 0.5) * 0.5
    tau = 0.3 * np.arange(5.0)
    a = np.linspace(1.0, 2.0, 8)
    A = a.sum()
    s = 3
    B = A * omega[s]
    K, Fh, _ = O.tables(tau, np.ones(5), np.ones(5), omega)
    R, _ = O.residual(K, Fh, a)
    ok, D, ap, as_, d = O.propose(K, Fh, omega, A, B, a, R, 6, s, 0.05)
    assert ok and ap == 0.95 * a[6]
    assert abs(as_ - (0.95 * a[s] + 0.05 * A)) < 1e-14 * A


def test_two_bin_model_is_frozen():
    """With two bins the two sum rules fix the spectrum: every move returns it unchanged,
    Delta chi2 = 0 and every move is accepted at any temperature."""
    tau = np.array([0.0, 0.5, 1.0])
    omega = np.array([0.5, 1.5])
    F = np.array([0.2, 0.1, 0.05])
    sig = np.full(3, 1e-3)
    A, B = 2.0, 1.3
    s = O.Schedule(n_sweeps=40, sweeps_per_block=10, resync_every=1000, T_start=1e-12, T_end=1e-12, seed=5)
    an = O.Anneal(tau, F, sig, omega, A, B, 3, s)
    a0 = an.a.copy()
    acc, _, _ = an.run(trace=True)
    assert np.all(acc == 2)
    np.testing.assert_allclose(an.a, a0, rtol=1e-13)


def _run_checking_every_sweep(P, sched, n_walkers):
    an = O.Anneal(P.tau, P.F, P.sigma, P.omega, P.A, P.B, n_walkers, sched)
    K, Fh = an.K, an.Fh
    prev = an.chi2.copy()
    for n in range(sched.n_sweeps):
        acc, _, _ = an.run(1, trace=True)
        assert np.all(an.a >= 0)
        np.testing.assert_allclose(an.a.sum(1), P.A, rtol=1e-12)
        np.testing.assert_allclose(an.a @ P.omega, P.B, rtol=1e-12)
        for w in range(n_walkers):
            R, chi2 = O.residual(K, Fh, an.a[w])
            np.testing.assert_allclose(an.R[w], R, rtol=1e-9, atol=1e-9 * np.abs(R).max())
            assert abs(an.chi2[w] - chi2) <= 1e-9 * max(chi2, np.abs(R).max() ** 2)
        yield an, acc, prev
        prev = an.chi2.copy()


def test_sweeps_keep_invariants_and_bookkeeping():
    """After every sweep: a >= 0, both sums hold to 1e-12 and the incrementally
    updated residual and chi2 equal a from-scratch recomputation (no resync runs)."""
    P = _small_problem(n_tau=8, n_omega=12)
    sched = O.Schedule(n_sweeps=30, sweeps_per_block=1000, resync_every=1000, T_start=1.0,
                       T_end=1e-3, move_scale=0.2, seed=11)
    n_acc = 0
    for an, acc, _ in _run_checking_every_sweep(P, sched, 6):
        n_acc += acc.sum()
    assert n_acc > 0


def test_zero_temperature_never_raises_chi2():
    P = _small_problem(n_tau=8, n_omega=12, seed=3)
    sched = O.Schedule(n_sweeps=20, sweeps_per_block=1000, resync_every=1000, T_start=1e-300,
                       T_end=1e-300, move_scale=0.2, seed=2)
    for an, acc, prev in _run_checking_every_sweep(P, sched, 4):
        assert np.all(an.chi2 <= prev * (1 + 1e-12))


def test_infinite_temperature_accepts_every_positive_move():
    P = _small_problem(n_tau=8, n_omega=12, seed=4)
    sched = O.Schedule(n_sweeps=10, sweeps_per_block=1000, resync_every=1000, T_start=1e300,
                       T_end=1e300, move_scale=0.05, seed=3)
    an = O.Anneal(P.tau, P.F, P.sigma, P.omega, P.A, P.B, 5, sched)
    acc, _, _ = an.run(trace=True)
    assert acc.sum() + an.n_pos.sum() == 10 * 5 * P.n_omega
    assert an.n_acc.sum() == acc.sum()


def test_temperature_schedule_is_geometric():
    s = O.Schedule(n_sweeps=101, T_start=10.0, T_end=1e-3)
    P = tiny_double_lorentz()
    an = O.Anneal(P.tau, P.F, P.sigma, P.omega, P.A, P.B, 2, s)
    T = np.array([an.temperature(n) for n in range(101)])
    assert abs(T[0] - 10 * an.chi2_0) <= 1e-15 * T[0]
    assert abs(T[-1] - 1e-3 * an.chi2_0) <= 1e-13 * T[-1]
    ratios = T[1:] / T[:-1]
    np.testing.assert_allclose(ratios, (1e-4) ** (1 / 100), rtol=1e-12)


def test_amplitude_heuristic():
    """Eq. (amplitude-acceptance-adjustment) with p = 1, m = 2: y = acceptance^2."""
    assert O.amplitude(64, 64) == 1.0
    assert O.amplitude(32, 64) == 0.25
    assert O.amplitude(16, 64, y_p=0.5, y_m=3.0) == 0.125
    assert O.amplitude(0, 64) == 1e-4
    assert abs(O.amplitude(10, 64, y_p=0.5, y_m=2.5) - (10 / 64 / 0.5) ** 2.5) < 1e-15
    assert O.amplitude(40, 64, y_p=0.5) == 1.0


def test_moves_follow_the_random_stream():
    """Same seed, same run; another seed, another run; walkers are independent of
    how many walkers share the run."""
    P = tiny_double_lorentz()
    s = O.Schedule(n_sweeps=20, sweeps_per_block=1000, resync_every=10, seed=9)
    a1 = O.Anneal(P.tau, P.F, P.sigma, P.omega, P.A, P.B, 6, s); a1.run()
    a2 = O.Anneal(P.tau, P.F, P.sigma, P.omega, P.A, P.B, 6, s); a2.run()
    a3 = O.Anneal(P.tau, P.F, P.sigma, P.omega, P.A, P.B, 3, s); a3.run()
    assert np.array_equal(a1.a, a2.a) and np.array_equal(a1.hash, a2.hash)
    assert np.array_equal(a1.a[:3], a3.a) and np.array_equal(a1.hash[:3], a3.hash)
    s.seed = 10
    a4 = O.Anneal(P.tau, P.F, P.sigma, P.omega, P.A, P.B, 6, s); a4.run()
    assert not np.array_equal(a1.hash, a4.hash)
