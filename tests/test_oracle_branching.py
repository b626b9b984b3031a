"""Pins for imprinted branching (Sec. 2.5) and the stochastic average (Sec. 1)."""

import numpy as np
import pytest

import oracle as O
from workloads import tiny_double_lorentz


def _brute_multipliers(z, xi, Delta):
    """The N smallest break points Delta z_l + ln(k - xi_l), k = 1..N, listed exhaustively."""
    n = len(z)
    pts = sorted((Delta * z[l] + np.log(k - xi[l]), l, k) for l in range(n) for k in range(1, n + 1))
    m = np.zeros(n, dtype=int)
    for _, l, _ in pts[:n]:
        m[l] += 1
    return m


@pytest.mark.parametrize("seed", range(6))
def test_multipliers_match_enumeration(seed):
    rng = np.random.default_rng(seed)
    n = 8
    z = rng.exponential(1.0, n)
    xi = rng.uniform(0, 1, n)
    for Delta in [0.0, 0.3, 1.0, 2.5, 7.0, 40.0]:
        m, Z = O.multipliers_at(z, xi, Delta)
        assert m.sum() == n
        np.testing.assert_array_equal(m, _brute_multipliers(z, xi, Delta))
        assert Z == int(np.sum(m == 0))


@pytest.mark.parametrize("seed", range(4))
def test_multipliers_have_the_papers_form(seed):
    """m_l = floor(w_l + xi_l) with w_l = exp[-Delta (z_l - P_r)] for one P_r."""
    rng = np.random.default_rng(10 + seed)
    n = 200
    z = rng.exponential(1.0, n)
    xi = rng.uniform(0, 1, n)
    Delta = 1.7
    m, _ = O.multipliers_at(z, xi, Delta)
    pts = np.sort(np.concatenate([Delta * z + np.log(k - xi) for k in range(1, n + 1)]))
    theta = 0.5 * (pts[n - 1] + pts[n])       # Delta * P_r, between the n-th and n+1-th point
    w = np.exp(theta - Delta * z)
    np.testing.assert_array_equal(np.floor(w + xi).astype(int), m)


def test_solve_hits_the_branching_fraction():
    rng = np.random.default_rng(4)
    for n, f in [(64, 0.25), (1000, 0.25), (257, 0.1), (4096, 0.25)]:
        chi2 = 100.0 * (1 + rng.exponential(1.0, n))
        xi = rng.uniform(0, 1, n)
        m, Delta = O.branch_multipliers(chi2, xi, f)
        assert m.sum() == n and np.all(m >= 0)
        assert int(np.sum(m == 0)) == int(np.floor(f * n + 0.5))
        assert Delta > 0
        # zero-multiplier walkers are on average the worse ones
        assert chi2[m == 0].mean() > chi2[m >= 2].mean()


def test_solve_degenerate_cases():
    n = 16
    xi = np.linspace(0.01, 0.99, n)
    m, Delta = O.branch_multipliers(np.full(n, 5.0), xi, 0.25)   # all equal: nothing to select
    assert m.sum() == n
    m, Delta = O.branch_multipliers(np.arange(1.0, n + 1), xi, 0.0)  # no branching requested
    assert np.all(m == 1) and Delta == 0.0


def test_pairing_lists_every_surplus_copy():
    m = np.array([0, 3, 1, 0, 0, 2, 1, 1], dtype=np.int32)
    zl, dl = O.pairs(m)
    assert list(zl) == [0, 3, 4]
    assert list(dl) == [1, 1, 5]


def test_branching_run_keeps_sums_and_residuals():
    """Imprinting mixes a and R linearly: after every block the sums still hold
    and the mixed residual equals a recomputation from the mixed spectrum."""
    P = tiny_double_lorentz()
    s = O.Schedule(n_sweeps=60, sweeps_per_block=20, resync_every=20, branching=True,
                   T_start=1.0, T_end=1e-3, seed=3)
    an = O.Anneal(P.tau, P.F, P.sigma, P.omega, P.A, P.B, 32, s)
    acc, mtr, dtr = an.run(trace=True)
    assert mtr.shape == (3, 32)
    assert np.all(mtr.sum(1) == 32) and np.all((mtr == 0).sum(1) == 8)
    np.testing.assert_allclose(an.a.sum(1), P.A, rtol=1e-12)
    np.testing.assert_allclose(an.a @ P.omega, P.B, rtol=1e-12)
    for w in range(32):
        R, chi2 = O.residual(an.K, an.Fh, an.a[w])
        np.testing.assert_allclose(an.R[w], R, rtol=1e-8, atol=1e-8 * np.abs(R).max())
        assert abs(an.chi2[w] - chi2) <= 1e-8 * chi2


def test_branching_draws_follow_the_stream():
    """The multipliers of block 0 are the solve applied to the block's chi2 and to
    xi_l from Philox counter (l, 0, 0, 1)."""
    P = tiny_double_lorentz()
    s = O.Schedule(n_sweeps=20, sweeps_per_block=10, resync_every=10, branching=True, seed=21)
    an = O.Anneal(P.tau, P.F, P.sigma, P.omega, P.A, P.B, 16, s)
    _, mtr, dtr = an.run(10, trace=True)
    s_off = O.Schedule(n_sweeps=20, sweeps_per_block=10, resync_every=10, branching=False, seed=21)
    ref = O.Anneal(P.tau, P.F, P.sigma, P.omega, P.A, P.B, 16, s_off)
    ref.run(10)
    m, Delta = O.branch_multipliers(ref.chi2, O.xi_for_block(21, 0, 16), 0.25)
    np.testing.assert_array_equal(mtr[0], m)
    assert dtr[0] == Delta
    # untouched walkers are identical, imprinted ones moved towards their donor
    zl, dl = O.pairs(m)
    keep = np.setdiff1d(np.arange(16), zl)
    np.testing.assert_array_equal(an.a[keep], ref.a[keep])
    np.testing.assert_allclose(an.a[zl], 0.1 * ref.a[dl] + 0.9 * ref.a[zl], rtol=1e-14)


def test_average_over_good_walkers():
    rng = np.random.default_rng(2)
    a = rng.uniform(0, 1, (10, 7))
    chi2 = np.array([1.0, 1.4, 1.6, 3.0, 1.2, 9.0, 1.5, 1.51, 2.0, 1.0])
    mean, err, used = O.average(a, chi2, 1.5)
    sel = chi2 <= 1.5
    assert used == sel.sum() == 5
    np.testing.assert_allclose(mean, a[sel].mean(0), rtol=1e-14)
    np.testing.assert_allclose(err, a[sel].std(0, ddof=1) / np.sqrt(5), rtol=1e-12)
    mean, err, used = O.average(a[:1], chi2[:1], 1.5)
    assert used == 1 and np.all(err == 0)
