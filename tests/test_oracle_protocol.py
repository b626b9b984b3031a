"""CPU pins of the oracle's anti-sawtooth protocol: self-cooling schedule (Sec. self-cooling),
acceptance-adaptive branching (Sec. 2.5, last paragraph) and smoothing with renormalisation
(Sec. smoothing).  Values below are worked by hand or follow from the sum rules."""
import numpy as np
import pytest

import oracle as O
from workloads import tiny_double_lorentz


# ---------------------------------------------------------------- smoothing

def test_smoothing_worked_example():
    """s = 0.1 on the symmetric spectrum 1,2,3,4,3,2,1 (worked by hand):
    ends (1-s) a_0 + s a_1 = 1.1; interior s a_{j-1} + (1-2s) a_j + s a_{j+1} = 2, 3, 3.8.
    The spectrum is symmetric, so the second sum rule is unchanged and the tilt is ~0."""
    x = (np.arange(7) + 0.5) * 0.25
    a = np.array([1.0, 2.0, 3.0, 4.0, 3.0, 2.0, 1.0])
    B = float(a @ x)
    out = O.smooth(x, B, 0.1, a)
    np.testing.assert_allclose(out, [1.1, 2.0, 3.0, 3.8, 3.0, 2.0, 1.1], rtol=1e-13)


def test_smoothing_boundary_delta_keeps_stencil_when_tilt_too_large():
    """All mass in bin 0: the stencil gives (1 - s, s, 0, ...); its first moment moved by
    s dw (a_0 - a_{N-1}) = s dw.  Restoring it would need a tilt factor 1 + beta (x - m) with
    |beta| span = 6 / (1 - s) > 1/2, so the renormalisation is skipped."""
    dw, s = 0.5, 0.05
    x = (np.arange(7) + 0.5) * dw
    a = np.zeros(7)
    a[0] = 1.0
    out = O.smooth(x, float(x[0]), s, a)
    np.testing.assert_array_equal(out, [1.0 - s, s, 0, 0, 0, 0, 0])
    assert out @ x - x[0] == pytest.approx(s * dw, rel=1e-12)


def test_smoothing_keeps_both_sum_rules():
    """A lopsided spectrum (a_0 != a_{N-1}): the stencil keeps sum a, the tilt restores
    sum a x = B; the result stays positive and close to the stencil alone."""
    rng = np.random.default_rng(4)
    n = 200
    dw = 0.05
    x = (np.arange(n) + 0.5) * dw
    a = np.exp(-((x - 3.0) / 1.5) ** 2) + 0.3 * np.exp(-x) + 0.01 * rng.random(n)
    A, B = a.sum(), float(a @ x)
    for s in (1e-3, 1e-2, 0.05):
        out = O.smooth(x, B, s, a)
        assert np.all(out >= 0)
        assert out.sum() == pytest.approx(A, rel=1e-13)
        assert out @ x == pytest.approx(B, rel=1e-13)
        # smoothing lowers the largest second difference (a sawtooth is damped)
        assert np.abs(np.diff(out, 2)).max() < np.abs(np.diff(a, 2)).max()


def test_smoothing_damps_a_sawtooth_by_one_minus_4s():
    """The stencil maps the alternating mode (-1)^j to (1 - 4s)(-1)^j in the interior: the
    sawtooth the paper counters (Sec. smoothing) decays geometrically."""
    n, s = 64, 0.02
    x = (np.arange(n) + 0.5) * 0.1
    base = 5.0 + 0.0 * x
    saw = 0.5 * (-1.0) ** np.arange(n)
    a = base + saw
    out = O.smooth(x, float(a @ x), s, a)
    interior = slice(2, n - 2)
    ratio = (out[interior] - out[interior].mean()) / saw[interior]
    np.testing.assert_allclose(ratio, 1.0 - 4.0 * s, rtol=1e-3)


# ---------------------------------------------------------------- self-cooling

def test_cooling_block_split():
    assert O.cooling_blocks(200, 0.1, 0.5) == (20, 100)
    assert O.cooling_blocks(10, 0.5, 0.2) == (5, 5)      # freeze-out never before cooling
    assert O.cooling_blocks(10, -1.0, 2.0) == (0, 10)     # clamped to the schedule


def test_self_cooling_phases():
    nb, bc, bf = 20, 4, 10
    cbar, cmin, Tf = 900.0, 100.0, 1e-3
    # boiling: the population's mean residue
    for b in range(1, bc):
        assert O.self_cooling(b, nb, bc, bf, cbar, cmin, Tf)[0] == cbar
    # cooling: geometric from the mean towards the minimum; x = 1/2 at b = bc + 2
    assert O.self_cooling(bc + 2, nb, bc, bf, cbar, cmin, Tf)[0] == pytest.approx(np.sqrt(cbar * cmin), rel=1e-14)
    assert O.self_cooling(bf - 1, nb, bc, bf, cbar, cmin, Tf)[0] == cmin
    Ts = [O.self_cooling(b, nb, bc, bf, cbar, cmin, Tf)[0] for b in range(bc, bf)]
    assert all(t1 > t2 for t1, t2 in zip(Ts, Ts[1:]))
    # freeze-out: from the minimum down by a constant factor per block to T_final at the end
    T, tf = O.self_cooling(bf, nb, bc, bf, cbar, cmin, Tf)
    ratio = (Tf / cmin) ** (1.0 / (nb - bf))
    assert tf == cmin and T == pytest.approx(cmin * ratio, rel=1e-13)
    Tz = [O.self_cooling(b, nb, bc, bf, cbar, 5.0, Tf, tf)[0] for b in range(bf, nb)]  # later minima do not move T_F
    np.testing.assert_allclose(np.array(Tz[1:]) / np.array(Tz[:-1]), ratio, rtol=1e-12)
    assert Tz[-1] == pytest.approx(Tf, rel=1e-13)
    # a population already colder than the end temperature is held where it is
    assert O.self_cooling(bf, nb, bc, bf, cbar, 1e-4, Tf)[0] == 1e-4
    assert O.self_cooling(bf, nb, bc, bf, cbar, 0.0, Tf)[0] == 0.0


def test_self_cooling_anneal_follows_population_statistics():
    """Without branching or smoothing the residues after a block are those the next block's
    temperature is taken from: T of block b+1 is the schedule function of block b's mean and
    minimum, and block 0 runs at chi2_0."""
    P = tiny_double_lorentz()
    k, nblocks = 10, 8
    s = O.Schedule(n_sweeps=k * nblocks, sweeps_per_block=k, resync_every=k, branching=False,
                   schedule_kind=1, cool_begin=0.25, freeze_begin=0.75, seed=12)
    an = O.Anneal(P.tau, P.F, P.sigma, P.omega, P.A, P.B, 12, s)
    assert np.all(an.T[:k] == an.chi2_0) and np.all(np.isnan(an.T[k:]))
    bc, bf = O.cooling_blocks(nblocks, 0.25, 0.75)
    tf = -1.0
    for b in range(nblocks - 1):
        an.run(k)
        cbar = 0.0
        for c in an.chi2:
            cbar += float(c)
        cbar /= len(an.chi2)
        T, tf = O.self_cooling(b + 1, nblocks, bc, bf, cbar, float(an.chi2.min()), an.chi2_0 * s.T_end, tf)
        assert np.all(an.T[(b + 1) * k:(b + 2) * k] == T)
    an.run()
    assert an.T[-1] < an.T[bf * k - 1]


# ---------------------------------------------------------------- adaptive branching

def test_adaptive_scale():
    assert O.adaptive_scale(0.3, 0.6) == 0.5
    assert O.adaptive_scale(0.7, 0.6) == 1.0
    assert O.adaptive_scale(0.3, 0.0) == 1.0
    assert O.adaptive_scale(0.0, 0.5) == 0.0


def test_adaptive_branching_scales_fraction_and_imprint():
    """Moves of negligible size (d = 1e-300) leave every spectrum as it is, so the state
    before a block's branching is the state after the previous block.  Block 0 runs hot
    (acceptance ~1), block 1 at T ~ 0 (about half the moves raise chi2 by a rounding-sized
    amount): its branching fraction and imprint strength are scaled by acc_1 / acc_0."""
    P = tiny_double_lorentz()
    W, k = 32, 5
    s = O.Schedule(n_sweeps=2 * k, sweeps_per_block=k, resync_every=k, branching=True, adaptive=True,
                   T_start=1e250, T_end=1e-250, move_scale=1e-300, branch_fraction=0.5, imprint_t=0.4,
                   seed=31)
    an = O.Anneal(P.tau, P.F, P.sigma, P.omega, P.A, P.B, W, s)
    rng = np.random.default_rng(8)
    a0 = an.a[0].copy()
    for w in range(W):
        an.a[w] = a0 * rng.uniform(0.5, 1.5, a0.size)
        R, c2 = O.residual(an.K, an.Fh, an.a[w])
        an.R[w] = R
        an.chi2[w] = c2
    proposed = k * W * P.n_omega
    _, m0, _ = an.run(k, trace=True)
    acc0 = an.n_acc.sum() / proposed
    assert (m0[0] == 0).sum() == 16                       # scale 1 in block 0
    before = an.a.copy()
    _, m1, _ = an.run(k, trace=True)
    acc1 = (an.n_acc.sum() - acc0 * proposed) / proposed
    scale = min(1.0, acc1 / acc0)
    assert 0.2 < scale < 0.9
    Z = (m1[0] == 0).sum()
    assert abs(Z - 0.5 * scale * W) <= 1.0
    zl, dl = O.pairs(m1[0])
    t = 0.4 * scale
    np.testing.assert_allclose(an.a[zl], t * before[dl] + (1.0 - t) * before[zl], rtol=1e-13)


# ---------------------------------------------------------------- smoothing in the anneal

def test_smoothing_in_the_anneal_keeps_sum_rules_and_residuals():
    P = tiny_double_lorentz()
    s = O.Schedule(n_sweeps=40, sweeps_per_block=10, resync_every=10, branching=True, adaptive=True,
                   schedule_kind=1, smooth_s=0.02, seed=7)
    an = O.Anneal(P.tau, P.F, P.sigma, P.omega, P.A, P.B, 16, s)
    an.run()
    assert np.all(an.a >= 0)
    np.testing.assert_allclose(an.a.sum(1), P.A, rtol=1e-12)
    np.testing.assert_allclose(an.a @ P.omega, P.B, rtol=1e-12)
    for w in range(16):
        R, c2 = O.residual(an.K, an.Fh, an.a[w])
        assert abs(an.chi2[w] - c2) <= 1e-9 * c2
