"""CPU pins of the oracle's shared-bin moves: the walkers of each group of W propose, at every
move, the bins drawn by the group's first walker, and keep their own amplitude and acceptance
draw.

Pins: W = 1 is the paper's move; with branching off the group's first walkers follow exactly
the trajectories they have with their own bins, while the others differ both from their own-bin
trajectory and from the first walker's (their amplitudes are their own); and at T = infinity
with the Hastings acceptance every walker still samples the uniform law on the polytope (a
walker's bins stay uniform and independent of its spectrum, so its chain is unchanged).
"""
import numpy as np
import pytest

import oracle as O
from tests.test_oracle_hastings import A6, B6, N6, X6, _uniform_polytope_samples

NT, NO, NW = 8, 24, 16


def _problem():
    tau = np.linspace(0.0, 4.0, NT)
    x = (np.arange(NO) + 0.5) * (6.0 / NO)
    a = np.exp(-((x - 2.0) ** 2))
    a /= a.sum()
    F = np.array([(a * np.exp(-t * x)).sum() for t in tau])
    return tau, F, 1e-3 * F, x, a.sum(), float(a @ x)


def _run(W, n_sweeps=20, seed=5, hastings=False):
    tau, F, sig, x, A, B = _problem()
    s = O.Schedule(n_sweeps=n_sweeps, sweeps_per_block=10, resync_every=5, T_start=1.0, T_end=1e-3,
                   seed=seed, hastings=hastings, shared_bins=W)
    an = O.Anneal(tau, F, sig, x, A, B, NW, s)
    an.run()
    return an


def _same(an, bn, w):
    return (np.array_equal(an.a[w], bn.a[w]) and np.array_equal(an.R[w], bn.R[w])
            and an.chi2[w] == bn.chi2[w] and an.hash[w] == bn.hash[w])


def test_one_walker_groups_are_the_paper_move():
    an, bn = _run(0), _run(1)
    assert all(_same(an, bn, w) for w in range(NW))


@pytest.mark.parametrize("W", [4, 8])
def test_first_walkers_follow_their_own_bins(W):
    own, sh = _run(0), _run(W)
    for w in range(NW):
        if w % W == 0:
            assert _same(own, sh, w), w
        else:
            assert not _same(own, sh, w), w
            # same start spectrum and the same bins as the group's first walker, but its own
            # amplitudes and acceptance draws
            assert not np.array_equal(sh.a[w], sh.a[w - w % W]), w


@pytest.mark.parametrize("hastings", [False, True])
def test_shared_bins_keep_the_sum_rules(hastings):
    tau, F, sig, x, A, B = _problem()
    an = _run(4, hastings=hastings)
    np.testing.assert_allclose(an.a.sum(1), A, rtol=1e-12)
    np.testing.assert_allclose(an.a @ x, B, rtol=1e-12)
    assert np.all(an.a >= 0)


def test_shared_bins_chain_samples_the_uniform_polytope():
    """Hastings acceptance at T = infinity, groups of 4: each walker's law is uniform on the
    polytope {a >= 0, sum a = A, sum a x = B}.  The group's first walkers and the others are
    tested apart (samples within a test are independent walkers)."""
    from scipy import stats
    S = _uniform_polytope_samples()
    tau = np.linspace(0.0, 2.0, 3)
    s = O.Schedule(n_sweeps=3000, sweeps_per_block=10 ** 6, resync_every=50, T_start=1e300, T_end=1e300,
                   hastings=True, y_p=1e-9, seed=6, shared_bins=4)
    an = O.Anneal(tau, np.ones(3), np.ones(3), X6, A6, B6, 4096, s)
    an.run()
    for part in (an.a[0::4], an.a[1::4]):
        for j in range(N6):
            assert stats.ks_2samp(part[:, j], S[:, j]).pvalue > 1e-3, j
