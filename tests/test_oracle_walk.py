"""CPU pins of the oracle's index walk (Sec. 2.3, selection of update frequencies).

The walk of L steps from a uniform start, proposing j' uniform and moving when
u a_j <= a_j', is a Markov chain with transition T_jk = min(1, a_k / a_j) / N (k != j).  Its
law after L steps is the uniform start times T^L, computed here by a matrix power (the
closed form), and compared with the oracle's empirical distribution of p and s.
"""
import numpy as np
import pytest

import oracle as O
from workloads import tiny_double_lorentz


def _transition(a, allowed):
    """Walk transition on the bins in `allowed` (proposals uniform over them)."""
    idx = np.flatnonzero(allowed)
    n = idx.size
    T = np.zeros((a.size, a.size))
    for j in idx:
        for k in idx:
            if k == j:
                continue
            T[j, k] = 1.0 / n if a[j] == 0 else min(1.0, a[k] / a[j]) / n
        T[j, j] = 1.0 - T[j].sum()
    return T


def _laws(a, L, rho):
    """Exact law of p, and of s (mixed over p), after L steps with admixture rho."""
    N = a.size
    uni = np.full(N, 1.0 / N)
    Tp = _transition(a, np.ones(N, bool))
    law_p = rho * uni + (1 - rho) * uni @ np.linalg.matrix_power(Tp, L)
    law_s = np.zeros(N)
    for p in range(N):
        allowed = np.ones(N, bool)
        allowed[p] = False
        start = allowed / allowed.sum()
        Ts = _transition(a, allowed)
        cond = rho * start + (1 - rho) * start @ np.linalg.matrix_power(Ts, L)
        law_s += law_p[p] * cond
    return law_p, law_s


def _sample(a, L, rho, n, seed):
    rng = np.random.default_rng(seed)
    w = rng.integers(0, 2 ** 32, (n, 2), dtype=np.uint64)
    ctr = rng.integers(0, 1 << 20, (n, 3))
    ps = np.array([O.move_bins(a, int(w[i, 0]), int(w[i, 1]), int(ctr[i, 0]), int(ctr[i, 1]), int(ctr[i, 2]),
                               walk_len=L, walk_uniform=rho, seed=77) for i in range(n)])
    return ps[:, 0], ps[:, 1]


def _chi2_ok(counts, law, n):
    exp = law * n
    keep = exp > 0
    assert np.all(counts[~keep] == 0)
    stat = np.sum((counts[keep] - exp[keep]) ** 2 / exp[keep])
    dof = keep.sum() - 1
    # a 5-sigma bound on the chi-square statistic
    assert stat < dof + 5 * np.sqrt(2 * dof), (stat, dof)


@pytest.mark.parametrize("L,rho", [(0, 0.0), (1, 0.0), (3, 0.0), (3, 0.3)])
def test_walk_law_matches_the_matrix_power(L, rho):
    a = np.array([0.0, 0.5, 3.0, 1.0, 0.0, 2.0, 0.1, 4.0, 0.0, 1.5])
    n = 40000
    p, s = _sample(a, L, rho, n, seed=L * 10 + int(rho * 10))
    assert np.all(p != s)
    law_p, law_s = _laws(a, L, rho)
    _chi2_ok(np.bincount(p, minlength=a.size), law_p, n)
    _chi2_ok(np.bincount(s, minlength=a.size), law_s, n)


def test_long_walk_approaches_a_over_A():
    """After many steps p is distributed as a_j / A (the walk's stationary law)."""
    a = np.array([1.0, 0.2, 0.0, 3.0, 0.8, 2.0])
    law_p, _ = _laws(a, 40, 0.0)
    np.testing.assert_allclose(law_p, a / a.sum(), atol=1e-6)


def test_zero_length_walk_is_the_uniform_rule():
    """L = 0: p = floor(w0 N / 2^32), s = floor(w1 (N-1) / 2^32) shifted past p; the spectrum
    is not read."""
    rng = np.random.default_rng(3)
    N = 37
    a = rng.random(N)
    for _ in range(200):
        w0, w1 = (int(v) for v in rng.integers(0, 2 ** 32, 2, dtype=np.uint64))
        p, s = O.move_bins(a, w0, w1, 1, 2, 3)
        assert p == (w0 * N) >> 32
        s_ = (w1 * (N - 1)) >> 32
        assert s == s_ + (s_ >= p)
        assert (p, s) == O.move_bins(np.zeros(N), w0, w1, 1, 2, 3)


def test_walk_anneal_keeps_invariants():
    P = tiny_double_lorentz()
    s = O.Schedule(n_sweeps=30, sweeps_per_block=10, resync_every=10, branching=True, walk_len=3,
                   walk_uniform=0.1, seed=5)
    an = O.Anneal(P.tau, P.F, P.sigma, P.omega, P.A, P.B, 16, s)
    an.run()
    assert np.all(an.a >= 0)
    np.testing.assert_allclose(an.a.sum(1), P.A, rtol=1e-12)
    np.testing.assert_allclose(an.a @ P.omega, P.B, rtol=1e-12)
    for w in range(16):
        R, c2 = O.residual(an.K, an.Fh, an.a[w])
        assert abs(an.chi2[w] - c2) <= 1e-8 * c2
