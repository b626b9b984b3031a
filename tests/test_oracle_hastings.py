"""CPU pins of the oracle's Hastings-corrected move (exact detailed balance for the move of
Sec. 2.2).

The move (a, eps) -> (r a + delta(eps), -eps / r), r = 1 - eps, is its own inverse; its
Jacobian on the manifold of the two sum rules, with the amplitude as the auxiliary variable,
is r^(N_omega - 4).  Pins: the inverse move restores the spectrum; a finite-difference
determinant of the map equals r^(N-4) and sets the acceptance threshold; and at T = infinity
the corrected chain samples the uniform law on the polytope {a >= 0, sum a = A,
sum a x = B} (checked against rejection sampling), which the uncorrected chain does not.
"""
import functools

import numpy as np
import pytest

import oracle as O

N6 = 6
X6 = np.arange(N6) + 0.5
A6, B6 = 1.0, 2.2


def _manifold(x, A, B):
    C = np.vstack([np.ones(x.size), x])
    _, _, Vt = np.linalg.svd(C)
    V = Vt[2:].T
    ac = np.linalg.lstsq(C, [A, B], rcond=None)[0]
    return V, ac


@functools.lru_cache(maxsize=1)
def _uniform_polytope_samples(n=20000):
    """Uniform points of {a >= 0, sum a = A, sum a x = B} by rejection from a box in manifold
    coordinates (the box holds the polytope: its points are within 0.7 of the centre)."""
    V, ac = _manifold(X6, A6, B6)
    rng = np.random.default_rng(0)
    out = []
    while sum(len(o) for o in out) < n:
        z = rng.uniform(-0.7, 0.7, (2_000_000, N6 - 2))
        a = ac + z @ V.T
        out.append(a[np.all(a >= 0, axis=1)])
    return np.concatenate(out)[:n]


def _move(a, p, s, eps, x, A, B):
    """The oracle's move applied to a (rescale all bins, then a_p', a_s')."""
    K = np.zeros((1, x.size))
    ok, _, ap, as_, _ = O.propose(K, np.zeros(1), x, A, B, a, np.zeros(1), p, s, eps)
    out = (1.0 - eps) * a
    out[p], out[s] = ap, as_
    return ok, out


def test_inverse_move_restores_the_spectrum():
    rng = np.random.default_rng(1)
    x = np.arange(9) + 0.5
    a = rng.uniform(0.5, 1.5, 9)
    A, B = a.sum(), float(a @ x)
    done = 0
    while done < 20:
        p, s = rng.choice(9, 2, replace=False)
        eps = rng.uniform(-0.02, 0.02)
        ok, a1 = _move(a, p, s, eps, x, A, B)
        if not ok:          # a bin would go negative: no move to invert
            continue
        ok, a2 = _move(a1, p, s, -eps / (1.0 - eps), x, A, B)
        assert ok
        np.testing.assert_allclose(a2, a, rtol=1e-12)
        done += 1


@pytest.mark.parametrize("eps", [0.07, -0.05])
def test_jacobian_is_r_to_the_n_minus_4(eps):
    """Finite-difference determinant of (z, eps) -> (z', eps') in manifold coordinates, and the
    oracle's acceptance threshold at Delta chi2 = 0 equal to it."""
    N = 7
    x = np.arange(N) + 0.5
    rng = np.random.default_rng(2)
    a0 = rng.uniform(0.5, 1.5, N)
    A, B = a0.sum(), float(a0 @ x)
    V, ac = _manifold(x, A, B)
    p, s = 1, 4

    def h(v):
        z, e = v[:-1], v[-1]
        _, a1 = _move(ac + V @ z, p, s, e, x, A, B)
        return np.concatenate([V.T @ (a1 - ac), [-e / (1.0 - e)]])

    v0 = np.concatenate([V.T @ (a0 - ac), [eps]])
    J = np.zeros((N - 1, N - 1))
    step = 1e-6
    for k in range(N - 1):
        dv = np.zeros(N - 1)
        dv[k] = step
        J[:, k] = (h(v0 + dv) - h(v0 - dv)) / (2 * step)
    r = 1.0 - eps
    det = abs(np.linalg.det(J))
    assert det == pytest.approx(r ** (N - 4), rel=1e-6)
    yd = 0.2
    thr = min(1.0, det)
    assert O.accept(N, yd, eps, 0.0, 1.0, thr * (1 - 1e-9), hastings=True)
    if thr < 1.0:
        assert not O.accept(N, yd, eps, 0.0, 1.0, thr * (1 + 1e-9), hastings=True)
    # a reverse amplitude |eps / r| beyond y d cannot be proposed: rejected
    assert not O.accept(N, abs(eps / r) * 0.999, eps, -1.0, 1.0, 1e-9, hastings=True)


def _chain(hastings, seed, n_sweeps=3000, W=2048):
    tau = np.linspace(0.0, 2.0, 3)
    # fixed move scale (y = 1): the adaptive amplitude of Eq. (amplitude-acceptance-adjustment)
    # makes the proposal depend on the chain's past
    s = O.Schedule(n_sweeps=n_sweeps, sweeps_per_block=10 ** 6, resync_every=50, T_start=1e300, T_end=1e300,
                   hastings=hastings, y_p=1e-9, seed=seed)
    an = O.Anneal(tau, np.ones(3), np.ones(3), X6, A6, B6, W, s)
    an.run()
    return an.a


def test_hastings_chain_samples_the_uniform_polytope():
    from scipy import stats
    S = _uniform_polytope_samples()
    a = _chain(True, seed=4)
    np.testing.assert_allclose(a.sum(1), A6, rtol=1e-13)
    np.testing.assert_allclose(a @ X6, B6, rtol=1e-13)
    for j in range(N6):
        assert stats.ks_2samp(a[:, j], S[:, j]).pvalue > 1e-3, j


def test_uncorrected_chain_does_not():
    from scipy import stats
    S = _uniform_polytope_samples()
    a = _chain(False, seed=4)
    assert min(stats.ks_2samp(a[:, j], S[:, j]).pvalue for j in range(N6)) < 1e-10
