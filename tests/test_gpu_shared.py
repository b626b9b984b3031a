"""GPU: shared-bin moves (the walkers of each group of W propose their first walker's bins)
through the C ABI.

The FP64 validation path takes every decision the oracle takes with shared bins, bit for bit.
The FP32 sweeps draw the same words as the oracle, so a walker's FP32 run takes the oracle's
decisions until rounding first flips one near a threshold: over a few sweeps nearly every
walker's accepted counts equal the oracle's (the own-bin FP32 kernel is checked the same way,
as a control).  At T = infinity with the Hastings acceptance the FP32 walkers sample the
uniform law on the polytope, and on the paper-scale grid the sum rules and the chi2 bookkeeping
hold.  Invalid combinations are refused.
"""
import numpy as np
import pytest

import oracle as O
import paper_1609_07936_gb300 as sail
from tests.test_oracle_hastings import A6, B6, N6, X6, _uniform_polytope_samples
from workloads import paper_scale_double_lorentz, tiny_double_lorentz

pytestmark = pytest.mark.gpu


def _pair(P, n_walkers, precision, W, hastings=False, loop=0, **kw):
    sched = O.Schedule(shared_bins=W, hastings=hastings, **kw)
    params = sail.Params(n_walkers=n_walkers, precision=precision, n_sweeps=sched.n_sweeps,
                         sweeps_per_block=sched.sweeps_per_block, resync_every=sched.resync_every,
                         branching=sched.branching, T_start=sched.T_start, T_end=sched.T_end,
                         A=P.A, B=P.B, seed=sched.seed, trace=True, shared_bins=W, hastings=hastings,
                         resync_kind=sail.RESYNC_FP32, sweep_loop=loop)
    an = O.Anneal(P.tau, P.F, P.sigma, P.omega, P.A, P.B, n_walkers, sched)
    g = sail.Sail(P.tau, P.F, P.sigma, P.omega, params)
    return an, g


@pytest.mark.parametrize("W,hastings,n_walkers", [(2, False, 37), (4, False, 48), (8, False, 61), (8, True, 40)])
def test_fp64_shared_bins_reproduce_every_decision(W, hastings, n_walkers):
    """Tiny workload, branching every 50 sweeps; 61 walkers leave the last group ragged."""
    P = tiny_double_lorentz()
    an, g = _pair(P, n_walkers, sail.PREC_FP64, W, hastings, n_sweeps=200, sweeps_per_block=50,
                  resync_every=25, branching=True, T_start=1.0, T_end=1e-4, seed=31)
    acc_o, m_o, d_o = an.run(trace=True)
    g.anneal()
    acc_g, m_g, d_g = g.trace()
    np.testing.assert_array_equal(acc_g, acc_o)
    np.testing.assert_array_equal(m_g, m_o)
    np.testing.assert_array_equal(d_g, d_o)
    a, R, chi2, _, h = g.state()
    np.testing.assert_array_equal(h, an.hash)
    np.testing.assert_array_equal(a, an.a)
    np.testing.assert_array_equal(R, an.R)
    np.testing.assert_array_equal(chi2, an.chi2)
    g.close()


_DECISION_CASES = [(0, False, 64), (2, False, 64), (4, False, 64), (8, False, 61), (8, True, 64), (4, True, 37),
                   (2, True, 33)]


# the move-loop choice (1 one move at a time, 2 look-ahead) applies to own bins only
@pytest.mark.parametrize("W,hastings,n_walkers,loop",
                         [c + (2,) for c in _DECISION_CASES] + [c + (1,) for c in _DECISION_CASES if c[0] == 0])
def test_fp32_sweep_takes_the_oracle_decisions(W, hastings, n_walkers, loop):
    """Tiny workload (32 tau points, 64 bins), 4 sweeps of 64 moves at T = chi2_0 / 2 with a
    recomputation every 2 sweeps, no branching: at least 90% of the walkers accept exactly
    the oracle's number of moves in every sweep, and those walkers end within 1e-4 of the
    oracle's spectra."""
    P = tiny_double_lorentz()
    an, g = _pair(P, n_walkers, sail.PREC_FP32, W, hastings, loop=loop, n_sweeps=4, sweeps_per_block=4,
                  resync_every=2, branching=False, T_start=0.5, T_end=0.5, seed=17)
    acc_o, _, _ = an.run(trace=True)
    g.anneal()
    acc_g, _, _ = g.trace()
    same = np.all(acc_g == acc_o, axis=0)
    assert same.mean() >= 0.9, same.mean()
    assert acc_o.sum() > 0 and (acc_o < P.n_omega).any()
    a = g.state()[0]
    for w in np.flatnonzero(same):
        np.testing.assert_allclose(a[w], an.a[w], rtol=0, atol=1e-4 * an.a[w].max())
    g.close()


def test_fp32_shared_hastings_samples_the_uniform_polytope():
    from scipy import stats
    S = _uniform_polytope_samples()
    tau = np.linspace(0.0, 2.0, 3)
    prm = sail.Params(n_walkers=4096, precision=sail.PREC_FP32, n_sweeps=3000, sweeps_per_block=10 ** 6,
                      resync_every=50, branching=False, T_start=1e20, T_end=1e20, A=A6, B=B6, y_p=1e-9,
                      seed=9, hastings=True, shared_bins=8, resync_kind=sail.RESYNC_FP32)
    g = sail.Sail(tau, np.ones(3), np.ones(3), X6, prm)
    g.anneal()
    a = g.state()[0]
    np.testing.assert_allclose(a.sum(1), A6, rtol=1e-5)
    np.testing.assert_allclose(a @ X6, B6, rtol=1e-5)
    # walkers of one group are correlated: test one walker per group, two positions
    for part in (a[0::8], a[5::8]):
        for j in range(N6):
            assert stats.ks_2samp(part[:, j], S[:, j]).pvalue > 1e-3, j
    g.close()


@pytest.mark.parametrize("W", [2, 4, 8])
def test_fp32_shared_paper_scale_keeps_sums_and_bookkeeping(W):
    """200 x 1000 grid, 4096 walkers, two blocks of 100 sweeps with branching and BF16
    tensor-core recomputation every 50."""
    P = paper_scale_double_lorentz(1e-4)
    prm = sail.Params(n_walkers=4096, precision=sail.PREC_FP32, n_sweeps=20000, sweeps_per_block=100,
                      resync_every=50, branching=True, T_start=10.0, T_end=1e-9, A=P.A, B=P.B, seed=2,
                      shared_bins=W, resync_kind=sail.RESYNC_TENSOR_BF16)
    g = sail.Sail(P.tau, P.F, P.sigma, P.omega, prm)
    stats = g.anneal(2)
    assert len(stats) == 2 and all(s["branch_zeros"] == 1024 for s in stats)
    assert 0.05 < stats[-1]["acceptance"] < 0.95
    a, R, chi2, _, _ = g.state()
    assert np.all(a >= 0)
    np.testing.assert_allclose(a.sum(1), P.A, rtol=2e-6)
    np.testing.assert_allclose(a @ P.omega, P.B, rtol=2e-6)
    K, Fh, _ = O.tables(P.tau, P.F, P.sigma, P.omega)
    for w in range(0, 4096, 173):
        model = K @ a[w]
        R_ref = Fh - model
        tol = 2e-6 * model + 6e-8 * np.abs(R_ref) + 1e-6
        c2 = np.sum(R_ref ** 2)
        assert abs(chi2[w] - c2) <= 2 * np.sum(np.abs(R_ref) * tol) + 1e-9 * c2
    g.close()


def test_invalid_shared_bin_combinations_are_refused():
    P = tiny_double_lorentz()
    base = dict(n_walkers=16, A=P.A, B=P.B, n_sweeps=10)
    for kw in (dict(shared_bins=3), dict(shared_bins=16), dict(shared_bins=4, index_walk_len=2)):
        with pytest.raises(sail.SailError):
            sail.Sail(P.tau, P.F, P.sigma, P.omega, sail.Params(**base, **kw))
    big = paper_scale_double_lorentz(1e-4, n_walkers=16, n_tau=300)
    with pytest.raises(sail.SailError):
        sail.Sail(big.tau, big.F, big.sigma, big.omega,
                  sail.Params(n_walkers=16, A=big.A, B=big.B, n_sweeps=10, precision=sail.PREC_FP32, shared_bins=8))
    prm = sail.Params(n_walkers=16, A=P.A, B=P.B, n_sweeps=10, precision=sail.PREC_FP32, shared_bins=8)
    with pytest.raises(sail.SailError):
        sail.Batch([(P.tau, P.F, P.sigma, P.omega, prm)], autotune=False)
