"""GPU: the index walk choosing the bins of a move (Sec. 2.3) through the C ABI.

The FP64 validation path takes every decision the oracle takes with the walk on (accepted
counts per sweep, the FNV hash of every move's outcome, branching multipliers, final
spectra, residuals and chi2, bit for bit).  The FP32 path keeps the sum rules and its chi2
bookkeeping, and a batch gives the same result as each problem alone.
"""
import numpy as np
import pytest

import oracle as O
import paper_1609_07936_gb300 as sail
from workloads import paper_scale_double_lorentz, tiny_double_lorentz

pytestmark = pytest.mark.gpu


def _pair(P, n_walkers, precision, **kw):
    sched = O.Schedule(**kw)
    params = sail.Params(n_walkers=n_walkers, precision=precision, n_sweeps=sched.n_sweeps,
                         sweeps_per_block=sched.sweeps_per_block, resync_every=sched.resync_every,
                         branching=sched.branching, T_start=sched.T_start, T_end=sched.T_end,
                         A=P.A, B=P.B, seed=sched.seed, trace=True, index_walk_len=sched.walk_len,
                         walk_uniform=sched.walk_uniform)
    an = O.Anneal(P.tau, P.F, P.sigma, P.omega, P.A, P.B, n_walkers, sched)
    g = sail.Sail(P.tau, P.F, P.sigma, P.omega, params)
    return an, g


@pytest.mark.parametrize("L,rho,n_sweeps", [(3, 0.2, 300), (7, 0.0, 250), (1, 1.0, 100)])
def test_fp64_walk_reproduces_every_decision(L, rho, n_sweeps):
    """Tiny double-Lorentzian workload, 48 walkers, branching every 50 sweeps, T 1 -> 1e-4.
    rho = 1 skips every walk: the bins are then the uniform ones."""
    P = tiny_double_lorentz()
    an, g = _pair(P, 48, sail.PREC_FP64, n_sweeps=n_sweeps, sweeps_per_block=50, resync_every=25,
                  branching=True, T_start=1.0, T_end=1e-4, walk_len=L, walk_uniform=rho, seed=11)
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


def test_fp32_walk_keeps_sums_and_bookkeeping():
    P = paper_scale_double_lorentz(1e-4, n_walkers=512)
    prm = sail.Params(n_walkers=512, precision=sail.PREC_FP32, n_sweeps=200, sweeps_per_block=50,
                      resync_every=25, branching=True, A=P.A, B=P.B, seed=12, index_walk_len=2,
                      walk_uniform=0.1, resync_kind=sail.RESYNC_TENSOR)
    g = sail.Sail(P.tau, P.F, P.sigma, P.omega, prm)
    stats = g.anneal()
    assert len(stats) == 4 and 0 < stats[-1]["acceptance"] < 1
    a, R, chi2, _, _ = g.state()
    assert np.all(a >= 0)
    np.testing.assert_allclose(a.sum(1), P.A, rtol=2e-6)
    np.testing.assert_allclose(a @ P.omega, P.B, rtol=2e-6)
    K, Fh, _ = O.tables(P.tau, P.F, P.sigma, P.omega)
    for w in range(0, 512, 37):
        model = K @ a[w]
        R_ref = Fh - model
        tol = 2e-6 * model + 6e-8 * np.abs(R_ref) + 1e-6
        c2 = np.sum(R_ref ** 2)
        assert abs(chi2[w] - c2) <= 2 * np.sum(np.abs(R_ref) * tol) + 1e-9 * c2
    g.close()


def test_batch_with_walk_equals_problems_alone():
    P1 = tiny_double_lorentz()
    P2 = paper_scale_double_lorentz(1e-4, n_walkers=64)
    items, alone = [], []
    for k, (P, W, L) in enumerate([(P1, 40, 2), (P2, 64, 0), (P2, 70, 3)]):
        prm = sail.Params(n_walkers=W, precision=sail.PREC_FP32, n_sweeps=60, sweeps_per_block=20,
                          resync_every=10, branching=True, A=P.A, B=P.B, seed=60 + k, index_walk_len=L,
                          walk_uniform=0.05, resync_kind=sail.RESYNC_TENSOR)
        items.append((P.tau, P.F, P.sigma, P.omega, prm))
        h = sail.Sail(P.tau, P.F, P.sigma, P.omega, prm)
        h.anneal()
        alone.append(h)
    batch = sail.Batch(items, autotune=False)
    batch.anneal()
    for k, h in enumerate(alone):
        a1, R1, c1, _, h1 = h.state()
        a2, R2, c2, _, h2 = batch.handles[k].state()
        np.testing.assert_array_equal(a2, a1)
        np.testing.assert_array_equal(R2, R1)
        np.testing.assert_array_equal(c2, c1)
        h.close()
    batch.close()
