"""GPU: the Hastings-corrected acceptance through the C ABI.

The FP64 validation path takes every decision the oracle takes with the correction on (and
puts the spectra back on the sum rules at the same recomputations), bit for bit.  The FP32
path, at T = infinity with a fixed move scale, samples the uniform law on the polytope
{a >= 0, sum a = A, sum a x = B}: its walkers' marginals match rejection samples of it.
"""
import numpy as np
import pytest

import oracle as O
import paper_1609_07936_gb300 as sail
from tests.test_oracle_hastings import A6, B6, N6, X6, _uniform_polytope_samples
from workloads import paper_scale_double_lorentz, tiny_double_lorentz

pytestmark = pytest.mark.gpu


def test_fp64_hastings_reproduces_every_decision():
    P = tiny_double_lorentz()
    sched = O.Schedule(n_sweeps=300, sweeps_per_block=50, resync_every=25, branching=True, T_start=1.0,
                       T_end=1e-4, hastings=True, seed=21)
    an = O.Anneal(P.tau, P.F, P.sigma, P.omega, P.A, P.B, 48, sched)
    acc_o, m_o, d_o = an.run(trace=True)
    g = sail.Sail(P.tau, P.F, P.sigma, P.omega,
                  sail.Params(n_walkers=48, precision=sail.PREC_FP64, n_sweeps=300, sweeps_per_block=50,
                              resync_every=25, branching=True, T_start=1.0, T_end=1e-4, A=P.A, B=P.B,
                              seed=21, trace=True, hastings=True))
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


def test_fp32_hastings_samples_the_uniform_polytope():
    from scipy import stats
    S = _uniform_polytope_samples()
    tau = np.linspace(0.0, 2.0, 3)
    prm = sail.Params(n_walkers=2048, precision=sail.PREC_FP32, n_sweeps=3000, sweeps_per_block=10 ** 6,
                      resync_every=50, branching=False, T_start=1e20, T_end=1e20, A=A6, B=B6, y_p=1e-9,
                      seed=8, hastings=True, resync_kind=sail.RESYNC_FP32)
    g = sail.Sail(tau, np.ones(3), np.ones(3), X6, prm)
    g.anneal()
    a = g.state()[0]
    np.testing.assert_allclose(a.sum(1), A6, rtol=1e-5)
    np.testing.assert_allclose(a @ X6, B6, rtol=1e-5)
    for j in range(N6):
        assert stats.ks_2samp(a[:, j], S[:, j]).pvalue > 1e-3, j
    g.close()


def test_batch_with_hastings_equals_problems_alone():
    P1 = tiny_double_lorentz()
    P2 = paper_scale_double_lorentz(1e-4, n_walkers=64)
    items, alone = [], []
    for k, (P, W) in enumerate([(P1, 40), (P2, 64)]):
        prm = sail.Params(n_walkers=W, precision=sail.PREC_FP32, n_sweeps=60, sweeps_per_block=20,
                          resync_every=10, branching=True, A=P.A, B=P.B, seed=80 + k, hastings=True,
                          resync_kind=sail.RESYNC_TENSOR)
        items.append((P.tau, P.F, P.sigma, P.omega, prm))
        h = sail.Sail(P.tau, P.F, P.sigma, P.omega, prm)
        h.anneal()
        alone.append(h)
    batch = sail.Batch(items, autotune=False)
    batch.anneal()
    for k, h in enumerate(alone):
        a1, R1, c1, _, _ = h.state()
        a2, R2, c2, _, _ = batch.handles[k].state()
        np.testing.assert_array_equal(a2, a1)
        np.testing.assert_array_equal(c2, c1)
        h.close()
    batch.close()
