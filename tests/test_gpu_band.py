"""GPU: the paper's band example (Eq. lorentzian-band with correlated undersampling noise,
Sec. resampling) through the C ABI against the oracle.

On the band problem — 160 tau points with correlated noise, 1000 bins of [0, 3.5], the band
[0.5, 2.5] — the FP64 validation path with the paper's protocol (self-cooling, adaptive
branching, smoothing) takes every decision the oracle takes; the FP32 path keeps the sum
rules, and the chi2 of its averaged spectrum is the oracle's chi2 of that spectrum.
"""
import numpy as np
import pytest

import oracle as O
import paper_1609_07936_gb300 as sail
from workloads import lorentzian_band, skew

pytestmark = pytest.mark.gpu


def test_fp64_band_protocol_reproduces_every_decision():
    P = lorentzian_band(1e-4, seed=2, n_walkers=24)
    sched = O.Schedule(n_sweeps=200, sweeps_per_block=50, resync_every=25, branching=True, T_start=1.0,
                       T_end=1e-6, seed=5, schedule_kind=1, adaptive=True, cool_begin=0.25, freeze_begin=0.5,
                       smooth_s=0.01)
    an = O.Anneal(P.tau, P.F, P.sigma, P.omega, P.A, P.B, 24, sched)
    acc_o, m_o, d_o = an.run(trace=True)
    prm = sail.Params(n_walkers=24, precision=sail.PREC_FP64, n_sweeps=200, sweeps_per_block=50, resync_every=25,
                      branching=True, T_start=1.0, T_end=1e-6, A=P.A, B=P.B, seed=5, trace=True, schedule_kind=1,
                      adaptive_branching=True, cool_begin=0.25, freeze_begin=0.5, smooth_s=0.01)
    g = sail.Sail(P.tau, P.F, P.sigma, P.omega, prm)
    stats = g.anneal()
    acc_g, m_g, d_g = g.trace()
    np.testing.assert_array_equal(acc_g, acc_o)
    np.testing.assert_array_equal(m_g, m_o)
    np.testing.assert_array_equal(d_g, d_o)
    for s in stats:
        assert s["T"] == an.T[s["sweep_end"] - 1]
    a, R, chi2, _, h = g.state()
    np.testing.assert_array_equal(h, an.hash)
    np.testing.assert_array_equal(a, an.a)
    np.testing.assert_array_equal(R, an.R)
    mean, err, used, c2 = g.average()
    mean_o, err_o, used_o, c2_o = an.average()
    np.testing.assert_array_equal(mean, mean_o)
    assert used == used_o and c2 == c2_o
    g.close()


def test_fp32_band_run_keeps_sum_rules_and_reports_the_oracle_chi2_of_its_average():
    P = lorentzian_band(1e-4, seed=2, n_walkers=256)
    prm = sail.Params(n_walkers=256, precision=sail.PREC_FP32, n_sweeps=400, sweeps_per_block=100, resync_every=50,
                      branching=True, T_start_abs=1e6, T_end_abs=0.03, move_scale=0.1 / P.n_omega, A=P.A, B=P.B,
                      seed=6, resync_kind=sail.RESYNC_TENSOR_BF16)
    g = sail.Sail(P.tau, P.F, P.sigma, P.omega, prm)
    g.anneal()
    a, R, chi2, _, _ = g.state()
    np.testing.assert_allclose(a.sum(1), P.A, rtol=2e-6)
    np.testing.assert_allclose(a @ P.omega, P.B, rtol=2e-6)
    mean, err, used, c2 = g.average()
    K, Fh, _ = O.tables(P.tau, P.F, P.sigma, P.omega)
    _, c2_ref = O.residual(K, Fh, mean)
    assert c2 == pytest.approx(c2_ref, rel=1e-9)
    assert 0.0 <= skew(mean, P.omega) <= 1.0
    g.close()
