"""GPU: the paper's protocol against the sawtooth instability through the C ABI --
self-cooling schedule (Sec. self-cooling), acceptance-adaptive branching (Sec. 2.5) and
smoothing with renormalisation (Sec. smoothing).

The FP64 validation path takes every decision the oracle takes: per-sweep accepted counts,
branching multipliers and Deltas, every block's temperature, final spectra, residuals and
chi2, bit for bit.  The FP32 path keeps the sum rules and its chi2 bookkeeping, and its
self-cooling temperatures follow its own population statistics; a batch gives the same
result as each problem alone.
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
                         branch_fraction=sched.branch_fraction, imprint_t=sched.imprint_t,
                         move_scale=sched.move_scale, y_p=sched.y_p, y_m=sched.y_m, y_min=sched.y_min,
                         A=P.A, B=P.B, seed=sched.seed, trace=True, schedule_kind=sched.schedule_kind,
                         adaptive_branching=sched.adaptive, cool_begin=sched.cool_begin,
                         freeze_begin=sched.freeze_begin, smooth_s=sched.smooth_s)
    an = O.Anneal(P.tau, P.F, P.sigma, P.omega, P.A, P.B, n_walkers, sched)
    g = sail.Sail(P.tau, P.F, P.sigma, P.omega, params)
    return an, g


@pytest.mark.parametrize("n_sweeps", [1000, 950])
def test_fp64_protocol_reproduces_every_decision(n_sweeps):
    """Tiny double-Lorentzian workload, 64 walkers, k = 100: self-cooling (boil 2 blocks,
    freeze-out from block 6), adaptive branching and smoothing s = 0.01.  950 sweeps end
    with a partial block (no branching or smoothing after it)."""
    P = tiny_double_lorentz()
    an, g = _pair(P, 64, sail.PREC_FP64, n_sweeps=n_sweeps, sweeps_per_block=100, resync_every=50,
                  branching=True, schedule_kind=1, adaptive=True, cool_begin=0.2, freeze_begin=0.6,
                  smooth_s=0.01, seed=3)
    acc_o, m_o, d_o = an.run(trace=True)
    stats = g.anneal()
    assert len(stats) == (n_sweeps + 99) // 100
    acc_g, m_g, d_g = g.trace()
    np.testing.assert_array_equal(acc_g, acc_o)
    np.testing.assert_array_equal(m_g, m_o)
    np.testing.assert_array_equal(d_g, d_o)
    # the temperature of every block, as the oracle set it from its own statistics
    for s in stats:
        assert s["T"] == an.T[s["sweep_end"] - 1]
    T_blocks = [s["T"] for s in stats]
    assert T_blocks[0] == an.chi2_0 and T_blocks[-1] < T_blocks[3]
    # adaptive branching imprinted fewer walkers as the acceptance fell
    zeros = [s["branch_zeros"] for s in stats if s["branch_zeros"] > 0]
    assert zeros[0] == 16 and min(zeros) < 16
    a, R, chi2, accp, h = g.state()
    np.testing.assert_array_equal(h, an.hash)
    np.testing.assert_array_equal(a, an.a)
    np.testing.assert_array_equal(R, an.R)
    np.testing.assert_array_equal(chi2, an.chi2)


def test_fp32_protocol_keeps_sums_and_follows_its_statistics():
    """Paper-scale grid (200 x 1000), 512 walkers, 8 blocks of 50 sweeps, FP32 moves with
    tensor-core resync.  With branching and smoothing off, the statistics a block reports
    are those the next block's temperature comes from."""
    P = paper_scale_double_lorentz(1e-4, n_walkers=512)
    k, nb = 50, 8
    prm = sail.Params(n_walkers=512, precision=sail.PREC_FP32, n_sweeps=k * nb, sweeps_per_block=k,
                      resync_every=25, branching=False, A=P.A, B=P.B, seed=5, schedule_kind=1,
                      cool_begin=0.25, freeze_begin=0.75, resync_kind=sail.RESYNC_TENSOR)
    g = sail.Sail(P.tau, P.F, P.sigma, P.omega, prm)
    stats = g.anneal()
    bc, bf = O.cooling_blocks(nb, 0.25, 0.75)
    assert stats[0]["T"] == g.info()["chi2_0"]
    tf = -1.0
    T_final = g.info()["chi2_0"] * prm.T_end
    for b in range(1, nb):
        prev = stats[b - 1]
        T, tf = O.self_cooling(b, nb, bc, bf, prev["chi2_mean"], prev["chi2_min"], T_final, tf)
        assert stats[b]["T"] == pytest.approx(T, rel=1e-12)
    g.close()


def test_fp32_smoothing_and_adaptive_branching_keep_sum_rules():
    P = paper_scale_double_lorentz(1e-4, n_walkers=512)
    prm = sail.Params(n_walkers=512, precision=sail.PREC_FP32, n_sweeps=400, sweeps_per_block=50,
                      resync_every=25, branching=True, adaptive_branching=True, smooth_s=0.01,
                      schedule_kind=1, A=P.A, B=P.B, seed=6, resync_kind=sail.RESYNC_TENSOR)
    g = sail.Sail(P.tau, P.F, P.sigma, P.omega, prm)
    stats = g.anneal()
    assert len(stats) == 8
    a, R, chi2, _, _ = g.state()
    assert np.all(a >= 0)
    np.testing.assert_allclose(a.sum(1), P.A, rtol=2e-6)
    np.testing.assert_allclose(a @ P.omega, P.B, rtol=2e-6)
    # chi2 as the tensor-core resync forms it: within the bound of its residuals' error
    # (2e-6 of the model value, the TF32 x3 split and FP32 accumulation, plus FP32 storage)
    K, Fh, _ = O.tables(P.tau, P.F, P.sigma, P.omega)
    for w in range(0, 512, 41):
        model = K @ a[w]
        R_ref = Fh - model
        tol = 2e-6 * model + 6e-8 * np.abs(R_ref) + 1e-6
        c2 = np.sum(R_ref ** 2)
        assert abs(chi2[w] - c2) <= 2 * np.sum(np.abs(R_ref) * tol) + 1e-9 * c2
    g.close()


def test_batch_with_protocol_equals_problems_alone():
    P1 = tiny_double_lorentz()
    P2 = paper_scale_double_lorentz(1e-4, n_walkers=96)
    items, alone = [], []
    for k, (P, W) in enumerate([(P1, 40), (P2, 96)]):
        prm = sail.Params(n_walkers=W, precision=sail.PREC_FP32, n_sweeps=120, sweeps_per_block=20,
                          resync_every=10, branching=True, adaptive_branching=True, smooth_s=0.02,
                          schedule_kind=1, A=P.A, B=P.B, seed=40 + k, resync_kind=sail.RESYNC_TENSOR)
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
        np.testing.assert_array_equal(R2, R1)
        np.testing.assert_array_equal(c2, c1)
        h.close()
    batch.close()
