"""GPU: checkpoint and resume in the middle of a schedule.

The random numbers are counter-based (Philox keyed by walker, sweep and move), so a run's
future depends only on its state: the spectra, residuals and chi2 as stored, the acceptance of
the last sweep, the schedule's position and, for the paper's protocol, the temperatures set so
far and the adaptive-branching and freeze-out state.  A handle that stops after some blocks,
writes a checkpoint, and a new handle that loads it and runs the remaining blocks end bit for
bit like one uninterrupted run: FP64 and FP32 paths, branching, the self-cooling schedule with
adaptive branching and smoothing, and the trace.
"""
import numpy as np
import pytest

import paper_1609_07936_gb300 as sail
from workloads import paper_scale_double_lorentz, tiny_double_lorentz

pytestmark = pytest.mark.gpu


def _params(P, precision, protocol, W):
    kw = dict(n_walkers=W, precision=precision, n_sweeps=700, sweeps_per_block=100, resync_every=50,
              branching=True, T_start=1.0, T_end=1e-6, A=P.A, B=P.B, seed=5, trace=True,
              resync_kind=sail.RESYNC_TENSOR_BF16)
    if protocol:
        kw.update(schedule_kind=sail.SCHEDULE_SELF_COOLING, adaptive_branching=True, smooth_s=1e-2)
    return sail.Params(**kw)


def _final(g):
    a, R, chi2, acc, h = g.state()
    acc_tr, m_tr, d_tr = g.trace()
    mean, err, used, c2 = g.average()
    return a, R, chi2, acc, h, acc_tr, m_tr, d_tr, mean, c2


@pytest.mark.parametrize("precision,protocol,W", [(sail.PREC_FP64, False, 32), (sail.PREC_FP64, True, 32),
                                                  (sail.PREC_FP32, False, 256), (sail.PREC_FP32, True, 256)])
def test_resumed_run_equals_the_uninterrupted_one(precision, protocol, W):
    P = tiny_double_lorentz() if precision == sail.PREC_FP64 else paper_scale_double_lorentz(1e-4, n_walkers=W)
    prm = _params(P, precision, protocol, W)
    whole = sail.Sail(P.tau, P.F, P.sigma, P.omega, prm)
    whole.anneal()
    ref = _final(whole)
    whole.close()

    first = sail.Sail(P.tau, P.F, P.sigma, P.omega, prm)
    first.anneal(3)
    blob = first.checkpoint()
    first.close()
    second = sail.Sail(P.tau, P.F, P.sigma, P.omega, prm)
    second.restore(blob)
    assert second.info()["sweeps_done"] == 300
    stats = second.anneal()
    assert len(stats) == 4 and stats[0]["block"] == 3
    out = _final(second)
    second.close()
    for x, y in zip(ref, out):
        np.testing.assert_array_equal(np.asarray(x), np.asarray(y))


def test_restore_refuses_another_problem():
    P = tiny_double_lorentz()
    prm = _params(P, sail.PREC_FP32, False, 16)
    g = sail.Sail(P.tau, P.F, P.sigma, P.omega, prm)
    g.anneal(1)
    blob = g.checkpoint()
    prm2 = _params(P, sail.PREC_FP32, False, 16)
    prm2.seed = 6
    h = sail.Sail(P.tau, P.F, P.sigma, P.omega, prm2)
    with pytest.raises(sail.SailError):
        h.restore(blob)
    with pytest.raises(sail.SailError):
        g.restore(blob[:100])
    g.close()
    h.close()
