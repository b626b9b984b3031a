"""GPU: FP64 acceptance near the threshold (fp64_accept).

With fp64_accept = 2 every feasible move's Metropolis decision is taken from Delta chi2 in
FP64 on the walker's FP32 state, so the recheck counter equals the number of feasible moves
and the flip counter the decisions that FP32 would have taken differently; with
fp64_accept = 1 only decisions within 1e-5 S of the threshold are taken again.  Where no
decision changes, the chain is the unguarded FP32 chain move for move (the FP32 Delta chi2 of
the guarded kernel is formed by the same operations), on both move loops.
"""
import numpy as np
import pytest

import paper_1609_07936_gb300 as sail
from workloads import paper_scale_double_lorentz, tiny_double_lorentz

pytestmark = pytest.mark.gpu


def _run(P, W, loop, guard, blocks, seed=3, **kw):
    prm = sail.Params(n_walkers=W, precision=sail.PREC_FP32, n_sweeps=blocks * 20, sweeps_per_block=20,
                      resync_every=10, branching=True, A=P.A, B=P.B, seed=seed, sweep_loop=loop,
                      fp64_accept=guard, **kw)
    g = sail.Sail(P.tau, P.F, P.sigma, P.omega, prm)
    stats = g.anneal(blocks)
    info = g.info()
    state = g.state()
    g.close()
    return stats, info, state


@pytest.mark.parametrize("loop", [1, 2])
def test_every_feasible_decision_is_rechecked_in_mode_2(loop):
    P = paper_scale_double_lorentz(1e-4, n_walkers=256)
    stats, info, _ = _run(P, 256, loop, 2, 2, T_start=1e-3, T_end=1e-5)
    per_block = 20 * P.n_omega * 256
    feasible = sum(per_block * (1.0 - b["positivity_rejected"]) for b in stats)
    assert info["fp64_rechecks"] == pytest.approx(feasible, abs=0.5 * len(stats))
    assert info["fp64_rechecks"] > 0
    # FP32 and FP64 decisions on the same state almost never differ
    assert info["fp64_flips"] <= 1e-4 * info["fp64_rechecks"]


@pytest.mark.parametrize("loop", [1, 2])
@pytest.mark.parametrize("mode", [1, 2])
def test_unchanged_decisions_keep_the_fp32_chain(loop, mode):
    P = tiny_double_lorentz()
    base = _run(P, 64, loop, 0, 3)
    guarded = _run(P, 64, loop, mode, 3)
    info = guarded[1]
    if mode == 2:
        assert info["fp64_rechecks"] > 0
    if info["fp64_flips"] == 0:
        a0, R0, c0, acc0, h0 = base[2]
        a1, R1, c1, acc1, h1 = guarded[2]
        np.testing.assert_array_equal(h0, h1)          # every decision
        np.testing.assert_array_equal(a0, a1)
        np.testing.assert_array_equal(R0, R1)
        # chi2 bookkeeping takes the FP64 value of a rechecked move
        np.testing.assert_allclose(c1, c0, rtol=1e-6)


def test_unguarded_run_reports_no_rechecks():
    P = tiny_double_lorentz()
    _, info, _ = _run(P, 64, 0, 0, 1)
    assert info["fp64_rechecks"] == 0 and info["fp64_flips"] == 0
