"""GPU: the FP32 look-ahead move loop at the edges of its proposal windows, through the C ABI.

Each walker keeps 16 proposals drawn (two windows of 8), takes the first feasible one by a
ballot and counts the infeasible ones before it as rejected; windows may run past the end of
a sweep, and a sweep may hold fewer proposals than one window.  Bin counts of 3 to 37 (fewer
than a window, partial last windows, sweeps of odd length) and a ragged tau count exercise
those paths; the FP32 sweep draws the oracle's words, so over a few sweeps nearly every
walker accepts exactly the oracle's number of moves in every sweep.  The shared-bin sweep is
run on the same cases, and a 300-point tau grid (10 chunks: the one-move loop, which takes
over where columns cannot be prefetched) on both.  The look-ahead loop and the one-move loop
(sweep_loop = 2 and 1) leave bit-identical states, with branching and recomputation.
"""
import numpy as np
import pytest

import oracle as O
import paper_1609_07936_gb300 as sail
from workloads import Peak, make_problem

pytestmark = pytest.mark.gpu


def _problem(n_omega, n_tau=40, n_walkers=64):
    tau = 3.0 * np.arange(n_tau, dtype=np.float64) / (n_tau - 1)
    peaks = [Peak("lorentz", 2.0, 0.4, 0.6), Peak("gauss", 5.0, 0.8, 0.4)]
    return make_problem(f"edges_{n_omega}", tau, n_omega, 10.0, peaks, 1e-4, 3, n_walkers)


@pytest.mark.parametrize("n_omega", [3, 5, 13, 17, 37])
@pytest.mark.parametrize("W,loop", [(0, 2), (0, 1), (2, 0), (8, 0)])
def test_fp32_windows_take_the_oracle_decisions(n_omega, W, loop):
    P = _problem(n_omega)
    kw = dict(n_sweeps=6, sweeps_per_block=6, resync_every=3, branching=False, T_start=0.5, T_end=0.5, seed=23)
    an = O.Anneal(P.tau, P.F, P.sigma, P.omega, P.A, P.B, 64, O.Schedule(shared_bins=W, **kw))
    acc_o, _, _ = an.run(trace=True)
    g = sail.Sail(P.tau, P.F, P.sigma, P.omega,
                  sail.Params(n_walkers=64, precision=sail.PREC_FP32, A=P.A, B=P.B, trace=True, shared_bins=W,
                              sweep_loop=loop, resync_kind=sail.RESYNC_FP32, **kw))
    g.anneal()
    acc_g, _, _ = g.trace()
    assert acc_g.shape == acc_o.shape
    same = np.all(acc_g == acc_o, axis=0)
    assert same.mean() >= 0.9, same.mean()
    # the runs took decisions both ways
    assert acc_o.sum() > 0 and (acc_o < n_omega).any()
    a = g.state()[0]
    np.testing.assert_allclose(a.sum(1), P.A, rtol=2e-6)
    np.testing.assert_allclose(a @ P.omega, P.B, rtol=2e-6)
    for w in np.flatnonzero(same):
        np.testing.assert_allclose(a[w], an.a[w], rtol=0, atol=1e-4 * an.a[w].max())
    g.close()


@pytest.mark.parametrize("n_omega", [5, 13])
def test_fp32_hastings_windows_take_the_oracle_decisions(n_omega):
    """The Hastings variant also skips proposals whose reverse move cannot be proposed."""
    P = _problem(n_omega)
    kw = dict(n_sweeps=6, sweeps_per_block=6, resync_every=3, branching=False, T_start=0.5, T_end=0.5, seed=29)
    an = O.Anneal(P.tau, P.F, P.sigma, P.omega, P.A, P.B, 64, O.Schedule(hastings=True, **kw))
    acc_o, _, _ = an.run(trace=True)
    g = sail.Sail(P.tau, P.F, P.sigma, P.omega,
                  sail.Params(n_walkers=64, precision=sail.PREC_FP32, A=P.A, B=P.B, trace=True, hastings=True,
                              sweep_loop=2, resync_kind=sail.RESYNC_FP32, **kw))
    g.anneal()
    acc_g, _, _ = g.trace()
    same = np.all(acc_g == acc_o, axis=0)
    assert same.mean() >= 0.9, same.mean()
    g.close()


@pytest.mark.parametrize("n_tau", [300, 512])
@pytest.mark.parametrize("W", [0, 2, 4])
def test_fp32_wide_tau_takes_the_oracle_decisions(W, n_tau):
    """300 tau points (10 chunks) and the library's maximum, 512 (16 chunks)."""
    P = _problem(37, n_tau=n_tau, n_walkers=32)
    kw = dict(n_sweeps=6, sweeps_per_block=6, resync_every=3, branching=False, T_start=0.5, T_end=0.5, seed=41)
    an = O.Anneal(P.tau, P.F, P.sigma, P.omega, P.A, P.B, 32, O.Schedule(shared_bins=W, **kw))
    acc_o, _, _ = an.run(trace=True)
    g = sail.Sail(P.tau, P.F, P.sigma, P.omega,
                  sail.Params(n_walkers=32, precision=sail.PREC_FP32, A=P.A, B=P.B, trace=True, shared_bins=W,
                              resync_kind=sail.RESYNC_FP32, **kw))
    g.anneal()
    assert g.info()["sweep_lanes"] == 16
    acc_g, _, _ = g.trace()
    same = np.all(acc_g == acc_o, axis=0)
    assert same.mean() >= 0.9, same.mean()
    assert acc_o.sum() > 0 and (acc_o < 37).any()
    g.close()


@pytest.mark.parametrize("n_tau", [5, 37, 230])
def test_quad_compact_columns_at_ragged_and_widest_tau(n_tau):
    """The one-move loop with 8 lanes per walker forms its columns from tables of every fourth
    tau point: 5 and 37 points end in a partial quad (rho zero past n_tau), 230 points are the
    widest 8-lane layout (8 chunks, rows of 64 floats).  The walkers take the oracle's decisions
    and keep the sum rules."""
    P = _problem(21, n_tau=n_tau)
    kw = dict(n_sweeps=6, sweeps_per_block=6, resync_every=3, branching=False, T_start=0.5, T_end=0.5, seed=53)
    an = O.Anneal(P.tau, P.F, P.sigma, P.omega, P.A, P.B, 64, O.Schedule(**kw))
    acc_o, _, _ = an.run(trace=True)
    g = sail.Sail(P.tau, P.F, P.sigma, P.omega,
                  sail.Params(n_walkers=64, precision=sail.PREC_FP32, A=P.A, B=P.B, trace=True, sweep_loop=1,
                              resync_kind=sail.RESYNC_FP32, **kw))
    assert g.info()["sweep_lanes"] == 8
    g.anneal()
    acc_g, _, _ = g.trace()
    same = np.all(acc_g == acc_o, axis=0)
    assert same.mean() >= 0.9, same.mean()
    assert acc_o.sum() > 0 and (acc_o < 21).any()
    a = g.state()[0]
    np.testing.assert_allclose(a.sum(1), P.A, rtol=2e-6)
    np.testing.assert_allclose(a @ P.omega, P.B, rtol=2e-6)
    g.close()


def test_uneven_tau_grid_runs_on_sixteen_lanes():
    """The 8-lane sweep forms its columns along a uniform tau grid; an uneven grid of 40 points
    (tau_i = 3 (i / 39)^1.5) takes the 16-lane sweep with full factor rows, which still takes
    the oracle's decisions, and an explicit request for 8 lanes is refused."""
    tau = 3.0 * (np.arange(40, dtype=np.float64) / 39) ** 1.5
    peaks = [Peak("lorentz", 2.0, 0.4, 0.6), Peak("gauss", 5.0, 0.8, 0.4)]
    P = make_problem("uneven_tau", tau, 37, 10.0, peaks, 1e-4, 3, 64)
    kw = dict(n_sweeps=6, sweeps_per_block=6, resync_every=3, branching=False, T_start=0.5, T_end=0.5, seed=47)
    an = O.Anneal(P.tau, P.F, P.sigma, P.omega, P.A, P.B, 64, O.Schedule(**kw))
    acc_o, _, _ = an.run(trace=True)
    g = sail.Sail(P.tau, P.F, P.sigma, P.omega,
                  sail.Params(n_walkers=64, precision=sail.PREC_FP32, A=P.A, B=P.B, trace=True,
                              resync_kind=sail.RESYNC_FP32, **kw))
    assert g.info()["sweep_lanes"] == 16
    g.anneal()
    acc_g, _, _ = g.trace()
    same = np.all(acc_g == acc_o, axis=0)
    assert same.mean() >= 0.9, same.mean()
    assert acc_o.sum() > 0 and (acc_o < 37).any()
    g.close()
    with pytest.raises(sail.SailError, match="uniform tau"):
        sail.Sail(P.tau, P.F, P.sigma, P.omega,
                  sail.Params(n_walkers=64, precision=sail.PREC_FP32, A=P.A, B=P.B, sweep_lanes=8, **kw))


@pytest.mark.parametrize("hastings", [False, True])
def test_lookahead_and_one_move_loops_are_the_same_chain(hastings):
    """Paper-scale grid (200 tau, 1000 bins), 512 walkers, two blocks of 50 sweeps with branching
    and tensor-core recomputation: both FP32 move loops end in the same bits.  They draw the same
    proposals and take the same decisions; the one-move loop forms its columns from the
    quad-compact tables (FP32 values that differ from the full rows' in the last bits), so the
    states agree bit for bit while no delta chi2 falls within rounding of its threshold, and the
    residuals are recomputed at the block ends."""
    from workloads import paper_scale_double_lorentz
    P = paper_scale_double_lorentz(1e-4, n_walkers=512)
    out = []
    for loop in (1, 2):
        prm = sail.Params(n_walkers=512, precision=sail.PREC_FP32, n_sweeps=100, sweeps_per_block=50,
                          resync_every=25, branching=True, T_start=10.0, T_end=1e-6, A=P.A, B=P.B, seed=13,
                          hastings=hastings, sweep_loop=loop, resync_kind=sail.RESYNC_TENSOR_BF16, trace=True)
        g = sail.Sail(P.tau, P.F, P.sigma, P.omega, prm)
        stats = g.anneal()
        a, R, chi2, acc, _ = g.state()
        out.append((a, R, chi2, acc, g.trace()[0], [s["positivity_rejected"] for s in stats]))
        g.close()
    for x, y in zip(out[0], out[1]):
        np.testing.assert_array_equal(np.asarray(x), np.asarray(y))


@pytest.mark.parametrize("W,loop", [(0, 1), (0, 2), (4, 0)])
def test_fp32_paper_grid_takes_the_oracle_decisions(W, loop):
    """The benchmark's grid (200 tau, 1000 bins, noise 1e-4), 64 walkers, 2 sweeps of 1000 moves
    at T = chi2_0 / 10: at least 90% of the walkers accept exactly the oracle's number of moves
    in both sweeps."""
    from workloads import paper_scale_double_lorentz
    P = paper_scale_double_lorentz(1e-4, n_walkers=64)
    kw = dict(n_sweeps=2, sweeps_per_block=2, resync_every=1, branching=False, T_start=0.1, T_end=0.1, seed=47)
    an = O.Anneal(P.tau, P.F, P.sigma, P.omega, P.A, P.B, 64, O.Schedule(shared_bins=W, **kw))
    acc_o, _, _ = an.run(trace=True)
    g = sail.Sail(P.tau, P.F, P.sigma, P.omega,
                  sail.Params(n_walkers=64, precision=sail.PREC_FP32, A=P.A, B=P.B, trace=True, shared_bins=W,
                              sweep_loop=loop, resync_kind=sail.RESYNC_FP32, **kw))
    g.anneal()
    acc_g, _, _ = g.trace()
    same = np.all(acc_g == acc_o, axis=0)
    assert same.mean() >= 0.9, same.mean()
    assert 0 < acc_o.mean() < P.n_omega
    g.close()


@pytest.mark.parametrize("W", [0, 4])
def test_spectra_in_global_memory_leave_the_same_bits(W):
    """512 tau x 1024 bins, no branching: 64 walkers leave their spectra staged in shared memory
    (factor tables 136 KB + 8 or 16 KB per walker group), 4096 walkers do not (7-14 groups per
    block), and each walker's chain depends only on its own index, so walkers 0..63 end in the
    same bits either way.  The one-move loop reads a move's b values one move ahead and patches
    them after an accepted move that wrote one of those bins; this compares that path in shared
    and in global memory."""
    from workloads import make_problem as mk
    tau = 8.0 * np.arange(512, dtype=np.float64) / 511
    P = mk("global_b", tau, 1024, 20.0, [Peak("lorentz", 2.0, 0.3, 0.6), Peak("lorentz", 5.0, 0.5, 0.4)],
           1e-4, 5, 64)
    out = []
    for n_walkers in (64, 4096):
        prm = sail.Params(n_walkers=n_walkers, precision=sail.PREC_FP32, n_sweeps=4, sweeps_per_block=4,
                          resync_every=2, branching=False, T_start=0.5, T_end=0.5, A=P.A, B=P.B, seed=53,
                          shared_bins=W, resync_kind=sail.RESYNC_FP32, trace=True)
        g = sail.Sail(P.tau, P.F, P.sigma, P.omega, prm)
        g.anneal()
        a, R, chi2, acc, _ = g.state()
        out.append((a[:64], R[:64], chi2[:64], acc[:64], g.trace()[0][:, :64]))
        g.close()
    assert out[0][4].sum() > 0 and (out[0][4] < 1024).any()
    for x, y in zip(out[0], out[1]):
        np.testing.assert_array_equal(x, y)


@pytest.mark.parametrize("schedule", ["paper", "to_target"])
def test_automatic_loop_follows_the_rejections_with_the_same_chain(schedule):
    """With sweep_loop = 0 and enough walkers for the look-ahead loop (16 a SM), the next
    block runs the look-ahead loop while the last block rejected at least 30% of its proposals
    for positivity (the paper's schedule, ~40%) and the one-move loop below (the to-target
    schedule, ~25%); either way the states equal those of the explicit loops bit for bit."""
    from workloads import paper_scale_double_lorentz
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    W = 16 * sms
    P = paper_scale_double_lorentz(1e-4, n_walkers=W)
    temps = (dict(T_start=10.0, T_end=1e-9) if schedule == "paper"
             else dict(T_start_abs=1e6, T_end_abs=0.03, move_scale=0.1 / P.n_omega))
    out = {}
    for loop in (0, 1):
        g = sail.Sail(P.tau, P.F, P.sigma, P.omega,
                      sail.Params(n_walkers=W, precision=sail.PREC_FP32, n_sweeps=20000, sweeps_per_block=20,
                                  resync_every=10, branching=True, A=P.A, B=P.B, seed=8, sweep_loop=loop,
                                  resync_kind=sail.RESYNC_TENSOR_BF16, **temps))
        first = g.info()["sweep_ahead"]
        stats = g.anneal(2)
        out[loop] = (first, g.info()["sweep_ahead"], stats[-1]["positivity_rejected"], g.state())
        g.close()
    first, nxt, pos, _ = out[0]
    assert first == 1                                   # create-time choice: enough walkers
    assert nxt == (1 if pos >= 0.30 else 0)
    assert (pos >= 0.30) == (schedule == "paper")
    assert out[1][1] == 0                               # explicit one-move loop
    for x, y in zip(out[0][3], out[1][3]):
        np.testing.assert_array_equal(x, y)


def test_bench_configuration_samples_take_the_oracle_decisions():
    """The bench's launch configuration at full size — 4096 walkers on the paper grid (the
    look-ahead loop, 8 lanes a walker, 7 warps a SM, spectra staged in shared memory, the
    tensor-core recomputation) — for 2 sweeps at T = chi2_0 / 10 without branching: the walkers
    0-63 and 4032-4095, run by the oracle as shards of the same population (their own random
    counters), accept exactly the oracle's number of moves in both sweeps for at least 90% of
    them."""
    from workloads import paper_scale_double_lorentz
    P = paper_scale_double_lorentz(1e-4, n_walkers=4096)
    kw = dict(n_sweeps=2, sweeps_per_block=2, resync_every=2, branching=False, T_start=0.1, T_end=0.1, seed=47)
    g = sail.Sail(P.tau, P.F, P.sigma, P.omega,
                  sail.Params(n_walkers=4096, precision=sail.PREC_FP32, A=P.A, B=P.B, trace=True,
                              resync_kind=sail.RESYNC_TENSOR_BF16, **kw))
    assert g.info()["sweep_lanes"] == 8 and g.info()["sweep_ahead"] == 1
    g.anneal()
    acc_g = g.trace()[0]
    g.close()
    for lo in (0, 4032):
        an = O.Anneal(P.tau, P.F, P.sigma, P.omega, P.A, P.B, 64, O.Schedule(walker_base=lo, **kw))
        acc_o, _, _ = an.run(trace=True)
        same = np.all(acc_g[:, lo:lo + 64] == acc_o, axis=0)
        assert same.mean() >= 0.9, (lo, same.mean())
        assert 0 < acc_o.mean() < P.n_omega
