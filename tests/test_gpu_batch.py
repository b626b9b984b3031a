"""GPU: many uneven inversions in one persistent sweep launch.

A problem's results must not depend on the batch: its random numbers are keyed by its own
seed and walker indices and its arithmetic is per walker or per problem, so every walker of
every problem ends bit-identical to the same problem annealed alone through a single handle,
whatever the autotuner picks for the walker-to-block mapping and the tensor-core tile width.
The batched sweep is also checked against the FP64 oracle directly, problem by problem.
"""
import numpy as np
import pytest

import paper_1609_07936_gb300 as sail
from workloads import Peak, make_problem, random_batch_problem

pytestmark = pytest.mark.gpu


def _problems():
    specs = [  # n_tau, n_omega, walkers, W, peaks, noise, seed
        (50, 200, 256, 10.0, [Peak("lorentz", 2.0, 0.4, 1.0)], 1e-3, 1),
        (77, 300, 301, 12.0, [Peak("gauss", 3.0, 0.8, 0.6), Peak("lorentz", 7.0, 0.5, 0.4)], 1e-4, 2),
        (200, 1000, 96, 20.0, [Peak("lorentz", 2.0, 0.3, 0.6), Peak("lorentz", 5.0, 0.5, 0.4)], 1e-4, 3),
        (300, 450, 130, 15.0, [Peak("gauss", 6.0, 1.5, 1.0)], 1e-5, 4),
    ]
    out = []
    for k, (nt, no, nw, W, peaks, lvl, seed) in enumerate(specs):
        tau = 6.0 * np.arange(nt, dtype=np.float64) / (nt - 1)
        P = make_problem(f"b{k}", tau, no, W, peaks, lvl, seed, nw)
        prm = sail.Params(n_walkers=nw, precision=sail.PREC_FP32, n_sweeps=60 + 20 * k, sweeps_per_block=20,
                          resync_every=10, branching=True, T_start=3.0, T_end=1e-6, A=P.A, B=P.B, seed=100 + k,
                          resync_kind=sail.RESYNC_TENSOR)
        out.append((P, prm))
    return out


@pytest.mark.parametrize("autotune", [True, False])
def test_batch_equals_problems_alone(autotune):
    probs = _problems()
    batch = sail.Batch([(P.tau, P.F, P.sigma, P.omega, prm) for P, prm in probs], autotune=autotune)
    blocks = batch.anneal(2)
    assert blocks == 2
    for k, (P, prm) in enumerate(probs):
        alone = sail.Sail(P.tau, P.F, P.sigma, P.omega, prm)
        alone.anneal(2)
        a1, R1, c1, acc1, _ = alone.state()
        a2, R2, c2, acc2, _ = batch.handles[k].state()
        np.testing.assert_array_equal(a2, a1)
        np.testing.assert_array_equal(R2, R1)
        np.testing.assert_array_equal(c2, c1)
        np.testing.assert_array_equal(acc2, acc1)
        m1 = alone.average()
        m2 = batch.handles[k].average()
        np.testing.assert_array_equal(m2[0], m1[0])
        assert m2[3] == m1[3]
        alone.close()
    t = batch.tuning()
    assert t["item_pairs"] in (4, 8, 16) and t["sweep_launches"] >= 4
    # run the batch to the end of every schedule: problems finish at different blocks
    batch.anneal()
    for k, (P, prm) in enumerate(probs):
        assert batch.handles[k].info()["sweeps_done"] == prm.n_sweeps
    batch.close()


def test_uneven_batch_recipe_runs():
    """Eight inversions drawn as in the uneven-batch workload (n_tau U{50..500}, n_omega
    U{200..2000}, walkers U{256..4096}, noise log-uniform) run a block and keep their sum rules."""
    probs = [random_batch_problem(i, seed=7) for i in range(8)]
    items = []
    for P in probs:
        prm = sail.Params(n_walkers=P.n_walkers, precision=sail.PREC_FP32, n_sweeps=100, sweeps_per_block=20,
                          resync_every=10, branching=True, T_start=1.0, T_end=1e-6, A=P.A, B=P.B,
                          resync_kind=sail.RESYNC_TENSOR)
        items.append((P.tau, P.F, P.sigma, P.omega, prm))
    batch = sail.Batch(items, autotune=True)
    batch.anneal(1)
    for k, P in enumerate(probs):
        a = batch.handles[k].state()[0]
        assert np.all(a >= 0)
        np.testing.assert_allclose(a.sum(1), P.A, rtol=2e-6)
        np.testing.assert_allclose(a @ P.omega, P.B, rtol=2e-6)
    batch.close()


def _oracle_decisions(P, prm, kw):
    """Per-sweep accepted counts of every walker from the FP64 oracle on the same schedule."""
    import oracle as O
    an = O.Anneal(P.tau, P.F, P.sigma, P.omega, P.A, P.B, prm.n_walkers, O.Schedule(seed=prm.seed, **kw))
    acc, _, _ = an.run(trace=True)
    return acc, an


def test_batch_takes_the_oracle_decisions():
    """Three problems inside one batch, in different classes of the batched sweep: 40 tau points
    (8 lanes per walker), 300 tau points (16 lanes per walker, 10 chunks) and 200 tau points with
    the 1000-bin paper grid; spectra stay in global memory.  Over 6 sweeps at a fixed temperature
    at least 90% of each problem's walkers accept exactly the oracle's number of moves in every
    sweep (Sec. 2.2: the FP32 sweep draws the oracle's Philox words; the few walkers that part
    are those where an FP32 rounding flips a decision), and those walkers' spectra agree with the
    oracle's."""
    kw = dict(n_sweeps=6, sweeps_per_block=6, resync_every=3, branching=False, T_start=0.5, T_end=0.5)
    specs = [(40, 37, 64, 3.0), (300, 60, 48, 6.0), (200, 1000, 32, 8.0)]
    probs = []
    for k, (nt, no, nw, tmax) in enumerate(specs):
        tau = tmax * np.arange(nt, dtype=np.float64) / (nt - 1)
        peaks = [Peak("lorentz", 2.0, 0.3, 0.6), Peak("lorentz", 5.0, 0.5, 0.4)]
        P = make_problem(f"bo{k}", tau, no, 10.0 if no < 1000 else 20.0, peaks, 1e-4, 11 + k, nw)
        prm = sail.Params(n_walkers=nw, precision=sail.PREC_FP32, A=P.A, B=P.B, seed=300 + k, trace=True,
                          resync_kind=sail.RESYNC_FP32, **kw)
        probs.append((P, prm))
    batch = sail.Batch([(P.tau, P.F, P.sigma, P.omega, prm) for P, prm in probs], autotune=False)
    batch.anneal()
    lanes = set()
    for k, (P, prm) in enumerate(probs):
        h = batch.handles[k]
        lanes.add(h.info()["sweep_lanes"])
        acc_g, _, _ = h.trace()
        acc_o, an = _oracle_decisions(P, prm, kw)
        assert acc_g.shape == acc_o.shape
        same = np.all(acc_g == acc_o, axis=0)
        assert same.mean() >= 0.9, (k, same.mean())
        assert acc_o.sum() > 0 and (acc_o < P.n_omega).any()
        a = h.state()[0]
        for w in np.flatnonzero(same):
            np.testing.assert_allclose(a[w], an.a[w], rtol=0, atol=1e-4 * an.a[w].max())
    assert lanes == {8, 16}
    batch.close()
