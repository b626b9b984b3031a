"""GPU: one inversion's population split over several handles, against one handle.

Two or three shards of the population live on this GPU and exchange through the in-process
communicator; on several GPUs the same driver runs one shard per rank over torch.distributed
(NCCL), and the donor rows land in the receiving GPU's memory the same way.  Every shard
draws its walkers' population-indexed random numbers, the branching solve runs on the device
(sail_branch_solve) over the gathered chi2, and receivers are imprinted from donor rows
(sail_walker_rows, sail_imprint_rows): the multipliers, Delta and every walker's final
spectrum, residual, chi2 and move hash equal the single handle's run with branching, bit for
bit, on the FP64 validation path and the FP32 production path (tensor-core recomputation).
"""
import numpy as np
import pytest

import paper_1609_07936_gb300 as sail
from paper_1609_07936_gb300.sharded import CudaShard, LocalComm, ShardedAnneal
from workloads import paper_scale_double_lorentz, tiny_double_lorentz

pytestmark = pytest.mark.gpu


def _run(P, prm, spans, blocks):
    whole = sail.Sail(P.tau, P.F, P.sigma, P.omega, prm)
    whole.anneal(blocks)
    ref = whole.state()
    m_ref, d_ref = whole.trace()[1:]
    whole.close()
    n_total = prm.n_walkers
    shards = [CudaShard(P.tau, P.F, P.sigma, P.omega, prm, o, n, n_total) for o, n in spans]
    run = ShardedAnneal(shards, [spans], LocalComm(), prm.branch_fraction, prm.imprint_t)
    for _ in range(blocks):
        run.block()
    for b, ev in enumerate(run.events):
        np.testing.assert_array_equal(ev["m"], m_ref[b])
        assert ev["delta"] == d_ref[b]
    for s in shards:
        a, R, chi2, acc, h = s.handle.state()
        sl = slice(s.offset, s.offset + s.n_walkers)
        for x, y in zip((a, R, chi2, acc, h), ref):
            np.testing.assert_array_equal(x, y[sl])
        s.close()
    assert any((m == 0).any() for m in m_ref)


def test_sharded_fp64_equals_one_handle():
    P = tiny_double_lorentz()
    prm = sail.Params(n_walkers=40, precision=sail.PREC_FP64, n_sweeps=60, sweeps_per_block=20, resync_every=10,
                      branching=True, T_start=1.0, T_end=1e-3, A=P.A, B=P.B, seed=21, trace=True)
    _run(P, prm, [(0, 13), (13, 27)], 3)


@pytest.mark.parametrize("spans", [[(0, 256), (256, 256)], [(0, 100), (100, 301), (401, 111)]])
def test_sharded_fp32_equals_one_handle(spans):
    P = paper_scale_double_lorentz(1e-4, n_walkers=512)
    prm = sail.Params(n_walkers=512, precision=sail.PREC_FP32, n_sweeps=300, sweeps_per_block=100,
                      resync_every=50, branching=True, T_start_abs=1e6, T_end_abs=0.03, move_scale=1e-4,
                      A=P.A, B=P.B, seed=22, trace=True, resync_kind=sail.RESYNC_TENSOR_BF16)
    _run(P, prm, spans, 3)


def test_shard_parameters_are_checked():
    P = tiny_double_lorentz()
    bad = sail.Params(n_walkers=16, precision=sail.PREC_FP32, n_sweeps=20, A=P.A, B=P.B, walker_offset=10,
                      walker_total=20)
    with pytest.raises(sail.SailError):
        sail.Sail(P.tau, P.F, P.sigma, P.omega, bad)
    ok = sail.Params(n_walkers=16, precision=sail.PREC_FP32, n_sweeps=20, A=P.A, B=P.B, walker_offset=4,
                     walker_total=20, branching=False)
    g = sail.Sail(P.tau, P.F, P.sigma, P.omega, ok)
    with pytest.raises(sail.SailError):
        g.branch_solve(np.ones(21), 0, 0.25)     # more than walker_total
    with pytest.raises(sail.SailError):
        g.imprint_rows([3, 3], *g.walker_rows([1, 2]), 0.1)   # a walker imprinted twice
    g.close()
