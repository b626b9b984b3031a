"""CPU: one inversion's population split over two gloo ranks (world size 2), against one rank.

The sharding driver (paper_1609_07936_gb300.sharded) orders the block-end steps of Sec. 2.5
over shards: gather every walker's chi2, the same branching solve on every rank, donor rows
sent point to point to the rank that holds the receiver, imprint there.  Its engine here is
the FP64 oracle (a shard = the oracle run on a contiguous range of walkers with their
population indices in the random counters, branching off), so the test checks the driver's
bookkeeping and exchange against the oracle's own single-population run with branching: the
multipliers, Delta and final spectra, residuals and chi2 of every walker are identical, bit for
bit, also with uneven shards and with a rank holding two shards.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

N_WALKERS, BLOCKS, K = 24, 3, 20


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _schedule(**kw):
    import oracle as O
    base = dict(n_sweeps=BLOCKS * K, sweeps_per_block=K, resync_every=10, T_start=1.0, T_end=1e-3, seed=7)
    base.update(kw)
    return O.Schedule(**base)


class OracleShard:
    """Walkers [offset, offset + n) of the population, annealed by the FP64 oracle."""

    def __init__(self, P, offset, n):
        import oracle as O
        self.O = O
        self.offset, self.n_walkers = offset, n
        self.n_omega, self.n_tau = P.n_omega, P.n_tau
        self.seed = 7
        self.an = O.Anneal(P.tau, P.F, P.sigma, P.omega, P.A, P.B, n,
                           _schedule(branching=False, walker_base=offset))

    def run_block(self):
        self.an.run(K)

    def chi2(self):
        return self.an.chi2.copy()

    def rows(self, idx):
        import torch
        return torch.as_tensor(self.an.a[idx].copy()), torch.as_tensor(self.an.R[idx].copy())

    def imprint(self, idx, a_rows, R_rows, t):
        for q, l in enumerate(idx):
            a, R, c2 = self.O.imprint(t, self.an.a[l], self.an.R[l], a_rows[q].numpy(), R_rows[q].numpy())
            self.an.a[l], self.an.R[l], self.an.chi2[l] = a, R, c2

    def solve(self, chi2_all, block, fraction):
        xi = self.O.xi_for_block(self.seed, block, chi2_all.size)
        m, delta = self.O.branch_multipliers(chi2_all, xi, fraction)
        zl, dl = self.O.pairs(m)
        return m, delta, zl, dl


def _rank(rank, world, port, layout, q):
    import torch.distributed as dist
    from paper_1609_07936_gb300.sharded import ShardedAnneal, TorchComm
    from workloads import tiny_double_lorentz
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    P = tiny_double_lorentz()
    shards = [OracleShard(P, o, n) for o, n in layout[rank]]
    run = ShardedAnneal(shards, layout, TorchComm(dist, "cpu"), branch_fraction=0.25, imprint_t=0.1)
    for _ in range(BLOCKS):
        run.block()
    q.put((rank, [(s.offset, s.an.a, s.an.R, s.an.chi2) for s in shards],
           [(e["m"], e["delta"]) for e in run.events]))
    dist.destroy_process_group()


@pytest.mark.parametrize("layout", [
    [[(0, 12)], [(12, 12)]],                    # even halves
    [[(0, 7)], [(7, 17)]],                      # uneven
    [[(0, 5), (5, 6)], [(11, 13)]],             # two shards on rank 0
])
def test_sharded_run_equals_one_population(layout):
    import oracle as O
    from workloads import tiny_double_lorentz
    P = tiny_double_lorentz()
    ref = O.Anneal(P.tau, P.F, P.sigma, P.omega, P.A, P.B, N_WALKERS, _schedule(branching=True))
    _, m_ref, d_ref = ref.run(trace=True)
    assert len(d_ref) == BLOCKS

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, layout, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict((r, (st, ev)) for r, st, ev in (q.get(timeout=300) for _ in range(2)))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # every rank solved the same branching events, equal to the single population's
    for r in range(2):
        events = out[r][1]
        assert len(events) == BLOCKS
        for b, (m, delta) in enumerate(events):
            np.testing.assert_array_equal(m, m_ref[b])
            assert delta == d_ref[b]
    # the shards' walkers end where the single population's do
    seen = 0
    for r in range(2):
        for offset, a, R, chi2 in out[r][0]:
            n = a.shape[0]
            np.testing.assert_array_equal(a, ref.a[offset:offset + n])
            np.testing.assert_array_equal(R, ref.R[offset:offset + n])
            np.testing.assert_array_equal(chi2, ref.chi2[offset:offset + n])
            seen += n
    assert seen == N_WALKERS
    # and branching did move walkers across the shard boundary in some event
    assert any((m_ref[b] == 0).any() for b in range(BLOCKS))


def test_layout_must_tile_the_population():
    from paper_1609_07936_gb300.sharded import LocalComm, ShardedAnneal

    class Dummy:
        def __init__(self, o, n):
            self.offset, self.n_walkers = o, n

    with pytest.raises(ValueError):
        ShardedAnneal([Dummy(0, 4)], [[(0, 4), (5, 3)]], LocalComm())
    with pytest.raises(ValueError):
        ShardedAnneal([Dummy(0, 5)], [[(0, 4)]], LocalComm())
