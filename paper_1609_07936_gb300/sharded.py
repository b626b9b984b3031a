"""One inversion's population of walkers split over several handles (shards), e.g. one per GPU.

Between branching events the walkers are independent (Sec. 2.2), so each shard anneals its own
contiguous range of the population; its random counters carry the walkers' population indices
(sail_params.walker_offset), so a shard draws exactly what the whole population would for
those walkers.  At every block end (Sec. 2.5):

  1. every shard's chi2 after the block's residual recomputation is gathered by every process;
  2. every process runs the same deterministic branching solve on the whole population's chi2
     (sail_branch_solve on one of its handles): multipliers, Delta, and the imprint pairs;
  3. the rows (spectrum, residual) of donors whose receivers live elsewhere are sent to the
     process that holds the receiver and land in that GPU's own memory;
  4. each shard imprints its receivers from those rows (sail_imprint_rows).

The result is the single-handle run's, bit for bit: the same draws, the same solve input, the
same imprint arithmetic.  This module only orders the steps and moves bytes; the arithmetic runs
in the library's kernels.  The geometric schedule is supported; the self-cooling schedule,
adaptive branching and smoothing need population statistics per block and are not.

Engines (duck-typed): offset, n_walkers, run_block(), chi2() -> float64 array,
rows(idx) -> (a_rows, R_rows), imprint(idx, a_rows, R_rows, t), solve(chi2_all, block, fraction)
-> (m, Delta, receivers, donors).  CudaShard is the library's; any object with these methods
(for instance a CPU model of the method) can be sharded the same way.
Communicators: LocalComm (all shards in one process) and TorchComm (torch.distributed, one or
more shards per rank; NCCL with CUDA tensors, gloo with CPU tensors).
"""
from __future__ import annotations

from typing import Dict, List, Sequence, Tuple

import numpy as np


class LocalComm:
    """Every shard of the population lives in this process."""

    rank, world = 0, 1

    def all_gather(self, local: np.ndarray, counts: Sequence[int]) -> List[np.ndarray]:
        return [np.asarray(local, dtype=np.float64)]

    def exchange(self, sends: Dict[int, object], recv_rows: Dict[int, int], width: int) -> Dict[int, object]:
        return {}


class TorchComm:
    """torch.distributed between processes: all_gather of chi2 and point-to-point rows."""

    def __init__(self, dist, device="cpu"):
        self.dist = dist
        self.device = device
        self.rank = dist.get_rank()
        self.world = dist.get_world_size()

    def all_gather(self, local: np.ndarray, counts: Sequence[int]) -> List[np.ndarray]:
        import torch
        n = max(counts)
        buf = torch.zeros(n, dtype=torch.float64, device=self.device)
        buf[: local.size] = torch.as_tensor(local, dtype=torch.float64, device=self.device)
        out = [torch.zeros(n, dtype=torch.float64, device=self.device) for _ in range(self.world)]
        self.dist.all_gather(out, buf)
        return [o[:c].cpu().numpy() for o, c in zip(out, counts)]

    def exchange(self, sends: Dict[int, object], recv_rows: Dict[int, int], width: int) -> Dict[int, object]:
        import torch
        ops, recvs = [], {}
        for src, k in sorted(recv_rows.items()):
            recvs[src] = torch.empty((k, width), dtype=torch.float64, device=self.device)
            ops.append(self.dist.P2POp(self.dist.irecv, recvs[src], src))
        for dst, t in sorted(sends.items()):
            ops.append(self.dist.P2POp(self.dist.isend, t.to(self.device).contiguous(), dst))
        if ops:
            for r in self.dist.batch_isend_irecv(ops):
                r.wait()
        return recvs


class CudaShard:
    """Walkers [offset, offset + n_walkers) of a population of n_total, on the current GPU."""

    def __init__(self, tau, F, sigma, omega, params, offset: int, n_walkers: int, n_total: int):
        import copy
        from ._capi import Sail
        p = copy.copy(params)
        p.n_walkers = int(n_walkers)
        p.branching = False
        p.walker_offset = int(offset)
        p.walker_total = int(n_total)
        self.offset, self.n_walkers = int(offset), int(n_walkers)
        self.handle = Sail(tau, F, sigma, omega, p)

    def run_block(self):
        self.handle.anneal(1)

    def chi2(self) -> np.ndarray:
        return self.handle.chi2()

    def rows(self, idx):
        return self.handle.walker_rows(idx)

    def imprint(self, idx, a_rows, R_rows, t: float):
        self.handle.imprint_rows(idx, a_rows, R_rows, t)

    def solve(self, chi2_all, block: int, fraction: float):
        return self.handle.branch_solve(chi2_all, block, fraction)

    def close(self):
        self.handle.close()


class ShardedAnneal:
    """Blocks of a population held by shards across processes.

    layout: for every process, in rank order, the (offset, n_walkers) of its shards; together
    they tile [0, n_total) in population order.  shards: this process's engines, in the order
    of its layout entry."""

    def __init__(self, shards: Sequence, layout: Sequence[Sequence[Tuple[int, int]]], comm,
                 branch_fraction: float = 0.25, imprint_t: float = 0.1):
        self.shards = list(shards)
        self.layout = [list(x) for x in layout]
        self.comm = comm
        self.fraction = float(branch_fraction)
        self.imprint_t = float(imprint_t)
        spans = sorted((o, n, r, k) for r, lst in enumerate(self.layout) for k, (o, n) in enumerate(lst))
        self.n_total = sum(n for _, n, _, _ in spans)
        pos = 0
        for o, n, _, _ in spans:
            if o != pos:
                raise ValueError("the shards must tile the population without gaps or overlaps")
            pos += n
        mine = self.layout[comm.rank]
        if [(s.offset, s.n_walkers) for s in self.shards] != [tuple(x) for x in mine]:
            raise ValueError("this process's shards do not match its layout entry")
        self.owner = np.empty(self.n_total, dtype=np.int64)      # process of every walker
        self.shard_of = np.empty(self.n_total, dtype=np.int64)   # shard index within its process
        for o, n, r, k in spans:
            self.owner[o:o + n] = r
            self.shard_of[o:o + n] = k
        self.counts = [sum(n for _, n in lst) for lst in self.layout]
        self.blocks = 0
        self.events: List[dict] = []

    def block(self) -> dict:
        for s in self.shards:
            s.run_block()
        # 1. the whole population's chi2, assembled in population order
        local = np.concatenate([s.chi2() for s in self.shards]) if self.shards else np.zeros(0)
        gathered = self.comm.all_gather(local, self.counts)
        chi2_all = np.empty(self.n_total)
        for r, vals in enumerate(gathered):
            q = 0
            for o, n in self.layout[r]:
                chi2_all[o:o + n] = vals[q:q + n]
                q += n
        # 2. the same solve on every process
        m, delta, zl, dl = self.shards[0].solve(chi2_all, self.blocks, self.fraction)
        # 3. donor rows: local ones read here, remote ones sent by their owners
        me = self.comm.rank
        t = self.imprint_t
        need_local = {}                   # donor -> rows, for receivers in this process
        sends: Dict[int, List[int]] = {}  # destination process -> donors it needs from here
        recvs: Dict[int, List[int]] = {}  # source process -> donors this process needs
        for l1, l2 in zip(zl.tolist(), dl.tolist()):
            r1, r2 = int(self.owner[l1]), int(self.owner[l2])
            if r2 == me and r1 != me:
                sends.setdefault(r1, [])
                if l2 not in sends[r1]:
                    sends[r1].append(l2)
            elif r1 == me and r2 != me:
                recvs.setdefault(r2, [])
                if l2 not in recvs[r2]:
                    recvs[r2].append(l2)
        for lst in list(sends.values()) + list(recvs.values()):
            lst.sort()

        def rows_of(donors):
            """Rows of donors held by this process's shards, in the order given."""
            out_a, out_R = [], []
            for k, s in enumerate(self.shards):
                sel = [l for l in donors if self.shard_of[l] == k and self.owner[l] == me]
                if sel:
                    a, R = s.rows(np.asarray(sel) - s.offset)
                    out_a.append((sel, a))
                    out_R.append((sel, R))
            rows = {}
            for (sel, a), (_, R) in zip(out_a, out_R):
                for q, l in enumerate(sel):
                    rows[l] = (a[q], R[q])
            return rows

        width = None
        send_t = {}
        if sends:
            import torch
            for dst, donors in sends.items():
                rows = rows_of(donors)
                send_t[dst] = torch.stack([torch.cat([rows[l][0], rows[l][1]]) for l in donors])
                width = send_t[dst].shape[1]
        local_donors = sorted({l2 for l1, l2 in zip(zl.tolist(), dl.tolist())
                               if self.owner[l1] == me and self.owner[l2] == me})
        need_local.update(rows_of(local_donors))
        if width is None:
            width = self._width()
        received = self.comm.exchange(send_t, {src: len(d) for src, d in recvs.items()}, width)
        n_omega = self._n_omega()
        for src, donors in recvs.items():
            block_rows = received[src]
            for q, l in enumerate(donors):
                need_local[l] = (block_rows[q, :n_omega], block_rows[q, n_omega:])
        # 4. imprint each shard's receivers (receivers are never donors: m = 0 vs m > 1)
        for k, s in enumerate(self.shards):
            pairs = [(l1, l2) for l1, l2 in zip(zl.tolist(), dl.tolist())
                     if self.owner[l1] == me and self.shard_of[l1] == k]
            if not pairs:
                continue
            import torch
            idx = np.asarray([l1 for l1, _ in pairs]) - s.offset
            a_rows = torch.stack([torch.as_tensor(need_local[l2][0]) for _, l2 in pairs])
            R_rows = torch.stack([torch.as_tensor(need_local[l2][1]) for _, l2 in pairs])
            s.imprint(idx, a_rows, R_rows, t)
        event = {"block": self.blocks, "m": m, "delta": delta, "receivers": zl, "donors": dl}
        self.events.append(event)
        self.blocks += 1
        return event

    def _n_omega(self) -> int:
        s = self.shards[0]
        return int(getattr(s, "n_omega", None) or s.handle.n_omega)

    def _width(self) -> int:
        s = self.shards[0]
        n_tau = int(getattr(s, "n_tau", None) or s.handle.n_tau)
        return self._n_omega() + n_tau
