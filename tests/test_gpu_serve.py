"""GPU: continuous batching of inversion requests.

Requests of different sizes arrive while others run; the server admits them in order as
slots and device memory free up (here a buffer that holds only a few at a time), keeps their
walkers on the device between blocks, and retires each one when its averaged spectrum
reaches its target chi2 or its schedule ends.  Each request's result must be the same,
bit for bit, as the same inversion annealed alone through a single handle.
"""
import numpy as np
import pytest

import paper_1609_07936_gb300 as sail
from workloads import Peak, make_problem

pytestmark = pytest.mark.gpu


def _requests():
    out = []
    for k in range(7):
        nt = [40, 64, 100, 33, 150, 80, 120][k]
        no = [128, 200, 300, 96, 400, 250, 180][k]
        nw = [128, 200, 64, 300, 96, 160, 222][k]
        tau = 5.0 * np.arange(nt, dtype=np.float64) / (nt - 1)
        peaks = [Peak("lorentz", 1.5 + 0.3 * k, 0.4, 0.7), Peak("gauss", 4.0, 0.6, 0.3)]
        P = make_problem(f"r{k}", tau, no, 10.0, peaks, 1e-4, 50 + k, nw)
        # even requests stop at their first block (any chi2 meets the target), odd ones run
        # their whole schedule (the target is never met)
        target = 1e300 if k % 2 == 0 else 1e-300
        prm = sail.Params(n_walkers=nw, precision=sail.PREC_FP32, n_sweeps=40 + 20 * (k % 3), sweeps_per_block=20,
                          resync_every=10, branching=True, T_start=3.0, T_end=1e-6, A=P.A, B=P.B, seed=900 + k,
                          target_chi2=target, resync_kind=sail.RESYNC_TENSOR)
        out.append((P, prm))
    return out


def test_served_results_equal_alone_runs():
    reqs = _requests()
    need = max(sail.workspace_size(P.n_tau, P.n_omega, prm) for P, prm in reqs)
    # a device buffer for about three requests at once: the rest wait in the queue
    server = sail.Server(workspace_bytes=3 * need + (8 << 20), max_resident=8, max_walkers=1 << 16,
                         sweeps_per_block=20, resync_every=10)
    ids, done, steps = [], {}, 0
    pending = list(range(len(reqs)))
    max_active = 0
    while pending or len(done) < len(reqs):
        # two arrivals per step while requests remain
        for _ in range(2):
            if pending:
                k = pending.pop(0)
                P, prm = reqs[k]
                ids.append(server.submit(P.tau, P.F, P.sigma, P.omega, prm))
        completed, active, queued = server.step()
        max_active = max(max_active, active)
        for rid in completed:
            done[rid] = server.result(rid)
        steps += 1
        assert steps < 200
    assert max_active <= 3
    for k, (P, prm) in enumerate(reqs):
        r = done[ids[k]]
        alone = sail.Sail(P.tau, P.F, P.sigma, P.omega, prm)
        alone.anneal()
        mean, err, used, c2 = alone.average()
        info = alone.info()
        np.testing.assert_array_equal(r["mean"], mean)
        np.testing.assert_array_equal(r["err"], err)
        assert r["chi2_of_mean"] == c2
        assert r["sweeps"] == info["sweeps_done"]
        assert r["converged"] == (k % 2 == 0)
        alone.close()
    server.close()
