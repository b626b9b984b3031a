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
        # a resident request reports the sweeps it has run: one block of 20 per step since its
        # admission (steps are numbered from 1)
        for rid in ids:
            inf = server.request_info(rid)
            if inf["state"] == 1:
                assert inf["sweeps"] == 20 * (steps + 1 - inf["admit_step"] + 1)
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


def test_served_request_takes_the_oracle_decisions():
    """A served request (trace on) next to two others, against the FP64 oracle: over 6 sweeps
    at a fixed temperature at least 90% of its walkers accept exactly the oracle's number of
    moves in every sweep (Sec. 2.2; the FP32 sweep draws the oracle's Philox words)."""
    import oracle as O
    reqs = _requests()[:2]
    kw = dict(n_sweeps=6, sweeps_per_block=6, resync_every=3, branching=False, T_start=0.5, T_end=0.5)
    tau = 4.0 * np.arange(120, dtype=np.float64) / 119
    P = make_problem("served_oracle", tau, 90, 10.0, [Peak("lorentz", 2.0, 0.3, 0.6), Peak("gauss", 5.0, 0.7, 0.4)],
                     1e-4, 17, 96)
    prm = sail.Params(n_walkers=96, precision=sail.PREC_FP32, A=P.A, B=P.B, seed=71, trace=True,
                      resync_kind=sail.RESYNC_FP32, **kw)
    server = sail.Server(workspace_bytes=256 << 20, max_resident=4, max_walkers=1 << 16, sweeps_per_block=6,
                         resync_every=3)
    others = []
    for Q, q in reqs:
        q.sweeps_per_block, q.resync_every = 6, 3
        others.append(server.submit(Q.tau, Q.F, Q.sigma, Q.omega, q))
    rid = server.submit(P.tau, P.F, P.sigma, P.omega, prm)
    done = set()
    for _ in range(100):
        completed, active, queued = server.step()
        done.update(completed)
        if rid in done:
            break
    assert rid in done
    acc_g, _, _ = server.trace(rid, 96)
    an = O.Anneal(P.tau, P.F, P.sigma, P.omega, P.A, P.B, 96, O.Schedule(seed=71, **kw))
    acc_o, _, _ = an.run(trace=True)
    assert acc_g.shape == acc_o.shape
    same = np.all(acc_g == acc_o, axis=0)
    assert same.mean() >= 0.9, same.mean()
    assert acc_o.sum() > 0 and (acc_o < P.n_omega).any()
    server.close()


def test_worker_thread_admits_mid_block_arrivals_at_the_next_boundary():
    """The server's worker thread drives the blocks while this thread submits: a request
    submitted while a block runs is admitted by the next step (admit_step = submit_step + 1
    when a slot and memory are free), and every result equals its lone run bit for bit."""
    import time
    reqs = _requests()
    for _, prm in reqs:
        prm.n_sweeps = 200          # long enough that later submissions land mid-run
        prm.target_chi2 = 0.0
    server = sail.Server(workspace_bytes=1 << 30, max_resident=8, max_walkers=1 << 16, sweeps_per_block=20,
                         resync_every=10)
    server.start()
    ids = []
    P0, prm0 = reqs[0]
    ids.append(server.submit(P0.tau, P0.F, P0.sigma, P0.omega, prm0))
    # wait until the first request is resident and the worker has begun its second step
    for _ in range(2000):
        inf = server.request_info(ids[0])
        if inf["state"] == 1 and server.request_info(ids[0])["admit_step"] >= 1:
            break
        time.sleep(0.001)
    for P, prm in reqs[1:]:
        ids.append(server.submit(P.tau, P.F, P.sigma, P.omega, prm))
        time.sleep(0.002)
    done = set()
    t0 = time.time()
    while len(done) < len(ids):
        completed, _, _ = server.poll()
        done.update(completed)
        assert time.time() - t0 < 300
        time.sleep(0.005)
    server.stop()
    for k, rid in enumerate(ids):
        inf = server.request_info(rid)
        assert inf["state"] == 2 and inf["admit_step"] == inf["submit_step"] + 1, inf
        assert inf["t_submit"] <= inf["t_admit"] <= inf["t_done"]
    # at least one request arrived while another was resident (it joined a running server)
    assert max(server.request_info(r)["submit_step"] for r in ids) >= 1
    for k, (P, prm) in enumerate(reqs):
        r = server.result(ids[k])
        alone = sail.Sail(P.tau, P.F, P.sigma, P.omega, prm)
        alone.anneal()
        mean, err, used, c2 = alone.average()
        np.testing.assert_array_equal(r["mean"], mean)
        assert r["chi2_of_mean"] == c2 and r["sweeps"] == alone.info()["sweeps_done"]
        alone.close()
    server.close()
