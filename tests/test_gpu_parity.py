"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the same inputs.

FP64 validation path: the same decision for every move (per-sweep accepted counts and an
FNV hash of every move's outcome per walker), and the same final spectra, residuals and
chi2, on the tiny double-Lorentzian workload (32 tau points, 64 bins, 64 walkers, 1000
sweeps, T 1 -> 1e-4), with and without branching.

FP32 production path: Delta chi2 of proposals evaluated on states the oracle produced
within 1e-5 of S = sum_i (|eps M_i| + |delta_p Khat_ip| + |delta_s Khat_is|)(2|R_i| + |d_i|),
the magnitude of the products the move adds (a forward-error bound of the computation is
a small multiple of the unit roundoff times S); sum rules, positivity and chi2 bookkeeping
at the paper-scale size; the ensemble average within twice its statistical error.
"""
import ctypes
import os
import subprocess
import tempfile

import numpy as np
import pytest

import oracle as O
import paper_1609_07936_gb300 as sail
from workloads import Peak, make_problem, paper_scale_double_lorentz, tiny_double_lorentz

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    sail.load()
    yield


def _pair(P, n_walkers, precision, **kw):
    """Oracle and GPU handle on the same problem and schedule."""
    sched = O.Schedule(**kw)
    params = sail.Params(n_walkers=n_walkers, precision=precision, n_sweeps=sched.n_sweeps,
                         sweeps_per_block=sched.sweeps_per_block, resync_every=sched.resync_every,
                         branching=sched.branching, T_start=sched.T_start, T_end=sched.T_end,
                         branch_fraction=sched.branch_fraction, imprint_t=sched.imprint_t,
                         move_scale=sched.move_scale, y_p=sched.y_p, y_m=sched.y_m, y_min=sched.y_min,
                         A=P.A, B=P.B, seed=sched.seed, trace=True)
    an = O.Anneal(P.tau, P.F, P.sigma, P.omega, P.A, P.B, n_walkers, sched)
    g = sail.Sail(P.tau, P.F, P.sigma, P.omega, params)
    return an, g


# ------------------------------------------------------------------ set-up and RNG

def test_start_state_and_tables_match():
    P = tiny_double_lorentz()
    an, g = _pair(P, 8, sail.PREC_FP64, n_sweeps=10)
    inf = g.info()
    assert inf["chi2_0"] == an.chi2_0
    assert inf["lambda0"] == an.lam
    assert abs(inf["d_omega"] - an.dw) == 0
    a, R, chi2, acc, h = g.state()
    np.testing.assert_array_equal(a, an.a)
    np.testing.assert_array_equal(R, an.R)
    np.testing.assert_array_equal(chi2, an.chi2)


def test_device_philox_matches_oracle_and_curand_header():
    rng = np.random.default_rng(0)
    ctr = rng.integers(0, 2 ** 32, (4096, 4), dtype=np.uint64).astype(np.uint32)
    ctr[:4] = [[0, 0, 0, 0], [1, 0, 0, 0], [0xFFFFFFFF] * 4, [7, 3, 5, 1]]
    seed = 0x0123456789ABCDEF
    ours = sail.philox(ctr, seed)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    want = np.array([O.philox4x32_10(c, key) for c in ctr[:512]])
    np.testing.assert_array_equal(ours[:512], want)
    # an independent implementation: the cuRAND device header, compiled here
    with tempfile.TemporaryDirectory() as td:
        so = os.path.join(td, "ref.so")
        subprocess.check_call(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-shared",
                               "-Xcompiler", "-fPIC", "-o", so, os.path.join(ROOT, "tests", "cuda", "curand_philox_ref.cu")])
        ref = ctypes.CDLL(so)
        import torch
        dc = torch.from_numpy(ctr.view(np.int32)).cuda()
        do = torch.empty_like(dc)
        torch.cuda.synchronize()
        rc = ref.curand_philox_ref(ctypes.c_int(ctr.shape[0]), ctypes.c_void_p(dc.data_ptr()),
                                   ctypes.c_uint64(seed), ctypes.c_void_p(do.data_ptr()))
        assert rc == 0
        theirs = do.cpu().numpy().view(np.uint32)
    np.testing.assert_array_equal(ours, theirs)


# ------------------------------------------------------------------ FP64 validation path

@pytest.mark.parametrize("branching", [False, True])
def test_fp64_path_reproduces_every_decision(branching):
    """Tiny double-Lorentzian workload: 64 walkers, 1000 sweeps, T 1 -> 1e-4 (units of chi2_0)."""
    P = tiny_double_lorentz()
    an, g = _pair(P, 64, sail.PREC_FP64, n_sweeps=1000, sweeps_per_block=100, resync_every=50,
                  branching=branching, T_start=1.0, T_end=1e-4, seed=0)
    acc_o, m_o, d_o = an.run(trace=True)
    stats = g.anneal()
    assert len(stats) == 10
    acc_g, m_g, d_g = g.trace()
    np.testing.assert_array_equal(acc_g, acc_o)
    a, R, chi2, accp, h = g.state()
    np.testing.assert_array_equal(h, an.hash)
    if branching:
        np.testing.assert_array_equal(m_g, m_o)
        np.testing.assert_array_equal(d_g, d_o)
        assert all(s["branch_zeros"] == 16 for s in stats)
    np.testing.assert_array_equal(a, an.a)
    np.testing.assert_array_equal(R, an.R)
    np.testing.assert_array_equal(chi2, an.chi2)
    mean, err, used, c2 = g.average()
    mo, eo, uo, c2o = an.average()
    assert used == uo
    np.testing.assert_array_equal(mean, mo)
    np.testing.assert_array_equal(err, eo)
    assert c2 == c2o


def test_fp64_path_ragged_sizes_and_partial_block():
    """n_tau spanning several 32-wide chunks with a ragged tail, n_omega not a multiple of 32,
    a schedule that ends mid-block and a resync period that does not divide the block."""
    tau = 0.05 * np.arange(77, dtype=np.float64)
    P = make_problem("ragged", tau, 45, 6.0, [Peak("gauss", 2.0, 0.6, 0.7), Peak("lorentz", 4.0, 0.4, 0.3)],
                     1e-3, 5, 24)
    an, g = _pair(P, 24, sail.PREC_FP64, n_sweeps=130, sweeps_per_block=40, resync_every=15,
                  branching=True, T_start=3.0, T_end=1e-3, seed=77)
    acc_o, m_o, _ = an.run(trace=True)
    g.anneal()
    acc_g, m_g, _ = g.trace()
    np.testing.assert_array_equal(acc_g, acc_o)
    np.testing.assert_array_equal(m_g, m_o)
    a, R, chi2, _, h = g.state()
    np.testing.assert_array_equal(h, an.hash)
    np.testing.assert_array_equal(a, an.a)
    np.testing.assert_array_equal(chi2, an.chi2)


def test_fp64_path_at_the_maximum_tau_count():
    """512 tau points (the library's maximum: 16 chunks of 32 per lane), a bin count that is not
    a multiple of 32, branching every 3 sweeps and a recomputation every 2: every decision,
    multiplier and final state bit-identical to the oracle."""
    tau = 8.0 * np.arange(512, dtype=np.float64) / 511
    P = make_problem("max_tau", tau, 45, 10.0, [Peak("lorentz", 2.0, 0.3, 0.6), Peak("gauss", 5.0, 0.5, 0.4)],
                     1e-4, 9, 8)
    an, g = _pair(P, 8, sail.PREC_FP64, n_sweeps=7, sweeps_per_block=3, resync_every=2,
                  branching=True, T_start=1.0, T_end=1e-2, seed=19)
    acc_o, m_o, d_o = an.run(trace=True)
    g.anneal()
    acc_g, m_g, d_g = g.trace()
    np.testing.assert_array_equal(acc_g, acc_o)
    np.testing.assert_array_equal(m_g, m_o)
    np.testing.assert_array_equal(d_g, d_o)
    assert acc_o.sum() > 0 and (acc_o < P.n_omega).any()
    a, R, chi2, _, h = g.state()
    np.testing.assert_array_equal(h, an.hash)
    np.testing.assert_array_equal(a, an.a)
    np.testing.assert_array_equal(R, an.R)
    np.testing.assert_array_equal(chi2, an.chi2)
    g.close()


def test_single_walker_and_edge_cases():
    """One walker (no branching possible) and a two-bin model (every move a no-op)."""
    P = tiny_double_lorentz()
    an, g = _pair(P, 1, sail.PREC_FP64, n_sweeps=50, sweeps_per_block=10, resync_every=10,
                  branching=True, seed=3)
    an.run()
    g.anneal()
    a, R, chi2, _, h = g.state()
    np.testing.assert_array_equal(h, an.hash)
    np.testing.assert_array_equal(a, an.a)
    tau = np.array([0.0, 0.5, 1.0])
    om = np.array([0.5, 1.5])
    for prec, T in ((sail.PREC_FP64, 1e-12), (sail.PREC_FP32, 1e12)):
        # FP64: every Delta chi2 is zero to rounding and passes even a tiny T; FP32 rounding
        # leaves Delta chi2 ~ 1e-3, so that path is run hot
        g2 = sail.Sail(tau, [0.2, 0.1, 0.05], [1e-3] * 3, om,
                       sail.Params(n_walkers=3, precision=prec, n_sweeps=20, sweeps_per_block=10,
                                   resync_every=10, A=2.0, B=1.3, T_start=T, T_end=T, trace=True))
        a0 = g2.state()[0]
        g2.anneal()
        acc, _, _ = g2.trace()
        assert np.all(acc == 2)
        np.testing.assert_allclose(g2.state()[0], a0, rtol=1e-6 if prec else 1e-13)


# ------------------------------------------------------------------ FP32 production path

def _oracle_states(P, n_walkers, sweeps, seed):
    an = O.Anneal(P.tau, P.F, P.sigma, P.omega, P.A, P.B, n_walkers,
                  O.Schedule(n_sweeps=2 * sweeps, sweeps_per_block=10 ** 6, resync_every=10 ** 6,
                             T_start=1.0, T_end=1e-6, seed=seed))
    an.run(sweeps)
    return an


@pytest.mark.parametrize("workload", ["tiny", "paper_scale"])
def test_fp32_delta_chi2_within_1e5(workload):
    if workload == "tiny":
        P = tiny_double_lorentz()
        W, sweeps = 32, 200
    else:
        P = paper_scale_double_lorentz(1e-4, n_walkers=16)
        W, sweeps = 16, 3
    an = _oracle_states(P, W, sweeps, seed=5)
    g = sail.Sail(P.tau, P.F, P.sigma, P.omega,
                  sail.Params(n_walkers=W, precision=sail.PREC_FP32, n_sweeps=10, A=P.A, B=P.B))
    g.set_state(an.a)
    a32 = g.state()[0]                     # the FP32 state the probe sees
    R32 = g.state()[1]
    rng = np.random.default_rng(9)
    n = 4000
    walker = rng.integers(0, W, n)
    p = rng.integers(0, P.n_omega, n)
    s = (p + rng.integers(1, P.n_omega, n)) % P.n_omega
    eps = rng.uniform(-1.0, 1.0, n) * 2.0 / P.n_omega
    delta, ok = g.probe(walker, p, s, eps)
    checked = 0
    for q in range(n):
        w = walker[q]
        good, D, ap, as_, d = O.propose(an.K, an.Fh, P.omega, P.A, P.B, a32[w], R32[w], p[q], s[q], eps[q])
        if good != ok[q]:
            # FP32 and FP64 disagree only when a bin lands within rounding of zero
            assert min(abs(ap), abs(as_)) <= 1e-5 * (abs(a32[w][p[q]]) + abs(a32[w][s[q]]) + 1e-30)
            continue
        if not good:
            continue
        x = P.omega
        dp = eps[q] * (P.B - P.A * x[s[q]]) / (x[p[q]] - x[s[q]])
        ds = eps[q] * (P.B - P.A * x[p[q]]) / (x[s[q]] - x[p[q]])
        M = an.Fh - R32[w]
        terms = np.abs(eps[q] * M) + np.abs(dp * an.K[:, p[q]]) + np.abs(ds * an.K[:, s[q]])
        scale = np.sum(terms * (2 * np.abs(R32[w]) + np.abs(d)))
        assert abs(delta[q] - D) <= 1e-5 * scale, (q, delta[q], D, scale)
        checked += 1
    assert checked > n // 4


def test_fp32_paper_scale_invariants():
    """200 tau points, 1000 bins, 4096 walkers, the bench launch configuration: after two
    blocks (200 sweeps, 4 resyncs, 2 branchings) the sum rules hold, a >= 0, and the
    chi2 and residuals the device keeps equal an FP64 recomputation from its spectra."""
    P = paper_scale_double_lorentz(1e-4)
    params = sail.Params(n_walkers=4096, precision=sail.PREC_FP32, n_sweeps=20000, sweeps_per_block=100,
                         resync_every=50, branching=True, T_start=10.0, T_end=1e-9, A=P.A, B=P.B, seed=1)
    g = sail.Sail(P.tau, P.F, P.sigma, P.omega, params)
    stats = g.anneal(2)
    assert len(stats) == 2 and all(s["branch_zeros"] == 1024 for s in stats)
    a, R, chi2, acc, h = g.state()
    assert np.all(a >= 0)
    # the block ends with a residual recomputation, which restores both sums
    np.testing.assert_allclose(a.sum(1), P.A, rtol=2e-6)
    np.testing.assert_allclose(a @ P.omega, P.B, rtol=2e-6)
    K, Fh, _ = O.tables(P.tau, P.F, P.sigma, P.omega)
    rng = np.random.default_rng(0)
    for w in rng.choice(4096, 24, replace=False):
        Rw, c2 = O.residual(K, Fh, a[w])
        assert abs(chi2[w] - c2) <= 1e-6 * c2 + 1e-3
        np.testing.assert_allclose(R[w], Rw, rtol=0, atol=1e-6 * np.abs(Rw).max() + 1e-3)


def test_fp32_ensemble_average_matches_oracle():
    """Independent walkers (no branching) on the tiny workload: the FP32 and FP64 ensemble
    means agree per bin within twice their combined standard error."""
    P = tiny_double_lorentz()
    W = 512
    kw = dict(n_sweeps=300, sweeps_per_block=100, resync_every=50, branching=False, T_start=1.0,
              T_end=1e-4, seed=11)
    an = O.Anneal(P.tau, P.F, P.sigma, P.omega, P.A, P.B, W, O.Schedule(**kw))
    an.run()
    params = sail.Params(n_walkers=W, precision=sail.PREC_FP32, A=P.A, B=P.B, avg_chi2_factor=1e300,
                         **{k: v for k, v in kw.items()})
    params.seed = 12345                      # an independent stream
    g = sail.Sail(P.tau, P.F, P.sigma, P.omega, params)
    g.anneal()
    mean_g, err_g, used_g, _ = g.average()
    mean_o, err_o, used_o = O.average(an.a, an.chi2, 1e300)
    assert used_g == used_o == W
    z = (mean_g - mean_o) / np.sqrt(err_g ** 2 + err_o ** 2)
    assert np.mean(np.abs(z) <= 2.0) >= 0.9, np.abs(z).max()
    assert np.abs(z).max() < 5.0
