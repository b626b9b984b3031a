"""GPU: the FP32-state residual recomputations against the FP64 oracle.

All paths compute R = Fhat - Khat a and chi2 = sum R^2 for every walker: the FP32-FMA GEMM
with FP64 sums over 32-bin chunks (resync_kind 0), the tcgen05 tensor-core GEMM in TF32
with a three-term operand split and an FP32 tensor-memory accumulator (resync_kind 1), and
the same in BF16 with three pieces per operand and six products (resync_kind 2), and the
plain FP64-FMA GEMM (resync_kind 3, the comparison path).
The error bound per element is relative to the model value m_i = sum_j Khat_ij a_j (all
terms are positive): 2e-6 m_i covers the FP32 accumulation of ~1000 terms and the ~2^-21
operand precision of the split, plus the FP32 storage of R (6e-8 |R_i|).
"""
import numpy as np
import pytest

import oracle as O
import paper_1609_07936_gb300 as sail
from workloads import paper_scale_double_lorentz, precision_random_peaks, tiny_double_lorentz

pytestmark = pytest.mark.gpu


def _check(P, W, kind, seed, rel=2e-6):
    rng = np.random.default_rng(seed)
    K, Fh, _ = O.tables(P.tau, P.F, P.sigma, P.omega)
    a0, _ = O.initial_spectrum(P.omega, P.A, P.B)
    # start spectra perturbed per walker, some bins emptied
    a = a0[None, :] * rng.uniform(0.2, 1.8, (W, P.n_omega))
    a[rng.random((W, P.n_omega)) < 0.1] = 0.0
    g = sail.Sail(P.tau, P.F, P.sigma, P.omega,
                  sail.Params(n_walkers=W, precision=sail.PREC_FP32, n_sweeps=10, A=P.A, B=P.B,
                              resync_kind=kind))
    g.set_state(a)
    a32, R, chi2, _, _ = g.state()
    g.close()
    for w in range(W):
        model = K @ a32[w]
        R_ref = Fh - model
        tol = rel * model + 6e-8 * np.abs(R_ref) + 1e-6
        assert np.all(np.abs(R[w] - R_ref) <= tol), (w, np.max(np.abs(R[w] - R_ref) / tol))
        c2 = np.sum(R_ref ** 2)
        assert abs(chi2[w] - c2) <= 2 * np.sum(np.abs(R_ref) * tol) + 1e-9 * c2


@pytest.mark.parametrize("kind", [sail.RESYNC_FP32, sail.RESYNC_TENSOR, sail.RESYNC_TENSOR_BF16])
def test_resync_paper_scale(kind):
    """200 tau x 1000 bins, 300 walkers (two full 128-walker tiles and a ragged one)."""
    _check(paper_scale_double_lorentz(1e-4, n_walkers=300), 300, kind, 1)


@pytest.mark.parametrize("kind", [sail.RESYNC_FP32, sail.RESYNC_TENSOR, sail.RESYNC_TENSOR_BF16])
def test_resync_tiny_and_wide(kind):
    """32 tau x 64 bins (one MMA of N = 32), and 512 tau x 2048 bins (two MMAs of N = 256)."""
    _check(tiny_double_lorentz(), 70, kind, 2)
    _check(precision_random_peaks(3, n_walkers=130), 130, kind, 3)


def test_anneal_with_tensor_core_resync():
    """A short FP32 anneal whose resyncs and block ends run on the tensor cores keeps the
    sum rules and chi2 bookkeeping, like the FP32-FMA path."""
    P = paper_scale_double_lorentz(1e-4, n_walkers=512)
    out = {}
    for kind in (0, 1, 2):
        g = sail.Sail(P.tau, P.F, P.sigma, P.omega,
                      sail.Params(n_walkers=512, precision=sail.PREC_FP32, n_sweeps=2000, sweeps_per_block=20,
                                  resync_every=10, branching=True, T_start=10.0, T_end=1e-9, A=P.A, B=P.B,
                                  seed=4, resync_kind=kind))
        stats = g.anneal(2)
        a, R, chi2, _, _ = g.state()
        out[kind] = (stats, a, chi2)
        np.testing.assert_allclose(a.sum(1), P.A, rtol=2e-6)
        np.testing.assert_allclose(a @ P.omega, P.B, rtol=2e-6)
        K, Fh, _ = O.tables(P.tau, P.F, P.sigma, P.omega)
        for w in range(0, 512, 37):
            _, c2 = O.residual(K, Fh, a[w])
            assert abs(chi2[w] - c2) <= 1e-5 * c2
    # the two paths see the same statistics to within the rounding-driven divergence of chains
    assert abs(out[0][0][-1]["acceptance"] - out[1][0][-1]["acceptance"]) < 0.02
    assert abs(out[0][0][-1]["acceptance"] - out[2][0][-1]["acceptance"]) < 0.02


def test_fp64_resync_of_fp32_state():
    """resync_kind 3 multiplies and sums in FP64: only the FP32 storage of R and FP64 rounding
    (order of 1e-16 per term over 1000-2048 terms) remain, on the paper grid, the tiny grid and
    the 512 x 2048 grid with ragged walker counts."""
    _check(paper_scale_double_lorentz(1e-4, n_walkers=300), 300, 3, 1, rel=1e-12)
    _check(tiny_double_lorentz(), 70, 3, 2, rel=1e-12)
    _check(precision_random_peaks(3, n_walkers=130), 130, 3, 3, rel=1e-12)


def test_bf16x6_resync_at_full_size_on_sampled_walkers():
    """512 tau x 2048 bins x 16384 walkers, the precision workload's size and launch
    configuration (128-column tiles, 128 walker blocks): the residuals and chi2 of 65 sampled
    walkers (every 256th and the last) against the FP64 oracle, within the bound of the other
    cases."""
    P = precision_random_peaks(3, n_walkers=16384)
    W = 16384
    rng = np.random.default_rng(9)
    K, Fh, _ = O.tables(P.tau, P.F, P.sigma, P.omega)
    a0, _ = O.initial_spectrum(P.omega, P.A, P.B)
    a = a0[None, :] * rng.uniform(0.2, 1.8, (W, P.n_omega))
    a[rng.random((W, P.n_omega)) < 0.1] = 0.0
    g = sail.Sail(P.tau, P.F, P.sigma, P.omega,
                  sail.Params(n_walkers=W, precision=sail.PREC_FP32, n_sweeps=10, A=P.A, B=P.B,
                              resync_kind=sail.RESYNC_TENSOR_BF16))
    g.set_state(a)
    a32, R, chi2, _, _ = g.state()
    g.close()
    for w in list(range(0, W, 256)) + [W - 1]:
        model = K @ a32[w]
        R_ref = Fh - model
        tol = 2e-6 * model + 6e-8 * np.abs(R_ref) + 1e-6
        assert np.all(np.abs(R[w] - R_ref) <= tol), (w, np.max(np.abs(R[w] - R_ref) / tol))
        c2 = np.sum(R_ref ** 2)
        assert abs(chi2[w] - c2) <= 2 * np.sum(np.abs(R_ref) * tol) + 1e-9 * c2
