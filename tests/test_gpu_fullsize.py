"""GPU: the precision configuration at its full size (512 tau x 2048 bins x 16384 walkers, FP32
moves, BF16 x6 tensor-core residual recomputation), in the launch configuration the benchmark
times, with the walkers' own bins and with bins shared by groups of 4.

After two blocks of 10 sweeps (a recomputation at each block end) every spectrum is
non-negative and on both sum rules, and for sampled walkers the residual and chi2 the device
keeps equal an FP64 recomputation from the spectrum (within the recomputation's error bound).
The acceptance counts of the last sweep are within [0, N_omega] and the run moved the walkers.
"""
import numpy as np
import pytest

import oracle as O
import paper_1609_07936_gb300 as sail
from workloads import precision_random_peaks

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("W", [0, 4])
def test_precision_configuration_full_size(W):
    P = precision_random_peaks(0)
    assert (P.n_tau, P.n_omega, P.n_walkers) == (512, 2048, 16384)
    prm = sail.Params(n_walkers=P.n_walkers, precision=sail.PREC_FP32, n_sweeps=20, sweeps_per_block=10,
                      resync_every=10, branching=True, T_start=10.0, T_end=1e-3, A=P.A, B=P.B, seed=7,
                      shared_bins=W, resync_kind=sail.RESYNC_TENSOR_BF16)
    g = sail.Sail(P.tau, P.F, P.sigma, P.omega, prm)
    chi2_0 = g.info()["chi2_0"]
    stats = g.anneal()
    assert len(stats) == 2
    a, R, chi2, acc, _ = g.state()
    assert np.all(a >= 0)
    np.testing.assert_allclose(a.sum(1), P.A, rtol=2e-6)
    np.testing.assert_allclose(a @ P.omega, P.B, rtol=2e-6)
    assert np.all((acc >= 0) & (acc <= P.n_omega)) and acc.mean() > 0
    assert chi2.min() < chi2_0
    K, Fh, _ = O.tables(P.tau, P.F, P.sigma, P.omega)
    rng = np.random.default_rng(1)
    for w in rng.choice(P.n_walkers, 16, replace=False):
        model = K @ a[w]
        R_ref = Fh - model
        tol = 2e-6 * model + 6e-8 * np.abs(R_ref) + 1e-6
        np.testing.assert_array_less(np.abs(R[w] - R_ref), tol + 1e-12)
        c2 = np.sum(R_ref ** 2)
        assert abs(chi2[w] - c2) <= 2 * np.sum(np.abs(R_ref) * tol) + 1e-9 * c2
    g.close()
