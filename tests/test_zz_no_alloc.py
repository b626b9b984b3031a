"""GPU test of sail_residue_noalloc, the one entry point that allocates nothing.

Every other entry point runs inside a device workspace its caller allocates.  Some callers
cannot do that: a plug-in inside a program whose allocator already owns the whole device
memory budget, or a service loop that must not pay for cudaMalloc / cudaFree.  For them
sail_residue_noalloc computes the residue chi2 (and the residuals) of given spectra with its
scratch in a fixed array inside the library.  Here its output is compared, on two calls in a
row with different sizes (so the second call runs on the array the first one filled), with
the residual recomputation a handle runs after sail_set_state, and with the FP64 oracle's
residual of the same spectra (an independent implementation of the kernel table and the
sums).  The device builds its table with its own exp, so the agreement is a relative 1e-10
rather than bit for bit.
"""
import ctypes

import numpy as np
import pytest

import paper_1609_07936_gb300 as sail
from paper_1609_07936_gb300 import _capi
from workloads import paper_scale_double_lorentz, tiny_double_lorentz

pytestmark = pytest.mark.gpu


def _noalloc(P, a):
    import torch
    dev = lambda x: torch.from_numpy(np.ascontiguousarray(x, dtype=np.float64)).cuda()
    tau, F, sig, om, da = dev(P.tau), dev(P.F), dev(P.sigma), dev(P.omega), dev(a)
    W = a.shape[0]
    chi2 = torch.empty(W, dtype=torch.float64, device="cuda")
    R = torch.empty((W, P.n_tau), dtype=torch.float64, device="cuda")
    st = torch.cuda.current_stream()
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    rc = sail.load().sail_residue_noalloc(p(tau), p(F), p(sig), P.n_tau, p(om), P.n_omega, p(da), W,
                                          p(chi2), p(R), ctypes.c_void_p(st.cuda_stream))
    assert rc == 0, sail.load().sail_last_error()
    st.synchronize()
    return chi2.cpu().numpy(), R.cpu().numpy()


def _reference(P, a):
    W = a.shape[0]
    g = sail.Sail(P.tau, P.F, P.sigma, P.omega,
                  sail.Params(n_walkers=W, precision=sail.PREC_FP64, n_sweeps=1, A=P.A, B=P.B))
    g.set_state(a)
    _, R, chi2, _, _ = g.state()
    g.close()
    return chi2, R


def test_noalloc_residue_matches_the_handle_recomputation():
    import torch
    assert torch.cuda.is_available()
    rng = np.random.default_rng(4)
    cases = [(paper_scale_double_lorentz(1e-4, n_walkers=48), 48),   # larger table first
             (tiny_double_lorentz(), 16)]                              # then a smaller one on the same array
    for P, W in cases:
        a = rng.uniform(0.0, 2.0 * P.A / P.n_omega, (W, P.n_omega))
        chi2, R = _noalloc(P, a)
        chi2_ref, R_ref = _reference(P, a)
        np.testing.assert_allclose(chi2, chi2_ref, rtol=1e-10)
        np.testing.assert_allclose(R, R_ref, rtol=1e-10, atol=1e-10 * np.abs(R_ref).max())
        import oracle as O
        K, Fh, _ = O.tables(P.tau, P.F, P.sigma, P.omega)
        for w in range(W):
            R_o, c2_o = O.residual(K, Fh, a[w])
            assert abs(chi2[w] - c2_o) <= 1e-10 * c2_o
            np.testing.assert_allclose(R[w], R_o, rtol=1e-10, atol=1e-10 * np.abs(R_o).max())


def test_noalloc_refuses_sizes_beyond_its_scratch():
    L = sail.load()
    one = ctypes.c_void_p(256)   # never dereferenced: the size check comes first
    rc = L.sail_residue_noalloc(one, one, one, 512, one, 2049, one, 1, one, None, None)
    assert rc == _capi.SAIL_EINVAL
    assert b"exceeds the fixed scratch" in L.sail_last_error()
