"""GPU failure handling without faulting the GPU.

A bounded device wait that runs out: the tensor-core resync's test hook withholds the first
tile's commit, so no MMA is in flight and its mbarrier wait expires after 1024 polls; the block
records the time-out in the status word, frees its tensor memory and returns, and sail_anneal
reports SAIL_ETIMEOUT.  The CUDA context stays usable: a fresh handle anneals normally.
Invalid inputs are refused on the host before any device work.
"""
import numpy as np
import pytest

import paper_1609_07936_gb300 as sail
from paper_1609_07936_gb300 import _capi
from workloads import tiny_double_lorentz

pytestmark = pytest.mark.gpu


def _params(P, **kw):
    base = dict(n_walkers=64, precision=sail.PREC_FP32, n_sweeps=40, sweeps_per_block=20, resync_every=10,
                A=P.A, B=P.B, resync_kind=sail.RESYNC_TENSOR)
    base.update(kw)
    return sail.Params(**base)


def test_timed_out_wait_is_reported_and_context_survives():
    P = tiny_double_lorentz()
    g = sail.Sail(P.tau, P.F, P.sigma, P.omega, _params(P, wait_test=1))
    with pytest.raises(sail.SailError) as e:
        g.anneal(1)
    assert e.value.code == _capi.SAIL_ETIMEOUT
    g.close()
    h = sail.Sail(P.tau, P.F, P.sigma, P.omega, _params(P))
    stats = h.anneal()
    assert len(stats) == 2
    a = h.state()[0]
    np.testing.assert_allclose(a.sum(1), P.A, rtol=2e-6)
    h.close()


@pytest.mark.parametrize("bad", ["sigma", "grid", "ratio", "tau", "nan"])
def test_invalid_inputs_are_refused(bad):
    P = tiny_double_lorentz()
    tau, F, sig, om = P.tau.copy(), P.F.copy(), P.sigma.copy(), P.omega.copy()
    prm = _params(P)
    if bad == "sigma":
        sig[3] = 0.0
    elif bad == "grid":
        om[5] += 0.01
    elif bad == "ratio":
        prm.B = P.A * (P.omega[-1] + 1.0)
    elif bad == "tau":
        tau[2] = -1.0
    elif bad == "nan":
        F[4] = np.nan
    with pytest.raises(sail.SailError) as e:
        sail.Sail(tau, F, sig, om, prm)
    assert e.value.code == _capi.SAIL_EINVAL
