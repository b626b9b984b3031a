"""CPU: every parameter check of the C ABI refuses its bad value with SAIL_EINVAL and a message,
through the size queries, which touch no device (sail_workspace_size for one inversion,
sail_batch_workspace_size for a batch)."""
import ctypes
import math

import pytest

import paper_1609_07936_gb300 as sail
from paper_1609_07936_gb300 import _capi

BAD = [
    ("n_walkers", 0, "n_walkers"), ("precision", 7, "precision"), ("n_sweeps", 0, "n_sweeps"),
    ("sweeps_per_block", 0, "sweeps_per_block"), ("resync_every", 0, "resync_every"),
    ("T_start", 0.0, "temperatures"), ("T_end", math.inf, "temperatures"), ("T_end_abs", -1.0, "T_end_abs"),
    ("branch_fraction", 1.0, "branch_fraction"), ("imprint_t", 1.5, "imprint_t"),
    ("y_p", 0.0, "amplitude"), ("y_m", 0.5, "amplitude"), ("y_min", 0.0, "amplitude"),
    ("move_scale", 1.0, "move_scale"), ("avg_chi2_factor", 0.9, "avg_chi2_factor"),
    ("resync_kind", 4, "resync_kind"), ("T_start_abs", -1.0, "T_start_abs"), ("sweep_lanes", 4, "sweep_lanes"), ("schedule_kind", 2, "schedule_kind"),
    ("adaptive_branching", 2, "adaptive_branching"), ("cool_begin", math.nan, "cool_begin"),
    ("smooth_s", 0.5, "smooth_s"), ("index_walk_len", 8, "index_walk_len"), ("walk_uniform", 1.5, "walk_uniform"),
    ("hastings", 2, "hastings"), ("shared_bins", 3, "shared_bins"), ("sweep_loop", 3, "sweep_loop"),
    ("fp64_accept", 3, "fp64_accept"),
]


def _size(n_tau, n_omega, prm):
    L = sail.load()
    out = ctypes.c_size_t(0)
    rc = L.sail_workspace_size(n_tau, n_omega, ctypes.byref(prm.c()), ctypes.byref(out))
    return rc, L.sail_last_error().decode()


def test_defaults_are_accepted():
    rc, _ = _size(200, 1000, sail.Params(B=1.0))
    assert rc == _capi.SAIL_OK


@pytest.mark.parametrize("field,value,word", BAD)
def test_bad_value_is_refused(field, value, word):
    prm = sail.Params(B=1.0)
    setattr(prm, field, value)
    rc, msg = _size(200, 1000, prm)
    assert rc == _capi.SAIL_EINVAL and word in msg, (rc, msg)


@pytest.mark.parametrize("case", ["lanes8_wide", "hastings_walk", "shared_walk", "shared8_wide", "shared4_wide",
                                  "fp64_accept_fp64", "fp64_accept_walk", "fp64_accept_hastings", "fp64_accept_shared"])
def test_combinations_are_refused(case):
    prm = sail.Params(B=1.0)
    n_tau = 200
    if case == "lanes8_wide":
        prm.sweep_lanes, n_tau = 8, 300
    elif case == "hastings_walk":
        prm.hastings, prm.index_walk_len = True, 2
    elif case == "shared_walk":
        prm.shared_bins, prm.index_walk_len = 4, 2
    elif case == "shared8_wide":
        prm.shared_bins, n_tau = 8, 300
    elif case == "shared4_wide":
        prm.shared_bins, n_tau = 4, 513
    elif case.startswith("fp64_accept"):
        prm.fp64_accept = 1
        if case.endswith("fp64"):
            prm.precision = sail.PREC_FP64
        elif case.endswith("walk"):
            prm.index_walk_len = 2
        elif case.endswith("hastings"):
            prm.hastings = True
        else:
            prm.shared_bins = 4
    rc, msg = _size(n_tau, 1000, prm)
    assert rc == _capi.SAIL_EINVAL and msg, (rc, msg)


def test_null_params_and_output_are_refused():
    L = sail.load()
    out = ctypes.c_size_t(0)
    assert L.sail_workspace_size(200, 1000, None, ctypes.byref(out)) == _capi.SAIL_EINVAL
    assert b"params" in L.sail_last_error()
    assert L.sail_workspace_size(200, 1000, ctypes.byref(sail.Params(B=1.0).c()), None) == _capi.SAIL_EINVAL


def _batch_size(params_list, n_tau=100, n_omega=300):
    L = sail.load()
    probs = (_capi.CProblem * len(params_list))()
    for k, prm in enumerate(params_list):
        probs[k].n_tau, probs[k].n_omega = n_tau, n_omega
        probs[k].params = prm.c()
    out = ctypes.c_size_t(0)
    rc = L.sail_batch_workspace_size(len(params_list), probs, ctypes.byref(out))
    return rc, L.sail_last_error().decode(), out.value


def test_batch_checks():
    ok = sail.Params(n_walkers=256, B=1.0)
    rc, _, nbytes = _batch_size([ok, ok])
    assert rc == _capi.SAIL_OK and nbytes > 0
    rc, msg, _ = _batch_size([ok, sail.Params(n_walkers=256, B=1.0, precision=sail.PREC_FP64)])
    assert rc == _capi.SAIL_EINVAL and "FP32" in msg
    rc, msg, _ = _batch_size([ok, sail.Params(n_walkers=256, B=1.0, resync_every=25)])
    assert rc == _capi.SAIL_EINVAL and "match" in msg
    rc, msg, _ = _batch_size([ok, sail.Params(n_walkers=256, B=1.0, shared_bins=4)])
    assert rc == _capi.SAIL_EINVAL and "shared bins" in msg
    rc, msg, _ = _batch_size([ok, sail.Params(n_walkers=256, B=1.0, fp64_accept=1)])
    assert rc == _capi.SAIL_EINVAL and "fp64_accept" in msg
    rc, msg, _ = _batch_size([])
    assert rc == _capi.SAIL_EINVAL
