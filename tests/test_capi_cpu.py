"""The C ABI without a GPU: the library loads, exports every declared entry point,
fills the paper's defaults and refuses bad arguments in its host-side checks."""
import ctypes
import json
import math
import os
import re

import pytest

import paper_1609_07936_gb300 as sail
from paper_1609_07936_gb300 import _capi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "sail.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sail_[a-z_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported():
    L = sail.load()
    names = _declared()
    assert len(names) >= 12
    for n in names:
        assert hasattr(L, n), n
    assert sorted(names) == sorted(_capi.EXPORTS)


def test_defaults_are_the_papers():
    gold = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_parameters.json")))
    p = sail.Params.library_defaults()
    for k in ("T_start", "sweeps_per_block", "branch_fraction", "imprint_t", "y_p", "y_m"):
        assert getattr(p, k) == gold[k]["value"], k
    assert math.isnan(p.A) and math.isnan(p.B)


def _c_layout(struct, fields):
    """sizeof and field offsets of a header struct, as the C compiler lays it out."""
    import subprocess
    import tempfile
    td = tempfile.mkdtemp()
    src = os.path.join(td, "layout.c")
    body = "".join(f'    printf("%zu\\n", offsetof({struct}, {f}));\n' for f in fields)
    open(src, "w").write('#include <stddef.h>\n#include <stdio.h>\n#include "sail.h"\n'
                         f'int main(void) {{\n    printf("%zu\\n", sizeof({struct}));\n{body}    return 0;\n}}\n')
    exe = os.path.join(td, "layout")
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), "-o", exe, src])
    out = [int(v) for v in subprocess.check_output([exe]).split()]
    return out[0], out[1:]


@pytest.mark.parametrize("struct,cls", [("sail_params", "CParams"), ("sail_block_stats", "CBlockStats"),
                                        ("sail_info", "CInfo"), ("sail_problem", "CProblem"),
                                        ("sail_request_info", "CRequestInfo")])
def test_struct_layouts_match_the_header(struct, cls):
    """Every ctypes mirror has the C compiler's size and field offsets."""
    C = getattr(_capi, cls)
    names = [f[0] for f in C._fields_]
    size, offs = _c_layout(struct, names)
    assert ctypes.sizeof(C) == size
    assert [getattr(C, n).offset for n in names] == offs


def test_workspace_size_and_refusals():
    p = sail.Params(n_walkers=4096, n_sweeps=20000)
    n = sail.workspace_size(200, 1000, p)
    # at least the FP32 spectra, residuals and both kernel tables
    assert n >= 4096 * 1000 * 4 + 4096 * 224 * 4 + 1000 * 224 * 12
    assert sail.workspace_size(200, 1000, sail.Params(n_walkers=4096, precision=sail.PREC_FP64)) > n
    with pytest.raises(sail.SailError) as e:
        sail.workspace_size(0, 1000, p)
    assert e.value.code == _capi.SAIL_EINVAL
    with pytest.raises(sail.SailError):
        sail.workspace_size(600, 1000, p)           # more than 512 tau points
    with pytest.raises(sail.SailError):
        sail.workspace_size(200, 1, p)              # one bin
    with pytest.raises(sail.SailError):
        sail.workspace_size(200, 1000, sail.Params(n_walkers=0))
    with pytest.raises(sail.SailError):
        sail.workspace_size(200, 1000, sail.Params(branch_fraction=1.0))
    with pytest.raises(sail.SailError):
        sail.workspace_size(200, 1000, sail.Params(T_start=-1.0))


def test_create_refuses_bad_inputs_before_touching_the_device():
    L = sail.load()
    import numpy as np
    tau = np.linspace(0, 1, 4)
    F = np.ones(4)
    sig = np.ones(4)
    om = (np.arange(8) + 0.5) * 0.5
    p = sail.Params(n_walkers=2, B=1.0, A=1.0).c()
    h = ctypes.c_void_p()
    dp = ctypes.POINTER(ctypes.c_double)
    ptr = lambda a: a.ctypes.data_as(dp)
    # NULL workspace
    rc = L.sail_create(ctypes.byref(h), ptr(tau), ptr(F), ptr(sig), 4, ptr(om), 8, ctypes.byref(p), None, 0, None)
    assert rc == _capi.SAIL_EINVAL
    # unaligned workspace pointer, refused before any copy
    rc = L.sail_create(ctypes.byref(h), ptr(tau), ptr(F), ptr(sig), 4, ptr(om), 8, ctypes.byref(p),
                       ctypes.c_void_p(16), 1 << 30, None)
    assert rc == _capi.SAIL_EINVAL and b"aligned" in L.sail_last_error()
    # too small
    rc = L.sail_create(ctypes.byref(h), ptr(tau), ptr(F), ptr(sig), 4, ptr(om), 8, ctypes.byref(p),
                       ctypes.c_void_p(256), 16, None)
    assert rc == _capi.SAIL_ENOMEM


def test_eight_lanes_need_a_uniform_tau_grid():
    """The 8-lane FP32 sweep forms its kernel columns along a uniform tau grid; asked for on an
    uneven grid, create refuses before touching the device."""
    L = sail.load()
    import numpy as np
    tau = np.array([0.0, 0.1, 0.3, 0.6])
    F = np.ones(4)
    sig = np.ones(4)
    om = (np.arange(8) + 0.5) * 0.5
    p = sail.Params(n_walkers=2, B=1.0, A=1.0, precision=sail.PREC_FP32, sweep_lanes=8).c()
    h = ctypes.c_void_p()
    dp = ctypes.POINTER(ctypes.c_double)
    ptr = lambda a: a.ctypes.data_as(dp)
    rc = L.sail_create(ctypes.byref(h), ptr(tau), ptr(F), ptr(sig), 4, ptr(om), 8, ctypes.byref(p),
                       ctypes.c_void_p(256), 1 << 40, None)
    assert rc == _capi.SAIL_EINVAL and b"uniform tau" in L.sail_last_error()
    # an evenly spaced but decreasing grid is not taken either
    down = np.array([0.6, 0.4, 0.2, 0.0])
    rc = L.sail_create(ctypes.byref(h), ptr(down), ptr(F), ptr(sig), 4, ptr(om), 8, ctypes.byref(p),
                       ctypes.c_void_p(256), 1 << 40, None)
    assert rc == _capi.SAIL_EINVAL and b"uniform tau" in L.sail_last_error()
