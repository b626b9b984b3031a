"""ctypes binding of libsail (include/sail.h): argument marshalling only.

Every computation runs in the CUDA library; this module converts numpy
arrays to pointers, gets device memory and a stream from PyTorch, and turns
error codes into exceptions.  Importing it loads libsail.so and raises if the
library is missing or was built without a symbol the header declares.
"""
from __future__ import annotations

import ctypes
import math
import os
from dataclasses import dataclass, fields
from typing import List, Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsail.so")

SAIL_OK = 0
SAIL_NOT_CONVERGED = 1
SAIL_EINVAL = -1
SAIL_ENOMEM = -2
SAIL_ECUDA = -3
SAIL_ESTATE = -4
SAIL_ETIMEOUT = -5
RESYNC_FP32 = 0
RESYNC_TENSOR = 1
RESYNC_TENSOR_BF16 = 2
RESYNC_FP64 = 3
SCHEDULE_GEOMETRIC = 0
SCHEDULE_SELF_COOLING = 1
PREC_FP64 = 0
PREC_FP32 = 1

# Every entry point include/sail.h declares.
EXPORTS = [
    "sail_default_params", "sail_workspace_size", "sail_create", "sail_anneal", "sail_average",
    "sail_get_info", "sail_get_state", "sail_set_state", "sail_get_trace", "sail_delta_probe",
    "sail_philox", "sail_probe_read_bandwidth", "sail_probe_smem_bandwidth", "sail_residue_noalloc",
    "sail_batch_workspace_size", "sail_batch_create", "sail_batch_anneal", "sail_batch_handle",
    "sail_batch_tuning", "sail_batch_destroy", "sail_server_create", "sail_server_submit", "sail_server_step",
    "sail_server_result", "sail_server_destroy", "sail_destroy", "sail_last_error",
    "sail_server_start", "sail_server_poll", "sail_server_stop", "sail_server_request_info", "sail_server_trace",
    "sail_checkpoint_size", "sail_checkpoint", "sail_restore",
    "sail_branch_solve", "sail_walker_rows", "sail_imprint_rows",
]


class CParams(ctypes.Structure):
    _fields_ = [
        ("n_walkers", ctypes.c_int), ("precision", ctypes.c_int), ("n_sweeps", ctypes.c_int),
        ("sweeps_per_block", ctypes.c_int), ("resync_every", ctypes.c_int), ("branching", ctypes.c_int),
        ("T_start", ctypes.c_double), ("T_end", ctypes.c_double), ("T_end_abs", ctypes.c_double),
        ("branch_fraction", ctypes.c_double),
        ("imprint_t", ctypes.c_double), ("move_scale", ctypes.c_double), ("y_p", ctypes.c_double),
        ("y_m", ctypes.c_double), ("y_min", ctypes.c_double), ("A", ctypes.c_double), ("B", ctypes.c_double),
        ("avg_chi2_factor", ctypes.c_double), ("target_chi2", ctypes.c_double), ("seed", ctypes.c_uint64),
        ("trace", ctypes.c_int), ("timing", ctypes.c_int), ("resync_kind", ctypes.c_int),
        ("wait_test", ctypes.c_int), ("sweep_lanes", ctypes.c_int), ("schedule_kind", ctypes.c_int),
        ("adaptive_branching", ctypes.c_int), ("cool_begin", ctypes.c_double), ("freeze_begin", ctypes.c_double),
        ("smooth_s", ctypes.c_double), ("index_walk_len", ctypes.c_int), ("hastings", ctypes.c_int),
        ("walk_uniform", ctypes.c_double), ("shared_bins", ctypes.c_int), ("sweep_loop", ctypes.c_int),
        ("T_start_abs", ctypes.c_double), ("walker_offset", ctypes.c_int), ("walker_total", ctypes.c_int),
        ("fp64_accept", ctypes.c_int),
    ]


class CProblem(ctypes.Structure):
    _fields_ = [
        ("tau", ctypes.POINTER(ctypes.c_double)), ("F", ctypes.POINTER(ctypes.c_double)),
        ("sigma", ctypes.POINTER(ctypes.c_double)), ("n_tau", ctypes.c_int),
        ("omega", ctypes.POINTER(ctypes.c_double)), ("n_omega", ctypes.c_int), ("params", CParams),
    ]


class CRequestInfo(ctypes.Structure):
    _fields_ = [
        ("state", ctypes.c_int), ("converged", ctypes.c_int), ("sweeps", ctypes.c_int), ("n_used", ctypes.c_int),
        ("submit_step", ctypes.c_longlong), ("admit_step", ctypes.c_longlong), ("done_step", ctypes.c_longlong),
        ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double),
        ("chi2_of_mean", ctypes.c_double),
    ]


class CBlockStats(ctypes.Structure):
    _fields_ = [
        ("block", ctypes.c_int), ("sweep_end", ctypes.c_int), ("T", ctypes.c_double),
        ("chi2_min", ctypes.c_double), ("chi2_mean", ctypes.c_double), ("acceptance", ctypes.c_double),
        ("positivity_rejected", ctypes.c_double), ("branch_delta", ctypes.c_double),
        ("branch_zeros", ctypes.c_int), ("reserved", ctypes.c_int),
    ]


class CInfo(ctypes.Structure):
    _fields_ = [
        ("n_tau", ctypes.c_int), ("n_omega", ctypes.c_int), ("n_walkers", ctypes.c_int),
        ("n_tau_pad", ctypes.c_int), ("precision", ctypes.c_int), ("sweeps_done", ctypes.c_int),
        ("blocks_done", ctypes.c_int), ("n_sweeps", ctypes.c_int), ("chi2_0", ctypes.c_double),
        ("d_omega", ctypes.c_double), ("A", ctypes.c_double), ("B", ctypes.c_double),
        ("lambda0", ctypes.c_double), ("kernel_launches", ctypes.c_longlong),
        ("workspace_bytes", ctypes.c_size_t), ("sweep_ms", ctypes.c_double), ("resync_ms", ctypes.c_double),
        ("branch_ms", ctypes.c_double), ("sweep_launches", ctypes.c_longlong),
        ("resync_launches", ctypes.c_longlong), ("branch_launches", ctypes.c_longlong),
        ("moves", ctypes.c_longlong), ("sweep_lanes", ctypes.c_int), ("sweep_ahead", ctypes.c_int),
        ("fp64_rechecks", ctypes.c_longlong), ("fp64_flips", ctypes.c_longlong),
    ]


_lib = None
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_u64p = ctypes.POINTER(ctypes.c_uint64)


def load(path: str = LIB_PATH):
    """Loads libsail.so (building it first if the sources are newer) and types its entry points."""
    global _lib
    if _lib is not None:
        return _lib
    from . import build as _build
    if not _build.up_to_date():
        _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"libsail.so not found at {path}; build it with paper_1609_07936_gb300.build")
    L = ctypes.CDLL(path)
    missing = [n for n in EXPORTS if not hasattr(L, n)]
    if missing:
        raise RuntimeError(f"libsail.so lacks {missing}")
    vp = ctypes.c_void_p
    L.sail_default_params.argtypes = [ctypes.POINTER(CParams)]
    L.sail_default_params.restype = None
    L.sail_workspace_size.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(CParams), ctypes.POINTER(ctypes.c_size_t)]
    L.sail_create.argtypes = [ctypes.POINTER(vp), _dp, _dp, _dp, ctypes.c_int, _dp, ctypes.c_int,
                              ctypes.POINTER(CParams), vp, ctypes.c_size_t, vp]
    L.sail_anneal.argtypes = [vp, ctypes.c_int, ctypes.POINTER(CBlockStats), _ip]
    L.sail_average.argtypes = [vp, _dp, _dp, _ip, _dp]
    L.sail_get_info.argtypes = [vp, ctypes.POINTER(CInfo)]
    L.sail_get_state.argtypes = [vp, _dp, _dp, _dp, _ip, _u64p]
    L.sail_set_state.argtypes = [vp, _dp, _ip]
    L.sail_get_trace.argtypes = [vp, _ip, _ip, _dp, _ip]
    L.sail_branch_solve.argtypes = [vp, ctypes.c_int, _dp, ctypes.c_int, ctypes.c_double, _ip, _dp, _ip, _ip, _ip]
    L.sail_walker_rows.argtypes = [vp, ctypes.c_int, _ip, vp, vp]
    L.sail_imprint_rows.argtypes = [vp, ctypes.c_int, _ip, vp, vp, ctypes.c_double]
    L.sail_checkpoint_size.argtypes = [vp, ctypes.POINTER(ctypes.c_size_t)]
    L.sail_checkpoint.argtypes = [vp, vp, ctypes.c_size_t]
    L.sail_restore.argtypes = [vp, vp, ctypes.c_size_t]
    L.sail_delta_probe.argtypes = [vp, ctypes.c_int, _ip, _ip, _ip, _dp, _dp, _ip]
    L.sail_philox.argtypes = [ctypes.c_int, vp, ctypes.c_uint64, vp, vp]
    L.sail_probe_read_bandwidth.argtypes = [vp, ctypes.c_size_t, ctypes.c_int, vp, vp]
    L.sail_probe_smem_bandwidth.argtypes = [ctypes.c_int, vp, vp, ctypes.POINTER(ctypes.c_double)]
    L.sail_residue_noalloc.argtypes = [vp, vp, vp, ctypes.c_int, vp, ctypes.c_int, vp, ctypes.c_int, vp, vp, vp]
    L.sail_batch_workspace_size.argtypes = [ctypes.c_int, ctypes.POINTER(CProblem), ctypes.POINTER(ctypes.c_size_t)]
    L.sail_batch_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.POINTER(CProblem), ctypes.c_int, vp,
                                    ctypes.c_size_t, vp]
    L.sail_batch_anneal.argtypes = [vp, ctypes.c_int, _ip]
    L.sail_batch_handle.argtypes = [vp, ctypes.c_int, ctypes.POINTER(vp)]
    L.sail_batch_tuning.argtypes = [vp, _ip, _dp, ctypes.POINTER(ctypes.c_longlong)]
    L.sail_batch_destroy.argtypes = [vp]
    L.sail_server_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.c_longlong, ctypes.c_int, ctypes.c_int,
                                     vp, ctypes.c_size_t, vp]
    L.sail_server_submit.argtypes = [vp, ctypes.POINTER(CProblem), _ip]
    L.sail_server_step.argtypes = [vp, _ip, ctypes.c_int, _ip, _ip, _ip]
    L.sail_server_result.argtypes = [vp, ctypes.c_int, _dp, _dp, _dp, _ip, _ip]
    L.sail_server_destroy.argtypes = [vp]
    L.sail_server_start.argtypes = [vp]
    L.sail_server_poll.argtypes = [vp, _ip, ctypes.c_int, _ip, _ip, _ip]
    L.sail_server_stop.argtypes = [vp]
    L.sail_server_request_info.argtypes = [vp, ctypes.c_int, ctypes.POINTER(CRequestInfo)]
    L.sail_server_trace.argtypes = [vp, ctypes.c_int, _ip, _ip, _dp, _ip, _ip]
    L.sail_destroy.argtypes = [vp]
    L.sail_last_error.argtypes = []
    L.sail_last_error.restype = ctypes.c_char_p
    for n in EXPORTS:
        if n not in ("sail_default_params", "sail_last_error"):
            getattr(L, n).restype = ctypes.c_int
    _lib = L
    return L


class SailError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"sail error {code}: {msg}")
        self.code = code


def _check(rc: int) -> int:
    if rc < 0:
        raise SailError(rc, load().sail_last_error().decode())
    return rc


def _ptr(a: Optional[np.ndarray], t=_dp):
    return None if a is None else a.ctypes.data_as(t)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


@dataclass
class Params:
    """Mirror of sail_params; defaults are sail_default_params()."""
    n_walkers: int = 1024
    precision: int = PREC_FP32
    n_sweeps: int = 20000
    sweeps_per_block: int = 100
    resync_every: int = 50
    branching: bool = True
    T_start: float = 10.0
    T_end: float = 1e-9
    T_end_abs: float = 0.0
    branch_fraction: float = 0.25
    imprint_t: float = 0.1
    move_scale: float = 0.0
    y_p: float = 1.0
    y_m: float = 2.0
    y_min: float = 1e-4
    A: float = math.nan
    B: float = math.nan
    avg_chi2_factor: float = 1.5
    target_chi2: float = 0.0
    seed: int = 0
    trace: bool = False
    timing: bool = False
    resync_kind: int = 0
    wait_test: int = 0
    sweep_lanes: int = 0
    schedule_kind: int = 0
    adaptive_branching: bool = False
    cool_begin: float = 0.1
    freeze_begin: float = 0.5
    smooth_s: float = 0.0
    index_walk_len: int = 0
    walk_uniform: float = 0.0
    hastings: bool = False
    shared_bins: int = 0
    sweep_loop: int = 0
    T_start_abs: float = 0.0
    walker_offset: int = 0
    walker_total: int = 0
    fp64_accept: int = 0

    def c(self) -> CParams:
        p = CParams()
        for f in fields(self):
            v = getattr(self, f.name)
            setattr(p, f.name, int(v) if isinstance(v, bool) else v)
        return p

    @staticmethod
    def library_defaults() -> "Params":
        cp = CParams()
        load().sail_default_params(ctypes.byref(cp))
        out = Params()
        for f in fields(out):
            v = getattr(cp, f.name)
            setattr(out, f.name, bool(v) if isinstance(getattr(out, f.name), bool) else v)
        return out


def workspace_size(n_tau: int, n_omega: int, params: Params) -> int:
    out = ctypes.c_size_t(0)
    _check(load().sail_workspace_size(n_tau, n_omega, ctypes.byref(params.c()), ctypes.byref(out)))
    return int(out.value)


class Sail:
    """One inversion on the current CUDA device; PyTorch supplies the workspace and stream."""

    def __init__(self, tau, F, sigma, omega, params: Params, stream=None, device=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("Sail needs a CUDA device")
        self.params = params
        self.lib = load()
        tau, F, sigma, omega = map(_f64, (tau, F, sigma, omega))
        self.n_tau, self.n_omega = tau.size, omega.size
        self.n_walkers = params.n_walkers
        nbytes = workspace_size(self.n_tau, self.n_omega, params)
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self._h = ctypes.c_void_p()
        cp = params.c()
        _check(self.lib.sail_create(ctypes.byref(self._h), _ptr(tau), _ptr(F), _ptr(sigma), self.n_tau,
                                    _ptr(omega), self.n_omega, ctypes.byref(cp),
                                    ctypes.c_void_p(self.workspace.data_ptr()), nbytes,
                                    ctypes.c_void_p(self.stream.cuda_stream)))

    @classmethod
    def _view(cls, handle, n_tau, n_omega, params: "Params", owner):
        """A handle owned by a batch: usable for queries, never destroyed here."""
        self = cls.__new__(cls)
        self.params = params
        self.lib = load()
        self.n_tau, self.n_omega, self.n_walkers = n_tau, n_omega, params.n_walkers
        self._h = handle
        self._owner = owner
        self.last_status = 0
        return self

    def close(self):
        if self._h and getattr(self, "_owner", None) is None:
            self.lib.sail_destroy(self._h)
        self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self) -> dict:
        ci = CInfo()
        _check(self.lib.sail_get_info(self._h, ctypes.byref(ci)))
        return {f[0]: getattr(ci, f[0]) for f in CInfo._fields_}

    def anneal(self, max_blocks: int = 1 << 30) -> List[dict]:
        """Runs up to max_blocks blocks; returns one stats dict per block run."""
        nb = max(0, min(max_blocks, self.params.n_sweeps // max(1, self.params.sweeps_per_block) + 1))
        stats = (CBlockStats * max(nb, 1))()
        done = ctypes.c_int(0)
        self.last_status = _check(self.lib.sail_anneal(self._h, nb, stats, ctypes.byref(done)))
        return [{f[0]: getattr(stats[b], f[0]) for f in CBlockStats._fields_ if f[0] != "reserved"}
                for b in range(done.value)]

    def average(self):
        """(mean, stderr, n_used, chi2 of the mean spectrum)."""
        mean = np.zeros(self.n_omega)
        err = np.zeros(self.n_omega)
        used = ctypes.c_int(0)
        c2 = ctypes.c_double(0)
        _check(self.lib.sail_average(self._h, _ptr(mean), _ptr(err), ctypes.byref(used), ctypes.byref(c2)))
        return mean, err, used.value, c2.value

    def state(self):
        """(a [W, N_omega], R [W, N_tau], chi2 [W], acc_prev [W], hash [W])."""
        W = self.n_walkers
        a = np.zeros((W, self.n_omega))
        R = np.zeros((W, self.n_tau))
        chi2 = np.zeros(W)
        acc = np.zeros(W, dtype=np.int32)
        h = np.zeros(W, dtype=np.uint64)
        _check(self.lib.sail_get_state(self._h, _ptr(a), _ptr(R), _ptr(chi2), _ptr(acc, _ip), _ptr(h, _u64p)))
        return a, R, chi2, acc, h

    def chi2(self) -> np.ndarray:
        """chi2 of every walker [W]."""
        chi2 = np.zeros(self.n_walkers)
        _check(self.lib.sail_get_state(self._h, None, None, _ptr(chi2), None, None))
        return chi2

    def set_state(self, a, acc_prev=None):
        a = _f64(a)
        acc = None if acc_prev is None else np.ascontiguousarray(acc_prev, dtype=np.int32)
        _check(self.lib.sail_set_state(self._h, _ptr(a), _ptr(acc, _ip)))

    def trace(self):
        """(accepted [sweeps, W], multipliers [events, W], Delta [events])."""
        inf = self.info()
        W = self.n_walkers
        acc = np.zeros((max(inf["sweeps_done"], 1), W), dtype=np.int32)
        n_ev_max = self.params.n_sweeps // max(1, self.params.sweeps_per_block) + 1
        m = np.zeros((n_ev_max, W), dtype=np.int32)
        d = np.zeros(n_ev_max)
        ne = ctypes.c_int(0)
        _check(self.lib.sail_get_trace(self._h, _ptr(acc, _ip), _ptr(m, _ip), _ptr(d), ctypes.byref(ne)))
        return acc[: inf["sweeps_done"]], m[: ne.value], d[: ne.value]

    def branch_solve(self, chi2_all, block: int, fraction: float):
        """The branching solve over a whole population's chi2 (sail_branch_solve):
        (multipliers, Delta, receivers, donors) with population indices."""
        c = _f64(chi2_all)
        n = c.size
        m = np.zeros(n, dtype=np.int32)
        zl = np.zeros(n, dtype=np.int32)
        dl = np.zeros(n, dtype=np.int32)
        delta, npairs = ctypes.c_double(0), ctypes.c_int(0)
        _check(self.lib.sail_branch_solve(self._h, n, _ptr(c), int(block), float(fraction), _ptr(m, _ip),
                                          ctypes.byref(delta), _ptr(zl, _ip), _ptr(dl, _ip), ctypes.byref(npairs)))
        return m, delta.value, zl[: npairs.value].copy(), dl[: npairs.value].copy()

    def walker_rows(self, idx):
        """Spectra and residuals of this handle's walkers idx, as FP64 device tensors."""
        import torch
        idx = np.ascontiguousarray(idx, dtype=np.int32)
        a = torch.empty((idx.size, self.n_omega), dtype=torch.float64, device="cuda")
        R = torch.empty((idx.size, self.n_tau), dtype=torch.float64, device="cuda")
        if idx.size:
            _check(self.lib.sail_walker_rows(self._h, idx.size, _ptr(idx, _ip), ctypes.c_void_p(a.data_ptr()),
                                             ctypes.c_void_p(R.data_ptr())))
        return a, R

    def imprint_rows(self, idx, a_rows, R_rows, t: float) -> None:
        """Imprints this handle's walkers idx with donor rows held on this GPU (FP64 tensors)."""
        idx = np.ascontiguousarray(idx, dtype=np.int32)
        if idx.size:
            a_rows, R_rows = a_rows.contiguous(), R_rows.contiguous()
            _check(self.lib.sail_imprint_rows(self._h, idx.size, _ptr(idx, _ip), ctypes.c_void_p(a_rows.data_ptr()),
                                              ctypes.c_void_p(R_rows.data_ptr()), float(t)))

    def checkpoint(self) -> bytes:
        """Everything the rest of the schedule depends on, as bytes (sail_checkpoint)."""
        n = ctypes.c_size_t(0)
        _check(self.lib.sail_checkpoint_size(self._h, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(n.value)
        _check(self.lib.sail_checkpoint(self._h, buf, n.value))
        return buf.raw

    def restore(self, blob: bytes) -> None:
        """Loads a checkpoint of a handle created from the same data and parameters."""
        buf = ctypes.create_string_buffer(blob, len(blob))
        _check(self.lib.sail_restore(self._h, buf, len(blob)))

    def probe(self, walker, p, s, eps):
        """Delta chi2 of proposals on the current state: (delta [n], ok [n])."""
        walker = np.ascontiguousarray(walker, dtype=np.int32)
        p = np.ascontiguousarray(p, dtype=np.int32)
        s = np.ascontiguousarray(s, dtype=np.int32)
        eps = _f64(eps)
        n = walker.size
        delta = np.zeros(n)
        ok = np.zeros(n, dtype=np.int32)
        _check(self.lib.sail_delta_probe(self._h, n, _ptr(walker, _ip), _ptr(p, _ip), _ptr(s, _ip), _ptr(eps),
                                         _ptr(delta), _ptr(ok, _ip)))
        return delta, ok.astype(bool)


class Batch:
    """Many independent inversions annealed together (one persistent sweep launch per segment)."""

    def __init__(self, problems, autotune: bool = True, stream=None):
        """problems: list of (tau, F, sigma, omega, Params); all FP32, same block and resync periods."""
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("Batch needs a CUDA device")
        self.lib = load()
        self._arrays = []
        cp = (CProblem * len(problems))()
        self.shapes = []
        for k, (tau, F, sigma, omega, prm) in enumerate(problems):
            arrs = [_f64(x) for x in (tau, F, sigma, omega)]
            self._arrays.append(arrs)
            cp[k].tau, cp[k].F, cp[k].sigma = (_ptr(a) for a in arrs[:3])
            cp[k].n_tau = arrs[0].size
            cp[k].omega = _ptr(arrs[3])
            cp[k].n_omega = arrs[3].size
            cp[k].params = prm.c()
            self.shapes.append((arrs[0].size, arrs[3].size, prm))
        nbytes = ctypes.c_size_t(0)
        _check(self.lib.sail_batch_workspace_size(len(problems), cp, ctypes.byref(nbytes)))
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.workspace = torch.empty(nbytes.value, dtype=torch.uint8, device="cuda")
        self._b = ctypes.c_void_p()
        _check(self.lib.sail_batch_create(ctypes.byref(self._b), len(problems), cp, int(autotune),
                                          ctypes.c_void_p(self.workspace.data_ptr()), nbytes.value,
                                          ctypes.c_void_p(self.stream.cuda_stream)))
        self.handles = []
        for k, (nt, no, prm) in enumerate(self.shapes):
            h = ctypes.c_void_p()
            _check(self.lib.sail_batch_handle(self._b, k, ctypes.byref(h)))
            self.handles.append(Sail._view(h, nt, no, prm, self))

    def anneal(self, max_blocks: int = 1 << 30) -> int:
        done = ctypes.c_int(0)
        _check(self.lib.sail_batch_anneal(self._b, int(max_blocks), ctypes.byref(done)))
        return done.value

    def tuning(self):
        ip = ctypes.c_int(0)
        ns = ctypes.c_double(0.0)
        nl = ctypes.c_longlong(0)
        _check(self.lib.sail_batch_tuning(self._b, ctypes.byref(ip), ctypes.byref(ns), ctypes.byref(nl)))
        return {"item_pairs": ip.value, "ns_per_move": ns.value, "sweep_launches": nl.value}

    def close(self):
        if self._b:
            for h in self.handles:
                h._h = ctypes.c_void_p()
            self.lib.sail_batch_destroy(self._b)
            self._b = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous batching of inversion requests on one device buffer of workspace_bytes."""

    def __init__(self, workspace_bytes: int, max_resident: int = 512, max_walkers: int = 1 << 21,
                 sweeps_per_block: int = 100, resync_every: int = 50, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("Server needs a CUDA device")
        self.lib = load()
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.workspace = torch.empty(int(workspace_bytes), dtype=torch.uint8, device="cuda")
        self._s = ctypes.c_void_p()
        _check(self.lib.sail_server_create(ctypes.byref(self._s), int(max_resident), int(max_walkers),
                                           int(sweeps_per_block), int(resync_every),
                                           ctypes.c_void_p(self.workspace.data_ptr()), int(workspace_bytes),
                                           ctypes.c_void_p(self.stream.cuda_stream)))
        self.n_omega = {}
        self.max_resident = max_resident

    def submit(self, tau, F, sigma, omega, params: "Params") -> int:
        arrs = [_f64(x) for x in (tau, F, sigma, omega)]
        cp = CProblem()
        cp.tau, cp.F, cp.sigma = (_ptr(a) for a in arrs[:3])
        cp.n_tau = arrs[0].size
        cp.omega = _ptr(arrs[3])
        cp.n_omega = arrs[3].size
        cp.params = params.c()
        rid = ctypes.c_int(-1)
        _check(self.lib.sail_server_submit(self._s, ctypes.byref(cp), ctypes.byref(rid)))
        self.n_omega[rid.value] = arrs[3].size
        return rid.value

    def step(self):
        """One admission / block / retirement round: (completed ids, active, queued)."""
        buf = (ctypes.c_int * self.max_resident)()
        nc, na, nq = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
        _check(self.lib.sail_server_step(self._s, buf, self.max_resident, ctypes.byref(nc), ctypes.byref(na),
                                         ctypes.byref(nq)))
        return [buf[i] for i in range(min(nc.value, self.max_resident))], na.value, nq.value

    def start(self):
        """Hands the steps to the server's worker thread (poll() then reports completions)."""
        _check(self.lib.sail_server_start(self._s))

    def stop(self):
        _check(self.lib.sail_server_stop(self._s))

    def poll(self):
        """Ids the worker retired since the last poll: (completed ids, active, queued)."""
        buf = (ctypes.c_int * self.max_resident)()
        nc, na, nq = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
        out = []
        while True:
            _check(self.lib.sail_server_poll(self._s, buf, self.max_resident, ctypes.byref(nc), ctypes.byref(na),
                                             ctypes.byref(nq)))
            out += [buf[i] for i in range(nc.value)]
            if nc.value < self.max_resident:
                return out, na.value, nq.value

    def request_info(self, rid: int) -> dict:
        ci = CRequestInfo()
        _check(self.lib.sail_server_request_info(self._s, int(rid), ctypes.byref(ci)))
        return {f[0]: getattr(ci, f[0]) for f in CRequestInfo._fields_}

    def trace(self, rid: int, n_walkers: int):
        """(accepted counts [sweeps, walkers], multipliers [events, walkers], Deltas) of a
        completed request created with trace=True."""
        ns, ne = ctypes.c_int(0), ctypes.c_int(0)
        _check(self.lib.sail_server_trace(self._s, int(rid), None, None, None, ctypes.byref(ns), ctypes.byref(ne)))
        acc = np.zeros((ns.value, n_walkers), dtype=np.int32)
        m = np.zeros((ne.value, n_walkers), dtype=np.int32)
        d = np.zeros(ne.value)
        _check(self.lib.sail_server_trace(self._s, int(rid), _ptr(acc, _ip), _ptr(m, _ip), _ptr(d), None, None))
        return acc, m, d

    def result(self, rid: int):
        n = self.n_omega[rid]
        mean, err = np.zeros(n), np.zeros(n)
        c2, conv, sw = ctypes.c_double(0), ctypes.c_int(0), ctypes.c_int(0)
        _check(self.lib.sail_server_result(self._s, int(rid), _ptr(mean), _ptr(err), ctypes.byref(c2),
                                           ctypes.byref(conv), ctypes.byref(sw)))
        return {"mean": mean, "err": err, "chi2_of_mean": c2.value, "converged": bool(conv.value),
                "sweeps": sw.value}

    def close(self):
        if self._s:
            self.lib.sail_server_destroy(self._s)
            self._s = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def read_bandwidth_probe(buf, reps: int, stream=None) -> None:
    """Launches the read-bandwidth probe over a CUDA tensor (timed by the caller)."""
    import torch
    st = stream if stream is not None else torch.cuda.current_stream()
    sink = torch.zeros(8, dtype=torch.uint8, device=buf.device)
    nbytes = buf.numel() * buf.element_size() // 16 * 16
    _check(load().sail_probe_read_bandwidth(ctypes.c_void_p(buf.data_ptr()), nbytes, int(reps),
                                            ctypes.c_void_p(sink.data_ptr()), ctypes.c_void_p(st.cuda_stream)))


def smem_bandwidth_probe(reps: int, stream=None) -> float:
    """Launches the shared-memory read probe; returns the bytes it reads (timed by the caller)."""
    import torch
    st = stream if stream is not None else torch.cuda.current_stream()
    sink = torch.zeros(8, dtype=torch.uint8, device="cuda")
    nbytes = ctypes.c_double(0.0)
    _check(load().sail_probe_smem_bandwidth(int(reps), ctypes.c_void_p(sink.data_ptr()),
                                            ctypes.c_void_p(st.cuda_stream), ctypes.byref(nbytes)))
    return nbytes.value


def philox(ctr: np.ndarray, seed: int):
    """Device Philox4x32-10 of counters ctr [n, 4] (uint32) under a 64-bit key."""
    import torch
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    n = ctr.shape[0]
    dc = torch.from_numpy(ctr.view(np.int32)).cuda()
    do = torch.empty_like(dc)
    st = torch.cuda.current_stream()
    _check(load().sail_philox(n, ctypes.c_void_p(dc.data_ptr()), ctypes.c_uint64(seed),
                              ctypes.c_void_p(do.data_ptr()), ctypes.c_void_p(st.cuda_stream)))
    st.synchronize()
    return do.cpu().numpy().view(np.uint32)
