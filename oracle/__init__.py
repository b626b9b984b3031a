"""FP64 CPU oracle for SAIL (arXiv:1609.07936): loader and Python front end.

TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check in __graft_entry__
and the CPU-baseline leg of bench.py may import this package.  The arithmetic
lives in sail_oracle.c (plain C, FP64, no contraction of products into fused
multiply-adds); this file only allocates numpy arrays and passes pointers.
It shares no code with the CUDA library and imports nothing from it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sail_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_u32p = ctypes.POINTER(ctypes.c_uint32)
_u64p = ctypes.POINTER(ctypes.c_uint64)
_i64p = ctypes.POINTER(ctypes.c_int64)


def build(force: bool = False) -> str:
    """Compile sail_oracle.c into liboracle.so next to it (gcc, FP64, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O3", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
                               "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class OrParams(ctypes.Structure):
    _fields_ = [
        ("n_sweeps", ctypes.c_int),
        ("sweeps_per_block", ctypes.c_int),
        ("resync_every", ctypes.c_int),
        ("branching", ctypes.c_int),
        ("T_start", ctypes.c_double),
        ("T_end", ctypes.c_double),
        ("branch_fraction", ctypes.c_double),
        ("imprint_t", ctypes.c_double),
        ("move_scale", ctypes.c_double),
        ("y_p", ctypes.c_double),
        ("y_m", ctypes.c_double),
        ("y_min", ctypes.c_double),
        ("seed", ctypes.c_uint64),
        ("schedule_kind", ctypes.c_int),
        ("adaptive", ctypes.c_int),
        ("cool_begin", ctypes.c_double),
        ("freeze_begin", ctypes.c_double),
        ("smooth_s", ctypes.c_double),
        ("walk_len", ctypes.c_int),
        ("walk_uniform", ctypes.c_double),
        ("hastings", ctypes.c_int),
        ("shared_bins", ctypes.c_int),
        ("walker_base", ctypes.c_int),
    ]


class OrState(ctypes.Structure):
    _fields_ = [
        ("T", ctypes.POINTER(ctypes.c_double)),
        ("T_final", ctypes.c_double),
        ("acc_ref", ctypes.c_double),
        ("T_freeze", ctypes.c_double),
        ("acc_before", ctypes.c_int64),
    ]


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        L.or_philox4x32_10.argtypes = [_u32p, _u32p, _u32p]
        L.or_tables.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp, _dp, _dp, _dp, _dp, _dp]
        L.or_tables.restype = ctypes.c_int
        L.or_residual.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp, _dp, _dp]
        L.or_residual.restype = ctypes.c_double
        L.or_initial_spectrum.argtypes = [ctypes.c_int, _dp, ctypes.c_double, ctypes.c_double, _dp, _dp]
        L.or_initial_spectrum.restype = ctypes.c_int
        L.or_propose.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp, _dp, ctypes.c_double,
                                 ctypes.c_double, _dp, _dp, ctypes.c_int, ctypes.c_int,
                                 ctypes.c_double, _dp, _dp, _dp, _dp]
        L.or_propose.restype = ctypes.c_int
        L.or_amplitude.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_double]
        L.or_amplitude.restype = ctypes.c_double
        L.or_multipliers_at.argtypes = [ctypes.c_int, _dp, _dp, ctypes.c_double, _ip, ctypes.c_void_p]
        L.or_multipliers_at.restype = ctypes.c_int
        L.or_branch_multipliers.argtypes = [ctypes.c_int, _dp, _dp, ctypes.c_double, _ip]
        L.or_branch_multipliers.restype = ctypes.c_double
        L.or_pairs.argtypes = [ctypes.c_int, _ip, _ip, _ip]
        L.or_pairs.restype = ctypes.c_int
        L.or_temperature.argtypes = [ctypes.POINTER(OrParams), ctypes.c_int, ctypes.c_double]
        L.or_temperature.restype = ctypes.c_double
        L.or_anneal.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp, _dp,
                                ctypes.c_double, ctypes.c_double, ctypes.POINTER(OrParams),
                                ctypes.POINTER(OrState), _dp, _dp, _dp, _ip, _u64p, _i64p, _i64p,
                                ctypes.c_int, ctypes.c_int, _ip, _ip, _dp]
        L.or_init_temperatures.argtypes = [ctypes.POINTER(OrParams), ctypes.c_double, _dp]
        L.or_init_temperatures.restype = None
        L.or_cooling_blocks.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, _ip, _ip]
        L.or_cooling_blocks.restype = None
        L.or_self_cooling.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_double, _dp]
        L.or_self_cooling.restype = ctypes.c_double
        L.or_adaptive_scale.argtypes = [ctypes.c_double, ctypes.c_double]
        L.or_adaptive_scale.restype = ctypes.c_double
        L.or_smooth.argtypes = [ctypes.c_int, _dp, ctypes.c_double, ctypes.c_double, _dp]
        L.or_smooth.restype = None
        L.or_move_bins.argtypes = [ctypes.POINTER(OrParams), ctypes.c_int, _dp, ctypes.c_uint32, ctypes.c_uint32,
                                   ctypes.c_int, ctypes.c_int, ctypes.c_int, _ip, _ip]
        L.or_move_bins.restype = None
        L.or_accept.argtypes = [ctypes.POINTER(OrParams), ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                ctypes.c_double, ctypes.c_double, ctypes.c_double]
        L.or_accept.restype = ctypes.c_int
        L.or_restore.argtypes = [ctypes.c_int, _dp, ctypes.c_double, ctypes.c_double, _dp]
        L.or_restore.restype = None
        L.or_anneal.restype = ctypes.c_int
        L.or_average.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp, ctypes.c_double, _dp, _dp]
        L.or_average.restype = ctypes.c_int
        L.or_imprint.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, _dp, _dp, _dp, _dp]
        L.or_imprint.restype = ctypes.c_double
        _lib = L
    return _lib


def _p(a: np.ndarray, t=_dp):
    return a.ctypes.data_as(t)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


# ---------------------------------------------------------------- primitives

def philox4x32_10(ctr, key) -> np.ndarray:
    """Philox4x32-10 of one 128-bit counter (4 words) under a 64-bit key (2 words)."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().or_philox4x32_10(_p(c, _u32p), _p(k, _u32p), _p(out, _u32p))
    return out


def tables(tau, F, sigma, omega):
    """Weighted kernel Khat [n_tau, n_omega], weighted data Fhat [n_tau] and bin width."""
    tau, F, sigma, omega = map(_f64, (tau, F, sigma, omega))
    n_tau, n_omega = tau.size, omega.size
    K = np.zeros((n_tau, n_omega))
    Fh = np.zeros(n_tau)
    dw = np.zeros(1)
    rc = lib().or_tables(n_tau, n_omega, _p(tau), _p(F), _p(sigma), _p(omega), _p(K), _p(Fh), _p(dw))
    if rc != 0:
        raise ValueError("invalid grid or data")
    return K, Fh, float(dw[0])


def residual(K, Fh, a):
    K, Fh, a = map(_f64, (K, Fh, a))
    R = np.zeros(K.shape[0])
    chi2 = lib().or_residual(K.shape[0], K.shape[1], _p(K), _p(Fh), _p(a), _p(R))
    return R, chi2


def initial_spectrum(omega, A, B):
    x = _f64(omega)
    a = np.zeros(x.size)
    lam = np.zeros(1)
    if lib().or_initial_spectrum(x.size, _p(x), float(A), float(B), _p(a), _p(lam)) != 0:
        raise ValueError("B/A outside the frequency window")
    return a, float(lam[0])


def propose(K, Fh, omega, A, B, a, R, p, s, eps):
    """One proposal on a given state: (ok, delta_chi2, a_p', a_s', d)."""
    K, Fh, x, a, R = map(_f64, (K, Fh, omega, a, R))
    d = np.zeros(K.shape[0])
    D, ap, as_ = np.zeros(1), np.zeros(1), np.zeros(1)
    ok = lib().or_propose(K.shape[0], K.shape[1], _p(K), _p(Fh), _p(x), float(A), float(B),
                          _p(a), _p(R), int(p), int(s), float(eps), _p(D), _p(ap), _p(as_), _p(d))
    return bool(ok), float(D[0]), float(ap[0]), float(as_[0]), d


def amplitude(accepted_prev, n_omega, y_p=1.0, y_m=2.0, y_min=1e-4):
    return lib().or_amplitude(int(accepted_prev), int(n_omega), y_p, y_m, y_min)


def multipliers_at(chi2_normalised, xi, Delta):
    z, xi = _f64(chi2_normalised), _f64(xi)
    m = np.zeros(z.size, dtype=np.int32)
    heap = (ctypes.c_byte * (16 * z.size))()
    Z = lib().or_multipliers_at(z.size, _p(z), _p(xi), float(Delta), _p(m, _ip), heap)
    return m, Z


def branch_multipliers(chi2, xi, fraction):
    chi2, xi = _f64(chi2), _f64(xi)
    m = np.zeros(chi2.size, dtype=np.int32)
    Delta = lib().or_branch_multipliers(chi2.size, _p(chi2), _p(xi), float(fraction), _p(m, _ip))
    return m, Delta


def pairs(m):
    m = np.ascontiguousarray(m, dtype=np.int32)
    zl = np.zeros(m.size, dtype=np.int32)
    dl = np.zeros(m.size, dtype=np.int32)
    n = lib().or_pairs(m.size, _p(m, _ip), _p(zl, _ip), _p(dl, _ip))
    return zl[:n], dl[:n]


def average(a, chi2, factor):
    a, chi2 = _f64(a), _f64(chi2)
    mean = np.zeros(a.shape[1])
    err = np.zeros(a.shape[1])
    used = lib().or_average(a.shape[0], a.shape[1], _p(a), _p(chi2), float(factor), _p(mean), _p(err))
    return mean, err, used


def imprint(t: float, a1, R1, a2, R2):
    """Walker 1 imprinted by walker 2 with strength t (Sec. 2.5): (a1', R1', chi2 of R1')."""
    a1, R1 = _f64(a1).copy(), _f64(R1).copy()
    a2, R2 = _f64(a2), _f64(R2)
    c2 = lib().or_imprint(a1.size, R1.size, float(t), _p(a1), _p(R1), _p(a2), _p(R2))
    return a1, R1, c2


def smooth(x, B: float, s: float, a) -> np.ndarray:
    """One spectrum smoothed by the three-point stencil of strength s and renormalised to
    the second sum rule B (Sec. smoothing)."""
    x = _f64(x)
    out = _f64(a).copy()
    lib().or_smooth(x.size, _p(x), float(B), float(s), _p(out))
    return out


def restore(x, A: float, B: float, a) -> np.ndarray:
    """A spectrum put back on both sum rules (the Hastings chain's projection)."""
    x = _f64(x)
    out = _f64(a).copy()
    lib().or_restore(x.size, _p(x), float(A), float(B), _p(out))
    return out


def accept(n_omega: int, yd: float, eps: float, D: float, T: float, u: float, hastings: bool = False) -> bool:
    """The acceptance decision of a move that passed the positivity test."""
    c = Schedule(hastings=hastings).c()
    return bool(lib().or_accept(ctypes.byref(c), int(n_omega), float(yd), float(eps), float(D), float(T), float(u)))


def cooling_blocks(n_blocks: int, cool_begin: float, freeze_begin: float):
    """First cooling block and first freeze-out block of a self-cooling schedule."""
    bc = np.zeros(1, dtype=np.int32)
    bf = np.zeros(1, dtype=np.int32)
    lib().or_cooling_blocks(int(n_blocks), float(cool_begin), float(freeze_begin), _p(bc, _ip), _p(bf, _ip))
    return int(bc[0]), int(bf[0])


def self_cooling(b: int, n_blocks: int, b_cool: int, b_freeze: int, cbar: float, cmin: float,
                 T_final: float, T_freeze: float = -1.0):
    """Temperature of block b >= 1 from the previous block's mean and smallest residues and
    the schedule's end temperature; returns (T, T_freeze after the call)."""
    tf = np.array([T_freeze], dtype=np.float64)
    T = lib().or_self_cooling(int(b), int(n_blocks), int(b_cool), int(b_freeze), float(cbar), float(cmin),
                              float(T_final), _p(tf))
    return T, float(tf[0])


def adaptive_scale(acc: float, acc_ref: float) -> float:
    """Factor on the branching fraction and imprint strength at acceptance acc."""
    return lib().or_adaptive_scale(float(acc), float(acc_ref))


def move_bins(a, w0: int, w1: int, mv: int, n: int, w: int, walk_len: int = 0, walk_uniform: float = 0.0,
              seed: int = 0):
    """Bins (p, s) of move mv of sweep n of walker w with spectrum a: the start words w0, w1
    and, for walk_len > 0, the index walk of Sec. 2.3."""
    a = _f64(a)
    sched = Schedule(walk_len=walk_len, walk_uniform=walk_uniform, seed=seed)
    c = sched.c()
    p = np.zeros(1, dtype=np.int32)
    s = np.zeros(1, dtype=np.int32)
    lib().or_move_bins(ctypes.byref(c), a.size, _p(a), int(w0), int(w1), int(mv), int(n), int(w), _p(p, _ip),
                       _p(s, _ip))
    return int(p[0]), int(s[0])


def xi_for_block(seed: int, block: int, n_walkers: int) -> np.ndarray:
    """The branching draws xi_l of one block, Philox counter (l, block, 0, 1)."""
    key = np.array([seed & 0xFFFFFFFF, seed >> 32], dtype=np.uint32)
    out = np.empty(n_walkers)
    for l in range(n_walkers):
        w = philox4x32_10([l, block, 0, 1], key)[0]
        out[l] = (float(w) + 0.5) * 2.0 ** -32
    return out


# ---------------------------------------------------------------- the anneal

@dataclass
class Schedule:
    n_sweeps: int = 1000
    sweeps_per_block: int = 100
    resync_every: int = 50
    branching: bool = False
    T_start: float = 1.0
    T_end: float = 1e-4
    branch_fraction: float = 0.25
    imprint_t: float = 0.1
    move_scale: float = 0.0      # 0 -> 1 / n_omega
    y_p: float = 1.0
    y_m: float = 2.0
    y_min: float = 1e-4
    seed: int = 0
    schedule_kind: int = 0       # 0 geometric, 1 self-cooling
    adaptive: bool = False       # acceptance-adaptive branching fraction and imprint strength
    cool_begin: float = 0.1
    freeze_begin: float = 0.5
    smooth_s: float = 0.0
    walk_len: int = 0            # steps of the index walk (Sec. 2.3)
    walk_uniform: float = 0.0    # probability an index skips its walk
    hastings: bool = False       # Metropolis-Hastings acceptance with the move's Jacobian
    shared_bins: int = 0         # W > 1: the walkers of each group of W propose the same bins
    walker_base: int = 0         # population index of walker 0 (a shard of a larger population)

    def c(self) -> OrParams:
        return OrParams(self.n_sweeps, self.sweeps_per_block, self.resync_every, int(self.branching),
                        self.T_start, self.T_end, self.branch_fraction, self.imprint_t,
                        self.move_scale, self.y_p, self.y_m, self.y_min, self.seed,
                        int(self.schedule_kind), int(self.adaptive), self.cool_begin, self.freeze_begin,
                        self.smooth_s, int(self.walk_len), self.walk_uniform, int(self.hastings),
                        int(self.shared_bins), int(self.walker_base))


class Anneal:
    """The whole method on one problem: tables, start state, sweeps, resyncs, branching."""

    def __init__(self, tau, F, sigma, omega, A, B, n_walkers: int, schedule: Schedule):
        self.K, self.Fh, self.dw = tables(tau, F, sigma, omega)
        self.x = _f64(omega)
        self.A, self.B = float(A), float(B)
        self.n_walkers = int(n_walkers)
        self.sched = schedule
        self._c = schedule.c()
        a0, self.lam = initial_spectrum(self.x, A, B)
        R0, self.chi2_0 = residual(self.K, self.Fh, a0)
        n_tau, n_omega = self.K.shape
        self.a = np.tile(a0, (n_walkers, 1))
        self.R = np.tile(R0, (n_walkers, 1))
        self.chi2 = np.full(n_walkers, self.chi2_0)
        self.acc_prev = np.full(n_walkers, n_omega, dtype=np.int32)
        self.hash = np.full(n_walkers, 0xCBF29CE484222325, dtype=np.uint64)
        self.n_acc = np.zeros(n_walkers, dtype=np.int64)
        self.n_pos = np.zeros(n_walkers, dtype=np.int64)
        self.sweep = 0
        # the temperature of every sweep (self-cooling fills each block's entries as it gets there)
        self.T = np.zeros(max(schedule.n_sweeps, 1))
        lib().or_init_temperatures(ctypes.byref(self._c), self.chi2_0, _p(self.T))
        self._st = OrState(_p(self.T), self.chi2_0 * schedule.T_end, -1.0, -1.0, 0)

    def temperature(self, n: int) -> float:
        return float(self.T[n])

    def run(self, n_sweeps: Optional[int] = None, trace: bool = False):
        """Advance n sweeps (default: to the end of the schedule).  With trace,
        returns (accepted counts [sweeps, walkers], multipliers [events, walkers], Deltas)."""
        end = self.sched.n_sweeps if n_sweeps is None else min(self.sweep + n_sweeps, self.sched.n_sweeps)
        n_run = end - self.sweep
        n_tau, n_omega = self.K.shape
        acc_tr = np.zeros((max(n_run, 1), self.n_walkers), dtype=np.int32)
        n_ev = n_run // self.sched.sweeps_per_block + 2
        m_tr = np.zeros((n_ev, self.n_walkers), dtype=np.int32)
        d_tr = np.zeros(n_ev)
        ev = lib().or_anneal(n_tau, n_omega, self.n_walkers, _p(self.K), _p(self.Fh), _p(self.x),
                             self.A, self.B, ctypes.byref(self._c), ctypes.byref(self._st),
                             _p(self.a), _p(self.R), _p(self.chi2), _p(self.acc_prev, _ip),
                             _p(self.hash, _u64p), _p(self.n_acc, _i64p), _p(self.n_pos, _i64p),
                             self.sweep, end,
                             _p(acc_tr, _ip) if trace else None,
                             _p(m_tr, _ip) if trace else None,
                             _p(d_tr) if trace else None)
        self.sweep = end
        if trace:
            return acc_tr[:n_run], m_tr[:ev], d_tr[:ev]
        return None

    def average(self, factor: float = 1.5):
        mean, err, used = average(self.a, self.chi2, factor)
        _, chi2_mean = residual(self.K, self.Fh, mean)
        return mean, err, used, chi2_mean
