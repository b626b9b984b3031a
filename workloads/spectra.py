"""Closed forms for the synthetic spectra that feed the annealing inversion.

A synthetic spectrum is a weighted sum of peaks, each cut to the frequency
window [0, W] on which the histogram model of Eq. (spectral-model) lives:

    S(w) = sum_k c_k * P_k(w) * 1[0 <= w <= W]   (or 1[lo <= w <= hi], a band inside it)

with P_k a unit-mass Lorentzian (centre w0, half width at half maximum G,
as in Eq. (lorentzian-band)) or a unit-mass Gaussian (mean mu, standard
deviation s).  This module gives, in closed form and in float64,

  * the Laplace transform of Eq. (transform), F(tau) = (1/2pi) int_0^W S(w) e^{-w tau} dw,
  * the mass int_0^W S dw and first moment int_0^W w S dw, from which the
    sum constants of Sec. 2.2 follow as A = mass / dw and B = moment / dw,
  * the mass of S inside each histogram bin.

These are the inputs to the problem, not the method: nothing here knows the
histogram kernel, the residue or the annealing.  The tests pin every formula
against adaptive quadrature.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Sequence

import numpy as np
from scipy import special

TWO_PI = 2.0 * np.pi


@dataclass(frozen=True)
class Peak:
    kind: str      # "lorentz" or "gauss"
    centre: float  # w0 (Lorentzian) or mu (Gaussian)
    width: float   # G = HWHM (Lorentzian) or s = standard deviation (Gaussian)
    weight: float  # c_k, the mass the untruncated peak would carry

    def density(self, w):
        w = np.asarray(w, dtype=np.float64)
        if self.kind == "lorentz":
            return self.weight * (self.width / np.pi) / ((w - self.centre) ** 2 + self.width ** 2)
        if self.kind == "gauss":
            z = (w - self.centre) / self.width
            return self.weight * np.exp(-0.5 * z * z) / (self.width * np.sqrt(TWO_PI))
        raise ValueError(self.kind)


# ---------------------------------------------------------------- Lorentzian

def _lorentz_mass(p: Peak, W: float) -> float:
    return p.weight / np.pi * (np.arctan((W - p.centre) / p.width) + np.arctan(p.centre / p.width))


def _lorentz_moment(p: Peak, W: float) -> float:
    # int_0^W w L dw = w0 * mass + (G / 2pi) ln(((W-w0)^2+G^2) / (w0^2+G^2))
    g, c = p.width, p.centre
    log_term = np.log(((W - c) ** 2 + g * g) / (c * c + g * g))
    return c * _lorentz_mass(p, W) + p.weight * g / TWO_PI * log_term


def _lorentz_laplace(p: Peak, W: float, tau: np.ndarray) -> np.ndarray:
    """(1/2pi) int_0^W L(w) e^{-w tau} dw via the exponential integral.

    L(w) = (1/pi) Im[1/(w - c)] with c = w0 + iG.  Substituting u = w - c,
    int_0^W e^{-w tau}/(w - c) dw = e^{-c tau} [E1(-c tau) - E1((W - c) tau)];
    the path in u runs parallel to the real axis at Im u = -G, so it never
    crosses the principal branch cut of E1 on the negative real axis.
    At tau = 0 the integral is log(W - c) - log(-c).
    """
    c = complex(p.centre, p.width)
    out = np.empty(tau.shape, dtype=np.float64)
    zero = tau == 0.0
    if np.any(zero):
        val = np.log(W - c) - np.log(-c)
        out[zero] = val.imag / np.pi
    t = tau[~zero]
    if t.size:
        val = np.exp(-c * t) * (special.exp1(-c * t) - special.exp1((W - c) * t))
        out[~zero] = val.imag / np.pi
    return p.weight * out / TWO_PI


# ------------------------------------------------------------------ Gaussian

def _ndtr_diff(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Phi(b) - Phi(a) for a <= b, without cancellation in either tail."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    upper = a > 0  # both in the upper tail: use the complementary form
    out = special.ndtr(b) - special.ndtr(a)
    if np.any(upper):
        out = np.where(upper, special.ndtr(-a) - special.ndtr(-b), out)
    return out


def _gauss_mass(p: Peak, W: float) -> float:
    s, m = p.width, p.centre
    return p.weight * float(_ndtr_diff((0.0 - m) / s, (W - m) / s))


def _gauss_moment(p: Peak, W: float) -> float:
    s, m = p.width, p.centre
    edge = s / np.sqrt(TWO_PI) * (np.exp(-0.5 * (m / s) ** 2) - np.exp(-0.5 * ((W - m) / s) ** 2))
    return m * _gauss_mass(p, W) + p.weight * edge


def _gauss_laplace(p: Peak, W: float, tau: np.ndarray) -> np.ndarray:
    """(1/2pi) int_0^W G(w) e^{-w tau} dw by completing the square.

    -(w-mu)^2/2s^2 - w tau = -(w - mu')^2/2s^2 - mu tau + s^2 tau^2/2 with
    mu' = mu - s^2 tau, so the integral is e^{-mu tau + s^2 tau^2/2} times
    Phi((W-mu')/s) - Phi(-mu'/s).  When both limits sit in the upper tail the
    product is rewritten with the scaled complementary error function erfcx:
    e^{-mu tau + s^2 tau^2/2} * erfc(x/sqrt2)/2 = erfcx(x/sqrt2)/2 * e^{-x^2/2 - mu tau + s^2 tau^2/2},
    which stays finite for any tau.
    """
    s, m = p.width, p.centre
    tau = np.asarray(tau, dtype=np.float64)
    mu_p = m - s * s * tau
    a = (0.0 - mu_p) / s   # lower limit in standard units
    b = (W - mu_p) / s     # upper limit in standard units
    log_pref = -m * tau + 0.5 * (s * tau) ** 2
    out = np.empty(tau.shape, dtype=np.float64)
    tail = a > 0
    if np.any(~tail):
        out[~tail] = np.exp(log_pref[~tail]) * (special.ndtr(b[~tail]) - special.ndtr(a[~tail]))
    if np.any(tail):
        at, bt, lp = a[tail], b[tail], log_pref[tail]
        r2 = np.sqrt(2.0)
        term_a = 0.5 * special.erfcx(at / r2) * np.exp(lp - 0.5 * at * at)
        term_b = 0.5 * special.erfcx(bt / r2) * np.exp(lp - 0.5 * bt * bt)
        out[tail] = term_a - term_b
    return p.weight * out / TWO_PI


# ---------------------------------------------------------------- interface

# A spectrum may also be cut to a band [lo, hi] inside [0, W] (Eq. lorentzian-band); every
# quantity over the band is the one over [0, hi] minus the one over [0, lo].

def _band(W: float, band):
    lo, hi = (0.0, W) if band is None else (float(band[0]), float(band[1]))
    if not (0.0 <= lo < hi <= W):
        raise ValueError("band must satisfy 0 <= lo < hi <= W")
    return lo, hi


def mass(peaks: Sequence[Peak], W: float, band=None) -> float:
    """int S(w) dw over [0, W] (or over the band [lo, hi])."""
    lo, hi = _band(W, band)
    f = lambda p, x: (_lorentz_mass(p, x) if p.kind == "lorentz" else _gauss_mass(p, x)) if x > 0 else 0.0
    return float(sum(f(p, hi) - f(p, lo) for p in peaks))


def first_moment(peaks: Sequence[Peak], W: float, band=None) -> float:
    """int w S(w) dw over [0, W] (or over the band [lo, hi])."""
    lo, hi = _band(W, band)
    f = lambda p, x: (_lorentz_moment(p, x) if p.kind == "lorentz" else _gauss_moment(p, x)) if x > 0 else 0.0
    return float(sum(f(p, hi) - f(p, lo) for p in peaks))


def laplace(peaks: Sequence[Peak], W: float, tau, band=None) -> np.ndarray:
    """F(tau) = (1/2pi) int S(w) e^{-w tau} dw (Eq. transform) over [0, W] or the band."""
    lo, hi = _band(W, band)
    tau = np.atleast_1d(np.asarray(tau, dtype=np.float64))
    out = np.zeros(tau.shape, dtype=np.float64)
    for p in peaks:
        f = _lorentz_laplace if p.kind == "lorentz" else _gauss_laplace
        out += f(p, hi, tau)
        if lo > 0:
            out -= f(p, lo, tau)
    return out


def bin_masses(peaks: Sequence[Peak], W: float, n_omega: int, band=None) -> np.ndarray:
    """int over bin j of S(w) dw for the n_omega equal bins of [0, W] (S cut to the band)."""
    lo, hi = _band(W, band)
    edges = np.clip(np.linspace(0.0, W, n_omega + 1), lo, hi)
    cum = np.zeros(n_omega + 1)
    for p in peaks:
        if p.kind == "lorentz":
            cum += p.weight / np.pi * (np.arctan((edges - p.centre) / p.width) + np.arctan(p.centre / p.width))
        else:
            z = (edges - p.centre) / p.width
            cum += p.weight * (special.ndtr(z) - special.ndtr(-p.centre / p.width))
    return np.diff(cum)
