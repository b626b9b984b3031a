"""Workload recipes: tau grid, omega bins, true spectrum, noisy F, sigma, A and B.

Every array is float64 and every random draw comes from
numpy.random.default_rng(seed), so the oracle and the CUDA path receive
bit-identical inputs.

Readings fixed here (the paper does not state them):
  * the true spectrum is cut to [0, W], the support of the histogram model
    (Sec. 2.1 sets S = 0 above w_max = N_w * dw; a Lorentzian's first moment
    diverges without the upper cut);
  * sigma_i = level * F_exact(tau_i) and F_i = F_exact(tau_i) + sigma_i * z_i
    with z_i independent standard normals (the random recipes hold sigma constant
    where F_exact falls below 1e-8 of its largest value, RANDOM_NOISE_FLOOR);
  * A = int_0^W S dw / dw and B = int_0^W w S dw / dw, the sum constants of
    Sec. 2.2 evaluated on the true spectrum;
  * omega is passed as the bin centres x_j = (j + 1/2) dw.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

from .spectra import Peak, first_moment, laplace, mass


@dataclass
class Problem:
    name: str
    tau: np.ndarray        # [n_tau] float64, >= 0
    F: np.ndarray          # [n_tau] noisy correlation data
    sigma: np.ndarray      # [n_tau] noise standard deviations
    omega: np.ndarray      # [n_omega] bin centres
    A: float
    B: float
    W: float               # upper edge of the frequency window
    peaks: List[Peak]
    F_exact: np.ndarray
    n_walkers: int = 64
    extra: dict = field(default_factory=dict)

    @property
    def n_tau(self) -> int:
        return int(self.tau.size)

    @property
    def n_omega(self) -> int:
        return int(self.omega.size)

    @property
    def d_omega(self) -> float:
        return self.W / self.n_omega


def make_problem(name: str, tau: np.ndarray, n_omega: int, W: float, peaks: List[Peak],
                 noise_level: float, seed: int, n_walkers: int, noise_floor: float = 0.0) -> Problem:
    """sigma_i = noise_level * max(F_exact(tau_i), noise_floor * max_k F_exact(tau_k))."""
    tau = np.asarray(tau, dtype=np.float64)
    omega = (np.arange(n_omega, dtype=np.float64) + 0.5) * (W / n_omega)
    F_exact = laplace(peaks, W, tau)
    sigma = noise_level * np.maximum(F_exact, noise_floor * F_exact.max())
    z = np.random.default_rng(seed).standard_normal(tau.size)
    F = F_exact + sigma * z
    dw = W / n_omega
    return Problem(name=name, tau=tau, F=F, sigma=sigma, omega=omega,
                   A=mass(peaks, W) / dw, B=first_moment(peaks, W) / dw, W=W,
                   peaks=list(peaks), F_exact=F_exact, n_walkers=n_walkers,
                   extra={"noise_level": noise_level, "seed": seed, "noise_floor": noise_floor})


def _double_lorentz() -> List[Peak]:
    return [Peak("lorentz", 2.0, 0.3, 0.6), Peak("lorentz", 5.0, 0.5, 0.4)]


def tiny_double_lorentz(seed: int = 0, n_walkers: int = 64) -> Problem:
    """32 tau points 4k/31 on [0, 4]; 64 bins on [0, 10]; two Lorentzians
    (centres 2.0 / 5.0, HWHM 0.3 / 0.5, weights 0.6 / 0.4); sigma = 1e-4 F."""
    tau = 4.0 * np.arange(32, dtype=np.float64) / 31.0
    return make_problem("tiny_double_lorentz", tau, 64, 10.0, _double_lorentz(), 1e-4, seed, n_walkers)


def paper_scale_double_lorentz(noise_level: float = 1e-4, seed: int = 0,
                               n_walkers: int = 4096, n_tau: int = 200,
                               n_omega: int = 1000) -> Problem:
    """200 tau points uniform on [0, 8] (end points included); 1000 bins on
    [0, 20]; the same double Lorentzian; relative noise 1e-3, 1e-4 or 1e-5."""
    tau = 8.0 * np.arange(n_tau, dtype=np.float64) / (n_tau - 1)
    return make_problem(f"paper_scale_double_lorentz_{noise_level:g}", tau, n_omega, 20.0,
                        _double_lorentz(), noise_level, seed, n_walkers)


def random_peaks(rng: np.random.Generator) -> List[Peak]:
    """1-4 peaks, each Lorentzian or Gaussian with probability 1/2, centres
    U[0.5, 15], widths U[0.05, 2], Dirichlet(1, ..., 1) weights."""
    k = int(rng.integers(1, 5))
    kinds = ["lorentz" if b else "gauss" for b in rng.random(k) < 0.5]
    centres = rng.uniform(0.5, 15.0, k)
    widths = rng.uniform(0.05, 2.0, k)
    weights = rng.dirichlet(np.ones(k))
    return [Peak(kd, float(c), float(w), float(a)) for kd, c, w, a in zip(kinds, centres, widths, weights)]


# Random peaks reach omega = 15 on tau in [0, 8], where F(8) / F(0) falls to 1e-40: a purely
# relative sigma would then weight the kernel's low-frequency columns by up to 1e43, past the
# range of an FP32 state.  The random recipes keep the noise relative down to 1e-8 of F's
# largest value and constant below it (reading of "noise sigma = level * F").
RANDOM_NOISE_FLOOR = 1e-8


def precision_random_peaks(seed: int = 0, n_tau: int = 512, n_omega: int = 2048,
                           n_walkers: int = 16384, noise_level: float = 1e-4) -> Problem:
    """512 tau points on [0, 8], 2048 bins on [0, 20], 1-4 random peaks."""
    rng = np.random.default_rng(seed)
    peaks = random_peaks(rng)
    tau = 8.0 * np.arange(n_tau, dtype=np.float64) / (n_tau - 1)
    return make_problem(f"precision_random_peaks_{seed}", tau, n_omega, 20.0, peaks,
                        noise_level, seed + 1, n_walkers, noise_floor=RANDOM_NOISE_FLOOR)


def random_batch_problem(index: int, seed: int = 0, rng: Optional[np.random.Generator] = None,
                         max_tau: int = 500, max_omega: int = 2000, max_walkers: int = 4096) -> Problem:
    """One inversion of the uneven batch: n_tau ~ U{50..500}, n_omega ~ U{200..2000},
    walkers ~ U{256..4096}, noise log-uniform on [1e-5, 1e-3].  The max_* arguments lower the
    upper ends of the three size ranges (same draws, same order)."""
    rng = rng or np.random.default_rng([seed, index])
    n_tau = int(rng.integers(50, max_tau + 1))
    n_omega = int(rng.integers(200, max_omega + 1))
    n_walkers = int(rng.integers(256, max_walkers + 1))
    level = float(10.0 ** rng.uniform(-5.0, -3.0))
    peaks = random_peaks(rng)
    tau = 8.0 * np.arange(n_tau, dtype=np.float64) / (n_tau - 1)
    return make_problem(f"batch_{seed}_{index}", tau, n_omega, 20.0, peaks, level,
                        int(rng.integers(0, 2**31)), n_walkers, noise_floor=RANDOM_NOISE_FLOOR)


def lorentzian_band_peaks() -> List[Peak]:
    """Eq. (lorentzian-band): two unit Lorentzians of HWHM 1 at 1 and 2, cut to [0.5, 2.5]."""
    return [Peak("lorentz", 1.0, 1.0, 1.0), Peak("lorentz", 2.0, 1.0, 1.0)]


LORENTZIAN_BAND = (0.5, 2.5)


def lorentzian_band(noise_level: float, seed: int = 0, n_walkers: int = 1500, n_tau: int = 160,
                    dtau: float = 0.05, n_omega: int = 1000, W: float = 3.5) -> Problem:
    """The paper's example (Sec. lorentzian-model): the band spectrum on 1000 bins of [0, 3.5]
    with correlated undersampling noise (Sec. resampling) of relative level noise_level at
    tau = 0; noise_level = 0 gives the exact data, weighted as if its noise were at 1e-8.
    Readings: the tau grid (unstated) is tau_i = i dtau, i < n_tau, and the sequences drawn
    for the noise have 2 n_tau points."""
    from .correlated import correlated_noise
    from .spectra import laplace as _laplace
    peaks = lorentzian_band_peaks()
    tau = dtau * np.arange(n_tau, dtype=np.float64)
    lags = dtau * np.arange(2 * n_tau, dtype=np.float64)
    F_lags = _laplace(peaks, W, lags, LORENTZIAN_BAND)
    F_exact = F_lags[:n_tau].copy()
    rng = np.random.default_rng(seed)
    F, sigma, M = correlated_noise(F_exact, F_lags, noise_level if noise_level > 0 else 1e-8, rng)
    if noise_level == 0:
        F = F_exact.copy()
    omega = (np.arange(n_omega, dtype=np.float64) + 0.5) * (W / n_omega)
    dw = W / n_omega
    return Problem(name=f"lorentzian_band_{noise_level:g}", tau=tau, F=F, sigma=sigma, omega=omega,
                   A=mass(peaks, W, LORENTZIAN_BAND) / dw, B=first_moment(peaks, W, LORENTZIAN_BAND) / dw,
                   W=W, peaks=peaks, F_exact=F_exact, n_walkers=n_walkers,
                   extra={"noise_level": noise_level, "seed": seed, "band": LORENTZIAN_BAND,
                          "sequences_equivalent": M})


def skew(a: np.ndarray, omega: np.ndarray, w_mid: float = 1.5) -> float:
    """The paper's skew of a histogram spectrum about w_mid (Sec. annealing results):
    |mass below - mass above| / total mass, the bin containing w_mid split at it."""
    a = np.asarray(a, dtype=np.float64)
    dw = omega[1] - omega[0]
    lo_edge = omega - 0.5 * dw
    frac_below = np.clip((w_mid - lo_edge) / dw, 0.0, 1.0)
    below = float(np.sum(a * frac_below))
    total = float(np.sum(a))
    return abs(below - (total - below)) / total
