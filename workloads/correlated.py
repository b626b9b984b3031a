"""Correlation data with an undersampling noise profile (Sec. resampling of the paper's example).

The paper emulates Monte Carlo correlation data as follows: take the Gaussian process whose
autocorrelation is the exact F(tau) of the known spectrum, draw a limited number of its
sequences, and use their sample autocorrelation as the data.  Noise then grows with tau
relative to F and is correlated between the tau points; the number of sequences sets its
level.

F(tau) = (1/2pi) int S(w) e^{-w |tau|} dw with S >= 0 is a positive mixture of the
exponential (Ornstein-Uhlenbeck) covariances e^{-w |tau|}, so the Toeplitz matrix
F(|i - j| dtau) is a valid covariance.

  * `sequences` draws Gaussian sequences with that covariance (Cholesky factor).
  * `autocorrelation` is the sample autocorrelation of each sequence at lags 0..n-1, with the
    mean known to be zero: c_k = mean_i x_i x_{i+k}.
  * `undersampled` is the procedure itself: the mean of c over n_sequences sequences, with
    sigma from their spread.
  * `correlated_noise` serves noise levels that would need millions of sequences: by the
    central limit theorem the mean of M independent c's is Gaussian with covariance
    Sigma_1 / M, Sigma_1 the covariance of one sequence's c (estimated here from a few
    thousand sequences); M is chosen so that the relative noise at tau = 0 is the requested
    level.

This module builds problem inputs; it holds none of the inversion's arithmetic.
"""
from __future__ import annotations

import numpy as np
from scipy import linalg


def covariance(F_lags: np.ndarray) -> np.ndarray:
    """Toeplitz covariance Cov(x_i, x_j) = F(|i - j| dtau) of a sequence of len(F_lags)."""
    return linalg.toeplitz(np.asarray(F_lags, dtype=np.float64))


def sequences(F_lags: np.ndarray, n: int, rng: np.random.Generator) -> np.ndarray:
    """n Gaussian sequences [n, L] with zero mean and covariance F(|i - j| dtau)."""
    C = covariance(F_lags)
    # a relative jitter of 1e-12 keeps the factorisation of a positive semidefinite matrix
    # whose smallest eigenvalues sit at rounding level
    L = np.linalg.cholesky(C + 1e-12 * C[0, 0] * np.eye(C.shape[0]))
    return rng.standard_normal((n, C.shape[0])) @ L.T


def autocorrelation(x: np.ndarray, n_lags: int) -> np.ndarray:
    """Sample autocorrelation of each row at lags 0..n_lags-1: c_k = mean_i x_i x_{i+k}."""
    x = np.asarray(x, dtype=np.float64)
    L = x.shape[1]
    return np.stack([(x[:, :L - k] * x[:, k:]).mean(axis=1) for k in range(n_lags)], axis=1)


def undersampled(F_lags: np.ndarray, n_lags: int, n_sequences: int, rng: np.random.Generator, chunk: int = 4096):
    """The paper's procedure: (F_hat, sigma) from n_sequences sequences of length len(F_lags)."""
    total = np.zeros(n_lags)
    total2 = np.zeros(n_lags)
    left = n_sequences
    while left > 0:
        m = min(chunk, left)
        c = autocorrelation(sequences(F_lags, m, rng), n_lags)
        total += c.sum(axis=0)
        total2 += (c * c).sum(axis=0)
        left -= m
    mean = total / n_sequences
    var = (total2 - n_sequences * mean * mean) / max(n_sequences - 1, 1)
    return mean, np.sqrt(np.maximum(var, 0.0) / n_sequences)


def single_sequence_covariance(F_lags: np.ndarray, n_lags: int, rng: np.random.Generator,
                               n_sample: int = 8192) -> np.ndarray:
    """Covariance Sigma_1 [n_lags, n_lags] of one sequence's sample autocorrelation."""
    c = autocorrelation(sequences(F_lags, n_sample, rng), n_lags)
    return np.cov(c, rowvar=False)


def correlated_noise(F_exact: np.ndarray, F_lags: np.ndarray, level: float, rng: np.random.Generator,
                     n_sample: int = 8192):
    """(F, sigma) for the tau points of F_exact (the first len(F_exact) lags of F_lags) with
    the noise of the mean of M sequences' autocorrelations, M such that sigma_0 / F_0 = level."""
    n = F_exact.size
    S1 = single_sequence_covariance(F_lags, n, rng, n_sample)
    M = S1[0, 0] / (level * F_exact[0]) ** 2
    Sm = S1 / M
    w, V = np.linalg.eigh(Sm)
    noise = V @ (np.sqrt(np.maximum(w, 0.0)) * rng.standard_normal(n))
    sigma = np.sqrt(np.diag(Sm))
    return F_exact + noise, sigma, M
