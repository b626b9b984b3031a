"""Pins for the synthetic input generator: closed forms against adaptive quadrature."""
import numpy as np
import pytest
from scipy import integrate

from workloads import (Peak, bin_masses, first_moment, laplace, mass, paper_scale_double_lorentz,
                       precision_random_peaks, random_batch_problem, tiny_double_lorentz)


def _quad(f, W, pts):
    v, _ = integrate.quad(f, 0.0, W, points=[p for p in pts if 0 < p < W], limit=500,
                          epsabs=0.0, epsrel=1e-13)
    return v


PEAK_SETS = [
    ([Peak("lorentz", 2.0, 0.3, 0.6), Peak("lorentz", 5.0, 0.5, 0.4)], 10.0),
    ([Peak("lorentz", 2.0, 0.3, 0.6), Peak("lorentz", 5.0, 0.5, 0.4)], 20.0),
    ([Peak("gauss", 3.0, 0.5, 0.7), Peak("gauss", 12.0, 0.05, 0.3)], 20.0),
    ([Peak("gauss", 0.5, 2.0, 0.5), Peak("lorentz", 14.5, 1.7, 0.5)], 20.0),
    ([Peak("lorentz", 0.6, 0.05, 1.0)], 3.5),
]


@pytest.mark.parametrize("peaks,W", PEAK_SETS)
@pytest.mark.parametrize("tau", [0.0, 0.05, 0.7, 3.0, 8.0])
def test_laplace_closed_form_matches_quadrature(peaks, W, tau):
    pts = [p.centre for p in peaks]
    q = _quad(lambda w: sum(p.density(w) for p in peaks) * np.exp(-w * tau) / (2 * np.pi), W, pts)
    c = laplace(peaks, W, tau)[0]
    assert abs(c - q) <= 1e-11 * abs(q)


@pytest.mark.parametrize("peaks,W", PEAK_SETS)
def test_mass_and_moment_match_quadrature(peaks, W):
    pts = [p.centre for p in peaks]
    m = _quad(lambda w: sum(p.density(w) for p in peaks), W, pts)
    m1 = _quad(lambda w: w * sum(p.density(w) for p in peaks), W, pts)
    assert abs(mass(peaks, W) - m) <= 1e-12 * m
    assert abs(first_moment(peaks, W) - m1) <= 1e-12 * m1
    # tau = 0 of the transform is the mass over 2 pi
    assert abs(laplace(peaks, W, 0.0)[0] * 2 * np.pi - m) <= 1e-12 * m
    bm = bin_masses(peaks, W, 37)
    assert abs(bm.sum() - m) <= 1e-12 * m and np.all(bm >= 0)


def test_tiny_problem_recipe():
    P = tiny_double_lorentz()
    assert P.n_tau == 32 and P.n_omega == 64
    np.testing.assert_allclose(P.tau, 4.0 * np.arange(32) / 31, rtol=0, atol=0)
    np.testing.assert_allclose(P.omega, 10.0 * (np.arange(64) + 0.5) / 64, rtol=0, atol=0)
    np.testing.assert_allclose(P.sigma, 1e-4 * P.F_exact)
    z = (P.F - P.F_exact) / P.sigma
    assert abs(z.mean()) < 0.6 and 0.5 < z.std() < 1.5
    # same seed, same data
    Q = tiny_double_lorentz()
    assert np.array_equal(P.F, Q.F)
    assert P.B / P.A > P.omega[0] and P.B / P.A < P.omega[-1]


def test_other_recipes_shapes():
    P = paper_scale_double_lorentz(1e-5)
    assert P.n_tau == 200 and P.n_omega == 1000 and P.tau[-1] == 8.0
    assert abs(P.d_omega - 0.02) < 1e-15
    Q = precision_random_peaks(3)
    assert Q.n_tau == 512 and Q.n_omega == 2048 and 1 <= len(Q.peaks) <= 4
    R = random_batch_problem(5, seed=1)
    assert 50 <= R.n_tau <= 500 and 200 <= R.n_omega <= 2000 and 256 <= R.n_walkers <= 4096
    assert 1e-5 <= R.extra["noise_level"] <= 1e-3
    # lowered size caps draw in the same order: the noise level and the peaks are unchanged
    for i in range(8):
        full = random_batch_problem(i, seed=77)
        small = random_batch_problem(i, seed=77, max_tau=200, max_omega=800, max_walkers=1024)
        assert 50 <= small.n_tau <= 200 and 200 <= small.n_omega <= 800 and 256 <= small.n_walkers <= 1024
        assert small.extra["noise_level"] == full.extra["noise_level"] and small.peaks == full.peaks
