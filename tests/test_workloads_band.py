"""CPU pins of the band-limited spectrum (Eq. lorentzian-band), the correlated undersampling
noise (Sec. resampling) and the skew of Sec. annealing results."""
import numpy as np
import pytest
from scipy import integrate

from workloads import bin_masses, first_moment, laplace, lorentzian_band, lorentzian_band_peaks, mass, skew
from workloads import correlated as CN

BAND = (0.5, 2.5)
W = 3.5


def _S(w):
    return sum(p.density(w) for p in lorentzian_band_peaks()) * ((w >= BAND[0]) & (w <= BAND[1]))


@pytest.mark.parametrize("tau", [0.0, 0.05, 1.0, 7.95])
def test_band_laplace_is_the_band_integral(tau):
    q = integrate.quad(lambda w: _S(np.array(w)) * np.exp(-w * tau) / (2 * np.pi), *BAND, epsabs=0, epsrel=1e-13)[0]
    assert laplace(lorentzian_band_peaks(), W, [tau], BAND)[0] == pytest.approx(q, rel=1e-12)


def test_band_mass_moment_and_bins():
    peaks = lorentzian_band_peaks()
    m = integrate.quad(lambda w: _S(np.array(w)), *BAND, epsrel=1e-13)[0]
    mom = integrate.quad(lambda w: w * _S(np.array(w)), *BAND, epsrel=1e-13)[0]
    assert mass(peaks, W, BAND) == pytest.approx(m, rel=1e-12)
    assert first_moment(peaks, W, BAND) == pytest.approx(mom, rel=1e-12)
    bm = bin_masses(peaks, W, 1000, BAND)
    assert bm.sum() == pytest.approx(m, rel=1e-12)
    x = (np.arange(1000) + 0.5) * W / 1000
    assert np.all(bm[x < BAND[0] - 0.002] == 0) and np.all(bm[x > BAND[1] + 0.002] == 0)


def test_process_covariance_is_positive_semidefinite():
    lags = 0.05 * np.arange(120)
    F = laplace(lorentzian_band_peaks(), W, lags, BAND)
    assert np.linalg.eigvalsh(CN.covariance(F)).min() > -1e-12 * F[0]


def test_sample_autocorrelation_is_unbiased():
    """The mean autocorrelation of many sequences is F, within its standard error."""
    lags = 0.05 * np.arange(64)
    F = laplace(lorentzian_band_peaks(), W, lags, BAND)
    mean, sigma = CN.undersampled(F, 16, 20000, np.random.default_rng(1))
    z = (mean - F[:16]) / sigma
    assert np.all(np.abs(z) < 5)
    assert np.all(np.diff(sigma / F[:16]) > 0)        # relative noise grows with tau


def test_clt_noise_matches_the_procedure():
    """For a moderate number of sequences the two forms give the same noise: sigma of the
    mean of M sequences equals sqrt(diag(Sigma_1) / M)."""
    lags = 0.05 * np.arange(64)
    F = laplace(lorentzian_band_peaks(), W, lags, BAND)
    rng = np.random.default_rng(2)
    S1 = CN.single_sequence_covariance(F, 16, rng, n_sample=20000)
    reps = np.array([CN.undersampled(F, 16, 200, rng)[0] for _ in range(400)])
    np.testing.assert_allclose(reps.std(axis=0, ddof=1), np.sqrt(np.diag(S1) / 200), rtol=0.15)
    # and the noise is correlated between tau points, as the procedure's is
    c_rep = np.corrcoef(reps[:, 0], reps[:, 8])[0, 1]
    c_clt = S1[0, 8] / np.sqrt(S1[0, 0] * S1[8, 8])
    assert c_rep == pytest.approx(c_clt, abs=0.15) and c_clt > 0.3


def test_band_problem_noise_level():
    P = lorentzian_band(1e-4, seed=3)
    assert P.sigma[0] / P.F_exact[0] == pytest.approx(1e-4, rel=1e-12)
    assert np.all(np.diff(P.sigma / P.F_exact) > 0)
    assert np.abs((P.F - P.F_exact) / P.sigma).max() < 6
    assert lorentzian_band(0.0, seed=3).F.tolist() == P.F_exact.tolist()


def test_skew():
    x = (np.arange(1000) + 0.5) * W / 1000
    bm = bin_masses(lorentzian_band_peaks(), W, 1000, BAND)
    assert skew(bm, x) < 1e-9                       # the band is symmetric about 1.5
    a = np.zeros(1000)
    a[100] = 1.0
    assert skew(a, x) == 1.0
    a[900] = 3.0
    assert skew(a, x) == pytest.approx(0.5)
