"""Pins for the oracle's model: kernel table, residual, start spectrum, Philox."""
import numpy as np
import pytest
from scipy import integrate

import oracle as O
from workloads import tiny_double_lorentz


def _grid(n_tau=7, n_omega=9, W=3.0, dtau=0.4):
    tau = dtau * np.arange(n_tau, dtype=np.float64)
    omega = (np.arange(n_omega) + 0.5) * (W / n_omega)
    return tau, omega


def test_kernel_is_the_bin_integral():
    """K_ij = (1/2pi) int_bin e^{-w tau} dw (Eq. correlation-model), checked by quadrature."""
    tau, omega = _grid()
    sigma = np.linspace(0.5, 2.0, tau.size)
    K, Fh, dw = O.tables(tau, np.ones_like(tau), sigma, omega)
    assert abs(dw - 3.0 / 9) < 1e-15
    for i, t in enumerate(tau):
        for j in range(omega.size):
            q, _ = integrate.quad(lambda w: np.exp(-w * t) / (2 * np.pi), j * dw, (j + 1) * dw,
                                  epsabs=0, epsrel=1e-13)
            assert abs(K[i, j] * sigma[i] - q) <= 1e-13 * q
    np.testing.assert_array_equal(Fh, 1.0 / sigma)


@pytest.mark.parametrize("tau0", [0.0, 0.3])
def test_kernel_factors_along_tau_in_quads(tau0):
    """The factorisation the 8-lane FP32 sweep builds its quad-compact column tables on: on a
    uniform grid tau_i = tau_0 + i dtau, with i0 = 4 floor(i / 4) and e = i - i0,
    Khat_{i,j} = Khat_{i0,j} (Khat_{i,0} / Khat_{i0,0}) e^{-j dw e dtau} (Eq. efficient-
    correlation-model read along tau), checked on the oracle's FP64 table with sigma varying
    along tau.  On an uneven grid it fails by far more than rounding, which is why the 8-lane
    sweep refuses one."""
    n_tau, n_omega, dtau = 37, 50, 8.0 / 199
    tau = tau0 + dtau * np.arange(n_tau, dtype=np.float64)
    omega = (np.arange(n_omega) + 0.5) * (20.0 / n_omega)
    sigma = 1e-4 * np.exp(-1.3 * tau) + 1e-9
    K, _, dw = O.tables(tau, np.ones_like(tau), sigma, omega)
    j = np.arange(n_omega)
    for i in range(n_tau):
        i0, e = i & ~3, i & 3
        pred = K[i0] * (K[i, 0] / K[i0, 0]) * np.exp(-j * dw * e * dtau)
        np.testing.assert_allclose(K[i], pred, rtol=1e-12, atol=0)
    uneven = tau0 + 8.0 * (np.arange(n_tau, dtype=np.float64) / (n_tau - 1)) ** 1.5
    Ku, _, _ = O.tables(uneven, np.ones_like(uneven), np.ones_like(uneven), omega)
    d = uneven[1] - uneven[0]
    pred = Ku[0] * (Ku[1, 0] / Ku[0, 0]) * np.exp(-j * dw * d)
    np.testing.assert_allclose(Ku[1], pred, rtol=1e-12)        # one step defines dtau
    pred3 = Ku[0] * (Ku[3, 0] / Ku[0, 0]) * np.exp(-j * dw * 3 * d)
    assert np.max(np.abs(Ku[3] / pred3 - 1.0)) > 1e-3


def test_fp32_column_forms_stay_within_a_few_ulp():
    """The FP32 sweeps form a kernel column element from FP32 factors, each rounded once from
    FP64: full rows as Qhi[j/32][i] * Qlo[j%32][i]; the quad-compact tables (uniform tau) as
    ((Qhi[j/32][i0] * Qlo[j%32][i0]) * X_j^e) * rho_i.  Emulated in float32 with those operation
    orders on the paper-scale grid, the full rows stay within 2 float32 ulp of the oracle's FP64
    table and the compact form (seven roundings) within 5, wherever the element is a normal
    float32: the two forms differ in the last bits only."""
    from workloads import paper_scale_double_lorentz
    P = paper_scale_double_lorentz(1e-4, n_walkers=1)
    K, _, dw = O.tables(P.tau, P.F, P.sigma, P.omega)         # [n_tau, n_omega], FP64
    n_tau, n_omega = K.shape
    dtau = P.tau[1] - P.tau[0]
    i = np.arange(n_tau)[:, None]
    j = np.arange(n_omega)[None, :]
    qhi = K[:, (j[0] // 32) * 32].astype(np.float32)          # Khat_{i, 32 h}
    qlo = np.exp(-(j % 32) * dw * P.tau[:, None]).astype(np.float32)
    full = qhi * qlo
    i0 = (i // 4) * 4
    e = i - i0
    x = np.exp(-j * dw * e * dtau).astype(np.float32)
    rho = (K[:, :1] / K[i0[:, 0], :1]).astype(np.float32)
    compact = ((qhi[i0[:, 0], :] * qlo[i0[:, 0], :]) * x) * rho
    normal = K > np.finfo(np.float32).tiny * 2 ** 8
    ulp = np.spacing(K.astype(np.float32)).astype(np.float64)
    for form, bound in ((full, 2), (compact, 5)):
        err = np.abs(form.astype(np.float64) - K)
        assert np.all(err[normal] <= bound * ulp[normal])


def test_kernel_matches_efficient_form():
    """Eq. (efficient-correlation-model): F(tau_i) = c_i sum_j a_j (e^{-dw dtau})^{ij} with
    c_0 = dw/2pi and c_i = (1 - e^{-i dw dtau}) / (2 pi i dtau) on a uniform tau grid."""
    tau, omega = _grid(n_tau=11, n_omega=13, W=5.0, dtau=0.25)
    K, _, dw = O.tables(tau, np.ones_like(tau), np.ones_like(tau), omega)
    q = np.exp(-dw * 0.25)
    for i in range(tau.size):
        c = dw / (2 * np.pi) if i == 0 else (1 - np.exp(-i * dw * 0.25)) / (2 * np.pi * i * 0.25)
        for j in range(omega.size):
            assert abs(K[i, j] - c * q ** (i * j)) <= 1e-13 * K[i, j]


def test_histogram_data_gives_zero_residue():
    """A histogram spectrum whose transform is the data has chi2 = 0 up to rounding."""
    P = tiny_double_lorentz()
    K, _, dw = O.tables(P.tau, P.F, P.sigma, P.omega)
    rng = np.random.default_rng(3)
    a_true = rng.uniform(0.0, 2.0, P.n_omega)
    F_hist = (K * P.sigma[:, None]) @ a_true
    K2, Fh2, _ = O.tables(P.tau, F_hist, P.sigma, P.omega)
    R, chi2 = O.residual(K2, Fh2, a_true)
    assert chi2 <= 1e-24 * np.sum(Fh2 ** 2)
    # and the residual is exactly the plain matrix-vector difference
    R2, c2 = O.residual(K2, Fh2, a_true * 1.01)
    np.testing.assert_allclose(R2, Fh2 - K2 @ (a_true * 1.01), rtol=1e-12, atol=1e-9)
    assert abs(c2 - np.sum(R2 ** 2)) <= 1e-12 * c2


def test_histogram_transform_by_quadrature():
    """K a equals the transform of the piecewise-constant spectrum computed by quadrature."""
    tau, omega = _grid(n_tau=5, n_omega=6, W=2.0, dtau=0.9)
    a = np.array([0.3, 1.2, 0.0, 2.5, 0.7, 0.1])
    K, _, dw = O.tables(tau, np.ones_like(tau), np.ones_like(tau), omega)
    for i, t in enumerate(tau):
        S = lambda w: a[min(int(w / dw), a.size - 1)]
        q = sum(integrate.quad(lambda w: S(w) * np.exp(-w * t) / (2 * np.pi), j * dw, (j + 1) * dw,
                               epsabs=0, epsrel=1e-13)[0] for j in range(a.size))
        assert abs(K[i] @ a - q) <= 1e-13 * q


def test_invalid_grids_are_refused():
    tau, omega = _grid()
    with pytest.raises(ValueError):
        O.tables(tau, np.ones_like(tau), np.ones_like(tau), omega + 0.01)   # bins not from 0
    bad = omega.copy(); bad[3] += 1e-3
    with pytest.raises(ValueError):
        O.tables(tau, np.ones_like(tau), np.ones_like(tau), bad)            # not uniform
    with pytest.raises(ValueError):
        O.tables(tau, np.ones_like(tau), -np.ones_like(tau), omega)         # sigma <= 0
    with pytest.raises(ValueError):
        O.tables(-tau - 1, np.ones_like(tau), np.ones_like(tau), omega)     # tau < 0


@pytest.mark.parametrize("ratio", [0.15, 0.5, 0.5000001, 0.8, 0.97])
def test_start_spectrum_sum_rules_and_max_entropy(ratio):
    omega = (np.arange(50) + 0.5) * 0.2
    A = 3.7
    B = A * (omega[0] + ratio * (omega[-1] - omega[0]))
    a, lam = O.initial_spectrum(omega, A, B)
    assert np.all(a > 0)
    assert abs(a.sum() - A) <= 1e-13 * A
    assert abs(a @ omega - B) <= 1e-13 * B
    # an exponential family: log a is affine in x, so its gradient is orthogonal to
    # every perturbation that keeps both sums, i.e. it is a stationary point of the entropy
    fit = np.polyfit(omega, np.log(a), 1)
    assert np.max(np.abs(np.polyval(fit, omega) - np.log(a))) < 1e-11
    assert abs(fit[0] + lam) < 1e-9 * max(1.0, abs(lam))
    # and a maximum: entropy falls along any moment-preserving direction
    rng = np.random.default_rng(1)
    big = a > 1e-3 * a.max()          # perturb where a is not negligibly small
    C = np.vstack([np.ones(big.sum()), omega[big]])
    for _ in range(5):
        v = np.zeros_like(a)
        u = rng.standard_normal(big.sum())
        v[big] = u - C.T @ np.linalg.solve(C @ C.T, C @ u)
        t = 1e-3 * a[big].min() / np.abs(v).max()
        H = lambda q: -np.sum(q * np.log(q))
        assert H(a + t * v) < H(a) and H(a - t * v) < H(a)


def test_start_spectrum_flat_at_midpoint_and_refusal():
    omega = (np.arange(40) + 0.5) * 0.25
    a, lam = O.initial_spectrum(omega, 2.0, 2.0 * omega.mean())
    assert abs(lam) < 1e-12
    np.testing.assert_allclose(a, 2.0 / 40, rtol=1e-12)
    with pytest.raises(ValueError):
        O.initial_spectrum(omega, 2.0, 2.0 * omega[-1] * 1.01)


# ------------------------------------------------------------------ Philox

M0, M1 = 0xD2511F53, 0xCD9E8D57
W0, W1 = 0x9E3779B9, 0xBB67AE85
MASK = 0xFFFFFFFF


def _unround(y, k):
    """Inverse of one Philox4x32 round (Salmon et al., SC'11): the low halves
    of the two products are outputs 1 and 3, and M0, M1 are odd, so the
    multiplied words come back through the inverses of M0, M1 mod 2^32."""
    x0 = (y[3] * pow(M0, -1, 2 ** 32)) & MASK
    x2 = (y[1] * pow(M1, -1, 2 ** 32)) & MASK
    hi0 = (M0 * x0) >> 32
    hi1 = (M1 * x2) >> 32
    x1 = y[0] ^ hi1 ^ k[0]
    x3 = y[2] ^ hi0 ^ k[1]
    return [x0, x1, x2, x3]


def test_philox_inverts_to_its_counter():
    """Running the published round structure backwards through the 10 round
    keys recovers the counter: pins both constants pairs, the word order and
    the round count of the oracle's Philox4x32-10."""
    rng = np.random.default_rng(7)
    for _ in range(50):
        ctr = [int(v) for v in rng.integers(0, 2 ** 32, 4, dtype=np.uint64)]
        key = [int(v) for v in rng.integers(0, 2 ** 32, 2, dtype=np.uint64)]
        y = [int(v) for v in O.philox4x32_10(ctr, key)]
        keys = []
        k = list(key)
        for r in range(10):
            keys.append(list(k))
            k = [(k[0] + W0) & MASK, (k[1] + W1) & MASK]
        for r in reversed(range(10)):
            y = _unround(y, keys[r])
        assert y == ctr


def test_philox_statistics():
    key = [0x12345678, 0x9ABCDEF0]
    words = np.array([O.philox4x32_10([i, 3, 5, 0], key) for i in range(20000)], dtype=np.uint64)
    flat = words.ravel()
    # byte histogram: chi-square with 255 dof stays far from its tails
    counts = np.bincount((flat >> 24).astype(np.int64), minlength=256)
    e = flat.size / 256
    chi = np.sum((counts - e) ** 2 / e)
    assert 180 < chi < 340
    # each bit is set half the time
    bits = ((flat[:, None] >> np.arange(32, dtype=np.uint64)) & 1).mean(0)
    assert np.all(np.abs(bits - 0.5) < 0.01)
    # avalanche: one flipped counter bit changes about half of the 128 output bits
    flips = []
    for i in range(200):
        a = O.philox4x32_10([i, 0, 0, 0], key)
        b = O.philox4x32_10([i ^ 1, 0, 0, 0], key)
        flips.append(sum(bin(int(u) ^ int(v)).count("1") for u, v in zip(a, b)))
    assert 60 < np.mean(flips) < 68
