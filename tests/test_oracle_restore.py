"""CPU pins of the oracle's sum-rule restoration (or_restore): a spectrum that has drifted off
the two sum rules of Sec. 2.2 (sum a_j = A, sum a_j x_j = B) is put back on both by the
reweighting a_j <- a_j kappa (1 + lambda (x_j - c)), c = B'/A'; the tilt is skipped when it
could turn a factor negative."""
import numpy as np

import oracle as O


def test_hand_worked_example():
    # four unit bins at x = 0.5 .. 3.5: A' = 4, B' = 8, c = 2, sum a (x - c)^2 = 5; the target
    # B = 8.4 needs lambda = (2.1 - 2) * 4 / 5 = 0.08, so a' = 1 + 0.08 (x - 2)
    x = np.array([0.5, 1.5, 2.5, 3.5])
    out = O.restore(x, 4.0, 8.4, np.ones(4))
    np.testing.assert_allclose(out, [0.88, 0.96, 1.04, 1.12], rtol=1e-15, atol=1e-15)


def test_both_sums_restored_and_the_factor_is_affine():
    rng = np.random.default_rng(5)
    x = (np.arange(200) + 0.5) * 0.05
    for _ in range(20):
        a = rng.uniform(0.1, 2.0, x.size)
        A1, B1 = a.sum(), a @ x
        A, B = A1 * (1 + rng.uniform(-1e-3, 1e-3)), B1 * (1 + rng.uniform(-1e-3, 1e-3))
        out = O.restore(x, A, B, a)
        assert abs(out.sum() - A) <= 1e-13 * A
        assert abs(out @ x - B) <= 1e-13 * B
        f = out / a                                  # kappa (1 + lambda (x - c)): a line in x
        coef = np.polyfit(x, f, 1)
        assert np.abs(np.polyval(coef, x) - f).max() <= 1e-13
        assert np.all(out > 0)


def test_identity_on_the_sum_rules():
    rng = np.random.default_rng(6)
    x = (np.arange(64) + 0.5) * 0.1
    a = rng.uniform(0.1, 1.0, x.size)
    out = O.restore(x, a.sum(), a @ x, a)
    np.testing.assert_allclose(out, a, rtol=1e-14)


def test_tilt_skipped_when_a_factor_could_turn_negative():
    # a first moment far off needs |lambda| (x_max - x_min) >= 1/2: only the scale is applied
    x = np.array([0.5, 1.5, 2.5, 3.5])
    a = np.ones(4)
    out = O.restore(x, 2.0, 2.0 * 3.4, a)
    np.testing.assert_allclose(out, 0.5 * a, rtol=1e-15)
    assert abs(out.sum() - 2.0) <= 1e-15
