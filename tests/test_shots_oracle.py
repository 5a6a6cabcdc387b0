"""Pins of the shot-noise oracle (Sec. 4.3.2) against what the mathematics
fixes: the Householder factor's identities, the exact sum of the Gaussian
sample, its mean and covariance (Monte Carlo, fixed seed), the degenerate
case, closed forms of the exact sampler and of the vector-Jacobian product."""
import numpy as np
import pytest

from oracle import shots as O


def rand_p(rng, k, zeros=0):
    p = rng.random(k)
    if zeros:
        p[rng.choice(k - 1, zeros, replace=False)] = 0.0
    return p / p.sum()


@pytest.mark.parametrize("k,seed", [(2, 1), (5, 2), (16, 3), (64, 4)])
def test_householder_identities(k, seed):
    rng = np.random.default_rng(seed)
    p = rand_p(rng, k)
    u = np.sqrt(p)
    v = O.householder_v(p)
    S = np.eye(k) - 2.0 * np.outer(v, v)
    e = np.zeros(k)
    e[-1] = 1.0
    np.testing.assert_allclose(S @ u, e, atol=1e-14)               # reflects u onto e_{k-1}
    np.testing.assert_allclose(S @ S.T, np.eye(k), atol=1e-14)     # orthogonal
    J = np.eye(k)
    J[-1, -1] = 0.0
    # covariance of x_n = S z with z_{k-1} = 0: I - u u^T (Sec. 4.3.2)
    np.testing.assert_allclose(S @ J @ S.T, np.eye(k) - np.outer(u, u), atol=1e-14)


@pytest.mark.parametrize("k,seed", [(3, 5), (32, 6), (257, 7)])
def test_gaussian_sum_is_n(k, seed):
    rng = np.random.default_rng(seed)
    p = rand_p(rng, k, zeros=min(3, k - 2))
    for n in (1.0, 1000.0, 1e6):
        y = O.shots_gaussian(p, n, rng.standard_normal(k - 1))
        assert abs(y.sum() - n) <= 1e-12 * n * k


def test_gaussian_degenerate_point_mass():
    k = 8
    p = np.zeros(k)
    p[-1] = 1.0
    np.testing.assert_array_equal(O.householder_v(p), np.zeros(k))
    y = O.shots_gaussian(p, 500.0, np.random.default_rng(1).standard_normal(k - 1))
    np.testing.assert_allclose(y, 500.0 * p, atol=1e-12)


def test_gaussian_moments_monte_carlo():
    """E[y] = n p and Cov[y] = n (diag p - p p^T), the multinomial's moments."""
    rng = np.random.default_rng(11)
    k, n, m = 6, 400.0, 40000
    p = rand_p(rng, k)
    Y = np.stack([O.shots_gaussian(p, n, rng.standard_normal(k - 1)) for _ in range(m)])
    cov = n * (np.diag(p) - np.outer(p, p))
    se_mean = np.sqrt(np.diag(cov) / m)
    assert np.all(np.abs(Y.mean(0) - n * p) < 5 * se_mean + 1e-9)
    emp = np.cov(Y.T)
    scale = np.sqrt(np.outer(np.diag(cov), np.diag(cov)) * 2.0 / m)  # standard error of a covariance entry
    assert np.all(np.abs(emp - cov) < 6 * scale + 1e-9)
    # the printed S = I - v v^T (no factor 2) gives the wrong covariance
    v = O.householder_v(p)
    S1 = np.eye(k) - np.outer(v, v)
    J = np.eye(k)
    J[-1, -1] = 0.0
    u = np.sqrt(p)
    assert np.max(np.abs(S1 @ J @ S1.T - (np.eye(k) - np.outer(u, u)))) > 0.05


def test_exact_sampler_closed_forms():
    k = 16
    # a point mass: every shot lands on it
    p = np.zeros(k)
    p[9] = 1.0
    u = np.random.default_rng(2).random(1000)
    assert np.all(O.sample_exact(p, u) == 9)
    # uniform p: the shot for u lies in floor(u k)
    p = np.full(k, 1.0 / k)
    u = (np.arange(k) + 0.5) / k
    np.testing.assert_array_equal(O.sample_exact(p, u), np.arange(k))
    # zero-probability outcomes are never drawn; unnormalised p is normalised
    p = np.array([0.0, 2.0, 0.0, 6.0])
    s = O.sample_exact(p, np.array([0.0, 0.24, 0.25, 0.26, 0.999999]))
    np.testing.assert_array_equal(s, [1, 1, 3, 3, 3])


def test_exact_sampler_chi_square():
    rng = np.random.default_rng(21)
    k, shots = 12, 200000
    p = rand_p(rng, k)
    s = O.sample_exact(p, rng.random(shots))
    counts = np.bincount(s, minlength=k)
    chi2 = np.sum((counts - shots * p) ** 2 / (shots * p))
    assert chi2 < 45.0  # 11 degrees of freedom: P(chi2 > 45) ~ 5e-6


def test_vjp_closed_form_without_noise():
    """z = 0: y = n p, so sum ybar y = n sum ybar |psi|^2 and
    dL/d conj(psi) = n ybar psi."""
    rng = np.random.default_rng(5)
    k = 8
    psi = rng.standard_normal(k) + 1j * rng.standard_normal(k)
    psi /= np.linalg.norm(psi)
    ybar = rng.standard_normal(k)
    lam = O.shots_gaussian_vjp_psi(psi, 300.0, np.zeros(k - 1), ybar)
    np.testing.assert_allclose(lam, 300.0 * ybar * psi, rtol=1e-6, atol=1e-8)
