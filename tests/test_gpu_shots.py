"""Shot noise on the GPU through the C ABI against the oracle (Sec. 4.3.2):
probabilities, exact samples from given uniforms, the Gaussian sample, its
seed for the reverse sweep, and the end-to-end gradient of a loss of the
shots against finite differences of the oracle."""
import numpy as np
import pytest
import torch

import oracle
from oracle import shots as OS
from paper_2511_19291_gb300 import workloads as W
from gpu_helpers import DTYPES, gpu_state, params_tensor, sim, to_numpy

pytestmark = pytest.mark.gpu


def ansatz_state(n, layers, dtype, seed=3):
    circ = W.hea_ansatz(n, layers)
    params = W.config_rng(seed).angles(circ.n_params)
    st, c, p = gpu_state(circ, params, "fused", dtype)
    return st, circ, params


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("n", [5, 13])
def test_probabilities(dtype, n):
    S = sim()
    st, _, _ = ansatz_state(n, 2, dtype)
    p = S.probabilities(st).cpu().numpy()
    np.testing.assert_allclose(p, OS.probabilities(to_numpy(st)), rtol=1e-14, atol=1e-300)


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("n,shots", [(6, 5000), (16, 20000), (21, 4000)])
def test_sample_matches_inverse_transform(dtype, n, shots):
    """Same uniforms on both sides: identical outcomes, except where a
    uniform sits within 1e-11 of a boundary of the oracle's cumulative
    distribution (the two sum in different orders)."""
    S = sim()
    st, _, _ = ansatz_state(n, 2, dtype)
    u = np.random.default_rng(100 + n).random(shots)
    got = S.sample(st, torch.tensor(u)).cpu().numpy()
    p = OS.probabilities(to_numpy(st))
    ref = OS.sample_exact(p, u)
    c = OS.cdf(p)
    bad = np.nonzero(got != ref)[0]
    for s in bad:
        j = min(ref[s], got[s])
        assert abs(u[s] - c[j]) < 1e-11, (s, u[s], got[s], ref[s])
    assert len(bad) <= max(1, shots // 10000)
    assert np.all(p[got] > 0)


def test_sample_basis_and_ghz():
    S = sim()
    n = 14
    st = S.State(n, torch.complex64).reset(12345)
    u = torch.tensor(np.random.default_rng(1).random(3000))
    assert torch.all(S.sample(st, u) == 12345)
    st2, _, _ = gpu_state(W.ghz_circuit(n), None, "fused", "c128")
    s = S.sample(st2, u).cpu().numpy()
    assert set(np.unique(s)) <= {0, (1 << n) - 1}
    assert abs(np.mean(s == 0) - 0.5) < 0.05
    assert S.sample(st2, torch.zeros(0, dtype=torch.float64)).numel() == 0


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("n,shots", [(4, 1000.0), (12, 1e5), (17, 2.5e6)])
def test_shots_gaussian(dtype, n, shots):
    S = sim()
    st, _, _ = ansatz_state(n, 2, dtype)
    z = np.random.default_rng(7 + n).standard_normal((1 << n) - 1)
    y = S.shots_gaussian(st, shots, torch.tensor(z)).cpu().numpy()
    ref = OS.shots_gaussian(OS.probabilities(to_numpy(st)), shots, z)
    np.testing.assert_allclose(y, ref, rtol=0, atol=1e-9 * np.sqrt(shots) + 1e-12 * shots)
    assert abs(y.sum() - ref.sum()) < 1e-9 * shots


def test_shots_gaussian_degenerate():
    S = sim()
    n = 6
    st = S.State(n, torch.complex128).reset((1 << n) - 1)  # p = e_{N-1}: v = 0
    y = S.shots_gaussian(st, 300.0, torch.randn((1 << n) - 1, dtype=torch.float64)).cpu().numpy()
    ref = np.zeros(1 << n)
    ref[-1] = 300.0
    np.testing.assert_allclose(y, ref, atol=1e-12)


@pytest.mark.parametrize("n", [3, 5])
def test_shots_gaussian_seed_against_finite_differences(n):
    S = sim()
    st, _, _ = ansatz_state(n, 2, "c128", seed=4)
    rng = np.random.default_rng(40 + n)
    z = rng.standard_normal((1 << n) - 1)
    ybar = rng.standard_normal(1 << n)
    lam = S.State(n, torch.complex128)
    S.shots_gaussian_backward(st, 700.0, torch.tensor(z), torch.tensor(ybar), lam)
    ref = OS.shots_gaussian_vjp_psi(to_numpy(st), 700.0, z, ybar)
    np.testing.assert_allclose(to_numpy(lam), ref, rtol=1e-6, atol=1e-6)


@pytest.mark.parametrize("dtype,rtol", [("c128", 1e-6), ("c64", 2e-3)])
def test_shots_gaussian_gradient(dtype, rtol):
    """d(sum_i w_i y_i)/dtheta through the autograd function against central
    differences of the oracle's forward (FP64, h = 1e-5)."""
    S = sim()
    n = 6
    circ = W.hea_ansatz(n, 2)
    params = np.array(W.config_rng(9).angles(circ.n_params))
    rng = np.random.default_rng(9)
    z = rng.standard_normal((1 << n) - 1)
    w = rng.standard_normal(1 << n)
    nshot = 2000.0
    c = S.Circuit(circ)
    p = params_tensor(params).requires_grad_(True)
    y = S.shots_gaussian_fn(p, c, nshot, torch.tensor(z, device="cuda"), dtype=DTYPES[dtype])
    (y * torch.tensor(w, device="cuda")).sum().backward()
    g = p.grad.cpu().numpy()

    def L(th):
        return float(np.dot(w, OS.shots_gaussian(OS.probabilities(oracle.run(circ, th)), nshot, z)))

    h = 1e-5
    ref = np.array([(L(params + h * e) - L(params - h * e)) / (2 * h) for e in np.eye(len(params))])
    scale = np.max(np.abs(ref))
    np.testing.assert_allclose(g, ref, rtol=0, atol=rtol * scale)
