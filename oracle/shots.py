"""Shot noise on the probability vector |psi|^2 (Sec. 4.3.2), plain numpy in
FP64.

TEST INFRASTRUCTURE ONLY: only tests/, __graft_entry__.smoke() and the CPU
legs of bench.py may import this module.  It shares no code with the CUDA
library.  Random numbers are inputs: the uniforms of the exact sampler and
the unit normals of the Gaussian sampler are drawn by the caller.

Functions and the passage each follows:

* ``probabilities``  -- p_b = |psi_b|^2 (measurement in the Z basis, Sec. 2.2.1)
* ``sample_exact``   -- exact samples of the multinomial over outcomes
  (Sec. 4.3.2, "Exact"): each shot is the outcome b whose cumulative interval
  [CDF(b-1), CDF(b)) of the normalised p holds the shot's uniform (inverse
  transform).  The paper's hierarchical scheme (group totals, then outcomes
  within groups) yields the same distribution; this is its single-machine
  form.
* ``shots_gaussian`` -- the approximate, differentiable sample (Sec. 4.3.2,
  "Approximate"): y = n p + sqrt(n) D S z with D = diag(sqrt(p)),
  u = sqrt(p), v = (e_{k-1} - u)/||e_{k-1} - u|| (v = 0 when u = e_{k-1}),
  S = I - 2 v v^T and z = (z_0, ..., z_{k-2}, 0).  Reading: the printed
  S = I - v v^T lacks the factor 2 (only the Householder reflection maps u to
  e_{k-1} and gives S diag(1..1, 0) S^T = I - u u^T, the covariance of x_n);
  the printed e_k^{(k)} is the last unit vector, index k - 1.
* ``shots_gaussian_vjp_psi`` -- d(sum_i ybar_i y_i)/d conj(psi) for the
  reverse sweep, lambda_b = ubar_b psi_b / (2 |psi_b|) (0 where psi_b = 0),
  with ubar = d(sum ybar y)/du by central differences of shots_gaussian in
  FP64 (slow; tiny states only).
"""
from __future__ import annotations

import numpy as np


def probabilities(psi: np.ndarray) -> np.ndarray:
    """p_b = |psi_b|^2."""
    return np.abs(np.asarray(psi, dtype=np.complex128)) ** 2


def cdf(p: np.ndarray) -> np.ndarray:
    """Cumulative distribution of the normalised p (FP64, left to right)."""
    c = np.cumsum(np.asarray(p, dtype=np.float64))
    return c / c[-1]


def sample_exact(p: np.ndarray, uniforms: np.ndarray) -> np.ndarray:
    """One outcome per uniform u in [0, 1): the smallest b with CDF(b) > u."""
    c = cdf(p)
    out = np.empty(len(uniforms), dtype=np.int64)
    for s, u in enumerate(np.asarray(uniforms, dtype=np.float64)):
        b = int(np.searchsorted(c, u, side="right"))
        out[s] = min(b, len(c) - 1)
    return out


def householder_v(p: np.ndarray) -> np.ndarray:
    """v = (e_{k-1} - u) / ||e_{k-1} - u||, u = sqrt(p); zero when u = e_{k-1}."""
    u = np.sqrt(np.asarray(p, dtype=np.float64))
    vt = -u.copy()
    vt[-1] += 1.0
    nrm = np.sqrt(np.sum(vt * vt))
    if nrm == 0.0:
        return np.zeros_like(u)
    return vt / nrm


def shots_gaussian(p: np.ndarray, n_shots: float, z: np.ndarray) -> np.ndarray:
    """y = n p + sqrt(n) D S z, z's last entry taken as 0 (z has k or k - 1 entries)."""
    p = np.asarray(p, dtype=np.float64)
    k = len(p)
    zz = np.zeros(k)
    zz[:k - 1] = np.asarray(z, dtype=np.float64)[:k - 1]
    v = householder_v(p)
    x = zz - 2.0 * v * np.dot(v, zz)          # S z
    return n_shots * p + np.sqrt(n_shots) * np.sqrt(p) * x


def shots_gaussian_vjp_psi(psi: np.ndarray, n_shots: float, z: np.ndarray, ybar: np.ndarray,
                           h: float = 1e-6) -> np.ndarray:
    """lambda = dL/d conj(psi) for L = sum_i ybar_i y_i(|psi|^2), by central
    differences in u = |psi| (each u_b moved by +-h)."""
    psi = np.asarray(psi, dtype=np.complex128)
    u = np.abs(psi)
    ybar = np.asarray(ybar, dtype=np.float64)

    def L(uu):
        return float(np.dot(ybar, shots_gaussian(uu * uu, n_shots, z)))

    ubar = np.empty_like(u)
    for b in range(len(u)):
        up, um = u.copy(), u.copy()
        up[b] += h
        um[b] -= h
        ubar[b] = (L(up) - L(um)) / (2 * h)
    lam = np.zeros_like(psi)
    nz = u > 0
    lam[nz] = ubar[nz] * psi[nz] / (2 * u[nz])
    return lam
