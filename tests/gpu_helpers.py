"""Shared helpers of the GPU parity tests (no arithmetic of the method)."""
import numpy as np
import torch

from paper_2511_19291_gb300 import workloads as W

DTYPES = {"c64": torch.complex64, "c128": torch.complex128}
# Tolerances of the CUDA path against the oracle: 1e-5 absolute on
# expectations and 1e-4 relative on gradients for complex64, 1e-12 for
# complex128 (gradients 1e-10 relative).
AMP_TOL = {"c64": 2e-6, "c128": 1e-12}
E_TOL = {"c64": 1e-5, "c128": 1e-12}
G_REL = {"c64": 1e-4, "c128": 1e-10}


def sim():
    from paper_2511_19291_gb300 import sim as S
    return S


def params_tensor(params):
    return torch.tensor(np.asarray(params, dtype=np.float64), dtype=torch.float64, device="cuda")


def gpu_state(circ, params, mode="fused", dtype="c64", basis=0, **kw):
    S = sim()
    c = S.Circuit(circ, mode=mode, **kw)
    st = S.State(circ.n_qubits, DTYPES[dtype]).reset(basis)
    p = params_tensor(params if params is not None else np.zeros(max(1, circ.n_params)))
    S.apply(st, c, p)
    return st, c, p


def to_numpy(state):
    torch.cuda.synchronize()
    return state.tensor.detach().cpu().numpy().astype(np.complex128)


def grad_close(g, ref, rel, hnorm=None):
    """|g - ref| <= rel * max(|ref|, 1e-2 * max|ref|) componentwise; with
    hnorm = ||H||_1 a component also passes when |g - ref| <= 1e-6 * ||H||_1
    (complex64 error stated against the observable's scale)."""
    g = np.asarray(g)
    ref = np.asarray(ref)
    floor = 1e-2 * (np.max(np.abs(ref)) if ref.size else 0.0)
    bound = rel * np.maximum(np.abs(ref), floor) + 1e-300
    if hnorm is not None:
        bound = np.maximum(bound, 1e-6 * hnorm)
    bad = np.abs(g - ref) > bound
    return not bad.any(), np.max(np.abs(g - ref) / bound) if ref.size else 0.0


def all_kinds_circuit(seed, n, ng, n_params=None):
    return W.random_circuit(W.SplitMix64(seed), n, ng, n_params=n_params)
