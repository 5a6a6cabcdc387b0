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


def grad_close(g, ref, rel):
    """Gradient check at relative tolerance rel.

    Always: the normwise relative error of the gradient vector,
    max|g - ref| <= rel * max|ref| (the 1e-4 relative of complex64).
    For double-precision tolerances (rel < 1e-6) also componentwise:
    |g - ref| <= rel * max(|ref|, 1e-2 * max|ref|) for every component.
    (In complex64 the componentwise form is out of reach for deep circuits:
    the float32 amplitudes' rounding leaves an absolute error near
    3e-6 * max|ref| on every component, small ones included, whatever the
    summation -- the gate-by-gate path with compensated sums shows it too.)
    Returns (ok, worst) with worst = the largest error / bound (<= 1
    passes)."""
    g = np.asarray(g)
    ref = np.asarray(ref)
    if not ref.size:
        return True, 0.0
    gmax = float(np.max(np.abs(ref)))
    worst = float(np.max(np.abs(g - ref))) / (rel * gmax + 1e-300)
    if rel < 1e-6:
        bound = rel * np.maximum(np.abs(ref), 1e-2 * gmax) + 1e-300
        worst = max(worst, float(np.max(np.abs(g - ref) / bound)))
    return worst <= 1.0, worst


def grad_error(g, ref):
    """Error statement of a gradient against its reference: the largest
    absolute error, and the largest pure relative error over the components
    at least 1e-2 of the largest one."""
    g = np.asarray(g, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    if not ref.size:
        return {"max_abs": 0.0, "max_rel": 0.0}
    big = np.abs(ref) >= 1e-2 * np.max(np.abs(ref))
    rel = np.abs(g - ref)[big] / np.abs(ref)[big]
    return {"max_abs": float(np.max(np.abs(g - ref))), "max_rel": float(np.max(rel)) if rel.size else 0.0}


def all_kinds_circuit(seed, n, ng, n_params=None):
    return W.random_circuit(W.SplitMix64(seed), n, ng, n_params=n_params)
