"""The headline workloads against stored oracle values.

``tests/golden/*.json`` hold values written by ``tests/golden/make_golden.py``,
which runs only the complex128 CPU oracle (gate by gate, Sec. 4.1 and
Algorithm 1; expectation by definition, Sec. 2.2.1; derivatives by the
parameter-shift rule, independent of any adjoint code).  Here the library's
complex64 path is run in the configuration the benchmark times and compared
with them: 1e-5 absolute on E, 1e-4 relative on every gradient component
(floor: 1e-2 of the largest reference component), and the error is printed
per result.
"""
import json
import os

import numpy as np
import pytest
import torch

from paper_2511_19291_gb300 import workloads as W
from gpu_helpers import E_TOL, G_REL, grad_close, grad_error, params_tensor, sim

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def value_and_grad_c64(w):
    """The benchmark's call: tqd_value_and_grad on complex64 states."""
    S = sim()
    c = S.Circuit(w.circuit)
    n = w.circuit.n_qubits
    psi = S.State(n, torch.complex64).reset(0)
    lam = S.State(n, torch.complex64)
    e, g = S.value_and_grad(psi, lam, c, params_tensor(w.params), w.terms)
    torch.cuda.synchronize()
    out = e.item(), g.cpu().numpy()
    del psi, lam, c
    torch.cuda.empty_cache()
    return out


def check_sampled(name, w, e, g):
    ref = load(name)
    assert ref["n_qubits"] == w.circuit.n_qubits and ref["n_params"] == w.circuit.n_params
    idx = np.array(ref["grad_indices"])
    g_ref = np.array(ref["grad"])
    de = abs(e - ref["energy"])
    err = grad_error(g[idx], g_ref)
    print(f"\n{name}: |E - E_oracle| = {de:.3e} (E_oracle {ref['energy']:.12f}); sampled gradient "
          f"max abs err {err['max_abs']:.3e}, max rel err {err['max_rel']:.3e}")
    assert de <= E_TOL["c64"], de
    ok, worst = grad_close(g[idx], g_ref, G_REL["c64"])
    assert ok, (worst, list(zip(idx.tolist(), g[idx].tolist(), g_ref.tolist())))


def test_main_workload_26q_against_oracle():
    """26 qubits, 20 layers, Ising H: E and 8 gradient components from
    tqd_value_and_grad (forward checkpoints, ring kernels, pass-specialised
    kernels) against the oracle's E and parameter-shift components."""
    w = W.workload_main()
    e, g = value_and_grad_c64(w)
    check_sampled("hea26x20_ising.json", w, e, g)


def test_grad_workload_24q_against_oracle():
    """24 qubits, 10 layers, Ising H through the autograd.Function (the
    benchmark's grad24 path) against the oracle's E and 8 parameter-shift
    components."""
    S = sim()
    w = W.workload_grad()
    c = S.Circuit(w.circuit)
    theta = params_tensor(w.params).requires_grad_(True)
    e = S.expval_fn(theta, c, w.terms)
    e.backward()
    torch.cuda.synchronize()
    check_sampled("hea24x10_ising.json", w, e.item(), theta.grad.cpu().numpy())


def test_grad_workload_form_20q_full_gradient_against_oracle():
    """The 24-qubit workload's form at 20 qubits (10 layers, 400 angles):
    every gradient component against the oracle's parameter shift."""
    ref = load("hea20x10_ising_grad.json")
    w = W.workload_hea(3, 20, 10, "ising")
    assert ref["n_params"] == w.circuit.n_params
    e, g = value_and_grad_c64(w)
    g_ref = np.array(ref["grad"])
    err = grad_error(g, g_ref)
    print(f"\n20q: |E - E_oracle| = {abs(e - ref['energy']):.3e}; gradient max abs err {err['max_abs']:.3e}, "
          f"max rel err {err['max_rel']:.3e} over {len(g_ref)} components")
    assert abs(e - ref["energy"]) <= E_TOL["c64"]
    ok, worst = grad_close(g, g_ref, G_REL["c64"])
    assert ok, worst


def test_small_workload_12q_against_oracle():
    """12 qubits, 4 layers, sum_i Z_i (one tile: the launch-bound end of the
    range): the forward evaluation's E through tqd_expval and the whole
    gradient through tqd_value_and_grad against the oracle's stored values."""
    S = sim()
    ref = load("hea12x4_sumz_grad.json")
    w = W.workload_small()
    assert ref["n_params"] == w.circuit.n_params
    c = S.Circuit(w.circuit)
    st = S.State(12, torch.complex64).reset(0)
    S.apply(st, c, params_tensor(w.params))
    e_fwd = S.expval(st, w.terms).item()
    e, g = value_and_grad_c64(w)
    g_ref = np.array(ref["grad"])
    err = grad_error(g, g_ref)
    print(f"\n12q: |E - E_oracle| = {abs(e_fwd - ref['energy']):.3e} (forward), {abs(e - ref['energy']):.3e} "
          f"(value_and_grad); gradient max abs err {err['max_abs']:.3e}, max rel err {err['max_rel']:.3e}")
    assert abs(e_fwd - ref["energy"]) <= E_TOL["c64"]
    assert abs(e - ref["energy"]) <= E_TOL["c64"]
    ok, worst = grad_close(g, g_ref, G_REL["c64"])
    assert ok, worst
