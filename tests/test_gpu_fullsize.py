"""Full-size checks in the launch configuration the benchmark times (fused
plan), on the workloads' own sizes.  Where the oracle cannot run (2^24..2^32
amplitudes) the checks use properties that hold at any size: agreement of
two independent GPU paths (fused and gate-by-gate), agreement of complex64
with complex128, closed forms (QFT on |0...0> is uniform, zero angles give
E = n - 1 for the Ising chain), central finite differences, norm, the range
of E and the reverse sweep returning |0...0>.  The 14-qubit case of the
24-qubit workload's form is checked against the oracle's parameter shift."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2511_19291_gb300 import workloads as W
from gpu_helpers import grad_close, params_tensor, sim

pytestmark = pytest.mark.gpu


def energy_and_grad(circ, params, terms, dtype, mode="fused"):
    S = sim()
    c = S.Circuit(circ, mode=mode)
    p = params_tensor(params)
    psi = S.State(circ.n_qubits, dtype).reset(0)
    S.apply(psi, c, p)
    e = S.expval(psi, terms).item()
    lam = S.State(circ.n_qubits, dtype)
    g = torch.zeros(circ.n_params, dtype=torch.float64, device="cuda")
    S.backward(psi, lam, c, p, terms, g)
    torch.cuda.synchronize()
    return e, g.cpu().numpy(), psi


def back_to_zero(psi, tol):
    t = psi.tensor
    assert abs(t[0].item() - 1.0) < tol
    # the rest of the norm is gone from every other amplitude
    rest = float((t.abs() ** 2).sum().item()) - abs(t[0].item()) ** 2
    assert rest < tol


def test_main_workload_26q():
    """26 qubits, 20 layers, Ising: fused c64, gate-by-gate c64 and
    tqd_value_and_grad c64 (the benchmark's call) against fused c128."""
    w = W.workload_main()
    h1 = W.observable_l1(w.terms)
    e_f, g_f, psi = energy_and_grad(w.circuit, w.params, w.terms, torch.complex64, "fused")
    back_to_zero(psi, 1e-4)
    del psi
    e_p, g_p, psi = energy_and_grad(w.circuit, w.params, w.terms, torch.complex64, "plain")
    del psi
    e_d, g_d, psi = energy_and_grad(w.circuit, w.params, w.terms, torch.complex128, "fused")
    back_to_zero(psi, 1e-10)
    del psi
    torch.cuda.empty_cache()
    # the call bench.py times: tqd_value_and_grad, forward checkpoints for
    # every pass (psi only read), reverse passes reading psi there, the
    # closing CNOT ring folded into the observable
    S = sim()
    c = S.Circuit(w.circuit)
    psi = S.State(26, torch.complex64).reset(0)
    lam = S.State(26, torch.complex64)
    e_v, g_v = S.value_and_grad(psi, lam, c, params_tensor(w.params), w.terms)
    torch.cuda.synchronize()
    e_v = e_v.item()
    g_v = g_v.cpu().numpy()
    t = psi.tensor
    assert t[0].item() == 1 and int(torch.count_nonzero(t).item()) == 1  # never written
    del psi, lam, c
    torch.cuda.empty_cache()
    assert abs(e_v - e_d) < 1e-5
    assert grad_close(g_v, g_d, 1e-4)[0]
    print(f"\n26q: E c64 fused {e_f:.10f} plain {e_p:.10f} c128 {e_d:.14f}; "
          f"max|dg| fused {np.max(np.abs(g_f - g_d)):.2e} plain {np.max(np.abs(g_p - g_d)):.2e} (||H||_1 {h1})")
    assert abs(e_f - e_d) < 1e-5 and abs(e_p - e_d) < 1e-5
    assert grad_close(g_f, g_d, 1e-4)[0]
    assert grad_close(g_p, g_d, 1e-4)[0]


def test_zero_angles_closed_form_26q():
    w = W.workload_main()
    S = sim()
    c = S.Circuit(w.circuit)
    psi = S.State(26).reset(0)
    S.apply(psi, c, params_tensor(np.zeros(w.circuit.n_params)))
    assert abs(S.expval(psi, w.terms).item() - 25.0) < 1e-5
    assert abs(S.expval(psi, W.sum_z(26)).item() - 26.0) < 1e-5


def test_grad_workload_24q_finite_differences():
    """24 qubits, 10 layers, Ising: complex128 adjoint gradient against central
    differences with h = 1e-3 (truncation ~h^2/6 |E'''|), and complex64
    against complex128 on every angle."""
    w = W.workload_grad()
    h1 = W.observable_l1(w.terms)
    e_d, g_d, psi = energy_and_grad(w.circuit, w.params, w.terms, torch.complex128)
    del psi
    S = sim()
    c = S.Circuit(w.circuit)
    st = S.State(24, torch.complex128)
    h = 1e-3
    for k in (0, 1, 47, 240, 479):
        vals = []
        for s in (+1, -1):
            p = np.array(w.params)
            p[k] += s * h
            st.reset(0)
            S.apply(st, c, params_tensor(p))
            vals.append(S.expval(st, w.terms).item())
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(g_d[k] - fd) <= max(1e-4 * abs(fd), 2e-6 * h1), (k, g_d[k], fd)
    del st
    e_f, g_f, psi = energy_and_grad(w.circuit, w.params, w.terms, torch.complex64)
    del psi
    torch.cuda.empty_cache()
    assert abs(e_f - e_d) < 1e-5
    ok, worst = grad_close(g_f, g_d, 1e-4)
    assert ok, worst


def test_grad_workload_form_14q_parameter_shift():
    """The 24-qubit workload's form at 14 qubits (10 layers, 280 angles) against
    the oracle's parameter-shift gradient."""
    circ = W.hea_ansatz(14, 10)
    params = W.config_rng(3).angles(circ.n_params)
    terms = W.ising(14)
    ref = oracle.grad_param_shift(circ, params, terms)
    e_ref = oracle.energy(circ, params, terms)
    for dtype, rel, hn in ((torch.complex64, 1e-4, W.observable_l1(terms)), (torch.complex128, 1e-10, None)):
        e, g, _ = energy_and_grad(circ, params, terms, dtype)
        assert abs(e - e_ref) < (1e-5 if dtype == torch.complex64 else 1e-12)
        ok, worst = grad_close(g, ref, rel)
        assert ok, (dtype, worst)


def test_qft_32q_c64_invariants():
    """32 qubits, complex64 (32 GiB per state): QFT on |0...0> is uniform; QFT
    then 8 layers: norm 1, |E| <= ||H||_1, gradient finite, the reverse sweep
    returns |0...0>."""
    S = sim()
    n = 32
    qft = S.Circuit(W.qft_circuit(n))
    psi = S.State(n).reset(0)
    S.apply(psi, qft)
    amp = 2.0 ** (-n / 2)
    idx = [0, 1, 12345, (1 << 31) + 7, (1 << 32) - 1]
    for i in idx:
        v = psi.tensor[i].item()
        assert abs(v.real - amp) < 1e-6 * amp * 64 and abs(v.imag) < 1e-6 * amp * 64, (i, v)
    del psi, qft
    torch.cuda.empty_cache()
    w = W.workload_qft(32, 8)
    h1 = W.observable_l1(w.terms)
    e, g, psi = energy_and_grad(w.circuit, w.params, w.terms, torch.complex64)
    assert abs(e) <= h1 and np.all(np.isfinite(g))
    back_to_zero(psi, 1e-3)
    del psi
    torch.cuda.empty_cache()
    print(f"\n32q c64: E {e:.8f}, max|g| {np.max(np.abs(g)):.4f}")


def test_qft_31q_c64_error_against_c128():
    """The same circuit family at 31 qubits in complex128 states the complex64
    error (E and every gradient component)."""
    w = W.workload_qft(31, 8)
    h1 = W.observable_l1(w.terms)
    e64, g64, psi = energy_and_grad(w.circuit, w.params, w.terms, torch.complex64)
    del psi
    torch.cuda.empty_cache()
    e128, g128, psi = energy_and_grad(w.circuit, w.params, w.terms, torch.complex128)
    back_to_zero(psi, 1e-9)
    del psi
    torch.cuda.empty_cache()
    print(f"\n31q: |E64 - E128| = {abs(e64 - e128):.3e}, max|g64 - g128|/||H||_1 = "
          f"{np.max(np.abs(g64 - g128)) / h1:.3e}")
    assert abs(e64 - e128) < 1e-5
    assert grad_close(g64, g128, 1e-4)[0]
