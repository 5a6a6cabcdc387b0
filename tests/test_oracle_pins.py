"""Pins of the CPU oracle against facts that do not come from the oracle.

Each check ties one part of the oracle to something fixed by the paper or by
mathematics: closed forms (GHZ, QFT on basis states, Bloch-sphere rotations),
textbook Pauli expectation values, an independent dense construction of every
gate (matrix exponentials of Pauli generators, projector forms of controlled
gates, the SWAP Pauli identity, MoveDim-style tensor contraction for general
unitaries), unitarity and invertibility (Sec. 4.4), three gradient routes that
share nothing (parameter shift, stored-activation reverse pass, central finite
differences), and the hand-derived result of the appendix's basic listing.
The planted-mistake tests at the end edit the oracle source and check that at
least one pin fails.
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.linalg as sla

import oracle
from paper_2511_19291_gb300 import workloads as W

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

# ----------------------------------------------------------------- dense kit
I2 = np.eye(2, dtype=complex)
PX = np.array([[0, 1], [1, 0]], dtype=complex)
PY = np.array([[0, -1j], [1j, 0]], dtype=complex)
PZ = np.array([[1, 0], [0, -1]], dtype=complex)
P0 = np.array([[1, 0], [0, 0]], dtype=complex)
P1 = np.array([[0, 0], [0, 1]], dtype=complex)


def on(n, q, m):
    """Full-space operator of a single-qubit matrix on qubit q (qubit 0 is the
    least significant bit, so it is the last Kronecker factor)."""
    out = np.array([[1.0 + 0j]])
    for k in range(n - 1, -1, -1):
        out = np.kron(out, m if k == q else I2)
    return out


def contract(n, wires, m):
    """Full-space operator of a k-qubit matrix through the tensor view of the
    state (Algorithm 1): reshape to [2]*n, move the wire axes to the front in
    order, multiply, move them back."""
    N = 1 << n
    U = np.empty((N, N), dtype=complex)
    k = len(wires)
    axes = [n - 1 - w for w in wires]  # tensor axis of qubit w (C order)
    for j in range(N):
        e = np.zeros(N, dtype=complex)
        e[j] = 1
        t = e.reshape([2] * n)
        t = np.moveaxis(t, axes, list(range(k)))
        t = (m @ t.reshape(1 << k, -1)).reshape([2] * n)
        t = np.moveaxis(t, list(range(k)), axes)
        U[:, j] = t.reshape(N)
    return U


def dense_gate(n, g, params):
    th = params[g.param] if g.param >= 0 else g.angle
    N = 1 << n
    Id = np.eye(N, dtype=complex)
    k, w = g.kind, g.wires
    if k == "H":
        return on(n, w[0], (PX + PZ) / math.sqrt(2))
    if k in ("X", "Y", "Z"):
        return on(n, w[0], {"X": PX, "Y": PY, "Z": PZ}[k])
    if k == "S":
        return on(n, w[0], sla.expm(1j * (math.pi / 2) * P1))
    if k == "T":
        return on(n, w[0], sla.expm(1j * (math.pi / 4) * P1))
    if k in ("RX", "RY", "RZ"):
        P = {"RX": PX, "RY": PY, "RZ": PZ}[k]
        return on(n, w[0], sla.expm(-0.5j * th * P))
    if k == "PHASE":
        return on(n, w[0], sla.expm(1j * th * P1))
    if k == "CNOT":
        c, t = w
        return on(n, c, P0) + on(n, c, P1) @ on(n, t, PX)
    if k == "CZ":
        a, b = w
        return Id - 2 * on(n, a, P1) @ on(n, b, P1)
    if k == "CPHASE":
        a, b = w
        return sla.expm(1j * th * on(n, a, P1) @ on(n, b, P1))
    if k == "SWAP":
        a, b = w
        return 0.5 * (Id + on(n, a, PX) @ on(n, b, PX) + on(n, a, PY) @ on(n, b, PY)
                      + on(n, a, PZ) @ on(n, b, PZ))
    if k in ("UNITARY1", "UNITARY2"):
        return contract(n, list(w), np.asarray(g.matrix))
    raise AssertionError(k)


def dense_pauli(n, term):
    m = np.eye(1 << n, dtype=complex)
    for q, p in term.ops:
        m = m @ on(n, q, {"X": PX, "Y": PY, "Z": PZ}[p])
    return term.coeff * m


def dense_observable(n, terms):
    return sum(dense_pauli(n, t) for t in terms)


# ------------------------------------------------------------ closed forms
@pytest.mark.parametrize("n", [1, 2, 3, 5, 8])
def test_ghz_closed_form(n):
    psi = oracle.run(W.ghz_circuit(n))
    ref = np.zeros(1 << n, dtype=complex)
    ref[0] = ref[-1] = 1 / math.sqrt(2)
    np.testing.assert_allclose(psi, ref, atol=1e-14)


def qft_closed_form(n, j):
    N = 1 << n
    k = np.arange(N)
    return np.exp(2j * math.pi * j * k / N) / math.sqrt(N)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6])
def test_qft_all_basis_states(n):
    circ = W.qft_circuit(n)
    for j in range(1 << n):
        np.testing.assert_allclose(oracle.run(circ, None, j), qft_closed_form(n, j), atol=1e-12)


def test_qft_sampled_basis_states_n12():
    circ = W.qft_circuit(12)
    for j in (0, 1, 7, 1234, 4095, 2048, 3001):
        np.testing.assert_allclose(oracle.run(circ, None, j), qft_closed_form(12, j), atol=1e-12)


def bloch(psi):
    terms = [W.PauliTerm(1.0, ((0, p),)) for p in "XYZ"]
    return oracle.expval(1, psi, terms)[1]


@pytest.mark.parametrize("th", [0.0, 0.3, 1.1, 2.5, -0.7, 4.0])
def test_rotation_directions_on_bloch_sphere(th):
    """R_P(t) = exp(-i t P/2) turns the Bloch vector by t about axis P
    (right-hand rule); |0> is (0, 0, 1), |+> = H|0> is (1, 0, 0)."""
    one = lambda k: W.Circuit(1, [W.Gate(k, (0,), param=0)], 1)
    np.testing.assert_allclose(bloch(oracle.run(one("RX"), [th])), [0, -math.sin(th), math.cos(th)], atol=1e-13)
    np.testing.assert_allclose(bloch(oracle.run(one("RY"), [th])), [math.sin(th), 0, math.cos(th)], atol=1e-13)
    np.testing.assert_allclose(bloch(oracle.run(one("RZ"), [th])), [0, 0, 1], atol=1e-13)
    for k in ("RZ", "PHASE"):
        c = W.Circuit(1, [W.Gate("H", (0,)), W.Gate(k, (0,), param=0)], 1)
        np.testing.assert_allclose(bloch(oracle.run(c, [th])), [math.cos(th), math.sin(th), 0], atol=1e-13)


def test_fixed_gates_on_bloch_sphere():
    def vec(*kinds):
        return bloch(oracle.run(W.Circuit(1, [W.Gate(k, (0,)) for k in kinds], 0)))
    np.testing.assert_allclose(vec("H"), [1, 0, 0], atol=1e-14)
    np.testing.assert_allclose(vec("X"), [0, 0, -1], atol=1e-14)
    np.testing.assert_allclose(vec("H", "S"), [0, 1, 0], atol=1e-14)       # S: quarter turn about z
    np.testing.assert_allclose(vec("H", "T"), [1 / math.sqrt(2), 1 / math.sqrt(2), 0], atol=1e-14)
    np.testing.assert_allclose(vec("H", "Z"), [-1, 0, 0], atol=1e-14)
    np.testing.assert_allclose(vec("Y"), [0, 0, -1], atol=1e-14)
    np.testing.assert_allclose(vec("H", "Y"), [-1, 0, 0], atol=1e-14)


def test_bell_state_pauli_values():
    c = W.Circuit(2, [W.Gate("H", (0,)), W.Gate("CNOT", (0, 1))], 0)
    psi = oracle.run(c)
    terms = [W.PauliTerm(1.0, ((0, "X"), (1, "X"))), W.PauliTerm(1.0, ((0, "Y"), (1, "Y"))),
             W.PauliTerm(1.0, ((0, "Z"), (1, "Z"))), W.PauliTerm(1.0, ((0, "Z"),)),
             W.PauliTerm(1.0, ((1, "X"),)), W.PauliTerm(1.0, ((0, "X"), (1, "Y")))]
    np.testing.assert_allclose(oracle.expval(2, psi, terms)[1], [1, -1, 1, 0, 0, 0], atol=1e-14)


def test_controlled_gates_truth_tables():
    # CNOT(c, t) flips t exactly when c is 1; wires[0] is the control.
    for c, t in ((0, 1), (1, 0), (0, 2), (2, 1)):
        circ = W.Circuit(3, [W.Gate("CNOT", (c, t))], 0)
        for j in range(8):
            out = np.abs(oracle.run(circ, None, j))
            expect = j ^ (1 << t) if (j >> c) & 1 else j
            assert out[expect] == pytest.approx(1.0) and out.sum() == pytest.approx(1.0)
    # SWAP exchanges bits; CZ and CPHASE act only on |11>.
    for j in range(8):
        out = oracle.run(W.Circuit(3, [W.Gate("SWAP", (0, 2))], 0), None, j)
        b0, b2 = j & 1, (j >> 2) & 1
        swapped = (j & 0b010) | (b0 << 2) | b2
        assert abs(out[swapped]) == pytest.approx(1.0)
        out = oracle.run(W.Circuit(3, [W.Gate("CPHASE", (2, 1), angle=0.7)], 0), None, j)
        phase = np.exp(0.7j) if (j >> 2) & 1 and (j >> 1) & 1 else 1.0
        assert out[j] == pytest.approx(phase)


def test_basic_example_golden():
    with open(os.path.join(GOLDEN, "basic_example.json")) as f:
        g = json.load(f)
    n = g["n_qubits"]
    gates = [W.Gate(k, tuple(w), angle=a) for k, w, a in g["gates"]]
    psi = oracle.run(W.Circuit(n, gates, 0))
    np.testing.assert_allclose(oracle.expval(n, psi, W.all_z_terms(n))[1], g["expected_allZ"], atol=1e-14)


def test_zero_angle_ansatz_values():
    for n in (3, 6, 9):
        circ = W.hea_ansatz(n, 3)
        zero = np.zeros(circ.n_params)
        assert oracle.energy(circ, zero, W.sum_z(n)) == pytest.approx(n, abs=1e-13)
        assert oracle.energy(circ, zero, W.ising(n)) == pytest.approx(n - 1, abs=1e-13)


# -------------------------------------------------- independent dense checks
@pytest.mark.parametrize("seed", range(4))
def test_every_gate_against_dense_construction(seed):
    rng = W.SplitMix64(100 + seed)
    n = 4
    circ, params = W.random_circuit(rng, n, 60)
    for g in circ.gates:
        np.testing.assert_allclose(oracle.gate_dense(n, g, params), dense_gate(n, g, params), atol=1e-13,
                                   err_msg=str(g))


@pytest.mark.parametrize("n,ng,seed", [(3, 40, 1), (5, 80, 2), (6, 120, 3), (8, 60, 4)])
def test_circuit_against_dense_product(n, ng, seed):
    rng = W.SplitMix64(200 + seed)
    circ, params = W.random_circuit(rng, n, ng)
    U = np.eye(1 << n, dtype=complex)
    for g in circ.gates:
        U = dense_gate(n, g, params) @ U
    for j in (0, (1 << n) - 1, 5 % (1 << n)):
        np.testing.assert_allclose(oracle.run(circ, params, j), U[:, j], atol=1e-12)


@pytest.mark.parametrize("n,seed", [(2, 1), (4, 2), (6, 3)])
def test_expval_and_observable_against_dense(n, seed):
    rng = W.SplitMix64(300 + seed)
    circ, params = W.random_circuit(rng, n, 30)
    psi = oracle.run(circ, params)
    terms = W.random_pauli_terms(rng, n, 12) + W.ising(n)
    H = dense_observable(n, terms)
    e, per = oracle.expval(n, psi, terms)
    assert e == pytest.approx(np.real(np.vdot(psi, H @ psi)), abs=1e-12)
    for t, v in zip(terms, per):
        assert v == pytest.approx(np.real(np.vdot(psi, dense_pauli(n, t) @ psi)) / t.coeff, abs=1e-12)
    np.testing.assert_allclose(oracle.apply_observable(n, psi, terms), H @ psi, atol=1e-12)


# ----------------------------------------------------- unitarity / inverse
@pytest.mark.parametrize("n,seed", [(7, 1), (10, 2)])
def test_norm_preserved_and_inverse_returns_start(n, seed):
    rng = W.SplitMix64(400 + seed)
    circ, params = W.random_circuit(rng, n, 200)
    psi = oracle.run(circ, params, 3)
    assert oracle.norm2(n, psi) == pytest.approx(1.0, abs=1e-13)
    back = oracle.unapply(circ, params, psi)
    ref = np.zeros(1 << n, dtype=complex)
    ref[3] = 1
    np.testing.assert_allclose(back, ref, atol=1e-12)


# ---------------------------------------------------------------- gradients
def test_gradient_closed_form_single_qubit():
    for k, f in (("RX", lambda t: -math.sin(t)), ("RY", lambda t: -math.sin(t))):
        c = W.Circuit(1, [W.Gate(k, (0,), param=0)], 1)
        for th in (0.2, 1.3, 2.9):
            g = oracle.grad_param_shift(c, [th], W.sum_z(1))
            assert g[0] == pytest.approx(f(th), abs=1e-13)
            assert oracle.grad_stored(c, [th], W.sum_z(1))[1][0] == pytest.approx(f(th), abs=1e-13)


def finite_difference(circ, params, terms, h=1e-4):
    g = np.zeros(circ.n_params)
    for k in range(circ.n_params):
        p = np.array(params, dtype=float)
        p[k] += h
        ep = oracle.energy(circ, p, terms)
        p[k] -= 2 * h
        em = oracle.energy(circ, p, terms)
        g[k] = (ep - em) / (2 * h)
    return g


@pytest.mark.parametrize("n,ng,seed", [(3, 30, 1), (5, 50, 2), (6, 40, 3)])
def test_three_gradient_routes_agree(n, ng, seed):
    rng = W.SplitMix64(500 + seed)
    circ, params = W.random_circuit(rng, n, ng, n_params=12)
    terms = W.random_pauli_terms(rng, n, 6) + W.ising(n)
    gs = oracle.grad_param_shift(circ, params, terms)
    e, ga = oracle.grad_stored(circ, params, terms)
    gf = finite_difference(circ, params, terms)
    assert e == pytest.approx(oracle.energy(circ, params, terms), abs=1e-12)
    np.testing.assert_allclose(gs, ga, atol=1e-11)
    np.testing.assert_allclose(gs, gf, atol=1e-6)


def test_ansatz_gradient_routes_agree():
    circ = W.hea_ansatz(6, 3)
    params = W.config_rng(3).angles(circ.n_params)
    terms = W.ising(6)
    gs = oracle.grad_param_shift(circ, params, terms)
    _, ga = oracle.grad_stored(circ, params, terms)
    np.testing.assert_allclose(gs, ga, atol=1e-11)
    np.testing.assert_allclose(gs, finite_difference(circ, params, terms), atol=1e-6)


# ------------------------------------------------------- planted mistakes
MUTATIONS = [
    ("RY sign", "case O_RY: M[0] = c; M[1] = -s; M[2] = s;", "case O_RY: M[0] = c; M[1] = s; M[2] = -s;"),
    ("RX phase", "case O_RX: M[0] = c; M[1] = -I * s;", "case O_RX: M[0] = c; M[1] = I * s;"),
    ("RZ half angle", "case O_RZ: M[0] = cexp(-0.5 * I * t);", "case O_RZ: M[0] = cexp(-1.0 * I * t);"),
    ("Y matrix", "case O_Y:  M[1] = -I; M[2] = I;", "case O_Y:  M[1] = I; M[2] = -I;"),
    ("CNOT wires", "case O_CNOT: M[0] = 1; M[5] = 1; M[11] = 1; M[14] = 1;",
     "case O_CNOT: M[0] = 1; M[15] = 1; M[6] = 1; M[9] = 1;"),
    ("wire order", "if ((l >> (k - 1 - i)) & 1)", "if ((l >> i) & 1)"),
    ("transposed matvec", "acc += M[r * d + c] * v[c];", "acc += M[c * d + r] * v[c];"),
    ("expval conj", "acc += conj(a[i]) * b[i];", "acc += a[i] * b[i];"),
    ("pauli Y", "if (op == 2) { P[1] = -I; P[2] = I; }", "if (op == 2) { P[1] = I; P[2] = -I; }"),
    ("dropped coeff", "total += coeffs[j] * e;", "total += e;"),
    ("shift half", "contrib[g] = 0.5 * (ep - em);", "contrib[g] = (ep - em);"),
    ("stored factor", "grad[gg->param] += 2.0 * creal(inner(n, lam, tmp));",
     "grad[gg->param] += creal(inner(n, lam, tmp));"),
    ("adjoint not conj", "Md[i * d + j] = conj(M[j * d + i]);", "Md[i * d + j] = M[j * d + i];"),
    ("dRY", "case O_RY: D[0] = -0.5 * s; D[1] = -0.5 * c; D[2] = 0.5 * c;",
     "case O_RY: D[0] = -0.5 * s; D[1] = 0.5 * c; D[2] = -0.5 * c;"),
]


def pin_suite():
    """A compact run of the pins above; returns the names that fail."""
    failed = []
    checks = {
        "bloch": lambda: [test_rotation_directions_on_bloch_sphere(t) for t in (0.3, 2.5)],
        "fixed": test_fixed_gates_on_bloch_sphere,
        "bell": test_bell_state_pauli_values,
        "truth": test_controlled_gates_truth_tables,
        "qft": lambda: test_qft_all_basis_states(3),
        "dense": lambda: test_every_gate_against_dense_construction(0),
        "product": lambda: test_circuit_against_dense_product(3, 40, 1),
        "observable": lambda: test_expval_and_observable_against_dense(4, 2),
        "inverse": lambda: test_norm_preserved_and_inverse_returns_start(7, 1),
        "grad": lambda: test_three_gradient_routes_agree(3, 30, 1),
        "grad1": test_gradient_closed_form_single_qubit,
    }
    for name, fn in checks.items():
        try:
            fn()
        except AssertionError:
            failed.append(name)
    return failed


def test_unmutated_source_passes_compact_pins():
    assert pin_suite() == []


@pytest.mark.parametrize("name,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_is_caught(tmp_path, name, old, new):
    src = oracle.oracle.source_text()
    assert src.count(old) == 1, f"mutation anchor for {name!r} not found exactly once"
    path = oracle.oracle.build_variant(src.replace(old, new), str(tmp_path / "mut.so"))
    with oracle.oracle.use_library(path):
        failed = pin_suite()
    assert failed, f"planted mistake {name!r} passed every pin"
