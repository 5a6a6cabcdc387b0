"""Seeded, synthetic circuit and observable builders.

This module only *describes* inputs: gate lists, angle vectors and Pauli-sum
observables.  It performs none of the simulation arithmetic (no gate
application, no expectation value, no gradient), so that the CUDA path and the
independent CPU oracle can both be fed from it without sharing any of the
method's computation.

Conventions (shared by every consumer of these descriptions):

* Qubit ``i`` is bit ``i`` of the flat amplitude index (qubit 0 = least
  significant bit).  The paper's state tensor (Sec. 4.1, "Tensor dimension
  order") does not fix which tensor dimension is which qubit; only raw
  amplitude dumps depend on this choice.
* A gate is the ordered pair (unitary, ordered qubit list) of Sec. 4.1.  For a
  multi-qubit gate, ``wires[0]`` is the most significant bit of the gate's
  local index (the first dimension moved to the front by MoveDim in
  Algorithm 1); for CNOT ``wires = (control, target)`` as in the appendix
  listings.
* Rotations are ``R_P(theta) = exp(-i theta P / 2)`` (the Pauli-rotation gates
  of Sec. 3, "Extensible"); ``PHASE(theta) = diag(1, e^{i theta})`` and
  ``CPHASE(theta) = diag(1, 1, 1, e^{i theta})``.
* Angles are drawn from a splitmix64 stream: 53-bit uniform doubles times 2*pi.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Iterable, Sequence

import numpy as np

GATE_KINDS = (
    "H", "X", "Y", "Z", "S", "T",
    "RX", "RY", "RZ", "PHASE",
    "CNOT", "CZ", "CPHASE", "SWAP",
    "UNITARY1", "UNITARY2",
)
GATE_ARITY = {
    "H": 1, "X": 1, "Y": 1, "Z": 1, "S": 1, "T": 1,
    "RX": 1, "RY": 1, "RZ": 1, "PHASE": 1,
    "CNOT": 2, "CZ": 2, "CPHASE": 2, "SWAP": 2,
    "UNITARY1": 1, "UNITARY2": 2,
}
PARAMETRIC = frozenset({"RX", "RY", "RZ", "PHASE", "CPHASE"})


@dataclass(frozen=True)
class Gate:
    """One gate: kind, ordered wires, and where its angle comes from.

    ``param >= 0`` reads the angle from the parameter vector at that index;
    ``param == -1`` uses ``angle``.  ``matrix`` (complex, row-major) is only
    used by UNITARY1 (2x2) and UNITARY2 (4x4).
    """
    kind: str
    wires: tuple
    param: int = -1
    angle: float = 0.0
    matrix: object = None

    def __post_init__(self):
        if self.kind not in GATE_ARITY:
            raise ValueError(f"unknown gate kind {self.kind!r}")
        if len(self.wires) != GATE_ARITY[self.kind]:
            raise ValueError(f"{self.kind} takes {GATE_ARITY[self.kind]} wires, got {self.wires}")
        if self.param >= 0 and self.kind not in PARAMETRIC:
            raise ValueError(f"{self.kind} has no angle")


@dataclass
class Circuit:
    n_qubits: int
    gates: list
    n_params: int
    name: str = ""

    def __len__(self):
        return len(self.gates)


@dataclass(frozen=True)
class PauliTerm:
    """``coeff * P`` with ``P`` a tensor product of single-qubit Paulis.

    ``ops`` is a tuple of ``(qubit, 'X'|'Y'|'Z')`` pairs; qubits not listed
    carry the identity.
    """
    coeff: float
    ops: tuple = ()


# ----------------------------------------------------------------------------
# Random numbers: splitmix64 (Steele, Lea, Flood 2014), the published mixer.
# ----------------------------------------------------------------------------
MASK64 = (1 << 64) - 1
SEED_BASE = 2511019291


class SplitMix64:
    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform01(self) -> float:
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)

    def angle(self) -> float:
        return self.uniform01() * 2.0 * math.pi

    def angles(self, count: int) -> np.ndarray:
        return np.array([self.angle() for _ in range(count)], dtype=np.float64)

    def randint(self, lo: int, hi: int) -> int:
        """Uniform integer in [lo, hi] inclusive."""
        span = hi - lo + 1
        return lo + min(int(self.uniform01() * span), span - 1)


def config_rng(config_index: int) -> SplitMix64:
    """Stream for the numbered workload (1-based), seed = 2511019291 + index."""
    return SplitMix64(SEED_BASE + config_index)


# ----------------------------------------------------------------------------
# Circuit families
# ----------------------------------------------------------------------------
def hea_ansatz(n: int, layers: int, first_param: int = 0) -> Circuit:
    """Hardware-efficient ansatz: per layer RY(theta) on every qubit, then
    RZ(phi) on every qubit, then the CNOT ring CNOT(i, (i+1) mod n), i = 0..n-1
    (the ring of the appendix's main example).  Angle index of layer l, qubit q:
    ``l*2n + 2q`` for RY and ``l*2n + 2q + 1`` for RZ."""
    gates = []
    for l in range(layers):
        base = first_param + l * 2 * n
        for q in range(n):
            gates.append(Gate("RY", (q,), param=base + 2 * q))
        for q in range(n):
            gates.append(Gate("RZ", (q,), param=base + 2 * q + 1))
        if n > 1:
            for q in range(n):
                t = (q + 1) % n
                if t != q:
                    gates.append(Gate("CNOT", (q, t)))
    return Circuit(n, gates, first_param + layers * 2 * n, name=f"hea{n}x{layers}")


def ladder_ansatz(n: int, layers: int, encoder: bool = True) -> Circuit:
    """The Fig. 1 ladder (CNOT + RY blocks) in the form of the appendix's main
    example: an RY encoder on every qubit (angles 0..n-1 are the encoder
    inputs), then ``layers`` repetitions of the CNOT ring followed by RY on
    every qubit (trainable angles after the inputs)."""
    gates = []
    p = 0
    if encoder:
        for q in range(n):
            gates.append(Gate("RY", (q,), param=p))
            p += 1
    for _ in range(layers):
        for q in range(n):
            t = (q + 1) % n
            if t != q:
                gates.append(Gate("CNOT", (q, t)))
        for q in range(n):
            gates.append(Gate("RY", (q,), param=p))
            p += 1
    return Circuit(n, gates, p, name=f"ladder{n}x{layers}")


def ghz_circuit(n: int) -> Circuit:
    gates = [Gate("H", (0,))] + [Gate("CNOT", (0, i)) for i in range(1, n)]
    return Circuit(n, gates, 0, name=f"ghz{n}")


def qft_circuit(n: int) -> Circuit:
    """Textbook QFT on the flat index (qubit n-1 is the most significant bit):
    H on qubit i followed by controlled phases pi/2^(i-j) from every lower
    qubit j, for i = n-1 .. 0, then the bit-reversal swaps."""
    gates = []
    for i in range(n - 1, -1, -1):
        gates.append(Gate("H", (i,)))
        for j in range(i - 1, -1, -1):
            gates.append(Gate("CPHASE", (j, i), angle=math.pi / (1 << (i - j))))
    for i in range(n // 2):
        gates.append(Gate("SWAP", (i, n - 1 - i)))
    return Circuit(n, gates, 0, name=f"qft{n}")


def concat(a: Circuit, b: Circuit, shift_b_params: bool = True) -> Circuit:
    assert a.n_qubits == b.n_qubits
    off = a.n_params if shift_b_params else 0
    gates = list(a.gates)
    for g in b.gates:
        gates.append(Gate(g.kind, g.wires, g.param + off if g.param >= 0 else -1, g.angle, g.matrix))
    return Circuit(a.n_qubits, gates, off + b.n_params, name=f"{a.name}+{b.name}")


def qft_then_hea(n: int, layers: int) -> Circuit:
    return concat(qft_circuit(n), hea_ansatz(n, layers))


# ----------------------------------------------------------------------------
# Observables
# ----------------------------------------------------------------------------
def sum_z(n: int) -> list:
    return [PauliTerm(1.0, ((i, "Z"),)) for i in range(n)]


def ising(n: int, hx: float = 0.5) -> list:
    """Open-chain transverse-field Ising: sum_i Z_i Z_{i+1} + hx * sum_i X_i."""
    terms = [PauliTerm(1.0, ((i, "Z"), (i + 1, "Z"))) for i in range(n - 1)]
    terms += [PauliTerm(hx, ((i, "X"),)) for i in range(n)]
    return terms


def all_z_terms(n: int) -> list:
    """The per-qubit Z terms measured by ``measure_allZ`` (one output each)."""
    return sum_z(n)


def observable_l1(terms: Sequence[PauliTerm]) -> float:
    return float(sum(abs(t.coeff) for t in terms))


def random_pauli_terms(rng: SplitMix64, n: int, count: int, max_weight: int = 4) -> list:
    terms = []
    for _ in range(count):
        w = rng.randint(1, min(max_weight, n))
        qubits = []
        while len(qubits) < w:
            q = rng.randint(0, n - 1)
            if q not in qubits:
                qubits.append(q)
        ops = tuple(sorted((q, "XYZ"[rng.randint(0, 2)]) for q in qubits))
        terms.append(PauliTerm(rng.uniform01() * 2.0 - 1.0, ops))
    return terms


# ----------------------------------------------------------------------------
# Random gate lists (tests): every kind, every wire order
# ----------------------------------------------------------------------------
def random_unitary(rng: SplitMix64, dim: int) -> np.ndarray:
    """Haar-ish random unitary from a QR of a seeded complex Gaussian matrix
    (Box-Muller on the splitmix64 stream)."""
    def gauss():
        u1 = max(rng.uniform01(), 1e-300)
        u2 = rng.uniform01()
        return math.sqrt(-2.0 * math.log(u1)) * math.cos(2.0 * math.pi * u2)
    a = np.array([[gauss() + 1j * gauss() for _ in range(dim)] for _ in range(dim)])
    q, r = np.linalg.qr(a)
    d = np.diag(r)
    return q * (d / np.abs(d))


def random_circuit(rng: SplitMix64, n: int, n_gates: int, kinds: Iterable[str] = GATE_KINDS,
                   n_params: int | None = None, fixed_fraction: float = 0.25) -> tuple:
    """Random gate list over ``kinds``; returns (Circuit, params)."""
    kinds = [k for k in kinds if GATE_ARITY[k] <= n]
    if n_params is None:
        n_params = max(1, n_gates // 2)
    gates = []
    for _ in range(n_gates):
        k = kinds[rng.randint(0, len(kinds) - 1)]
        ar = GATE_ARITY[k]
        wires = []
        while len(wires) < ar:
            q = rng.randint(0, n - 1)
            if q not in wires:
                wires.append(q)
        if k in PARAMETRIC:
            if rng.uniform01() < fixed_fraction:
                gates.append(Gate(k, tuple(wires), -1, rng.angle()))
            else:
                gates.append(Gate(k, tuple(wires), rng.randint(0, n_params - 1)))
        elif k == "UNITARY1":
            gates.append(Gate(k, tuple(wires), matrix=random_unitary(rng, 2)))
        elif k == "UNITARY2":
            gates.append(Gate(k, tuple(wires), matrix=random_unitary(rng, 4)))
        else:
            gates.append(Gate(k, tuple(wires)))
    params = rng.angles(n_params)
    return Circuit(n, gates, n_params, name=f"random{n}x{n_gates}"), params


# ----------------------------------------------------------------------------
# The numbered workloads (synthetic stand-ins; the paper ships no dataset)
# ----------------------------------------------------------------------------
@dataclass
class Workload:
    name: str
    circuit: Circuit
    params: np.ndarray
    terms: list
    extra: dict = field(default_factory=dict)


def workload_hea(config_index: int, n: int, layers: int, observable: str) -> Workload:
    circ = hea_ansatz(n, layers)
    params = config_rng(config_index).angles(circ.n_params)
    terms = sum_z(n) if observable == "sum_z" else ising(n)
    return Workload(f"hea n={n} L={layers} {observable}", circ, params, terms)


def workload_small() -> Workload:
    """12 qubits, 4 layers (96 angles), observable sum_i Z_i."""
    return workload_hea(1, 12, 4, "sum_z")


def workload_main() -> Workload:
    """26 qubits, 20 layers (1040 angles), open-chain Ising observable."""
    return workload_hea(2, 26, 20, "ising")


def workload_grad() -> Workload:
    """24 qubits, 10 layers (480 angles), open-chain Ising observable."""
    return workload_hea(3, 24, 10, "ising")


def workload_qft(n: int = 32, layers: int = 8) -> Workload:
    circ = qft_then_hea(n, layers)
    params = config_rng(5).angles(circ.n_params)
    return Workload(f"qft+hea n={n} L={layers} ising", circ, params, ising(n))


def batched_workload(count: int = 512, wmin: int = 10, wmax: int = 20,
                     dmin: int = 2, dmax: int = 12, config_index: int = 4) -> list:
    """Ragged batch: for each circuit in turn the stream draws its width, its
    depth, then its 2*width*depth angles.  Observable sum_i Z_i."""
    rng = config_rng(config_index)
    out = []
    for c in range(count):
        w = rng.randint(wmin, wmax)
        d = rng.randint(dmin, dmax)
        circ = hea_ansatz(w, d)
        params = rng.angles(circ.n_params)
        out.append(Workload(f"batch[{c}] w={w} d={d}", circ, params, sum_z(w)))
    return out
