"""ctypes front end of the complex128 CPU oracle (``tqd_oracle.c``).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this module.  It shares no
code with the CUDA library: it marshals the gate descriptions of
``paper_2511_19291_gb300.workloads`` into its own C structures and calls its
own C functions.

Functions and the passage each follows:

* ``run``            -- psi_L = G_L ... G_1 e_j, gate by gate (Sec. 4.1, Algorithm 1)
* ``expval``         -- E = sum_j c_j psi^* P_j psi (Sec. 2.2.1, measurement)
* ``apply_observable`` -- H psi
* ``grad_param_shift`` -- parameter-shift gradient (exact for the gate set)
* ``grad_stored``    -- stored-activation reverse pass (Sec. 4.4, first form)
* ``unapply``        -- applies G^dagger in reverse order (Sec. 4.4, x = U^* y)
"""
from __future__ import annotations

import contextlib
import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tqd_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libtqd_oracle.so")
_lock = threading.Lock()
_lib = None

KIND_CODES = {
    "H": 0, "X": 1, "Y": 2, "Z": 3, "S": 4, "T": 5,
    "RX": 6, "RY": 7, "RZ": 8, "PHASE": 9,
    "CNOT": 10, "CZ": 11, "CPHASE": 12, "SWAP": 13,
    "UNITARY1": 14, "UNITARY2": 15,
}
PAULI_CODES = {"X": 1, "Y": 2, "Z": 3}


class OrcGate(C.Structure):
    _fields_ = [
        ("kind", C.c_int32),
        ("nwires", C.c_int32),
        ("wires", C.c_int32 * 3),
        ("param", C.c_int32),
        ("angle", C.c_double),
        ("mat", C.c_int32),
        ("pad", C.c_int32),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C11, optional OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:4] + ["-fopenmp"] + base[4:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load(path):
    L = C.CDLL(path)
    ip, vp = C.c_int, C.c_void_p
    L.orc_run.argtypes = [ip, vp, ip, vp, vp, C.c_uint64, vp]
    L.orc_apply_gates.argtypes = [ip, vp, vp, ip, ip, vp, vp, ip]
    L.orc_expval.argtypes = [ip, vp, ip, vp, vp, vp]
    L.orc_expval.restype = C.c_double
    L.orc_apply_observable.argtypes = [ip, vp, ip, vp, vp, vp]
    L.orc_grad_param_shift.argtypes = [ip, vp, ip, vp, ip, vp, C.c_uint64, ip, vp, vp, vp]
    L.orc_grad_stored.argtypes = [ip, vp, ip, vp, ip, vp, C.c_uint64, ip, vp, vp, vp]
    L.orc_grad_stored.restype = C.c_double
    L.orc_norm2.argtypes = [ip, vp]
    L.orc_norm2.restype = C.c_double
    L.orc_gate_dense.argtypes = [ip, vp, vp, vp, vp]
    return L


_override = []


def lib():
    global _lib
    if _override:
        return _override[-1]
    with _lock:
        if _lib is None:
            _lib = _load(build())
    return _lib


@contextlib.contextmanager
def use_library(path: str):
    """Temporarily route every oracle call to another build of the oracle
    source (the tests use it to plant mistakes and check that the pins
    catch them)."""
    _override.append(_load(path))
    try:
        yield
    finally:
        _override.pop()


def build_variant(source_text: str, out_path: str) -> str:
    """Compile an edited copy of the oracle source (test use only)."""
    src = out_path + ".c"
    with open(src, "w") as f:
        f.write(source_text)
    subprocess.run(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", src, "-o", out_path, "-lm"],
                   check=True, capture_output=True)
    return out_path


def source_text() -> str:
    with open(_SRC) as f:
        return f.read()


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


class _Marshalled:
    """Gate array + matrix table + parameter vector kept alive together."""

    def __init__(self, circuit, params):
        gates = circuit.gates
        self.ng = len(gates)
        self.arr = (OrcGate * max(1, self.ng))()
        table = []
        for i, g in enumerate(gates):
            og = self.arr[i]
            og.kind = KIND_CODES[g.kind]
            og.nwires = len(g.wires)
            for j, w in enumerate(g.wires):
                og.wires[j] = int(w)
            og.param = int(g.param)
            og.angle = float(g.angle)
            og.mat = -1
            if g.kind in ("UNITARY1", "UNITARY2"):
                og.mat = len(table)
                table.extend(np.asarray(g.matrix, dtype=np.complex128).reshape(-1).tolist())
        self.table = np.array(table if table else [0j], dtype=np.complex128)
        p = np.asarray(params if params is not None else [], dtype=np.float64)
        self.params = np.ascontiguousarray(p if p.size else np.zeros(1))
        self.n_params = int(circuit.n_params)


class _MarshalledTerms:
    def __init__(self, n, terms):
        self.nt = len(terms)
        self.ops = np.zeros((max(1, self.nt), n), dtype=np.int8)
        self.coeffs = np.zeros(max(1, self.nt), dtype=np.float64)
        for j, t in enumerate(terms):
            self.coeffs[j] = t.coeff
            for q, p in t.ops:
                if self.ops[j, q] != 0:
                    raise ValueError("qubit listed twice in a Pauli term")
                self.ops[j, q] = PAULI_CODES[p]


def run(circuit, params=None, init_index: int = 0) -> np.ndarray:
    m = _Marshalled(circuit, params)
    psi = np.empty(1 << circuit.n_qubits, dtype=np.complex128)
    lib().orc_run(circuit.n_qubits, C.cast(m.arr, C.c_void_p), m.ng, _ptr(m.params), _ptr(m.table),
                  init_index, _ptr(psi))
    return psi


def apply_gates(circuit, params, psi: np.ndarray, first: int = 0, last: int | None = None,
                adjoint: bool = False) -> np.ndarray:
    """Apply gates[first:last] (or their adjoints in reverse) to a copy of psi."""
    m = _Marshalled(circuit, params)
    out = np.array(psi, dtype=np.complex128, copy=True)
    last = m.ng if last is None else last
    lib().orc_apply_gates(circuit.n_qubits, _ptr(out), C.cast(m.arr, C.c_void_p), first, last,
                          _ptr(m.params), _ptr(m.table), int(adjoint))
    return out


def unapply(circuit, params, psi: np.ndarray) -> np.ndarray:
    return apply_gates(circuit, params, psi, adjoint=True)


def expval(n: int, psi: np.ndarray, terms) -> tuple:
    """Returns (E, per-term <P_j>)."""
    t = _MarshalledTerms(n, terms)
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    per = np.zeros(max(1, t.nt))
    e = lib().orc_expval(n, _ptr(psi), t.nt, _ptr(t.ops), _ptr(t.coeffs), _ptr(per))
    return float(e), per[: t.nt].copy()


def apply_observable(n: int, psi: np.ndarray, terms) -> np.ndarray:
    t = _MarshalledTerms(n, terms)
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    out = np.empty_like(psi)
    lib().orc_apply_observable(n, _ptr(psi), t.nt, _ptr(t.ops), _ptr(t.coeffs), _ptr(out))
    return out


def grad_param_shift(circuit, params, terms, init_index: int = 0) -> np.ndarray:
    m = _Marshalled(circuit, params)
    t = _MarshalledTerms(circuit.n_qubits, terms)
    g = np.zeros(max(1, m.n_params))
    lib().orc_grad_param_shift(circuit.n_qubits, C.cast(m.arr, C.c_void_p), m.ng, _ptr(m.params),
                               m.n_params, _ptr(m.table), init_index, t.nt, _ptr(t.ops),
                               _ptr(t.coeffs), _ptr(g))
    return g[: m.n_params].copy()


def grad_stored(circuit, params, terms, init_index: int = 0) -> tuple:
    """Returns (E, gradient) by the stored-activation reverse pass."""
    m = _Marshalled(circuit, params)
    t = _MarshalledTerms(circuit.n_qubits, terms)
    g = np.zeros(max(1, m.n_params))
    e = lib().orc_grad_stored(circuit.n_qubits, C.cast(m.arr, C.c_void_p), m.ng, _ptr(m.params),
                              m.n_params, _ptr(m.table), init_index, t.nt, _ptr(t.ops),
                              _ptr(t.coeffs), _ptr(g))
    return float(e), g[: m.n_params].copy()


def norm2(n: int, psi: np.ndarray) -> float:
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    return float(lib().orc_norm2(n, _ptr(psi)))


def gate_dense(n: int, gate, params=None) -> np.ndarray:
    """2^n x 2^n matrix of one gate, built by the oracle's own apply loop."""
    from types import SimpleNamespace
    circ = SimpleNamespace(gates=[gate], n_params=len(params) if params is not None else 0)
    m = _Marshalled(circ, params)
    N = 1 << n
    U = np.empty((N, N), dtype=np.complex128)
    lib().orc_gate_dense(n, C.cast(m.arr, C.c_void_p), _ptr(m.params), _ptr(m.table), _ptr(U))
    return U


def energy(circuit, params, terms, init_index: int = 0) -> float:
    return expval(circuit.n_qubits, run(circuit, params, init_index), terms)[0]
