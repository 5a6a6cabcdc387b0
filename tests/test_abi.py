"""The C ABI library loads and exports every symbol ``include/tqd.h`` declares;
host-side argument validation rejects bad requests before any device work
(no GPU needed)."""
import ctypes as C
import os
import re

import pytest

from paper_2511_19291_gb300 import _lib, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _lib.load()


def header_functions():
    text = open(os.path.join(ROOT, "include", "tqd.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tqd_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_what_binding_lists():
    assert header_functions() == sorted(_lib.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    missing = [name for name in header_functions() if not hasattr(lib, name)]
    assert missing == []


def test_version_and_error_strings(lib):
    assert lib.tqd_version().startswith(b"tqd")
    assert isinstance(lib.tqd_last_error(), bytes)


def make_gates(specs):
    arr = (_lib.Gate * max(1, len(specs)))()
    for i, (kind, wires, param) in enumerate(specs):
        arr[i].kind = _lib.KIND_CODES[kind]
        arr[i].nwires = len(wires)
        for j, w in enumerate(wires):
            arr[i].wires[j] = w
        arr[i].param_idx = param
        arr[i].fixed = 0.0
        arr[i].mat_idx = -1
    return arr


@pytest.mark.parametrize("specs,n,n_params,needle", [
    ([("RY", [5], -1)], 4, 0, b"wire 5 >= n_qubits 4"),
    ([("CNOT", [1, 1], -1)], 4, 0, b"duplicate wire"),
    ([("RY", [0], 3)], 4, 2, b"param_idx 3 >= n_params 2"),
    ([("H", [0], 0)], 4, 1, b"takes no angle"),
    ([("UNITARY1", [0], -1)], 4, 0, b"matrix index"),
])
def test_circuit_validation(lib, specs, n, n_params, needle):
    arr = make_gates(specs)
    h = C.c_void_p()
    st = lib.tqd_circuit_create(n, C.cast(arr, C.c_void_p), len(specs), n_params, None, 0, None, C.byref(h))
    assert st == 1  # TQD_ERR_INVALID_ARG
    assert needle in lib.tqd_last_error()
    assert not h.value


@pytest.mark.parametrize("field,value,needle", [
    ("tile_qubits", 10, b"tile_qubits 10"),
    ("low_qubits", 3, b"low_qubits 3"),
    ("buffers", 5, b"buffers 5"),
    ("jit", 3, b"jit 3"),
    ("mode", 7, b"unknown plan mode"),
])
def test_plan_option_validation(lib, field, value, needle):
    """Plan options outside what the kernels implement are rejected on the
    host, before any device work (the tile width is fixed at 12 qubits)."""
    arr = make_gates([("RY", [0], 0)])
    opts = _lib.PlanOpts()
    opts.mode = _lib.PLAN_FUSED
    setattr(opts, field, value)
    h = C.c_void_p()
    st = lib.tqd_circuit_create(14, C.cast(arr, C.c_void_p), 1, 1, None, 0, C.byref(opts), C.byref(h))
    assert st == 1, st
    assert needle in lib.tqd_last_error()
    assert not h.value


def test_wrong_arity_and_qubit_range(lib):
    arr = make_gates([("RY", [0], -1)])
    arr[0].nwires = 2
    h = C.c_void_p()
    assert lib.tqd_circuit_create(3, C.cast(arr, C.c_void_p), 1, 0, None, 0, None, C.byref(h)) == 1
    assert lib.tqd_circuit_create(40, C.cast(arr, C.c_void_p), 0, 0, None, 0, None, C.byref(h)) == 1
    assert lib.tqd_state_alloc(3, 0, None, 64, C.byref(h)) == 1
    assert lib.tqd_state_alloc(3, 0, C.c_void_p(0x1001), 64, C.byref(h)) == 1
    assert b"aligned" in lib.tqd_last_error()
    assert lib.tqd_state_alloc(10, 0, C.c_void_p(0x1000), 64, C.byref(h)) == 1
    assert b"need" in lib.tqd_last_error()


def test_nonfinite_angle_rejected(lib):
    arr = make_gates([("RY", [0], -1)])
    arr[0].fixed = float("nan")
    h = C.c_void_p()
    assert lib.tqd_circuit_create(3, C.cast(arr, C.c_void_p), 1, 0, None, 0, None, C.byref(h)) == 6


def test_null_handles_rejected(lib):
    assert lib.tqd_apply_circuit(None, None, None, None) == 1
    assert lib.tqd_expval(None, None, 0, None, None) == 1
    assert lib.tqd_backward(None, None, None, None, None, 0, None, 1.0, None, None) == 1
    assert lib.tqd_state_free(None) == 0
    assert lib.tqd_circuit_free(None) == 0
    assert lib.tqd_circuit_test_stall(None, 1) == 1
    assert lib.tqd_circuit_check(None, None) == 1


def test_specialised_pass_kernels_compile(lib):
    """The pass-specialised kernels the library generates compile for sm_103a
    (NVRTC, no GPU): the ansatz form and a random gate list over every kind,
    both precisions and both directions."""
    from paper_2511_19291_gb300 import sim as S
    from paper_2511_19291_gb300 import workloads as W
    assert S.jit_check(W.hea_ansatz(14, 2)) >= 4
    circ, _ = W.random_circuit(W.SplitMix64(77), 13, 60, n_params=20)
    assert S.jit_check(circ) >= 4


def test_specialised_check_rejects_small_and_bad_arch(lib):
    from paper_2511_19291_gb300 import sim as S
    from paper_2511_19291_gb300 import workloads as W
    with pytest.raises(_lib.TqdError, match="INVALID_ARG"):
        S.jit_check(W.hea_ansatz(8, 1))
    with pytest.raises(_lib.TqdError, match="INVALID_ARG"):
        S.jit_check(W.hea_ansatz(14, 1), arch=7)
