"""ctypes loader for ``libtqd.so`` (the C ABI of ``include/tqd.h``).

There is no fallback: if the library is missing or fails to load, every call
raises ``TqdLibraryError``.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libtqd.so")

TQD_OK = 0
STATUS_NAMES = {0: "TQD_OK", 1: "TQD_ERR_INVALID_ARG", 2: "TQD_ERR_UNSUPPORTED", 3: "TQD_ERR_CUDA",
                4: "TQD_ERR_OOM", 5: "TQD_ERR_TIMEOUT", 6: "TQD_ERR_NUMERIC"}
KIND_CODES = {
    "H": 0, "X": 1, "Y": 2, "Z": 3, "S": 4, "T": 5,
    "RX": 6, "RY": 7, "RZ": 8, "PHASE": 9,
    "CNOT": 10, "CZ": 11, "CPHASE": 12, "SWAP": 13,
    "UNITARY1": 14, "UNITARY2": 15,
}
C64, C128 = 0, 1
PLAN_PLAIN, PLAN_FUSED, PLAN_TC = 0, 1, 2
CHECKPOINTS_NONE = 0xFFFFFFFF

# Every symbol include/tqd.h declares (checked by the ABI test).
EXPORTS = (
    "tqd_state_alloc", "tqd_state_reset", "tqd_state_free",
    "tqd_circuit_create", "tqd_circuit_free", "tqd_circuit_info", "tqd_circuit_check", "tqd_circuit_test_stall",
    "tqd_jit_check",
    "tqd_plan_check",
    "tqd_apply_circuit",
    "tqd_expval", "tqd_expval_terms", "tqd_expval_noalloc", "tqd_apply_observable",
    "tqd_backward", "tqd_value_and_grad", "tqd_backward_seeded", "tqd_probabilities", "tqd_sample",
    "tqd_shots_gaussian", "tqd_shots_gaussian_backward", "tqd_batch_create", "tqd_batch_buffers", "tqd_batch_run", "tqd_batch_info", "tqd_batch_tiling",
    "tqd_batch_free",
    "tqd_profile_enable", "tqd_profile_read", "tqd_last_error", "tqd_version",
)


class TqdLibraryError(RuntimeError):
    pass


class TqdError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class Gate(C.Structure):
    _fields_ = [
        ("kind", C.c_uint32),
        ("nwires", C.c_uint32),
        ("wires", C.c_uint32 * 3),
        ("param_idx", C.c_int32),
        ("fixed", C.c_double),
        ("mat_idx", C.c_int32),
        ("reserved", C.c_uint32),
    ]


class PauliTerm(C.Structure):
    _fields_ = [("xmask", C.c_uint64), ("zmask", C.c_uint64), ("coeff", C.c_double)]


class ProfileEntry(C.Structure):
    _fields_ = [("name", C.c_char * 32), ("launches", C.c_int64), ("total_ms", C.c_double),
                ("bytes", C.c_double)]


class BatchOpts(C.Structure):
    _fields_ = [("small_max_qubits", C.c_uint32), ("small_threads", C.c_uint32), ("streams", C.c_uint32),
                ("autotune", C.c_uint32), ("plain", C.c_uint32), ("reserved", C.c_uint32 * 3)]


class PlanOpts(C.Structure):
    _fields_ = [("mode", C.c_uint32), ("tile_qubits", C.c_uint32), ("low_qubits", C.c_uint32),
                ("buffers", C.c_uint32), ("jit", C.c_uint32), ("max_blocks", C.c_uint32),
                ("checkpoints", C.c_uint32), ("reserved", C.c_uint32 * 1)]


_lock = threading.Lock()
_lib = None


def load(path: str | None = None):
    """Load libtqd once; raises TqdLibraryError when it is missing."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or os.environ.get("TQD_LIBRARY") or LIB_PATH
        if not os.path.exists(p):
            raise TqdLibraryError(
                f"libtqd.so not found at {p}; build it with `python -m paper_2511_19291_gb300.build` "
                "(there is no CPU fallback)")
        try:
            L = C.CDLL(p)
        except OSError as e:
            raise TqdLibraryError(f"cannot load {p}: {e}") from e
        vp, i32, sz, u64, dbl = C.c_void_p, C.c_int, C.c_size_t, C.c_uint64, C.c_double
        st = C.c_int
        L.tqd_state_alloc.argtypes = [i32, i32, vp, sz, C.POINTER(vp)]
        L.tqd_state_reset.argtypes = [vp, u64, vp]
        L.tqd_state_free.argtypes = [vp]
        L.tqd_circuit_create.argtypes = [i32, vp, sz, i32, vp, sz, vp, C.POINTER(vp)]
        L.tqd_circuit_free.argtypes = [vp]
        L.tqd_circuit_info.argtypes = [vp, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32)]
        L.tqd_circuit_check.argtypes = [vp, C.POINTER(i32)]
        L.tqd_circuit_test_stall.argtypes = [vp, i32]
        L.tqd_jit_check.argtypes = [i32, vp, sz, i32, vp, sz, i32, C.POINTER(i32)]
        L.tqd_plan_check.argtypes = [i32, vp, sz, i32, vp, sz, vp, u64, C.POINTER(dbl), C.POINTER(dbl),
                                     C.POINTER(i32), C.POINTER(i32)]
        L.tqd_apply_circuit.argtypes = [vp, vp, vp, vp]
        L.tqd_expval.argtypes = [vp, vp, sz, vp, vp]
        L.tqd_expval_terms.argtypes = [vp, vp, sz, vp, vp]
        L.tqd_expval_noalloc.argtypes = [vp, vp, sz, vp, vp]
        L.tqd_apply_observable.argtypes = [vp, vp, sz, vp, vp, vp]
        L.tqd_backward.argtypes = [vp, vp, vp, vp, vp, sz, vp, dbl, vp, vp]
        L.tqd_value_and_grad.argtypes = [vp, vp, vp, vp, vp, sz, vp, vp, vp]
        L.tqd_backward_seeded.argtypes = [vp, vp, vp, vp, vp, vp]
        L.tqd_probabilities.argtypes = [vp, vp, vp]
        L.tqd_sample.argtypes = [vp, vp, sz, vp, vp]
        L.tqd_shots_gaussian.argtypes = [vp, dbl, vp, vp, vp]
        L.tqd_shots_gaussian_backward.argtypes = [vp, dbl, vp, vp, vp, vp]
        L.tqd_batch_create.argtypes = [i32, vp, vp, vp, vp, C.POINTER(vp)]
        L.tqd_batch_buffers.argtypes = [vp, C.POINTER(vp), C.POINTER(vp), C.POINTER(vp), vp]
        L.tqd_batch_run.argtypes = [vp, vp]
        L.tqd_batch_info.argtypes = [vp] + [C.POINTER(i32)] * 5
        L.tqd_batch_free.argtypes = [vp]
        L.tqd_batch_tiling.argtypes = [vp, i32, C.POINTER(i32), C.POINTER(i32)]
        L.tqd_profile_enable.argtypes = [i32]
        L.tqd_profile_read.argtypes = [vp, i32, C.POINTER(i32)]
        for name in ("tqd_state_alloc", "tqd_state_reset", "tqd_state_free", "tqd_circuit_create",
                     "tqd_circuit_free", "tqd_circuit_info", "tqd_circuit_check", "tqd_circuit_test_stall",
                     "tqd_apply_circuit", "tqd_expval",
                     "tqd_expval_terms", "tqd_expval_noalloc", "tqd_apply_observable", "tqd_backward", "tqd_value_and_grad",
                     "tqd_backward_seeded", "tqd_probabilities", "tqd_sample", "tqd_shots_gaussian",
                     "tqd_shots_gaussian_backward",
                     "tqd_batch_create", "tqd_batch_buffers", "tqd_batch_run", "tqd_batch_info",
                     "tqd_batch_tiling",
                     "tqd_batch_free", "tqd_profile_enable", "tqd_jit_check", "tqd_plan_check",
                     "tqd_profile_read"):
            getattr(L, name).restype = st
        L.tqd_last_error.restype = C.c_char_p
        L.tqd_last_error.argtypes = []
        L.tqd_version.restype = C.c_char_p
        L.tqd_version.argtypes = []
        _lib = L
        return _lib


def check(status: int):
    if status != TQD_OK:
        msg = load().tqd_last_error().decode(errors="replace")
        raise TqdError(status, msg)
