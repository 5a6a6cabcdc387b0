"""Python front end of libtqd: argument marshalling only.

Every step of the simulation runs in the CUDA library; this module turns
torch tensors and the gate/term descriptions of ``workloads`` into the C ABI
arguments (device pointers, sizes, the current CUDA stream).

* ``State``      -- a 2^n complex64/complex128 CUDA tensor wrapped as a tqd_state
* ``Circuit``    -- a planned gate list (tqd_circuit)
* ``Observable`` -- a marshalled Pauli sum
* ``apply``, ``expval``, ``expval_terms``, ``apply_observable``, ``backward``
* ``expval_fn``  -- differentiable E(theta) (torch.autograd.Function)
* ``measure_allz_fn`` -- differentiable per-qubit <Z_i> (the appendix's measure_allZ)
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib
from . import workloads as W


def _L():
    return _lib.load()


def _stream(device) -> C.c_void_p:
    return C.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def pauli_masks(term: W.PauliTerm) -> tuple:
    """(xmask, zmask): X sets the x bit, Z the z bit, Y both."""
    x = z = 0
    for q, p in term.ops:
        bit = 1 << q
        if p == "X":
            x |= bit
        elif p == "Z":
            z |= bit
        elif p == "Y":
            x |= bit
            z |= bit
        else:
            raise ValueError(f"unknown Pauli {p!r}")
    return x, z


class Observable:
    """A Pauli sum marshalled once into the tqd_pauli_term layout."""

    def __init__(self, terms):
        if isinstance(terms, Observable):
            terms = terms.terms
        self.terms = list(terms)
        self.arr = (_lib.PauliTerm * max(1, len(self.terms)))()
        for j, t in enumerate(self.terms):
            x, z = pauli_masks(t)
            self.arr[j].xmask = x
            self.arr[j].zmask = z
            self.arr[j].coeff = float(t.coeff)

    def __len__(self):
        return len(self.terms)

    @property
    def ptr(self):
        return C.cast(self.arr, C.c_void_p)


def as_observable(obs) -> Observable:
    return obs if isinstance(obs, Observable) else Observable(obs)


class State:
    """An n-qubit state over a contiguous CUDA tensor of 2^n complex amplitudes."""

    def __init__(self, n: int, dtype=torch.complex64, device="cuda", tensor: torch.Tensor | None = None):
        if tensor is None:
            tensor = torch.empty(1 << n, dtype=dtype, device=device)
        if not tensor.is_cuda:
            raise ValueError("state tensor must be on a CUDA device")
        if tensor.dtype not in (torch.complex64, torch.complex128):
            raise ValueError("state tensor must be complex64 or complex128")
        if tensor.numel() != (1 << n) or not tensor.is_contiguous():
            raise ValueError("state tensor must be contiguous with 2^n elements")
        self.n = n
        self.tensor = tensor
        self.device = tensor.device
        self.dtype_code = _lib.C64 if tensor.dtype == torch.complex64 else _lib.C128
        h = C.c_void_p()
        _lib.check(_L().tqd_state_alloc(n, self.dtype_code, C.c_void_p(tensor.data_ptr()),
                                        tensor.numel() * tensor.element_size(), C.byref(h)))
        self._h = h

    @property
    def handle(self):
        return self._h

    def reset(self, basis_index: int = 0):
        with torch.cuda.device(self.device):
            _lib.check(_L().tqd_state_reset(self._h, basis_index, _stream(self.device)))
        return self

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            try:
                _L().tqd_state_free(h)
            except Exception:
                pass
            self._h = None


def _gate_array(circuit: W.Circuit):
    """The gate list as tqd_gate records, and the matrix table (re, im pairs)."""
    gates = circuit.gates
    arr = (_lib.Gate * max(1, len(gates)))()
    table = []
    for i, g in enumerate(gates):
        a = arr[i]
        a.kind = _lib.KIND_CODES[g.kind]
        a.nwires = len(g.wires)
        for j, w in enumerate(g.wires):
            a.wires[j] = int(w)
        a.param_idx = int(g.param)
        a.fixed = float(g.angle)
        a.mat_idx = -1
        if g.kind in ("UNITARY1", "UNITARY2"):
            a.mat_idx = len(table)
            table.extend(np.asarray(g.matrix, dtype=np.complex128).reshape(-1).tolist())
    mats = np.array([[v.real, v.imag] for v in table], dtype=np.float64).reshape(-1)
    return arr, mats, len(table)


def jit_check(circuit: W.Circuit, arch: int = 103) -> int:
    """Compiles the circuit's pass-specialised kernels for compute capability
    `arch` without a GPU (tqd_jit_check); returns how many distinct kernels."""
    arr, mats, n_entries = _gate_array(circuit)
    n = C.c_int32()
    _lib.check(_L().tqd_jit_check(
        circuit.n_qubits, C.cast(arr, C.c_void_p), len(circuit.gates), circuit.n_params,
        mats.ctypes.data_as(C.c_void_p) if n_entries else None, n_entries, arch, C.byref(n)))
    return n.value


def plan_check(circuit: W.Circuit, params=None, seed: int = 1) -> dict:
    """Runs the circuit's fused plan on the host from its encoded descriptors
    and compares it with the gates applied one by one (tqd_plan_check, no
    GPU): largest amplitude error after the forward passes and after the
    reverse sweep, and the plan's pass and stage counts."""
    arr, mats, n_entries = _gate_array(circuit)
    p = np.ascontiguousarray(np.zeros(max(1, circuit.n_params)) if params is None else params, dtype=np.float64)
    ef, er = C.c_double(), C.c_double()
    npass, nstage = C.c_int32(), C.c_int32()
    _lib.check(_L().tqd_plan_check(
        circuit.n_qubits, C.cast(arr, C.c_void_p), len(circuit.gates), circuit.n_params,
        mats.ctypes.data_as(C.c_void_p) if n_entries else None, n_entries, p.ctypes.data_as(C.c_void_p),
        seed, C.byref(ef), C.byref(er), C.byref(npass), C.byref(nstage)))
    return {"err_forward": ef.value, "err_reverse": er.value, "passes": npass.value, "stages": nstage.value}


class Circuit:
    """A gate list planned by the library (plain gate-by-gate or fused passes)."""

    def __init__(self, circuit: W.Circuit, mode: str = "fused", tile_qubits: int = 0, low_qubits: int = 0,
                 device=None, buffers: int = 0, jit: int = 0, max_blocks: int = 0, checkpoints: int | None = None):
        """checkpoints: forward checkpoints of value_and_grad; None = as many
        passes as fit in half the free device memory, 0 = none, k = at most k
        passes."""
        self.spec = circuit
        self.n = circuit.n_qubits
        self.n_params = circuit.n_params
        self.mode = mode
        gates = circuit.gates
        arr, mats, n_entries = _gate_array(circuit)
        opts = _lib.PlanOpts()
        opts.mode = {"plain": _lib.PLAN_PLAIN, "fused": _lib.PLAN_FUSED, "tc": _lib.PLAN_TC}[mode]
        opts.tile_qubits = tile_qubits
        opts.low_qubits = low_qubits
        opts.buffers = buffers
        opts.jit = jit
        opts.max_blocks = max_blocks
        if checkpoints is not None and checkpoints < 0:
            raise ValueError("checkpoints must be None or >= 0")
        opts.checkpoints = 0 if checkpoints is None else (_lib.CHECKPOINTS_NONE if checkpoints == 0 else checkpoints)
        h = C.c_void_p()
        dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        with torch.cuda.device(dev):
            _lib.check(_L().tqd_circuit_create(
                self.n, C.cast(arr, C.c_void_p), len(gates), self.n_params,
                mats.ctypes.data_as(C.c_void_p) if n_entries else None, n_entries,
                C.byref(opts), C.byref(h)))
        self._h = h
        self._mats = mats

    @property
    def handle(self):
        return self._h

    def info(self) -> dict:
        a, b, c = C.c_int(), C.c_int(), C.c_int()
        _lib.check(_L().tqd_circuit_info(self._h, C.byref(a), C.byref(b), C.byref(c)))
        return {"passes": a.value, "launches_apply": b.value, "launches_backward": c.value}

    def check(self) -> int:
        """Synchronize, return the device error word (0 = all launches of
        this circuit since the last check completed normally) and clear it;
        raises on a non-zero word."""
        v = C.c_int()
        _lib.check(_L().tqd_circuit_check(self._h, C.byref(v)))
        return v.value

    def test_stall(self, enable: bool) -> None:
        """Test hook: while enabled, block 0 of every fused tile pass waits for
        a tile copy that is never issued, runs out its time limit and
        returns (the launch's results are invalid)."""
        _lib.check(_L().tqd_circuit_test_stall(self._h, int(bool(enable))))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            try:
                _L().tqd_circuit_free(h)
            except Exception:
                pass
            self._h = None


def _params_ptr(params: torch.Tensor | None, n_params: int):
    if n_params == 0:
        return None
    if params is None or not params.is_cuda or params.dtype != torch.float64 or not params.is_contiguous():
        raise ValueError("params must be a contiguous float64 CUDA tensor")
    if params.numel() < n_params:
        raise ValueError(f"params has {params.numel()} entries, circuit needs {n_params}")
    return C.c_void_p(params.data_ptr())


def apply(state: State, circuit: Circuit, params: torch.Tensor | None = None) -> State:
    with torch.cuda.device(state.device):
        _lib.check(_L().tqd_apply_circuit(state.handle, circuit.handle, _params_ptr(params, circuit.n_params),
                                          _stream(state.device)))
    return state


def expval(state: State, obs, out: torch.Tensor | None = None) -> torch.Tensor:
    obs = as_observable(obs)
    if out is None:
        out = torch.empty((), dtype=torch.float64, device=state.device)
    with torch.cuda.device(state.device):
        _lib.check(_L().tqd_expval(state.handle, obs.ptr, len(obs), C.c_void_p(out.data_ptr()),
                                   _stream(state.device)))
    return out


def expval_terms(state: State, obs, out: torch.Tensor | None = None) -> torch.Tensor:
    obs = as_observable(obs)
    if out is None:
        out = torch.empty(len(obs), dtype=torch.float64, device=state.device)
    with torch.cuda.device(state.device):
        _lib.check(_L().tqd_expval_terms(state.handle, obs.ptr, len(obs),
                                         C.c_void_p(out.data_ptr()) if len(obs) else None, _stream(state.device)))
    return out


def apply_observable(state: State, obs, weights: torch.Tensor | None = None, out: State | None = None) -> State:
    obs = as_observable(obs)
    if out is None:
        out = State(state.n, state.tensor.dtype, state.device)
    with torch.cuda.device(state.device):
        _lib.check(_L().tqd_apply_observable(state.handle, obs.ptr, len(obs), _weights_ptr(weights, len(obs)),
                                             out.handle, _stream(state.device)))
    return out


def _weights_ptr(weights, n_terms):
    if weights is None:
        return None
    if not weights.is_cuda or weights.dtype != torch.float64 or not weights.is_contiguous() or \
            weights.numel() < n_terms:
        raise ValueError("weights must be a contiguous float64 CUDA tensor with one entry per term")
    return C.c_void_p(weights.data_ptr())


def backward(psi: State, lam: State, circuit: Circuit, params: torch.Tensor | None, obs,
             grads: torch.Tensor | None, weights: torch.Tensor | None = None, scale: float = 1.0) -> torch.Tensor:
    """Adjoint sweep: grads += d(scale * sum_j w_j c_j <P_j>)/dparams; psi is restored to
    the circuit's input state."""
    obs = as_observable(obs)
    if grads is None:
        grads = torch.zeros(max(circuit.n_params, 0), dtype=torch.float64, device=psi.device)
    gptr = C.c_void_p(grads.data_ptr()) if circuit.n_params else None
    with torch.cuda.device(psi.device):
        _lib.check(_L().tqd_backward(psi.handle, lam.handle, circuit.handle, _params_ptr(params, circuit.n_params),
                                     obs.ptr, len(obs), _weights_ptr(weights, len(obs)), float(scale), gptr,
                                     _stream(psi.device)))
    return grads


def value_and_grad(psi: State, lam: State, circuit: Circuit, params: torch.Tensor | None, obs,
                   energy: torch.Tensor | None = None, grads: torch.Tensor | None = None):
    """One gradient evaluation (tqd_value_and_grad): psi <- U psi, energy =
    <psi|H|psi> (a float64 scalar tensor on the device), grads += dE/dparams;
    psi is restored to its input state.  Returns (energy, grads)."""
    obs = as_observable(obs)
    if energy is None:
        energy = torch.zeros((), dtype=torch.float64, device=psi.device)
    if grads is None:
        grads = torch.zeros(max(circuit.n_params, 0), dtype=torch.float64, device=psi.device)
    gptr = C.c_void_p(grads.data_ptr()) if circuit.n_params else None
    with torch.cuda.device(psi.device):
        _lib.check(_L().tqd_value_and_grad(psi.handle, lam.handle, circuit.handle,
                                           _params_ptr(params, circuit.n_params), obs.ptr, len(obs),
                                           C.c_void_p(energy.data_ptr()), gptr, _stream(psi.device)))
    return energy, grads


def backward_seeded(psi: State, lam: State, circuit: Circuit, params: torch.Tensor | None,
                    grads: torch.Tensor | None = None) -> torch.Tensor:
    """Reverse sweep from the seed in lam (dL/d conj(psi_L)): grads += dL/dparams;
    psi is restored to the circuit's input state (tqd_backward_seeded)."""
    if grads is None:
        grads = torch.zeros(max(circuit.n_params, 0), dtype=torch.float64, device=psi.device)
    gptr = C.c_void_p(grads.data_ptr()) if circuit.n_params else None
    with torch.cuda.device(psi.device):
        _lib.check(_L().tqd_backward_seeded(psi.handle, lam.handle, circuit.handle,
                                            _params_ptr(params, circuit.n_params), gptr, _stream(psi.device)))
    return grads


# --------------------------------------------------------------- shot noise
def probabilities(state: State) -> torch.Tensor:
    """p_b = |psi_b|^2 (FP64, 2^n values) (tqd_probabilities)."""
    p = torch.empty(1 << state.n, dtype=torch.float64, device=state.device)
    with torch.cuda.device(state.device):
        _lib.check(_L().tqd_probabilities(state.handle, C.c_void_p(p.data_ptr()), _stream(state.device)))
    return p


def sample(state: State, uniforms: torch.Tensor) -> torch.Tensor:
    """Exact measurement samples: one outcome index per uniform in [0, 1)
    (inverse transform of |psi|^2's cumulative distribution; tqd_sample)."""
    u = uniforms.to(device=state.device, dtype=torch.float64).contiguous()
    out = torch.empty(u.numel(), dtype=torch.int64, device=state.device)
    with torch.cuda.device(state.device):
        _lib.check(_L().tqd_sample(state.handle, C.c_void_p(u.data_ptr()), u.numel(), C.c_void_p(out.data_ptr()),
                                   _stream(state.device)))
    return out


def _normals(z: torch.Tensor, n: int, device) -> torch.Tensor:
    z = z.to(device=device, dtype=torch.float64).contiguous()
    if z.numel() not in ((1 << n) - 1, 1 << n):
        raise ValueError(f"z needs 2^n - 1 or 2^n entries, got {z.numel()}")
    return z


def shots_gaussian(state: State, n_shots: float, z: torch.Tensor) -> torch.Tensor:
    """Approximate shots y = n p + sqrt(n) D S z (tqd_shots_gaussian); z: unit normals."""
    z = _normals(z, state.n, state.device)
    y = torch.empty(1 << state.n, dtype=torch.float64, device=state.device)
    with torch.cuda.device(state.device):
        _lib.check(_L().tqd_shots_gaussian(state.handle, float(n_shots), C.c_void_p(z.data_ptr()),
                                           C.c_void_p(y.data_ptr()), _stream(state.device)))
    return y


def shots_gaussian_backward(state: State, n_shots: float, z: torch.Tensor, ybar: torch.Tensor,
                            lam: State) -> State:
    """lam = d(sum ybar y)/d conj(psi), the seed of backward_seeded."""
    z = _normals(z, state.n, state.device)
    yb = ybar.to(device=state.device, dtype=torch.float64).contiguous()
    with torch.cuda.device(state.device):
        _lib.check(_L().tqd_shots_gaussian_backward(state.handle, float(n_shots), C.c_void_p(z.data_ptr()),
                                                    C.c_void_p(yb.data_ptr()), lam.handle, _stream(state.device)))
    return lam


# ------------------------------------------------------------------ autograd
class _ShotsGaussFn(torch.autograd.Function):
    """Gaussian shots of the circuit's output state, differentiable in the
    angles (the reparameterisation of Sec. 4.3.2 with the reverse sweep of
    Sec. 4.4 seeded by the shots' cotangent)."""

    @staticmethod
    def forward(ctx, params, circuit, n_shots, z, dtype, basis_index):
        psi = State(circuit.n, dtype, params.device).reset(basis_index)
        apply(psi, circuit, params)
        y = shots_gaussian(psi, n_shots, z)
        ctx.save_for_backward(params)
        ctx.psi, ctx.circuit, ctx.n_shots, ctx.z = psi, circuit, n_shots, z
        return y

    @staticmethod
    def backward(ctx, ybar):
        (params,) = ctx.saved_tensors
        psi = ctx.psi
        if psi is None:
            raise RuntimeError("these shots' backward already ran (the saved state is consumed)")
        lam = State(psi.n, psi.tensor.dtype, psi.device)
        shots_gaussian_backward(psi, ctx.n_shots, ctx.z, ybar.contiguous(), lam)
        grads = torch.zeros_like(params)
        backward_seeded(psi, lam, ctx.circuit, params, grads)
        ctx.psi = None
        return grads, None, None, None, None, None


def shots_gaussian_fn(params: torch.Tensor, circuit: Circuit, n_shots: float, z: torch.Tensor,
                      dtype=torch.complex64, basis_index: int = 0) -> torch.Tensor:
    """Differentiable approximate shots y (2^n values) of the circuit's
    output state for unit normals z."""
    return _ShotsGaussFn.apply(params, circuit, float(n_shots), z, dtype, basis_index)


class _ExpvalFn(torch.autograd.Function):
    """E(theta) = <psi_L|H|psi_L>, a scalar, so dL/dtheta = (dL/dE) dE/dtheta.
    When theta needs a gradient, forward runs the whole gradient evaluation
    at once (tqd_value_and_grad: the forward passes, E read off lambda = H
    psi_L, the adjoint reverse sweep of Sec. 4.4) and keeps only dE/dtheta;
    backward scales it.  Otherwise forward applies the circuit and measures E.
    No intermediate state is kept between the two."""

    @staticmethod
    def forward(ctx, params, circuit, obs, dtype, basis_index):
        psi = State(circuit.n, dtype, params.device).reset(basis_index)
        if not ctx.needs_input_grad[0]:
            apply(psi, circuit, params)
            return expval(psi, obs)
        lam = State(circuit.n, dtype, params.device)
        p64 = params.detach().to(torch.float64).contiguous()
        e, g = value_and_grad(psi, lam, circuit, p64, obs)
        ctx.save_for_backward(g)
        ctx.param_dtype = params.dtype
        return e

    @staticmethod
    def backward(ctx, grad_e):
        (g,) = ctx.saved_tensors
        return (grad_e.to(torch.float64) * g).to(ctx.param_dtype), None, None, None, None


class _MeasureFn(torch.autograd.Function):
    """Per-term values <P_j> (e.g. <Z_i>), differentiable with a vector grad."""

    @staticmethod
    def forward(ctx, params, circuit, obs, dtype, basis_index):
        psi = State(circuit.n, dtype, params.device).reset(basis_index)
        apply(psi, circuit, params)
        out = expval_terms(psi, obs)
        ctx.save_for_backward(params)
        ctx.psi, ctx.circuit, ctx.obs = psi, circuit, obs
        return out

    @staticmethod
    def backward(ctx, grad_out):
        (params,) = ctx.saved_tensors
        psi = ctx.psi
        if psi is None:
            raise RuntimeError("this measurement's backward already ran (the saved state is consumed)")
        lam = State(psi.n, psi.tensor.dtype, psi.device)
        # The per-term outputs <P_j> carry no coefficient, so the seed is
        # sum_j grad_j P_j psi: the same Pauli strings with unit coefficients,
        # weighted by the incoming gradient.
        unit = Observable([W.PauliTerm(1.0, t.ops) for t in ctx.obs.terms])
        w = grad_out.to(torch.float64).contiguous()
        grads = torch.zeros_like(params)
        backward(psi, lam, ctx.circuit, params, unit, grads, weights=w)
        ctx.psi = None
        return grads, None, None, None, None


def expval_fn(params: torch.Tensor, circuit: Circuit, obs, dtype=torch.complex64, basis_index: int = 0):
    return _ExpvalFn.apply(params, circuit, as_observable(obs), dtype, basis_index)


def measure_allz_fn(params: torch.Tensor, circuit: Circuit, dtype=torch.complex64, basis_index: int = 0):
    obs = Observable(W.all_z_terms(circuit.n))
    return _MeasureFn.apply(params, circuit, obs, dtype, basis_index)


# ------------------------------------------------------------------ profiling
def profile_enable(on: bool = True):
    _lib.check(_L().tqd_profile_enable(1 if on else 0))


def profile_read() -> list:
    """Per-kernel-class launches, total device ms and algorithmic bytes since
    the last enable/read (waits for the recorded events)."""
    cap = 64
    arr = (_lib.ProfileEntry * cap)()
    n = C.c_int()
    _lib.check(_L().tqd_profile_read(C.cast(arr, C.c_void_p), cap, C.byref(n)))
    return [{"name": arr[i].name.decode(), "launches": int(arr[i].launches), "ms": float(arr[i].total_ms),
             "bytes": float(arr[i].bytes)} for i in range(min(n.value, cap))]


# -------------------------------------------------------------------- batches
class _DevView:
    """Zero-copy torch view of a float64 device buffer owned by the library."""

    def __init__(self, ptr, n):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": "<f8", "data": (ptr, False), "version": 3,
                                         "strides": None}


class Batch:
    """Many independent circuits evaluated together (forward, E_c and the
    adjoint gradient of every E_c) by one CUDA-graph launch per run.

    ``circuits``: planned ``Circuit`` objects (distinct, complex64);
    ``observables``: one Pauli-term list per circuit.  After ``set_params``,
    ``run()`` fills ``energies`` and ``grads`` (device views; circuit c's
    angles and gradient at ``offsets[c]``)."""

    def __init__(self, circuits, observables, small_max_qubits=0, small_threads=0, streams=0, autotune=False,
                 plain=False):
        self.circuits = list(circuits)
        self.obs = [as_observable(o) for o in observables]
        n = len(self.circuits)
        handles = (C.c_void_p * n)(*[c.handle.value for c in self.circuits])
        tptrs = (C.c_void_p * n)(*[o.ptr.value for o in self.obs])
        counts = (C.c_size_t * n)(*[len(o) for o in self.obs])
        opts = _lib.BatchOpts()
        opts.small_max_qubits = small_max_qubits
        opts.small_threads = small_threads
        opts.streams = streams
        opts.autotune = 1 if autotune else 0
        opts.plain = 1 if plain else 0
        h = C.c_void_p()
        self.device = torch.device("cuda", torch.cuda.current_device())
        _lib.check(_L().tqd_batch_create(n, C.cast(handles, C.c_void_p), C.cast(tptrs, C.c_void_p),
                                         C.cast(counts, C.c_void_p), C.byref(opts), C.byref(h)))
        self._h = h
        p, e, g = C.c_void_p(), C.c_void_p(), C.c_void_p()
        offs = (C.c_size_t * n)()
        _lib.check(_L().tqd_batch_buffers(h, C.byref(p), C.byref(e), C.byref(g), C.cast(offs, C.c_void_p)))
        self.offsets = [int(x) for x in offs]
        self.n_params_total = sum(c.n_params for c in self.circuits)
        np_ = max(1, self.n_params_total)
        self.params = torch.as_tensor(_DevView(p.value, np_), device=self.device)
        self.energies = torch.as_tensor(_DevView(e.value, n), device=self.device)
        self.grads = torch.as_tensor(_DevView(g.value, np_), device=self.device)

    def set_params(self, arrays):
        flat = np.concatenate([np.asarray(a, dtype=np.float64).reshape(-1)[: c.n_params]
                               for a, c in zip(arrays, self.circuits)]) if self.n_params_total else np.zeros(0)
        if flat.size:
            self.params[: flat.size].copy_(torch.from_numpy(flat))

    def run(self):
        with torch.cuda.device(self.device):
            _lib.check(_L().tqd_batch_run(self._h, _stream(self.device)))

    def grads_of(self, c):
        return self.grads[self.offsets[c]: self.offsets[c] + self.circuits[c].n_params]

    def info(self) -> dict:
        v = [C.c_int() for _ in range(5)]
        _lib.check(_L().tqd_batch_info(self._h, *[C.byref(x) for x in v]))
        out = dict(zip(["small", "large", "small_max_qubits", "small_threads", "graph_nodes"], [x.value for x in v]))
        # the wider circuits' work items on the persistent kernel, by width
        tiling = {}
        for w in range(27):
            t, k = C.c_int(), C.c_int()
            _lib.check(_L().tqd_batch_tiling(self._h, w, C.byref(t), C.byref(k)))
            if k.value:
                tiling[w] = {"tiles_per_item": t.value, "items_per_stage": k.value}
        out["tiling"] = tiling
        return out

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            try:
                _L().tqd_batch_free(h)
            except Exception:
                pass
            self._h = None
