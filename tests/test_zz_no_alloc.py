"""tqd_expval_noalloc against tqd_expval, through the C ABI.

The no-allocation variant exists for callers that may not allocate device
memory while they run (fixed memory budgets, latency-sensitive loops, hosts
that own the allocator).  It must give the same expectation value as the
allocating entry point, call after call, even though every call reuses the
same fixed scratch array.  This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2511_19291_gb300 import _lib
from paper_2511_19291_gb300 import workloads as W
from gpu_helpers import E_TOL, gpu_state, sim

pytestmark = pytest.mark.gpu


def noalloc_expval(state, obs):
    out = torch.full((), float("nan"), dtype=torch.float64, device=state.device)
    st = _lib.load().tqd_expval_noalloc(state.handle, obs.ptr, len(obs), C.c_void_p(out.data_ptr()),
                                        C.c_void_p(torch.cuda.current_stream(state.device).cuda_stream))
    _lib.check(st)
    return out


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_noalloc_matches_expval_two_calls_in_a_row(dtype):
    S = sim()
    cases = []
    for seed, n in ((1, 14), (2, 9)):
        rng = W.SplitMix64(7000 + seed)
        circ, params = W.random_circuit(rng, n, 80)
        terms = W.random_pauli_terms(rng, n, 25) + W.ising(n)
        st, _, _ = gpu_state(circ, params, "fused", dtype)
        cases.append((st, S.Observable(terms)))
    # two calls in a row on different states and observables, then repeat
    for _ in range(2):
        for st, obs in cases:
            got = noalloc_expval(st, obs).item()
            ref = S.expval(st, obs).item()
            assert np.isfinite(got)
            assert abs(got - ref) <= E_TOL[dtype], (got, ref)


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_noalloc_against_oracle(dtype):
    """Directly against the oracle's expectation value (Sec. 2.2.1), twice in
    a row on the same state."""
    import oracle
    S = sim()
    n = 13
    rng = W.SplitMix64(7100)
    circ, params = W.random_circuit(rng, n, 70)
    terms = W.random_pauli_terms(rng, n, 20) + W.ising(n)
    st, _, _ = gpu_state(circ, params, "fused", dtype)
    ref = oracle.expval(n, oracle.run(circ, params), terms)[0]
    obs = S.Observable(terms)
    for _ in range(2):
        got = noalloc_expval(st, obs).item()
        assert abs(got - ref) <= E_TOL[dtype], (got, ref)


def test_noalloc_empty_and_too_large():
    S = sim()
    st, _, _ = gpu_state(W.hea_ansatz(12, 1), np.zeros(24), "fused", "c64")
    assert noalloc_expval(st, S.Observable([])).item() == 0.0
    # more distinct x masks than the fixed scratch can hold: clear rejection.
    # At 16 qubits a launch uses 128 blocks, so 1100 masks need 1100 * 129
    # doubles > TQD_NOALLOC_SCRATCH_DOUBLES.
    n = 16
    big, _, _ = gpu_state(W.hea_ansatz(n, 1), np.zeros(2 * n), "fused", "c64")
    many = [W.PauliTerm(1.0, tuple((q, "X") for q in range(n) if (m >> q) & 1)) for m in range(1, 1101)]
    with pytest.raises(_lib.TqdError, match="scratch"):
        noalloc_expval(big, S.Observable(many))
    # a request that fits still works after the rejection
    few = S.Observable(many[:40])
    assert abs(noalloc_expval(big, few).item() - S.expval(big, few).item()) <= 1e-5
