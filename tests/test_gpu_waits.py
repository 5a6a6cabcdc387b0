"""The give-up path of the bounded device waits.

Every spin wait in the tile kernels gives up after about one second of
elapsed time (the device's global timer), records code 1 in the circuit's
error word and lets its block return.  Here the test hook
tqd_circuit_test_stall makes block 0 of every fused pass wait for a tile
copy that is never issued (its barrier is armed, nothing will complete it):
the launch must end by itself, tqd_circuit_check must report
TQD_ERR_TIMEOUT, and the context must stay usable -- the same circuit then
gives the oracle's state again.  No kernel traps, faults or hangs: the wait
that runs out is the library's own bounded wait.
"""
import ctypes as C
import time

import numpy as np
import pytest
import torch

import oracle
from paper_2511_19291_gb300 import _lib
from paper_2511_19291_gb300 import workloads as W
from gpu_helpers import AMP_TOL, params_tensor, sim, to_numpy

pytestmark = pytest.mark.gpu


def one_pass_circuit(n):
    """RY layers and CNOT chains on qubits 0..11 only, ending in RY (no
    permutation tail): one fused pass."""
    gates = []
    p = 0
    for layer in range(2):
        for q in range(12):
            gates.append(W.Gate("RY", (q,), param=p))
            p += 1
        if layer < 1:
            for q in range(11):
                gates.append(W.Gate("CNOT", (q, q + 1)))
    return W.Circuit(n, gates, p, name=f"stall{n}")


@pytest.mark.parametrize("n", [21, 22])
def test_stalled_tile_wait_runs_out_and_reports_timeout(n):
    """n = 21: the generic ring kernel; n = 22: the pass-specialised one."""
    S = sim()
    circ = one_pass_circuit(n)
    params = W.config_rng(11).angles(circ.n_params)
    c = S.Circuit(circ)
    assert c.info()["passes"] == 1
    p = params_tensor(params)
    st = S.State(n, torch.complex64).reset(0)
    c.test_stall(True)
    t0 = time.time()
    S.apply(st, c, p)
    with pytest.raises(_lib.TqdError) as ei:
        c.check()
    waited = time.time() - t0
    assert ei.value.status == 5  # TQD_ERR_TIMEOUT
    assert "gave up" in str(ei.value)
    assert 0.5 < waited < 30.0, waited
    # the word was cleared by the check; the context still works
    c.test_stall(False)
    assert c.check() == 0
    st.reset(0)
    S.apply(st, c, p)
    assert c.check() == 0
    ref = oracle.run(circ, params)
    got = to_numpy(st)
    assert np.max(np.abs(got - ref)) <= AMP_TOL["c64"]


def test_stalled_reverse_sweep_reports_timeout():
    """The reverse ring (two groups sharing three buffers, so a buffer passes
    between groups and its next taker waits on a tile count as well): the
    stalled group's partner and the TMA warpgroup wait for tiles that never
    come, run out too, and the block still returns."""
    S = sim()
    n = 22
    circ = one_pass_circuit(n)
    params = W.config_rng(12).angles(circ.n_params)
    terms = W.sum_z(n)
    c = S.Circuit(circ)
    p = params_tensor(params)
    psi = S.State(n, torch.complex64).reset(0)
    lam = S.State(n, torch.complex64)
    c.test_stall(True)
    S.value_and_grad(psi, lam, c, p, terms)
    with pytest.raises(_lib.TqdError) as ei:
        c.check()
    assert ei.value.status == 5
    c.test_stall(False)
    psi.reset(0)
    e, g = S.value_and_grad(psi, lam, c, p, terms)
    assert c.check() == 0
    assert abs(e.item() - oracle.energy(circ, params, terms)) <= 1e-5
    assert np.all(np.isfinite(g.cpu().numpy()))
