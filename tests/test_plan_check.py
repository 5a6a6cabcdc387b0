"""The fused planner on the host: every circuit's encoded passes, executed
from their descriptors (tile gathering, stage address tables, op positions,
forward and reverse), against the gates applied one by one, for both
precisions' descriptors.  No GPU: tqd_plan_check runs on the CPU.  It also
checks every barrier flag against the address tables: a point marked
"none" must keep every thread on its own amplitudes, one marked "warp" every
warp on its own (a weaker flag than the tables allow fails the check)."""
import numpy as np
import pytest

from paper_2511_19291_gb300 import sim as S
from paper_2511_19291_gb300 import workloads as W

TOL = 1e-12


def check(circ, params, seed=1):
    r = S.plan_check(circ, params, seed)
    assert r["err_forward"] < TOL, r
    assert r["err_reverse"] < TOL, r
    assert r["passes"] >= 1 and r["stages"] >= r["passes"]
    return r


@pytest.mark.parametrize("n,layers", [(12, 4), (13, 3), (14, 5), (16, 4), (18, 3)])
def test_ansatz_plans(n, layers):
    circ = W.hea_ansatz(n, layers)
    check(circ, W.config_rng(2).angles(circ.n_params))


@pytest.mark.parametrize("n,ng,seed", [(12, 150, 1), (13, 200, 2), (14, 300, 3), (16, 250, 4), (17, 120, 5)])
def test_random_plans_every_gate_kind(n, ng, seed):
    rng = W.SplitMix64(9100 + seed)
    circ, params = W.random_circuit(rng, n, ng, n_params=max(2, ng // 3))
    check(circ, params, seed)


@pytest.mark.parametrize("n", [12, 15])
def test_qft_then_ansatz_plan(n):
    circ = W.qft_then_hea(n, 2)
    check(circ, W.config_rng(5).angles(circ.n_params))


def test_ladder_plan():
    circ = W.ladder_ansatz(14, 4)
    check(circ, W.config_rng(4).angles(circ.n_params))


def test_permutation_only_plan():
    # CNOT rings and SWAPs only: whole passes are address maps (stages
    # without ops, folded loads and stores)
    n = 14
    gates = []
    for r in range(3):
        gates += [W.Gate("CNOT", (q, (q + 1 + r) % n)) for q in range(n)]
        gates += [W.Gate("SWAP", (q, (q + 5) % n)) for q in range(0, n, 3)]
        gates += [W.Gate("X", (q,)) for q in range(r, n, 4)]
    check(W.Circuit(n, gates, 0), np.zeros(1))


def test_plan_check_rejects_small_and_large():
    with pytest.raises(Exception):
        S.plan_check(W.hea_ansatz(8, 1), np.zeros(16))
    with pytest.raises(Exception):
        S.plan_check(W.hea_ansatz(21, 1), np.zeros(42))


def permutation_heavy(seed, n, ng):
    """Dense CNOT, SWAP and X among RY and RZ: many permutations folded into
    the stages' load and store maps, so every kind of barrier point occurs."""
    rng = W.SplitMix64(seed)
    gates, n_params = [], 0
    for _ in range(ng):
        r = rng.randint(0, 9)
        a = rng.randint(0, n - 1)
        b = (a + 1 + rng.randint(0, n - 2)) % n
        if r <= 3:
            gates.append(W.Gate("CNOT", (a, b)))
        elif r <= 5:
            gates.append(W.Gate("SWAP", (a, b)))
        elif r == 6:
            gates.append(W.Gate("X", (a,)))
        elif r == 7:
            gates.append(W.Gate("RY", (a,), param=n_params))
            n_params += 1
        else:
            gates.append(W.Gate("RZ", (a,), param=n_params))
            n_params += 1
    return W.Circuit(n, gates, n_params), rng.angles(max(1, n_params))


@pytest.mark.parametrize("n,ng,seed", [(12, 200, 1), (14, 300, 2), (16, 250, 3), (19, 150, 4)])
def test_permutation_heavy_plans(n, ng, seed):
    circ, params = permutation_heavy(9300 + seed, n, ng)
    check(circ, params, seed)


@pytest.mark.parametrize("n,layers", [(20, 2), (20, 6)])
def test_ansatz_plans_20_qubits(n, layers):
    """The ansatz at the largest host-checkable width, where windows of the
    26-qubit workload's kind (overlapping 8-qubit sets) appear."""
    circ = W.hea_ansatz(n, layers)
    check(circ, W.config_rng(5).angles(circ.n_params))


def diagonal_heavy(seed, n, ng):
    """Diagonal gates of every kind (RZ, PHASE, CPHASE, CZ, Z, S, T) on any
    qubits, among RY and H: many diagonal gates land on qubits outside a
    pass's set and are applied from the tile's index bits."""
    rng = W.SplitMix64(seed)
    gates, n_params = [], 0
    for _ in range(ng):
        r = rng.randint(0, 11)
        a = rng.randint(0, n - 1)
        b = (a + 1 + rng.randint(0, n - 2)) % n
        if r <= 2:
            gates.append(W.Gate("CPHASE", (a, b), param=n_params))
            n_params += 1
        elif r == 3:
            gates.append(W.Gate("CZ", (a, b)))
        elif r == 4:
            gates.append(W.Gate("RZ", (a,), param=n_params))
            n_params += 1
        elif r == 5:
            gates.append(W.Gate("PHASE", (a,), param=n_params))
            n_params += 1
        elif r == 6:
            gates.append(W.Gate(("Z", "S", "T")[rng.randint(0, 2)], (a,)))
        elif r == 7:
            gates.append(W.Gate("CPHASE", (a, b), angle=rng.angle()))
        elif r <= 9:
            gates.append(W.Gate("RY", (a,), param=n_params))
            n_params += 1
        else:
            gates.append(W.Gate("H", (a,)))
    return W.Circuit(n, gates, n_params), rng.angles(max(1, n_params))


@pytest.mark.parametrize("n,ng,seed", [(12, 200, 1), (16, 300, 2), (18, 400, 3), (20, 250, 4)])
def test_diagonal_heavy_plans(n, ng, seed):
    circ, params = diagonal_heavy(9400 + seed, n, ng)
    check(circ, params, seed)


@pytest.mark.parametrize("n", [16, 18, 20])
def test_qft_passes(n):
    """The QFT's controlled phases on qubits outside a pass's set are applied
    from the tile's bits, so each pass takes the Hadamards of 8 new qubits
    (Q = qubits 0..3 and 8 others): ceil((n - 4) / 8) + 1 passes, the last of
    them the bit-reversal swaps."""
    r = check(W.qft_circuit(n), np.zeros(1))
    assert r["passes"] <= -(-(n - 4) // 8) + 2, r


@pytest.mark.parametrize("n,seed", [(17, 1), (19, 2), (20, 3)])
def test_scattered_qubit_plans(n, seed):
    """Dense two-qubit gates between distant qubits: passes whose first gate
    forces a scattered qubit set (runs and gaps beyond the tensor map's five
    dimensions, so separate box copies in one precision or both), while the
    rest of each set avoids them; every pass still reproduces the gates."""
    rng = W.SplitMix64(9300 + seed)
    gates, p = [], 0
    for layer in range(4):
        for k in range(n // 2):
            a = rng.randint(4, n - 1)
            b = rng.randint(4, n - 1)
            if a == b:
                continue
            gates.append(W.Gate("UNITARY2", (a, b), matrix=W.random_unitary(rng, 4)))
            gates.append(W.Gate("RY", (a,), param=p))
            p += 1
        gates += [W.Gate("CNOT", (q, (q + 7) % n)) for q in range(0, n, 3)]
    circ = W.Circuit(n, gates, p)
    check(circ, W.config_rng(6).angles(p), seed)


@pytest.mark.parametrize("n,layers", [(12, 4), (14, 6)])
def test_small_state_long_passes(n, layers):
    """States of at most 14 qubits take up to 104 angles per pass: the
    12-qubit, 4-layer ansatz plans to its 96 angles' pass and the closing
    CNOT ring's pass."""
    circ = W.hea_ansatz(n, layers)
    r = check(circ, W.config_rng(1).angles(circ.n_params))
    if (n, layers) == (12, 4):
        assert r["passes"] == 2, r
