"""GPU parity: the CUDA path through the C ABI against the CPU oracle, element
by element on the same seeded inputs (states, expectations, H psi, gradients),
for both plans (gate-by-gate and fused) and both precisions."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2511_19291_gb300 import workloads as W
from gpu_helpers import (AMP_TOL, DTYPES, E_TOL, G_REL, all_kinds_circuit, gpu_state, grad_close,
                         params_tensor, sim, to_numpy)

pytestmark = pytest.mark.gpu
MODES = ["plain", "fused"]


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("n,ng,seed", [(1, 12, 1), (2, 30, 2), (3, 60, 3), (4, 80, 4), (5, 120, 5),
                                       (8, 200, 6), (11, 300, 7), (13, 300, 8), (14, 250, 9), (17, 120, 10)])
def test_state_parity_all_gate_kinds(mode, dtype, n, ng, seed):
    circ, params = all_kinds_circuit(1000 + seed, n, ng)
    st, _, _ = gpu_state(circ, params, mode, dtype, basis=(seed * 7919) % (1 << n))
    ref = oracle.run(circ, params, (seed * 7919) % (1 << n))
    got = to_numpy(st)
    tol = AMP_TOL[dtype] * math.sqrt(ng / 100 + 1)
    np.testing.assert_allclose(got, ref, atol=tol, rtol=0)


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("n,layers", [(4, 2), (12, 4), (13, 3), (15, 2)])
def test_ansatz_state_parity(mode, n, layers):
    circ = W.hea_ansatz(n, layers)
    params = W.config_rng(1).angles(circ.n_params)
    st, _, _ = gpu_state(circ, params, mode, "c64")
    np.testing.assert_allclose(to_numpy(st), oracle.run(circ, params), atol=4e-6, rtol=0)


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("n,seed", [(1, 1), (3, 2), (6, 3), (12, 4), (15, 5)])
def test_expval_parity(dtype, n, seed):
    S = sim()
    rng = W.SplitMix64(2000 + seed)
    circ, params = W.random_circuit(rng, n, 40 + 10 * n)
    terms = W.random_pauli_terms(rng, n, 30) + (W.ising(n) if n > 1 else []) + W.sum_z(n)
    st, _, _ = gpu_state(circ, params, "fused", dtype)
    psi = oracle.run(circ, params)
    e_ref, per_ref = oracle.expval(n, psi, terms)
    e = S.expval(st, terms).item()
    per = S.expval_terms(st, terms).cpu().numpy()
    assert abs(e - e_ref) <= E_TOL[dtype], (e, e_ref)
    np.testing.assert_allclose(per, per_ref, atol=E_TOL[dtype], rtol=0)


def spin_terms(rng, n, kind):
    """Observables of the shapes the tile expectation kernels distinguish:
    one-qubit X fields alone; Z strings (ZZ chain, Z fields, a long Z string)
    with X fields; and the same plus two-qubit X strings and a Y term (the
    general kernel).  Coefficients random in [-1, 1)."""
    c = lambda: rng.uniform01() * 2.0 - 1.0
    xs = [W.PauliTerm(c(), ((i, "X"),)) for i in range(n)]
    if kind == "x":
        return xs
    zs = [W.PauliTerm(c(), ((i, "Z"), (i + 1, "Z"))) for i in range(n - 1)]
    zs += [W.PauliTerm(c(), ((i, "Z"),)) for i in range(0, n, 3)]
    zs += [W.PauliTerm(c(), tuple((q, "Z") for q in range(0, n, 2)))]
    if kind == "zx":
        return zs + xs
    return zs + xs + [W.PauliTerm(c(), ((i, "X"), (i + 5, "X"))) for i in range(0, n - 5, 4)] + \
        [W.PauliTerm(c(), ((1, "Y"), (n - 1, "Z")))]


@pytest.mark.parametrize("kind", ["x", "zx", "general"])
@pytest.mark.parametrize("n", [12, 14, 17])
def test_expval_tile_kernels_parity(kind, n):
    """E of the spin-model shapes on 12..17 qubits (every tile launch: the
    X-only kernel with its three register layouts, the one that also carries
    the real diagonal group, and the general kernel) against the oracle, in
    complex64 and complex128."""
    S = sim()
    rng = W.SplitMix64(5100 + n)
    circ, params = W.random_circuit(rng, n, 60 + 10 * n)
    terms = spin_terms(rng, n, kind)
    psi = oracle.run(circ, params)
    e_ref, _ = oracle.expval(n, psi, terms)
    for dtype in ("c64", "c128"):
        st, _, _ = gpu_state(circ, params, "fused", dtype)
        e = S.expval(st, terms).item()
        assert abs(e - e_ref) <= E_TOL[dtype], (dtype, e, e_ref)


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("n,seed", [(2, 1), (7, 2), (13, 3)])
def test_apply_observable_parity(dtype, n, seed):
    S = sim()
    rng = W.SplitMix64(3000 + seed)
    circ, params = W.random_circuit(rng, n, 60)
    terms = W.random_pauli_terms(rng, n, 20) + W.ising(n)
    st, _, _ = gpu_state(circ, params, "fused", dtype)
    out = S.apply_observable(st, terms)
    ref = oracle.apply_observable(n, oracle.run(circ, params), terms)
    np.testing.assert_allclose(to_numpy(out), ref, atol=AMP_TOL[dtype] * 30, rtol=0)
    w = np.linspace(-1.5, 2.0, len(terms))
    outw = S.apply_observable(st, terms, weights=params_tensor(w))
    terms_w = [W.PauliTerm(t.coeff * wi, t.ops) for t, wi in zip(terms, w)]
    refw = oracle.apply_observable(n, oracle.run(circ, params), terms_w)
    np.testing.assert_allclose(to_numpy(outw), refw, atol=AMP_TOL[dtype] * 60, rtol=0)


def gpu_grad(circ, params, terms, mode, dtype, weights=None, scale=1.0, **kw):
    S = sim()
    st, c, p = gpu_state(circ, params, mode, dtype, **kw)
    lam = S.State(circ.n_qubits, DTYPES[dtype])
    g = torch.zeros(circ.n_params, dtype=torch.float64, device="cuda")
    S.backward(st, lam, c, p, terms, g, weights=weights, scale=scale)
    torch.cuda.synchronize()
    return g.cpu().numpy(), st


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("n,ng,seed", [(1, 10, 1), (2, 20, 2), (3, 40, 3), (5, 60, 4), (6, 80, 5), (9, 60, 6)])
def test_gradient_parity_random(mode, dtype, n, ng, seed):
    rng = W.SplitMix64(4000 + seed)
    circ, params = W.random_circuit(rng, n, ng, n_params=max(2, ng // 3))
    terms = W.random_pauli_terms(rng, n, 8) + W.sum_z(n)
    ref = oracle.grad_param_shift(circ, params, terms)
    g, st = gpu_grad(circ, params, terms, mode, dtype)
    ok, worst = grad_close(g, ref, G_REL[dtype])
    assert ok, f"worst relative error {worst}"
    # the reverse sweep leaves the input state |0...0> behind
    back = to_numpy(st)
    e0 = np.zeros(1 << n, dtype=complex)
    e0[0] = 1
    np.testing.assert_allclose(back, e0, atol=AMP_TOL[dtype] * 10 * math.sqrt(ng), rtol=0)


TILE_VARIANTS = {"generic": dict(jit=1), "generic_2buf": dict(jit=1, buffers=2), "specialised": dict(jit=2),
                 "generic_ring": dict(jit=1, buffers=3, max_blocks=2),
                 "specialised_ring": dict(jit=2, buffers=3, max_blocks=2),
                 # the ring with a TMA warpgroup whose registers go to the groups
                 "generic_ring_tma": dict(jit=1, buffers=4, max_blocks=2),
                 "specialised_ring_tma": dict(jit=2, buffers=4, max_blocks=3)}


@pytest.mark.parametrize("variant", list(TILE_VARIANTS))
@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("n,ng,seed", [(12, 80, 1), (14, 120, 2), (16, 60, 3)])
def test_fused_tile_variants_random(variant, dtype, n, ng, seed):
    """Fused passes through the generic kernel with one and two tile buffers
    per block, and through the pass-specialised kernels: random gate lists
    over every kind (several passes, ragged stage schedules), forward state
    and gradient against the oracle."""
    kw = TILE_VARIANTS[variant]
    rng = W.SplitMix64(6000 + seed)
    circ, params = W.random_circuit(rng, n, ng, n_params=max(2, ng // 3))
    terms = W.random_pauli_terms(rng, n, 6) + W.sum_z(n)
    st, _, _ = gpu_state(circ, params, "fused", dtype, **kw)
    tol = AMP_TOL[dtype] * math.sqrt(ng / 100 + 1)
    np.testing.assert_allclose(to_numpy(st), oracle.run(circ, params), atol=tol, rtol=0)
    del st
    ref = oracle.grad_param_shift(circ, params, terms)
    g, st = gpu_grad(circ, params, terms, "fused", dtype, **kw)
    ok, worst = grad_close(g, ref, G_REL[dtype])
    assert ok, f"worst relative error {worst}"
    back = to_numpy(st)
    e0 = np.zeros(1 << n, dtype=complex)
    e0[0] = 1
    np.testing.assert_allclose(back, e0, atol=AMP_TOL[dtype] * 10 * math.sqrt(ng), rtol=0)


@pytest.mark.parametrize("jit", [1, 2])
@pytest.mark.parametrize("buffers", [3, 4])
@pytest.mark.parametrize("n,layers,max_blocks", [(15, 2, 1), (17, 2, 3)])
def test_ring_many_tiles_per_block(jit, buffers, n, layers, max_blocks):
    """Ring kernels with few blocks, so that each block cycles through many
    tiles: buffers are refilled after their stores and (reverse sweep: 3
    buffers, 2 groups) handed from one group to the other.  The ansatz with
    the Ising observable, energy and gradient against the oracle."""
    circ = W.hea_ansatz(n, layers)
    params = W.config_rng(3).angles(circ.n_params)
    terms = W.ising(n)
    ref = oracle.grad_param_shift(circ, params, terms)
    e_ref = oracle.energy(circ, params, terms)
    kw = dict(jit=jit, buffers=buffers, max_blocks=max_blocks)
    st, _, _ = gpu_state(circ, params, "fused", "c64", **kw)
    assert abs(sim().expval(st, terms).item() - e_ref) < E_TOL["c64"]
    np.testing.assert_allclose(to_numpy(st), oracle.run(circ, params), atol=AMP_TOL["c64"] * 4, rtol=0)
    del st
    g, st = gpu_grad(circ, params, terms, "fused", "c64", **kw)
    ok, worst = grad_close(g, ref, G_REL["c64"])
    assert ok, f"worst relative error {worst}"
    back = to_numpy(st)
    e0 = np.zeros(1 << n, dtype=complex)
    e0[0] = 1
    np.testing.assert_allclose(back, e0, atol=AMP_TOL["c64"] * 40, rtol=0)


@pytest.mark.parametrize("jit", [1, 2])
def test_specialised_ansatz_ising_14q(jit):
    """The ansatz workload's form at 14 qubits through the generic and the
    pass-specialised kernels: energy and gradient against the oracle."""
    circ = W.hea_ansatz(14, 3)
    params = W.config_rng(3).angles(circ.n_params)
    terms = W.ising(14)
    ref = oracle.grad_param_shift(circ, params, terms)
    e_ref = oracle.energy(circ, params, terms)
    for dtype in ("c64", "c128"):
        st, _, _ = gpu_state(circ, params, "fused", dtype, jit=jit)
        assert abs(sim().expval(st, terms).item() - e_ref) < E_TOL[dtype]
        del st
        g, _ = gpu_grad(circ, params, terms, "fused", dtype, jit=jit)
        ok, worst = grad_close(g, ref, G_REL[dtype])
        assert ok, f"{dtype}: worst relative error {worst}"


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("n,layers", [(6, 3), (12, 2), (14, 2)])
def test_gradient_parity_ansatz_ising(mode, n, layers):
    circ = W.hea_ansatz(n, layers)
    params = W.config_rng(3).angles(circ.n_params)
    terms = W.ising(n)
    ref = oracle.grad_param_shift(circ, params, terms)
    for dtype in ("c64", "c128"):
        g, _ = gpu_grad(circ, params, terms, mode, dtype)
        ok, worst = grad_close(g, ref, G_REL[dtype])
        assert ok, f"{dtype}: worst relative error {worst}"


@pytest.mark.parametrize("mode", MODES)
def test_gradient_weights_and_scale(mode):
    n = 7
    rng = W.SplitMix64(4500)
    circ, params = W.random_circuit(rng, n, 70, n_params=20)
    terms = W.random_pauli_terms(rng, n, 6)
    w = np.array([0.5, -1.0, 2.0, 0.0, 1.5, -0.25])
    scale = 0.75
    ref = oracle.grad_param_shift(circ, params, [W.PauliTerm(t.coeff * wi * scale, t.ops) for t, wi in zip(terms, w)])
    g, _ = gpu_grad(circ, params, terms, mode, "c128", weights=params_tensor(w), scale=scale)
    ok, worst = grad_close(g, ref, 1e-10)
    assert ok, worst


def test_gradients_accumulate():
    n = 5
    circ = W.hea_ansatz(n, 2)
    params = W.config_rng(3).angles(circ.n_params)
    ref = oracle.grad_param_shift(circ, params, W.sum_z(n))
    S = sim()
    st, c, p = gpu_state(circ, params, "fused", "c128")
    lam = S.State(n, torch.complex128)
    g = torch.full((circ.n_params,), 1.0, dtype=torch.float64, device="cuda")
    S.backward(st, lam, c, p, W.sum_z(n), g)
    np.testing.assert_allclose(g.cpu().numpy(), ref + 1.0, atol=1e-11)


@pytest.mark.parametrize("mode", MODES)
def test_autograd_function(mode):
    S = sim()
    n = 10
    circ = W.hea_ansatz(n, 3)
    params = W.config_rng(3).angles(circ.n_params)
    c = S.Circuit(circ, mode=mode)
    p = params_tensor(params).requires_grad_(True)
    e = S.expval_fn(p, c, W.ising(n))
    (2.5 * e).backward()
    ref_e = oracle.energy(circ, params, W.ising(n))
    ref_g = oracle.grad_param_shift(circ, params, W.ising(n))
    assert abs(e.item() - ref_e) < 1e-5
    ok, worst = grad_close(p.grad.cpu().numpy(), 2.5 * ref_g, 1e-4)
    assert ok, worst


@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_autograd_function_paths(dtype):
    """expval_fn with angles that need no gradient (apply and measure only),
    with float32 angles (the gradient comes back in float32) and on a
    complex128 state, against the oracle; a second backward through the same
    graph is refused by torch as usual."""
    S = sim()
    n = 13
    circ = W.hea_ansatz(n, 2)
    params = W.config_rng(8).angles(circ.n_params)
    terms = W.ising(n)
    c = S.Circuit(circ)
    ref_e = oracle.energy(circ, params, terms)
    ref_g = oracle.grad_param_shift(circ, params, terms)
    e0 = S.expval_fn(params_tensor(params), c, terms, dtype=DTYPES[dtype])
    assert not e0.requires_grad and abs(e0.item() - ref_e) < E_TOL[dtype], (e0.item(), ref_e)
    p32 = torch.tensor(params, dtype=torch.float32, device="cuda", requires_grad=True)
    e = S.expval_fn(p32, c, terms, dtype=DTYPES[dtype])
    (-0.5 * e).backward()
    assert p32.grad.dtype == torch.float32
    # float32 angles: compare with the oracle at the rounded angles
    p_r = p32.detach().double().cpu().numpy()
    ok, worst = grad_close(p32.grad.double().cpu().numpy(), -0.5 * oracle.grad_param_shift(circ, p_r, terms),
                           1e-4)
    assert ok, worst
    p64 = params_tensor(params).requires_grad_(True)
    e = S.expval_fn(p64, c, terms, dtype=DTYPES[dtype])
    e.backward(retain_graph=False)
    ok, worst = grad_close(p64.grad.cpu().numpy(), ref_g, G_REL[dtype])
    assert ok, worst
    with pytest.raises(RuntimeError):
        e.backward()


def test_measure_allz_autograd():
    S = sim()
    n = 6
    circ = W.ladder_ansatz(n, 3)
    params = W.config_rng(2).angles(circ.n_params)
    c = S.Circuit(circ)
    p = params_tensor(params).requires_grad_(True)
    z = S.measure_allz_fn(p, c, dtype=torch.complex128)
    psi = oracle.run(circ, params)
    _, ref = oracle.expval(n, psi, W.all_z_terms(n))
    np.testing.assert_allclose(z.detach().cpu().numpy(), ref, atol=1e-12)
    wts = torch.linspace(-1, 1, n, dtype=torch.float64, device="cuda")
    (z * wts).sum().backward()
    terms = [W.PauliTerm(float(wi), t.ops) for t, wi in zip(W.all_z_terms(n), wts.cpu().numpy())]
    ok, worst = grad_close(p.grad.cpu().numpy(), oracle.grad_param_shift(circ, params, terms), 1e-10)
    assert ok, worst


def test_basic_example_allz():
    import json, os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "basic_example.json")))
    n = g["n_qubits"]
    gates = [W.Gate(k, tuple(w), angle=a) for k, w, a in g["gates"]]
    st, _, _ = gpu_state(W.Circuit(n, gates, 0), None, "fused", "c64")
    z = sim().expval_terms(st, W.all_z_terms(n)).cpu().numpy()
    np.testing.assert_allclose(z, g["expected_allZ"], atol=1e-6)


def test_empty_circuit_and_empty_observable():
    S = sim()
    for n in (1, 5, 13):
        st, _, _ = gpu_state(W.Circuit(n, [], 0), None, "fused", "c64", basis=1)
        got = to_numpy(st)
        ref = np.zeros(1 << n, dtype=complex)
        ref[1] = 1
        np.testing.assert_array_equal(got, ref)
        assert S.expval(st, []).item() == 0.0
        assert S.expval(st, [W.PauliTerm(1.0, ((0, "Z"),))]).item() == pytest.approx(-1.0)


def test_small_workload_config():
    """12 qubits, 4 layers, sum_i Z_i: complex64 against the complex128 oracle."""
    S = sim()
    w = W.workload_small()
    st, _, _ = gpu_state(w.circuit, w.params, "fused", "c64")
    e = S.expval(st, w.terms).item()
    assert abs(e - oracle.energy(w.circuit, w.params, w.terms)) <= 1e-5


def test_invalid_state_use_raises():
    S = sim()
    circ = W.hea_ansatz(4, 1)
    c = S.Circuit(circ)
    st = S.State(5)
    with pytest.raises(Exception, match="qubits"):
        S.apply(st, c, params_tensor(np.zeros(circ.n_params)))
    with pytest.raises(Exception, match="qubit"):
        S.expval(st, [W.PauliTerm(1.0, ((7, "Z"),))])


def tc_circuit(seed, n, blocks):
    """Runs of 40 random gates (every kind) on qubits 0..5, each followed by RY
    on the other qubits and two CNOTs that leave the block."""
    rng = W.SplitMix64(seed)
    gates, n_params = [], 0
    for _ in range(blocks):
        c6, _ = W.random_circuit(rng, 6, 40, n_params=8)
        for g in c6.gates:
            gates.append(W.Gate(g.kind, g.wires, g.param + n_params if g.param >= 0 else -1, g.angle, g.matrix))
        n_params += 8
        for q in range(6, n):
            gates.append(W.Gate("RY", (q,), param=n_params))
            n_params += 1
        gates.append(W.Gate("CNOT", (5, 6)))
        gates.append(W.Gate("CNOT", (n - 1, 0)))
    return W.Circuit(n, gates, n_params), rng.angles(n_params)


@pytest.mark.parametrize("n,blocks,seed", [(12, 2, 1), (14, 3, 2), (17, 2, 3)])
def test_tensor_core_blocks(n, blocks, seed):
    tensor_core_case(n, blocks, seed)


@pytest.mark.parametrize("n,blocks,max_blocks,seed", [(15, 2, 2, 4), (17, 3, 3, 5), (16, 1, 1, 6)])
def test_tensor_core_blocks_pipelined(n, blocks, max_blocks, seed):
    """Few blocks, so that each block runs many 64-column tiles through the
    double-buffered loads and accumulators (tile k's MMAs overlapping tile
    k - 1's epilogue and the loads of tiles k + 1, k + 2)."""
    tensor_core_case(n, blocks, seed, max_blocks=max_blocks)


def tensor_core_case(n, blocks, seed, **kw):
    """Fused 6-qubit blocks on the tensor cores (split-precision TF32) in the
    forward pass; the reverse sweep runs the same gates through tile passes."""
    S = sim()
    circ, params = tc_circuit(8000 + seed, n, blocks)
    terms = W.ising(n) + W.random_pauli_terms(W.SplitMix64(seed), n, 5)
    S.profile_enable(True)
    st, c, p = gpu_state(circ, params, "tc", "c64", **kw)
    torch.cuda.synchronize()
    prof = {q["name"]: q for q in S.profile_read()}
    S.profile_enable(False)
    assert prof.get("tc_block", {}).get("launches", 0) >= 1
    ref = oracle.run(circ, params)
    # the amplitude bar of the other parity tests: TF32 hi/lo products with
    # FP32 accumulation lose about 2^-21 of each 128-term dot product, well
    # inside it
    err = float(np.max(np.abs(to_numpy(st) - ref)))
    tol = AMP_TOL["c64"] * math.sqrt(len(circ.gates) / 100 + 1)
    print(f"\ntensor-core block, n={n}: max amplitude error {err:.2e} (bar {tol:.2e})")
    assert err <= tol, (err, tol)
    e_ref, g_ref = oracle.grad_stored(circ, params, terms)
    assert abs(S.expval(st, terms).item() - e_ref) < 1e-5
    lam = S.State(n, torch.complex64)
    g = torch.zeros(circ.n_params, dtype=torch.float64, device="cuda")
    S.backward(st, lam, c, p, terms, g)
    ok, worst = grad_close(g.cpu().numpy(), g_ref, 1e-4)
    assert ok, worst
    # complex128 states take the tile path for the same plan
    st2, _, _ = gpu_state(circ, params, "tc", "c128", **kw)
    np.testing.assert_allclose(to_numpy(st2), ref, atol=1e-12, rtol=0)


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("n,layers,extra", [(13, 3, False), (15, 2, True)])
def test_value_and_grad(mode, dtype, n, layers, extra):
    """tqd_value_and_grad (E read off lambda = H psi) against the oracle's
    energy and parameter-shift gradient, and psi restored.  `extra` adds
    Pauli strings that flip more than 8 qubits above qubit 3 (groups outside
    the 12-qubit tiles: E then comes from a separate pass over psi and
    lambda)."""
    S = sim()
    circ = W.hea_ansatz(n, layers)
    params = W.config_rng(3).angles(circ.n_params)
    terms = W.ising(n)
    if extra:
        wide = tuple((q, "X") for q in range(4, n)) + ((0, "Y"),)
        terms = terms + [W.PauliTerm(0.3, wide)] + W.random_pauli_terms(W.SplitMix64(77), n, 4)
    e_ref = oracle.energy(circ, params, terms)
    g_ref = oracle.grad_param_shift(circ, params, terms)
    c = S.Circuit(circ, mode=mode)
    psi = S.State(n, DTYPES[dtype]).reset(0)
    lam = S.State(n, DTYPES[dtype])
    p = params_tensor(params)
    for rep in range(2):  # twice in a row: the state comes back to |0...0>
        e, g = S.value_and_grad(psi, lam, c, p, terms)
        torch.cuda.synchronize()
        assert abs(e.item() - e_ref) < E_TOL[dtype], (rep, e.item(), e_ref)
        ok, worst = grad_close(g.cpu().numpy(), g_ref, G_REL[dtype])
        assert ok, worst
    back = to_numpy(psi)
    e0 = np.zeros(1 << n, dtype=complex)
    e0[0] = 1
    np.testing.assert_allclose(back, e0, atol=AMP_TOL[dtype] * 200, rtol=0)


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("checkpoints", [None, 0, 2])
def test_value_and_grad_permutation_tail(dtype, checkpoints):
    """A circuit ending in CNOT, SWAP and X gates: tqd_value_and_grad skips
    the tail passes and conjugates the observable through them (Pauli
    strings with X, Y and Z, so every sign rule is used)."""
    S = sim()
    n = 14
    circ = W.hea_ansatz(n, 2)
    tail = [W.Gate("SWAP", (0, 5)), W.Gate("X", (3,)), W.Gate("CNOT", (2, 7)), W.Gate("SWAP", (4, 13)),
            W.Gate("X", (12,)), W.Gate("CNOT", (13, 1)), W.Gate("CNOT", (6, 11)), W.Gate("X", (6,))]
    circ = W.Circuit(n, list(circ.gates) + tail, circ.n_params)
    params = W.config_rng(4).angles(circ.n_params)
    terms = W.ising(n) + W.random_pauli_terms(W.SplitMix64(91), n, 8)
    e_ref = oracle.energy(circ, params, terms)
    g_ref = oracle.grad_param_shift(circ, params, terms)
    c = S.Circuit(circ, mode="fused", checkpoints=checkpoints)
    psi = S.State(n, DTYPES[dtype]).reset(0)
    lam = S.State(n, DTYPES[dtype])
    e, g = S.value_and_grad(psi, lam, c, params_tensor(params), terms)
    torch.cuda.synchronize()
    assert abs(e.item() - e_ref) < E_TOL[dtype], (e.item(), e_ref)
    ok, worst = grad_close(g.cpu().numpy(), g_ref, G_REL[dtype])
    assert ok, worst
    back = to_numpy(psi)
    assert abs(back[0] - 1) < AMP_TOL[dtype] * 200


def _adj_bytes_expected(n, dtype, n_passes, k):
    """Algorithmic bytes of a reverse sweep whose last k passes read psi from
    forward checkpoints (psi read, lambda read and written) and whose others
    recompute psi in place (psi and lambda read and written)."""
    sb = (1 << n) * (8 if dtype == "c64" else 16)
    return sb * (3 * k + 4 * (n_passes - k))


@pytest.mark.parametrize("dtype", ["c64", "c128"])
@pytest.mark.parametrize("checkpoints", [None, 0, 1, 3])
@pytest.mark.parametrize("jit", [1, 2])
def test_value_and_grad_checkpoints(dtype, checkpoints, jit):
    """Forward checkpoints (all passes, none, the last one, the last three):
    the same energy and gradient as the oracle; psi is never written when
    every pass has a checkpoint and comes back by recomputation otherwise;
    the reverse passes that read a checkpoint move 3 states, the others 4."""
    S = sim()
    n = 14
    circ = W.hea_ansatz(n, 3)
    params = W.config_rng(6).angles(circ.n_params)
    terms = W.ising(n) + W.random_pauli_terms(W.SplitMix64(17), n, 4)
    e_ref = oracle.energy(circ, params, terms)
    g_ref = oracle.grad_param_shift(circ, params, terms)
    c = S.Circuit(circ, mode="fused", checkpoints=checkpoints, jit=jit)
    psi = S.State(n, DTYPES[dtype]).reset(0)
    lam = S.State(n, DTYPES[dtype])
    for rep in range(2):
        S.profile_enable(True)
        e, g = S.value_and_grad(psi, lam, c, params_tensor(params), terms)
        torch.cuda.synchronize()
        prof = {q["name"]: q for q in S.profile_read()}
        S.profile_enable(False)
        assert abs(e.item() - e_ref) < E_TOL[dtype], (rep, e.item(), e_ref)
        ok, worst = grad_close(g.cpu().numpy(), g_ref, G_REL[dtype])
        assert ok, worst
        # the passes that run: those before the ansatz's closing CNOT ladder
        # (a permutation the observable is conjugated through)
        n_passes = prof["tile_adj"]["launches"]
        assert prof["tile_fwd"]["launches"] == n_passes <= c.info()["passes"]
        k = n_passes if checkpoints is None else min(checkpoints, n_passes)
        assert prof["tile_adj"]["bytes"] == _adj_bytes_expected(n, dtype, n_passes, k)
        back = to_numpy(psi)
        if k == n_passes:
            assert back[0] == 1 and np.count_nonzero(back) == 1  # untouched
        else:
            e0 = np.zeros(1 << n, dtype=complex)
            e0[0] = 1
            np.testing.assert_allclose(back, e0, atol=AMP_TOL[dtype] * 200, rtol=0)


@pytest.mark.parametrize("kw", [dict(max_blocks=5), dict(buffers=4, jit=2), dict(buffers=3, jit=2, max_blocks=7),
                                dict(buffers=1, jit=1)])
def test_value_and_grad_checkpoints_ring(kw):
    """21 qubits: the generic ring kernels with the TMA warpgroup (default
    below 22 qubits), the pass-specialised ones with and without it (their
    reverse kernels for passes that read psi from a checkpoint store lambda
    only in the last stage) and the one-buffer generic kernel: checkpoints for
    the last 5 passes against none, energy against the oracle."""
    S = sim()
    n = 21
    circ = W.hea_ansatz(n, 2)
    params = W.config_rng(7).angles(circ.n_params)
    terms = W.ising(n)
    e_ref = oracle.energy(circ, params, terms)
    out = {}
    for ck in (0, 5):
        c = S.Circuit(circ, mode="fused", checkpoints=ck, **kw)
        psi = S.State(n, torch.complex64).reset(0)
        lam = S.State(n, torch.complex64)
        e, g = S.value_and_grad(psi, lam, c, params_tensor(params), terms)
        torch.cuda.synchronize()
        # complex64 rounding over ~100 gates: a few 1e-7 of the observable's norm
        assert abs(e.item() - e_ref) < 2e-6 * W.observable_l1(terms), (ck, e.item(), e_ref)
        assert abs(to_numpy(psi)[0] - 1) < 1e-4
        out[ck] = (g.cpu().numpy(), to_numpy(lam))
    scale = np.abs(out[0][0]).max()
    np.testing.assert_allclose(out[5][0], out[0][0], atol=1e-4 * scale, rtol=0)
    np.testing.assert_allclose(out[5][1], out[0][1], atol=1e-5 * W.observable_l1(terms), rtol=0)


def prefix_then_hea(n, rounds, layers, seed):
    """An angle-free state preparation (rounds of H on every qubit, a CNOT
    ring and a fixed controlled phase) that fills whole fused passes, then
    the ansatz with the Ising observable."""
    gates = []
    for r in range(rounds):
        gates += [W.Gate("H", (q,)) for q in range(n)]
        gates += [W.Gate("CNOT", (q, (q + 1) % n)) for q in range(n)]
        gates.append(W.Gate("CPHASE", (0, n - 1), angle=0.3 + r))
    h = W.hea_ansatz(n, layers)
    circ = W.Circuit(n, gates + list(h.gates), h.n_params)
    return W.Workload(f"prefix+hea n={n}", circ, W.config_rng(seed).angles(h.n_params), W.ising(n))


@pytest.mark.parametrize("checkpoints", [None, 0, 1, 2])
@pytest.mark.parametrize("dtype", ["c64", "c128"])
def test_value_and_grad_angle_free_prefix(checkpoints, dtype):
    """A prefix without angles (it fills the first fused pass), then the
    ansatz: the reverse sweep of tqd_value_and_grad ends at the first pass
    with an angle (Sec. 4.4: the gradient needs lambda and psi only where an
    angle acts).  psi comes back as the input state: untouched when every
    pass is checkpointed, else from a copy kept in a checkpoint slot
    (checkpoints 1: every pass in place; 2: one checkpoint and the copy);
    checkpoints 0 (none) keeps the whole sweep.  E and the gradient against
    the oracle, psi restored, and the number of reverse passes."""
    S = sim()
    n = 14
    w = prefix_then_hea(n, 2, 2, 31)
    e_ref, g_ref = oracle.grad_stored(w.circuit, w.params, w.terms)
    c = S.Circuit(w.circuit, checkpoints=checkpoints)
    full = S.Circuit(w.circuit, checkpoints=0)
    psi = S.State(n, DTYPES[dtype]).reset(0)
    lam = S.State(n, DTYPES[dtype])
    S.profile_enable(True)
    e_full, g_full = S.value_and_grad(psi, lam, full, params_tensor(w.params), w.terms)
    torch.cuda.synchronize()
    adj_full = {q["name"]: q for q in S.profile_read()}.get("tile_adj", {}).get("launches", 0)
    psi.reset(0)
    e, g = S.value_and_grad(psi, lam, c, params_tensor(w.params), w.terms)
    torch.cuda.synchronize()
    adj = {q["name"]: q for q in S.profile_read()}.get("tile_adj", {}).get("launches", 0)
    S.profile_enable(False)
    assert adj_full >= 1
    if checkpoints == 0:
        assert adj == adj_full
    else:
        assert 1 <= adj < adj_full, (adj, adj_full)  # the QFT's passes are not un-applied
    assert abs(e.item() - e_ref) <= E_TOL[dtype]
    ok, worst = grad_close(g.cpu().numpy(), g_ref, G_REL[dtype])
    assert ok, worst
    # the same passes take the derivatives either way (psi from a checkpoint
    # or recomputed in place: rounding only)
    ok, worst = grad_close(g.cpu().numpy(), g_full.cpu().numpy(), G_REL[dtype])
    assert ok, worst
    e0 = np.zeros(2 ** n, dtype=np.complex128)
    e0[0] = 1
    back = np.max(np.abs(to_numpy(psi) - e0))
    assert back <= (1e-12 if dtype == "c128" else AMP_TOL["c64"] * math.sqrt(2 * len(w.circuit.gates) / 100 + 1)), back


def test_value_and_grad_checkpoints_tensor_core():
    """Forward passes on the tensor cores write their checkpoint through a copy
    of the previous state (the kernel works in place)."""
    S = sim()
    n = 14
    circ, params = tc_circuit(8100, n, 2)
    terms = W.ising(n) + W.random_pauli_terms(W.SplitMix64(5), n, 3)
    e_ref, g_ref = oracle.grad_stored(circ, params, terms)
    c = S.Circuit(circ, mode="tc")
    psi = S.State(n, torch.complex64).reset(0)
    lam = S.State(n, torch.complex64)
    S.profile_enable(True)
    e, g = S.value_and_grad(psi, lam, c, params_tensor(params), terms)
    torch.cuda.synchronize()
    prof = {q["name"]: q for q in S.profile_read()}
    S.profile_enable(False)
    assert prof.get("tc_block", {}).get("launches", 0) >= 1
    assert abs(e.item() - e_ref) < 1e-5
    ok, worst = grad_close(g.cpu().numpy(), g_ref, 1e-4)
    assert ok, worst
    back = to_numpy(psi)
    assert back[0] == 1 and np.count_nonzero(back) == 1


def tc_fixed_circuit(seed, n, blocks):
    """As tc_circuit, but every block is 40 fixed gates (no angle) on qubits
    0..5: the reverse sweep then un-applies each block on the tensor cores
    (tqd_value_and_grad's sweep ends at the first pass with an angle, so it
    does not reach the first block)."""
    rng = W.SplitMix64(seed)
    gates, n_params = [], 0
    for _ in range(blocks):
        c6, _ = W.random_circuit(rng, 6, 40, n_params=1, fixed_fraction=1.0)
        gates.extend(c6.gates)
        for q in range(6, n):
            gates.append(W.Gate("RY", (q,), param=n_params))
            n_params += 1
        gates.append(W.Gate("CNOT", (5, 6)))
        gates.append(W.Gate("CNOT", (n - 1, 0)))
    return W.Circuit(n, gates, n_params), rng.angles(n_params)


@pytest.mark.parametrize("checkpoints", [None, 0])
def test_reverse_sweep_tensor_core_fixed_blocks(checkpoints):
    """Blocks of fixed gates have no angle derivative, so the reverse sweep
    un-applies them as x = U^dagger y (Sec. 4.4) with one tensor-core product
    per state: lambda only when psi comes from a forward checkpoint, psi and
    lambda when psi is recomputed in place.  E and the gradient against the
    oracle's parameter shift, psi restored, and the launch count of the
    tensor-core kernel."""
    S = sim()
    n, blocks = 14, 3
    circ, params = tc_fixed_circuit(8200, n, blocks)
    terms = W.ising(n) + W.random_pauli_terms(W.SplitMix64(9), n, 4)
    e_ref, g_ref = oracle.grad_stored(circ, params, terms)
    c = S.Circuit(circ, mode="tc", checkpoints=checkpoints)

    def tc_launches(run):
        S.profile_enable(True)
        out = run()
        torch.cuda.synchronize()
        prof = {q["name"]: q for q in S.profile_read()}
        S.profile_enable(False)
        return out, prof.get("tc_block", {}).get("launches", 0)

    psi = S.State(n, torch.complex64).reset(0)
    _, n_blocks = tc_launches(lambda: S.apply(psi, c, params_tensor(params)))
    assert n_blocks >= 1
    psi.reset(0)
    lam = S.State(n, torch.complex64)
    (e, g), launches = tc_launches(lambda: S.value_and_grad(psi, lam, c, params_tensor(params), terms))
    # forward: one launch per block; reverse: every block but the first (the
    # circuit opens with it: no angle before it, so the sweep ends there) on
    # lambda when psi comes from checkpoints; without checkpoints the whole
    # sweep runs, on psi and lambda
    want = 2 * n_blocks - 1 if checkpoints is None else 3 * n_blocks
    assert launches == want, (launches, n_blocks)
    assert abs(e.item() - e_ref) < 1e-5
    ok, worst = grad_close(g.cpu().numpy(), g_ref, 1e-4)
    assert ok, worst
    # psi back at e_0: the amplitude bar of the tensor-core forward test for
    # the 2 x ng gates of the round trip, twice (the reverse sweep's rounding
    # adds to the forward's rather than cancelling it)
    bar = 2 * AMP_TOL["c64"] * math.sqrt(2 * len(circ.gates) / 100 + 1)
    e0 = np.zeros(2 ** n, dtype=np.complex128)
    e0[0] = 1
    err = float(np.max(np.abs(to_numpy(psi) - e0)))
    # tqd_backward over the same plan: psi_L in, psi_0 back, the same gradient
    st, c2, p = gpu_state(circ, params, "tc", "c64")
    lam2 = S.State(n, torch.complex64)
    g2 = torch.zeros(circ.n_params, dtype=torch.float64, device="cuda")
    _, back_launches = tc_launches(lambda: S.backward(st, lam2, c2, p, terms, g2))
    assert back_launches == 2 * n_blocks  # tqd_backward un-applies every block, on psi and lambda
    ok, worst = grad_close(g2.cpu().numpy(), g_ref, 1e-4)
    assert ok, worst
    err2 = float(np.max(np.abs(to_numpy(st) - e0)))
    print(f"\ntensor-core reverse, {n_blocks} blocks: psi restored to {err:.2e} (value_and_grad), "
          f"{err2:.2e} (backward); bar {bar:.2e}")
    assert err <= bar and err2 <= bar, (err, err2, bar)


@pytest.mark.parametrize("nq,dtype", [(6, "c128"), (12, "c64")])
def test_main_example_ladder_encoder_batch(nq, dtype):
    """The appendix's main example: a batch of 16 inputs x[b, i] fed to RY
    encoders, three CNOT-ladder + RY layers, out = measure_allZ per sample,
    loss = sum |out|, gradient with respect to the inputs; against the
    oracle (per-term values; parameter shift with the terms weighted by
    sign(out)), then three Adam steps that lower the loss."""
    S = sim()
    batch, layers = 16, 3
    circ = W.ladder_ansatz(nq, layers)
    rng = np.random.default_rng(nq)
    weights = rng.random(circ.n_params - nq) * np.pi
    x = torch.nn.Parameter(torch.tensor(rng.random((batch, nq)) * np.pi / 3, device="cuda"))
    c = S.Circuit(circ)
    w_dev = torch.tensor(weights, device="cuda")
    tol_e = 1e-10 if dtype == "c128" else 2e-5

    def forward(xv):
        outs = [S.measure_allz_fn(torch.cat([xv[b], w_dev]), c, dtype=DTYPES[dtype]) for b in range(batch)]
        return torch.stack(outs)

    out = forward(x)
    loss = out.abs().sum()
    loss.backward()
    g = x.grad.detach().cpu().numpy()
    xs = x.detach().cpu().numpy()
    for b in (0, 7, 15):
        params = np.concatenate([xs[b], weights])
        _, ref = oracle.expval(nq, oracle.run(circ, params), W.all_z_terms(nq))
        np.testing.assert_allclose(out[b].detach().cpu().numpy(), ref, atol=tol_e)
        terms = [W.PauliTerm(float(np.sign(r)), t.ops) for t, r in zip(W.all_z_terms(nq), ref)]
        gref = oracle.grad_param_shift(circ, params, terms)[:nq]
        np.testing.assert_allclose(g[b], gref, atol=1e-9 if dtype == "c128" else 1e-4)
    opt = torch.optim.Adam([x], lr=0.05)
    losses = [loss.item()]
    for _ in range(3):
        opt.zero_grad()
        l2 = forward(x).abs().sum()
        l2.backward()
        opt.step()
        losses.append(l2.item())
    assert losses[-1] < losses[0]


_CACHE_SCRIPT = r"""
import sys, torch
sys.path.insert(0, {root!r})
from paper_2511_19291_gb300 import sim as S, workloads as W
n = 22
circ = W.hea_ansatz(n, 2)
params = torch.tensor(W.config_rng(9).angles(circ.n_params), dtype=torch.float64, device="cuda")
c = S.Circuit(circ)
psi, lam = S.State(n).reset(0), S.State(n)
e, g = S.value_and_grad(psi, lam, c, params, W.ising(n))
torch.cuda.synchronize()
print(repr(e.item()), repr(float(g.abs().sum().item())))
"""


def test_jit_disk_cache(tmp_path):
    """Pass-specialised kernels persist across processes: a first process
    fills an empty cache directory, a second one loads them (nothing is
    rewritten; the same energy bit for bit), and a third, after every entry
    was truncated, compiles them again and still agrees."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, TQD_JIT_CACHE_DIR=str(tmp_path / "jit"))
    script = _CACHE_SCRIPT.format(root=root)

    def run():
        r = subprocess.run([sys.executable, "-c", script], env=env, capture_output=True, text=True, timeout=900)
        assert r.returncode == 0, r.stderr[-2000:]
        return r.stdout.strip().splitlines()[-1]

    def same(a, b):
        # the energy's reduction is deterministic; the gradient partials are
        # summed with shared-memory atomics, whose order varies run to run
        (ea, ga), (eb, gb) = (map(float, x.split()) for x in (a, b))
        return ea == eb and abs(ga - gb) <= 1e-9 * abs(ga)

    first = run()
    entries = sorted((tmp_path / "jit").glob("*.cubin"))
    assert entries, "no cache entries written"
    stamps = {p: p.stat().st_mtime_ns for p in entries}
    assert same(run(), first)
    assert all(p.stat().st_mtime_ns == stamps[p] for p in entries)  # read, not rewritten
    for p in entries:
        p.write_bytes(p.read_bytes()[:20])
    assert same(run(), first)
    assert all(p.stat().st_size > 20 for p in entries)  # rewritten whole
