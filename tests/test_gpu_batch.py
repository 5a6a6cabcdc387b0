"""Batched ragged circuits (one CUDA-graph launch): energies and gradients of
every circuit against the CPU oracle, for the small-circuit kernel, the wider
circuits' fused passes, the gate-by-gate baseline and an autotuned batch."""
import numpy as np
import pytest
import torch

import oracle
from paper_2511_19291_gb300 import workloads as W
from gpu_helpers import grad_close, sim

pytestmark = pytest.mark.gpu


def ragged(seed, count, wmin, wmax, dmin, dmax):
    rng = W.SplitMix64(seed)
    out = []
    for _ in range(count):
        w = rng.randint(wmin, wmax)
        d = rng.randint(dmin, dmax)
        circ = W.hea_ansatz(w, d)
        out.append((circ, rng.angles(circ.n_params), W.sum_z(w) if rng.uniform01() < 0.5 else W.ising(w)))
    return out


def reference(circ, params, terms):
    """The oracle's stored-activation gradient up to 14 qubits; wider circuits
    use the single-circuit complex128 path (itself checked against the oracle)."""
    if circ.n_qubits <= 14:
        return oracle.grad_stored(circ, params, terms)
    S = sim()
    c = S.Circuit(circ)
    p = torch.tensor(params, dtype=torch.float64, device="cuda").requires_grad_(True)
    e = S.expval_fn(p, c, terms, dtype=torch.complex128)
    e.backward()
    return e.item(), p.grad.cpu().numpy()


def check_batch(items, batch):
    batch.set_params([p for _, p, _ in items])
    batch.run()
    batch.run()  # a replay of the captured graph gives the same numbers
    torch.cuda.synchronize()
    energies = batch.energies.cpu().numpy()
    for c, (circ, params, terms) in enumerate(items):
        e_ref, g_ref = reference(circ, params, terms)
        assert abs(energies[c] - e_ref) < 1e-5, (c, circ.n_qubits, energies[c], e_ref)
        g = batch.grads_of(c).cpu().numpy()
        ok, worst = grad_close(g, g_ref, 1e-4)
        assert ok, (c, circ.n_qubits, len(circ.gates), worst, float(np.max(np.abs(g - g_ref))),
                    float(np.max(np.abs(g_ref))))


@pytest.mark.parametrize("small_max", [0, 11])
def test_batch_mixed_widths(small_max):
    S = sim()
    items = ragged(91 + small_max, 20, 4, 15, 1, 3)
    circs = [S.Circuit(c) for c, _, _ in items]
    b = S.Batch(circs, [t for _, _, t in items], small_max_qubits=small_max, streams=4)
    info = b.info()
    assert info["small"] + info["large"] == len(items)
    # every wider circuit runs on the persistent work-queue kernel
    wide = sorted({c.n_qubits for c, _, _ in items if c.n_qubits > info["small_max_qubits"]})
    assert sorted(info["tiling"]) == wide, info
    for w, t in info["tiling"].items():
        tiles = 1 << (w - 12)
        assert 1 <= t["tiles_per_item"] <= tiles and t["items_per_stage"] * t["tiles_per_item"] >= tiles
    check_batch(items, b)


def test_batch_wide_fallback_to_streams():
    """A wider circuit without a fused plan (here a gate-by-gate one) sends
    the batch's wider circuits back to their per-pass launches on streams:
    same results, no persistent-kernel tiling."""
    S = sim()
    items = ragged(92, 8, 12, 15, 1, 2)  # widths 14, 12, 14, 13, 15, 13, 15, 14
    circs = [S.Circuit(c, mode="plain" if k == 0 else "fused") for k, (c, _, _) in enumerate(items)]
    b = S.Batch(circs, [t for _, _, t in items], small_max_qubits=11, streams=4)
    assert b.info()["tiling"] == {}
    check_batch(items, b)


def test_batch_gate_by_gate_baseline():
    S = sim()
    items = ragged(93, 8, 4, 13, 1, 2)
    circs = [S.Circuit(c, mode="plain") for c, _, _ in items]
    b = S.Batch(circs, [t for _, _, t in items], plain=True)
    assert b.info()["small"] == 0
    check_batch(items, b)


def test_batch_autotune():
    S = sim()
    items = ragged(95, 12, 10, 14, 1, 2)
    circs = [S.Circuit(c) for c, _, _ in items]
    b = S.Batch(circs, [t for _, _, t in items], autotune=True, streams=4)
    info = b.info()
    assert info["small_threads"] in (128, 256, 512) and info["small_max_qubits"] in (11, 12, 13)
    for w, t in info["tiling"].items():
        assert t["tiles_per_item"] in (1, 2, 4)  # 2^(w - 12) tiles for w <= 14
    check_batch(items, b)


def test_batched_workload_sample():
    """The 512-circuit workload's generator (widths 10..20, depths 2..12): the
    first circuits, checked against the oracle."""
    S = sim()
    wl = W.batched_workload(count=6)
    items = [(w.circuit, w.params, w.terms) for w in wl]
    circs = [S.Circuit(c) for c, _, _ in items]
    b = S.Batch(circs, [t for _, _, t in items], streams=4)
    check_batch(items, b)


def test_batch_sharded_across_ranks():
    """The batched workload's split across ranks (bench.py --gpus N): each of
    3 ranks' shares, run here one after the other as its own batch, gives
    every circuit the energy and gradient of the whole batch and of the
    oracle; the shares cover the batch once."""
    from paper_2511_19291_gb300 import shard as SH
    S = sim()
    items = ragged(97, 15, 4, 14, 1, 3)
    costs = [SH.circuit_cost(c.n_qubits, len(c.gates)) for c, _, _ in items]
    parts = SH.partition(costs, 3)
    assert sorted(i for p in parts for i in p) == list(range(len(items)))
    whole = S.Batch([S.Circuit(c) for c, _, _ in items], [t for _, _, t in items], streams=4)
    check_batch(items, whole)
    e_whole = whole.energies.cpu().numpy()
    for part in parts:
        sub = [items[i] for i in part]
        b = S.Batch([S.Circuit(c) for c, _, _ in sub], [t for _, _, t in sub], streams=4)
        check_batch(sub, b)
        e = b.energies.cpu().numpy()
        for k, i in enumerate(part):
            assert abs(e[k] - e_whole[i]) < 1e-6, (i, e[k], e_whole[i])
            np.testing.assert_allclose(b.grads_of(k).cpu().numpy(), whole.grads_of(i).cpu().numpy(),
                                       atol=1e-6 * W.observable_l1(items[i][2]), rtol=0)
