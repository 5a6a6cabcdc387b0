"""Writes the stored oracle values of the full-size workloads.

Every number written here comes from the complex128 CPU oracle (``oracle/``)
run on the seeded inputs of ``paper_2511_19291_gb300.workloads``; nothing is
taken from the CUDA library.  The GPU tests compare the library's complex64
results with these files.

Files (all under ``tests/golden/``):

* ``hea26x20_ising.json`` -- the 26-qubit, 20-layer ansatz (1040 angles,
  seed index 2) with the open-chain Ising observable: E, and the
  parameter-shift derivative dE/dtheta_k = (E(theta_k + pi/2) -
  E(theta_k - pi/2)) / 2 (exact for R_P(t) = exp(-i t P / 2)) for a fixed
  sample of angles (first, middle and last RY and RZ).
* ``hea24x10_ising.json`` -- the 24-qubit, 10-layer workload (480 angles,
  seed index 3): E and the same kind of sample.
* ``hea20x10_ising_grad.json`` -- the same family at 20 qubits, 10 layers
  (400 angles, seed index 3): E and the whole parameter-shift gradient.
* ``hea12x4_sumz_grad.json`` -- the small workload: 12 qubits, 4 layers (96
  angles, seed index 1) with the observable sum_i Z_i: E and the whole
  parameter-shift gradient.

Each evaluation is one gate-by-gate oracle run (Sec. 4.1, Algorithm 1)
followed by the oracle's expectation value (Sec. 2.2.1); the derivatives use
the parameter-shift rule, which does not touch any adjoint code.

Usage: ``python tests/golden/make_golden.py [--procs P] [--only NAME]``.
The 26-qubit file takes about 17 oracle evaluations of roughly 7 minutes
each on one core; they run as P independent processes (default: the host's
cores, capped by free memory at about 2.5 GB per 26-qubit process).
"""
from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def sample_indices(n: int, layers: int) -> list:
    """First, middle and last RY and RZ angles, plus the last qubit of the
    first layer and the first qubit of the last layer (8 angles)."""
    per = 2 * n
    mid = layers // 2
    q_mid = n // 2
    idx = [0, 1,                                   # layer 0, qubit 0: RY, RZ
           2 * (n - 1),                            # layer 0, last qubit: RY
           mid * per + 2 * q_mid, mid * per + 2 * q_mid + 1,
           (layers - 1) * per + 1,                 # last layer, qubit 0: RZ
           (layers - 1) * per + 2 * (n - 1), (layers - 1) * per + 2 * (n - 1) + 1]
    return idx


def _energy_job(args):
    """One oracle evaluation: E(params) for the named workload."""
    name, shift_index, shift = args
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    from paper_2511_19291_gb300 import workloads as W
    from oracle import oracle as O
    wl = _workload(W, name)
    p = wl.params.copy()
    if shift_index >= 0:
        p[shift_index] += shift
    t0 = time.time()
    e = O.energy(wl.circuit, p, wl.terms)
    return name, shift_index, shift, e, time.time() - t0


def _workload(W, name):
    if name == "hea26x20_ising":
        return W.workload_main()
    if name == "hea24x10_ising":
        return W.workload_grad()
    if name == "hea20x10_ising":
        return W.workload_hea(3, 20, 10, "ising")
    if name == "hea12x4_sumz":
        return W.workload_small()
    raise KeyError(name)


def _describe(W, name):
    wl = _workload(W, name)
    c = wl.circuit
    return {"workload": wl.name, "n_qubits": c.n_qubits, "gates": len(c.gates), "n_params": c.n_params,
            "observable": ("sum_i Z_i" if name.endswith("sumz")
                           else "open-chain Ising: sum_i Z_i Z_{i+1} + 0.5 sum_i X_i"),
            "terms": len(wl.terms)}


def sampled(name: str, n: int, layers: int, procs: int) -> dict:
    from paper_2511_19291_gb300 import workloads as W
    idx = sample_indices(n, layers)
    jobs = [(name, -1, 0.0)]
    for k in idx:
        jobs += [(name, k, 0.5 * math.pi), (name, k, -0.5 * math.pi)]
    ctx = mp.get_context("spawn")
    res = {}
    secs = []
    with ctx.Pool(processes=min(procs, len(jobs))) as pool:
        for nm, k, s, e, dt in pool.imap_unordered(_energy_job, jobs):
            res[(k, s)] = e
            secs.append(dt)
            print(f"  {nm} shift[{k}] {s:+.4f}: E = {e:.15g} ({dt:.0f} s)", flush=True)
    grads = {str(k): 0.5 * (res[(k, 0.5 * math.pi)] - res[(k, -0.5 * math.pi)]) for k in idx}
    out = _describe(W, name)
    out.update({
        "energy": res[(-1, 0.0)],
        "grad_indices": idx,
        "grad": [grads[str(k)] for k in idx],
        "method": "oracle complex128: E by gate-by-gate run + expectation; dE/dtheta_k by parameter shift "
                  "(E(theta_k + pi/2) - E(theta_k - pi/2)) / 2",
        "oracle_seconds_per_evaluation": round(sum(secs) / len(secs), 1),
    })
    return out


def full_gradient(name: str) -> dict:
    from paper_2511_19291_gb300 import workloads as W
    from oracle import oracle as O
    wl = _workload(W, name)
    t0 = time.time()
    e = O.energy(wl.circuit, wl.params, wl.terms)
    g = O.grad_param_shift(wl.circuit, wl.params, wl.terms)
    out = _describe(W, name)
    out.update({
        "energy": e,
        "grad": [float(x) for x in g],
        "method": "oracle complex128: E by gate-by-gate run + expectation; every dE/dtheta_k by parameter shift",
        "oracle_seconds": round(time.time() - t0, 1),
    })
    return out


def write(name: str, data: dict) -> None:
    path = os.path.join(HERE, name + ".json")
    with open(path, "w") as f:
        json.dump(data, f, indent=1)
        f.write("\n")
    print("wrote", path, flush=True)


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--procs", type=int, default=0)
    ap.add_argument("--only", default="")
    a = ap.parse_args()
    from oracle import oracle as O
    O.build()
    cores = len(os.sched_getaffinity(0))
    procs = a.procs or cores
    try:
        avail_gb = os.sysconf("SC_AVPHYS_PAGES") * os.sysconf("SC_PAGE_SIZE") / 2**30
        procs = max(1, min(procs, int(avail_gb // 2.5)))
    except (ValueError, OSError):
        pass
    todo = [a.only] if a.only else ["hea12x4_sumz", "hea20x10_ising", "hea24x10_ising", "hea26x20_ising"]
    for name in todo:
        t0 = time.time()
        print(f"{name}: {procs} processes", flush=True)
        if name in ("hea20x10_ising", "hea12x4_sumz"):
            data = full_gradient(name)
        elif name == "hea24x10_ising":
            data = sampled(name, 24, 10, procs)
        else:
            data = sampled(name, 26, 20, procs)
        data["script"] = "python tests/golden/make_golden.py --only " + name
        write(name + ("_grad" if name in ("hea20x10_ising", "hea12x4_sumz") else ""), data)
        print(f"{name}: {time.time() - t0:.0f} s", flush=True)


if __name__ == "__main__":
    main()
