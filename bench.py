#!/usr/bin/env python
"""Benchmark of the differentiable state-vector hot path on GB300.

One step = one gradient evaluation of the 26-qubit, 20-layer hardware-efficient
ansatz (1040 angles, complex64 amplitudes) with the open-chain Ising
observable, through tqd_value_and_grad: reset |0...0>, apply the circuit,
lambda = H psi with E = Re <psi|lambda> read off its last pass, reverse sweep
with the angle derivatives.  Inputs (angles) are resident in HBM during
the timed region; the 512 MiB state is larger than L2, so no flush is needed.

The JSON line reports grad-evals/s of the fused plan (value), the
gate-by-gate plan measured on the same workload (plain), the dominant
kernel's achieved HBM bandwidth against the measured peak (roofline), the
same metric end to end with host buffers (e2e), and the CPU oracle timed on
a bounded sample of the workload (cpu_baseline).

Multi-GPU: the single-state path does not shard (replicas only): every rank
runs its own replica; value = steps of all ranks / max time over ranks.  The
batched measurement shards its circuits over the ranks (no collective on the
data path) and reports all circuits / the slowest rank's time.

``--impl reference`` times the CPU oracle on the same workload (bounded
samples extrapolated to grad-evals/s); under torchrun only rank 0 runs it.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "HBM GB/s vs peak per gate sweep; grad-evals/sec fused vs plain at ≤1e-5 error"
UNIT = "grad-evals/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--plan", choices=["fused", "plain"], default="fused")
    ap.add_argument("--plain-steps", type=int, default=2, help="steps of the gate-by-gate comparison (0 = skip)")
    ap.add_argument("--n", type=int, default=26)
    ap.add_argument("--layers", type=int, default=20)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--tile-qubits", type=int, default=0)
    ap.add_argument("--low-qubits", type=int, default=0)
    ap.add_argument("--buffers", type=int, default=0, choices=[0, 1, 2],
                    help="tile buffers per block in the fused passes (0 = library default)")
    ap.add_argument("--jit", type=int, default=0, choices=[0, 1, 2],
                    help="fused passes: 1 generic kernel, 2 pass-specialised kernels, 0 library default")
    ap.add_argument("--sweep-n", type=int, default=30, help="qubits of the plain gate-sweep measurement (0 = skip)")
    ap.add_argument("--batch-count", type=int, default=512, help="circuits of the batched measurement (0 = skip)")
    ap.add_argument("--tc-gates", type=int, default=200, help="gates of the tensor-core block measurement (0 = skip)")
    ap.add_argument("--qft-n", type=int, default=32, help="qubits of the QFT + ansatz measurement (0 = skip)")
    ap.add_argument("--small", type=int, default=1, choices=(0, 1),
                    help="time the 12-qubit, 4-layer workload's forward and gradient evaluations (0 = skip)")
    ap.add_argument("--forward-expval", type=int, default=1, choices=[0, 1],
                    help="time the workload's forward evaluation with E = <H> alone, fused and gate by gate (0 = skip)")
    ap.add_argument("--grad-fn", type=int, default=1, choices=[0, 1],
                    help="time the 24-qubit workload's gradient through the autograd.Function (0 = skip)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload(args):
    from paper_2511_19291_gb300 import workloads as W
    if args.n == 26 and args.layers == 20:
        return W.workload_main()
    return W.workload_hea(2, args.n, args.layers, "ising")


def config_of(args, w, plan, amplitudes="complex64"):
    reductions = ("fp64 (the oracle's own sums)" if amplitudes == "complex128" else
                  "gradients: fp32 inside one tile (a thread's 16 amplitudes, then the warp's 32 shares), fp64 "
                  "across tiles and blocks; expectations: fp32 per-thread partials, fp64 across threads and blocks")
    return {
        "workload": f"hea ansatz n={args.n} layers={args.layers} ({w.circuit.n_params} angles), "
                    f"open-chain Ising H ({len(w.terms)} terms), forward + expval + adjoint gradient",
        "n_qubits": args.n, "layers": args.layers, "n_params": w.circuit.n_params,
        "gates": len(w.circuit.gates), "plan": plan, "tile_buffers": args.buffers or "default",
        "pass_kernels": {0: "default", 1: "generic", 2: "specialised"}[args.jit],
        "amplitudes": amplitudes,
        "reductions": reductions,
        "l2": "inputs larger than L2 (state 2^n x 8 B; no flush needed)",
        "parallelism": "replicas",
    }


# --------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index, period_ms=100, lead_s=0.3):
        self.index = index
        self.period_ms = period_ms
        self.lead_s = lead_s
        self.proc = None
        self.stamped = []  # (host time of arrival, line)

    def _read(self):
        for line in self.proc.stdout:
            if line.strip():
                self.stamped.append((time.monotonic(), line))

    def __enter__(self):
        import threading
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", str(self.period_ms)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.reader = threading.Thread(target=self._read, daemon=True)
            self.reader.start()
            time.sleep(self.lead_s)  # nvidia-smi is up and sampling before the timed region starts
        except Exception:
            self.proc = None
        self.t0 = time.monotonic()
        return self

    def __exit__(self, *a):
        self.t1 = time.monotonic()
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.reader.join(timeout=5)
            # the samples that arrived while the timed work ran
            self.lines = [l for t, l in self.stamped if self.t0 <= t <= self.t1 + self.period_ms / 1000.0]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def stored_traffic(kernel):
    """DRAM bytes per launch from a committed ncu summary, valid only while the
    library source is unchanged since the capture."""
    try:
        import hashlib
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            t = json.load(f)
        h = hashlib.sha256()
        for rel in t.get("source_files", []):
            with open(os.path.join(ROOT, rel), "rb") as g:
                h.update(g.read())
        if t.get("source_digest") != h.hexdigest():
            return None
        return t.get("kernels", {}).get(kernel)
    except Exception:
        return None


# ------------------------------------------------------------ CPU oracle
def oracle_sample(w, gate_sample=6, term_sample=2):
    """Times the oracle on a bounded sample of the workload and extrapolates to
    one parameter-shift gradient evaluation: (2P + 1) forward passes plus
    expectations.  Single-threaded calls."""
    import numpy as np
    import oracle
    n = w.circuit.n_qubits
    psi = np.zeros(1 << n, dtype=np.complex128)
    psi[0] = 1
    from paper_2511_19291_gb300 import workloads as W
    sub = W.Circuit(n, w.circuit.gates[:gate_sample], w.circuit.n_params)
    t0 = time.perf_counter()
    psi = oracle.apply_gates(sub, w.params, psi)
    t_gates = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.expval(n, psi, w.terms[:term_sample])
    t_terms = time.perf_counter() - t0
    per_gate = t_gates / gate_sample
    per_term = t_terms / term_sample
    t_eval = per_gate * len(w.circuit.gates) + per_term * len(w.terms)
    t_grad = (2 * w.circuit.n_params + 1) * t_eval
    sample = (f"{gate_sample} gates and {term_sample} terms of the {n}-qubit workload on 1 host thread "
              f"({per_gate:.3f} s/gate, {per_term:.3f} s/term), extrapolated to one parameter-shift gradient "
              f"= (2*{w.circuit.n_params}+1) x ({len(w.circuit.gates)} gates + {len(w.terms)} terms)")
    return 1.0 / t_grad, sample, t_gates + t_terms


def oracle_all_cores(n, layers, gate_sample=6, term_sample=2, procs=None, deadline_s=300.0):
    """The same oracle, unchanged, as one process per host core, each timing
    the bounded sample of the n-qubit, `layers`-layer workload at once (a
    parameter-shift gradient's 2P + 1 evaluations are independent, so a CPU
    run would spread them this way): the rate is the sum of the processes'
    extrapolated rates.  Plain subprocesses with a deadline: one that dies
    or overruns turns the measurement into an 'unavailable' note."""
    try:
        cores = len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        cores = os.cpu_count() or 1
    procs = procs or cores
    try:  # about 3 states per process (the state and numpy temporaries), in half the free memory
        avail = os.sysconf("SC_AVPHYS_PAGES") * os.sysconf("SC_PAGE_SIZE")
        procs = max(1, min(procs, int(avail / 2 // (3 * 16 << n))))
    except (ValueError, OSError, AttributeError):
        pass
    # each process builds its inputs, then waits for a line on stdin before
    # timing, so that the timed samples of all processes overlap
    code = ("import json, sys; sys.path.insert(0, {root!r}); import bench; "
            "from paper_2511_19291_gb300 import workloads as W; "
            "wl = W.workload_hea(2, {n}, {layers}, 'ising'); sys.stdin.readline(); "
            "v, _, t = bench.oracle_sample(wl, {g}, {t}); "
            "print(json.dumps([v, t]))").format(root=ROOT, n=n, layers=layers, g=gate_sample, t=term_sample)
    ps = [subprocess.Popen([sys.executable, "-c", code], stdin=subprocess.PIPE, stdout=subprocess.PIPE,
                           stderr=subprocess.DEVNULL, text=True) for _ in range(procs)]
    end = time.monotonic() + deadline_s
    values = []
    try:
        time.sleep(min(5.0, deadline_s / 10))  # imports and inputs ready
        for p in ps:
            try:
                p.stdin.write("go\n")
                p.stdin.flush()
            except (BrokenPipeError, OSError):
                pass
        for p in ps:
            out, _ = p.communicate(timeout=max(0.01, end - time.monotonic()))
            if p.returncode != 0:
                return {"unavailable": f"an oracle process exited with {p.returncode}"}
            values.append(json.loads(out.strip().splitlines()[-1])[0])
    except subprocess.TimeoutExpired:
        return {"unavailable": f"oracle processes ran past {deadline_s:g} s"}
    finally:
        for p in ps:
            if p.poll() is None:
                p.kill()
                p.wait()
    sample = (f"{gate_sample} gates and {term_sample} terms of the {n}-qubit workload in each of {procs} "
              f"concurrent single-threaded processes ({cores} host cores available; processes capped by free "
              f"memory), started together, each extrapolated to one parameter-shift gradient; rate = sum over "
              f"processes")
    return {"value": sum(values), "unit": UNIT, "cores": procs, "host_cores": cores, "kind": "oracle",
            "sample": sample}


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return 0
    w = workload(args)
    vals = []
    total = 0.0
    for i in range(args.warmup + args.steps):
        v, sample, spent = oracle_sample(w, gate_sample=2, term_sample=1)
        total += spent
        if i >= args.warmup:
            vals.append(v)
    value = statistics.median(vals)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 / value,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
        "data": "synthetic", "config": config_of(args, w, "oracle", amplitudes="complex128"),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# -------------------------------------------------- plain sweep measurement
def dram_bytes(kind, t, c, n, amp=8):
    """Bytes HBM must move for one gate sweep on an n-qubit state: reads in
    128-byte lines, writes in 32-byte sectors (ncu on GB300 at 28 qubits:
    CNOT with control bit <= 3 reads every line of the state although it needs
    half the amplitudes; writes follow 32-byte sectors).  RY and RZ read and
    write every amplitude; CNOT(c, t) reads and writes the amplitudes with
    bit c set."""
    A = (1 << n) * amp
    if kind in ("RY", "RZ"):
        return 2 * A
    lines = A if (1 << c) * amp < 128 else A // 2      # lines holding an amplitude with bit c set
    sectors = A if (1 << c) * amp < 32 else A // 2     # sectors written
    return lines + sectors


def sweep_bench(S, torch, dev, n, barrier, reps=5):
    """Achieved HBM bandwidth of single gate sweeps (gate-by-gate kernels) on
    an n-qubit complex64 state: RY (dense), RZ (diagonal) and CNOT at several
    targets.  `gbs` counts the algorithmic bytes (the library's accounting:
    the amplitudes the gate changes, read and written); `dram_gbs` counts the
    bytes HBM must move at its access granularity (dram_bytes), which the
    fractions of peak use."""
    from paper_2511_19291_gb300 import workloads as W
    st = S.State(n, torch.complex64, dev).reset(0)
    targets = sorted({0, 1, 4, n // 2, n - 2, n - 1})
    rows = []
    for kind in ("RY", "RZ", "CNOT"):
        for t in targets:
            if kind == "CNOT":
                g = W.Gate("CNOT", ((t + 1) % n, t))
            else:
                g = W.Gate(kind, (t,), angle=0.37)
            c = S.Circuit(W.Circuit(n, [g] * reps, 0), mode="plain", device=dev)
            S.apply(st, c)
            barrier()
            S.profile_enable(True)
            S.apply(st, c)
            torch.cuda.synchronize(dev)
            prof = {p["name"]: p for p in S.profile_read()}
            S.profile_enable(False)
            k = {"RY": "dense1", "RZ": "diag1", "CNOT": "perm2"}[kind]
            p = prof[k]
            sec = p["ms"] / 1000.0 / p["launches"]
            db = dram_bytes(kind, t, (t + 1) % n, n)
            rows.append({"gate": kind, "target": t, "gbs": round(p["bytes"] / (p["ms"] / 1000.0) / 1e9, 1),
                         "dram_gbs": round(db / sec / 1e9, 1), "us": round(1e6 * sec, 1)})
    del st
    torch.cuda.empty_cache()
    peak, src = peaks()
    for r in rows:
        r["frac"] = round(r["gbs"] / peak, 3)
        r["frac_dram"] = round(r["dram_gbs"] / peak, 3)
    return {"n_qubits": n, "rows": rows,
            "min_frac": min(r["gbs"] for r in rows) / peak, "max_frac": max(r["gbs"] for r in rows) / peak,
            "min_frac_dram": min(r["dram_gbs"] for r in rows) / peak,
            "max_frac_dram": max(r["dram_gbs"] for r in rows) / peak,
            "frac_bytes": "frac: algorithmic bytes (the amplitudes the gate changes, read and written); "
                          "frac_dram: bytes HBM moves at its granularity (reads in 128-byte lines, writes in "
                          "32-byte sectors)",
            "peak": peak, "peak_source": f"{src} hbm_gbs"}


# ------------------------------------------------------- batched measurement
def batch_bench(S, torch, dev, count, barrier, reps=3, rank=0, world=1):
    """512 ragged circuits (widths 10..20, depths 2..12, sum_i Z_i): forward +
    adjoint gradient of every circuit per run.  Fused: one CUDA-graph launch
    (autotuned); plain: every gate its own launch, issued by the host.  With
    several ranks the circuits are sharded (greedy by 2^width x gates, no
    collective on the data path); the time is the slowest rank's and the rate
    counts all circuits (the total work is fixed: strong scaling)."""
    from paper_2511_19291_gb300 import shard as SH
    from paper_2511_19291_gb300 import workloads as W
    wl_all = W.batched_workload(count=count)
    mine = SH.shard(SH.workload_costs(wl_all), world, rank)
    wl = [wl_all[i] for i in mine]
    out = {"circuits": count, "widths": "10..20", "depths": "2..12", "observable": "sum_i Z_i",
           "ranks": world, "scaling": "strong" if world > 1 else None, "circuits_this_rank": len(wl)}

    def slowest(ms):
        if world > 1:
            t = torch.tensor([ms], dtype=torch.float64, device=dev)
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            ms = float(t.item())
        return ms

    for mode in ("fused", "plain"):
        k = reps if mode == "fused" else 1
        info = {}
        if wl:
            circs = [S.Circuit(w.circuit, mode=mode, device=dev) for w in wl]
            b = S.Batch(circs, [w.terms for w in wl], autotune=(mode == "fused"), plain=(mode == "plain"))
            b.set_params([w.params for w in wl])
            b.run()
        barrier()
        a = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(k if wl else 0):
            b.run()
        e.record()
        barrier()
        ms = slowest(a.elapsed_time(e) / k)
        out[mode] = {"grad_evals_per_s": count / (ms / 1000.0), "ms_per_batch": ms, "runs": k}
        if wl:
            if mode == "fused":
                out[mode].update(b.info())
            del b, circs
    out["fused_over_plain"] = out["fused"]["grad_evals_per_s"] / out["plain"]["grad_evals_per_s"]
    return out


# ------------------------------------------- gradient through autograd.Function
def grad_fn_bench(S, torch, dev, barrier, reps=10):
    """The 24-qubit, 10-layer ansatz with the Ising observable (480 angles),
    differentiated through the autograd.Function the way a training loop
    does: e = expval_fn(theta); e.backward().  grad-evals/s over `reps`
    evaluations after two warm-up ones."""
    from paper_2511_19291_gb300 import workloads as W
    w = W.workload_grad()
    c = S.Circuit(w.circuit, device=dev)
    obs = S.Observable(w.terms)
    p = torch.tensor(w.params, dtype=torch.float64, device=dev, requires_grad=True)

    def step():
        p.grad = None
        e = S.expval_fn(p, c, obs)
        e.backward()
        return e

    for _ in range(2):
        step()
    barrier()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        e = step()
    b.record()
    barrier()
    ms = a.elapsed_time(b) / reps
    return {"workload": w.name, "n_qubits": w.circuit.n_qubits, "n_params": w.circuit.n_params,
            "path": "expval_fn + backward (autograd.Function)", "grad_evals_per_s": 1000.0 / ms,
            "ms_per_grad_eval": ms, "energy": e.item()}


# ------------------------------------------------ tensor-core block measurement
def forward_expval_bench(S, torch, dev, w, barrier, reps=5):
    """Forward evaluation of the workload without a gradient (reset, the
    circuit, E = <H> by tqd_expval): time per evaluation for the fused plan
    and the gate-by-gate one, and the expectation kernels' own time and
    bandwidth (the bytes they read: psi once per 12-qubit set of x masks)."""
    n = w.circuit.n_qubits
    obs = S.Observable(w.terms)
    params = torch.tensor(w.params, dtype=torch.float64, device=dev)
    st = S.State(n, torch.complex64, dev)
    out = {"workload": w.name, "observable_terms": len(w.terms)}
    peak, src = peaks()
    for mode in ("fused", "plain"):
        c = S.Circuit(w.circuit, mode=mode, device=dev)
        k = reps if mode == "fused" else 1
        e = torch.zeros((), dtype=torch.float64, device=dev)

        def one():
            st.reset(0)
            S.apply(st, c, params)
            S.expval(st, obs, out=e)

        one()
        barrier()
        S.profile_enable(True)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(k):
            one()
        b.record()
        torch.cuda.synchronize(dev)
        prof = {p["name"]: p for p in S.profile_read()}
        S.profile_enable(False)
        r = {"ms_per_eval": a.elapsed_time(b) / k, "energy": float(e.item())}
        if mode == "fused" and "expval" in prof:
            p = prof["expval"]
            ms = p["ms"] / k
            r["expval"] = {"ms_per_eval": ms, "launches_per_eval": p["launches"] // k,
                           "gbs": p["bytes"] / (p["ms"] / 1000.0) / 1e9,
                           "frac": p["bytes"] / (p["ms"] / 1000.0) / 1e9 / peak, "peak_source": f"{src} hbm_gbs"}
        out[mode] = r
        del c
    out["fused_over_plain"] = out["plain"]["ms_per_eval"] / out["fused"]["ms_per_eval"]
    del st
    torch.cuda.empty_cache()
    return out


def small_bench(S, torch, dev, barrier, reps=200):
    """The small workload (12 qubits, 4 layers, 96 angles, sum_i Z_i: one
    2^12-amplitude tile, so launch- and latency-bound): time per forward
    evaluation (reset, circuit, tqd_expval) and per gradient evaluation
    (tqd_value_and_grad), each over `reps` back-to-back calls, and both results
    against the stored oracle values (tests/golden/hea12x4_sumz_grad.json)."""
    import numpy as np
    from paper_2511_19291_gb300 import workloads as W
    w = W.workload_small()
    n = w.circuit.n_qubits
    c = S.Circuit(w.circuit, device=dev)
    obs = S.Observable(w.terms)
    params = torch.tensor(w.params, dtype=torch.float64, device=dev)
    psi = S.State(n, torch.complex64, dev)
    lam = S.State(n, torch.complex64, dev)
    e = torch.zeros((), dtype=torch.float64, device=dev)
    eg = torch.zeros((), dtype=torch.float64, device=dev)
    g = torch.zeros(w.circuit.n_params, dtype=torch.float64, device=dev)

    def fwd():
        psi.reset(0)
        S.apply(psi, c, params)
        S.expval(psi, obs, out=e)

    def grad():
        psi.reset(0)
        S.value_and_grad(psi, lam, c, params, obs, eg, g)

    out = {"workload": w.name, "n_qubits": n, "layers": 4, "n_params": w.circuit.n_params,
           "observable": "sum_i Z_i", "reps": reps}
    for name, fn in (("forward", fwd), ("gradient", grad)):
        for _ in range(3):
            fn()
        barrier()
        S.profile_enable(True)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            fn()
        b.record()
        torch.cuda.synchronize(dev)
        launches = sum(p["launches"] for p in S.profile_read())
        S.profile_enable(False)
        out[name] = {"us_per_eval": a.elapsed_time(b) * 1000.0 / reps, "launches_per_eval": launches / reps}
        out[name]["api_calls"] = "through the Python binding, one library call after another (host-bound)"
    # the same calls captured once into a CUDA graph (the circuit's matrices are
    # built on the device from the angles, so the graph stays valid), replayed;
    # then with the pass-specialised kernels (compiled at run time; by default
    # they serve states of 22 qubits and more)
    cs = S.Circuit(w.circuit, device=dev, jit=2)

    def fwd_s():
        psi.reset(0)
        S.apply(psi, cs, params)
        S.expval(psi, obs, out=e)

    def grad_s():
        psi.reset(0)
        S.value_and_grad(psi, lam, cs, params, obs, eg, g)

    out["passes"] = c.info()["passes"]
    for name, fn, key in (("forward", fwd, "graph_us_per_eval"), ("gradient", grad, "graph_us_per_eval"),
                          ("forward", fwd_s, "graph_specialised_us_per_eval"),
                          ("gradient", grad_s, "graph_specialised_us_per_eval")):
        per = 50
        try:
            side = torch.cuda.Stream(dev)
            side.wait_stream(torch.cuda.current_stream(dev))
            with torch.cuda.stream(side):
                fn()
            torch.cuda.current_stream(dev).wait_stream(side)
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph):
                for _ in range(per):
                    fn()
            graph.replay()
            barrier()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            for _ in range(reps // per):
                graph.replay()
            b.record()
            torch.cuda.synchronize(dev)
            out[name][key] = a.elapsed_time(b) * 1000.0 / ((reps // per) * per)
            del graph
        except Exception as ex:  # a call that cannot be captured: report it
            out[name][key] = None
            out[name]["graph_error"] = str(ex)[:200]
    # the batch path with this one circuit: the whole circuit in one block's
    # shared memory, forward + E + gradient in one graph launch
    try:
        bt = S.Batch([c], [w.terms])
        bt.set_params([w.params])
        bt.run()
        barrier()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            bt.run()
        b.record()
        torch.cuda.synchronize(dev)
        out["batch_one_circuit"] = {"us_per_grad_eval": a.elapsed_time(b) * 1000.0 / reps,
                                    "energy": float(bt.energies[0].item()), **{k: v for k, v in bt.info().items()
                                                                              if k != "tiling"}}
        del bt
    except Exception as ex:
        out["batch_one_circuit"] = {"error": str(ex)[:200]}
    # one clean gradient evaluation (g accumulates) for the error statement
    g.zero_()
    grad()
    e_f, e_g, g_h = float(e.item()), float(eg.item()), g.cpu().numpy()
    path = os.path.join(ROOT, "tests", "golden", "hea12x4_sumz_grad.json")
    if os.path.exists(path):
        with open(path) as f:
            ref = json.load(f)
        g_ref = np.array(ref["grad"])
        out["error"] = {"reference": "complex128 oracle, tests/golden/hea12x4_sumz_grad.json (E and every "
                                     "dE/dtheta by parameter shift)",
                        "energy_forward_abs_err": abs(e_f - ref["energy"]),
                        "energy_grad_eval_abs_err": abs(e_g - ref["energy"]),
                        "grad_max_abs_err": float(np.max(np.abs(g_h - g_ref))),
                        "grad_norm_rel_err": float(np.max(np.abs(g_h - g_ref)) / np.max(np.abs(g_ref)))}
    del psi, lam, c, cs
    torch.cuda.empty_cache()
    return out


def tc_bench(S, torch, dev, n, n_gates, barrier, reps=5):
    """One run of `n_gates` gates on qubits 0..5 of an n-qubit complex64 state:
    the fused 64 x 64 block on the tensor cores against the same gates in one
    tile pass.  Achieved bandwidth counts one read and one write of the state."""
    from paper_2511_19291_gb300 import workloads as W
    rng = W.SplitMix64(2511)
    gates = []
    for i in range(n_gates):
        r = i % 3
        if r == 0:
            gates.append(W.Gate("RY", (i % 6,), angle=rng.angle()))
        elif r == 1:
            gates.append(W.Gate("RZ", ((i + 2) % 6,), angle=rng.angle()))
        else:
            gates.append(W.Gate("CNOT", (i % 6, (i + 1) % 6)))
    circ = W.Circuit(n, gates, 0)
    st = S.State(n, torch.complex64, dev).reset(0)
    out = {"n_qubits": n, "gates": n_gates}
    for mode, kern in (("tc", "tc_block"), ("fused", "tile_fwd")):
        c = S.Circuit(circ, mode=mode, device=dev)
        S.apply(st, c)
        barrier()
        S.profile_enable(True)
        for _ in range(reps):
            S.apply(st, c)
        torch.cuda.synchronize(dev)
        prof = {p["name"]: p for p in S.profile_read()}
        S.profile_enable(False)
        p = prof[kern]
        ms = p["ms"] / p["launches"]
        out[mode] = {"kernel": kern, "ms_per_pass": ms, "gbs": 2.0 * 8 * (1 << n) / (ms / 1000.0) / 1e9,
                     "passes_per_apply": p["launches"] // reps}
    peak, src = peaks()
    out["tc"]["frac_of_hbm"] = out["tc"]["gbs"] / peak
    out["tc_over_tile"] = out["fused"]["ms_per_pass"] * out["fused"]["passes_per_apply"] / \
        (out["tc"]["ms_per_pass"] * out["tc"]["passes_per_apply"])
    del st
    return out


# ------------------------------------------------ QFT + ansatz at 32 qubits
def qft_bench(S, torch, dev, n, barrier, layers=8, mode="fused"):
    """One gradient evaluation of the QFT followed by `layers` ansatz layers
    (Ising H) on an n-qubit complex64 state: psi and lambda (2 x 2^n x 8 B,
    64 GiB at 32 qubits) resident in HBM.  Reports the step time and the
    fused passes' achieved bandwidth (algorithmic bytes over CUDA-event time).
    mode "tc": the same workload planned with tensor-core blocks for runs of
    at least 16 gates on qubits 0..5 (forward, and the reverse sweep of such
    a block when its gates are fixed)."""
    from paper_2511_19291_gb300 import workloads as W
    w = W.workload_qft(n, layers)
    c = S.Circuit(w.circuit, mode=mode, device=dev)
    obs = S.Observable(w.terms)
    psi = S.State(n, torch.complex64, dev)
    lam = S.State(n, torch.complex64, dev)
    p = torch.tensor(w.params, dtype=torch.float64, device=dev)
    g = torch.zeros(w.circuit.n_params, dtype=torch.float64, device=dev)
    e = torch.zeros((), dtype=torch.float64, device=dev)

    def step():
        psi.reset(0)
        S.value_and_grad(psi, lam, c, p, obs, e, g)

    step()  # compiles the pass kernels
    barrier()
    S.profile_enable(True)
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record()
    step()
    b.record()
    barrier()
    ms = a.elapsed_time(b)
    prof = {q["name"]: q for q in S.profile_read()}
    S.profile_enable(False)
    peak, src = peaks()
    out = {"n_qubits": n, "layers": layers, "gates": len(w.circuit.gates), "n_params": w.circuit.n_params,
           "plan": mode, "passes": c.info()["passes"], "ms_per_grad_eval": ms, "energy": float(e.item()),
           "peak": peak, "peak_source": f"{src} hbm_gbs"}
    for k in ("tile_fwd", "tile_adj", "tc_block"):
        if k in prof and prof[k]["ms"] > 0:
            gbs = prof[k]["bytes"] / (prof[k]["ms"] / 1000.0) / 1e9
            out[k] = {"launches": prof[k]["launches"], "ms": prof[k]["ms"], "gbs": gbs, "frac": gbs / peak}
    del psi, lam
    torch.cuda.empty_cache()
    return out


# ----------------------------------------------------------- error statement
def error_statement(args, e_step, e_check, g_step):
    """The step's E against a separate tqd_expval of a fresh forward pass, and
    E and the gradient against the stored complex128 oracle values of this
    workload (tests/golden, written by tests/golden/make_golden.py from the
    oracle alone: E, and parameter-shift derivatives at a sample of angles)."""
    import numpy as np
    out = {"energy_step": e_step, "energy_expval": e_check, "energy_step_vs_expval": abs(e_step - e_check)}
    name = {(26, 20): "hea26x20_ising.json", (24, 10): "hea24x10_ising.json"}.get((args.n, args.layers))
    path = os.path.join(ROOT, "tests", "golden", name) if name else None
    if not path or not os.path.exists(path):
        out["oracle"] = None
        return out
    with open(path) as f:
        ref = json.load(f)
    idx = np.array(ref["grad_indices"])
    g_ref = np.array(ref["grad"])
    dg = np.abs(g_step[idx] - g_ref)
    big = np.abs(g_ref) >= 1e-2 * np.max(np.abs(g_ref))
    out["oracle"] = {
        "reference": f"complex128 oracle, tests/golden/{name}: E and dE/dtheta by parameter shift at "
                     f"{len(idx)} angles {idx.tolist()}",
        "energy": ref["energy"], "energy_abs_err": abs(e_step - ref["energy"]),
        "grad_max_abs_err": float(np.max(dg)),
        "grad_norm_rel_err": float(np.max(dg) / np.max(np.abs(g_ref))),
        "grad_max_rel_err": float(np.max(dg[big] / np.abs(g_ref[big]))),
        "tolerance": "1e-5 absolute on E; 1e-4 relative on the gradient (max|dg| / max|g|)",
    }
    return out


# ------------------------------------------------------------- our path
def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    from paper_2511_19291_gb300 import build as B
    if rank == 0 or world == 1:
        B.build()
    if world > 1:
        torch.distributed.barrier()
    from paper_2511_19291_gb300 import sim as S

    w = workload(args)
    n = w.circuit.n_qubits
    obs = S.Observable(w.terms)
    circ = S.Circuit(w.circuit, mode=args.plan, tile_qubits=args.tile_qubits, low_qubits=args.low_qubits,
                     device=dev, buffers=args.buffers, jit=args.jit)
    psi = S.State(n, torch.complex64, dev)
    lam = S.State(n, torch.complex64, dev)
    params = torch.tensor(w.params, dtype=torch.float64, device=dev)
    grads = torch.zeros(w.circuit.n_params, dtype=torch.float64, device=dev)
    e_out = torch.zeros((), dtype=torch.float64, device=dev)

    def step(c):
        # one gradient evaluation: psi <- U|0...0>, E = <H>, dE/dtheta (the
        # energy read off lambda = H psi, which the reverse sweep needs)
        psi.reset(0)
        S.value_and_grad(psi, lam, c, params, obs, e_out, grads)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    def timed(fn, k):
        barrier()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(k):
            fn()
        b.record()
        barrier()
        ms = a.elapsed_time(b)
        if world > 1:
            t = torch.tensor([ms], dtype=torch.float64, device=dev)
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            ms = float(t.item())
        return ms

    # warm-up, and one profiled step to count launches
    for _ in range(args.warmup):
        step(circ)
    S.profile_enable(True)
    step(circ)
    torch.cuda.synchronize(dev)
    prof1 = S.profile_read()
    launches_per_step = sum(p["launches"] for p in prof1)

    # main timed region (per-kernel events recorded on the launching stream)
    S.profile_enable(True)
    with ClockSampler(local) as clk:
        ms = timed(lambda: step(circ), args.steps)
    prof = S.profile_read()
    S.profile_enable(False)
    ms_per_step = ms / args.steps
    value = world * args.steps / (ms / 1000.0)

    # end to end: angles from pinned host memory in, E and gradient back out
    params_host = torch.tensor(w.params, dtype=torch.float64).pin_memory()
    e_host = torch.zeros((), dtype=torch.float64).pin_memory()
    g_host = torch.zeros(w.circuit.n_params, dtype=torch.float64).pin_memory()

    def step_e2e():
        params.copy_(params_host, non_blocking=True)
        step(circ)
        e_host.copy_(e_out, non_blocking=True)
        g_host.copy_(grads, non_blocking=True)

    step_e2e()
    ms_e2e = timed(step_e2e, args.steps)
    e2e_value = world * args.steps / (ms_e2e / 1000.0)

    # gate-by-gate comparison on the same workload
    plain = None
    if args.plain_steps > 0 and args.plan == "fused":
        circ_plain = S.Circuit(w.circuit, mode="plain", device=dev)
        step(circ_plain)
        ms_plain = timed(lambda: step(circ_plain), args.plain_steps)
        plain = {"value": world * args.plain_steps / (ms_plain / 1000.0), "unit": UNIT,
                 "ms_per_step": ms_plain / args.plain_steps, "steps": args.plain_steps}

    # plain gate sweeps at 30 qubits: one full-state kernel per gate, GB/s per (gate, target)
    sweep = None
    if args.sweep_n > 0:
        sweep = sweep_bench(S, torch, dev, args.sweep_n, barrier)

    tcb = None
    if args.tc_gates > 0:
        tcb = tc_bench(S, torch, dev, args.n, args.tc_gates, barrier)

    batched = None
    if args.batch_count > 0:
        batched = batch_bench(S, torch, dev, args.batch_count, barrier, rank=rank, world=world)

    grad_fn = grad_fn_bench(S, torch, dev, barrier) if args.grad_fn else None

    fwd_e = forward_expval_bench(S, torch, dev, w, barrier) if args.forward_expval else None

    small = small_bench(S, torch, dev, barrier) if args.small else None

    qft = None
    if args.qft_n > 0:
        del psi, lam
        torch.cuda.empty_cache()
        qft = qft_bench(S, torch, dev, args.qft_n, barrier)
        # the same workload planned with tensor-core blocks: which passes and
        # tensor-core launches that plan makes, and its time
        t = qft_bench(S, torch, dev, args.qft_n, barrier, mode="tc")
        qft["tc_plan"] = {"passes": t["passes"], "tc_block_launches": t.get("tc_block", {}).get("launches", 0),
                          "ms_per_grad_eval": t["ms_per_grad_eval"], "energy": t["energy"]}
        psi = S.State(n, torch.complex64, dev)
        lam = S.State(n, torch.complex64, dev)

    # the numbers being timed: one clean step (the gradient buffer accumulates
    # over steps), its E against a fresh forward's tqd_expval, and both E and
    # the gradient against the oracle's stored values for this workload
    grads.zero_()
    step(circ)
    e_step = float(e_out.item())
    g_step = grads.cpu().numpy()
    psi.reset(0)
    S.apply(psi, circ, params)
    e_check = S.expval(psi, obs).item()
    error = error_statement(args, e_step, e_check, g_step)

    if rank != 0:
        if world > 1:
            torch.distributed.barrier()
            torch.distributed.destroy_process_group()
        return 0

    # roofline of the dominant kernel class
    peak, peak_src = peaks()
    dom = max(prof, key=lambda p: p["ms"])
    per_launch_ms = dom["ms"] / max(1, dom["launches"])
    per_launch_bytes = dom["bytes"] / max(1, dom["launches"])
    achieved = per_launch_bytes / (per_launch_ms / 1000.0) / 1e9 if per_launch_ms > 0 else 0.0
    total_ms = sum(p["ms"] for p in prof)
    roofline = {
        "bound": "hbm", "kernel": dom["name"], "achieved": achieved, "peak": peak, "unit": "GB/s",
        "frac": achieved / peak, "peak_source": f"{peak_src} hbm_gbs",
        "traffic": stored_traffic(dom["name"]),
        "bytes_per_launch": per_launch_bytes, "ms_per_launch": per_launch_ms,
        "share_of_step": dom["ms"] / total_ms if total_ms > 0 else None,
    }
    kernels = sorted(({"name": p["name"], "launches": p["launches"], "ms": round(p["ms"], 3),
                       "gbs": round(p["bytes"] / (p["ms"] / 1000.0) / 1e9, 1) if p["ms"] > 0 and p["bytes"] > 0
                       else None} for p in prof), key=lambda d: -d["ms"])

    cpu = cpu_all = None
    if not args.no_cpu_baseline and world == 1:
        v, sample, _ = oracle_sample(w)
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample}
        try:
            cpu_all = oracle_all_cores(args.n, args.layers)
        except Exception as exc:  # context only: never fails the line
            cpu_all = {"unavailable": repr(exc)[:200]}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "c64", "data": "synthetic",
        "config": config_of(args, w, args.plan),
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(params_host.numel() * 8),
                "d2h_bytes_per_step": int(8 + g_host.numel() * 8), "ms_per_step": ms_e2e / args.steps},
        "gpu_launches": int(launches_per_step * args.steps),
        "roofline": roofline,
        "cpu_baseline": cpu,
        "cpu_baseline_all_cores": cpu_all,
        "plain": plain,
        "fused_over_plain": (value / plain["value"]) if plain else None,
        "sweep": sweep,
        "batched": batched,
        "tc_block": tcb,
        "grad24": grad_fn,
        "forward_expval": fwd_e,
        "qft32": qft,
        "small12": small,
        "clocks": clk.summary(),
        "kernels": kernels,
        "energy": e_step,
        "error": error,
    }
    print(json.dumps(line))
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
