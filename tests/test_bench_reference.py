"""The benchmark's reference arm on the CPU: one JSON line with the contract's
keys (the CPU oracle timed on a bounded sample of the 26-qubit workload), and
under torchrun only rank 0 prints it."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_reference(extra_env=None):
    env = dict(os.environ)
    env.pop("RANK", None)
    env.pop("WORLD_SIZE", None)
    env.update(extra_env or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                           "--warmup", "0"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def test_reference_arm_line():
    sys.path.insert(0, ROOT)
    import bench
    r = run_reference()
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT == "grad-evals/s"
    assert d["higher_is_better"] is True and d["steps"] == 1 and d["warmup"] == 0
    assert d["value"] > 0 and abs(d["ms_per_step"] - 1000.0 / d["value"]) < 1e-6 * d["ms_per_step"]
    assert d["config"]["n_qubits"] == 26 and d["config"]["layers"] == 20
    assert d["dtype"] == "c128" and d["config"]["amplitudes"] == "complex128"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_exit_quietly():
    r = run_reference({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert r.returncode == 0, r.stderr[-2000:]
    assert not [l for l in r.stdout.splitlines() if l.startswith("{")]


def test_oracle_on_all_cores_small():
    """The all-core oracle baseline: one process per core, rates summed; a
    deadline it cannot meet turns it into an 'unavailable' note and leaves no
    process behind."""
    sys.path.insert(0, ROOT)
    import bench
    r = bench.oracle_all_cores(14, 2, gate_sample=4, term_sample=2, procs=2)
    assert r["cores"] == 2 and r["kind"] == "oracle" and r["unit"] == "grad-evals/s" and r["value"] > 0
    assert r["host_cores"] == len(os.sched_getaffinity(0))
    slow = bench.oracle_all_cores(24, 10, gate_sample=6, term_sample=2, procs=2, deadline_s=0.01)
    assert "unavailable" in slow
    left = subprocess.run(["ps", "-eo", "args"], capture_output=True, text=True).stdout
    assert "workload_hea(2, 24, 10" not in left
