"""Builds ``libtqd.so`` in-tree with nvcc for sm_103a.

Each ``csrc/*.cu`` file is compiled in parallel to an object file, then the
objects are linked into ``_build/libtqd.so`` (static CUDA runtime, C ABI of
``include/tqd.h``).  ``python -m paper_2511_19291_gb300.build`` builds it.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import hashlib
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(BUILD, "libtqd.so")
GEN = os.path.join(BUILD, "gen")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# device headers handed to the run-time compiler for the pass-specialised kernels
JIT_HEADERS = ["common.cuh", "tile_desc.h", "tile_dev.cuh"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _write_jit_headers() -> None:
    """Embeds the device headers' text in the library (``tqd_jit_headers.inc``)."""
    os.makedirs(GEN, exist_ok=True)
    srcs = []
    for name in JIT_HEADERS:
        with open(os.path.join(CSRC, name)) as f:
            text = f.read()
        if ")TQDSRC" in text:
            raise RuntimeError(f"{name} contains the raw-string delimiter")
        srcs.append(text)
    out = ["// Generated by build.py from csrc/: header texts for the run-time compiler.",
           "static const char *const k_jit_header_names[] = {" + ", ".join(f'"{n}"' for n in JIT_HEADERS) + "};",
           "static const char *const k_jit_header_srcs[] = {"]
    out += [f'R"TQDSRC({t})TQDSRC",' for t in srcs]
    out += ["};", f"static const int k_jit_n_headers = {len(JIT_HEADERS)};", ""]
    path = os.path.join(GEN, "tqd_jit_headers.inc")
    with open(path + ".tmp", "w") as f:
        f.write("\n".join(out))
    os.replace(path + ".tmp", path)


def _flags(verbose_ptxas: bool) -> list:
    f = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2", "-I", INCLUDE, "-I", CSRC, "-I", GEN,
                "--expt-relaxed-constexpr", "-DNDEBUG"]
    if os.environ.get("TQD_CHECKED") == "1":
        # kernels check their shared-memory indices and record failures
        f += ["-DTQD_CHECKED"]
    if verbose_ptxas:
        f += ["-Xptxas", "-v"]
    return f


def _digest() -> str:
    h = hashlib.sha256()
    h.update(b"checked" if os.environ.get("TQD_CHECKED") == "1" else b"release")
    for p in sorted(glob.glob(os.path.join(CSRC, "*")) + [os.path.join(INCLUDE, "tqd.h"), __file__]):
        with open(p, "rb") as f:
            h.update(os.path.basename(p).encode())
            h.update(f.read())
    return h.hexdigest()


def build(force: bool = False, verbose_ptxas: bool = False, jobs: int | None = None) -> str:
    os.makedirs(BUILD, exist_ok=True)
    stamp = os.path.join(BUILD, "libtqd.sha256")
    digest = _digest()
    if not force and os.path.exists(LIB) and os.path.exists(stamp):
        with open(stamp) as f:
            if f.read().strip() == digest:
                return LIB
    _write_jit_headers()
    sources = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    cc = nvcc()
    flags = _flags(verbose_ptxas)
    log_lines = []

    def compile_one(src):
        obj = os.path.join(BUILD, os.path.basename(src)[:-3] + ".o")
        cmd = [cc, *flags, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {os.path.basename(src)}:\n{r.stdout}\n{r.stderr}")
        return obj, r.stderr

    jobs = jobs or min(len(sources), os.cpu_count() or 4)
    with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
        results = list(ex.map(compile_one, sources))
    objs = [o for o, _ in results]
    for _, err in results:
        if err:
            log_lines.append(err)
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs, "-lcuda" if False else "-lcudart_static", "-ldl", "-lpthread",
           "-lrt"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    with open(stamp, "w") as f:
        f.write(digest)
    with open(os.path.join(BUILD, "ptxas.log"), "w") as f:
        f.write("\n".join(log_lines))
    return LIB


if __name__ == "__main__":
    v = "-v" in sys.argv
    print(build(force="--force" in sys.argv, verbose_ptxas=v))
    if v:
        print(open(os.path.join(BUILD, "ptxas.log")).read())
