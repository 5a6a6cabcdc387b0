"""The ctypes structures of the binding against the C header: every struct of
include/tqd.h compiled with the host C compiler, its size and each field's
offset compared with the binding's mirror (no GPU, no library needed)."""
import ctypes as C
import os
import shutil
import subprocess

import pytest

from paper_2511_19291_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# C struct -> (binding class, the binding's field names in order)
STRUCTS = {
    "tqd_gate": _lib.Gate,
    "tqd_pauli_term": _lib.PauliTerm,
    "tqd_plan_opts": _lib.PlanOpts,
    "tqd_batch_opts": _lib.BatchOpts,
    "tqd_profile_entry": _lib.ProfileEntry,
}


def _c_layouts(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "tqd.h"', "int main(void) {"]
    for cname, cls in STRUCTS.items():
        lines.append(f'    printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'    printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True,
                   capture_output=True, text=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    got = {}
    for line in out.splitlines():
        cname, key, value = line.split()
        got[(cname, key)] = int(value)
    return got


def test_binding_structs_match_header(tmp_path):
    got = _c_layouts(tmp_path)
    for cname, cls in STRUCTS.items():
        assert got[(cname, "size")] == C.sizeof(cls), (cname, got[(cname, "size")], C.sizeof(cls))
        for fname, _ in cls._fields_:
            assert got[(cname, fname)] == getattr(cls, fname).offset, (cname, fname)


def test_checkpoint_option_codes():
    # the binding's "no checkpoints" code is the header's TQD_CHECKPOINTS_NONE
    with open(os.path.join(ROOT, "include", "tqd.h")) as f:
        header = f.read()
    assert "#define TQD_CHECKPOINTS_NONE 0xFFFFFFFFu" in header
    assert _lib.CHECKPOINTS_NONE == 0xFFFFFFFF
