"""The ctypes option and statistics structures of the Python binding have the layout of their
C declarations in include/chem.h: every field at the same offset, every structure the same
size.  A small C program compiled with the host compiler against the header prints the C
side (no GPU, no CUDA headers: chem.h is plain C)."""
import ctypes
import os
import shutil
import subprocess

import pytest

from conftest import ROOT

# ctypes class name in chem.py -> C typedef in chem.h
PAIRS = {
    "DiOpts": "chem_di_opts",
    "TrainOpts": "chem_train_opts",
    "TrainEpochOpts": "chem_train_epoch_opts",
    "AnnOpts": "chem_ann_opts",
    "ServerOpts": "chem_server_opts",
    "ServerStats": "chem_server_stats",
    "HfrdOpts": "chem_hfrd_opts",
}


def _c_layout(tmp_path):
    from paper_2402_18858_gb300 import chem
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "chem.h"', "int main(void) {"]
    for py, c in PAIRS.items():
        cls = getattr(chem, py)
        lines.append(f'  printf("{py} size %zu\\n", sizeof({c}));')
        for name, _ in cls._fields_:
            lines.append(f'  printf("{py} {name} %zu\\n", offsetof({c}, {name}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    got = {}
    for ln in out.splitlines():
        py, field, val = ln.split()
        got[(py, field)] = int(val)
    return got


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs a host C compiler")
def test_ctypes_structures_match_the_header(tmp_path):
    from paper_2402_18858_gb300 import chem
    c = _c_layout(tmp_path)
    for py in PAIRS:
        cls = getattr(chem, py)
        assert ctypes.sizeof(cls) == c[(py, "size")], py
        for name, _ in cls._fields_:
            assert getattr(cls, name).offset == c[(py, name)], (py, name)
