"""The C-ABI library builds, loads, and exports every function include/fs1.h
declares; the ctypes structures match the header's layout.  No GPU calls."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2202_10042_gb300 import build as pkg_build
from paper_2202_10042_gb300 import fs1

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fs1.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(fs1_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    pkg_build.build()
    return fs1.load()


def test_header_declares_expected(lib):
    assert set(_declared()) == set(fs1.EXPORTED)


def test_every_declared_symbol_exported(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", fs1.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (fs1_[a-z0-9_]+)", out))
    for name in _declared():
        assert name in exported, name
        assert hasattr(lib, name)


def test_struct_layout_matches_header():
    """Compile a C probe of the header's struct sizes / offsets and compare with ctypes."""
    probe = r'''
#include <stddef.h>
#include <stdio.h>
#include "fs1.h"
int main(void) {
  printf("%zu %zu %zu\n", sizeof(fs1_config), sizeof(fs1_problem), sizeof(fs1_info));
  printf("%zu %zu %zu %zu\n", offsetof(fs1_problem, n), offsetof(fs1_problem, a),
         offsetof(fs1_problem, g_init), offsetof(fs1_info, w1));
  printf("%zu %zu %zu %zu %zu\n", offsetof(fs1_config, spin_cap), offsetof(fs1_config, stream),
         offsetof(fs1_config, autotune), offsetof(fs1_config, use_graph), offsetof(fs1_config, tau));
  printf("%zu\n", offsetof(fs1_config, grid2d));
  return 0;
}
'''
    import tempfile
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "p.c")
        exe = os.path.join(d, "p")
        open(c, "w").write(probe)
        subprocess.run(["cc", "-I" + os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        vals = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()
    vals = [int(v) for v in vals]
    assert vals[0] == ctypes.sizeof(fs1.fs1_config)
    assert vals[1] == ctypes.sizeof(fs1.fs1_problem)
    assert vals[2] == ctypes.sizeof(fs1.fs1_info)
    assert vals[3] == fs1.fs1_problem.n.offset
    assert vals[4] == fs1.fs1_problem.a.offset
    assert vals[5] == fs1.fs1_problem.g_init.offset
    assert vals[6] == fs1.fs1_info.w1.offset
    assert vals[7] == fs1.fs1_config.spin_cap.offset
    assert vals[8] == fs1.fs1_config.stream.offset
    assert vals[9] == fs1.fs1_config.autotune.offset
    assert vals[10] == fs1.fs1_config.use_graph.offset
    assert vals[11] == fs1.fs1_config.tau.offset
    assert vals[12] == fs1.fs1_config.grid2d.offset


def test_status_strings_and_version(lib):
    # host-only entry points: no device needed
    assert fs1.fs1_status_string(fs1.FS1_OK) == "FS1_OK"
    assert fs1.fs1_status_string(fs1.FS1_ENUMERIC) == "FS1_ENUMERIC"
    assert fs1.fs1_version().startswith("fs1-gb300")
    cfg = fs1.fs1_config_default()
    assert cfg.variant == fs1.FS1_VARIANT_LOG and cfg.precision == fs1.FS1_FP32
    assert cfg.check_every == 1 and cfg.spin_cap > 0 and cfg.autotune == 1 and cfg.trial_iters > 0
    assert cfg.use_graph == 1 and cfg.tau == 1e10


def test_missing_library_fails_loudly(tmp_path):
    with pytest.raises(RuntimeError):
        fs1._lib_backup = fs1._lib
        try:
            fs1._lib = None
            fs1.load(str(tmp_path / "nope.so"))
        finally:
            fs1._lib = fs1._lib_backup
