"""The C-ABI library builds, loads and exports every symbol include/*.h declares.

CPU only: nothing here calls into CUDA (loading the library does not need a GPU).
"""
import glob
import os
import re

import pytest

from paper_1502_02935_gb300 import build, mhd

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"\b(mhd_\w+)\s*\(", src)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("mhd_init_grid", "mhd_set_sources", "mhd_step", "mhd_cfl_dt", "mhd_get_state"):
        assert required in names


def test_library_exports_every_declared_symbol():
    path = build.build()
    assert os.path.exists(path)
    L = mhd.lib()
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_binding_wraps_every_export():
    assert set(declared_functions()) <= set(mhd.EXPORTS)
