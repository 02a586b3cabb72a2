"""The C-ABI library loads and exports every entry point include/wslda_td.h
declares (no GPU needed: nothing is called)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "wslda_td.h")
LIB = os.path.join(ROOT, "paper_2602_08982_b300", "_lib", "libwslda_td.so")


def declared():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"\b(wslda_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(LIB):
        from paper_2602_08982_b300 import build
        build.build()
    return ctypes.CDLL(LIB)


def test_header_declares_the_entry_points():
    names = declared()
    for n in ("wslda_create", "wslda_add_box", "wslda_load_states", "wslda_start", "wslda_step",
              "wslda_get_densities", "wslda_get_energy", "wslda_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_loads_without_touching_the_gpu():
    from paper_2602_08982_b300 import wslda
    assert wslda.lattice_supported(wslda.MIXED, 32, 32, 32)
    assert wslda.lattice_supported(wslda.FP64, 16, 16, 16)
    assert not wslda.lattice_supported(wslda.FP64, 14, 14, 14)
