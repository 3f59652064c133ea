"""The C-ABI library builds, loads without a GPU and exports every function include/fdtd.h
declares; the Python binding covers the same set (no compute calls here)."""
import ctypes
import os
import re

import pytest

from paper_2609_30039_gb300 import build as B
from paper_2609_30039_gb300 import fdtd

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    txt = open(os.path.join(ROOT, "include", "fdtd.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(fdtd_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    path = B.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared()
    for must in ("fdtd_create", "fdtd_step_forward", "fdtd_step_adjoint", "fdtd_dft_read", "fdtd_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_header():
    assert sorted(fdtd.declared_functions()) == declared()
    for n in declared():
        assert hasattr(fdtd, n), n


def _declared_arity():
    txt = open(os.path.join(ROOT, "include", "fdtd.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    out = {}
    for name, params in re.findall(r"\b(fdtd_[a-z0-9_]+)\s*\(([^;{]*?)\)\s*;", txt, flags=re.S):
        params = " ".join(params.split())
        out[name] = 0 if params in ("", "void") else params.count(",") + 1
    return out


def test_binding_argument_counts_match_header():
    # every ctypes signature has as many arguments as the C declaration
    arity = _declared_arity()
    assert set(arity) == set(declared())
    for name, n in arity.items():
        assert len(fdtd._SIGS[name]) == n, (name, len(fdtd._SIGS[name]), n)


def test_version_and_null_context_calls():
    fdtd.load()
    assert "sm_103a" in fdtd.fdtd_version()
    lib = fdtd.load()
    assert lib.fdtd_destroy(None) == fdtd.FDTD_OK
    assert lib.fdtd_step_forward(None, 1) == fdtd.FDTD_EINVAL
    assert isinstance(lib.fdtd_last_error(None), bytes)


def test_struct_layouts_match_c():
    # offsets fixed by the C declarations (natural alignment on LP64)
    assert ctypes.sizeof(fdtd.fdtd_grid) == 48 and fdtd.fdtd_grid.dx.offset == 16
    assert ctypes.sizeof(fdtd.fdtd_cpml) == 56 and fdtd.fdtd_cpml.m.offset == 24
    assert ctypes.sizeof(fdtd.fdtd_pole) == 32
    assert ctypes.sizeof(fdtd.fdtd_material) == 48 and fdtd.fdtd_material.pole_mask.offset == 40
