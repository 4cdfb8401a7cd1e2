"""The C-ABI library builds, loads without a GPU, and exports every entry point that
include/pet.h declares; the binding covers them all (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "pet.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pet_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpet():
    from paper_2111_07886_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_entry_points():
    names = declared_functions()
    for must in ("pet_geometry_create", "pet_forward_subset", "pet_back_subset", "pet_subiter",
                 "pet_reconstruct", "pet_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol(libpet):
    missing = [n for n in declared_functions() if not hasattr(libpet, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2111_07886_gb300 import pet
    assert set(declared_functions()) <= set(pet.SIGNATURES), \
        set(declared_functions()) - set(pet.SIGNATURES)


def test_invalid_geometry_rejected_without_gpu(libpet):
    """Argument validation happens on the host before any CUDA call."""
    from paper_2111_07886_gb300 import pet
    L = pet.lib()
    d = pet.GeometryDesc(0, 1, 1.0, 10, 10, 1.0, 1, 1.0)
    h = ctypes.c_void_p()
    assert L.pet_geometry_create(ctypes.byref(d), None, ctypes.byref(h)) == pet.ERR_INVALID
    assert b"invalid geometry" in L.pet_last_error()
    d = pet.GeometryDesc(16, 1, 1.0, 10, 10, 1.0, 11, 1.0)          # M > V
    assert L.pet_geometry_create(ctypes.byref(d), None, ctypes.byref(h)) == pet.ERR_INVALID
    assert L.pet_subiter(None, None) == pet.ERR_INVALID


def test_oracle_is_not_linked_by_the_library(libpet):
    """The product library shares no code with the oracle: no ora_* symbol is exported."""
    assert not hasattr(libpet, "ora_forward")
