"""Host-side checks of the C-ABI library that need no GPU: it builds for
sm_103a, loads, exports every function include/bhgrav.h declares, and its
argument checks that run before any CUDA call behave as documented."""
import ctypes
import os
import re

import pytest

from paper_1509_07370_gb300 import bhgrav as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(bh_\w+)\s*\(", txt))
    return names


def test_library_builds_and_exports_every_declared_symbol():
    lib = B.load()
    declared = _declared()
    assert {"bh_create", "bh_build", "bh_potential", "bh_destroy"} <= declared
    for name in declared:
        assert hasattr(lib, name), name
    assert set(B.EXPORTED) == declared


def test_default_options():
    o = B.bh_default_options()
    assert (o.precision, o.criterion, o.kahan) == (B.BH_PREC_F32, B.BH_CRIT_PER_CELL, 1)


def test_null_arguments_fail_without_touching_the_gpu():
    lib = B.load()
    assert lib.bh_create(None, None, 0, None) == B.BH_ERR_ARG
    assert lib.bh_build(None, 1, None, None, None, 1.0, None, 0) == B.BH_ERR_ARG
    assert lib.bh_potential(None, 0.5, 1.0, None) == B.BH_ERR_ARG
    assert lib.bh_walk_counts(None, 0.5, None, None, None) == B.BH_ERR_ARG
    assert lib.bh_tree_size(None, None, None, None) == B.BH_ERR_ARG
    assert lib.bh_export_nodes(None, None, None, None, None, None) == B.BH_ERR_ARG
    assert lib.bh_last_error(None) == b"null context"
    lib.bh_destroy(None)


def test_bad_options_rejected_before_device_use():
    lib = B.load()
    h = ctypes.c_void_p()
    o = B.bh_default_options()
    o.precision = 7
    assert lib.bh_create(ctypes.byref(h), ctypes.byref(o), 0, None) == B.BH_ERR_ARG
    o = B.bh_default_options()
    o.criterion = -1
    assert lib.bh_create(ctypes.byref(h), ctypes.byref(o), 0, None) == B.BH_ERR_ARG
    # periodic boundaries: the binary32 per-cell monopole walk only
    for field, value in (("quadrupole", 1), ("learned", 1), ("precision", B.BH_PREC_F64),
                         ("criterion", B.BH_CRIT_WARP_VOTE)):
        o = B.bh_default_options()
        o.periodic = 1
        setattr(o, field, value)
        assert lib.bh_create(ctypes.byref(h), ctypes.byref(o), 0, None) == B.BH_ERR_ARG
    o = B.bh_default_options()
    o.periodic = 2
    assert lib.bh_create(ctypes.byref(h), ctypes.byref(o), 0, None) == B.BH_ERR_ARG
    assert not h.value
    assert lib.bh_set_ewald(None, 64, 3) == B.BH_ERR_ARG
    assert lib.bh_ewald_eval(None, 0, None, None) == B.BH_ERR_ARG


def test_library_is_built_for_sm103a():
    B.load()
    objs = [f for f in os.listdir(os.path.dirname(B.library_path())) if f.endswith(".o")]
    assert objs
    # the build command pins the architecture; the flag list is the contract
    from paper_1509_07370_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in build.ARCH


def test_product_code_never_reaches_the_oracle():
    """The library and its binding neither import, load nor name the oracle."""
    pkg = os.path.join(ROOT, "paper_1509_07370_gb300")
    for dirpath, _, files in os.walk(pkg):
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                src = open(os.path.join(dirpath, fn)).read()
                assert not re.search(r"^\s*(from|import)\s+oracle", src, re.M), fn
                assert "liboracle" not in src and "bh_oracle" not in src, fn
