"""C-ABI library: builds, loads and exports every entry point declared in
include/psdf.h; host-side validation that runs before any CUDA call.  CPU only."""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np
import pytest

from paper_2607_04310_b300 import build as libbuild
from paper_2607_04310_b300 import psdf
from paper_2607_04310_b300 import scenegen as sg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(psdf_[a-z0-9_]+)\s*\(", txt))
    return names


@pytest.fixture(scope="module")
def lib():
    libbuild.build()
    return psdf.load()


def test_every_declared_symbol_is_exported(lib):
    declared = _declared()
    assert {"psdf_eval", "psdf_eval_grad", "psdf_backward", "psdf_scene_create_csr"} <= declared
    for name in sorted(declared):
        assert hasattr(lib, name), name
    # and the binding knows all of them
    assert declared <= set(psdf.exported_symbols())


def test_debug_build_exports_the_same_symbols():
    """The index-checking build (loaded by the GPU tests in a process of its
    own) declares the same ABI."""
    dbg = ctypes.CDLL(psdf.LIB_DEBUG_PATH)
    for name in sorted(_declared()):
        assert hasattr(dbg, name), name


def test_version_and_workspace(lib):
    assert lib.psdf_version() >= 100
    assert psdf.psdf_workspace_bytes(0) >= 256 + 8
    assert psdf.psdf_workspace_bytes(1000) >= 256 + 8000
    assert psdf.psdf_workspace_bytes(1000) % 256 == 0


def _create(edges, offs):
    e = np.ascontiguousarray(edges, dtype=np.float32)
    o = np.ascontiguousarray(offs, dtype=np.int32)
    out = ctypes.c_void_p()
    rc = psdf.load().psdf_scene_create_csr(e.ctypes.data, o.ctypes.data, len(o) - 1, 0, None,
                                           None, ctypes.byref(out))
    return rc, psdf.last_error()


def test_layout_validation_before_any_cuda_call(lib):
    e, o = sg.rects(sg.rng(0), 3, 0.2, 1.0, 0.0, 5.0)
    # unclosed polygon
    bad = e.copy()
    bad[1, 2] += 0.01
    rc, msg = _create(bad, o)
    assert rc == psdf.PSDF_ERR_LAYOUT and "not closed" in msg
    # clockwise polygon
    cw = e.copy()
    cw[0:4] = e[0:4][::-1][:, [2, 3, 0, 1]]
    rc, msg = _create(cw, o)
    assert rc == psdf.PSDF_ERR_LAYOUT
    # two-edge obstacle
    rc, msg = _create(e[:6], np.array([0, 2, 6], dtype=np.int32))
    assert rc == psdf.PSDF_ERR_LAYOUT and "2 edges" in msg
    # decreasing offsets
    rc, _ = _create(e, np.array([0, 8, 4, 12], dtype=np.int32))
    assert rc == psdf.PSDF_ERR_LAYOUT
    # degenerate (zero-length) segment
    seg = np.array([[1.0, 1.0, 1.0, 1.0]], dtype=np.float32)
    rc, msg = _create(seg, np.array([0, 1], dtype=np.int32))
    assert rc == psdf.PSDF_ERR_DEGENERATE_EDGE
    # non-finite coordinate
    nan = e.copy()
    nan[5, 0] = np.nan
    rc, _ = _create(nan, o)
    assert rc == psdf.PSDF_ERR_ARG
    # offsets[0] != 0
    rc, _ = _create(e, np.array([1, 4, 8, 12], dtype=np.int32))
    assert rc == psdf.PSDF_ERR_LAYOUT


def test_binding_fails_loudly_without_library(tmp_path):
    saved = psdf._lib
    psdf._lib = None
    try:
        with pytest.raises(RuntimeError, match="not built"):
            psdf.load(str(tmp_path / "missing.so"))
    finally:
        psdf._lib = saved


def test_binding_constants_match_the_header():
    """Every integer #define of include/psdf.h that the binding mirrors (under
    its own name or without the PSDF_ prefix) has the same value there."""
    txt = open(os.path.join(ROOT, "include", "psdf.h")).read()
    defs = dict(re.findall(r"#define\s+(PSDF_[A-Z0-9_]+)\s+(0x[0-9A-Fa-f]+|\d+)u?\b", txt))
    assert "PSDF_NOALLOC_MAX_POSES" in defs and "PSDF_ERR_CAPACITY" in defs
    mirrored = 0
    for name, val in defs.items():
        for py in (name, name[len("PSDF_"):]):
            if hasattr(psdf, py):
                assert getattr(psdf, py) == int(val, 0), (name, getattr(psdf, py), val)
                mirrored += 1
                break
    assert hasattr(psdf, "NOALLOC_MAX_POSES") and mirrored >= 12, mirrored
