"""FP64 CPU oracle for the PSDF -- TEST INFRASTRUCTURE ONLY.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never imports it and shares no code with it.

The arithmetic lives in ``psdf_oracle.c`` (plain C, FP64, OpenMP over poses)
and ``mlp.py`` (the tile-proposal network in numpy FP64).  This module only
builds/loads the C library and marshals numpy arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Dict, Optional, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "psdf_oracle.c")
_LIB = os.path.join(_HERE, "libpsdf_oracle.so")
_lib = None

PID_NONE = 0xFFFFFFFF


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (FP64, no FMA contraction, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC",
               "-shared", _SRC, "-o", tmp, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [("eps_seg", ctypes.c_double), ("eps_axis", ctypes.c_double),
                ("eps_sat", ctypes.c_double), ("eta", ctypes.c_double)]


def _bind(path: str):
    """Load a compiled oracle library and declare its C signatures."""
    lib = ctypes.CDLL(path)
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int)
    up = ctypes.POINTER(ctypes.c_uint)
    lib.oracle_psdf_eval.argtypes = [dp, ctypes.c_int, dp, ip, ctypes.c_int, dp, ctypes.c_long,
                                     ctypes.POINTER(_Params), dp, up, dp, dp, dp, up,
                                     ctypes.c_int]
    lib.oracle_psdf_backward.argtypes = [dp, ctypes.c_int, dp, ip, ctypes.c_int, dp,
                                         ctypes.c_long, ctypes.POINTER(_Params), dp, dp, dp,
                                         ctypes.c_int]
    lib.oracle_psdf_obstacle_sd.argtypes = [dp, ctypes.c_int, dp, ip, ctypes.c_int, dp,
                                            ctypes.c_long, ctypes.POINTER(_Params), dp,
                                            ctypes.c_int]
    lib.oracle_max_threads.restype = ctypes.c_int
    return lib


def compile_variant(src_text: str, out_path: str) -> str:
    """Compile an edited copy of the oracle source (used by the tests that
    plant mistakes in the oracle to show the pins catch them)."""
    cpath = out_path + ".c"
    with open(cpath, "w") as f:
        f.write(src_text)
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared",
                           cpath, "-o", out_path, "-lm"])
    return out_path


def source_text() -> str:
    with open(_SRC) as f:
        return f.read()


_variant = None


def use_library(path: Optional[str]) -> None:
    """Route the functions below to another build of the oracle (None = default)."""
    global _variant
    _variant = _bind(path) if path else None


def _load():
    global _lib
    if _variant is not None:
        return _variant
    if _lib is None:
        lib = _bind(build())
        _lib = lib
    return _lib


def _d(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _ptr(a: np.ndarray, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _params(eps_seg, eps_axis, eps_sat, eta) -> _Params:
    return _Params(float(eps_seg), float(eps_axis), float(eps_sat), float(eta))


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def psdf_eval(footprint, edges, offsets, poses, eps_seg=0.0, eps_axis=0.0, eps_sat=0.0,
              eta=0.0, nthreads: int = 0) -> Dict[str, np.ndarray]:
    """phi, active pair id, d phi / d pose, tie margin, edge-attribution
    margin and antiparallel-twin pair id for every pose (float64 inputs;
    float32 inputs are widened exactly)."""
    lib = _load()
    fp = _d(footprint)
    ed = _d(edges).reshape(-1, 4)
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int32))
    ps = _d(poses).reshape(-1, 3)
    P = ps.shape[0]
    M = len(off) - 1
    phi = np.empty(P)
    pair = np.empty(P, dtype=np.uint32)
    grad = np.empty((P, 3))
    margin = np.empty(P)
    egap = np.empty(P)
    twin = np.empty(P, dtype=np.uint32)
    prm = _params(eps_seg, eps_axis, eps_sat, eta)
    rc = lib.oracle_psdf_eval(_ptr(fp, ctypes.c_double), fp.shape[0], _ptr(ed, ctypes.c_double),
                              _ptr(off, ctypes.c_int), M, _ptr(ps, ctypes.c_double), P,
                              ctypes.byref(prm), _ptr(phi, ctypes.c_double),
                              _ptr(pair, ctypes.c_uint), _ptr(grad, ctypes.c_double),
                              _ptr(margin, ctypes.c_double), _ptr(egap, ctypes.c_double),
                              _ptr(twin, ctypes.c_uint), int(nthreads))
    if rc != 0:
        raise ValueError("oracle_psdf_eval: invalid input (code %d)" % rc)
    return {"phi": phi, "pair": pair, "grad": grad, "margin": margin, "egap": egap,
            "twin": twin}


def psdf_backward(footprint, edges, offsets, poses, grad_phi, eps_seg=0.0, eps_axis=0.0,
                  eps_sat=0.0, eta=0.0, nthreads: int = 0) -> Tuple[np.ndarray, np.ndarray]:
    """(grad_pose [P,3], grad_edges [E,4]) of sum_p grad_phi[p] * phi[p]."""
    lib = _load()
    fp = _d(footprint)
    ed = _d(edges).reshape(-1, 4)
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int32))
    ps = _d(poses).reshape(-1, 3)
    gphi = _d(grad_phi).reshape(-1)
    P = ps.shape[0]
    gp = np.empty((P, 3))
    ge = np.empty_like(ed)
    prm = _params(eps_seg, eps_axis, eps_sat, eta)
    rc = lib.oracle_psdf_backward(_ptr(fp, ctypes.c_double), fp.shape[0],
                                  _ptr(ed, ctypes.c_double), _ptr(off, ctypes.c_int),
                                  len(off) - 1, _ptr(ps, ctypes.c_double), P, ctypes.byref(prm),
                                  _ptr(gphi, ctypes.c_double), _ptr(gp, ctypes.c_double),
                                  _ptr(ge, ctypes.c_double), int(nthreads))
    if rc != 0:
        raise ValueError("oracle_psdf_backward: invalid input (code %d)" % rc)
    return gp, ge


def obstacle_sd(footprint, edges, offsets, poses, eps_seg=0.0, eps_axis=0.0, eps_sat=0.0,
                eta=0.0, nthreads: int = 0) -> np.ndarray:
    """Per-obstacle signed distances [P, M] (before the minimum over obstacles)."""
    lib = _load()
    fp = _d(footprint)
    ed = _d(edges).reshape(-1, 4)
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int32))
    ps = _d(poses).reshape(-1, 3)
    P, M = ps.shape[0], len(off) - 1
    sd = np.empty((P, M))
    prm = _params(eps_seg, eps_axis, eps_sat, eta)
    rc = lib.oracle_psdf_obstacle_sd(_ptr(fp, ctypes.c_double), fp.shape[0],
                                     _ptr(ed, ctypes.c_double), _ptr(off, ctypes.c_int), M,
                                     _ptr(ps, ctypes.c_double), P, ctypes.byref(prm),
                                     _ptr(sd, ctypes.c_double), int(nthreads))
    if rc != 0:
        raise ValueError("oracle_psdf_obstacle_sd: invalid input (code %d)" % rc)
    return sd


def pair_fields(pid: int) -> Tuple[int, int, int]:
    """(edge, kind, l) of an active pair id."""
    pid = int(pid)
    return pid >> 8, (pid >> 4) & 0xF, pid & 0xF
