"""Thin ctypes binding of libpsdf_b300.so (C ABI in include/psdf.h).

Argument marshalling only: every step of the PSDF runs in the library's CUDA
kernels.  Functions carry the C names; device buffers are torch CUDA tensors
(PyTorch supplies memory and streams), host inputs are numpy arrays.  If the
library is missing this module raises -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Tuple

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# PSDF_LIBRARY names another build of the library for this process (the
# tests run the batched kernels' index-checking build, LIB_DEBUG_PATH, so)
LIB_PATH = os.environ.get("PSDF_LIBRARY") or os.path.join(HERE, "libpsdf_b300.so")
LIB_DEBUG_PATH = os.path.join(HERE, "libpsdf_b300_debug.so")

PSDF_OK = 0
PSDF_ERR_ARG = 1
PSDF_ERR_FOOTPRINT = 2
PSDF_ERR_DEGENERATE_EDGE = 3
PSDF_ERR_LAYOUT = 4
PSDF_ERR_CUDA = 5
PSDF_ERR_TIMEOUT = 6
PSDF_ERR_CAPACITY = 7
PAIR_NONE = 0xFFFFFFFF

KINDS = {0: "robot vertex -> obstacle edge", 1: "obstacle vertex A -> robot edge",
         2: "segment B -> robot edge", 3: "robot axis, obstacle max - robot min",
         4: "robot axis, robot max - obstacle min", 5: "robot axis (B), obstacle max - robot min",
         6: "robot axis (B), robot max - obstacle min",
         7: "obstacle axis, obstacle max - robot min",
         8: "obstacle axis, robot max - obstacle min"}


class PsdfError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("psdf error %d: %s" % (code, msg))
        self.code = code


class Params(ctypes.Structure):
    _fields_ = [("eps_seg", ctypes.c_float), ("eps_axis", ctypes.c_float),
                ("eps_sat", ctypes.c_float), ("eta", ctypes.c_float)]


class CullGridInfo(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("entries", ctypes.c_int64),
                ("x0", ctypes.c_float), ("y0", ctypes.c_float), ("cell", ctypes.c_float),
                ("reach", ctypes.c_float), ("inv_cell", ctypes.c_float)]


class SceneInfo(ctypes.Structure):
    _fields_ = [("n_edges", ctypes.c_int64), ("n_obstacles", ctypes.c_int32),
                ("n_tiles", ctypes.c_int32), ("tile_edges", ctypes.c_int32),
                ("max_obstacle_edges", ctypes.c_int32), ("bbox", ctypes.c_float * 4),
                ("device_bytes", ctypes.c_int64)]


class PlanConfig(ctypes.Structure):
    _fields_ = [("threads", ctypes.c_int32), ("tiles_per_item", ctypes.c_int32)]


class PlanInfo(ctypes.Structure):
    _fields_ = [("n_inst", ctypes.c_int32), ("n_tiles", ctypes.c_int32),
                ("n_poses", ctypes.c_int64), ("n_rows", ctypes.c_int64),
                ("n_items", ctypes.c_int32), ("n_blocks", ctypes.c_int32),
                ("grid", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("config", PlanConfig), ("device_bytes", ctypes.c_size_t)]


_lib = None
_vp = ctypes.c_void_p
_SIGS = {
    "psdf_last_error": (ctypes.c_char_p, []),
    "psdf_version": (ctypes.c_int, []),
    "psdf_scene_create_csr": (ctypes.c_int, [_vp, _vp, ctypes.c_int32, ctypes.c_int32, _vp, _vp,
                                             ctypes.POINTER(_vp)]),
    "psdf_scene_create_padded": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int32, ctypes.c_int32,
                                                ctypes.c_int32, _vp, _vp, ctypes.POINTER(_vp)]),
    "psdf_scene_destroy": (ctypes.c_int, [_vp]),
    "psdf_scene_get_info": (ctypes.c_int, [_vp, ctypes.POINTER(SceneInfo)]),
    "psdf_scene_cull_grid": (ctypes.c_int, [_vp, ctypes.POINTER(CullGridInfo)]),
    "psdf_scene_cull_grid_copy": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "psdf_workspace_bytes": (ctypes.c_size_t, [ctypes.c_int64]),
    "psdf_workspace_status": (ctypes.c_int, [_vp, _vp]),
    "psdf_eval": (ctypes.c_int, [_vp, ctypes.c_int32, _vp, _vp, ctypes.c_int64, _vp, _vp, _vp,
                                 _vp, ctypes.c_size_t, _vp]),
    "psdf_eval_grad": (ctypes.c_int, [_vp, ctypes.c_int32, _vp, _vp, ctypes.c_int64, _vp, _vp,
                                      _vp, _vp, _vp, ctypes.c_size_t, _vp]),
    "psdf_backward": (ctypes.c_int, [_vp, ctypes.c_int32, _vp, _vp, ctypes.c_int64, _vp, _vp,
                                     _vp, _vp, _vp, _vp]),
    "psdf_eval_grad_save": (ctypes.c_int, [_vp, ctypes.c_int32, _vp, _vp, ctypes.c_int64, _vp,
                                           _vp, _vp, _vp, _vp, _vp, ctypes.c_size_t, _vp]),
    "psdf_backward_saved": (ctypes.c_int, [_vp, _vp, ctypes.c_int64, _vp, _vp, _vp, _vp]),
    "psdf_eval_keys": (ctypes.c_int, [_vp, ctypes.c_int32, _vp, _vp, ctypes.c_int64, _vp,
                                      ctypes.c_int64, _vp, _vp, ctypes.c_size_t, _vp]),
    "psdf_merge_keys": (ctypes.c_int, [_vp, _vp, ctypes.c_int64, _vp]),
    "psdf_finish_keys": (ctypes.c_int, [_vp, ctypes.c_int32, _vp, _vp, ctypes.c_int64, _vp,
                                        ctypes.c_int64, ctypes.c_int32, _vp, _vp, _vp, _vp,
                                        _vp]),
    "psdf_stage_params": (ctypes.c_int, [_vp, ctypes.c_int32, _vp, _vp, ctypes.c_int64, _vp,
                                         ctypes.c_float, _vp, _vp, _vp, ctypes.c_size_t, _vp]),
    "psdf_stage_params_batched": (ctypes.c_int, [_vp, _vp, ctypes.c_float, _vp, _vp, _vp]),
    "psdf_eval_grad_noalloc": (ctypes.c_int, [_vp, ctypes.c_int32, _vp, _vp, ctypes.c_int64,
                                              _vp, _vp, _vp, _vp, _vp]),
    "psdf_mlp_create": (ctypes.c_int, [_vp, _vp, ctypes.c_float, ctypes.POINTER(_vp)]),
    "psdf_mlp_destroy": (ctypes.c_int, [_vp]),
    "psdf_tile_features": (ctypes.c_int, [_vp, ctypes.c_int32, _vp, _vp, ctypes.c_int64, _vp,
                                          _vp]),
    "psdf_mlp_scores": (ctypes.c_int, [_vp, _vp, ctypes.c_int32, _vp, _vp, ctypes.c_int64, _vp,
                                       _vp]),
    "psdf_tile_values": (ctypes.c_int, [_vp, ctypes.c_int32, _vp, _vp, ctypes.c_int64, _vp,
                                        _vp, _vp]),
    "psdf_tile_lower_bounds": (ctypes.c_int, [_vp, ctypes.c_int32, _vp, _vp, ctypes.c_int64,
                                              _vp, _vp]),
    "psdf_cull_workspace_bytes": (ctypes.c_size_t, [ctypes.c_int64, _vp]),
    "psdf_eval_culled": (ctypes.c_int, [_vp, ctypes.c_int32, _vp, _vp, _vp, _vp,
                                        ctypes.c_int64, _vp, _vp, _vp, _vp, _vp,
                                        ctypes.c_size_t, _vp]),
    "psdf_eval_culled_save": (ctypes.c_int, [_vp, ctypes.c_int32, _vp, _vp, _vp, _vp,
                                             ctypes.c_int64, _vp, _vp, _vp, _vp, _vp, _vp,
                                             ctypes.c_size_t, _vp]),
    "psdf_cull_stats_read": (ctypes.c_int, [_vp, _vp, _vp]),
    "psdf_trainer_create": (ctypes.c_int, [_vp, _vp, ctypes.c_float, ctypes.c_float,
                                           ctypes.POINTER(_vp)]),
    "psdf_trainer_destroy": (ctypes.c_int, [_vp]),
    "psdf_trainer_set_lr": (ctypes.c_int, [_vp, ctypes.c_float]),
    "psdf_trainer_grad": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int64, _vp, _vp, _vp]),
    "psdf_trainer_step": (ctypes.c_int, [_vp, _vp, _vp, _vp, ctypes.c_int64, _vp, _vp]),
    "psdf_trainer_get": (ctypes.c_int, [_vp, _vp, _vp, _vp, ctypes.POINTER(ctypes.c_int64)]),
    "psdf_trainer_set": (ctypes.c_int, [_vp, _vp, _vp, _vp, ctypes.c_int64]),
    "psdf_plan_create": (ctypes.c_int, [ctypes.c_int32, _vp, _vp, _vp, _vp, _vp, _vp,
                                        ctypes.c_int32, _vp, _vp, ctypes.POINTER(_vp)]),
    "psdf_plan_destroy": (ctypes.c_int, [_vp]),
    "psdf_plan_get_info": (ctypes.c_int, [_vp, ctypes.POINTER(PlanInfo)]),
    "psdf_plan_set_config": (ctypes.c_int, [_vp, ctypes.POINTER(PlanConfig), _vp]),
    "psdf_plan_autotune": (ctypes.c_int, [_vp, _vp, ctypes.c_int32, _vp,
                                          ctypes.POINTER(PlanConfig),
                                          ctypes.POINTER(ctypes.c_int32)]),
    "psdf_eval_batched": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "psdf_plan_status": (ctypes.c_int, [_vp, _vp]),
    "psdf_plan_debug_read": (ctypes.c_int, [ctypes.POINTER(ctypes.c_uint64),
                                            ctypes.POINTER(ctypes.c_int32)]),
    "psdf_backward_batched": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "psdf_debug_set_wait_limit": (ctypes.c_int, [ctypes.c_uint32,
                                                 ctypes.POINTER(ctypes.c_uint32)]),
    "psdf_measure_fp32_peak": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                              ctypes.POINTER(ctypes.c_double),
                                              ctypes.POINTER(ctypes.c_double), _vp]),
    "psdf_profile_enable": (ctypes.c_int, [ctypes.c_int]),
    "psdf_profile_reset": (ctypes.c_int, []),
    "psdf_profile_read": (ctypes.c_int, [ctypes.c_char_p, ctypes.POINTER(ctypes.c_int64),
                                         ctypes.POINTER(ctypes.c_double)]),
}


def load(path: str = LIB_PATH):
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError("%s is not built; run `python -m paper_2607_04310_b300.build` "
                               "(there is no CPU fallback)" % path)
        lib = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def exported_symbols():
    return list(_SIGS)


def last_error() -> str:
    return load().psdf_last_error().decode()


def _check(rc: int) -> None:
    if rc != PSDF_OK:
        raise PsdfError(rc, last_error())


def _ptr(t) -> Optional[int]:
    """Device/host address of a torch tensor or numpy array (None -> NULL)."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def _stream(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def make_params(eps_seg=0.0, eps_axis=0.0, eps_sat=0.0, eta=0.0) -> Params:
    return Params(eps_seg, eps_axis, eps_sat, eta)


# --------------------------------------------------------------------------
# scene
# --------------------------------------------------------------------------
class Scene:
    """Owns a psdf_scene (device copy of the edge set and its precompute)."""

    def __init__(self, handle: int, n_rows: int, params: Params):
        self.handle = ctypes.c_void_p(handle)
        self.n_rows = n_rows
        self.params = params

    @classmethod
    def from_csr(cls, edges, offsets, tile_edges: int = 0, params: Optional[Params] = None,
                 stream=None) -> "Scene":
        e = np.ascontiguousarray(edges, dtype=np.float32).reshape(-1, 4)
        o = np.ascontiguousarray(offsets, dtype=np.int32)
        prm = params or Params()
        out = ctypes.c_void_p()
        _check(load().psdf_scene_create_csr(_ptr(e), _ptr(o), len(o) - 1, tile_edges,
                                            ctypes.byref(prm), _stream(stream),
                                            ctypes.byref(out)))
        return cls(out.value, e.shape[0], prm)

    @classmethod
    def from_padded(cls, A, B, S, tile_edges: int = 0, params: Optional[Params] = None,
                    stream=None) -> "Scene":
        A = np.ascontiguousarray(A, dtype=np.float32)
        B = np.ascontiguousarray(B, dtype=np.float32)
        S = np.ascontiguousarray(S, dtype=np.uint8)
        Mbar, mbar = S.shape
        prm = params or Params()
        out = ctypes.c_void_p()
        _check(load().psdf_scene_create_padded(_ptr(A), _ptr(B), _ptr(S), Mbar, mbar,
                                               tile_edges, ctypes.byref(prm), _stream(stream),
                                               ctypes.byref(out)))
        return cls(out.value, Mbar * mbar, prm)

    def info(self) -> SceneInfo:
        inf = SceneInfo()
        _check(load().psdf_scene_get_info(self.handle, ctypes.byref(inf)))
        return inf

    def cull_grid(self) -> CullGridInfo:
        inf = CullGridInfo()
        _check(load().psdf_scene_cull_grid(self.handle, ctypes.byref(inf)))
        return inf

    def cull_grid_lists(self):
        """(offsets [nx*ny+1], tiles [entries], tile AABBs [T,4]) on the host."""
        g = self.cull_grid()
        T = self.info().n_tiles
        off = np.zeros(max(g.nx * g.ny + 1, 1), dtype=np.int32)
        tl = np.zeros(max(int(g.entries), 1), dtype=np.int32)
        ab = np.zeros((max(T, 1), 4), dtype=np.float32)
        _check(load().psdf_scene_cull_grid_copy(self.handle, off.ctypes.data, tl.ctypes.data,
                                                ab.ctypes.data))
        return off[:g.nx * g.ny + 1], tl[:int(g.entries)], ab[:T]

    def close(self) -> None:
        if self.handle and self.handle.value:
            load().psdf_scene_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# --------------------------------------------------------------------------
# C entry points, same names (device buffers = torch CUDA tensors)
# --------------------------------------------------------------------------
def psdf_workspace_bytes(P: int) -> int:
    return int(load().psdf_workspace_bytes(int(P)))


def psdf_workspace_status(workspace, stream=None) -> int:
    return int(load().psdf_workspace_status(_ptr(workspace), _stream(stream)))


def psdf_eval(footprint: np.ndarray, scene: Scene, poses, params: Params, phi, active,
              workspace, stream=None) -> None:
    fp = np.ascontiguousarray(footprint, dtype=np.float32)
    _check(load().psdf_eval(_ptr(fp), fp.shape[0], scene.handle, _ptr(poses), poses.shape[0],
                            ctypes.byref(params), _ptr(phi), _ptr(active), _ptr(workspace),
                            workspace.numel(), _stream(stream)))


def psdf_eval_grad(footprint: np.ndarray, scene: Scene, poses, params: Params, phi, dphi,
                   active, workspace, stream=None) -> None:
    fp = np.ascontiguousarray(footprint, dtype=np.float32)
    _check(load().psdf_eval_grad(_ptr(fp), fp.shape[0], scene.handle, _ptr(poses),
                                 poses.shape[0], ctypes.byref(params), _ptr(phi), _ptr(dphi),
                                 _ptr(active), _ptr(workspace), workspace.numel(),
                                 _stream(stream)))


def psdf_stage_params(footprint: np.ndarray, scene: Scene, poses, params: Params, d_min: float,
                      stage, active, workspace, stream=None) -> None:
    fp = np.ascontiguousarray(footprint, dtype=np.float32)
    _check(load().psdf_stage_params(_ptr(fp), fp.shape[0], scene.handle, _ptr(poses),
                                    poses.shape[0], ctypes.byref(params), float(d_min),
                                    _ptr(stage), _ptr(active), _ptr(workspace), workspace.numel(),
                                    _stream(stream)))


def psdf_eval_keys(footprint: np.ndarray, scene: Scene, poses, params: Params, row_offset: int,
                   keys, workspace, stream=None) -> None:
    """Per-pose 64-bit keys of a scene part (keys: int64 tensor holding the
    unsigned bits), ranks offset by row_offset."""
    fp = np.ascontiguousarray(footprint, dtype=np.float32)
    _check(load().psdf_eval_keys(_ptr(fp), fp.shape[0], scene.handle, _ptr(poses),
                                 poses.shape[0], ctypes.byref(params), int(row_offset),
                                 _ptr(keys), _ptr(workspace), workspace.numel(),
                                 _stream(stream)))


def psdf_merge_keys(a, b, stream=None) -> None:
    """b = min(a, b) over the unsigned key bits."""
    _check(load().psdf_merge_keys(_ptr(a), _ptr(b), b.numel(), _stream(stream)))


def psdf_finish_keys(footprint: np.ndarray, scene: Scene, poses, params: Params,
                     row_offset: int, own_empty: bool, keys, phi, dphi, active,
                     stream=None) -> None:
    fp = np.ascontiguousarray(footprint, dtype=np.float32)
    _check(load().psdf_finish_keys(_ptr(fp), fp.shape[0], scene.handle, _ptr(poses),
                                   poses.shape[0], ctypes.byref(params), int(row_offset),
                                   1 if own_empty else 0, _ptr(keys), _ptr(phi), _ptr(dphi),
                                   _ptr(active), _stream(stream)))


def psdf_backward(footprint: np.ndarray, scene: Scene, poses, params: Params, active, grad_phi,
                  grad_pose, grad_edges, stream=None) -> None:
    fp = np.ascontiguousarray(footprint, dtype=np.float32)
    _check(load().psdf_backward(_ptr(fp), fp.shape[0], scene.handle, _ptr(poses),
                                poses.shape[0], ctypes.byref(params), _ptr(active),
                                _ptr(grad_phi), _ptr(grad_pose), _ptr(grad_edges),
                                _stream(stream)))


# floats per pose of a saved backward record (psdf_eval_grad_save,
# psdf_eval_culled_save -> psdf_backward_saved)
SAVED_FLOATS = 16


def psdf_eval_grad_save(footprint: np.ndarray, scene: Scene, poses, params: Params, phi, dphi,
                        active, saved, workspace, stream=None) -> None:
    fp = np.ascontiguousarray(footprint, dtype=np.float32)
    _check(load().psdf_eval_grad_save(_ptr(fp), fp.shape[0], scene.handle, _ptr(poses),
                                      poses.shape[0], ctypes.byref(params), _ptr(phi),
                                      _ptr(dphi), _ptr(active), _ptr(saved), _ptr(workspace),
                                      workspace.numel(), _stream(stream)))


def psdf_backward_saved(scene: Scene, saved, grad_phi, grad_pose, grad_edges,
                        stream=None) -> None:
    _check(load().psdf_backward_saved(scene.handle, _ptr(saved), saved.shape[0],
                                      _ptr(grad_phi), _ptr(grad_pose), _ptr(grad_edges),
                                      _stream(stream)))


NOALLOC_MAX_POSES = 262144
PROPOSE_BOUND = 1
PROPOSE_MLP = 2
PROPOSE_CIRCLES = 3


class CullOpts(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("k", ctypes.c_int32)]


class CullStats(ctypes.Structure):
    _fields_ = [("evaluated_obstacles", ctypes.c_int64), ("evaluated_edges", ctypes.c_int64),
                ("proposed_items", ctypes.c_int64), ("fallback_items", ctypes.c_int64),
                ("fallback_poses", ctypes.c_int64), ("bound_evaluations", ctypes.c_int64),
                ("circle_evaluations", ctypes.c_int64)]


class Mlp:
    """Owns a psdf_mlp (tile-proposal network weights on the device)."""

    def __init__(self, W1, w2, b2: float):
        W1 = np.ascontiguousarray(W1, dtype=np.float32).reshape(64, 16)
        w2 = np.ascontiguousarray(w2, dtype=np.float32).reshape(64)
        out = ctypes.c_void_p()
        _check(load().psdf_mlp_create(_ptr(W1), _ptr(w2), float(b2), ctypes.byref(out)))
        self.handle = out
        self.W1, self.w2, self.b2 = W1, w2, float(b2)

    def close(self):
        if self.handle and self.handle.value:
            load().psdf_mlp_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def psdf_tile_features(footprint, scene: Scene, poses, out, stream=None) -> None:
    fp = np.ascontiguousarray(footprint, dtype=np.float32)
    _check(load().psdf_tile_features(_ptr(fp), fp.shape[0], scene.handle, _ptr(poses),
                                     poses.shape[0], _ptr(out), _stream(stream)))


def psdf_mlp_scores(mlp: Mlp, footprint, scene: Scene, poses, out, stream=None) -> None:
    fp = np.ascontiguousarray(footprint, dtype=np.float32)
    _check(load().psdf_mlp_scores(mlp.handle, _ptr(fp), fp.shape[0], scene.handle, _ptr(poses),
                                  poses.shape[0], _ptr(out), _stream(stream)))


def psdf_tile_values(footprint, scene: Scene, poses, params: Params, out, stream=None) -> None:
    fp = np.ascontiguousarray(footprint, dtype=np.float32)
    _check(load().psdf_tile_values(_ptr(fp), fp.shape[0], scene.handle, _ptr(poses),
                                   poses.shape[0], ctypes.byref(params), _ptr(out),
                                   _stream(stream)))


def psdf_tile_lower_bounds(footprint, scene: Scene, poses, out, stream=None) -> None:
    fp = np.ascontiguousarray(footprint, dtype=np.float32)
    _check(load().psdf_tile_lower_bounds(_ptr(fp), fp.shape[0], scene.handle, _ptr(poses),
                                         poses.shape[0], _ptr(out), _stream(stream)))


def psdf_cull_workspace_bytes(P: int, scene: Scene) -> int:
    return int(load().psdf_cull_workspace_bytes(int(P), scene.handle))


def psdf_eval_culled(footprint, scene: Scene, mlp: Optional[Mlp], opts: CullOpts, poses,
                     params: Params, phi, dphi, active, workspace, stream=None) -> None:
    fp = np.ascontiguousarray(footprint, dtype=np.float32)
    _check(load().psdf_eval_culled(_ptr(fp), fp.shape[0], scene.handle,
                                   mlp.handle if mlp is not None else None, ctypes.byref(opts),
                                   _ptr(poses), poses.shape[0], ctypes.byref(params), _ptr(phi),
                                   _ptr(dphi), _ptr(active), _ptr(workspace), workspace.numel(),
                                   _stream(stream)))


def psdf_eval_culled_save(footprint, scene: Scene, mlp: Optional[Mlp], opts: CullOpts, poses,
                          params: Params, phi, dphi, active, saved, workspace,
                          stream=None) -> None:
    fp = np.ascontiguousarray(footprint, dtype=np.float32)
    _check(load().psdf_eval_culled_save(_ptr(fp), fp.shape[0], scene.handle,
                                        mlp.handle if mlp is not None else None,
                                        ctypes.byref(opts), _ptr(poses), poses.shape[0],
                                        ctypes.byref(params), _ptr(phi), _ptr(dphi),
                                        _ptr(active), _ptr(saved), _ptr(workspace),
                                        workspace.numel(), _stream(stream)))


def psdf_cull_stats_read(workspace, stream=None) -> CullStats:
    st = CullStats()
    _check(load().psdf_cull_stats_read(_ptr(workspace), _stream(stream), ctypes.byref(st)))
    return st


def eval_culled(scene: Scene, footprint, poses, mlp: Optional[Mlp] = None, k: int = 2,
                params: Optional[Params] = None, grad: bool = True, ws=None, stream=None,
                mode: Optional[int] = None):
    """(phi, dphi or None, active, workspace) through the exact tile cull;
    mode defaults to PROPOSE_MLP with a network, else PROPOSE_BOUND."""
    import torch
    prm = params or scene.params
    P = poses.shape[0]
    if mode is None:
        mode = PROPOSE_MLP if mlp is not None else PROPOSE_BOUND
    opts = CullOpts(mode, k)
    phi = torch.empty(P, dtype=torch.float32, device=poses.device)
    act = torch.empty(P, dtype=torch.int32, device=poses.device)
    dphi = torch.empty((P, 3), dtype=torch.float32, device=poses.device) if grad else None
    if ws is None:
        ws = torch.empty(psdf_cull_workspace_bytes(P, scene), dtype=torch.uint8,
                         device=poses.device)
    psdf_eval_culled(footprint, scene, mlp, opts, poses, prm, phi, dphi, act, ws, stream)
    return phi, dphi, act, ws


def psdf_eval_grad_noalloc(footprint: np.ndarray, scene: Scene, poses, params: Params, phi,
                           dphi, active, stream=None) -> int:
    """psdf_eval_grad with the library's built-in scratch (no allocation).
    Returns the status code (0 = PSDF_OK) without raising."""
    fp = np.ascontiguousarray(footprint, dtype=np.float32)
    return int(load().psdf_eval_grad_noalloc(_ptr(fp), fp.shape[0], scene.handle, _ptr(poses),
                                             poses.shape[0], ctypes.byref(params), _ptr(phi),
                                             _ptr(dphi), _ptr(active), _stream(stream)))


def psdf_measure_fp32_peak(paired: bool, iters: int = 200000, reps: int = 5,
                           stream=None) -> Tuple[float, float]:
    """(TFLOP/s, ms) of the library's FP32 FMA microbenchmark (best of reps)."""
    tf = ctypes.c_double()
    ms = ctypes.c_double()
    _check(load().psdf_measure_fp32_peak(1 if paired else 0, int(iters), int(reps),
                                         ctypes.byref(tf), ctypes.byref(ms), _stream(stream)))
    return float(tf.value), float(ms.value)


DEFAULT_WAIT_LIMIT = 1 << 22


def psdf_debug_set_wait_limit(polls: int) -> int:
    """Polls every bounded device-side wait makes before it gives up, for
    launches issued afterwards (0 = give up at once); returns the previous
    limit."""
    prev = ctypes.c_uint32()
    _check(load().psdf_debug_set_wait_limit(int(polls), ctypes.byref(prev)))
    return int(prev.value)


def psdf_profile_enable(on: bool) -> None:
    _check(load().psdf_profile_enable(1 if on else 0))


def psdf_profile_reset() -> None:
    _check(load().psdf_profile_reset())


def psdf_profile_read(kernel: str) -> Tuple[int, float]:
    """(launches, total device milliseconds) of a traced kernel."""
    n = ctypes.c_int64()
    ms = ctypes.c_double()
    _check(load().psdf_profile_read(kernel.encode(), ctypes.byref(n), ctypes.byref(ms)))
    return int(n.value), float(ms.value)


# --------------------------------------------------------------------------
# allocation helpers (torch owns the memory; the library computes)
# --------------------------------------------------------------------------
def workspace(P: int, device="cuda"):
    import torch
    return torch.empty(psdf_workspace_bytes(P), dtype=torch.uint8, device=device)


def eval_grad(scene: Scene, footprint: np.ndarray, poses, params: Optional[Params] = None,
              grad: bool = True, ws=None, stream=None) -> Tuple:
    """(phi [P], dphi [P,3] or None, active [P] int32 view of the uint32 ids)."""
    import torch
    prm = params or scene.params
    P = poses.shape[0]
    phi = torch.empty(P, dtype=torch.float32, device=poses.device)
    active = torch.empty(P, dtype=torch.int32, device=poses.device)
    ws = workspace(P, poses.device) if ws is None else ws
    if grad:
        dphi = torch.empty((P, 3), dtype=torch.float32, device=poses.device)
        psdf_eval_grad(footprint, scene, poses, prm, phi, dphi, active, ws, stream)
        return phi, dphi, active
    psdf_eval(footprint, scene, poses, prm, phi, active, ws, stream)
    return phi, None, active


def pair_ids(active) -> np.ndarray:
    """uint32 pair ids from the int32 tensor the helpers return."""
    a = active.detach().cpu().numpy() if hasattr(active, "detach") else np.asarray(active)
    return a.view(np.uint32) if a.dtype == np.int32 else a.astype(np.uint32)


# --------------------------------------------------------------------------
# batched plan
# --------------------------------------------------------------------------
class Plan:
    """Owns a psdf_plan: many instances (footprint, own edge set, run of poses)
    evaluated by one persistent launch.  `instances` is a sequence of
    (footprint [m][2], edges [E][4], offsets [M+1], n_poses)."""

    def __init__(self, instances, tile_edges: int = 0, params: Optional[Params] = None,
                 stream=None):
        fps, fpo, edges, obs_off, inst_obs, pose_off = [], [0], [], [0], [0], [0]
        row = 0
        for fp, e, off, n in instances:
            fp = np.asarray(fp, dtype=np.float32).reshape(-1, 2)
            e = np.asarray(e, dtype=np.float32).reshape(-1, 4)
            off = np.asarray(off, dtype=np.int64)
            fps.append(fp)
            fpo.append(fpo[-1] + fp.shape[0])
            edges.append(e)
            obs_off.extend((row + off[1:]).tolist())
            inst_obs.append(inst_obs[-1] + len(off) - 1)
            pose_off.append(pose_off[-1] + int(n))
            row += e.shape[0]
        self.footprints = np.ascontiguousarray(np.concatenate(fps) if fps else
                                               np.zeros((0, 2), np.float32))
        self.fp_offsets = np.asarray(fpo, dtype=np.int32)
        self.edges = np.ascontiguousarray(np.concatenate(edges) if edges else
                                          np.zeros((0, 4), np.float32))
        self.obs_offsets = np.asarray(obs_off, dtype=np.int32)
        self.inst_obs = np.asarray(inst_obs, dtype=np.int32)
        self.pose_offsets = np.asarray(pose_off, dtype=np.int64)
        self.row_offsets = np.concatenate([[0], np.cumsum([e.shape[0] for e in edges])]).astype(
            np.int64) if edges else np.zeros(1, np.int64)
        self.params = params or Params()
        out = ctypes.c_void_p()
        _check(load().psdf_plan_create(len(instances), _ptr(self.footprints),
                                       _ptr(self.fp_offsets), _ptr(self.edges),
                                       _ptr(self.obs_offsets), _ptr(self.inst_obs),
                                       _ptr(self.pose_offsets), tile_edges,
                                       ctypes.byref(self.params), _stream(stream),
                                       ctypes.byref(out)))
        self.handle = ctypes.c_void_p(out.value)

    @property
    def n_poses(self) -> int:
        return int(self.pose_offsets[-1])

    def info(self) -> PlanInfo:
        inf = PlanInfo()
        _check(load().psdf_plan_get_info(self.handle, ctypes.byref(inf)))
        return inf

    def close(self) -> None:
        if self.handle and self.handle.value:
            load().psdf_plan_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def psdf_plan_set_config(plan: Plan, threads: int, tiles_per_item: int, stream=None) -> None:
    cfg = PlanConfig(threads, tiles_per_item)
    _check(load().psdf_plan_set_config(plan.handle, ctypes.byref(cfg), _stream(stream)))


def psdf_plan_autotune(plan: Plan, poses, reps: int = 3, stream=None) -> Tuple[PlanConfig, bool]:
    cfg = PlanConfig()
    hit = ctypes.c_int32(0)
    _check(load().psdf_plan_autotune(plan.handle, _ptr(poses), reps, _stream(stream),
                                     ctypes.byref(cfg), ctypes.byref(hit)))
    return cfg, bool(hit.value)


def psdf_eval_batched(plan: Plan, poses, phi, dphi=None, active=None, stream=None) -> None:
    _check(load().psdf_eval_batched(plan.handle, _ptr(poses), _ptr(phi), _ptr(dphi),
                                    _ptr(active), _stream(stream)))


def psdf_stage_params_batched(plan: Plan, poses, d_min: float, stage, active=None,
                              stream=None) -> None:
    _check(load().psdf_stage_params_batched(plan.handle, _ptr(poses), float(d_min), _ptr(stage),
                                            _ptr(active), _stream(stream)))


def psdf_plan_debug_read() -> Tuple[int, bool]:
    """(first recorded index violation, whether this is a debug build)."""
    v = ctypes.c_uint64(0)
    en = ctypes.c_int32(0)
    _check(load().psdf_plan_debug_read(ctypes.byref(v), ctypes.byref(en)))
    return int(v.value), bool(en.value)


def psdf_plan_status(plan: Plan, stream=None) -> int:
    return int(load().psdf_plan_status(plan.handle, _stream(stream)))


def psdf_backward_batched(plan: Plan, poses, active, grad_phi, grad_pose=None, grad_edges=None,
                          stream=None) -> None:
    _check(load().psdf_backward_batched(plan.handle, _ptr(poses), _ptr(active), _ptr(grad_phi),
                                        _ptr(grad_pose), _ptr(grad_edges), _stream(stream)))


def eval_batched(plan: Plan, poses, stream=None):
    """phi, dphi, active for every pose of the plan (allocates the outputs)."""
    import torch
    P = plan.n_poses
    dev = poses.device
    phi = torch.empty(P, device=dev)
    dphi = torch.empty((P, 3), device=dev)
    act = torch.empty(P, dtype=torch.int32, device=dev)
    psdf_eval_batched(plan, poses, phi, dphi, act, stream)
    return phi, dphi, act
