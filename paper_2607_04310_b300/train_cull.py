"""Training of the tile-proposal network (the learned part of the exact cull).

    python -m paper_2607_04310_b300.train_cull --scenes 10000 --epochs 3 \
        --out paper_2607_04310_b300/data/tile_mlp.json

Data: seeded training scenes (1,024 random-yaw rectangles = 16 tiles of 256
edges at the dense-clutter density, 64 uniform poses; `scenegen.training_scene`).
For every (pose, tile) the inputs come from psdf_tile_features and the label
from psdf_tile_values (the exact per-tile minimum signed distance computed by
the CUDA kernels), clamped to [-0.5, 5] m.  Training runs in the library's own
kernels (psdf_trainer_*: forward, fixed-order gradient reduction, Adam).
Checkpoints hold the parameters, both Adam moments, the step and the epoch in
a flat binary with a JSON header; resuming from one reproduces the
uninterrupted run bit for bit.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import math
import os
import struct
import time
from typing import Optional, Tuple

import numpy as np

from . import psdf
from . import scenegen as sg

N_PARAMS = 1089
TARGET_LO, TARGET_HI = -0.5, 5.0
CKPT_FORMAT = "psdf-tile-mlp-checkpoint-v1"
WEIGHTS_FORMAT = "psdf-tile-mlp-weights-v1"
HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_WEIGHTS = os.path.join(HERE, "data", "tile_mlp.json")            # STR tiles
MORTON_WEIGHTS = os.path.join(HERE, "data", "tile_mlp_morton.json")      # Morton tiles
TILE_MORTON = 0x10000  # PSDF_TILE_MORTON


def init_weights(seed: int) -> Tuple[np.ndarray, np.ndarray, float]:
    """He-normal hidden layer (bias = column 15 starts at 0), small output."""
    g = np.random.default_rng(seed)
    W1 = g.normal(scale=math.sqrt(2.0 / 16), size=(64, 16)).astype(np.float32)
    W1[:, 15] = 0.0
    w2 = g.normal(scale=math.sqrt(1.0 / 64), size=64).astype(np.float32)
    return W1, w2, 1.0


def split_params(p: np.ndarray):
    p = np.asarray(p, dtype=np.float32)
    return p[:1024].reshape(64, 16).copy(), p[1024:1088].copy(), float(p[1088])


class Trainer:
    """Owns a psdf_trainer (FP32 parameters and Adam state on the device)."""

    def __init__(self, W1, w2, b2: float, lr: float = 2e-3):
        W1 = np.ascontiguousarray(W1, dtype=np.float32).reshape(64, 16)
        w2 = np.ascontiguousarray(w2, dtype=np.float32).reshape(64)
        out = ctypes.c_void_p()
        psdf._check(psdf.load().psdf_trainer_create(W1.ctypes.data, w2.ctypes.data, float(b2),
                                                    float(lr), ctypes.byref(out)))
        self.handle = out

    def close(self):
        if self.handle and self.handle.value:
            psdf.load().psdf_trainer_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_lr(self, lr: float):
        psdf._check(psdf.load().psdf_trainer_set_lr(self.handle, float(lr)))

    def grad(self, X, y, N: Optional[int] = None):
        import torch
        N = X.shape[0] if N is None else N
        g = torch.empty(N_PARAMS, dtype=torch.float32, device=X.device)
        loss = torch.empty(1, dtype=torch.float32, device=X.device)
        psdf._check(psdf.load().psdf_trainer_grad(self.handle, X.data_ptr(), y.data_ptr(), N,
                                                  g.data_ptr(), loss.data_ptr(),
                                                  psdf._stream(None)))
        return g, loss

    def step(self, X, y, idx, N: int, loss=None):
        psdf._check(psdf.load().psdf_trainer_step(self.handle, X.data_ptr(), y.data_ptr(),
                                                  idx.data_ptr() if idx is not None else None,
                                                  N, loss.data_ptr() if loss is not None else None,
                                                  psdf._stream(None)))

    def get_state(self):
        p = np.empty(N_PARAMS, np.float32)
        m = np.empty(N_PARAMS, np.float32)
        v = np.empty(N_PARAMS, np.float32)
        st = ctypes.c_int64()
        psdf._check(psdf.load().psdf_trainer_get(self.handle, p.ctypes.data, m.ctypes.data,
                                                 v.ctypes.data, ctypes.byref(st)))
        return {"params": p, "m": m, "v": v, "step": int(st.value)}

    def set_state(self, state):
        p = np.ascontiguousarray(state["params"], np.float32)
        m = np.ascontiguousarray(state["m"], np.float32)
        v = np.ascontiguousarray(state["v"], np.float32)
        psdf._check(psdf.load().psdf_trainer_set(self.handle, p.ctypes.data, m.ctypes.data,
                                                 v.ctypes.data, int(state["step"])))


# --------------------------------------------------------------------------
# checkpoints and weights files
# --------------------------------------------------------------------------
def save_checkpoint(path: str, trainer: Trainer, meta: dict) -> None:
    st = trainer.get_state()
    header = dict(meta)
    header.update({"format": CKPT_FORMAT, "params": N_PARAMS, "step": st["step"],
                   "arrays": ["params", "m", "v"], "dtype": "float32-le"})
    hb = json.dumps(header, sort_keys=True).encode()
    tmp = path + ".tmp"
    with open(tmp, "wb") as f:
        f.write(struct.pack("<Q", len(hb)))
        f.write(hb)
        for name in ("params", "m", "v"):
            f.write(np.asarray(st[name], dtype="<f4").tobytes())
    os.replace(tmp, path)


def load_checkpoint(path: str):
    with open(path, "rb") as f:
        n = struct.unpack("<Q", f.read(8))[0]
        header = json.loads(f.read(n).decode())
        if header.get("format") != CKPT_FORMAT:
            raise ValueError("not a tile-MLP checkpoint: %s" % path)
        arrs = {}
        for name in header["arrays"]:
            arrs[name] = np.frombuffer(f.read(4 * N_PARAMS), dtype="<f4").astype(np.float32)
    state = {"params": arrs["params"], "m": arrs["m"], "v": arrs["v"], "step": header["step"]}
    return state, header


def save_weights(path: str, W1, w2, b2: float, meta: dict) -> None:
    """Weights rounded to FP16 (what the inference kernel uses), as JSON text."""
    h = lambda a: np.asarray(a, dtype=np.float32).astype(np.float16).astype(np.float32)
    doc = dict(meta)
    doc.update({"format": WEIGHTS_FORMAT, "W1": h(W1).tolist(), "w2": h(w2).tolist(),
                "b2": float(b2)})
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    with open(path, "w") as f:
        json.dump(doc, f, indent=0, sort_keys=True)


def load_weights(path: str = DEFAULT_WEIGHTS):
    with open(path) as f:
        doc = json.load(f)
    if doc.get("format") != WEIGHTS_FORMAT:
        raise ValueError("not a tile-MLP weights file: %s" % path)
    return (np.asarray(doc["W1"], np.float32), np.asarray(doc["w2"], np.float32),
            float(doc["b2"]), doc)


# --------------------------------------------------------------------------
# data
# --------------------------------------------------------------------------
def build_dataset(n_scenes: int, first: int = 0, device="cuda", log=None, tile_flags: int = 0):
    """(X [R, 16], y [R]) on the device for training scenes first..first+n-1
    (tile_flags: 0 = sort-tile-recursive tiles, TILE_MORTON = Morton tiles)."""
    import torch
    Xs, ys = [], []
    t0 = time.time()
    for i in range(n_scenes):
        w = sg.training_scene(first + i)
        scene = psdf.Scene.from_csr(w.edges, w.offsets, tile_edges=tile_flags)
        T = scene.info().n_tiles
        poses = torch.as_tensor(w.poses, device=device)
        feats = torch.empty((w.P, T, 16), dtype=torch.float32, device=device)
        vals = torch.empty((w.P, T), dtype=torch.float32, device=device)
        psdf.psdf_tile_features(w.footprint, scene, poses, feats)
        psdf.psdf_tile_values(w.footprint, scene, poses, scene.params, vals)
        Xs.append(feats.reshape(-1, 16))
        ys.append(vals.reshape(-1).clamp(TARGET_LO, TARGET_HI))
        scene.close()
        if log and (i + 1) % 1000 == 0:
            log("dataset: %d / %d scenes, %.1f s" % (i + 1, n_scenes, time.time() - t0))
    X = torch.cat(Xs).contiguous()
    y = torch.cat(ys).contiguous()
    torch.cuda.synchronize()
    return X, y


def epoch_permutation(seed: int, epoch: int, rows: int) -> np.ndarray:
    return np.random.default_rng([seed, epoch]).permutation(rows).astype(np.int32)


def lr_at(epoch: int, epochs: int, lr: float) -> float:
    return lr if epoch < epochs - 1 else lr * 0.1


def train(X, y, epochs: int, batch: int, lr: float, seed: int, trainer: Optional[Trainer] = None,
          start_epoch: int = 0, checkpoint: Optional[str] = None, log=None,
          stop_after_epoch: Optional[int] = None) -> Trainer:
    import torch
    rows = X.shape[0]
    if trainer is None:
        W1, w2, b2 = init_weights(seed)
        trainer = Trainer(W1, w2, b2, lr)
    steps = rows // batch
    loss = torch.empty(1, device=X.device)
    for e in range(start_epoch, epochs):
        trainer.set_lr(lr_at(e, epochs, lr))
        perm = torch.as_tensor(epoch_permutation(seed, e, rows), device=X.device)
        acc = 0.0
        for i in range(steps):
            trainer.step(X, y, perm[i * batch:(i + 1) * batch], batch, loss)
            if i % 50 == 0:
                acc = float(loss.item())
        if log:
            log("epoch %d: loss %.5f (last sampled), %d steps" % (e, acc, steps))
        if checkpoint:
            save_checkpoint(checkpoint, trainer, {"epoch_done": e, "epochs": epochs,
                                                  "batch": batch, "lr": lr, "seed": seed,
                                                  "rows": rows})
        if stop_after_epoch is not None and e >= stop_after_epoch:
            break
    return trainer


def resume(path: str, X, y, log=None) -> Trainer:
    state, meta = load_checkpoint(path)
    W1, w2, b2 = split_params(state["params"])
    tr = Trainer(W1, w2, b2, meta["lr"])
    tr.set_state(state)
    return train(X, y, meta["epochs"], meta["batch"], meta["lr"], meta["seed"], trainer=tr,
                 start_epoch=meta["epoch_done"] + 1, log=log)


# --------------------------------------------------------------------------
# evaluation: how often the proposal's first tile holds the nearest obstacle
# --------------------------------------------------------------------------
def evaluate(W1, w2, b2, n_scenes: int = 100, first: int = 20000, device="cuda",
             tile_flags: int = 0):
    import torch
    mlp = psdf.Mlp(W1, w2, b2)
    hit_mlp = hit_lb = total = 0
    for i in range(n_scenes):
        w = sg.training_scene(first + i)
        scene = psdf.Scene.from_csr(w.edges, w.offsets, tile_edges=tile_flags)
        T = scene.info().n_tiles
        poses = torch.as_tensor(w.poses, device=device)
        vals = torch.empty((w.P, T), device=device)
        sc = torch.empty((w.P, T), device=device)
        lb = torch.empty((w.P, T), device=device)
        psdf.psdf_tile_values(w.footprint, scene, poses, scene.params, vals)
        psdf.psdf_mlp_scores(mlp, w.footprint, scene, poses, sc)
        psdf.psdf_tile_lower_bounds(w.footprint, scene, poses, lb)
        best = vals.argmin(dim=1)
        hit_mlp += int((sc.argmin(dim=1) == best).sum())
        hit_lb += int((lb.argmin(dim=1) == best).sum())
        total += w.P
        scene.close()
    return {"top1_mlp": hit_mlp / total, "top1_bound": hit_lb / total, "poses": total}


def main():
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--scenes", type=int, default=10000)
    ap.add_argument("--epochs", type=int, default=3)
    ap.add_argument("--batch", type=int, default=16384)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--out", default=DEFAULT_WEIGHTS)
    ap.add_argument("--checkpoint", default=None)
    ap.add_argument("--eval-scenes", type=int, default=200)
    ap.add_argument("--morton", action="store_true", help="train for Morton-packed tiles")
    a = ap.parse_args()
    flags = TILE_MORTON if a.morton else 0
    torch.cuda.init()
    log = lambda s: print(s, flush=True)
    t0 = time.time()
    X, y = build_dataset(a.scenes, log=log, tile_flags=flags)
    log("dataset: %d rows in %.1f s" % (X.shape[0], time.time() - t0))
    t1 = time.time()
    tr = train(X, y, a.epochs, a.batch, a.lr, a.seed, checkpoint=a.checkpoint, log=log)
    torch.cuda.synchronize()
    log("training: %.1f s" % (time.time() - t1))
    W1, w2, b2 = split_params(tr.get_state()["params"])
    ev = evaluate(W1, w2, b2, a.eval_scenes, tile_flags=flags)
    log("held-out: %s" % json.dumps(ev))
    save_weights(a.out, W1, w2, b2, {"scenes": a.scenes, "epochs": a.epochs, "batch": a.batch,
                                     "lr": a.lr, "seed": a.seed, "heldout": ev,
                                     "tiles": "morton" if a.morton else "sort-tile-recursive",
                                     "target_clamp": [TARGET_LO, TARGET_HI]})
    log("wrote %s" % a.out)


if __name__ == "__main__":
    main()
