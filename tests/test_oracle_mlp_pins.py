"""Pins of the tile-proposal network reference (oracle/mlp.py) on the CPU.

The network is not from the paper: it is the learned proposal of the exact
tile cull, defined by the library's header (inputs), the tensor-core forward
(FP16 inputs, weights and ReLU activations, FP32 accumulation) and the
training loss (mean squared error of s = w2 . relu(W1 x) + b2).  These tests
fix the reference against values worked out by hand from those definitions
and against central finite differences of its loss, and plant plausible
mistakes in a copy of the module to show that every one is caught.
"""
from __future__ import annotations

import inspect
import math
import types

import numpy as np
import pytest

from oracle import mlp as omlp


# ---------------------------------------------------------------------------
# pins, each taking the module under test
# ---------------------------------------------------------------------------
def pin_loss_hand(m) -> bool:
    """Two rows, two live hidden units, worked by hand.

    W1 row 0 = e0 (a0 = x0), row 1 = -e1 (a1 = -x1), w2 = (2, 3), b2 = 0.5.
    Row A: x = (1, 2), y = 1  -> a = (1, -2), h = (1, 0), s = 2.5,  r = 1.5
    Row B: x = (-1, -4), y = 0 -> a = (-1, 4), h = (0, 4), s = 12.5, r = 12.5
    loss = (1.5^2 + 12.5^2) / 2 = 79.25; ds = 2 r / N = (1.5, 12.5)
    dw2 = h^T ds = (1.5, 50); db2 = 14
    dh = ds w2^T masked by a > 0: row A (3, 0), row B (0, 37.5)
    dW1 row 0 = 3 x_A = (3, 6); row 1 = 37.5 x_B = (-37.5, -150).
    """
    X = np.zeros((2, 16))
    X[0, :2] = (1, 2)
    X[1, :2] = (-1, -4)
    y = np.array([1.0, 0.0])
    W1 = np.zeros((64, 16))
    W1[0, 0] = 1.0
    W1[1, 1] = -1.0
    w2 = np.zeros(64)
    w2[:2] = (2.0, 3.0)
    loss, dW1, dw2, db2 = m.loss_and_grads(X, y, W1, w2, 0.5)
    eW1 = np.zeros((64, 16))
    eW1[0, :2] = (3, 6)
    eW1[1, :2] = (-37.5, -150)
    ew2 = np.zeros(64)
    ew2[:2] = (1.5, 50)
    return (loss == 79.25 and db2 == 14.0 and np.array_equal(dw2, ew2) and
            np.array_equal(dW1, eW1))


def _fd_case(seed):
    g = np.random.default_rng(seed)
    N = 24
    X = g.normal(size=(N, 16))
    X[:, 15] = 1.0
    y = g.normal(size=N)
    W1, w2, b2 = m_init(seed)
    b2 = 0.3
    # push a few units negative on most rows, so that the ReLU mask matters
    W1[:8, 15] -= 2.5
    return X, y, W1, w2, b2


def m_init(seed):
    g = np.random.default_rng(1000 + seed)
    return g.normal(scale=0.5, size=(64, 16)), g.normal(scale=0.5, size=64), 0.0


def pin_loss_fd(m, seed: int = 0, h: float = 1e-6) -> bool:
    """Every gradient component equals the central difference of the loss
    (FP64, step h) to 1e-6 of the largest component.  The case keeps every
    pre-activation farther than 1e-4 from the ReLU kink (so that the
    difference is smooth; a case that does not is a failure, never a pass)."""
    X, y, W1, w2, b2 = _fd_case(seed)
    a = X @ W1.T
    if np.min(np.abs(a)) < 1e-4:
        return False
    inactive = np.mean(a <= 0)
    if not 0.2 < inactive < 0.8:
        return False  # the case must exercise both branches of the mask
    loss, dW1, dw2, db2 = m.loss_and_grads(X, y, W1, w2, b2)

    def L(W1_, w2_, b2_):
        return m.loss_and_grads(X, y, W1_, w2_, b2_)[0]

    fd_W1 = np.zeros_like(W1)
    for i in range(64):
        for j in range(16):
            Wp = W1.copy(); Wp[i, j] += h
            Wm = W1.copy(); Wm[i, j] -= h
            fd_W1[i, j] = (L(Wp, w2, b2) - L(Wm, w2, b2)) / (2 * h)
    fd_w2 = np.zeros_like(w2)
    for i in range(64):
        wp = w2.copy(); wp[i] += h
        wm = w2.copy(); wm[i] -= h
        fd_w2[i] = (L(W1, wp, b2) - L(W1, wm, b2)) / (2 * h)
    fd_b2 = (L(W1, w2, b2 + h) - L(W1, w2, b2 - h)) / (2 * h)
    scale = max(np.abs(dW1).max(), np.abs(dw2).max(), abs(db2))
    tol = 1e-6 * scale + 1e-7
    return (np.abs(fd_W1 - dW1).max() <= tol and np.abs(fd_w2 - dw2).max() <= tol and
            abs(fd_b2 - db2) <= tol)


def pin_forward_hand(m) -> bool:
    """Inputs x0 = 0.1, x1 = 2; W1 row 0 = (3, 0), row 1 = (1, -1); w2 =
    (2, 5); b2 = 0.25.  FP16(0.1) = 1638 / 16384 = 0.0999755859375 (0.1 =
    1.6 * 2^-4, 1.6 * 1024 = 1638.4 rounds to 1638).  a0 = 3 * that =
    0.2999267578125 = 1.19970703125 * 2^-2, whose 10-bit mantissa
    0.19970703125 * 1024 = 204.5 ties to the even 204: FP16(a0) =
    1.19921875 / 4 = 0.2998046875.  a1 = 0.0999755859375 - 2 < 0 -> 0.
    s = 2 * 0.2998046875 + 0.25 = 0.849609375 exactly.  (Without the hidden
    rounding s would be 0.849853515625; without the input rounding,
    2 * FP16(0.3) + 0.25 = 0.85009765625.)"""
    X = np.zeros((1, 16))
    X[0, :2] = (0.1, 2.0)
    W1 = np.zeros((64, 16))
    W1[0, 0] = 3.0
    W1[1, 0], W1[1, 1] = 1.0, -1.0
    w2 = np.zeros(64)
    w2[:2] = (2.0, 5.0)
    s = m.forward_f16(X, W1, w2, 0.25)
    return s.shape == (1,) and s[0] == 0.849609375


def pin_features_hand(m) -> bool:
    """AABB [xmin, ymin, xmax, ymax] = [1, 2, 3, 5], footprint radius 0.36,
    a tile of 128 edges.  Corners in the header's order: (1,2) (3,2) (3,5)
    (1,5).

    Pose (0, 0, 0): local = world.  Features 0..7 = 0.1 (1, 2, 3, 2, 3, 5,
    1, 5); 8..11 = 0.1 (sqrt 5, sqrt 13, sqrt 34, sqrt 26); 12 = 0.1 sqrt 5
    (nearest AABB point (1, 2)); 13 = 0.36; 14 = 0.5; 15 = 1.

    Pose (0, 0, pi/2): local (x, y) = (dy, -dx), so the corners become (2,
    -1) (2, -3) (5, -3) (5, -1); distances unchanged.

    Pose (2, 3, 0) inside the AABB: local corners (-1, -1) (1, -1) (1, 2)
    (-1, 2); distances (sqrt 2, sqrt 2, sqrt 5, sqrt 5); AABB distance 0.

    Pose (-250, 2, 0): corner x offsets 251 and 253 clamp to 20 -> 2.0;
    distances above 30 clamp to 3.0; AABB distance 251 -> 3.0."""
    ab = np.array([[1.0, 2.0, 3.0, 5.0]])
    poses = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, math.pi / 2], [2.0, 3.0, 0.0],
                      [-250.0, 2.0, 0.0]])
    F = m.tile_features(ab, [128], poses, 0.36)
    if F.shape != (4, 1, 16):
        return False
    r5, r13, r34, r26, r2 = map(math.sqrt, (5, 13, 34, 26, 2))
    tail = [0.36, 0.5, 1.0]
    exp = [
        [0.1, 0.2, 0.3, 0.2, 0.3, 0.5, 0.1, 0.5, 0.1 * r5, 0.1 * r13, 0.1 * r34, 0.1 * r26,
         0.1 * r5] + tail,
        [0.2, -0.1, 0.2, -0.3, 0.5, -0.3, 0.5, -0.1, 0.1 * r5, 0.1 * r13, 0.1 * r34, 0.1 * r26,
         0.1 * r5] + tail,
        [-0.1, -0.1, 0.1, -0.1, 0.1, 0.2, -0.1, 0.2, 0.1 * r2, 0.1 * r2, 0.1 * math.sqrt(5),
         0.1 * math.sqrt(5), 0.0] + tail,
        [2.0, 0.0, 2.0, 0.0, 2.0, 0.3, 2.0, 0.3, 3.0, 3.0, 3.0, 3.0, 3.0] + tail,
    ]
    return bool(np.allclose(F[:, 0, :], np.array(exp), rtol=0, atol=1e-12))


PINS = {
    "loss_hand": pin_loss_hand,
    "loss_fd": pin_loss_fd,
    "forward_hand": pin_forward_hand,
    "features_hand": pin_features_hand,
}


# ---------------------------------------------------------------------------
# the reference passes its pins
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("name", sorted(PINS))
def test_mlp_reference_pin(name):
    assert PINS[name](omlp), name


@pytest.mark.parametrize("seed", [1, 2])
def test_mlp_loss_fd_more_seeds(seed):
    assert pin_loss_fd(omlp, seed=seed)


# ---------------------------------------------------------------------------
# planted mistakes in a copy of the module are caught
# ---------------------------------------------------------------------------
MUTATIONS = {
    "relu_mask_dropped": ("dh = np.outer(ds, w2) * (a > 0)", "dh = np.outer(ds, w2)"),
    "ds_halved": ("ds = 2.0 * r / N", "ds = r / N"),
    "corner_swapped": (
        "np.stack([ab[:, 2], ab[:, 1]], 1), np.stack([ab[:, 2], ab[:, 3]], 1), "
        "np.stack([ab[:, 0], ab[:, 3]], 1)",
        "np.stack([ab[:, 0], ab[:, 3]], 1), np.stack([ab[:, 2], ab[:, 3]], 1), "
        "np.stack([ab[:, 2], ab[:, 1]], 1)"),
    "hidden_not_rounded": ("h = f16(np.maximum(h, 0.0))", "h = np.maximum(h, 0.0)"),
    "input_not_rounded": ("h = f16(X) @ f16(W1).T", "h = np.asarray(X) @ f16(W1).T"),
    "frame_rotation_sign": ("ly = -s * d[..., 0] + c * d[..., 1]",
                            "ly = s * d[..., 0] + c * d[..., 1]"),
    "bias_grad_dropped": ("db2 = float(ds.sum())", "db2 = 0.0"),
    "aabb_distance_from_centre": (
        "out[:, :, 12] = 0.1 * np.minimum(np.hypot(gx, gy), 30)",
        "out[:, :, 12] = 0.1 * np.minimum(np.hypot(gx + 1.0, gy), 30)"),
}


def _mutant(old: str, new: str):
    src = inspect.getsource(omlp)
    # the replaced text may be split over lines in the source: match it with
    # the source's own whitespace collapsed
    flat = " ".join(src.split())
    assert " ".join(old.split()) in flat, "mutation anchor not found: %r" % old
    if old in src:
        msrc = src.replace(old, new, 1)
    else:
        # rebuild the statement on one line (only the corner list spans lines)
        i = src.index("corners = np.stack(")
        j = src.index("# [T, 4, 2]", i)
        stmt = " ".join(src[i:j].split())
        msrc = src[:i] + stmt.replace(" ".join(old.split()), new, 1) + "  " + src[j:]
    mod = types.ModuleType("mlp_mutant")
    exec(compile(msrc, "<mlp_mutant>", "exec"), mod.__dict__)
    return mod


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mlp_mistake_is_caught(name):
    mod = _mutant(*MUTATIONS[name])
    caught = []
    for pname, pin in PINS.items():
        try:
            ok = pin(mod)
        except Exception:
            ok = False
        if not ok:
            caught.append(pname)
    assert caught, "planted mistake %s passed every pin" % name
