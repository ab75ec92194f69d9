"""Training kernels of the tile-proposal network: gradients against the FP64
numpy reference, learning on exact labels, bit-exact checkpoint/resume."""
from __future__ import annotations

import numpy as np
import pytest

from oracle import mlp as omlp
from paper_2607_04310_b300 import train_cull as tc

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not torch.cuda.is_available(), reason="needs a CUDA device")]


@pytest.fixture(scope="module")
def small_data():
    X, y = tc.build_dataset(40)
    return X, y


def test_gradients_match_fp64_reference(small_data):
    X, y = small_data
    W1, w2, b2 = tc.init_weights(3)
    # FP16-representable weights: the same values the inference kernel uses
    W1 = W1.astype(np.float16).astype(np.float32)
    w2 = w2.astype(np.float16).astype(np.float32)
    tr = tc.Trainer(W1, w2, b2)
    N = 20000
    g, loss = tr.grad(X[:N], y[:N])
    torch.cuda.synchronize()
    Xn = X[:N].cpu().numpy().astype(np.float64)
    yn = y[:N].cpu().numpy().astype(np.float64)
    rl, dW1, dw2, db2 = omlp.loss_and_grads(Xn, yn, W1.astype(np.float64), w2.astype(np.float64), b2)
    ref = np.concatenate([dW1.reshape(-1), dw2, [db2]])
    got = g.cpu().numpy().astype(np.float64)
    scale = np.abs(ref).max()
    assert np.max(np.abs(got - ref)) <= 1e-4 * scale, np.max(np.abs(got - ref)) / scale
    assert abs(loss.item() - rl) <= 1e-4 * max(1.0, rl)


def test_training_reduces_loss_and_beats_the_bound(small_data):
    X, y = small_data
    tr = tc.train(X, y, epochs=4, batch=4096, lr=3e-3, seed=0)
    W1, w2, b2 = tc.split_params(tr.get_state()["params"])
    g0, l0 = tc.Trainer(*tc.init_weights(0)).grad(X, y)
    g1, l1 = tc.Trainer(W1, w2, b2).grad(X, y)
    assert l1.item() < 0.5 * l0.item()
    ev = tc.evaluate(W1, w2, b2, n_scenes=20)
    assert ev["top1_mlp"] > 0.3


def test_checkpoint_resume_is_bit_exact(small_data, tmp_path):
    X, y = small_data
    X, y = X[:80000].contiguous(), y[:80000].contiguous()
    ck = str(tmp_path / "ck.bin")
    full = tc.train(X, y, epochs=3, batch=4096, lr=2e-3, seed=5)
    ref = full.get_state()
    part = tc.train(X, y, epochs=3, batch=4096, lr=2e-3, seed=5, checkpoint=ck,
                    stop_after_epoch=0)
    resumed = tc.resume(ck, X, y)
    got = resumed.get_state()
    assert got["step"] == ref["step"]
    for k in ("params", "m", "v"):
        assert np.array_equal(got[k].view(np.uint32), ref[k].view(np.uint32)), k
    state, meta = tc.load_checkpoint(ck)
    assert meta["format"] == tc.CKPT_FORMAT and meta["epoch_done"] == 0
