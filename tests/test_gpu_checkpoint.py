"""Checkpoint / resume of the learned-guess training (library state: FP32
parameters, Adam moments, step; trainer state: iteration and window
generator). A run resumed from a checkpoint taken half-way must reproduce the
uninterrupted run bit for bit (every training step sums its partial
gradients in a fixed order)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1904_08510_gb300 import learned as Lrn  # noqa: E402
from paper_1904_08510_gb300 import sdcef as S  # noqa: E402


def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return "cuda:0"


def data(rows, d):
    g = torch.Generator(device="cpu").manual_seed(3)
    X = torch.randn(rows, 32, generator=g)
    X[:, 25:] = 0.0
    W = torch.randn(32, 2, generator=g) * 0.1
    T = torch.tanh(X @ W) + 0.01 * torch.randn(rows, 2, generator=g)
    return X.to(torch.bfloat16).to(d), T.float().to(d)


def test_state_round_trip_is_exact():
    d = dev()
    X, T = data(4096, d)
    mlp, _ = Lrn.train(X, T, steps=5, batch=1024, seed=2)
    st = mlp.get_state()
    assert st["step"] == 5 and np.abs(st["adam_v"]).max() > 0
    other = S.MLP(1024)
    other.set_state(st)
    back = other.get_state()
    for k in ("params", "adam_m", "adam_v"):
        np.testing.assert_array_equal(back[k], st[k])
    assert back["step"] == 5


def test_resumed_training_matches_uninterrupted(tmp_path):
    d = dev()
    X, T = data(16384, d)
    kw = dict(steps=40, batch=2048, seed=4, lr=2e-3)
    a, _ = Lrn.train(X, T, **kw)
    ck = str(tmp_path / "ck.npz")
    b, _ = Lrn.train(X, T, checkpoint=ck, checkpoint_every=20, **kw)
    c, _ = Lrn.train(X, T, resume=ck, **kw)
    pa, pb, pc = a.get_params(), b.get_params(), c.get_params()
    assert c.get_state()["step"] == 40
    np.testing.assert_array_equal(pb, pa)
    np.testing.assert_array_equal(pc, pa)
    # and it differs from simply restarting the schedule
    r, _ = Lrn.train(X, T, steps=20, batch=2048, seed=4, lr=2e-3,
                     params=Lrn.load_checkpoint(ck)[0]["params"])
    assert np.abs(r.get_params() - pa).max() > np.abs(pc - pa).max()
