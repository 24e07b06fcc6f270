"""Failure path of the tensor-core kernels' bounded waits.

Every mbarrier wait of the tcgen05 kernels (guess, inference forward, fused
training step) is bounded; a wait that runs out makes the kernel set an error
word, write NaN for the rows (or the partial gradient) it was computing, skip
the rest of its work and, after bounded waits that let issued MMAs finish,
free its tensor memory. The poll
count of the main waits is a handle setting; at 0 every such wait gives up at
once, exactly as one that ran out, with no GPU fault and no hang. The test
drives that path and checks that the context stays usable: with the default
restored, the next calls reproduce the results of the calls made before.
"""
import numpy as np
import pytest

from oracle import mlp as M
from paper_1904_08510_gb300.workload import make_batch

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1904_08510_gb300 import sdcef as S  # noqa: E402


def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return "cuda:0"


def params(seed=13):
    p = M.init_params(seed)
    rng = np.random.default_rng(seed)
    for k in ("b1", "b2", "b3"):
        p[k] = 0.1 * rng.standard_normal(p[k].shape)
    p["W1"][:, 25:] = 0.0
    return S.pack_params(p).astype(np.float32)


def test_wait_that_runs_out_sets_error_and_nan_then_recovers():
    d = dev()
    b = make_batch("ragged", 6, 21, n_range=(100, 600))
    db = S.DeviceBatch.from_host(b, d)
    n = 3000
    mlp = S.MLP(max(b.ncells, n))
    mlp.set_params(params())
    rng = np.random.default_rng(4)
    Xh = M.bf16_round(rng.standard_normal((n, 32)))
    Xh[:, 25:] = 0.0
    X = torch.as_tensor(Xh, dtype=torch.float32, device=d).to(torch.bfloat16)
    T = torch.as_tensor(rng.standard_normal((n, 2)), dtype=torch.float32, device=d)
    # reference calls with the default bound
    ne0, _ = mlp.guess(db, components=S.GUESS_NE)
    g0, _ = mlp.grad(X, T)
    mlp.check()
    ne0, g0 = ne0.cpu().numpy(), g0.cpu().numpy()
    assert np.isfinite(ne0).all() and np.isfinite(g0).all()

    mlp.set_wait_polls(0)
    sentinel = 12345.0
    ne_f = torch.full((b.ncells,), sentinel, dtype=torch.float64, device=d)
    ph_f = torch.full_like(ne_f, sentinel)
    mlp.guess(db, ne_f, ph_f, components=S.GUESS_NE)
    with pytest.raises(S.SdcefError) as e:
        mlp.check()
    assert e.value.code == S.ERR_CUDA
    nef, phf = ne_f.cpu().numpy(), ph_f.cpu().numpy()
    # the rows a worker was computing hold NaN; no row holds a result
    assert np.isnan(nef).any()
    assert np.all(np.isnan(nef) | (nef == sentinel))
    assert np.all((phf == sentinel) | (phf == b.phi_old))
    g1, _ = mlp.grad(X, T)
    with pytest.raises(S.SdcefError) as e:
        mlp.check()
    assert e.value.code == S.ERR_CUDA
    assert np.isnan(g1.cpu().numpy()).any()

    mlp.set_wait_polls(-1)
    ne2, _ = mlp.guess(db, components=S.GUESS_NE)
    g2, _ = mlp.grad(X, T)
    mlp.check()                       # the error word was cleared by the last check
    assert np.array_equal(ne2.cpu().numpy(), ne0)
    # the training step sums its partial gradients in a fixed order: bit-identical
    assert np.array_equal(g2.cpu().numpy(), g0)
    mlp.close()
