"""Pins of the FP64 MLP oracle (learned Newton initial guess)."""
import numpy as np
import pytest

from oracle import mlp as M
from paper_1904_08510_gb300.workload import make_batch


def test_backward_matches_central_differences():
    rng = np.random.default_rng(0)
    p = M.init_params(3)
    for k in p:
        p[k] = p[k] + 0.05 * rng.standard_normal(p[k].shape)
    X = rng.standard_normal((7, M.NF_PAD))
    T = rng.standard_normal((7, M.NOUT))

    def loss(pp):
        return M.mse(M.forward(pp, X)[0], T)[0]
    Y, cache = M.forward(p, X)
    _, dY = M.mse(Y, T)
    g = M.backward(p, cache, dY)
    for k in p:
        flat = p[k].reshape(-1)
        idx = rng.choice(flat.size, size=min(6, flat.size), replace=False)
        for i in idx:
            h = 1e-6 * max(1.0, abs(flat[i]))
            q = {kk: vv.copy() for kk, vv in p.items()}
            q[k].reshape(-1)[i] += h
            lp = loss(q)
            q[k].reshape(-1)[i] -= 2 * h
            lm = loss(q)
            fd = (lp - lm) / (2 * h)
            assert g[k].reshape(-1)[i] == pytest.approx(fd, rel=1e-6, abs=1e-10), (k, i)


def test_silu_closed_form():
    z = np.array([-3.0, 0.0, 1.0, 4.0])
    np.testing.assert_allclose(M.silu(z), z / (1 + np.exp(-z)))
    assert M.silu(0.0) == 0.0
    assert M.silu_grad(np.array([0.0]))[0] == pytest.approx(0.5)
    h = 1e-6
    np.testing.assert_allclose(M.silu_grad(z), (M.silu(z + h) - M.silu(z - h)) / (2 * h), rtol=1e-8)


def test_bf16_rounding():
    v = np.array([1.0, 1 + 2.0 ** -8, 1 + 3 * 2.0 ** -9, -2.5, 3.0e38])
    r = M.bf16_round(v)
    assert r[0] == 1.0
    assert r[1] == 1.0                    # halfway, ties to even
    assert r[2] == 1 + 2.0 ** -7
    assert r[3] == -2.5


def test_adam_first_step_is_lr_times_sign():
    p = dict(w=np.array([1.0, -2.0, 0.5]))
    g = dict(w=np.array([0.3, -4.0, 1e-3]))
    m = dict(w=np.zeros(3))
    v = dict(w=np.zeros(3))
    M.adam_step(p, g, m, v, t=1, lr=1e-2, eps=0.0)
    np.testing.assert_allclose(p["w"], [1.0 - 1e-2, -2.0 + 1e-2, 0.5 - 1e-2])


def test_features_follow_the_stencil_definition():
    b = make_batch("single", 1, 4, n_cells=5)
    X = M.features(b)
    sn, sp = M.column_scales(b)
    assert X.shape == (5, 32) and np.all(X[:, 25:] == 0)
    # cell 0, offset -2 mirrors to cell 1; offset -1 to cell 0
    assert X[0, 0] == pytest.approx(b.ne_old[1] / sn[0])
    assert X[0, 5] == pytest.approx(b.ne_old[0] / sn[0])
    # centre of cell 2 and its field: E h = -(phi_3 - phi_1)/2
    assert X[2, 10] == pytest.approx(b.ne_old[2] / sn[0])
    assert X[2, 13] == pytest.approx(b.T[2] / 2000.0)
    assert X[2, 14] == pytest.approx(-(b.phi_old[3] - b.phi_old[1]) / 2 / sp[0])
    # last cell, offset +2 mirrors to cell N-2 = 3
    assert X[4, 20] == pytest.approx(b.ne_old[3] / sn[0])


def test_guess_inverts_targets():
    b = make_batch("ragged", 3, 2, n_range=(10, 30))
    rng = np.random.default_rng(1)
    ne = b.ne_old * (1 + 0.1 * rng.standard_normal(b.ncells))
    phi = b.phi_old + rng.standard_normal(b.ncells)
    Y = M.targets(b, ne, phi)
    g_ne, g_phi = M.guess(b, Y)
    np.testing.assert_allclose(g_ne, ne, rtol=1e-12)
    np.testing.assert_allclose(g_phi, phi, rtol=1e-12, atol=1e-12)
