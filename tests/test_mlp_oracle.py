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
    assert X.shape == (5, 32)
    # column context: position, density level, voltage, resolution, time step
    np.testing.assert_allclose(X[:, 25], (np.arange(5) + 0.5) / 5)
    assert np.all(X[:, 26] == np.log10(sn[0]) - 16.0)
    assert np.all(X[:, 27] == (b.v_right[0] - b.v_left[0]) / 1000.0)
    assert np.all(X[:, 28] == (np.log2(5.0) - 10.0) / 2.0)
    np.testing.assert_allclose(X[:, 29], 0.0, atol=1e-15)   # dt = 1e-5 s
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


# --------------------------------------------------------------------------
# Poisson potential of the guess (root of F_phi) and the ion-field features
def _parabola(x, L, vl, vr, rho_over_eps):
    """phi'' = -rho/eps0 with phi(0) = V_L, phi(L) = V_R, uniform rho."""
    return vl + (vr - vl) * x / L + 0.5 * rho_over_eps * x * (L - x)


@pytest.mark.parametrize("N", [2, 3, 7, 64])
def test_poisson_potential_of_uniform_charge_is_the_parabola(N):
    """Interior second differences and the one-sided second-order electrode
    faces are exact for quadratics, so the discrete root equals the exact
    solution at the cell centres."""
    L, vl, vr = 0.01, 37.0, -250.0
    h = L / N
    n, f = 3e15, 8e15                      # net charge e (f - n)
    x = (np.arange(N) + 0.5) * h
    phi = M.poisson_potential(np.full(N, n - f), h, vl, vr)
    ref = _parabola(x, L, vl, vr, M.E_CHARGE * (f - n) / M.EPS0)
    np.testing.assert_allclose(phi, ref, rtol=1e-11, atol=1e-9 * np.abs(ref).max())


def test_ion_field_of_uniform_ions_is_the_parabola_and_its_slope():
    N, L, f = 40, 0.01, 2e16
    h = L / N
    x = (np.arange(N) + 0.5) * h
    phi, E = M.ion_field(np.full(N, f), h)
    a = M.E_CHARGE * f / M.EPS0
    np.testing.assert_allclose(phi, 0.5 * a * x * (L - x), rtol=1e-11)
    # mean of the two face slopes of a quadratic = its slope at the centre
    np.testing.assert_allclose(E, -0.5 * a * (L - 2 * x), rtol=1e-9, atol=1e-9 * a * L)


def test_poisson_start_zeroes_the_residual_of_the_c_oracle():
    """The potential of guess bit 2 makes the C oracle's Poisson residual vanish
    (an independent implementation of F_phi), with n_e from the network."""
    import oracle as O
    b = make_batch("ragged", 3, 12, n_range=(2, 300))
    rng = np.random.default_rng(3)
    Y = 0.05 * rng.standard_normal((b.ncells, 2))
    ne, phi = M.guess(b, Y, components=5)
    ne1, _ = M.guess(b, Y, components=1)
    np.testing.assert_array_equal(ne, ne1)
    _, Fp = O.residual(b, ne, phi, O.default_params())
    fphi = np.atleast_2d(b.n_ion).sum(axis=0)
    for c in range(b.ncol):
        s = slice(b.col_off[c], b.col_off[c + 1])
        scale = max(np.abs(ne[s]).max(), np.abs(fphi[s]).max())
        assert np.abs(Fp[s]).max() <= 1e-9 * scale, c
    # bit 2 alone keeps n_e^n and solves for its charge
    ne4, phi4 = M.guess(b, Y, components=4)
    np.testing.assert_array_equal(ne4, b.ne_old)
    _, Fp4 = O.residual(b, ne4, phi4, O.default_params())
    assert np.abs(Fp4).max() <= 1e-9 * max(np.abs(b.ne_old).max(), np.abs(fphi).max())


def test_context_features_of_the_ion_field():
    b = make_batch("ragged", 2, 40, n_range=(30, 90))
    X = M.features(b)
    sn, sp = M.column_scales(b)
    for c in range(b.ncol):
        a0, a1 = int(b.col_off[c]), int(b.col_off[c + 1])
        N, L = a1 - a0, b.length[c]
        phi, E = M.ion_field(b.n_ion[0, a0:a1], L / N)
        np.testing.assert_allclose(X[a0:a1, 30], np.arcsinh(phi / sp[c]))
        np.testing.assert_allclose(X[a0:a1, 31], np.arcsinh(E * L / sp[c]))
        # the ion potential is positive inside (positive charge, grounded electrodes)
        assert np.all(phi > 0)
