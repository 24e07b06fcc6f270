"""Pins of the oracle's field-dependent electron transport (Sec. 2.2: mobility
and diffusivity from two-dimensional tables over the progress variable c and
the reduced field |E|/N; synthetic tables stand in for BOLSIG+): bilinear
interpolation is exact for bilinear data and clamps outside the table; the
constant-mobility model written as a table reproduces the constant path
(residual, Jacobian, root); the current in a uniform plasma follows the table
at a node (Ohm's law with mu(c, E/N)); JFNK roots satisfy the table residual."""
import numpy as np
import pytest

import oracle as O
from paper_1904_08510_gb300.workload import (constant_transport_table, make_batch,
                                             transport_table, uniform_batch)

NA = 6.02214076e23


def test_bilinear_lookup_is_exact_for_bilinear_data_and_clamps():
    nc, nx, en_max = 7, 13, 300.0
    c = np.linspace(0, 1, nc)[:, None]
    x = np.linspace(0, en_max, nx)[None, :]
    f = lambda c, x: 2.0 + 3.0 * c - 0.01 * x + 0.05 * c * x
    t = f(c, x)
    rng = np.random.default_rng(0)
    for cc, xx in zip(rng.uniform(0, 1, 50), rng.uniform(0, en_max, 50)):
        assert abs(O.tab_lookup(t, en_max, cc, xx) - f(cc, xx)) <= 1e-13 * abs(f(cc, xx))
    assert O.tab_lookup(t, en_max, -0.5, 1e6) == pytest.approx(f(0.0, en_max), rel=1e-14)
    assert O.tab_lookup(t, en_max, 2.0, -3.0) == pytest.approx(f(1.0, 0.0), rel=1e-14)


def test_constant_table_reproduces_the_constant_model():
    """mu constant and D = mu k_B T(c)/e is linear in c, so the face values
    (means of the cells' c) equal the constant path's face values."""
    b = make_batch("single", 3, 2, n_cells=128, dt=1e-7)
    Pc = O.default_params(precond=O.PREC_EXACT, eps_F=1e-12)
    Pt = O.default_params(precond=O.PREC_EXACT, eps_F=1e-12, table=constant_transport_table())
    rng = np.random.default_rng(1)
    ne = b.ne_old * (1 + 0.1 * rng.standard_normal(b.ncells))
    phi = b.phi_old + rng.standard_normal(b.ncells)
    for u, v in zip(O.residual(b, ne, phi, Pc), O.residual(b, ne, phi, Pt)):
        assert np.abs(u - v).max() <= 1e-12 * np.abs(u).max()
    for u, v in zip(O.jacobian_blocks(b, ne, phi, Pc), O.jacobian_blocks(b, ne, phi, Pt)):
        assert np.abs(u - v).max() <= 1e-12 * np.abs(u).max()
    rc, rt = O.solve(b, Pc), O.solve(b, Pt)
    np.testing.assert_array_equal(rc["newton_it"], rt["newton_it"])
    for k in ("ne", "phi"):
        assert np.abs(rc[k] - rt[k]).max() <= 1e-12 * np.abs(rc[k]).max()


def test_uniform_plasma_current_follows_the_table():
    """Uniform n, T and rho, linear phi: interior faces carry J- = e n mu E
    with mu = the table value at (c, E/N); T and the field are chosen on table
    nodes, so mu is the generating formula itself."""
    tab = transport_table()
    T, n, L = 1150.0, 2e15, 0.01                     # c = 0.5, a node
    b = uniform_batch(1, 64, ne=n, n_ion=n, T=T, v_left=0.0, v_right=1.0, dt=1e-7)
    N = b.rho[0] * NA / 0.028
    dv = 20.0 * 1e-21 * N * L                        # E/N = 20 Td, a node
    b = uniform_batch(1, 64, ne=n, n_ion=n, T=T, v_left=0.0, v_right=dv, dt=1e-7)
    en_td = (dv / L) / N / 1e-21
    P = O.default_params(table=tab)
    jp, jn = O.current(b, b.ne_old, b.phi_old, 4e-3, P)
    c = (T - tab["T_in"]) / (tab["T_max"] - tab["T_in"])
    mu = 0.4 * (1 + 0.25 * (c - 0.5)) / np.sqrt(1 + (en_td / 20.0) ** 2)
    np.testing.assert_allclose(jn[1:-1], O.E_CHARGE * n * mu * (-dv / L), rtol=1e-9)
    # off-node: within the interpolation error of the smooth formula
    e2 = 21.3
    mu2 = 0.4 * (1 + 0.25 * (c - 0.5)) / np.sqrt(1 + (e2 / 20.0) ** 2)
    assert abs(mu2 - O.tab_lookup(tab["mu"], tab["en_max_td"], c, e2)) < 2e-3 * mu2


def test_field_dependent_roots_satisfy_the_table_residual():
    b = make_batch("single", 4, 3, n_cells=200, dt=1e-7)
    P = O.default_params(precond=O.PREC_EXACT, table=transport_table())
    r = O.solve(b, P)
    assert (r["status"] == 0).all()
    Fe, Fp = O.residual(b, r["ne"], r["phi"], P)
    Fe0, Fp0 = O.residual(b, b.ne_old, b.phi_old, P)
    for c in range(b.ncol):
        sl = slice(b.col_off[c], b.col_off[c + 1])
        sFe = max(np.abs(Fe0[sl]).max(), np.abs(b.ne_old[sl]).max())
        sFp = max(np.abs(Fp0[sl]).max(), np.abs(b.n_ion[0, sl]).max())
        assert max(np.abs(Fe[sl]).max() / sFe, np.abs(Fp[sl]).max() / sFp) < 1e-10
    # the field dependence changes the root (mobility falls with E/N)
    rc = O.solve(b, O.default_params(precond=O.PREC_EXACT))
    assert np.abs(r["ne"] - rc["ne"]).max() > 1e-4 * np.abs(rc["ne"]).max()


def test_table_jacobian_matches_central_differences():
    """The analytic Jacobian with transport tables carries the interpolant's
    slopes mu'(G), D'(G): it matches central differences of the table residual
    (steps small enough that no face crosses a table node)."""
    b = make_batch("single", 1, 3, n_cells=14, dt=1e-7)
    n = b.ncells
    rng = np.random.default_rng(4)
    ne = b.ne_old * (1 + 0.2 * rng.standard_normal(n)) + 1e14
    phi = b.phi_old * 20.0 + 30.0 * rng.standard_normal(n)     # E/N of tens of Td
    b.v_right = b.v_right * 20.0
    P = O.default_params(table=transport_table())
    A, B, L = O.jacobian_blocks(b, ne, phi, P)
    d = lambda T: np.diag(T[1]) + np.diag(T[0][1:], -1) + np.diag(T[2][:-1], 1)
    J = np.block([[d(A), d(B)], [-np.eye(n), d(L)]])
    F = lambda X: np.concatenate(O.residual(b, X[:n], X[n:], P))
    X = np.concatenate([ne, phi])
    scale = np.concatenate([np.full(n, 1e16), np.full(n, 100.0)])
    Jfd = np.zeros_like(J)
    for j in range(2 * n):
        h = 1e-8 * scale[j]
        Xp, Xm = X.copy(), X.copy()
        Xp[j] += h
        Xm[j] -= h
        Jfd[:, j] = (F(Xp) - F(Xm)) / (2 * h)
    rowmax = np.abs(Jfd).max(axis=1, keepdims=True)
    assert np.all(np.abs(J - Jfd) <= 1e-6 * rowmax)
    # at these fields mu' G / mu is O(1) (the mobility falls with E/N over
    # 20 Td), so a Jacobian with frozen coefficients would miss by far more
    G = np.abs(np.diff(phi)) / (b.length[0] / n)
    N = b.rho[0] * 6.02214076e23 / 0.028
    assert np.median(G / N / 1e-21) > 10.0
