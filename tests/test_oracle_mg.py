"""Pins of the oracle's multigrid block solver (Sec. 4.2: V-cycles with two
red-black Gauss-Seidel relaxations down and up, to a tolerance gamma_MG).

The references are independent of the oracle's multigrid code: a closed-form
Galerkin stencil, the Schur complement and ideal transfers computed by dense
linear algebra (numpy), direct solves, a textbook convergence rate, and the
recast preconditioner with exact (Thomas) block solves.
"""
import numpy as np
import pytest

import oracle as O
from paper_1904_08510_gb300.workload import make_batch


def dense_tri(sub, dia, sup):
    M = np.diag(dia).astype(float)
    M += np.diag(sub[1:], -1)
    M += np.diag(sup[:-1], 1)
    return M


def poisson(n):
    sub, dia, sup = np.ones(n), -2.0 * np.ones(n), np.ones(n)
    sub[0] = 0.0
    sup[-1] = 0.0
    return sub, dia, sup


def random_mmatrix(n, seed):
    """Non-symmetric, strictly diagonally dominant tridiagonal (upwind-like)."""
    rng = np.random.default_rng(seed)
    sub = rng.uniform(0.0, 5.0, n)
    sup = rng.uniform(0.0, 0.5, n)
    sub[0] = 0.0
    sup[-1] = 0.0
    dia = -(sub + sup) - rng.uniform(0.1, 1.0, n)
    return sub, dia, sup


def column_blocks(seed=7, n_cells=512, dt=1e-6, col=0):
    """(A, S~) tridiagonals of one synthetic flame column, built at X^n."""
    b = make_batch("single", 2, seed, n_cells=n_cells, dt=dt)
    A, B, L = O.jacobian_blocks(b, b.ne_old, b.phi_old)
    sl = slice(b.col_off[col], b.col_off[col + 1])
    Ab = tuple(A[k][sl] for k in range(3))
    Sb = tuple(L[k][sl] - B[k][sl] for k in range(3))
    return Ab, Sb


def rel_res(T, x, b):
    return np.linalg.norm(b - dense_tri(*T) @ x) / np.linalg.norm(b)


# --------------------------------------------------------------------------
def test_linear_galerkin_coarse_poisson_stencil():
    """Linear interpolation P (1/2, 1, 1/2) and R = P^T applied to the stencil
    [1, -2, 1]: T P e_I is 1/2 at fine 2I-1, -1 at 2I+1, 1/2 at 2I+3 and 0 at the
    even unknowns, so R T P has the interior stencil [1/2, -1, 1/2]."""
    lev = O.mg_hierarchy(*poisson(64), transfer=O.MG_LINEAR)
    assert [len(l[1]) for l in lev] == [64, 32, 16, 8]
    sub, dia, sup = lev[1]
    np.testing.assert_array_equal(sub[1:-1], 0.5)
    np.testing.assert_array_equal(dia[1:-1], -1.0)
    np.testing.assert_array_equal(sup[1:-1], 0.5)


@pytest.mark.parametrize("n", [17, 64, 101])
def test_operator_transfers_are_the_ideal_ones(n):
    """Black-box transfers on a non-symmetric tridiagonal T equal the ideal
    interpolation [-T_FF^-1 T_FC; I] and restriction [-T_CF T_FF^-1, I]
    (F = even, fine-only unknowns; C = odd unknowns), computed densely."""
    T = random_mmatrix(n, n)
    M = dense_tri(*T)
    P, R = O.mg_transfers(*T, transfer=O.MG_OPERATOR)
    F = np.arange(0, n, 2)
    C = np.arange(1, 2 * (n // 2), 2)
    Pi = np.zeros((n, n // 2))
    Pi[C, np.arange(n // 2)] = 1.0
    Pi[F] = -np.linalg.solve(M[np.ix_(F, F)], M[np.ix_(F, C)])
    Ri = np.zeros((n // 2, n))
    Ri[np.arange(n // 2), C] = 1.0
    Ri[:, F] = -M[np.ix_(C, F)] @ np.linalg.inv(M[np.ix_(F, F)])
    np.testing.assert_allclose(P, Pi, rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(R, Ri, rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("n", [16, 63, 200])
def test_operator_coarse_operator_is_schur_complement(n):
    """With the ideal transfers, R T P = T_CC - T_CF T_FF^-1 T_FC."""
    T = random_mmatrix(n, 100 + n)
    M = dense_tri(*T)
    F = np.arange(0, n, 2)
    C = np.arange(1, 2 * (n // 2), 2)
    S = M[np.ix_(C, C)] - M[np.ix_(C, F)] @ np.linalg.solve(M[np.ix_(F, F)], M[np.ix_(F, C)])
    lev = O.mg_hierarchy(*T, transfer=O.MG_OPERATOR)
    np.testing.assert_allclose(dense_tri(*lev[1]), S, rtol=1e-12, atol=1e-12 * np.abs(S).max())


@pytest.mark.parametrize("transfer", [O.MG_OPERATOR, O.MG_LINEAR])
def test_mg_converges_to_the_direct_solution(transfer):
    rng = np.random.default_rng(3)
    for T in (poisson(1000), column_blocks()[1]) + ((column_blocks()[0],) if transfer == O.MG_OPERATOR else ()):
        b = rng.standard_normal(len(T[1]))
        x, k = O.mg_solve_tri(*T, b, 1e-12, max_cycles=200, transfer=transfer)
        xe = np.linalg.solve(dense_tri(*T), b)
        assert k >= 1
        assert np.abs(x - xe).max() <= 1e-9 * np.abs(xe).max()


def test_operator_v_cycle_is_exact_in_one_cycle():
    """In 1D the ideal transfers make the coarse problem the Schur complement,
    so after one V-cycle (post-relaxation of the fine-only unknowns last) the
    residual is at rounding level, for any 3-point operator."""
    rng = np.random.default_rng(5)
    for T in (poisson(777), random_mmatrix(500, 1)) + column_blocks():
        b = rng.standard_normal(len(T[1]))
        x, k = O.mg_solve_tri(*T, b, 0.0, max_cycles=1, transfer=O.MG_OPERATOR)
        assert k == 1
        assert rel_res(T, x, b) < 1e-9


def test_linear_v_cycle_rate_on_the_schur_block():
    """Textbook V(2,2) with red-black Gauss-Seidel: each cycle reduces the
    residual by well under 1/3 on the elliptic S~ block (Gauss-Seidel alone
    reduces it by a factor ~1 - O(h^2) per sweep, so a broken coarse-grid
    correction fails this)."""
    T = column_blocks()[1]
    b = np.random.default_rng(9).standard_normal(len(T[1]))
    prev = 1.0
    for k in range(1, 6):
        x, kk = O.mg_solve_tri(*T, b, 0.0, max_cycles=k, transfer=O.MG_LINEAR)
        r = rel_res(T, x, b)
        assert r < prev / 3.0
        prev = r


def test_tolerance_and_cycle_count():
    T = column_blocks()[1]
    b = np.random.default_rng(1).standard_normal(len(T[1]))
    counts = []
    for g in (1e-1, 1e-2, 1e-4, 1e-8):
        x, k = O.mg_solve_tri(*T, b, g, transfer=O.MG_LINEAR)
        assert rel_res(T, x, b) <= g
        x1, _ = O.mg_solve_tri(*T, b, 0.0, max_cycles=k - 1, transfer=O.MG_LINEAR) if k > 1 else (np.zeros_like(b), 0)
        assert k == 1 or rel_res(T, x1, b) > g      # the first cycle count that meets gamma
        counts.append(k)
    assert counts == sorted(counts) and counts[-1] > counts[0]


def test_no_progress_stops_and_undoes():
    """An unreachable tolerance stops at the rounding floor (a cycle that does
    not lower the residual is undone), not at the cycle cap; linear transfers
    on the upwind-dominated electron block diverge, and the solve returns the
    start x = 0 after the one (undone) cycle."""
    A, S = column_blocks()
    b = np.random.default_rng(2).standard_normal(len(S[1]))
    x, k = O.mg_solve_tri(*S, b, 1e-30, max_cycles=100, transfer=O.MG_OPERATOR)
    assert k < 10
    assert rel_res(S, x, b) < 1e-9
    x, k = O.mg_solve_tri(*A, b, 1e-4, max_cycles=100, transfer=O.MG_LINEAR)
    assert k == 1
    assert np.all(x == 0.0)


def test_mg_preconditioner_equals_recast_with_exact_blocks():
    """Preconditioner 3 (multigrid blocks, operator transfers, gamma = 1e-4)
    applies the recast form of Eq. prec_recast; with one exact V-cycle per block
    it matches the Thomas-based recast form to rounding. Linear transfers on
    S~ (A exact) at gamma = 1e-10 match to ~gamma."""
    b = make_batch("single", 3, 11, n_cells=300, dt=1e-6)
    rng = np.random.default_rng(0)
    v1 = rng.standard_normal(b.ncells) * 1e10
    v2 = rng.standard_normal(b.ncells) * 1e9
    for c in range(b.ncol):
        sl = slice(b.col_off[c], b.col_off[c + 1])
        ref = O.prec_apply(b, c, b.ne_old, b.phi_old, v1[sl], v2[sl], O.default_params(precond=O.PREC_RECAST))
        x1, x2, k = O.prec_apply(b, c, b.ne_old, b.phi_old, v1[sl], v2[sl],
                                 O.default_params(precond=O.PREC_MG), return_cycles=True)
        assert k == 3          # three block solves of one V-cycle each
        for u, r in zip((x1, x2), ref):
            assert np.abs(u - r).max() <= 1e-9 * np.abs(r).max()
        P = O.default_params(precond=O.PREC_MG, mg_transfer=O.MG_LINEAR, mg_gamma_A=0.0,
                             mg_gamma_S=1e-10)
        x1, x2, k = O.prec_apply(b, c, b.ne_old, b.phi_old, v1[sl], v2[sl], P, return_cycles=True)
        assert k > 1
        for u, r in zip((x1, x2), ref):
            assert np.abs(u - r).max() <= 1e-6 * np.abs(r).max()


def test_mg_jfnk_reaches_the_recast_root():
    b = make_batch("single", 4, 21, n_cells=256, dt=3e-7)
    ref = O.solve(b, O.default_params(precond=O.PREC_RECAST))
    for P in (O.default_params(precond=O.PREC_MG),
              O.default_params(precond=O.PREC_MG, mg_transfer=O.MG_LINEAR, mg_gamma_A=0.0)):
        r = O.solve(b, P)
        assert (r["status"] == 0).all() and (ref["status"] == 0).all()
        assert (r["mg_cycles"] > 0).all()
        for k in ("ne", "phi"):
            assert np.abs(r[k] - ref[k]).max() <= 1e-8 * np.abs(ref[k]).max()
    # operator transfers: one exact V-cycle per block solve, the same Krylov path
    r = O.solve(b, O.default_params(precond=O.PREC_MG))
    np.testing.assert_array_equal(r["krylov_it"], ref["krylov_it"])
    np.testing.assert_array_equal(r["newton_it"], ref["newton_it"])
