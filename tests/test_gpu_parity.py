"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Floating-point bar: relative 1e-9 per column and field for FP64 results and
1e-7 for the mixed-precision mode (max-norm error over the column divided by
the column's max-norm), the roots being compared at a residual tolerance
(1e-12) where both solvers sit well inside those bounds.
"""
import numpy as np
import pytest

import oracle as O
from paper_1904_08510_gb300.workload import make_batch, uniform_batch

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1904_08510_gb300 import sdcef as S  # noqa: E402


def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return "cuda:0"


def colerr(b, a, ref):
    e = []
    for c in range(b.ncol):
        s = slice(b.col_off[c], b.col_off[c + 1])
        e.append(np.abs(a[s] - ref[s]).max() / max(np.abs(ref[s]).max(), 1e-300))
    return np.array(e)


def solver_for(b, **kw):
    return S.Solver(S.default_params(**kw), max_cols=max(b.ncol, 1), max_cells=max(b.ncells, 2),
                    max_col_cells=max(int(b.lengths().max()) if b.ncol else 2, 2))


def with_extras(b, seed=0):
    """Add advection, an electron source and a second (negative) ion species."""
    rng = np.random.default_rng(seed)
    n = b.ncells
    b.u_adv = 0.4 * np.sin(np.arange(n) * 0.01)
    b.i_re = 1e19 * np.abs(rng.standard_normal(n))
    b.n_ion = np.vstack([b.n_ion, 0.05 * b.n_ion * np.abs(rng.standard_normal(n))])
    b.valence = np.array([1, -1], dtype=np.int32)
    return b


# --------------------------------------------------------------------------
def test_bernoulli_matches_oracle_and_cuda_expm1():
    """The solver's Bernoulli function (series below 1e-3, table-driven e^a - 1
    above, B(-a) = a + B(a)) against the oracle's x / expm1(x) (host libm) and
    against the same formula with CUDA's expm1 (torch on the GPU): B within
    2e-15 relative (a few ulp of each side), B' within 1e-11 relative (the
    derivative formulas differ and 1 - a - B cancels ~11 bits at a = 1e-3).
    Beyond |x| = 709 the exponential is treated as infinite, so B(x) < 1e-305
    is returned as 0: the absolute floor 1e-300 covers that."""
    d = dev()
    rng = np.random.default_rng(5)
    ln2_128 = np.log(2.0) / 128
    pos = np.concatenate([
        np.logspace(-9, np.log10(740.0), 4000), rng.uniform(1e-3, 10.0, 20000),
        rng.uniform(10.0, 700.0, 5000), np.arange(1, 2000) * ln2_128,
        np.nextafter(np.arange(1, 2000) * ln2_128, 0.0), [1e-3, np.nextafter(1e-3, 0.0), 708.99, 709.0]])
    x = np.concatenate([pos, -pos, [0.0]])
    s = S.Solver(S.default_params(), max_cols=1, max_cells=2, max_col_cells=2)
    xt = torch.as_tensor(x, device=d)
    b, db = s.bernoulli(xt)
    torch.cuda.synchronize()
    b, db = b.cpu().numpy(), db.cpu().numpy()
    ref_b = np.array([O.bern(v) for v in x])
    ref_db = np.array([O.bern_deriv(v) for v in x])
    big = np.abs(x) >= 1e-3
    xc = xt[torch.as_tensor(big, device=d)]
    cuda_b = (xc / torch.expm1(xc)).cpu().numpy()
    tol = lambda r, rel: rel * np.abs(r) + 1e-300
    assert np.all(np.abs(b - ref_b) <= tol(ref_b, 2e-15)), np.max(np.abs(b - ref_b) / np.abs(ref_b))
    assert np.all(np.abs(b[big] - cuda_b) <= tol(cuda_b, 2e-15))
    m = np.abs(x) <= 700.0
    assert np.all(np.abs(db[m] - ref_db[m]) <= tol(ref_db[m], 1e-11))
    s.close()


# --------------------------------------------------------------------------
@pytest.mark.parametrize("bc", [S.BC_ABSORBING, S.BC_ZERO_GRADIENT])
@pytest.mark.parametrize("extras", [False, True])
def test_residual_matches_oracle(bc, extras):
    d = dev()
    b = make_batch("ragged", 9, 300, n_range=(2, 700))
    if extras:
        b = with_extras(b, 1)
    rng = np.random.default_rng(5)
    ne = np.abs(b.ne_old * (1 + 0.3 * rng.standard_normal(b.ncells)))
    phi = b.phi_old + 10 * rng.standard_normal(b.ncells)
    s = solver_for(b, bc_electron=bc)
    db = S.DeviceBatch.from_host(b, d)
    Fe, Fp = s.residual(db, torch.as_tensor(ne, device=d), torch.as_tensor(phi, device=d))
    torch.cuda.synchronize()
    Pe = O.default_params(bc_electron=bc)
    Fe_r, Fp_r = O.residual(b, ne, phi, Pe)
    for c in range(b.ncol):
        sl = slice(b.col_off[c], b.col_off[c + 1])
        scale_e = np.abs(Fe_r[sl]).max() + np.abs(ne[sl]).max()
        scale_p = np.abs(Fp_r[sl]).max() + np.abs(ne[sl]).max()
        assert np.abs(Fe.cpu().numpy()[sl] - Fe_r[sl]).max() <= 1e-12 * scale_e, c
        assert np.abs(Fp.cpu().numpy()[sl] - Fp_r[sl]).max() <= 1e-12 * scale_p, c


def _dense_prec_inverse(bc_, P):
    """The oracle's preconditioner as a dense matrix (applied to identity columns)."""
    n = bc_.ncells
    M = np.zeros((2 * n, 2 * n))
    for j in range(2 * n):
        e = np.zeros(2 * n)
        e[j] = 1.0
        x1, x2 = O.prec_apply(bc_, 0, bc_.ne_old, bc_.phi_old, e[:n], e[n:], P)
        M[:, j] = np.concatenate([x1, x2])
    return M


@pytest.mark.parametrize("precond,oprec", [(S.PREC_EXACT, 2), (S.PREC_RECAST, 1)])
@pytest.mark.parametrize("precision", [S.FP64, S.MIXED, S.MIXED_DF])
@pytest.mark.parametrize("tpc", [0, 32, 256])
def test_preconditioner_matches_oracle(precond, oprec, precision, tpc):
    """FP64: forward error <= 1e-9 against the oracle. FP32 (mixed mode): the
    forward error of a block solve is up to cond x 6e-8 (cond ~ N^2 for the
    Poisson-like Schur block), so the check is the backward error: the oracle's
    preconditioner matrix P applied to the GPU result reproduces r to 1e-4 of
    ||P|| ||x||. Double-float (~48-bit significand, unit roundoff ~2^-44 for
    its products and sums): backward error <= 1e-10, and the forward error
    stays below cond x 1e-12."""
    d = dev()
    b = make_batch("ragged", 5, 77, n_range=(2, 400), dt=1e-7)
    rng = np.random.default_rng(2)
    r_e = rng.standard_normal(b.ncells) * 1e18
    r_p = rng.standard_normal(b.ncells) * 1e14
    s = solver_for(b, precond=precond, precision=precision, threads_per_column=tpc)
    db = S.DeviceBatch.from_host(b, d)
    t = lambda a: torch.as_tensor(a, device=d)
    xe, xp = s.precond_apply(db, t(b.ne_old), t(b.phi_old), t(r_e), t(r_p))
    torch.cuda.synchronize()
    xe, xp = xe.cpu().numpy(), xp.cpu().numpy()
    P = O.default_params(precond=oprec)
    for c in range(b.ncol):
        sl = slice(b.col_off[c], b.col_off[c + 1])
        bc_ = b.column(c)
        if precision == S.FP64:
            re_, rp_ = O.prec_apply(bc_, 0, bc_.ne_old, bc_.phi_old, r_e[sl], r_p[sl], P)
            assert np.abs(xe[sl] - re_).max() <= 1e-9 * np.abs(re_).max(), c
            assert np.abs(xp[sl] - rp_).max() <= 1e-9 * np.abs(rp_).max(), c
        else:
            n = bc_.ncells
            # row/column scaling of the typical magnitudes keeps the norms meaningful
            sr = np.concatenate([np.full(n, 1e18), np.full(n, 1e14)])
            sx = np.concatenate([np.full(n, np.abs(xe[sl]).max()), np.full(n, np.abs(xp[sl]).max())])
            Pm = np.linalg.inv(_dense_prec_inverse(bc_, P))
            Ph = Pm * sx[None, :] / sr[:, None]
            x = np.concatenate([xe[sl], xp[sl]]) / sx
            r = np.concatenate([r_e[sl], r_p[sl]]) / sr
            berr = np.abs(Ph @ x - r).max() / (np.abs(Ph).sum(axis=1).max() * np.abs(x).max())
            re_, rp_ = O.prec_apply(bc_, 0, bc_.ne_old, bc_.phi_old, r_e[sl], r_p[sl], P)
            ferr = max(np.abs(xe[sl] - re_).max() / np.abs(re_).max(),
                       np.abs(xp[sl] - rp_).max() / np.abs(rp_).max())
            cond = np.linalg.cond(Ph, p=np.inf)
            print(f"precond precision={precision} col {c} n={n} tpc={tpc} mode={precond}: "
                  f"backward {berr:.2e} forward {ferr:.2e} cond {cond:.2e}")
            if precision == S.MIXED:
                assert berr <= 1e-4, (c, berr)
            else:
                assert berr <= 1e-10, (c, berr)
                assert ferr <= max(cond, 1.0) * 1e-12, (c, ferr, cond)


# --------------------------------------------------------------------------
def _solve_both(b, gpu_kw, ora_kw, guess=None):
    d = dev()
    s = solver_for(b, **gpu_kw)
    db = S.DeviceBatch.from_host(b, d, guess=guess)
    out = s.solve(db)
    torch.cuda.synchronize()
    ref = O.solve(b, O.default_params(**ora_kw), guess=guess)
    return {k: v.cpu().numpy() for k, v in out.items()}, ref


def _converged_or_at_floor(out, ok):
    """eps_F = 1e-12 lies at the FP64 round-off floor of the scaled residual of
    some columns (the oracle itself stops on a line-search failure for a quarter
    of this batch), so whether such a column reaches 1e-12 or stalls just above
    it depends on the rounding order of the arithmetic. A column the oracle
    converged must converge here too or stall at that floor (line-search
    failure with a final residual below 1e-11), at most two of them; the root
    is compared with the oracle's either way."""
    st, fr = out["status"][ok], out["final_res"][ok]
    conv = st == S.STATUS_OK
    floor = (st == S.STATUS_LINESEARCH_FAIL) & (fr < 1e-11)
    assert (conv | floor).all(), (out["status"], out["final_res"])
    assert conv.sum() >= len(st) - 2, out["status"]
    assert (fr[conv] < 1e-12).all()


@pytest.mark.parametrize("tpc", [0, 32, 64, 256])
def test_fp64_solve_matches_oracle_ragged(tpc):
    b = make_batch("ragged", 24, 1000, n_range=(2, 900))
    out, ref = _solve_both(b, dict(eps_F=1e-12, threads_per_column=tpc),
                           dict(precond=2, eps_F=1e-12))
    ok = (ref["status"] == 0)
    _converged_or_at_floor(out, ok)
    assert colerr(b, out["ne"], ref["ne"])[ok].max() <= 1e-9
    assert colerr(b, out["phi"], ref["phi"])[ok].max() <= 1e-9


def test_fp64_single_column_256_cells():
    b = make_batch("single", 1, 1)
    out, ref = _solve_both(b, dict(eps_F=1e-12), dict(precond=2, eps_F=1e-12))
    assert out["status"][0] == S.STATUS_OK and ref["status"][0] == 0
    assert colerr(b, out["ne"], ref["ne"])[0] <= 1e-9
    assert colerr(b, out["phi"], ref["phi"])[0] <= 1e-9


def test_recast_preconditioner_solve_in_paper_regime():
    """Eq. prec_recast with GMRES(30) at an ion-CFL-sized step (dt = 1e-7 s)."""
    b = make_batch("ragged", 8, 500, n_range=(100, 700), dt=1e-7)
    out, ref = _solve_both(b, dict(eps_F=1e-12, precond=S.PREC_RECAST, restart_m=30),
                           dict(precond=1, eps_F=1e-12, restart_m=30))
    assert (out["status"] == S.STATUS_OK).all(), out["status"]
    assert colerr(b, out["ne"], ref["ne"]).max() <= 1e-9
    assert colerr(b, out["phi"], ref["phi"]).max() <= 1e-9
    # the recast form needs several GMRES iterations per Newton step, the exact one ~1
    assert (out["krylov_it"] > out["newton_it"]).all()


def test_mixed_precision_matches_fp64_oracle():
    b = make_batch("single", 16, 1)
    out, ref = _solve_both(b, dict(eps_F=1e-12, precision=S.MIXED),
                           dict(precond=2, eps_F=1e-12))
    assert (out["status"] == S.STATUS_OK).all(), out["status"]
    assert colerr(b, out["ne"], ref["ne"]).max() <= 1e-7
    assert colerr(b, out["phi"], ref["phi"]).max() <= 1e-7


@pytest.mark.parametrize("precond,oprec", [(S.PREC_EXACT, 2), (S.PREC_RECAST, 1)])
@pytest.mark.parametrize("tpc", [0, 32, 256])
def test_double_float_preconditioner_solve_matches_fp64_oracle(precond, oprec, tpc):
    """SDCEF_MIXED_DF: residuals, JVP, Newton update and stopping test in FP64,
    preconditioner in double-float. The root is the FP64 root, so the FP64 bar
    (1e-9) applies."""
    if precond == S.PREC_RECAST:
        b = make_batch("ragged", 8, 500, n_range=(2, 700), dt=1e-7)
        kw = dict(restart_m=30)
    else:
        b = make_batch("ragged", 24, 1000, n_range=(2, 900))
        kw = {}
    out, ref = _solve_both(b, dict(eps_F=1e-12, precision=S.MIXED_DF, precond=precond,
                                   threads_per_column=tpc, **kw),
                           dict(precond=oprec, eps_F=1e-12, **kw))
    # eps_F = 1e-12 is below the FP64 round-off floor of a few columns, where the
    # oracle itself stops (line search); the comparison is on the others
    ok = (ref["status"] == 0)
    assert ok.sum() >= b.ncol // 2, ref["status"]
    _converged_or_at_floor(out, ok)
    assert colerr(b, out["ne"], ref["ne"])[ok].max() <= 1e-9
    assert colerr(b, out["phi"], ref["phi"])[ok].max() <= 1e-9
    # the double-float preconditioner costs at most a few extra GMRES iterations
    kg, ko = out["krylov_it"][ok].sum(), ref["krylov_it"][ok].sum()
    assert kg <= 1.1 * ko + ok.sum(), (kg, ko)


def test_extras_advection_source_two_species():
    b = with_extras(make_batch("ragged", 6, 42, n_range=(50, 400)), 3)
    out, ref = _solve_both(b, dict(eps_F=1e-12), dict(precond=2, eps_F=1e-12))
    ok = ref["status"] == 0
    assert ok.all()
    assert (out["status"] == S.STATUS_OK).all()
    assert colerr(b, out["ne"], ref["ne"]).max() <= 1e-9
    assert colerr(b, out["phi"], ref["phi"]).max() <= 1e-9


def test_guess_at_root_takes_no_newton_step():
    b = make_batch("single", 3, 9, n_cells=128)
    ref = O.solve(b, O.default_params(precond=2, eps_F=1e-13, max_linesearch=6))
    out, _ = _solve_both(b, dict(eps_F=1e-10), dict(precond=2), guess=(ref["ne"], ref["phi"]))
    assert (out["status"] == S.STATUS_OK).all()
    assert (out["newton_it"] == 0).all()


def _scaled_res(b, ne, phi):
    """||S_F^-1 F||_inf per column by the oracle, with the solver's scaling."""
    Fe, Fp = O.residual(b, ne, phi)
    F0e, F0p = O.residual(b, b.ne_old, b.phi_old)
    out = []
    for c in range(b.ncol):
        sl = slice(b.col_off[c], b.col_off[c + 1])
        sn = max(np.abs(b.ne_old[sl]).max(), np.abs(b.n_ion[0, sl]).max(), 1.0)
        sFe = max(np.abs(F0e[sl]).max(), np.abs(b.ne_old[sl]).max(), 1e-12 * sn)
        sFp = max(np.abs(F0p[sl]).max(), np.abs(b.n_ion[0, sl]).max(), 1e-12 * sn)
        out.append(max(np.abs(Fe[sl]).max() / sFe, np.abs(Fp[sl]).max() / sFp))
    return np.array(out)


def test_bench_tolerance_reaches_residual_target():
    """At eps_F = 1e-10 (the bench setting) every column converges and matches the
    oracle run with the same algorithm and tolerance to 1e-9 (max-norm relative).

    The solver's iterate carries phi as phi_ref + psi; the returned phi is that
    sum rounded to double, so the oracle's residual at the returned (n, phi) is
    checked against 1e-10 plus the residual the same rounding leaves at the
    oracle's own fully converged root. Against that root a residual of 1e-10
    bounds the error only through the conditioning of J; it is printed and
    bounded loosely."""
    b = make_batch("ragged", 48, 4242)
    out, same = _solve_both(b, dict(), dict(precond=2))
    ref = O.solve(b, O.default_params(precond=2, eps_F=1e-13, max_linesearch=6))
    assert (out["status"] == S.STATUS_OK).all()
    assert (out["final_res"] < 1e-10).all()
    r_gpu = _scaled_res(b, out["ne"], out["phi"])
    r_floor = _scaled_res(b, ref["ne"], ref["phi"])
    assert (r_gpu <= 1e-10 + 2.0 * r_floor).all(), (r_gpu.max(), r_floor.max())
    sn, sp = colerr(b, out["ne"], same["ne"]), colerr(b, out["phi"], same["phi"])
    en, ep = colerr(b, out["ne"], ref["ne"]), colerr(b, out["phi"], ref["phi"])
    print("eps_F=1e-10 vs oracle at 1e-10: ne max %.2e phi max %.2e; vs converged root: "
          "ne median %.2e max %.2e, phi median %.2e max %.2e"
          % (sn.max(), sp.max(), np.median(en), en.max(), np.median(ep), ep.max()))
    assert sn.max() <= 1e-9 and sp.max() <= 1e-9
    assert en.max() <= 1e-8 and ep.max() <= 1e-8


# --------------------------------------------------------------------------
def test_edge_cases_status():
    d = dev()
    b = make_batch("ragged", 6, 3, n_range=(2, 40))
    # column 1: one cell (rejected); column 2: NaN input; column 3: T <= 0; column 4: dt <= 0
    lens = b.lengths()
    b2 = make_batch("ragged", 6, 3, n_range=(2, 40))
    off = b2.col_off
    b2.ne_old[off[2]] = np.nan
    b2.T[off[3] + 1] = -5.0
    b2.dt[4] = 0.0
    s = solver_for(b2)
    out = s.solve(S.DeviceBatch.from_host(b2, d))
    torch.cuda.synchronize()
    st = out["status"].cpu().numpy()
    assert st[2] == S.STATUS_BAD_INPUT and st[3] == S.STATUS_BAD_INPUT and st[4] == S.STATUS_BAD_INPUT
    assert st[0] == S.STATUS_OK and st[5] == S.STATUS_OK
    assert (lens >= 2).all()
    # one-cell column
    one = uniform_batch(1, 2, ne=1e15, n_ion=1e15, T=1000.0, v_left=0.0, v_right=1.0, dt=1e-6)
    one.col_off = np.array([0, 1], dtype=np.int64)
    one.ne_old = one.ne_old[:1]; one.phi_old = one.phi_old[:1]; one.T = one.T[:1]
    one.rho = one.rho[:1]; one.n_ion = one.n_ion[:, :1]
    s1 = S.Solver(S.default_params(), max_cols=1, max_cells=2, max_col_cells=2)
    o1 = s1.solve(S.DeviceBatch.from_host(one, d))
    torch.cuda.synchronize()
    assert o1["status"].cpu().numpy()[0] == S.STATUS_BAD_INPUT


def test_column_longer_than_capacity_is_rejected():
    d = dev()
    b = make_batch("ragged", 3, 8, n_range=(10, 60))
    s = S.Solver(S.default_params(), max_cols=3, max_cells=b.ncells,
                 max_col_cells=int(b.lengths().min()))
    out = s.solve(S.DeviceBatch.from_host(b, d))
    torch.cuda.synchronize()
    st = out["status"].cpu().numpy()
    lens = b.lengths()
    assert ((st == S.STATUS_BAD_INPUT) == (lens > lens.min())).all()


def test_two_cell_column_and_empty_batch():
    d = dev()
    b = make_batch("ragged", 2, 1, n_range=(2, 2))
    out, ref = _solve_both(b, dict(eps_F=1e-12), dict(precond=2, eps_F=1e-12))
    assert (out["status"] == S.STATUS_OK).all()
    assert colerr(b, out["ne"], ref["ne"]).max() <= 1e-9
    empty = make_batch("ragged", 0, 1)
    s = S.Solver(S.default_params(), max_cols=1, max_cells=2, max_col_cells=2)
    s.solve(S.DeviceBatch.from_host(empty, d))   # returns without launching


def test_iteration_caps_and_unreachable_tolerance_report_status():
    b = make_batch("single", 4, 12)
    out, _ = _solve_both(b, dict(max_newton=1), dict(precond=2))
    assert (out["status"] == S.STATUS_MAX_NEWTON).all()
    assert (out["newton_it"] == 1).all()
    out2, _ = _solve_both(b, dict(eps_F=1e-300, max_linesearch=3, max_newton=40), dict(precond=2))
    assert np.isin(out2["status"], [S.STATUS_LINESEARCH_FAIL, S.STATUS_MAX_NEWTON]).all()


def test_host_entry_point_matches_device_entry_point():
    d = dev()
    b = make_batch("ragged", 10, 66, n_range=(64, 500))
    s = solver_for(b)
    out_d = s.solve(S.DeviceBatch.from_host(b, d))
    torch.cuda.synchronize()
    out_h = s.solve_host(b)
    assert np.array_equal(out_h["ne"], out_d["ne"].cpu().numpy())
    assert np.array_equal(out_h["phi"], out_d["phi"].cpu().numpy())
    assert np.array_equal(out_h["status"], out_d["status"].cpu().numpy())


def test_pipelined_host_batches_match_one_call_per_batch():
    """sdcef_solve_batches_host overlaps the copies of neighbouring batches
    with each solve; every batch's results equal those of its own call."""
    dev()
    bs = [make_batch("ragged", 7, 70, n_range=(64, 400)),
          make_batch("ragged", 0, 71),
          make_batch("ragged", 12, 72, n_range=(32, 500)),
          make_batch("ragged", 3, 73, n_range=(200, 260)),
          make_batch("ragged", 9, 74, n_range=(64, 128))]
    s = S.Solver(S.default_params(), max_cols=12, max_cells=max(b.ncells for b in bs),
                 max_col_cells=500)
    many = s.solve_host_many(bs)
    for b, got in zip(bs, many):
        if b.ncol == 0:
            continue
        ref = s.solve_host(b)
        for k in ("ne", "phi", "status", "newton_it", "krylov_it", "final_res"):
            assert np.array_equal(got[k], ref[k]), k
    # a batch the context cannot hold fails the whole call before any copy
    big = make_batch("ragged", 13, 75, n_range=(64, 128))
    with pytest.raises(S.SdcefError):
        s.solve_host_many([bs[0], big])
    assert s.solve_host_many([]) == []
    # one batch through the pipelined call equals the single-batch call
    one = s.solve_host_many([bs[2]])[0]
    assert np.array_equal(one["ne"], s.solve_host(bs[2])["ne"])


def test_outputs_may_alias_inputs():
    d = dev()
    b = make_batch("ragged", 5, 90, n_range=(64, 300))
    s = solver_for(b)
    db = S.DeviceBatch.from_host(b, d)
    ref = s.solve(db)
    out = s.alloc_result(db)
    out["ne"] = db.tensors["ne_old"]
    out["phi"] = db.tensors["phi_old"]
    s.solve(db, out)
    torch.cuda.synchronize()
    assert torch.equal(out["ne"], ref["ne"]) and torch.equal(out["phi"], ref["phi"])


def test_autotune_picks_a_candidate_and_keeps_results():
    d = dev()
    b = make_batch("ragged", 40, 321, n_range=(64, 700))
    s = solver_for(b)
    db = S.DeviceBatch.from_host(b, d)
    ref = s.solve(db)
    torch.cuda.synchronize()
    ref = {k: v.cpu().numpy() for k, v in ref.items()}
    tpb, ms = s.autotune(db, reps=1)
    assert tpb in (32, 64, 128, 256) and ms[tpb] == min(ms.values())
    out = s.solve(db)
    torch.cuda.synchronize()
    assert (out["status"].cpu().numpy() == ref["status"]).all()
    assert colerr(b, out["ne"].cpu().numpy(), ref["ne"]).max() <= 1e-9


def test_bad_guess_is_judged_and_replaced_by_plain_start():
    """A start far from the root (rough noise in n_e and phi) fails Newton. The
    solver judges a supplied start three times: its residual against the plain
    start's before the first step (guess_reject_ratio), the residual reduction
    of each step (guess_progress) and its convergence within guess_newton_cap
    steps; each judge alone brings the column back to X^n, and it converges to
    the same root as the plain solve."""
    d = dev()
    b = make_batch("single", 6, 77, n_cells=300)
    rng = np.random.default_rng(9)
    g_ne = b.ne_old * (1 + 0.2 * rng.standard_normal(b.ncells))
    g_phi = b.phi_old + 5.0 * rng.standard_normal(b.ncells)
    plain, _ = _solve_both(b, dict(eps_F=1e-12), dict(precond=2, eps_F=1e-12))
    judged, _ = _solve_both(b, dict(eps_F=1e-12), dict(precond=2), guess=(g_ne, g_phi))
    raw, _ = _solve_both(b, dict(eps_F=1e-12, guess_newton_cap=0, guess_reject_ratio=0.0,
                                 max_newton=20), dict(precond=2), guess=(g_ne, g_phi))
    ratio_only, _ = _solve_both(b, dict(eps_F=1e-12, guess_newton_cap=0), dict(precond=2),
                                guess=(g_ne, g_phi))
    cap_only, _ = _solve_both(b, dict(eps_F=1e-12, guess_reject_ratio=0.0, guess_progress=0.0),
                              dict(precond=2), guess=(g_ne, g_phi))
    # the progress judge alone: a wandering step sends the column back to X^n
    # long before a cap of 40 steps
    prog_only, _ = _solve_both(b, dict(eps_F=1e-12, guess_reject_ratio=0.0, guess_newton_cap=40,
                                       guess_progress=0.3), dict(precond=2), guess=(g_ne, g_phi))
    assert (plain["status"] == S.STATUS_OK).all()
    assert (judged["status"] == S.STATUS_OK).all()
    assert (raw["status"] != S.STATUS_OK).any()
    assert (ratio_only["status"] == S.STATUS_OK).all()   # rejected before the first step
    assert (cap_only["status"] == S.STATUS_OK).all()     # restarted after the cap
    assert (prog_only["status"] == S.STATUS_OK).all()    # restarted after a wandering step
    assert prog_only["newton_it"].max() < 40 + plain["newton_it"].max()
    assert colerr(b, prog_only["ne"], plain["ne"]).max() <= 1e-9
    assert colerr(b, judged["ne"], plain["ne"]).max() <= 1e-9
    assert colerr(b, judged["phi"], plain["phi"]).max() <= 1e-9
