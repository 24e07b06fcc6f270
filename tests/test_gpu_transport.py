"""GPU parity of the field-dependent electron transport (SDCEF_TRANSPORT_TABLE,
Sec. 2.2) against the oracle through the C ABI: residual, roots, iteration
behaviour, charge flux, and the constant model written as a table."""
import numpy as np
import pytest

import oracle as O
from paper_1904_08510_gb300.workload import (constant_transport_table, make_batch,
                                             transport_table)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1904_08510_gb300 import sdcef as S  # noqa: E402


def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return "cuda:0"


def solver(b, table, **kw):
    s = S.Solver(S.default_params(transport=S.TRANSPORT_TABLE, **kw), max_cols=b.ncol,
                 max_cells=b.ncells, max_col_cells=int(b.lengths().max()))
    s.set_transport_table(table)
    return s


def colerr(b, a, ref):
    return np.array([np.abs(a[s] - ref[s]).max() / max(np.abs(ref[s]).max(), 1e-300)
                     for s in (slice(b.col_off[c], b.col_off[c + 1]) for c in range(b.ncol))])


def test_table_residual_matches_oracle():
    """F(X) at a perturbed state: every face looks up mu and D at its own E/N."""
    d = dev()
    b = make_batch("ragged", 10, 12, n_range=(2, 900), dt=1e-7)
    tab = transport_table()
    rng = np.random.default_rng(3)
    ne = b.ne_old * (1 + 0.1 * rng.standard_normal(b.ncells))
    phi = b.phi_old + 30.0 * np.sin(np.arange(b.ncells) * 0.05)
    s = solver(b, tab)
    db = S.DeviceBatch.from_host(b, d)
    t = lambda a: torch.as_tensor(a, device=d)
    Fe, Fp = s.residual(db, t(ne), t(phi))
    torch.cuda.synchronize()
    re_, rp_ = O.residual(b, ne, phi, O.default_params(table=tab))
    for c in range(b.ncol):
        sl = slice(b.col_off[c], b.col_off[c + 1])
        if sl.stop - sl.start < 2:
            continue
        se = max(np.abs(re_[sl]).max(), np.abs(b.ne_old[sl]).max())
        sp = max(np.abs(rp_[sl]).max(), np.abs(b.n_ion[0, sl]).max())
        assert np.abs(Fe.cpu().numpy()[sl] - re_[sl]).max() <= 1e-11 * se, c
        assert np.abs(Fp.cpu().numpy()[sl] - rp_[sl]).max() <= 1e-11 * sp, c


@pytest.mark.parametrize("precond,oprec", [(S.PREC_EXACT, O.PREC_EXACT), (S.PREC_RECAST, O.PREC_RECAST)])
def test_table_roots_match_oracle(precond, oprec):
    d = dev()
    b = make_batch("ragged", 12, 44, n_range=(64, 800), dt=1e-7)
    tab = transport_table()
    s = solver(b, tab, eps_F=1e-12, precond=precond, restart_m=30 if precond == S.PREC_RECAST else 8)
    out = s.solve(S.DeviceBatch.from_host(b, d))
    torch.cuda.synchronize()
    ref = O.solve(b, O.default_params(eps_F=1e-12, precond=oprec, table=tab))
    assert (out["status"].cpu().numpy() == 0).all() and (ref["status"] == 0).all()
    assert colerr(b, out["ne"].cpu().numpy(), ref["ne"]).max() <= 1e-9
    assert colerr(b, out["phi"].cpu().numpy(), ref["phi"]).max() <= 1e-9


def test_constant_table_reproduces_the_constant_kernel():
    d = dev()
    b = make_batch("ragged", 16, 5, n_range=(100, 1500), dt=1e-5)
    db = S.DeviceBatch.from_host(b, d)
    rc = S.Solver(S.default_params(threads_per_column=128), max_cols=b.ncol, max_cells=b.ncells,
                  max_col_cells=int(b.lengths().max())).solve(db)
    rt = solver(b, constant_transport_table()).solve(db)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(rc["status"].cpu().numpy(), rt["status"].cpu().numpy())
    np.testing.assert_array_equal(rc["newton_it"].cpu().numpy(), rt["newton_it"].cpu().numpy())
    for k in ("ne", "phi"):
        assert colerr(b, rt[k].cpu().numpy(), rc[k].cpu().numpy()).max() <= 1e-11


def test_table_current_matches_oracle():
    d = dev()
    b = make_batch("ragged", 8, 17, n_range=(2, 700), dt=1e-7)
    tab = transport_table()
    s = solver(b, tab)
    db = S.DeviceBatch.from_host(b, d)
    phi = b.phi_old + 10.0 * np.cos(np.arange(b.ncells) * 0.07)
    t = lambda a: torch.as_tensor(a, device=d)
    jp, jn = s.current(db, t(b.ne_old), t(phi))
    torch.cuda.synchronize()
    rp, rn = O.current(b, b.ne_old, phi, 4e-3, O.default_params(table=tab))
    for c in range(b.ncol):
        f = slice(b.col_off[c] + c, b.col_off[c + 1] + c + 1)
        sc = max(np.abs(rn[f]).max(), np.abs(rp[f]).max(), 1e-300)
        assert np.abs(jn.cpu().numpy()[f] - rn[f]).max() <= 1e-10 * sc
        assert np.abs(jp.cpu().numpy()[f] - rp[f]).max() <= 1e-10 * sc


def test_table_parameter_validation():
    d = dev()
    b = make_batch("single", 2, 1, n_cells=64, dt=1e-7)
    db = S.DeviceBatch.from_host(b, d)
    s = S.Solver(S.default_params(transport=S.TRANSPORT_TABLE), max_cols=2, max_cells=b.ncells,
                 max_col_cells=64)
    with pytest.raises(RuntimeError):        # no table set
        s.solve(db)
    for kw in (dict(precision=S.MIXED), dict(precond=S.PREC_MG), dict(gas_molar_mass=0.0)):
        with pytest.raises(RuntimeError):
            S.Solver(S.default_params(transport=S.TRANSPORT_TABLE, **kw), max_cols=1, max_cells=8,
                     max_col_cells=8)
    bad = transport_table()
    bad["mu"] = bad["mu"].copy()
    bad["mu"][3, 4] = -1.0
    with pytest.raises(RuntimeError):
        s.set_transport_table(bad)
    out = s.alloc_result(db)
    with pytest.raises(RuntimeError):
        S.solve_noalloc(S.default_params(transport=S.TRANSPORT_TABLE), db, out, 64)
