"""Krylov vectors in shared memory (sdcef_params.krylov_on_chip = 1).

The solver kernel may keep a column's GMRES vectors (Algorithm 2: w, v_0,
z_0 = P^-1 v_0, the error test's correction, the correction sum, then v_i, z_i)
in the shared memory it leaves unused at its occupancy instead of in the
column's workspace slot. Only where the vectors live changes, not one
operation, so every result must be bit-identical to the slot-only solve: for
every precision and preconditioner, for columns short enough to hold all
vectors on chip, long enough to hold none, and in between, and on solves that
restart GMRES (which use every vector of the cycle and the correction sum).
"""
import numpy as np
import pytest

from paper_1904_08510_gb300.workload import make_batch

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1904_08510_gb300 import sdcef as S  # noqa: E402

KEYS = ("ne", "phi", "status", "newton_it", "krylov_it", "res_evals")


def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return "cuda:0"


def solve(b, db, **kw):
    s = S.Solver(S.default_params(**kw), max_cols=b.ncol, max_cells=b.ncells,
                 max_col_cells=int(b.lengths().max()))
    out = s.solve(db)
    torch.cuda.synchronize()
    r = {k: out[k].cpu().numpy() for k in KEYS}
    s.close()
    return r


CASES = [
    ("fp64_auto", dict()),
    ("fp64_tpc32", dict(threads_per_column=32)),
    ("fp64_tpc256", dict(threads_per_column=256)),
    ("mixed_m16", dict(precision=S.MIXED, restart_m=16)),
    ("mixed_df", dict(precision=S.MIXED_DF)),
    ("recast_m30", dict(precond=S.PREC_RECAST, restart_m=30)),
    ("multigrid", dict(precond=S.PREC_MG, restart_m=30)),
    # unpreconditioned GMRES(4): restarts, every V_i / z_i and the correction sum
    ("none_m4_restarts", dict(precond=S.PREC_NONE, restart_m=4, max_newton=3, max_krylov=40)),
]


@pytest.mark.parametrize("name,kw", CASES, ids=[c[0] for c in CASES])
def test_on_chip_solve_is_bit_identical_to_slot_solve(name, kw):
    d = dev()
    small_dt = name.startswith(("recast", "multigrid", "none"))
    b = make_batch("ragged", 36, 7711, n_range=(2, 2600), dt=1e-7 if small_dt else 1e-5)
    db = S.DeviceBatch.from_host(b, d)
    ref = solve(b, db, krylov_on_chip=0, **kw)
    got = solve(b, db, krylov_on_chip=1, **kw)
    if not name.startswith("none"):
        assert (ref["status"] == S.STATUS_OK).sum() >= b.ncol - 1
    for k in KEYS:
        assert np.array_equal(got[k], ref[k]), k


def test_autotune_on_chip_keeps_the_faster_and_the_results():
    d = dev()
    b = make_batch("ragged", 300, 4242)
    db = S.DeviceBatch.from_host(b, d)
    s = S.Solver(S.default_params(), max_cols=b.ncol, max_cells=b.ncells,
                 max_col_cells=int(b.lengths().max()))
    choice, ms = s.autotune_on_chip(db, reps=1)
    assert choice in (0, 1)
    assert ms[0] > 0.0 and ms[1] > 0.0
    assert choice == (1 if ms[1] < ms[0] else 0)
    assert s.params.krylov_on_chip == choice
    out = s.solve(db)
    torch.cuda.synchronize()
    got = {k: out[k].cpu().numpy() for k in KEYS}
    s.close()
    ref = solve(b, db, krylov_on_chip=1 - choice)
    for k in KEYS:
        assert np.array_equal(got[k], ref[k]), k


def test_on_chip_noalloc_is_bit_identical_to_slot_noalloc():
    d = dev()
    b = make_batch("ragged", 30, 3131, n_range=(2, 1800))
    db = S.DeviceBatch.from_host(b, d)
    mcc = int(b.lengths().max())
    s = S.Solver(S.default_params(), max_cols=b.ncol, max_cells=b.ncells, max_col_cells=mcc)
    res = []
    for oc in (0, 1):
        out = s.alloc_result(db)
        for v in out.values():
            v.fill_(-7)
        S.solve_noalloc(S.default_params(krylov_on_chip=oc), db, out, mcc)
        torch.cuda.synchronize()
        res.append({k: out[k].cpu().numpy() for k in KEYS})
    s.close()
    assert (res[0]["status"] == S.STATUS_OK).all()
    for k in KEYS:
        assert np.array_equal(res[1][k], res[0][k]), k
