"""The allocation-free solve entry point against the context-based one.

sdcef_solve_batch_noalloc serves callers that cannot call cudaMalloc when they
solve (an application whose device memory belongs to its own arena allocator,
or a code that forbids allocation after start-up). It must give the same
results as sdcef_solve_batch on the same batch; it is called twice in a row
because every call reuses the library's one scratch array and must not depend
on what the previous call left there. This file is collected last so that a
run stopping at the first failure has already run every other test.
"""
import numpy as np
import pytest

from paper_1904_08510_gb300.workload import make_batch

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1904_08510_gb300 import sdcef as S  # noqa: E402


def _colerr(b, a, ref):
    e = []
    for c in range(b.ncol):
        s = slice(b.col_off[c], b.col_off[c + 1])
        e.append(np.abs(a[s] - ref[s]).max() / max(np.abs(ref[s]).max(), 1e-300))
    return np.array(e)


@pytest.mark.parametrize("precision", [S.FP64, S.MIXED, S.MIXED_DF])
def test_noalloc_solve_matches_context_solve_twice(precision):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    d = "cuda:0"
    # two different batches, so the second call runs over the first call's leftovers
    batches = [make_batch("ragged", 40, 5150, n_range=(2, 1500)),
               make_batch("ragged", 25, 9311, n_range=(100, 3000))]
    tol = 1e-7 if precision == S.MIXED else 1e-9
    for b in batches:
        p = S.default_params(precision=precision)
        mcc = int(b.lengths().max())
        ref_solver = S.Solver(p, max_cols=b.ncol, max_cells=b.ncells, max_col_cells=mcc)
        db = S.DeviceBatch.from_host(b, d)
        ref = ref_solver.solve(db)
        torch.cuda.synchronize()
        ref = {k: v.cpu().numpy() for k, v in ref.items()}
        for _call in range(2):
            out = ref_solver.alloc_result(db)
            for v in out.values():
                v.fill_(-7)
            S.solve_noalloc(p, db, out, mcc)
            torch.cuda.synchronize()
            got = {k: v.cpu().numpy() for k, v in out.items()}
            assert np.array_equal(got["status"], ref["status"])
            assert np.array_equal(got["newton_it"], ref["newton_it"])
            ok = ref["status"] == S.STATUS_OK
            if precision != S.MIXED:
                assert ok.all()
            assert ok.any()
            assert _colerr(b, got["ne"], ref["ne"])[ok].max() <= tol
            assert _colerr(b, got["phi"], ref["phi"])[ok].max() <= tol
        ref_solver.close()


def test_noalloc_rejects_sizes_beyond_its_limits():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    b = make_batch("ragged", 3, 1, n_range=(10, 20))
    db = S.DeviceBatch.from_host(b, "cuda:0")
    out = {k: torch.empty(1, device="cuda:0") for k in ("ne", "phi")}
    out.update({k: None for k in ("status", "newton_it", "krylov_it", "res_evals", "final_res")})
    with pytest.raises(S.SdcefError) as e:
        S.solve_noalloc(S.default_params(), db, out, S.NOALLOC_MAX_COL_CELLS + 1)
    assert e.value.code == S.ERR_CAPACITY


def test_noalloc_reports_a_column_longer_than_max_col_cells():
    """max_col_cells comes from the caller here, so the kernel's own length check
    is the only guard on the slot size: a longer column is BAD_INPUT and the
    others still match the context solve."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    d = "cuda:0"
    b = make_batch("ragged", 12, 6060, n_range=(64, 400))
    lens = b.lengths()
    long_col = int(np.argmax(lens))
    mcc = int(np.sort(lens)[-2])            # every column fits but the longest
    assert lens[long_col] > mcc
    p = S.default_params()
    ref_solver = S.Solver(p, max_cols=b.ncol, max_cells=b.ncells, max_col_cells=int(lens.max()))
    db = S.DeviceBatch.from_host(b, d)
    ref = {k: v.cpu().numpy() for k, v in ref_solver.solve(db).items()}
    out = ref_solver.alloc_result(db)
    S.solve_noalloc(p, db, out, mcc)
    torch.cuda.synchronize()
    got = {k: v.cpu().numpy() for k, v in out.items()}
    others = np.arange(b.ncol) != long_col
    assert got["status"][long_col] == S.STATUS_BAD_INPUT
    assert (got["status"][others] == S.STATUS_OK).all()
    assert _colerr(b, got["ne"], ref["ne"])[others].max() <= 1e-9
    assert _colerr(b, got["phi"], ref["phi"])[others].max() <= 1e-9
    ref_solver.close()


def test_noalloc_single_column_matches_context_solve():
    """One column: the path that launches no column-order kernel."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    d = "cuda:0"
    b = make_batch("ragged", 1, 777, n_range=(300, 900))
    p = S.default_params()
    n = int(b.ncells)
    ref_solver = S.Solver(p, max_cols=1, max_cells=n, max_col_cells=n)
    db = S.DeviceBatch.from_host(b, d)
    ref = {k: v.cpu().numpy() for k, v in ref_solver.solve(db).items()}
    out = ref_solver.alloc_result(db)
    S.solve_noalloc(p, db, out, n)
    torch.cuda.synchronize()
    got = {k: v.cpu().numpy() for k, v in out.items()}
    assert got["status"][0] == S.STATUS_OK and ref["status"][0] == S.STATUS_OK
    assert got["newton_it"][0] == ref["newton_it"][0]
    assert np.array_equal(got["ne"], ref["ne"]) and np.array_equal(got["phi"], ref["phi"])
    ref_solver.close()
