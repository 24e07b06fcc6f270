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
