"""The learned-start solve against the oracle's converged root.

The path under test is a learned Newton start (the BF16 network's n_e
increment and the potential of the guessed charge, tcgen05 inference kernel)
followed by the batched solve at the
bench tolerance ||S_F^-1 F||_inf < 1e-10 with the error test of the stop
(eps_E = 5e-10, the default), in FP64, with the double-float preconditioner
and with the FP32 Krylov solve and preconditioner. The plain start (X^n) is
checked the same way. Every batch is solved whole on the GPU; sampled columns
(the shortest, the longest, the eight with the smallest |V_R|, whose scaled
Jacobian is worst conditioned, and a seeded draw) are compared element by
element with the oracle's root, converged to its rounding floor
(eps_F = 1e-13, error test at 1e-14), as max-norm relative errors per column
and field. Bars: 1e-9 for FP64 and double-float, 1e-7 for FP32.
"""
import numpy as np
import pytest

import oracle as O
from paper_1904_08510_gb300.workload import make_batch

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1904_08510_gb300 import sdcef as S  # noqa: E402
from paper_1904_08510_gb300 import learned as Lrn  # noqa: E402


def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return "cuda:0"


def sample_columns(b, n_rand=24, seed=0):
    lens = b.lengths()
    cols = {int(np.argmin(lens)), int(np.argmax(lens))}
    cols |= set(int(c) for c in np.argsort(np.abs(b.v_right))[:8])
    rng = np.random.default_rng(seed)
    cols |= set(int(c) for c in rng.choice(b.ncol, n_rand, replace=False))
    return sorted(cols)


def converged_root(sub):
    r = O.solve(sub, O.default_params(precond=2, eps_F=1e-13, max_linesearch=6, eps_E=1e-14))
    # the floor of eps_F = 1e-13 ends most columns in the line search, after the
    # residual has passed 1e-10 on the way
    assert np.isin(r["status"], [O.OK, O.LINESEARCH_FAIL]).all(), r["status"]
    assert (r["final_res"] < 1e-10).all()
    return r


def column_errors(b, cols, out, ref):
    en, ep = [], []
    for k, c in enumerate(cols):
        s = slice(b.col_off[c], b.col_off[c + 1])
        a, e = int(b.col_off[c]), int(b.col_off[c + 1])
        r = slice(int(ref["off"][k]), int(ref["off"][k + 1]))
        assert e - a == r.stop - r.start
        en.append(np.abs(out["ne"][s] - ref["ne"][r]).max() / np.abs(ref["ne"][r]).max())
        ep.append(np.abs(out["phi"][s] - ref["phi"][r]).max() / np.abs(ref["phi"][r]).max())
    return np.array(en), np.array(ep)


MODES = [("fp64", S.FP64, 8, 1e-9), ("mixed_df", S.MIXED_DF, 8, 1e-9), ("mixed", S.MIXED, 16, 1e-7)]


@pytest.mark.parametrize("family", ["headline", "holdout"])
def test_learned_start_matches_converged_oracle_root(family):
    d = dev()
    if family == "headline":
        b = make_batch("ragged", 4096, 2_000_000)
        weights = Lrn.WEIGHTS_RAGGED
    else:
        b = make_batch("single", 4096, 2_000_000, n_range=(512, 2048))
        weights = Lrn.WEIGHTS
    cols = sample_columns(b)
    sub = b.subset(cols)
    ref = converged_root(sub)
    ref["off"] = sub.col_off
    db = S.DeviceBatch.from_host(b, d)
    mlp = S.MLP(b.ncells)
    mlp.set_params(Lrn.load(weights))
    ne_g, ph_g = mlp.guess(db, components=S.GUESS_NE | S.GUESS_PHI_POISSON)
    mlp.check()
    gdb = db.with_guess(ne_g, ph_g)
    lmax = int(b.lengths().max())
    report = []
    for name, prec, m, bar in MODES:
        s = S.Solver(S.default_params(precision=prec, restart_m=m), max_cols=b.ncol,
                     max_cells=b.ncells, max_col_cells=lmax)
        for start, batch in (("plain", db), ("learned", gdb)):
            out = s.solve(batch)
            torch.cuda.synchronize()
            out = {k: v.cpu().numpy() for k, v in out.items()}
            assert (out["status"] == S.STATUS_OK).all(), (name, start, np.bincount(out["status"]))
            assert (out["final_res"] < 1e-10).all()
            en, ep = column_errors(b, cols, out, ref)
            report.append("%s %s %s: ne max %.2e phi max %.2e (newton %.3f)" % (
                family, name, start, en.max(), ep.max(), out["newton_it"].mean()))
            assert en.max() <= bar and ep.max() <= bar, report[-1]
        s.close()
    mlp.close()
    print("\n".join(report))


def test_error_test_off_leaves_the_low_voltage_error():
    """Without the error test (eps_E = 0) the residual test alone leaves a column
    of the bench batch with |V_R| = 1.6 V at a potential error above 1e-8 (the
    scaled Jacobian's conditioning), which the default error test removes."""
    d = dev()
    full = make_batch("ragged", 4096, 2_000_000)
    b = full.subset([444])
    assert abs(b.v_right[0]) < 2.0
    ref = converged_root(b)
    ref["off"] = b.col_off
    db = S.DeviceBatch.from_host(b, d)
    errs = {}
    for eps_E in (0.0, 5e-10):
        s = S.Solver(S.default_params(eps_E=eps_E), max_cols=1, max_cells=b.ncells,
                     max_col_cells=b.ncells)
        out = s.solve(db)
        torch.cuda.synchronize()
        out = {k: v.cpu().numpy() for k, v in out.items()}
        assert out["status"][0] == S.STATUS_OK
        en, ep = column_errors(b, [0], out, ref)
        errs[eps_E] = max(en[0], ep[0])
        s.close()
    assert errs[0.0] > 1e-8, errs
    assert errs[5e-10] <= 1e-9, errs
