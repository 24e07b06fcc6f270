"""Seeded randomized parity sweep: GPU solve against the oracle over random
combinations of column sizes, time step, voltage range, electron boundary
condition, preconditioner form, precision mode, threads per column, and
optional advection / electron source / second ion species. Where both sides
converge the roots agree at the FP64 bar (1e-9; 1e-8 for the double-float
preconditioner, whose iterates round differently); a column converges on the
GPU wherever it converges in the oracle, up to columns stalling within a
decade of the residual target (the stopping test sits near the round-off
floor for some of them)."""
import numpy as np
import pytest

import oracle as O
from paper_1904_08510_gb300.workload import make_batch

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1904_08510_gb300 import sdcef as S  # noqa: E402


def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return "cuda:0"


def case(seed):
    rng = np.random.default_rng(seed)
    kind = ["single", "ragged"][rng.integers(2)]
    lo = int(rng.choice([2, 16, 128]))
    hi = int(rng.choice([200, 700, 1500]))
    dt = float(rng.choice([1e-7, 1e-6, 1e-5]))
    b = make_batch(kind, 10, 10_000 * seed, n_range=(lo, hi), dt=dt)
    extras = bool(rng.integers(2))
    if extras:
        n = b.ncells
        b.u_adv = 0.5 * np.sin(np.arange(n) * 0.013)
        b.i_re = 1e19 * np.abs(rng.standard_normal(n))
        b.n_ion = np.vstack([b.n_ion, 0.05 * b.n_ion * np.abs(rng.standard_normal(n))])
        b.valence = np.array([1, -1], dtype=np.int32)
    bc = int(rng.integers(2))
    precond = [S.PREC_EXACT, S.PREC_RECAST][rng.integers(2)] if dt < 1e-5 else S.PREC_EXACT
    precision = [S.FP64, S.MIXED_DF][rng.integers(2)]
    tpc = int(rng.choice([32, 64, 128, 256]))
    return b, dict(bc_electron=bc, precond=precond, precision=precision, threads_per_column=tpc,
                   restart_m=30 if precond == S.PREC_RECAST else 8)


@pytest.mark.parametrize("seed", range(1, 13))
def test_random_configuration_matches_oracle(seed):
    d = dev()
    b, kw = case(seed)
    s = S.Solver(S.default_params(**kw), max_cols=b.ncol, max_cells=max(b.ncells, 2),
                 max_col_cells=max(int(b.lengths().max()), 2))
    out = s.solve(S.DeviceBatch.from_host(b, d))
    torch.cuda.synchronize()
    out = {k: v.cpu().numpy() for k, v in out.items()}
    oprec = O.PREC_EXACT if kw["precond"] == S.PREC_EXACT else O.PREC_RECAST
    ref = O.solve(b, O.default_params(bc_electron=kw["bc_electron"], precond=oprec))
    tol = 1e-8 if kw["precision"] == S.MIXED_DF else 1e-9
    for c in range(b.ncol):
        sl = slice(b.col_off[c], b.col_off[c + 1])
        if sl.stop - sl.start < 2:
            assert out["status"][c] == S.STATUS_BAD_INPUT and ref["status"][c] == O.BAD_INPUT
            continue
        if ref["status"][c] == O.OK:
            assert out["status"][c] == S.STATUS_OK or out["final_res"][c] < 1e-9, (seed, c, kw)
        if ref["status"][c] == O.OK and out["status"][c] == S.STATUS_OK:
            for k in ("ne", "phi"):
                e = np.abs(out[k][sl] - ref[k][sl]).max() / max(np.abs(ref[k][sl]).max(), 1e-300)
                assert e <= tol, (seed, c, k, e, kw)
