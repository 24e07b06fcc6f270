"""GPU parity of the SDC electric sweep (provisional ions + k_max solves)."""
import numpy as np
import pytest

import oracle as O
from paper_1904_08510_gb300.workload import make_batch, sdc_batch

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1904_08510_gb300 import sdcef as S  # noqa: E402


def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return "cuda:0"


def colerr(b, a, ref):
    return np.array([np.abs(a[s] - ref[s]).max() / max(np.abs(ref[s]).max(), 1e-300)
                     for s in (slice(b.col_off[c], b.col_off[c + 1]) for c in range(b.ncol))])


def test_ion_update_matches_oracle():
    d = dev()
    b = make_batch("ragged", 7, 91, n_range=(2, 500))
    b.n_ion = np.vstack([b.n_ion, 0.3 * b.n_ion])
    b.valence = np.array([1, -1], dtype=np.int32)
    rng = np.random.default_rng(4)
    phi = b.phi_old + 20 * rng.standard_normal(b.ncells)
    s = S.Solver(S.default_params(), max_cols=b.ncol, max_cells=b.ncells,
                 max_col_cells=int(b.lengths().max()))
    db = S.DeviceBatch.from_host(b, d)
    out = s.ion_update(db, torch.as_tensor(phi, device=d), 4e-3)
    torch.cuda.synchronize()
    ref = O.ion_update(b, phi, 4e-3)
    np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


def test_ion_provisional_matches_oracle():
    """The paper's provisional ion transport (second-order Godunov advection,
    implicit diffusion, SDC correction) on ragged columns of 0..600 cells with
    two species of opposite valence and an advection velocity, from n^n and
    from a previous iterate."""
    d = dev()
    b = make_batch("ragged", 9, 92, n_range=(0, 600), dt=2e-6)
    rng = np.random.default_rng(6)
    b.n_ion = np.vstack([b.n_ion, 0.3 * b.n_ion + 1e12])
    b.valence = np.array([1, -1], dtype=np.int32)
    b.u_adv = 0.5 * np.cos(np.arange(b.ncells) * 0.02)
    phi = b.phi_old + 20 * rng.standard_normal(b.ncells)
    prev = b.n_ion * (1.0 + 0.1 * rng.standard_normal(b.n_ion.shape))
    s = S.Solver(S.default_params(), max_cols=b.ncol, max_cells=max(b.ncells, 2),
                 max_col_cells=max(int(b.lengths().max()), 2))
    db = S.DeviceBatch.from_host(b, d)
    t = lambda a: torch.as_tensor(a, device=d)
    for npv in (None, prev):
        out = s.ion_provisional(db, t(phi), None if npv is None else t(npv), 4e-3)
        torch.cuda.synchronize()
        ref = O.ion_provisional(b, phi, npv, 4e-3)
        np.testing.assert_allclose(out.cpu().numpy(), ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


@pytest.mark.parametrize("precond,precision,scheme", [
    (S.PREC_EXACT, S.FP64, S.ION_GODUNOV), (S.PREC_RECAST, S.FP64, S.ION_GODUNOV),
    (S.PREC_EXACT, S.MIXED_DF, S.ION_GODUNOV), (S.PREC_EXACT, S.FP64, S.ION_DRIFT_UPWIND)])
def test_sdc_sweep_matches_oracle(precond, precision, scheme):
    """Every SDC iteration's solve at the FP64 bar, with either provisional ion
    update; the double-float preconditioner mode reaches the same roots."""
    d = dev()
    b = sdc_batch(12, 777, n_cells=256)
    P = S.default_params(eps_F=1e-12, precond=precond, precision=precision,
                         restart_m=30 if precond == S.PREC_RECAST else 8, ion_scheme=scheme)
    s = S.Solver(P, max_cols=b.ncol, max_cells=b.ncells, max_col_cells=256)
    db = S.DeviceBatch.from_host(b, d)
    out = s.sdc_sweep(db, k_max=4)
    torch.cuda.synchronize()
    ne_r, phi_r, hist = O.sdc_sweep(b, 4, 4e-3, O.default_params(precond=2, eps_F=1e-12),
                                    scheme="godunov" if scheme == S.ION_GODUNOV else "drift")
    assert all((h["status"] == 0).all() for h in hist)
    assert (out["status"].cpu().numpy() == S.STATUS_OK).all()
    assert colerr(b, out["ne"].cpu().numpy(), ne_r).max() <= 1e-9
    assert colerr(b, out["phi"].cpu().numpy(), phi_r).max() <= 1e-9


def test_sdc_poisson_start_keeps_the_roots_and_saves_gmres():
    """Iterations k >= 2 start from the previous n_e with the potential of its
    charge under the new provisional ions (sdc_poisson_start = 1, the default)
    or from the previous iterate as it is (0): the same roots (the oracle's
    sweep at 1e-9), fewer GMRES iterations in the last SDC iteration."""
    d = dev()
    b = sdc_batch(64, 778, n_cells=512)
    db = S.DeviceBatch.from_host(b, d)
    outs = {}
    for ps in (0, 1):
        s = S.Solver(S.default_params(eps_F=1e-12, sdc_poisson_start=ps), max_cols=b.ncol,
                     max_cells=b.ncells, max_col_cells=512)
        o = s.sdc_sweep(db, k_max=4)
        torch.cuda.synchronize()
        outs[ps] = {k: v.cpu().numpy() for k, v in o.items()}
        assert (outs[ps]["status"] == S.STATUS_OK).all()
        s.close()
    ne_r, phi_r, hist = O.sdc_sweep(b, 4, 4e-3, O.default_params(precond=2, eps_F=1e-12))
    for ps in (0, 1):
        assert colerr(b, outs[ps]["ne"], ne_r).max() <= 1e-9
        assert colerr(b, outs[ps]["phi"], phi_r).max() <= 1e-9
    assert outs[1]["krylov_it"].mean() <= outs[0]["krylov_it"].mean()


@pytest.mark.parametrize("precision", [S.FP64, S.MIXED_DF])
def test_sdc_sweep_graph_replay_matches_eager(precision):
    d = dev()
    b = sdc_batch(64, 31, n_cells=512)
    s = S.Solver(S.default_params(precision=precision), max_cols=b.ncol, max_cells=b.ncells,
                 max_col_cells=512)
    db = S.DeviceBatch.from_host(b, d)
    eager = s.sdc_sweep(db, k_max=4)
    torch.cuda.synchronize()
    eager = {k: v.clone() for k, v in eager.items()}
    out = s.alloc_result(db)
    work = s.sweep_work(db)
    stream = torch.cuda.Stream()
    s2 = S.Solver(S.default_params(precision=precision), max_cols=b.ncol, max_cells=b.ncells,
                  max_col_cells=512, stream=stream)
    s2.sdc_sweep(db, k_max=4, work=work, out=out)     # first call outside capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        s2.sdc_sweep(db, k_max=4, work=work, out=out)
    for v in out.values():
        v.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(out["ne"], eager["ne"]) and torch.equal(out["phi"], eager["phi"])
    assert torch.equal(out["status"], eager["status"])
