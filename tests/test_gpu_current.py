"""GPU parity of the charge-flux diagnostic (sdcef_current_batch, Sec. 4.4)
against the oracle, through the C ABI.

Both sides evaluate the same face formulas in FP64; the GPU's Bernoulli
function agrees with the host's x / expm1(x) to a few ulp (see the Bernoulli
parity test), and the electron flux is a difference of two such terms, so the
comparison is made relative to the larger of the two Scharfetter-Gummel terms
of the column (the flux scale), at 1e-12."""
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


def with_species(b, seed):
    rng = np.random.default_rng(seed)
    n = b.ncells
    b.u_adv = 0.4 * np.sin(np.arange(n) * 0.01)
    b.n_ion = np.vstack([b.n_ion, 0.05 * b.n_ion * np.abs(rng.standard_normal(n))])
    b.valence = np.array([1, -1], dtype=np.int32)
    return b


def flux_scale(b, c, ne):
    """e (D/h) max n of column c: the size of each Scharfetter-Gummel term."""
    sl = slice(b.col_off[c], b.col_off[c + 1])
    h = b.length[c] / (sl.stop - sl.start)
    D = 0.4 * O.K_B * b.T[sl].max() / O.E_CHARGE
    return O.E_CHARGE * D / h * max(np.abs(ne[sl]).max(), np.abs(b.n_ion[:, sl]).max())


@pytest.mark.parametrize("bc", [S.BC_ABSORBING, S.BC_ZERO_GRADIENT])
def test_current_matches_oracle(bc):
    d = dev()
    b = with_species(make_batch("ragged", 24, 41, n_range=(0, 900), dt=1e-7), 3)
    s = S.Solver(S.default_params(bc_electron=bc), max_cols=b.ncol, max_cells=max(b.ncells, 2),
                 max_col_cells=max(int(b.lengths().max()), 2))
    db = S.DeviceBatch.from_host(b, d)
    ne = b.ne_old * (1.0 + 0.1 * np.sin(np.arange(b.ncells)))
    phi = b.phi_old + 3.0 * np.cos(np.arange(b.ncells) * 0.05)
    t = lambda a: torch.as_tensor(a, device=d)
    jp, jn = s.current(db, t(ne), t(phi), 4e-3)
    torch.cuda.synchronize()
    jp, jn = jp.cpu().numpy(), jn.cpu().numpy()
    rp, rn = O.current(b, ne, phi, 4e-3, O.default_params(bc_electron=bc))
    for c in range(b.ncol):
        f = slice(b.col_off[c] + c, b.col_off[c + 1] + c + 1)
        if b.col_off[c + 1] - b.col_off[c] < 2:
            assert (jp[f] == 0).all() and (jn[f] == 0).all()
            continue
        sc = flux_scale(b, c, ne)
        assert np.abs(jp[f] - rp[f]).max() <= 1e-12 * sc, c
        assert np.abs(jn[f] - rn[f]).max() <= 1e-12 * sc, c


def test_current_of_the_solved_state_matches_oracle():
    d = dev()
    b = make_batch("ragged", 16, 8, n_range=(100, 1200), dt=3e-7)
    s = S.Solver(S.default_params(eps_F=1e-12), max_cols=b.ncol, max_cells=b.ncells,
                 max_col_cells=int(b.lengths().max()))
    db = S.DeviceBatch.from_host(b, d)
    out = s.solve(db)
    jp, jn = s.current(db, out["ne"], out["phi"])
    torch.cuda.synchronize()
    ne, phi = out["ne"].cpu().numpy(), out["phi"].cpu().numpy()
    rp, rn = O.current(b, ne, phi)
    jp, jn = jp.cpu().numpy(), jn.cpu().numpy()
    for c in range(b.ncol):
        f = slice(b.col_off[c] + c, b.col_off[c + 1] + c + 1)
        sc = flux_scale(b, c, ne)
        assert np.abs(jp[f] - rp[f]).max() <= 1e-12 * sc
        assert np.abs(jn[f] - rn[f]).max() <= 1e-12 * sc
    # the electron current divergence matches the solved density change
    for c in range(b.ncol):
        sl = slice(b.col_off[c], b.col_off[c + 1])
        f = slice(b.col_off[c] + c, b.col_off[c + 1] + c + 1)
        h, dt = b.length[c] / (sl.stop - sl.start), b.dt[c]
        lhs = np.diff(jn[f])
        rhs = -O.E_CHARGE * (h / dt) * (b.ne_old[sl] - ne[sl])
        assert np.abs(lhs - rhs).max() <= 1e-9 * O.E_CHARGE * (h / dt) * np.abs(b.ne_old[sl]).max()
