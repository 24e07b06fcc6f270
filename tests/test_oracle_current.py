"""Pins of the oracle's charge-flux diagnostic (Sec. 4.4: J_m = nu_m e Gamma_m,
J+ over positive ions, J- over negative species and electrons) against closed
forms (Ohm's law in a uniform plasma, Fick's law for linear profiles, the sign
of the electrode outflow) and against the residual of Eq. nls at a converged
root (the divergence of the electron flux equals the density change)."""
import numpy as np

import oracle as O
from paper_1904_08510_gb300.workload import make_batch, uniform_batch

E = O.E_CHARGE
KB = O.K_B
MU = 0.4
KAPPA = 4e-3


def faces(b, c):
    return slice(b.col_off[c] + c, b.col_off[c + 1] + c + 1)


def test_ohms_law_uniform_plasma():
    """Uniform n_e = n_i = n and T, linear phi: every interior face carries
    J+ = e n kappa E and J- = e n mu E (the Scharfetter-Gummel flux of a
    uniform density is n v exactly, B(-x) - B(x) = x)."""
    n, dv, L = 3e15, 250.0, 0.01
    b = uniform_batch(2, 80, ne=n, n_ion=n, T=1200.0, v_left=0.0, v_right=dv, dt=1e-7)
    jp, jn = O.current(b, b.ne_old, b.phi_old, KAPPA)
    Ef = -dv / L
    for c in range(b.ncol):
        f = faces(b, c)
        np.testing.assert_allclose(jp[f][1:-1], E * n * KAPPA * Ef, rtol=1e-12)
        np.testing.assert_allclose(jn[f][1:-1], E * n * MU * Ef, rtol=1e-10)


def test_ficks_law_linear_profiles():
    """No field (phi = 0 everywhere), uniform T, linear densities: J- = e D_e
    dn_e/dx and J+ = -e D_i dn_i/dx at interior faces, D = mobility k_B T / e."""
    N, L, T = 64, 0.01, 900.0
    b = uniform_batch(1, N, ne=1e15, n_ion=1e15, T=T, v_left=0.0, v_right=0.0, dt=1e-7)
    x = (np.arange(N) + 0.5) * L / N
    ne = 1e15 + 4e16 * x
    b.n_ion = (2e15 - 1e17 * x)[None, :]
    jp, jn = O.current(b, ne, np.zeros(N), KAPPA)
    De, Di = MU * KB * T / E, KAPPA * KB * T / E
    np.testing.assert_allclose(jn[1:-1], E * De * 4e16, rtol=1e-10)
    np.testing.assert_allclose(jp[1:-1], -E * Di * (-1e17), rtol=1e-10)


def test_electrode_faces_pass_outgoing_drift_only():
    """V_R > V_L: electrons drift toward the right electrode and leave there,
    positive ions drift toward the left one; neither enters (absorbing)."""
    n, N = 2e15, 40
    b = uniform_batch(1, N, ne=n, n_ion=n, T=1500.0, v_left=0.0, v_right=100.0, dt=1e-7)
    jp, jn = O.current(b, b.ne_old, b.phi_old, KAPPA)
    G = 100.0 / 0.01                    # the electrode stencil is exact for linear phi
    assert jn[0] == 0.0 and jp[-1] == 0.0
    np.testing.assert_allclose(jn[-1], -E * (MU * G) * n, rtol=1e-12)
    np.testing.assert_allclose(jp[0], E * (-KAPPA * G) * n, rtol=1e-12)


def test_electron_current_divergence_matches_the_root():
    """At a root of Eq. nls (I_Re = 0): (dt/h)(Gam_{i+1/2} - Gam_{i-1/2}) =
    n_e^n_i - n_i, i.e. J-_{i+1/2} - J-_{i-1/2} = -e (h/dt)(n^n_i - n_i) with one
    positive ion species (J- is the electron current alone)."""
    b = make_batch("single", 3, 5, n_cells=200, dt=1e-7)
    r = O.solve(b, O.default_params(eps_F=1e-12))
    assert (r["status"] == 0).all()
    jp, jn = O.current(b, r["ne"], r["phi"], KAPPA)
    for c in range(b.ncol):
        sl = slice(b.col_off[c], b.col_off[c + 1])
        h, dt = b.length[c] / (sl.stop - sl.start), b.dt[c]
        lhs = np.diff(jn[faces(b, c)])
        rhs = -E * (h / dt) * (b.ne_old[sl] - r["ne"][sl])
        scale = E * (h / dt) * np.abs(b.ne_old[sl]).max()
        assert np.abs(lhs - rhs).max() <= 1e-9 * scale
