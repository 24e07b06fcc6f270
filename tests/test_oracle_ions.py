"""Pins of the oracle's provisional ion update (Sec. 3.1 / Algorithm 1:
effective-velocity advection by a second-order Godunov scheme, implicit ion
diffusion, the SDC diffusion correction (D n^n - D n^(k)) / 2) against exact
solutions: a shift by one cell at CFL 1, conservation up to the electrode
outflow, the decay of a discrete Neumann eigenmode under backward-Euler
diffusion, the correction term on an eigenmode, and third-order one-step
error (second-order scheme) for a smooth monotone profile."""
import numpy as np
import pytest

import oracle as O
from paper_1904_08510_gb300.workload import uniform_batch

KAPPA = 4e-3
L = 0.01


def column(N, *, T=1500.0, dv=0.0, dt=1e-7, n_ion=None):
    b = uniform_batch(1, N, ne=1e14, n_ion=1e15, T=T, v_left=0.0, v_right=dv, dt=dt)
    if n_ion is not None:
        b.n_ion = np.atleast_2d(np.asarray(n_ion, dtype=float))
    return b


def test_cfl_one_is_an_exact_shift():
    """Uniform field pushing the cation to the right at CFL 1 and negligible
    diffusion (T = 1e-9 K): every value moves one cell; nothing enters at the
    left electrode and the last cell's content leaves at the right one."""
    N = 50
    n0 = np.random.default_rng(1).uniform(1e14, 1e16, N)
    dv = -300.0                              # E = 3e4 V/m > 0, w = kappa E
    w = KAPPA * (-dv / L)
    b = column(N, T=1e-9, dv=dv, dt=(L / N) / w, n_ion=n0)
    out = O.ion_provisional(b, b.phi_old, kappa_ion=KAPPA)[0]
    np.testing.assert_allclose(out, np.concatenate([[0.0], n0[:-1]]), rtol=1e-11, atol=1e-13 * n0.max())


def test_conservation_up_to_electrode_outflow():
    N = 120
    rng = np.random.default_rng(2)
    b = column(N, T=1800.0, dv=200.0, dt=2e-6, n_ion=rng.uniform(1e14, 1e16, N))
    b.phi_old = b.phi_old + 5.0 * np.sin(np.arange(N) * 0.3)
    prev = b.n_ion * (1.0 + 0.2 * rng.standard_normal(N))
    out = O.ion_provisional(b, b.phi_old, n_prev=prev, kappa_ion=KAPPA)[0]
    h, p = L / N, b.phi_old
    GL = (-8.0 * 0.0 + 9.0 * p[0] - p[1]) / (3.0 * h)
    GR = (8.0 * 200.0 - 9.0 * p[-1] + p[-2]) / (3.0 * h)
    wl, wr = -KAPPA * GL, -KAPPA * GR
    out_l = -wl * b.n_ion[0, 0] if wl < 0 else 0.0
    out_r = wr * b.n_ion[0, -1] if wr > 0 else 0.0
    expect = b.n_ion[0].sum() - b.dt[0] / h * (out_l + out_r)
    assert abs(out.sum() - expect) <= 1e-12 * b.n_ion[0].sum()


@pytest.mark.parametrize("j", [1, 3, 10])
def test_backward_euler_diffusion_of_a_neumann_mode(j):
    """No field, uniform T: v_i = cos(pi j (i + 1/2) / N) satisfies
    D_h v = -(4 D / h^2) sin^2(pi j / (2N)) v with no-flux ends, so
    n~ = 1 + v / (1 + dt (4D/h^2) sin^2(pi j / 2N))."""
    N, T, dt = 64, 1500.0, 3e-4
    i = np.arange(N)
    v = 1e14 * np.cos(np.pi * j * (i + 0.5) / N)
    b = column(N, T=T, dv=0.0, dt=dt, n_ion=1e15 + v)
    out = O.ion_provisional(b, np.zeros(N), kappa_ion=KAPPA)[0]
    D = KAPPA * O.K_B * T / O.E_CHARGE
    h = L / N
    lam = -(4.0 * D / h ** 2) * np.sin(np.pi * j / (2 * N)) ** 2
    np.testing.assert_allclose(out, 1e15 + v / (1.0 - dt * lam), rtol=1e-12)


def test_sdc_diffusion_correction_on_an_eigenmode():
    """n_prev = n^n + d with D_h d = lam d: the right-hand side gains
    -(dt/2) lam d, so n~ changes by -(dt/2) lam d / (1 - dt lam)."""
    N, T, dt, j = 48, 1200.0, 2e-4, 5
    i = np.arange(N)
    d = 1e13 * np.cos(np.pi * j * (i + 0.5) / N)
    b = column(N, T=T, dv=0.0, dt=dt, n_ion=np.full(N, 1e15))
    base = O.ion_provisional(b, np.zeros(N), kappa_ion=KAPPA)[0]
    corr = O.ion_provisional(b, np.zeros(N), n_prev=b.n_ion + d, kappa_ion=KAPPA)[0]
    D = KAPPA * O.K_B * T / O.E_CHARGE
    lam = -(4.0 * D / (L / N) ** 2) * np.sin(np.pi * j / (2 * N)) ** 2
    np.testing.assert_allclose(corr - base, -0.5 * dt * lam * d / (1.0 - dt * lam),
                               rtol=1e-9, atol=1e-9 * 1e13)


def test_second_order_godunov_one_step_error():
    """A tanh front (monotone, so the limiter keeps the central slope except
    in the flat tails) advected one step at CFL 0.5 with negligible
    diffusion: the error against the exact shifted cell averages falls as h^3
    (local error of a second-order scheme), against h^2 for first-order
    upwinding (the drift-only update)."""
    ell, x0, dv = 8e-4, 4e-3, -200.0
    w = KAPPA * (-dv / L)
    errs, errs1 = [], []
    for N in (128, 256, 512):
        h = L / N
        dt = 0.5 * h / w
        xf = np.arange(N + 1) * h
        prim = lambda x: ell * np.log(np.cosh((x - x0) / ell))
        avg = lambda s: 1e15 * (1.5 + (prim(xf[1:] - s) - prim(xf[:-1] - s)) / h)
        b = column(N, T=1e-9, dv=dv, dt=dt, n_ion=avg(0.0))
        out = O.ion_provisional(b, b.phi_old, kappa_ion=KAPPA)[0]
        first = O.ion_update(b, b.phi_old, KAPPA)[0]
        ex = avg(w * dt)
        inner = slice(N // 8, N - N // 8)
        errs.append(np.abs(out - ex)[inner].max())
        errs1.append(np.abs(first - ex)[inner].max())
    order = np.log2(errs[0] / errs[1]), np.log2(errs[1] / errs[2])
    order1 = np.log2(errs1[0] / errs1[1]), np.log2(errs1[1] / errs1[2])
    assert min(order) > 2.6, order
    assert max(order1) < 2.3, order1
    assert errs[-1] < 0.05 * errs1[-1]
