"""Seeded synthetic inputs for the implicit electron / potential solve.

This module only draws the input fields of a batch of independent 1D
columns; it contains none of the solver's arithmetic, so the CPU oracle and
the CUDA path can both be fed from it.

Profiles (per column, uniform cells on a domain of length L):
  T(x)   = 300 + 1700 (1 + tanh((x - x_f) / 0.5 mm)) / 2          [K]
  rho(x) = p0 W / (R_u T)   with p0 = 101325 Pa, W = 28 g/mol        [kg/m^3]
           (ideal-gas equation of state, Sec. 2.1 Eq. EOS)
  n_ion  = A exp(-((x - x_f) / w)^2 / 2),  w = 0.3 mm (std. dev.)   [m^-3]
  n_e    = max(0, n_ion (1 - 0.01 N(0,1)))  (independent per cell)   [m^-3]
  phi    = V_L + (V_R - V_L) x / L,  V_L = 0                         [V]
The paper's own flame set-up (Sec. 4.1, Table 1: L = 1 cm, n_x in
[128, 2048]) fixes L and the range of cell counts; the flame itself needs a
chemical mechanism and is replaced by these profiles.

Each column c draws from its own PCG64 stream seeded with ``seed + c`` so a
column's inputs do not depend on the batch it sits in.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

L_DOMAIN = 0.01          # m (Table 1)
P0 = 101325.0            # Pa
W_MIX = 0.028            # kg/mol
R_U = 8.314462618        # J/(mol K)
T_FLAME_WIDTH = 0.0005   # m, tanh half-width of the temperature rise
ION_WIDTH = 0.0003       # m, Gaussian standard deviation of the ion peak


@dataclass
class Batch:
    """Structure-of-arrays batch: per-cell fields packed column after column."""
    col_off: np.ndarray            # int64 [ncol+1]
    length: np.ndarray             # float64 [ncol]  (m)
    dt: np.ndarray                 # float64 [ncol]  (s)
    v_left: np.ndarray             # float64 [ncol]  (V)
    v_right: np.ndarray            # float64 [ncol]  (V)
    ne_old: np.ndarray             # float64 [cells] (m^-3)
    phi_old: np.ndarray            # float64 [cells] (V)
    n_ion: np.ndarray              # float64 [n_species, cells] (m^-3)
    valence: np.ndarray            # int32 [n_species]
    T: np.ndarray                  # float64 [cells] (K)
    rho: np.ndarray                # float64 [cells] (kg/m^3)
    u_adv: np.ndarray | None = None   # float64 [cells] (m/s) or None
    i_re: np.ndarray | None = None    # float64 [cells] (m^-3 s^-1) or None
    meta: dict = field(default_factory=dict)

    @property
    def ncol(self) -> int:
        return int(self.col_off.shape[0] - 1)

    @property
    def ncells(self) -> int:
        return int(self.col_off[-1])

    def lengths(self) -> np.ndarray:
        return np.diff(self.col_off)

    def column(self, c: int) -> "Batch":
        """The single-column batch holding column ``c``."""
        a, b = int(self.col_off[c]), int(self.col_off[c + 1])
        sl = slice(a, b)
        return Batch(
            col_off=np.array([0, b - a], dtype=np.int64),
            length=self.length[c:c + 1].copy(), dt=self.dt[c:c + 1].copy(),
            v_left=self.v_left[c:c + 1].copy(), v_right=self.v_right[c:c + 1].copy(),
            ne_old=self.ne_old[sl].copy(), phi_old=self.phi_old[sl].copy(),
            n_ion=self.n_ion[:, sl].copy(), valence=self.valence.copy(),
            T=self.T[sl].copy(), rho=self.rho[sl].copy(),
            u_adv=None if self.u_adv is None else self.u_adv[sl].copy(),
            i_re=None if self.i_re is None else self.i_re[sl].copy(),
            meta=dict(self.meta, column=c))

    def subset(self, cols) -> "Batch":
        """A batch made of the listed columns, in the given order."""
        cols = [int(c) for c in cols]
        lens = np.array([self.col_off[c + 1] - self.col_off[c] for c in cols], dtype=np.int64)
        off = np.zeros(len(cols) + 1, dtype=np.int64)
        np.cumsum(lens, out=off[1:])
        idx = np.concatenate([np.arange(self.col_off[c], self.col_off[c + 1]) for c in cols]) \
            if cols else np.zeros(0, dtype=np.int64)
        return Batch(
            col_off=off, length=self.length[cols].copy(), dt=self.dt[cols].copy(),
            v_left=self.v_left[cols].copy(), v_right=self.v_right[cols].copy(),
            ne_old=self.ne_old[idx].copy(), phi_old=self.phi_old[idx].copy(),
            n_ion=self.n_ion[:, idx].copy(), valence=self.valence.copy(),
            T=self.T[idx].copy(), rho=self.rho[idx].copy(),
            u_adv=None if self.u_adv is None else self.u_adv[idx].copy(),
            i_re=None if self.i_re is None else self.i_re[idx].copy(),
            meta=dict(self.meta, subset=len(cols)))


def _column_fields(n, length, x_f, amp, v_left, v_right, rng):
    h = length / n
    x = (np.arange(n) + 0.5) * h
    T = 300.0 + 1700.0 * (1.0 + np.tanh((x - x_f) / T_FLAME_WIDTH)) / 2.0
    rho = P0 * W_MIX / (R_U * T)
    n_ion = amp * np.exp(-0.5 * ((x - x_f) / ION_WIDTH) ** 2)
    ne = np.maximum(0.0, n_ion * (1.0 - 0.01 * rng.standard_normal(n)))
    phi = v_left + (v_right - v_left) * x / length
    return ne, phi, n_ion, T, rho


def make_batch(kind: str, ncol: int, seed: int, *, n_cells=None, n_range=None,
               dt: float = 1e-5) -> Batch:
    """Draw ``ncol`` columns of one of the synthetic profile families.

    kind = "single": flame at 5 mm, ion peak 1e16 * U(0.5, 1.5), V_R ~ U(-300, 300),
                     n_cells cells per column (default 256), or cells ~ U{n_range}.
    kind = "ragged": cells ~ U{n_range} (default 128..2048), flame ~ U(3, 7) mm,
                     ion peak log-uniform in [1e15, 1e17], V_R ~ U(-500, 500).
    """
    cols = []
    for c in range(ncol):
        rng = np.random.Generator(np.random.PCG64(seed + c))
        if kind == "single":
            if n_range is not None and n_cells is None:
                n = int(rng.integers(n_range[0], n_range[1] + 1))
            else:
                n = 256 if n_cells is None else int(n_cells)
            amp = 1e16 * rng.uniform(0.5, 1.5)
            v_right = rng.uniform(-300.0, 300.0)
            x_f = 0.005
        elif kind == "ragged":
            lo, hi = (128, 2048) if n_range is None else n_range
            n = int(rng.integers(lo, hi + 1)) if n_cells is None else int(n_cells)
            x_f = rng.uniform(0.003, 0.007)
            amp = 10.0 ** rng.uniform(15.0, 17.0)
            v_right = rng.uniform(-500.0, 500.0)
        else:
            raise ValueError(f"unknown kind {kind!r}")
        fields = _column_fields(n, L_DOMAIN, x_f, amp, 0.0, v_right, rng)
        cols.append((n, v_right, fields))
    lens = np.array([c[0] for c in cols], dtype=np.int64)
    off = np.zeros(ncol + 1, dtype=np.int64)
    np.cumsum(lens, out=off[1:])
    cat = lambda k: np.concatenate([c[2][k] for c in cols]) if cols else np.zeros(0)
    return Batch(
        col_off=off,
        length=np.full(ncol, L_DOMAIN), dt=np.full(ncol, dt),
        v_left=np.zeros(ncol), v_right=np.array([c[1] for c in cols], dtype=np.float64),
        ne_old=cat(0), phi_old=cat(1), n_ion=cat(2)[None, :].copy(),
        valence=np.array([1], dtype=np.int32), T=cat(3), rho=cat(4),
        meta={"kind": kind, "seed": seed, "dt": dt})


def uniform_batch(ncol: int, n: int, *, ne: float, n_ion: float, T: float, v_left: float,
                  v_right: float, dt: float, length: float = L_DOMAIN) -> Batch:
    """Spatially uniform fields (used by closed-form checks)."""
    h = length / n
    x = (np.arange(n) + 0.5) * h
    phi = v_left + (v_right - v_left) * x / length
    off = np.arange(ncol + 1, dtype=np.int64) * n
    rep = lambda a: np.tile(a, ncol)
    return Batch(
        col_off=off, length=np.full(ncol, length), dt=np.full(ncol, dt),
        v_left=np.full(ncol, v_left), v_right=np.full(ncol, v_right),
        ne_old=np.full(ncol * n, ne), phi_old=rep(phi), n_ion=np.full((1, ncol * n), n_ion),
        valence=np.array([1], dtype=np.int32), T=np.full(ncol * n, T),
        rho=np.full(ncol * n, P0 * W_MIX / (R_U * T)), meta={"kind": "uniform"})


KAPPA_ION = 4e-3   # m^2/(V s): H3O+ mobility implied by the relaxation-time table (Sec. 4.4)


def transport_table(nc: int = 21, nx: int = 161, en_max_td: float = 400.0, t_in: float = 300.0,
                    t_max: float = 2000.0, mu_th: float = 0.4, e_mu: float = 20.0) -> dict:
    """Synthetic electron transport tables over the progress variable c and the
    reduced field E/N, standing in for the BOLSIG+ tables of the paper (not
    available): the thermal mobility mu_th (1 + (c - 1/2)/4) at low field,
    falling as 1/sqrt(1 + (E/N / e_mu)^2) with field heating; D = mu eps_k
    with the characteristic energy eps_k = k_B T(c)/e + 0.02 (E/N)^2 / (30 +
    E/N) V (E/N in Td), i.e. Einstein's relation at low field. Nodes: c_k =
    k/(nc - 1), E/N_j = j en_max/(nx - 1) Td."""
    kb_e = 1.380649e-23 / 1.602176634e-19
    c = np.linspace(0.0, 1.0, nc)[:, None]
    x = np.linspace(0.0, en_max_td, nx)[None, :]
    T = t_in + c * (t_max - t_in)
    mu = mu_th * (1.0 + 0.25 * (c - 0.5)) / np.sqrt(1.0 + (x / e_mu) ** 2)
    eps_k = kb_e * T + 0.02 * x ** 2 / (30.0 + x)
    return {"mu": np.ascontiguousarray(mu), "D": np.ascontiguousarray(mu * eps_k),
            "en_max_td": en_max_td, "T_in": t_in, "T_max": t_max}


def constant_transport_table(mobility: float = 0.4, nc: int = 11, nx: int = 5,
                             en_max_td: float = 400.0, t_in: float = 300.0,
                             t_max: float = 2000.0) -> dict:
    """The constant-mobility model written as a table: mu = mobility and
    Einstein D = mobility k_B T(c)/e, linear in c and independent of E/N."""
    kb_e = 1.380649e-23 / 1.602176634e-19
    c = np.linspace(0.0, 1.0, nc)[:, None]
    T = t_in + c * (t_max - t_in)
    mu = np.full((nc, nx), mobility)
    return {"mu": mu, "D": mobility * kb_e * T * np.ones((1, nx)), "en_max_td": en_max_td,
            "T_in": t_in, "T_max": t_max}


def sdc_batch(ncol: int, seed: int, *, n_cells: int = 1024, cfl: float = 0.5,
              kappa_ion: float = KAPPA_ION) -> Batch:
    """Columns of the "ragged" profile family with a fixed cell count and a time
    step set by the ion drift CFL: dt = cfl h / (kappa_ion |V_R - V_L| / L),
    the constant-CFL stepping of the paper's runs (Sec. 4.2)."""
    b = make_batch("ragged", ncol, seed, n_cells=n_cells)
    h = b.length / n_cells
    e = np.maximum(np.abs(b.v_right - b.v_left) / b.length, 1e3)
    b.dt = cfl * h / (kappa_ion * e)
    b.meta.update(kind="sdc", cfl=cfl, kappa_ion=kappa_ion)
    return b
