"""CPU FP64 oracle for the implicit electron / potential JFNK solve.

TEST INFRASTRUCTURE: only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package. The CUDA product path
never does, and the two share no code.

The arithmetic lives in ``oracle.c`` (plain C, IEEE double, one column per
OpenMP thread); this module compiles it with gcc on first use and marshals
numpy arrays through ctypes. Every function follows Sec. 3.2 and Algorithm 2
of arXiv:1904.08510 as documented in ``oracle.c``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, MAX_NEWTON, MAX_KRYLOV, LINESEARCH_FAIL, NONFINITE, BAD_INPUT = range(6)
BC_ABSORBING, BC_ZERO_GRADIENT = 0, 1

# physical constants (SI, CODATA 2018) as used by oracle.c
E_CHARGE = 1.602176634e-19
K_B = 1.380649e-23
EPS0 = 8.8541878128e-12


class Params(C.Structure):
    _fields_ = [("eps_F", C.c_double), ("eps_X", C.c_double), ("gamma", C.c_double),
                ("mobility", C.c_double), ("ls_alpha", C.c_double), ("eps_r", C.c_double),
                ("restart_m", C.c_int), ("max_newton", C.c_int), ("max_krylov", C.c_int),
                ("max_linesearch", C.c_int), ("bc_electron", C.c_int), ("precond", C.c_int),
                ("mg_gamma_A", C.c_double), ("mg_gamma_S", C.c_double),
                ("mg_max_cycles", C.c_int), ("mg_transfer", C.c_int),
                ("transport", C.c_int), ("tab_mu", C.c_void_p), ("tab_D", C.c_void_p),
                ("tab_nc", C.c_int), ("tab_nx", C.c_int), ("tab_en_max", C.c_double),
                ("T_in", C.c_double), ("T_max", C.c_double), ("gas_molar_mass", C.c_double),
                ("eps_E", C.c_double)]

PREC_NONE, PREC_RECAST, PREC_EXACT, PREC_MG = 0, 1, 2, 3
MG_OPERATOR, MG_LINEAR = 0, 1
TRANSPORT_CONSTANT, TRANSPORT_TABLE = 0, 1


class _Batch(C.Structure):
    _fields_ = [("ncol", C.c_int64), ("col_off", C.c_void_p), ("length", C.c_void_p),
                ("dt", C.c_void_p), ("v_left", C.c_void_p), ("v_right", C.c_void_p),
                ("ne_old", C.c_void_p), ("phi_old", C.c_void_p), ("n_species", C.c_int),
                ("valence", C.c_void_p), ("n_ion", C.c_void_p), ("T", C.c_void_p),
                ("u_adv", C.c_void_p), ("i_re", C.c_void_p), ("rho", C.c_void_p)]


def default_params(**kw) -> Params:
    """Defaults: eps_F = 1e-10, error test eps_E = 5e-10 (see or_jfnk_col),
    gamma = 1e-4 (Table 1), mobility 0.4 m^2/(V s)
    (Sec. 2.2), GMRES(30), 50 Newton steps, 200 Krylov iterations per step,
    20 line-search halvings, absorbing electrodes, recast Schur preconditioner;
    with precond=PREC_MG its blocks are solved by V-cycles to gamma_MG = 1e-4
    (Sec. 4.2), at most 100 per block solve."""
    p = dict(eps_F=1e-10, eps_X=0.0, gamma=1e-4, mobility=0.4, ls_alpha=1e-4, eps_r=1.0,
             restart_m=30, max_newton=50, max_krylov=200, max_linesearch=20,
             bc_electron=BC_ABSORBING, precond=PREC_RECAST, mg_gamma_A=1e-4, mg_gamma_S=1e-4,
             mg_max_cycles=100, mg_transfer=MG_OPERATOR, transport=TRANSPORT_CONSTANT,
             gas_molar_mass=0.028, T_in=300.0, T_max=2000.0, eps_E=5e-10)
    table = kw.pop("table", None)
    p.update(kw)
    P = Params(**p)
    if table is not None:
        set_table(P, table)
    return P


def tab_lookup(t, en_max, c, x):
    """The oracle's bilinear table interpolation at (c, E/N = x Td)."""
    t = np.ascontiguousarray(t, dtype=np.float64)
    return lib().or_tab_lookup(_ptr(t), t.shape[0], t.shape[1], float(en_max), float(c), float(x))


def set_table(P, table):
    """Point P at a transport table (dict mu, D [nc, nx] arrays, en_max_td,
    T_in, T_max) and switch P to TRANSPORT_TABLE. The arrays are kept alive on P."""
    mu = np.ascontiguousarray(table["mu"], dtype=np.float64)
    D = np.ascontiguousarray(table["D"], dtype=np.float64)
    P._keep = (mu, D)
    P.transport = TRANSPORT_TABLE
    P.tab_mu, P.tab_D = mu.ctypes.data, D.ctypes.data
    P.tab_nc, P.tab_nx = mu.shape
    P.tab_en_max = float(table["en_max_td"])
    P.T_in, P.T_max = float(table["T_in"]), float(table["T_max"])
    return P


def build(force: bool = False) -> str:
    """Compile oracle.c into a shared library (gcc, -O2, OpenMP)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            os.makedirs(_BUILD, exist_ok=True)
            tmp = _LIB + f".{os.getpid()}.tmp"
            subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
                                   "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        P = C.POINTER(Params)
        B = C.POINTER(_Batch)
        vp = C.c_void_p
        L.or_bern.restype = C.c_double
        L.or_bern.argtypes = [C.c_double]
        L.or_bern_deriv.restype = C.c_double
        L.or_bern_deriv.argtypes = [C.c_double]
        L.or_residual_batch.argtypes = [P, B, vp, vp, vp, vp]
        L.or_jacobian_batch.argtypes = [P, B, vp, vp, vp, vp, vp]
        L.or_prec_apply_col.argtypes = [P, B, C.c_int64, vp, vp, vp, vp, vp, vp, vp]
        L.or_solve_batch.argtypes = [P, B, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, C.c_int]
        L.or_mg_solve_tri.restype = C.c_int
        L.or_mg_solve_tri.argtypes = [C.c_int, vp, vp, vp, vp, vp, C.c_double, C.c_int, C.c_int]
        L.or_mg_hierarchy.restype = C.c_int
        L.or_mg_hierarchy.argtypes = [C.c_int, vp, vp, vp, C.c_int, vp, vp]
        L.or_mg_transfers.argtypes = [C.c_int, vp, vp, vp, C.c_int, vp, vp]
        L.or_thomas.argtypes = [C.c_int, vp, vp, vp, vp, vp, vp]
        L.or_gmres_dense.restype = C.c_int
        L.or_gmres_dense.argtypes = [C.c_int, vp, vp, vp, C.c_int, C.c_double, C.c_int,
                                     C.POINTER(C.c_int), C.POINTER(C.c_double)]
        L.or_max_threads.restype = C.c_int
        L.or_ion_update_batch.argtypes = [B, vp, C.c_double, vp]
        L.or_current_batch.argtypes = [P, B, vp, vp, C.c_double, vp, vp]
        L.or_tab_lookup.restype = C.c_double
        L.or_tab_lookup.argtypes = [vp, C.c_int, C.c_int, C.c_double, C.c_double, C.c_double]
        L.or_ion_provisional_batch.argtypes = [B, vp, vp, C.c_double, vp]
        _lib = L
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return None if a is None else a.ctypes.data


class _Keep:
    """Holds the contiguous copies referenced by a ctypes batch struct."""

    def __init__(self, batch):
        self.col_off = np.ascontiguousarray(batch.col_off, dtype=np.int64)
        self.length = _f64(batch.length)
        self.dt = _f64(batch.dt)
        self.v_left = _f64(batch.v_left)
        self.v_right = _f64(batch.v_right)
        self.ne_old = _f64(batch.ne_old)
        self.phi_old = _f64(batch.phi_old)
        self.n_ion = _f64(np.atleast_2d(batch.n_ion))
        self.valence = np.ascontiguousarray(batch.valence, dtype=np.int32)
        self.T = _f64(batch.T)
        self.u_adv = None if batch.u_adv is None else _f64(batch.u_adv)
        self.i_re = None if batch.i_re is None else _f64(batch.i_re)
        self.rho = None if getattr(batch, "rho", None) is None else _f64(batch.rho)
        self.s = _Batch(self.col_off.shape[0] - 1, _ptr(self.col_off), _ptr(self.length),
                        _ptr(self.dt), _ptr(self.v_left), _ptr(self.v_right),
                        _ptr(self.ne_old), _ptr(self.phi_old), self.n_ion.shape[0],
                        _ptr(self.valence), _ptr(self.n_ion), _ptr(self.T),
                        _ptr(self.u_adv), _ptr(self.i_re), _ptr(self.rho))


def bern(x: float) -> float:
    """B(x) = x / (e^x - 1) as evaluated by the oracle."""
    return lib().or_bern(float(x))


def bern_deriv(x: float) -> float:
    return lib().or_bern_deriv(float(x))


def residual(batch, ne, phi, params: Params | None = None):
    """F(X) of Eq. nls for every column: returns (F_e, F_phi), each [cells]."""
    P = params or default_params()
    k = _Keep(batch)
    ne, phi = _f64(ne), _f64(phi)
    Fe = np.zeros(batch.ncells)
    Fp = np.zeros(batch.ncells)
    lib().or_residual_batch(C.byref(P), C.byref(k.s), _ptr(ne), _ptr(phi), _ptr(Fe), _ptr(Fp))
    return Fe, Fp


def jacobian_blocks(batch, ne, phi, params: Params | None = None):
    """Analytic tridiagonal blocks (A, B, L), each an array [3, cells] of
    (sub, diag, sup); C = dF_phi/dn = -I (Eq. linear_nls)."""
    P = params or default_params()
    k = _Keep(batch)
    ne, phi = _f64(ne), _f64(phi)
    n = batch.ncells
    A = np.zeros((3, n))
    B = np.zeros((3, n))
    Lm = np.zeros((3, n))
    lib().or_jacobian_batch(C.byref(P), C.byref(k.s), _ptr(ne), _ptr(phi), _ptr(A), _ptr(B),
                            _ptr(Lm))
    return A, B, Lm


def prec_apply(batch, c, ne, phi, v1, v2, params: Params | None = None, *,
               return_cycles: bool = False):
    """Preconditioner params.precond (recast Schur form of Eq. prec_recast by
    default) of column c built at X, applied to (v1, v2) in unscaled units. With
    return_cycles, also the V-cycles the multigrid block solves took."""
    P = params or default_params()
    k = _Keep(batch)
    ne, phi, v1, v2 = _f64(ne), _f64(phi), _f64(v1), _f64(v2)
    x1 = np.zeros_like(v1)
    x2 = np.zeros_like(v2)
    cyc = C.c_int(0)
    lib().or_prec_apply_col(C.byref(P), C.byref(k.s), int(c), _ptr(ne), _ptr(phi), _ptr(v1),
                            _ptr(v2), _ptr(x1), _ptr(x2), C.addressof(cyc))
    return (x1, x2, cyc.value) if return_cycles else (x1, x2)


def mg_solve_tri(sub, dia, sup, b, gamma, max_cycles=100, transfer=MG_OPERATOR):
    """Multigrid V-cycles (Sec. 4.2) on one tridiagonal system from x = 0 until
    ||b - T x||_2 <= gamma ||b||_2 (or no progress); returns (x, cycles)."""
    sub, dia, sup, b = _f64(sub), _f64(dia), _f64(sup), _f64(b)
    x = np.zeros_like(b)
    k = lib().or_mg_solve_tri(b.shape[0], _ptr(sub), _ptr(dia), _ptr(sup), _ptr(b), _ptr(x),
                              float(gamma), int(max_cycles), int(transfer))
    return x, int(k)


def mg_hierarchy(sub, dia, sup, transfer=MG_OPERATOR):
    """The multigrid levels of a tridiagonal matrix: a list of (sub, dia, sup)."""
    sub, dia, sup = _f64(sub), _f64(dia), _f64(sup)
    n = sub.shape[0]
    sizes = np.zeros(64, dtype=np.int32)
    out = np.zeros(3 * 2 * n + 64)
    nl = lib().or_mg_hierarchy(n, _ptr(sub), _ptr(dia), _ptr(sup), int(transfer), _ptr(sizes),
                               _ptr(out))
    levels, o = [], 0
    for m in sizes[:nl]:
        levels.append((out[o:o + m].copy(), out[o + m:o + 2 * m].copy(), out[o + 2 * m:o + 3 * m].copy()))
        o += 3 * m
    return levels


def mg_transfers(sub, dia, sup, transfer=MG_OPERATOR):
    """Dense prolongation P (n x n/2) and restriction R (n/2 x n) of the finest level."""
    sub, dia, sup = _f64(sub), _f64(dia), _f64(sup)
    n = sub.shape[0]
    P = np.zeros((n, n // 2))
    R = np.zeros((n // 2, n))
    lib().or_mg_transfers(n, _ptr(sub), _ptr(dia), _ptr(sup), int(transfer), _ptr(P), _ptr(R))
    return P, R


def thomas(sub, dia, sup, d):
    sub, dia, sup, d = _f64(sub), _f64(dia), _f64(sup), _f64(d)
    n = d.shape[0]
    x = np.zeros(n)
    w = np.zeros(2 * n)
    lib().or_thomas(n, _ptr(sub), _ptr(dia), _ptr(sup), _ptr(d), _ptr(x), _ptr(w))
    return x


def gmres_dense(M, b, m, tol, maxit):
    """The oracle's GMRES routine on a dense operator (no preconditioner)."""
    M = _f64(M)
    b = _f64(b)
    n = b.shape[0]
    x = np.zeros(n)
    it = C.c_int(0)
    est = C.c_double(0)
    conv = lib().or_gmres_dense(n, _ptr(M), _ptr(b), _ptr(x), int(m), float(tol), int(maxit),
                                C.byref(it), C.byref(est))
    return x, bool(conv), it.value, est.value


def solve(batch, params: Params | None = None, *, guess=None, threads: int = 0):
    """JFNK (Algorithm 2) on every column. Returns a dict with ne, phi, status,
    newton_it, krylov_it, res_evals, final_res and mg_cycles (V-cycles of the
    multigrid block solves, precond=PREC_MG)."""
    P = params or default_params()
    k = _Keep(batch)
    n = batch.ncells
    ncol = batch.ncol
    ne = np.zeros(n)
    phi = np.zeros(n)
    status = np.zeros(ncol, dtype=np.int32)
    newton = np.zeros(ncol, dtype=np.int32)
    krylov = np.zeros(ncol, dtype=np.int32)
    evals = np.zeros(ncol, dtype=np.int32)
    fres = np.zeros(ncol)
    mgc = np.zeros(ncol, dtype=np.int32)
    g_ne = g_phi = None
    if guess is not None:
        g_ne, g_phi = _f64(guess[0]), _f64(guess[1])
    lib().or_solve_batch(C.byref(P), C.byref(k.s), _ptr(g_ne), _ptr(g_phi), _ptr(ne), _ptr(phi),
                         _ptr(status), _ptr(newton), _ptr(krylov), _ptr(evals), _ptr(fres),
                         _ptr(mgc), int(threads))
    return dict(ne=ne, phi=phi, status=status, newton_it=newton, krylov_it=krylov,
                res_evals=evals, final_res=fres, mg_cycles=mgc)


def max_threads() -> int:
    return int(lib().or_max_threads())


def ion_update(batch, phi, kappa_ion=4e-3):
    """Provisional ion densities after one explicit upwind drift step in the field
    of phi ([n_species, cells])."""
    k = _Keep(batch)
    phi = _f64(phi)
    out = np.zeros_like(k.n_ion)
    lib().or_ion_update_batch(C.byref(k.s), _ptr(phi), float(kappa_ion), _ptr(out))
    return out


def ion_provisional(batch, phi, n_prev=None, kappa_ion=4e-3):
    """Provisional ion densities of an SDC iteration with second-order Godunov
    drift/advection, implicit diffusion and the SDC diffusion correction
    against the previous iterate n_prev ([n_species, cells]; None = n^n)."""
    k = _Keep(batch)
    phi = _f64(phi)
    npv = None if n_prev is None else _f64(np.atleast_2d(n_prev))
    out = np.zeros_like(k.n_ion)
    lib().or_ion_provisional_batch(C.byref(k.s), _ptr(phi), _ptr(npv), float(kappa_ion), _ptr(out))
    return out


def current(batch, ne, phi, kappa_ion=4e-3, params: Params | None = None):
    """Charge flux density through every face (Sec. 4.4): (J+, J-) [A/m^2], each
    [cells + ncol], the N + 1 faces of column c starting at col_off[c] + c."""
    P = params or default_params()
    k = _Keep(batch)
    ne, phi = _f64(ne), _f64(phi)
    jp = np.zeros(batch.ncells + batch.ncol)
    jn = np.zeros_like(jp)
    lib().or_current_batch(C.byref(P), C.byref(k.s), _ptr(ne), _ptr(phi), float(kappa_ion),
                           _ptr(jp), _ptr(jn))
    return jp, jn


def sdc_sweep(batch, k_max=4, kappa_ion=4e-3, params: Params | None = None, guess=None,
              scheme="godunov"):
    """The electric part of one MISDC step (Algorithm 1): for k = 1..k_max the
    provisional ions are advanced from n_ion^n in the field of the previous
    iterate (scheme "godunov": ion_provisional with the previous iteration's
    provisional ions as n^(k); "drift": ion_update) and the implicit
    electron/potential system is solved from the previous iterate (X^0 = X^n,
    or the given guess for k = 1)."""
    from copy import copy
    P = params or default_params()
    ne, phi = batch.ne_old.copy(), batch.phi_old.copy()
    start = guess
    hist = []
    prev = None
    for k in range(k_max):
        bk = copy(batch)
        if scheme == "godunov":
            bk.n_ion = ion_provisional(batch, phi, prev, kappa_ion)
            prev = bk.n_ion
        else:
            bk.n_ion = ion_update(batch, phi, kappa_ion)
        g = start if start is not None else ((ne, phi) if k > 0 else None)
        r = solve(bk, P, guess=g)
        ne, phi = r["ne"], r["phi"]
        start = None
        hist.append(r)
    return ne, phi, hist
