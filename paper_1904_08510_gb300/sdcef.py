"""Python binding of the sdcef C ABI (include/sdcef.h): argument marshalling only.

Every step of the solve runs in libsdcef.so; this module converts torch CUDA
tensors into the plain pointers of the C structs and raises when the
library is missing (there is no CPU fallback).
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# SDCEF_LIB selects another build of the library (the bounds-checking one in
# _build_checks/ for its tests); default: the in-tree _build/libsdcef.so
LIB_PATH = os.environ.get("SDCEF_LIB") or os.path.join(_HERE, "_build", "libsdcef.so")

SUCCESS = 0
ERR_INVALID, ERR_CUDA, ERR_CAPACITY, ERR_NOMEM = -1, -2, -3, -4
STATUS_OK, STATUS_MAX_NEWTON, STATUS_MAX_KRYLOV, STATUS_LINESEARCH_FAIL, \
    STATUS_NONFINITE, STATUS_BAD_INPUT = range(6)
FP64, MIXED, MIXED_DF = 0, 1, 2
PREC_EXACT, PREC_RECAST, PREC_NONE, PREC_MG = 0, 1, 2, 3
MG_OPERATOR, MG_LINEAR = 0, 1
ION_DRIFT_UPWIND, ION_GODUNOV = 0, 1
TRANSPORT_CONSTANT, TRANSPORT_TABLE = 0, 1
BC_ABSORBING, BC_ZERO_GRADIENT = 0, 1
MAX_RESTART = 32
MAX_SPECIES = 16

# every function declared in include/sdcef.h
EXPORTS = ("sdcef_default_params", "sdcef_create", "sdcef_destroy", "sdcef_set_params",
           "sdcef_solve_batch", "sdcef_solve_batch_host", "sdcef_residual_batch",
           "sdcef_precond_apply_batch", "sdcef_last_error", "sdcef_last_launch_count",
           "sdcef_solve_batch_noalloc", "sdcef_ion_update_batch", "sdcef_sdc_sweep",
           "sdcef_autotune", "sdcef_bernoulli_batch", "sdcef_current_batch",
           "sdcef_ion_provisional_batch", "sdcef_set_transport_table",
           "sdcef_mlp_create", "sdcef_mlp_destroy",
           "sdcef_mlp_set_params", "sdcef_mlp_get_params", "sdcef_mlp_features",
           "sdcef_mlp_targets", "sdcef_mlp_forward", "sdcef_mlp_grad", "sdcef_mlp_train_step",
           "sdcef_mlp_guess", "sdcef_mlp_last_launch_count", "sdcef_mlp_get_state",
           "sdcef_mlp_set_state", "sdcef_mlp_check", "sdcef_fma_peak_probe",
           "sdcef_mlp_set_wait_polls", "sdcef_checks_compiled", "sdcef_check_word",
           "sdcef_mlp_check_word", "sdcef_autotune_on_chip", "sdcef_solve_batches_host")
MLP_NPARAM = 20994
GUESS_NE, GUESS_PHI, GUESS_PHI_POISSON = 1, 2, 4
NOALLOC_SCRATCH_BYTES = 32 << 20
NOALLOC_MAX_COLS = 65536
NOALLOC_MAX_COL_CELLS = 4096


class Params(C.Structure):
    _fields_ = [("eps_F", C.c_double), ("eps_X", C.c_double), ("gamma", C.c_double),
                ("mobility", C.c_double), ("ls_alpha", C.c_double), ("eps_r", C.c_double),
                ("restart_m", C.c_int), ("max_newton", C.c_int), ("max_krylov", C.c_int),
                ("max_linesearch", C.c_int), ("precision", C.c_int), ("precond", C.c_int),
                ("bc_electron", C.c_int), ("threads_per_column", C.c_int),
                ("guess_newton_cap", C.c_int), ("guess_reject_ratio", C.c_double),
                ("mg_gamma_A", C.c_double), ("mg_gamma_S", C.c_double),
                ("mg_max_cycles", C.c_int), ("mg_transfer", C.c_int), ("ion_scheme", C.c_int),
                ("transport", C.c_int), ("gas_molar_mass", C.c_double), ("eps_E", C.c_double),
                ("stall_ratio", C.c_double), ("krylov_on_chip", C.c_int),
                ("guess_progress", C.c_double), ("sdc_poisson_start", C.c_int)]


class BatchC(C.Structure):
    _fields_ = [("ncol", C.c_int64), ("col_off", C.c_void_p), ("length", C.c_void_p),
                ("dt", C.c_void_p), ("v_left", C.c_void_p), ("v_right", C.c_void_p),
                ("ne_old", C.c_void_p), ("phi_old", C.c_void_p), ("n_species", C.c_int),
                ("valence", C.c_void_p), ("n_ion", C.c_void_p), ("T", C.c_void_p),
                ("rho", C.c_void_p), ("u_adv", C.c_void_p), ("i_re", C.c_void_p),
                ("ne_guess", C.c_void_p), ("phi_guess", C.c_void_p)]


class ResultC(C.Structure):
    _fields_ = [("ne_out", C.c_void_p), ("phi_out", C.c_void_p), ("status", C.c_void_p),
                ("newton_it", C.c_void_p), ("krylov_it", C.c_void_p), ("res_evals", C.c_void_p),
                ("final_res", C.c_void_p), ("mg_cycles", C.c_void_p)]


_lib = None


def lib():
    """Load libsdcef.so (built by paper_1904_08510_gb300.build); raise if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libsdcef.so not found at {LIB_PATH}; run "
                               "`python -c 'import __graft_entry__ as g; g.build()'` first")
        L = C.CDLL(LIB_PATH)
        P = C.POINTER(Params)
        B = C.POINTER(BatchC)
        R = C.POINTER(ResultC)
        vp = C.c_void_p
        L.sdcef_default_params.argtypes = [P]
        L.sdcef_default_params.restype = None
        L.sdcef_create.argtypes = [C.POINTER(vp), P, C.c_int64, C.c_int64, C.c_int, vp]
        L.sdcef_destroy.argtypes = [vp]
        L.sdcef_set_params.argtypes = [vp, P]
        L.sdcef_solve_batch.argtypes = [vp, B, R]
        L.sdcef_solve_batch_host.argtypes = [vp, B, R]
        L.sdcef_solve_batches_host.argtypes = [vp, C.c_int, vp, vp]
        L.sdcef_solve_batches_host.restype = C.c_int
        L.sdcef_residual_batch.argtypes = [vp, B, vp, vp, vp, vp]
        L.sdcef_bernoulli_batch.argtypes = [vp, vp, vp, vp, C.c_int64]
        L.sdcef_bernoulli_batch.restype = C.c_int
        L.sdcef_precond_apply_batch.argtypes = [vp, B, vp, vp, vp, vp, vp, vp, vp]
        L.sdcef_last_error.restype = C.c_char_p
        L.sdcef_last_error.argtypes = []
        L.sdcef_last_launch_count.argtypes = [vp]
        L.sdcef_solve_batch_noalloc.argtypes = [P, B, R, C.c_int, vp]
        L.sdcef_ion_update_batch.argtypes = [vp, B, vp, C.c_double, vp]
        L.sdcef_current_batch.argtypes = [vp, B, vp, vp, C.c_double, vp, vp]
        L.sdcef_ion_provisional_batch.argtypes = [vp, B, vp, vp, C.c_double, vp, vp]
        L.sdcef_set_transport_table.argtypes = [vp, C.c_int, C.c_int, C.c_double, C.c_double,
                                                C.c_double, vp, vp]
        L.sdcef_sdc_sweep.argtypes = [vp, B, C.c_int, C.c_double, vp, R]
        L.sdcef_ion_update_batch.restype = C.c_int
        L.sdcef_autotune.argtypes = [vp, B, R, C.c_int, C.POINTER(C.c_int), vp]
        L.sdcef_autotune.restype = C.c_int
        L.sdcef_autotune_on_chip.argtypes = [vp, B, R, C.c_int, C.POINTER(C.c_int), vp]
        L.sdcef_autotune_on_chip.restype = C.c_int
        L.sdcef_sdc_sweep.restype = C.c_int
        L.sdcef_fma_peak_probe.argtypes = [C.c_int, C.c_int, vp, C.POINTER(C.c_double)]
        L.sdcef_fma_peak_probe.restype = C.c_int
        i64 = C.c_int64
        L.sdcef_mlp_create.argtypes = [C.POINTER(vp), i64, vp]
        L.sdcef_mlp_destroy.argtypes = [vp]
        L.sdcef_mlp_set_params.argtypes = [vp, vp]
        L.sdcef_mlp_get_params.argtypes = [vp, vp]
        L.sdcef_mlp_features.argtypes = [vp, B, vp]
        L.sdcef_mlp_targets.argtypes = [vp, B, vp, vp, vp]
        L.sdcef_mlp_forward.argtypes = [vp, vp, i64, vp]
        L.sdcef_mlp_grad.argtypes = [vp, vp, vp, i64, vp, vp]
        L.sdcef_mlp_train_step.argtypes = [vp, vp, vp, i64, C.c_float, vp]
        L.sdcef_mlp_guess.argtypes = [vp, B, i64, C.c_int, vp, vp]
        L.sdcef_mlp_last_launch_count.argtypes = [vp]
        L.sdcef_mlp_check.argtypes = [vp]
        L.sdcef_mlp_set_wait_polls.argtypes = [vp, C.c_int]
        L.sdcef_checks_compiled.argtypes = []
        L.sdcef_checks_compiled.restype = C.c_int
        L.sdcef_check_word.argtypes = [vp, C.POINTER(C.c_uint)]
        L.sdcef_check_word.restype = C.c_int
        L.sdcef_mlp_check_word.argtypes = [vp, C.POINTER(C.c_uint)]
        L.sdcef_mlp_check_word.restype = C.c_int
        L.sdcef_mlp_get_state.argtypes = [vp, vp, vp, vp, C.POINTER(C.c_int64)]
        L.sdcef_mlp_set_state.argtypes = [vp, vp, vp, vp, i64]
        for f in ("sdcef_mlp_create", "sdcef_mlp_destroy", "sdcef_mlp_set_params",
                  "sdcef_mlp_get_params", "sdcef_mlp_features", "sdcef_mlp_targets",
                  "sdcef_mlp_forward", "sdcef_mlp_grad", "sdcef_mlp_train_step",
                  "sdcef_mlp_guess", "sdcef_mlp_last_launch_count", "sdcef_mlp_get_state",
                  "sdcef_mlp_set_state", "sdcef_mlp_check", "sdcef_mlp_set_wait_polls"):
            getattr(L, f).restype = C.c_int
        for f in ("sdcef_create", "sdcef_destroy", "sdcef_set_params", "sdcef_solve_batch",
                  "sdcef_solve_batch_host", "sdcef_residual_batch", "sdcef_precond_apply_batch",
                  "sdcef_last_launch_count", "sdcef_solve_batch_noalloc"):
            getattr(L, f).restype = C.c_int
        _lib = L
    return _lib


class SdcefError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"sdcef error {code}: {msg}")
        self.code = code


def _check(rc):
    if rc != SUCCESS:
        raise SdcefError(rc, lib().sdcef_last_error().decode())
    return rc


def default_params(**kw) -> Params:
    p = Params()
    lib().sdcef_default_params(C.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def _ptr(t):
    return None if t is None else t.data_ptr()


@dataclass
class DeviceBatch:
    """A workload.Batch resident on the GPU (torch tensors) plus its C struct."""
    ncol: int
    ncells: int
    tensors: dict
    valence: np.ndarray

    @classmethod
    def from_host(cls, b, device="cuda", guess=None):
        import torch
        t = lambda a: None if a is None else torch.as_tensor(np.ascontiguousarray(a)).to(device)
        ts = dict(col_off=t(b.col_off.astype(np.int64)), length=t(b.length), dt=t(b.dt),
                  v_left=t(b.v_left), v_right=t(b.v_right), ne_old=t(b.ne_old),
                  phi_old=t(b.phi_old), n_ion=t(np.atleast_2d(b.n_ion)), T=t(b.T),
                  rho=t(b.rho), u_adv=t(b.u_adv), i_re=t(b.i_re),
                  ne_guess=None if guess is None else t(guess[0]),
                  phi_guess=None if guess is None else t(guess[1]))
        return cls(b.ncol, b.ncells, ts, np.ascontiguousarray(b.valence, dtype=np.int32))

    def cstruct(self) -> BatchC:
        ts = self.tensors
        return BatchC(self.ncol, _ptr(ts["col_off"]), _ptr(ts["length"]), _ptr(ts["dt"]),
                      _ptr(ts["v_left"]), _ptr(ts["v_right"]), _ptr(ts["ne_old"]),
                      _ptr(ts["phi_old"]), int(self.valence.shape[0]),
                      self.valence.ctypes.data, _ptr(ts["n_ion"]), _ptr(ts["T"]),
                      _ptr(ts["rho"]), _ptr(ts["u_adv"]), _ptr(ts["i_re"]),
                      _ptr(ts["ne_guess"]), _ptr(ts["phi_guess"]))

    def with_guess(self, ne, phi) -> "DeviceBatch":
        ts = dict(self.tensors, ne_guess=ne, phi_guess=phi)
        return DeviceBatch(self.ncol, self.ncells, ts, self.valence)


class Solver:
    """Owns one sdcef context (workspace sized at construction)."""

    def __init__(self, params: Params | None = None, *, max_cols: int, max_cells: int,
                 max_col_cells: int, stream=None):
        import torch
        self.params = params or default_params()
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = C.c_void_p()
        _check(lib().sdcef_create(C.byref(h), C.byref(self.params), int(max_cols),
                                  int(max_cells), int(max_col_cells),
                                  C.c_void_p(stream.cuda_stream)))
        self.h = h
        self.max_cols, self.max_cells = max_cols, max_cells

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            lib().sdcef_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, p: Params):
        _check(lib().sdcef_set_params(self.h, C.byref(p)))
        self.params = p

    def launches(self) -> int:
        return int(lib().sdcef_last_launch_count(self.h))

    def check_word(self) -> int:
        """sdcef_check_word: the bounds-checking build's failed-check site (0 = none);
        synchronises and clears it."""
        w = C.c_uint(0)
        _check(lib().sdcef_check_word(self.h, C.byref(w)))
        return int(w.value)

    def alloc_result(self, db: DeviceBatch):
        import torch
        dev = db.tensors["ne_old"].device
        return dict(ne=torch.empty(db.ncells, dtype=torch.float64, device=dev),
                    phi=torch.empty(db.ncells, dtype=torch.float64, device=dev),
                    status=torch.empty(db.ncol, dtype=torch.int32, device=dev),
                    newton_it=torch.empty(db.ncol, dtype=torch.int32, device=dev),
                    krylov_it=torch.empty(db.ncol, dtype=torch.int32, device=dev),
                    res_evals=torch.empty(db.ncol, dtype=torch.int32, device=dev),
                    final_res=torch.empty(db.ncol, dtype=torch.float64, device=dev),
                    mg_cycles=torch.empty(db.ncol, dtype=torch.int32, device=dev))

    def solve(self, db: DeviceBatch, out: dict | None = None) -> dict:
        """sdcef_solve_batch on device tensors; asynchronous on the solver stream."""
        out = out or self.alloc_result(db)
        bs = db.cstruct()
        rs = ResultC(_ptr(out["ne"]), _ptr(out["phi"]), _ptr(out["status"]),
                     _ptr(out["newton_it"]), _ptr(out["krylov_it"]), _ptr(out["res_evals"]),
                     _ptr(out["final_res"]), _ptr(out.get("mg_cycles")))
        _check(lib().sdcef_solve_batch(self.h, C.byref(bs), C.byref(rs)))
        return out

    @staticmethod
    def _host_structs(b, out, guess, keep):
        """BatchC / ResultC of host arrays (numpy or pinned torch); the arrays
        that back the pointers are appended to keep."""
        def h(a, dt=np.float64):
            if a is None:
                return None
            if hasattr(a, "data_ptr"):
                keep.append(a)
                return a.data_ptr()
            arr = np.ascontiguousarray(a, dtype=dt)
            keep.append(arr)
            return arr.ctypes.data
        val = np.ascontiguousarray(b.valence, dtype=np.int32)
        keep.append(val)
        bs = BatchC(b.ncol, h(b.col_off, np.int64), h(b.length), h(b.dt), h(b.v_left),
                    h(b.v_right), h(b.ne_old), h(b.phi_old), int(val.shape[0]), val.ctypes.data,
                    h(np.atleast_2d(b.n_ion) if not hasattr(b.n_ion, "data_ptr") else b.n_ion),
                    h(b.T), None, h(b.u_adv), h(b.i_re),
                    h(None if guess is None else guess[0]), h(None if guess is None else guess[1]))
        if out is None:
            out = dict(ne=np.empty(b.ncells), phi=np.empty(b.ncells),
                       status=np.empty(b.ncol, np.int32), newton_it=np.empty(b.ncol, np.int32),
                       krylov_it=np.empty(b.ncol, np.int32), res_evals=np.empty(b.ncol, np.int32),
                       final_res=np.empty(b.ncol))
        rs = ResultC(*[h(out[k], None) if k in out else None for k in
                       ("ne", "phi", "status", "newton_it", "krylov_it", "res_evals", "final_res")])
        return bs, rs, out

    def solve_host(self, b, out: dict | None = None, guess=None) -> dict:
        """sdcef_solve_batch_host: numpy (or pinned torch) host arrays in and out."""
        keep = []
        bs, rs, out = self._host_structs(b, out, guess, keep)
        _check(lib().sdcef_solve_batch_host(self.h, C.byref(bs), C.byref(rs)))
        return out

    def solve_host_many(self, batches, outs=None) -> list:
        """sdcef_solve_batches_host: several host batches, the copies of the next
        and previous batch overlapping each solve; returns the result dicts."""
        keep = []
        outs = outs if outs is not None else [None] * len(batches)
        structs = [self._host_structs(b, o, None, keep) for b, o in zip(batches, outs)]
        barr = (BatchC * len(structs))(*[st[0] for st in structs])
        rarr = (ResultC * len(structs))(*[st[1] for st in structs])
        _check(lib().sdcef_solve_batches_host(self.h, len(structs), C.cast(barr, C.c_void_p),
                                              C.cast(rarr, C.c_void_p)))
        return [st[2] for st in structs]

    def autotune(self, db: DeviceBatch, reps: int = 2):
        """sdcef_autotune: pick threads per column for this batch by timing."""
        out = self.alloc_result(db)
        bs = db.cstruct()
        rs = ResultC(_ptr(out["ne"]), _ptr(out["phi"]), None, None, None, None, None)
        tpb = C.c_int(0)
        ms = (C.c_float * 4)()
        _check(lib().sdcef_autotune(self.h, C.byref(bs), C.byref(rs), int(reps), C.byref(tpb),
                                    C.cast(ms, C.c_void_p)))
        self.params.threads_per_column = tpb.value
        return tpb.value, {t: float(m) for t, m in zip((32, 64, 128, 256), ms)}

    def autotune_on_chip(self, db: DeviceBatch, reps: int = 2):
        """sdcef_autotune_on_chip: Krylov vectors in shared memory or in the slot,
        whichever solves this batch faster; returns (choice, {0: ms, 1: ms})."""
        out = self.alloc_result(db)
        bs = db.cstruct()
        rs = ResultC(_ptr(out["ne"]), _ptr(out["phi"]), None, None, None, None, None)
        oc = C.c_int(0)
        ms = (C.c_float * 2)()
        _check(lib().sdcef_autotune_on_chip(self.h, C.byref(bs), C.byref(rs), int(reps),
                                            C.byref(oc), C.cast(ms, C.c_void_p)))
        self.params.krylov_on_chip = oc.value
        return oc.value, {0: float(ms[0]), 1: float(ms[1])}

    def ion_update(self, db: DeviceBatch, phi, kappa_ion: float = 4e-3):
        import torch
        out = torch.empty_like(db.tensors["n_ion"])
        bs = db.cstruct()
        _check(lib().sdcef_ion_update_batch(self.h, C.byref(bs), _ptr(phi), float(kappa_ion),
                                            _ptr(out)))
        return out

    def current(self, db: DeviceBatch, ne, phi, kappa_ion: float = 4e-3):
        """sdcef_current_batch: (J+, J-) [A/m^2] through every face, [cells + ncol]
        each; the N + 1 faces of column c start at col_off[c] + c."""
        import torch
        jp = torch.empty(db.ncells + db.ncol, dtype=torch.float64, device=ne.device)
        jn = torch.empty_like(jp)
        bs = db.cstruct()
        _check(lib().sdcef_current_batch(self.h, C.byref(bs), _ptr(ne), _ptr(phi),
                                         float(kappa_ion), _ptr(jp), _ptr(jn)))
        return jp, jn

    def set_transport_table(self, table: dict):
        """sdcef_set_transport_table from a dict with mu, D ([nc, nx] arrays),
        en_max_td, T_in, T_max (workload.transport_table's format)."""
        mu = np.ascontiguousarray(table["mu"], dtype=np.float64)
        D = np.ascontiguousarray(table["D"], dtype=np.float64)
        _check(lib().sdcef_set_transport_table(self.h, mu.shape[0], mu.shape[1],
                                               float(table["en_max_td"]), float(table["T_in"]),
                                               float(table["T_max"]), mu.ctypes.data, D.ctypes.data))

    def sweep_work(self, db: DeviceBatch):
        """Device scratch of sdcef_sdc_sweep for this context's ion scheme:
        3 n_species x max_cells doubles (Godunov) or n_species x cells."""
        import torch
        nsp = int(db.tensors["n_ion"].shape[0]) if db.tensors["n_ion"].dim() > 1 else 1
        n = 3 * nsp * self.max_cells if self.params.ion_scheme == ION_GODUNOV else nsp * db.ncells
        return torch.empty(n, dtype=torch.float64, device=db.tensors["ne_old"].device)

    def ion_provisional(self, db: DeviceBatch, phi, n_prev=None, kappa_ion: float = 4e-3):
        """sdcef_ion_provisional_batch: provisional ions with the paper's
        transport; n_prev = the previous SDC iterate (None: n^n)."""
        import torch
        out = torch.empty_like(db.tensors["n_ion"])
        scratch = torch.empty_like(db.tensors["n_ion"])
        bs = db.cstruct()
        _check(lib().sdcef_ion_provisional_batch(self.h, C.byref(bs), _ptr(phi), _ptr(n_prev),
                                                 float(kappa_ion), _ptr(scratch), _ptr(out)))
        return out

    def sdc_sweep(self, db: DeviceBatch, k_max: int = 4, kappa_ion: float = 4e-3,
                  work=None, out: dict | None = None) -> dict:
        """sdcef_sdc_sweep: k_max SDC iterations of the electric solve; work, if
        given, as sized by sweep_work."""
        out = out or self.alloc_result(db)
        work = self.sweep_work(db) if work is None else work
        bs = db.cstruct()
        rs = ResultC(_ptr(out["ne"]), _ptr(out["phi"]), _ptr(out["status"]),
                     _ptr(out["newton_it"]), _ptr(out["krylov_it"]), _ptr(out["res_evals"]),
                     _ptr(out["final_res"]))
        _check(lib().sdcef_sdc_sweep(self.h, C.byref(bs), int(k_max), float(kappa_ion),
                                     _ptr(work), C.byref(rs)))
        return out

    def residual(self, db: DeviceBatch, ne, phi):
        import torch
        Fe = torch.empty_like(ne)
        Fp = torch.empty_like(phi)
        bs = db.cstruct()
        _check(lib().sdcef_residual_batch(self.h, C.byref(bs), _ptr(ne), _ptr(phi), _ptr(Fe),
                                          _ptr(Fp)))
        return Fe, Fp

    def bernoulli(self, x):
        """sdcef_bernoulli_batch: B(x) = x / (e^x - 1) and B'(x) as the residual
        kernel evaluates them (x: FP64 device tensor)."""
        import torch
        b = torch.empty_like(x)
        db = torch.empty_like(x)
        _check(lib().sdcef_bernoulli_batch(self.h, _ptr(x), _ptr(b), _ptr(db), int(x.numel())))
        return b, db

    def precond_apply(self, db: DeviceBatch, ne, phi, r_e, r_phi, *, return_cycles=False):
        """x = P^-1 r (physical units) of the configured preconditioner built at
        (ne, phi); with return_cycles also the V-cycles per column (PREC_MG)."""
        import torch
        xe = torch.empty_like(r_e)
        xp = torch.empty_like(r_phi)
        cyc = torch.zeros(db.ncol, dtype=torch.int32, device=r_e.device)
        bs = db.cstruct()
        _check(lib().sdcef_precond_apply_batch(self.h, C.byref(bs), _ptr(ne), _ptr(phi),
                                               _ptr(r_e), _ptr(r_phi), _ptr(xe), _ptr(xp),
                                               _ptr(cyc)))
        return (xe, xp, cyc) if return_cycles else (xe, xp)


def fma_peak_probe(precision: int = FP64, iters: int = 300, stream=None) -> float:
    """sdcef_fma_peak_probe: measured FMA throughput (TFLOP/s) of this GPU in FP64
    (precision=FP64) or FP32 (precision=MIXED); synchronises."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    t = C.c_double(0.0)
    _check(lib().sdcef_fma_peak_probe(int(precision), int(iters), C.c_void_p(stream.cuda_stream),
                                      C.byref(t)))
    return float(t.value)


def solve_noalloc(params: Params, db: DeviceBatch, out: dict, max_col_cells: int, stream=None):
    """sdcef_solve_batch_noalloc: the solve without a context, its workspace in the
    library's fixed device scratch array (for callers that cannot allocate)."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    bs = db.cstruct()
    rs = ResultC(_ptr(out["ne"]), _ptr(out["phi"]), _ptr(out["status"]),
                 _ptr(out["newton_it"]), _ptr(out["krylov_it"]), _ptr(out["res_evals"]),
                 _ptr(out["final_res"]), _ptr(out.get("mg_cycles")))
    _check(lib().sdcef_solve_batch_noalloc(C.byref(params), C.byref(bs), C.byref(rs),
                                           int(max_col_cells), C.c_void_p(stream.cuda_stream)))
    return out


class MLP:
    """The learned Newton initial guess (sdcef_mlp_* of include/sdcef.h)."""

    def __init__(self, max_rows: int, stream=None):
        import torch
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = C.c_void_p()
        _check(lib().sdcef_mlp_create(C.byref(h), int(max_rows), C.c_void_p(stream.cuda_stream)))
        self.h = h
        self.max_rows = int(max_rows)

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            lib().sdcef_mlp_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, flat: np.ndarray):
        a = np.ascontiguousarray(flat, dtype=np.float32)
        assert a.shape == (MLP_NPARAM,)
        _check(lib().sdcef_mlp_set_params(self.h, a.ctypes.data))

    def get_params(self) -> np.ndarray:
        a = np.empty(MLP_NPARAM, dtype=np.float32)
        _check(lib().sdcef_mlp_get_params(self.h, a.ctypes.data))
        return a

    def get_state(self) -> dict:
        """Training checkpoint: parameters, Adam moments and step (host arrays)."""
        p, m, v = (np.empty(MLP_NPARAM, dtype=np.float32) for _ in range(3))
        step = C.c_int64(0)
        _check(lib().sdcef_mlp_get_state(self.h, p.ctypes.data, m.ctypes.data, v.ctypes.data,
                                         C.byref(step)))
        return {"params": p, "adam_m": m, "adam_v": v, "step": int(step.value)}

    def set_state(self, state: dict):
        """Restore a checkpoint taken by get_state."""
        p, m, v = (np.ascontiguousarray(state[k], dtype=np.float32)
                   for k in ("params", "adam_m", "adam_v"))
        assert p.shape == m.shape == v.shape == (MLP_NPARAM,)
        _check(lib().sdcef_mlp_set_state(self.h, p.ctypes.data, m.ctypes.data, v.ctypes.data,
                                         int(state["step"])))

    def launches(self) -> int:
        return int(lib().sdcef_mlp_last_launch_count(self.h))

    def check(self):
        """Raise if a tensor-core wait of an earlier call ran out (synchronises)."""
        _check(lib().sdcef_mlp_check(self.h))

    def check_word(self) -> int:
        """sdcef_mlp_check_word (see Solver.check_word)."""
        w = C.c_uint(0)
        _check(lib().sdcef_mlp_check_word(self.h, C.byref(w)))
        return int(w.value)

    def set_wait_polls(self, polls: int):
        """Polls of the kernels' main bounded waits (test hook; < 0 = default,
        0 = every such wait gives up at once)."""
        _check(lib().sdcef_mlp_set_wait_polls(self.h, int(polls)))

    def features(self, db: DeviceBatch):
        import torch
        X = torch.empty((db.ncells, 32), dtype=torch.bfloat16, device=db.tensors["ne_old"].device)
        bs = db.cstruct()
        _check(lib().sdcef_mlp_features(self.h, C.byref(bs), _ptr(X)))
        return X

    def targets(self, db: DeviceBatch, ne_star, phi_star):
        import torch
        T = torch.empty((db.ncells, 2), dtype=torch.float32, device=ne_star.device)
        bs = db.cstruct()
        _check(lib().sdcef_mlp_targets(self.h, C.byref(bs), _ptr(ne_star), _ptr(phi_star), _ptr(T)))
        return T

    def forward(self, X):
        import torch
        Y = torch.empty((X.shape[0], 2), dtype=torch.float32, device=X.device)
        _check(lib().sdcef_mlp_forward(self.h, _ptr(X), int(X.shape[0]), _ptr(Y)))
        return Y

    def grad(self, X, T):
        import torch
        g = torch.empty(MLP_NPARAM, dtype=torch.float32, device=X.device)
        loss = torch.empty(1, dtype=torch.float32, device=X.device)
        _check(lib().sdcef_mlp_grad(self.h, _ptr(X), _ptr(T), int(X.shape[0]), _ptr(g), _ptr(loss)))
        return g, loss

    def train_step(self, X, T, lr: float, loss=None):
        _check(lib().sdcef_mlp_train_step(self.h, _ptr(X), _ptr(T), int(X.shape[0]),
                                          float(lr), _ptr(loss)))

    def guess(self, db: DeviceBatch, ne=None, phi=None, components: int = 3):
        import torch
        dev = db.tensors["ne_old"].device
        ne = torch.empty(db.ncells, dtype=torch.float64, device=dev) if ne is None else ne
        phi = torch.empty(db.ncells, dtype=torch.float64, device=dev) if phi is None else phi
        bs = db.cstruct()
        _check(lib().sdcef_mlp_guess(self.h, C.byref(bs), int(db.ncells), int(components),
                                     _ptr(ne), _ptr(phi)))
        return ne, phi


def pack_params(p: dict) -> np.ndarray:
    """Flatten {W1, b1, W2, b2, W3, b3} in the order of the C ABI."""
    return np.concatenate([np.asarray(p[k], dtype=np.float64).reshape(-1)
                           for k in ("W1", "b1", "W2", "b2", "W3", "b3")])


def unpack_params(flat) -> dict:
    flat = np.asarray(flat, dtype=np.float64)
    shapes = (("W1", (128, 32)), ("b1", (128,)), ("W2", (128, 128)), ("b2", (128,)),
              ("W3", (2, 128)), ("b3", (2,)))
    out, o = {}, 0
    for k, sh in shapes:
        n = int(np.prod(sh))
        out[k] = flat[o:o + n].reshape(sh).copy()
        o += n
    return out
