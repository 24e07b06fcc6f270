"""The C ABI library builds, loads and exports every symbol include/sdcef.h declares
(no GPU needed: nothing here launches a kernel)."""
import os
import re
import subprocess

import pytest

from paper_1904_08510_gb300 import build as B
from paper_1904_08510_gb300 import sdcef as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libpath():
    return B.build()


def declared_functions():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            names |= set(re.findall(r"\b(sdcef_[a-z_0-9]+)\s*\(", txt))
    return names


def test_library_exports_every_declared_function(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(sdcef_[a-z_0-9]+)$", out, re.M))
    declared = declared_functions()
    assert declared, "no declarations found"
    missing = declared - exported
    assert not missing, missing
    assert set(S.EXPORTS) == declared


def test_library_loads_and_reports_defaults(libpath):
    p = S.default_params()
    assert p.eps_F == 1e-10 and p.gamma == 1e-4 and p.mobility == 0.4
    assert p.precond == S.PREC_EXACT and p.precision == S.FP64


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    monkeypatch.setattr(S, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(S, "_lib", None)
    with pytest.raises(RuntimeError):
        S.lib()


def test_default_build_carries_no_bounds_checks(libpath):
    """The in-tree library is the production build; the bounds-checking one is
    built separately (build(checks=True)) and loaded through SDCEF_LIB."""
    assert S.lib().sdcef_checks_compiled() == 0
    p = S.default_params()
    assert p.eps_E == 5e-10


def _struct_members(name):
    """Member names of a typedef'd struct of include/sdcef.h, in order."""
    txt = open(os.path.join(ROOT, "include", "sdcef.h")).read()
    end = re.search(r"\}\s*" + name + r";", txt).start()
    body = txt[txt.rindex("typedef struct {", 0, end) + len("typedef struct {"):end]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    return re.findall(r"([A-Za-z_][A-Za-z_0-9]*)\s*;", body)


@pytest.mark.parametrize("cname,pyname", [("sdcef_params", "Params"), ("sdcef_batch", "BatchC"),
                                          ("sdcef_result", "ResultC")])
def test_binding_structs_follow_the_header(cname, pyname):
    assert [f[0] for f in getattr(S, pyname)._fields_] == _struct_members(cname)


def test_every_default_crosses_the_boundary(libpath):
    """The C defaults read through the ctypes layout: a field out of place
    would show as a wrong value here."""
    p = S.default_params()
    assert (p.restart_m, p.max_newton, p.max_krylov, p.max_linesearch) == (8, 50, 200, 20)
    assert p.eps_X == 0.0 and p.ls_alpha == 1e-4 and p.eps_r == 1.0
    assert p.bc_electron == S.BC_ABSORBING and p.threads_per_column == 0
    assert p.guess_newton_cap == 8 and p.guess_reject_ratio == 30.0
    assert p.mg_gamma_A == 1e-4 and p.mg_gamma_S == 1e-4 and p.mg_max_cycles == 50
    assert p.gas_molar_mass == 0.028 and p.stall_ratio == 0.9
    assert p.krylov_on_chip == 0 and p.guess_progress == 0.3 and p.sdc_poisson_start == 1
