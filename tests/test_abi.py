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
