"""The bounds-checking build of the library (-DSDCEF_CHECKS; csrc/checks.cuh),
the stand-in for a device memory checker: every plane, level, shared-memory
and global index of the solver, block solver, multigrid, ion, current and MLP
kernels is tested before use and a failing test records its site in a check
word. The parity cases of every preconditioner, precision, transport model,
the error test, a rejected start, the field kernels, the SDC sweep and the
learned-guess kernels run against that build (in a child process that loads
it through SDCEF_LIB); every check word must stay 0 and the results must still
match the oracle to the usual bars."""
import json
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

BARS = {"mixed_fp32": 1e-7, "fields_and_sweep": 1e-8, "mlp": 2e-2}


def test_checked_build_runs_parity_cases_without_a_failed_check():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1904_08510_gb300 import build as B
    lib = B.build(checks=True)
    env = dict(os.environ, SDCEF_LIB=lib, PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, os.path.join(HERE, "checked_build_cases.py")], cwd=ROOT,
                       env=env, capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, r.stderr[-4000:]
    res = json.loads(r.stdout.strip().splitlines()[-1])
    assert len(res) >= 12
    for case, v in res.items():
        assert v["word"] == 0, (case, v)                  # no index left its array
        assert v["ok"] >= max(1, v["ncol"] // 2), (case, v)
        assert v["err"] <= BARS.get(case, 1e-9), (case, v)
