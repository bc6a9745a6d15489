"""The bounds-checked build (-DGMG_CHECKED) on the configuration-0 and -1 parity
cases: the checked kernels record any index outside its buffer in a sticky
device word instead of accessing memory out of range; the cases must leave
every word clear and still agree with the oracle (apply 1e-6, same pass/fail,
iterations within max(2, 10 %), displacement 1e-5).  The checked library runs
in a fresh process of its own (GMG_LIBRARY names it)."""

import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_bounds_checked_build_parity_cases():
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2604_26441_b300 import build
    lib = build.build_checked_library()
    env = dict(os.environ, GMG_LIBRARY=lib)
    out = subprocess.run([sys.executable, os.path.join(HERE, "checked_cases.py")], env=env, capture_output=True,
                         text=True, timeout=1200)
    assert out.returncode == 0, out.stderr[-3000:]
    recs = [json.loads(line) for line in out.stdout.splitlines() if line.startswith("{")]
    assert [r["case"] for r in recs] == ["c0", "c1"]
    for r in recs:
        assert r["site"] == 0, r
        assert r["apply_err"] < 1e-6, r
        assert (r["status"] == 0) == r["oracle_ok"], r
        assert abs(r["iterations"] - r["oracle_iterations"]) <= max(2, 0.1 * r["oracle_iterations"]), r
        assert r["u_err"] < 1e-5, r
