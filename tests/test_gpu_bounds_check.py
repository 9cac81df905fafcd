"""The index-checking debug build (libhubhmc_check.so, -DHH_BOUNDS_CHECK) on
the GPU: its self-test records an index past its range (without accessing
it), and the parity cases of the other tests (tiny lattices with N_x = 2, 3,
applies in both precisions, FP64 and mixed solves, the multi-vector apply,
trajectories, a mixed-dimension batch) run through it with no failed check
and results that still match the oracle."""
import json
import math
import os
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def checked_lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1007_3432_gb300 import build
    return build.build(bounds_check=True)


def test_checked_build_runs_the_parity_cases_clean(checked_lib):
    env = dict(os.environ, HH_BOUNDS_CHECK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "_bounds_worker.py")], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    from paper_1007_3432_gb300.binding import HH_EBOUNDS, HH_OK
    # self-test: check code 15, index 1000 recorded; the read clears it
    assert out["selftest"] == [HH_EBOUNDS, 1, (15 << 32) | 1000], out["selftest"]
    assert out["after_selftest"] == [HH_OK, 0], out["after_selftest"]
    assert out["final"] == [HH_OK, 1, 0], out["final"]
    w = out["worst"]
    assert w["apply_M_f64"] <= 1e-12 and w["apply_MT_f64"] <= 1e-12 and w["apply_MTM_f64"] <= 1e-12, w
    assert w["apply_M_f32"] <= 1e-5 and w["apply_MT_f32"] <= 1e-5 and w["apply_MTM_f32"] <= 1e-5, w
    assert w["apply_multi"] <= 1e-5, w
    assert w["solve_fp64"] <= 1e-10 * 1.0001 and w["solve_mixed"] <= 1e-10 * 1.0001, w
    assert w["batch_solve"] <= 1e-10 * 1.0001 and out["batch_status"] == [0, 0], out
    assert math.isfinite(w["traj_dH_1"]) and math.isfinite(w["traj_dH_3"]), w
