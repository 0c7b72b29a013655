"""The checked build (-DABP_CHECKED, the substitute for a device memory
checker): every grid node index the kernels read or write is bounds-checked
and out-of-grid indices are counted. Every form of the library (windowed WT
and mABP, per-step fused with coordination numbers, phased on a shared
grid, the closed loop fused and phased, the plain form, the allocation-free
step, the server) runs on small cases under the checked build and under
the normal one, each in its own process: the checked build must count no
out-of-grid index, and both builds must give the same bits (to FP64
rounding on the shared grid, whose hills are added by atomics)."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(lib, out):
    env = dict(os.environ, ABP_LIBRARY=lib)
    r = subprocess.run([sys.executable, "-m", "tests.checked_workloads", out], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_checked_build_sees_no_out_of_grid_index_and_changes_no_bit(tmp_path):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1609_09833_gb300 import build

    normal = build.build()
    checked = build.build(checked=True)
    rc = _run(checked, str(tmp_path / "checked.npz"))
    rn = _run(normal, str(tmp_path / "normal.npz"))
    assert rc == {"violations": 0, "checked": True}, rc
    assert rn == {"violations": 0, "checked": False}, rn
    a = np.load(tmp_path / "checked.npz")
    b = np.load(tmp_path / "normal.npz")
    assert sorted(a.files) == sorted(b.files) and len(a.files) > 20
    for k in a.files:
        if k.startswith(("big_", "mdbig_")):
            # a shared grid's FP64 atomics add a step's hills in any order
            scale = max(np.abs(b[k]).max(), 1e-30)
            assert np.abs(a[k] - b[k]).max() <= 1e-6 * scale, k
        else:
            assert np.array_equal(a[k], b[k]), k
    assert np.any(a["md_x"] != 0) and np.any(a["win_F"] != 0) and np.any(a["serve_F"] != 0)
