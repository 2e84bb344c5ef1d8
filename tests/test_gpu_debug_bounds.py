"""The bounds-checked debug build (libdv_debug.so, -DDV_DEBUG): in a child process that loads it,
the instrumented kernels run on small ragged, split and list cases; no indexed access falls
outside its buffer (the debug record is empty) and the results still match the FP64 oracle.
The checks record and skip an out-of-range access instead of faulting, so a wrong index shows up
here as a report."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_debug_build_reports_no_out_of_range_access(cuda_device):
    from paper_2407_11272_b300 import build

    build.build(debug=True)
    env = dict(os.environ, DV_DEBUG="1")
    r = subprocess.run([sys.executable, os.path.join(HERE, "_debug_bounds_case.py")], env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    res = json.loads([ln for ln in r.stdout.splitlines() if ln.startswith("{")][-1])
    assert res["report"] is not None and res["report"]["count"] == 0, res["report"]
    e = res["errors"]
    for k in ("grid_fp32", "grid_kahan", "grid_mixed", "list_kahan", "list_mixed"):
        assert e[k] <= 1e-4, (k, e[k])
    assert e["grid_fp16"] <= 1e-2
    for k in ("grad_grid_face", "grad_grid_boundary", "grad_long_rows_face", "grad_long_rows_boundary",
              "grad_list_face"):
        assert e[k] <= 1e-3, (k, e[k])
    assert e["dipole"] <= 1e-4
    assert e["batch_occ_mismatch"] == 0
