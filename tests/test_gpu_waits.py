"""The bounded waits of the shared-memory copy pipelines give up after their limit and report
DV_ERR_TIMEOUT instead of hanging; the CUDA context stays usable afterwards. The failure is made
by waiting on a barrier phase that nothing completes (no fault, no trap, no unbounded loop)."""
import time

import numpy as np
import pytest

import oracle
from _util import make_mesh
from paper_2407_11272_b300 import dv, meshgen

pytestmark = pytest.mark.gpu


def test_bounded_wait_completes_when_the_phase_completes(cuda_device):
    assert dv.dv_selftest_bounded_wait(200_000, True) == 0


def test_bounded_wait_times_out_and_context_survives(cuda_device):
    t0 = time.perf_counter()
    st = dv.dv_selftest_bounded_wait(50_000, False)  # 50 ms limit, nothing ever arrives
    dt = time.perf_counter() - t0
    assert st == 5  # DV_ERR_TIMEOUT
    assert 0.04 <= dt < 5.0
    # the context still runs real work correctly
    V, F = meshgen.icosphere(1, 0.5)
    mesh = make_mesh(V, F, cuda_device)
    grid = dv.Grid.cube(6)
    w = dv.dv_winding(mesh, grid=grid, precision="kahan").cpu().numpy()
    w64 = oracle.winding(V, F, oracle.grid_queries(grid.lo, grid.hi, grid.n))
    assert np.abs(w - w64).max() < 1e-5
    assert dv.dv_selftest_bounded_wait(200_000, True) == 0
