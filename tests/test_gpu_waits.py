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


def test_forward_pipeline_gives_up_on_a_tile_that_never_arrives(cuda_device):
    """The real grid forward (strip order, 96-event tiles in a 4-stage copy ring), with the copy
    of tile 1 of every CTA never issued and a 50 ms wait limit: each CTA gives up on that tile as
    one, drains the copies it issued, and the mesh's error word reports DV_ERR_TIMEOUT once. The
    next ordinary call on the same mesh and context matches the oracle."""
    import torch

    from _util import W_TOL, oracle_grid

    V, F = meshgen.icosphere(3, 0.8)  # 1 280 faces: the event range is split over 8 CTAs of 1-3 tiles
    mesh = make_mesh(V, F, cuda_device)
    grid = dv.Grid.cube(8)
    out = torch.empty(grid.num_queries, dtype=torch.float32, device=cuda_device)
    t0 = time.perf_counter()
    st = dv.dv_selftest_forward_timeout(mesh, grid, out, skip_tile=1, limit_us=50_000)
    dt = time.perf_counter() - t0
    assert st == 5  # DV_ERR_TIMEOUT
    assert 0.04 <= dt < 10.0
    with pytest.raises(dv.DvError) as exc:
        dv.dv_mesh_check(mesh)
    assert exc.value.status == 5
    dv.dv_mesh_check(mesh)  # reported once, then cleared
    _, w64, d = oracle_grid(V, F, grid)
    far = d > 1e-3
    # a skipped tile beyond every CTA's last tile: an ordinary forward
    assert dv.dv_selftest_forward_timeout(mesh, grid, out, skip_tile=1 << 20, limit_us=2_000_000) == 0
    assert np.abs(out.cpu().numpy() - w64)[far].max() <= W_TOL
    w = dv.dv_winding(mesh, grid=grid, precision="kahan").cpu().numpy()
    assert np.abs(w - w64)[far].max() <= W_TOL
    dv.dv_mesh_check(mesh)
    mesh.close()
