"""Algorithm 2 (flipped duplication) on the GPU against the oracle's restatement, and the
voxelization of the duplicated open mesh against the oracle (§2.3: an open mesh voxelizes as an
almost closed thin shell)."""
import numpy as np
import pytest

import oracle
from _util import check_forward, make_mesh, to_dev
from paper_2407_11272_b300 import dv, meshgen

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("eps", [0.01, 0.03])
def test_flipped_duplication_matches_oracle(cuda_device, eps):
    V, F = meshgen.open_cap(freq=10, radius=0.6, max_polar=1.1)
    mesh = make_mesh(V, F, cuda_device)
    V2, F2 = dv.dv_flipped_duplication(mesh, to_dev(V, cuda_device), eps)
    V2r, F2r = oracle.flipped_duplication(V, F, eps)
    assert np.array_equal(F2.cpu().numpy(), F2r)
    np.testing.assert_allclose(V2.cpu().numpy(), V2r, atol=1e-6, rtol=0)


def test_duplicated_open_surface_voxelizes_as_shell(cuda_device):
    V, F = meshgen.open_cap(freq=10, radius=0.6, max_polar=1.1)
    eps = 0.03
    mesh = make_mesh(V, F, cuda_device)
    V2, F2 = dv.dv_flipped_duplication(mesh, to_dev(V, cuda_device), eps)
    dup = dv.dv_mesh_create(V2, F2)
    grid = dv.Grid.cube(40, -0.8, 0.8)
    w, occ, _ = dv.dv_voxelize_grid(dup, grid, precision="mixed")
    V2r, F2r = oracle.flipped_duplication(V, F, eps)
    Q = oracle.grid_queries(grid.lo, grid.hi, grid.n)
    w64 = oracle.winding(V2r, F2r, Q)
    d = oracle.point_mesh_distance(V2r, F2r, Q)
    check_forward(w.cpu().numpy(), w64, d, "mixed", occ.cpu().numpy(), "flipdup")
    # queries inside the slit between the two layers are occupied
    r = np.linalg.norm(Q, axis=1)
    pol = np.arccos(np.clip(Q[:, 2] / np.maximum(r, 1e-12), -1, 1))
    slit = (r > 0.6 - eps + 0.005) & (r < 0.6 - 0.005) & (pol < 0.8)
    assert slit.any()
    assert occ.cpu().numpy()[slit].all()
    # and far from the cap nothing is
    far = d > 0.1
    assert not occ.cpu().numpy()[far].any()
