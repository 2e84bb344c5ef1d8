"""FP16 ablation of the forward (the paper computed in half precision, §3.1): its error against
the FP64 oracle is measured and bounded loosely (it is expected to miss the 1e-4 bar), and it
must still get the occupancy of queries far from the threshold right."""
import numpy as np
import pytest

from _util import make_mesh, oracle_grid
from paper_2407_11272_b300 import dv, meshgen

pytestmark = pytest.mark.gpu


def test_fp16_error_against_oracle(cuda_device):
    V, F = meshgen.jittered_torus(nu=60, nv=30, sigma=0.01, delete_frac=0.1, seed=0)
    grid = dv.Grid.cube(40)
    Q, w64, d = oracle_grid(V, F, grid)
    mesh = make_mesh(V, F, cuda_device)
    w16, occ16, _ = dv.dv_voxelize_grid(mesh, grid, precision="fp16")
    w32, _, _ = dv.dv_voxelize_grid(mesh, grid, precision="kahan")
    w16 = w16.cpu().numpy().astype(np.float64)
    w32 = w32.cpu().numpy().astype(np.float64)
    far = d > 1e-2
    e16 = np.abs(w16 - w64)[far]
    e32 = np.abs(w32 - w64)[far]
    print(f"fp16: max {e16.max():.3e} mean {e16.mean():.3e}; fp32-kahan: max {e32.max():.3e} mean {e32.mean():.3e}")
    assert np.all(np.isfinite(w16))
    assert e16.max() < 5e-2
    assert e32.max() < e16.max()
    safe = far & (np.abs(w64 - 0.5) > 0.1)
    assert np.array_equal(occ16.cpu().numpy()[safe], (w64[safe] > 0.5).astype(np.uint8))


def test_fp16_list_path_is_rejected(cuda_device):
    V, F = meshgen.icosphere(1, 0.5)
    mesh = make_mesh(V, F, cuda_device)
    import torch

    with pytest.raises(dv.DvError) as e:
        dv.dv_winding(mesh, queries=torch.zeros((4, 3), device=cuda_device), precision="fp16")
    assert e.value.status == 6
