"""Request server on the GPU: every request's result served in a mix (batched into CUDA graphs,
several batches in flight, requests arriving while others run) equals the same request run
alone through the single-request entry points, and matches the oracle."""
import numpy as np
import pytest
import torch

import oracle
from _util import TIE
from paper_2407_11272_b300 import dv, meshgen
from paper_2407_11272_b300.serve import Server, make_workload

pytestmark = pytest.mark.gpu


def _alone(r, dev):
    mesh = dv.dv_mesh_create(torch.from_numpy(r.verts).to(dev), torch.from_numpy(r.faces).to(dev))
    grid = dv.Grid.cube(r.n)
    _, occ, _ = dv.dv_voxelize_grid(mesh, grid, precision="mixed", want_w=False)
    dV = None
    if r.want_grad:
        g = torch.from_numpy(meshgen.upstream_gradient(r.queries, seed=r.upstream_seed)).to(dev)
        dV = dv.dv_winding_backward(mesh, g, grid=grid).cpu().numpy()
    torch.cuda.synchronize()
    return occ.cpu().numpy(), dV


@pytest.mark.parametrize("realtime,rate", [(False, 0.0), (True, 60.0)])
def test_mix_equals_alone(cuda_device, realtime, rate):
    reqs = make_workload(12, rate=rate, seed=11, f_lo=300, f_hi=6000, grids=(16, 24, 32), grad_frac=0.5)
    srv = Server(device=cuda_device, max_batch=4, max_inflight=2)
    results, stats = srv.run(reqs, realtime=realtime)
    assert stats["requests"] == len(reqs) and stats["batches"] >= 3
    by_id = {r.rid: r for r in reqs}
    for res in results:
        occ, dV = _alone(by_id[res.rid], cuda_device)
        assert np.array_equal(res.occ, occ), res.rid
        if dV is not None:
            assert np.array_equal(res.dverts, dV), res.rid
        else:
            assert res.dverts is None
    # one request against the oracle
    r = by_id[results[0].rid]
    grid = dv.Grid.cube(r.n)
    w64 = oracle.winding(r.verts, r.faces, oracle.grid_queries(grid.lo, grid.hi, grid.n))
    tie = np.abs(w64 - 0.5) <= TIE
    assert np.all((results[0].occ == (w64 > 0.5)) | tie)
