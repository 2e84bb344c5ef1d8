"""Child process of test_gpu_debug_bounds.py: with DV_DEBUG=1 the binding loads the bounds-checked
debug library. Runs the instrumented entry points on small inputs (ragged grid, split event
ranges, query lists with queries on the mesh, all precisions, both adjoints on odd rows and on
rows longer than the adjoint's window, the Eq. 4 kernels, one batch) and prints one JSON line:
the debug library's bounds report and the largest errors against the FP64 oracle."""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)
sys.path.insert(0, os.path.dirname(HERE))

import numpy as np  # noqa: E402
import torch  # noqa: E402

import oracle  # noqa: E402
from paper_2407_11272_b300 import dv, meshgen  # noqa: E402


def main():
    assert dv.library_path().name == "libdv_debug.so", dv.library_path()
    dev = torch.device("cuda:0")
    V, F = meshgen.jittered_torus(nu=30, nv=15, sigma=0.01, delete_frac=0.1, seed=5)
    grid = dv.Grid((21, 18, 10), (-1.0, -0.9, -0.5), (1.0, 0.9, 0.5))
    Vd, Fd = torch.from_numpy(V).to(dev), torch.from_numpy(F).to(dev)
    mesh = dv.dv_mesh_create(Vd, Fd)
    dv.dv_debug_report(clear=True)
    Q = oracle.grid_queries(grid.lo, grid.hi, grid.n)
    w64 = oracle.winding(V, F, Q)
    far = oracle.point_mesh_distance(V, F, Q) > 1e-3
    out = {"errors": {}}
    for prec in ("fp32", "kahan", "mixed", "fp16"):
        w, occ, _ = dv.dv_voxelize_grid(mesh, grid, precision=prec)
        tol_far = np.abs(w.cpu().numpy().astype(np.float64) - w64)[far].max()
        out["errors"][f"grid_{prec}"] = float(tol_far)
    rng = np.random.default_rng(11)
    Ql = np.concatenate([rng.uniform(-1, 1, size=(997, 3)), V[:4].astype(np.float64)]).astype(np.float32)
    wl64 = oracle.winding(V, F, Ql)
    farl = oracle.point_mesh_distance(V, F, Ql) > 1e-3
    for prec in ("kahan", "mixed"):
        wl = dv.dv_winding(mesh, queries=torch.from_numpy(Ql).to(dev), precision=prec).cpu().numpy()
        out["errors"][f"list_{prec}"] = float(np.abs(wl.astype(np.float64) - wl64)[farl].max())
    g = meshgen.upstream_gradient(grid.num_queries, seed=3).astype(np.float64) * far
    G64 = oracle.winding_grad(V, F, Q, g)
    gd = torch.from_numpy(g.astype(np.float32)).to(dev)
    for name, fn in (("face", dv.dv_winding_backward), ("boundary", dv.dv_winding_backward_boundary)):
        G = fn(mesh, gd, grid=grid).cpu().numpy().astype(np.float64)
        out["errors"][f"grad_grid_{name}"] = float(np.linalg.norm(G - G64) / np.linalg.norm(G64))
    # rows longer than the adjoint's window: a full piece of 2048 queries and an odd piece of one
    grid_l = dv.Grid((2049, 3, 2), (-1.0, -0.9, -0.5), (1.0, 0.9, 0.5))
    Qr = oracle.grid_queries(grid_l.lo, grid_l.hi, grid_l.n)
    gr = meshgen.upstream_gradient(grid_l.num_queries, seed=4).astype(np.float64)
    gr *= oracle.point_mesh_distance(V, F, Qr) > 1e-3
    Gr64 = oracle.winding_grad(V, F, Qr, gr)
    grd = torch.from_numpy(gr.astype(np.float32)).to(dev)
    for name, fn in (("face", dv.dv_winding_backward), ("boundary", dv.dv_winding_backward_boundary)):
        G = fn(mesh, grd, grid=grid_l).cpu().numpy().astype(np.float64)
        out["errors"][f"grad_long_rows_{name}"] = float(np.linalg.norm(G - Gr64) / np.linalg.norm(Gr64))
    gl = rng.normal(size=len(Ql)) * farl
    Gl64 = oracle.winding_grad(V, F, Ql, gl)
    Gl = dv.dv_winding_backward(mesh, torch.from_numpy(gl.astype(np.float32)).to(dev),
                                queries=torch.from_numpy(Ql).to(dev)).cpu().numpy().astype(np.float64)
    out["errors"]["grad_list_face"] = float(np.linalg.norm(Gl - Gl64) / np.linalg.norm(Gl64))
    wd = dv.dv_dipole_winding(mesh, grid=grid).cpu().numpy().astype(np.float64)
    out["errors"]["dipole"] = float(np.abs(wd - oracle.dipole_winding(V, F, Q)).max())
    dv.dv_dipole_backward(mesh, gd, grid=grid)
    occ_b = torch.empty(grid.num_queries, dtype=torch.uint8, device=dev)
    dv_b = torch.empty((len(V), 3), dtype=torch.float32, device=dev)
    side = torch.cuda.Stream()  # a batch is captured as a CUDA graph: not on the default stream
    side.wait_stream(torch.cuda.current_stream())
    dv.dv_run_batch([{"mesh": mesh, "grid": grid, "occ": occ_b, "upstream": gd, "dverts": dv_b}], precision="mixed",
                    stream=side)
    torch.cuda.synchronize()
    tie = np.abs(w64 - 0.5) <= 1e-9
    out["errors"]["batch_occ_mismatch"] = int(((occ_b.cpu().numpy() != (w64 > 0.5)) & ~tie).sum())
    dv.dv_mesh_check(mesh)
    out["report"] = dv.dv_debug_report()
    mesh.close()
    print(json.dumps(out))


if __name__ == "__main__":
    main()
