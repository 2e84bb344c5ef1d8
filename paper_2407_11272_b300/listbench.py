"""Query-list path timing: the winding number and its adjoint for arbitrary query points.

    python -m paper_2407_11272_b300.listbench [--queries 2097152] [--mesh torus] [--reps 3]

Seeded uniform points in [-1, 1]^3 against one of the benchmark meshes (the 36 000-face
jittered open torus or the 204 020-face SH sphere); per precision the forward through
`dv_winding` with a query buffer, then the adjoint through `dv_winding_backward`. Times are
CUDA events on the launching stream after warm-up calls, averaged over `--reps` calls; the
per-kernel split comes from the library's own event timing. Prints one JSON line.
"""
from __future__ import annotations

import argparse
import json

import numpy as np


def main(argv=None):
    import torch

    from paper_2407_11272_b300 import dv, meshgen

    ap = argparse.ArgumentParser()
    ap.add_argument("--queries", type=int, default=2097152)
    ap.add_argument("--mesh", choices=["torus", "sh_sphere"], default="torus")
    ap.add_argument("--seed", type=int, default=7)
    ap.add_argument("--reps", type=int, default=3)
    a = ap.parse_args(argv)
    if not torch.cuda.is_available():
        raise SystemExit("listbench needs a CUDA device")
    dev = torch.device("cuda")
    V, F = meshgen.jittered_torus() if a.mesh == "torus" else meshgen.sh_sphere()
    rng = np.random.default_rng(a.seed)
    Q = torch.from_numpy(rng.uniform(-1, 1, size=(a.queries, 3)).astype(np.float32)).to(dev)
    g = torch.from_numpy(meshgen.upstream_gradient(a.queries, seed=1)).to(dev)
    mesh = dv.dv_mesh_create(torch.from_numpy(V).to(dev), torch.from_numpy(F).to(dev))
    dv.dv_mesh_reserve(mesh, None, a.queries)
    stream = torch.cuda.current_stream()
    pairs = a.queries * len(F)

    def timed(fn):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        dv.dv_profile_reset()
        dv.dv_profile_enable(True)
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(a.reps):
            fn()
        t1.record(stream)
        torch.cuda.synchronize()
        dv.dv_profile_enable(False)
        ms = t0.elapsed_time(t1) / a.reps
        kernels = {k: round(v[0] / max(v[1], 1), 3) for k, v in dv.dv_profile_read().items()}
        return {"ms": ms, "pairs_per_s": pairs / (ms * 1e-3), "kernels_ms": kernels}

    w = torch.empty(a.queries, dtype=torch.float32, device=dev)
    out = {"mesh": a.mesh, "faces": len(F), "queries": a.queries, "pairs": pairs}
    for prec in ("kahan", "mixed"):
        out[prec] = timed(lambda: dv.dv_winding(mesh, queries=Q, out=w, precision=prec))
    dV = torch.empty((len(V), 3), dtype=torch.float32, device=dev)
    out["adjoint"] = timed(lambda: dv.dv_winding_backward(mesh, g, queries=Q, out=dV))
    print(json.dumps(out))


if __name__ == "__main__":
    main()
