"""Benchmark of the winding-number hot path on B300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference] [--workload NAME]

One step = the whole hot path on one synthetic mesh and grid:
  face packing (dv_mesh_update_verts), forward winding numbers with compensated
  FP32 sums, near-surface / near-threshold selection, FP64 re-evaluation of the
  selected queries, occupancy (dv_voxelize_grid, mixed precision), and the
  adjoint dL/dV for an N(0,1) upstream (dv_winding_backward).
Metric: query x face pairs per second, counting each pair once for its forward
and backward evaluation (pairs = queries x faces per step).

Default workload ``torus_128``: jittered torus R=0.6, r=0.25, 200x100 grid, 10 %
faces deleted (36 000 faces, open), 128^3 cell-centred grid on [-1,1]^3.
Under torchrun each rank runs its own replica of the workload (the queries of
different meshes are independent; there is no data-path collective): the
value is the work of all ranks over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "query×face solid-angle pairs/s fwd & fwd+bwd, served p50/p99 ms, |Δw|≤1e-4"
UNIT = "pairs/s"
# FP32 lane operations per pair (FMA = 1): the direct formula's count for the forward (offsets,
# lengths, N, dots, D, atan2, accumulate) and for the adjoint (no atan2, ~2x the algebra).
OPS_FWD = 59
OPS_BWD = 120
# FP32 lane operations the grid adjoint kernel executes per pair (counted from its code, FMA = 1):
# 42 for a face alone, 38.5 for a face of an edge-sharing pair (distances and dots shared).
EXEC_BWD_SINGLE = 42.0
EXEC_BWD_PAIRED = 38.5

# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum) from one ncu capture of
# the dominant kernel on the full workload, keyed by (workload, kernel). Each entry records the
# SHA-256 of the kernel's source file at capture time: if that file has changed since, the
# counters no longer describe the kernel and the bench line reports traffic as null.
TRAFFIC = {
    ("torus_128", "bwd_grid"): (11298304, "paper_2407_11272_b300/csrc/winding_bwd.cu",
                                "b6c3d3a58e597cc97d82f06b22944d858cd3bc9d5611dd9cbd4ca087a86631da"),
}

WORKLOADS = {
    "torus_128": dict(desc="jittered open torus R=0.6 r=0.25 200x100, 10% faces deleted (36000 faces), "
                           "128^3 grid on [-1,1]^3, fwd(mixed: Kahan FP32 + FP64 re-eval) + bwd",
                      n=128),
    "shsphere_256": dict(desc="SH-displaced geodesic sphere r=0.7 (204020 faces), 256^3 grid on [-1,1]^3, "
                              "fwd(mixed) + bwd", n=256),
    "torus_64": dict(desc="the torus_128 mesh (36000 faces) on a 64^3 grid on [-1,1]^3, fwd(mixed) + bwd; "
                          "the small case for profiler captures", n=64),
    "icosphere_32": dict(desc="icosphere k=3 r=0.8 (1280 faces), 32^3 grid on [-1,1]^3, fwd(mixed) + bwd", n=32),
}


def _mesh_for(name):
    from paper_2407_11272_b300 import meshgen

    if name in ("torus_128", "torus_64"):
        return meshgen.jittered_torus()
    if name == "shsphere_256":
        return meshgen.sh_sphere()
    if name == "icosphere_32":
        return meshgen.icosphere(3, 0.8)
    raise SystemExit(f"unknown workload {name}")


def _traffic(workload, kernel):
    """Captured DRAM bytes per launch of `kernel` on `workload`, or None if not captured or if the
    kernel's source changed after the capture."""
    import hashlib

    ent = TRAFFIC.get((workload, kernel))
    if not ent:
        return None
    nbytes, src, digest = ent
    path = os.path.join(ROOT, src)
    if not os.path.exists(path):
        return None
    with open(path, "rb") as fh:
        if hashlib.sha256(fh.read()).hexdigest() != digest:
            return None
    return nbytes


def _dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            return json.load(fh), "measured"
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "sm_max_mhz": 2032.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if not self.path or not os.path.exists(self.path):
            return out
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return out
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower().startswith("active")})
        out.update(sm_mhz=statistics.median(sm) if sm else None, sm_max_mhz=max(mx) if mx else None,
                   reasons=reasons, samples=len(rows))
        return out


def _cpu_baseline(V, F, grid_n, budget_s=12.0, seed=4):
    """The FP64 oracle as it stands, on this host's cores: forward + gradient on a seeded query
    sample sized (from two calibration runs) to about budget_s seconds."""
    import oracle
    from paper_2407_11272_b300 import meshgen

    nq = grid_n ** 3
    g = meshgen.upstream_gradient(nq, seed=1).astype(np.float64)

    def run(idx):
        Q = oracle.grid_points([-1.0] * 3, [1.0] * 3, [grid_n] * 3, idx)
        t0 = time.perf_counter()
        oracle.winding(V, F, Q)
        oracle.winding_grad(V, F, Q, g[idx])
        return max(time.perf_counter() - t0, 1e-4)

    per_q = run(meshgen.query_subsample(nq, 512, seed=seed + 1)) / 512
    n2 = int(np.clip(1.5 / per_q, 512, nq))
    per_q = run(meshgen.query_subsample(nq, n2, seed=seed + 2)) / n2
    n = int(np.clip(budget_s / per_q, 512, nq))
    dt = run(meshgen.query_subsample(nq, n, seed=seed))
    return {"value": n * len(F) / dt, "unit": UNIT, "cores": oracle.max_threads(), "kind": "oracle",
            "sample": f"{n} seeded grid queries (of {nq}) x all {len(F)} faces, FP64 forward + gradient, "
                      f"{dt:.1f} s"}


def aggregate_ranks(local_ms: float, pairs_per_step: int, steps: int, ws: int, device=None):
    """Whole-job throughput: every rank ran its own replica of `steps` steps; the job time is the
    slowest rank's (max over ranks), and the value counts the pairs of all ranks.
    Returns (job_ms, pairs_per_second). Works with any initialized process group (NCCL or gloo)."""
    job_ms = float(local_ms)
    if ws > 1:
        import torch
        import torch.distributed as dist

        t = torch.tensor([job_ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        job_ms = float(t.item())
    return job_ms, ws * pairs_per_step * steps / (job_ms * 1e-3)


def run_reference(args):
    ws, rank, _ = _dist_env()
    if rank != 0:
        return 0
    V, F = _mesh_for(args.workload)
    n = WORKLOADS[args.workload]["n"]
    import oracle
    from paper_2407_11272_b300 import meshgen

    nq = n ** 3
    g = meshgen.upstream_gradient(nq, seed=1).astype(np.float64)

    def cells(idx):  # voxel centres of the sampled cells only (the full grid may not fit)
        return oracle.grid_points([-1.0] * 3, [1.0] * 3, [n] * 3, idx)

    # size each step to a few seconds of CPU work
    probe = meshgen.query_subsample(nq, 512, seed=6)
    t0 = time.perf_counter()
    oracle.winding(V, F, cells(probe))
    oracle.winding_grad(V, F, cells(probe), g[probe])
    per_q = max(time.perf_counter() - t0, 1e-4) / 512
    nsamp = int(np.clip(4.0 / per_q, 32, nq))
    times = []
    for step in range(args.warmup + args.steps):
        idx = meshgen.query_subsample(nq, nsamp, seed=100 + step)
        Qs = cells(idx)
        t0 = time.perf_counter()
        oracle.winding(V, F, Qs)
        oracle.winding_grad(V, F, Qs, g[idx])
        if step >= args.warmup:
            times.append(time.perf_counter() - t0)
    total = sum(times)
    value = nsamp * len(F) * len(times) / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "desc": WORKLOADS[args.workload]["desc"], "faces": int(len(F)),
                   "grid": n, "sample_queries_per_step": nsamp},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.max_threads(), "kind": "oracle",
                         "sample": f"{nsamp} seeded grid queries per step x all {len(F)} faces, FP64 forward + "
                                   f"gradient"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def run_native(args):
    import torch

    from paper_2407_11272_b300 import build, dv, meshgen

    ws, rank, local = _dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    build.build()
    V, F = _mesh_for(args.workload)
    n = WORKLOADS[args.workload]["n"]
    grid = dv.Grid.cube(n)
    nq, nf = grid.num_queries, len(F)
    pairs = nq * nf
    Vd = torch.from_numpy(V).to(dev)
    Fd = torch.from_numpy(F).to(dev)
    g = torch.from_numpy(meshgen.upstream_gradient(nq, seed=1)).to(dev)
    mesh = dv.dv_mesh_create(Vd, Fd)
    dv.dv_mesh_reserve(mesh, grid)
    w = torch.empty(nq, dtype=torch.float32, device=dev)
    occ = torch.empty(nq, dtype=torch.uint8, device=dev)
    dV = torch.empty((len(V), 3), dtype=torch.float32, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # 256 MB > 126 MB L2
    stream = torch.cuda.current_stream()
    # The forward (+ FP64 re-evaluation) and the adjoint are independent given the packed mesh and
    # use separate scratch, so they can run on two streams: the FP64 pass (FP64 pipe) then overlaps
    # the adjoint (FP32 pipe). The forward stream has the higher priority so its CTAs are placed first.
    s_fwd = torch.cuda.Stream(device=dev, priority=-1)
    s_bwd = torch.cuda.Stream(device=dev, priority=0)

    def step():
        dv.dv_mesh_update_verts(mesh, Vd, stream=stream)
        if args.streams == 1:
            dv.dv_voxelize_grid(mesh, grid, out_w=w, out_occ=occ, precision=args.precision, stream=stream)
            dv.dv_winding_backward(mesh, g, grid=grid, out=dV, stream=stream)
            return
        s_fwd.wait_stream(stream)
        s_bwd.wait_stream(stream)
        dv.dv_voxelize_grid(mesh, grid, out_w=w, out_occ=occ, precision=args.precision, stream=s_fwd)
        dv.dv_winding_backward(mesh, g, grid=grid, out=dV, stream=s_bwd)
        stream.wait_stream(s_fwd)
        stream.wait_stream(s_bwd)

    for _ in range(args.warmup):
        flush.fill_(1.0)
        step()
    torch.cuda.synchronize()
    # one report outside the timed region: how many queries the FP64 pass re-evaluates
    _, _, rep = dv.dv_voxelize_grid(mesh, grid, out_w=w, out_occ=occ, precision=args.precision, report=True)

    if ws > 1:
        import torch.distributed as dist

        dist.barrier()
    torch.cuda.synchronize()
    dv.dv_profile_reset()
    launches0 = dv.dv_launch_count()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        dv.dv_profile_enable(True)
        for a, b in evs:
            flush.fill_(1.0)  # L2 flush between timed steps, outside the events
            a.record(stream)
            step()
            b.record(stream)
        torch.cuda.synchronize()
        dv.dv_profile_enable(False)
    launches = dv.dv_launch_count() - launches0
    times_ms = [a.elapsed_time(b) for a, b in evs]
    prof = dv.dv_profile_read()
    total_ms, value = aggregate_ranks(float(sum(times_ms)), pairs, args.steps, ws, dev)
    bnd = _boundary_adjoint(mesh, g, grid, dV, prof, stream, dev)

    # roofline of the dominant kernel: algorithmic FP32 lane operations per launch / measured duration
    peaks, peak_src = _peaks()
    sm_mhz = float(peaks.get("sm_max_mhz", 2032.0))
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    fp32_peak = sms * 128 * sm_mhz * 1e6  # lane-ops/s, FMA counted once
    dom = max(prof.items(), key=lambda kv: kv[1][0]) if prof else ("none", (0.0, 1))
    dname, (dms, dn) = dom
    ops = {"fwd_grid_kahan": OPS_FWD, "fwd_grid": OPS_FWD, "fwd_grid_fp16": OPS_FWD, "fwd_strip_kahan": OPS_FWD,
           "fwd_strip": OPS_FWD, "bwd_grid": OPS_BWD}.get(dname, OPS_FWD)
    avg_s = dms / max(dn, 1) * 1e-3
    achieved = ops * pairs / avg_s if avg_s > 0 else 0.0
    traffic = _traffic(args.workload, dname)
    roof = {"bound": "alu", "kernel": dname, "achieved": achieved / 1e12, "peak": fp32_peak / 1e12,
            "unit": "Tlane-op/s (FP32, FMA=1)", "frac": achieved / fp32_peak if fp32_peak else None,
            "traffic": traffic, "ops_per_pair": ops,
            "peak_note": f"{sms} SMs x 128 FP32 lanes x {sm_mhz:.0f} MHz ({peak_src} sm_max_mhz)"}
    if dname == "bwd_grid" and avg_s > 0:
        # the same rate on the basis of the operations the kernel executes (faces in pairs and alone)
        pair_recs, singles = dv.dv_build_face_pairs(F, len(V))
        exec_ops = (EXEC_BWD_PAIRED * 2 * len(pair_recs) + EXEC_BWD_SINGLE * len(singles)) / nf
        roof["executed_ops_per_pair"] = exec_ops
        roof["frac_executed"] = exec_ops * pairs / avg_s / fp32_peak
    kernels = {k: {"ms_total": v[0], "launches": v[1], "share": v[0] / max(sum(x[0] for x in prof.values()), 1e-9)}
               for k, v in sorted(prof.items(), key=lambda kv: -kv[1][0])}

    # end to end through the public API on every rank at once; the job time is the slowest rank's
    e2e = None
    if not args.no_e2e:
        e2e = _e2e(args, V, F, grid, dev)
        e2e_ms, e2e_value = aggregate_ranks(e2e["ms_per_step"], pairs, 1, ws, dev)
        e2e.update(value=e2e_value, ms_per_step=e2e_ms, h2d_bytes_per_step=ws * e2e["h2d_bytes_per_step"],
                   d2h_bytes_per_step=ws * e2e["d2h_bytes_per_step"])
    line = None
    if rank == 0:
        cpu = None if args.no_cpu_baseline else _cpu_baseline(V, F, n)
        ck = clk.summary()
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": args.workload, "desc": WORKLOADS[args.workload]["desc"], "faces": nf,
                       "queries": nq, "pairs_per_step": pairs, "parallelism": f"replicas{ws}",
                       "l2": "flushed between timed steps (256 MB write)", "streams": args.streams,
                       "precision": args.precision,
                       "fp64_reevaluated_queries": rep["n_flagged"]},
            "roofline": roof, "kernels": kernels, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": int(launches),
            "adjoint_boundary": bnd,
            "clocks": {"sm_mhz": ck["sm_mhz"], "sm_max_mhz": ck["sm_max_mhz"], "reasons": ck["reasons"],
                       "samples": ck["samples"]},
        }
        print(json.dumps(line))
    if ws > 1:
        import torch.distributed as dist

        dist.barrier()
        dist.destroy_process_group()
    mesh.close()
    return 0


def _boundary_adjoint(mesh, g, grid, dV_faces, prof, stream, dev):
    """Outside the timed step: the boundary form of the adjoint (dv_winding_backward_boundary) on
    the same upstream, its time per call and its difference from the face-by-face result."""
    import torch

    from paper_2407_11272_b300 import dv

    out = torch.empty_like(dV_faces)
    dv.dv_winding_backward_boundary(mesh, g, grid=grid, out=out, stream=stream)
    torch.cuda.synchronize(dev)
    reps = 3
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(reps):
        dv.dv_winding_backward_boundary(mesh, g, grid=grid, out=out, stream=stream)
    b.record(stream)
    torch.cuda.synchronize(dev)
    ms = a.elapsed_time(b) / reps
    ref = dV_faces.double()
    rel = float(torch.linalg.norm(out.double() - ref) / torch.linalg.norm(ref).clamp_min(1e-300))
    face_ms = prof["bwd_grid"][0] / max(prof["bwd_grid"][1], 1) if "bwd_grid" in prof else None
    nb = dv.dv_mesh_num_boundary_edges(mesh)
    note = "same dL/dV from the boundary edges; not part of the timed step"
    if nb == 0:
        note += "; closed mesh: the exact gradient is 0 and the face adjoint's value is cancellation noise"
    return {"ms_per_call": ms, "face_adjoint_ms": face_ms, "boundary_edges": nb, "rel_diff_vs_face_adjoint": rel,
            "face_adjoint_norm": float(torch.linalg.norm(ref)), "note": note}


def _e2e(args, V, F, grid, dev):
    """Same step through the public API from pinned host buffers: H2D of the mesh and upstream,
    mesh creation (validation + packing), voxelization, adjoint, D2H of w, occupancy and dL/dV."""
    import torch

    from paper_2407_11272_b300 import dv, meshgen

    nq = grid.num_queries
    hV = torch.from_numpy(V).pin_memory()
    hF = torch.from_numpy(F).pin_memory()
    hg = torch.from_numpy(meshgen.upstream_gradient(nq, seed=1)).pin_memory()
    hw = torch.empty(nq, dtype=torch.float32).pin_memory()
    ho = torch.empty(nq, dtype=torch.uint8).pin_memory()
    hd = torch.empty((len(V), 3), dtype=torch.float32).pin_memory()
    h2d = hV.numel() * 4 + hF.numel() * 4 + hg.numel() * 4
    d2h = hw.numel() * 4 + ho.numel() + hd.numel() * 4

    def one():
        Vd = hV.to(dev, non_blocking=True)
        Fd = hF.to(dev, non_blocking=True)
        gd = hg.to(dev, non_blocking=True)
        mesh = dv.dv_mesh_create(Vd, Fd)
        w, occ, _ = dv.dv_voxelize_grid(mesh, grid, precision=args.precision)
        dV = dv.dv_winding_backward(mesh, gd, grid=grid)
        hw.copy_(w, non_blocking=True)
        ho.copy_(occ, non_blocking=True)
        hd.copy_(dV, non_blocking=True)
        torch.cuda.synchronize()
        mesh.close()

    one()
    k = max(1, min(args.steps, 3))
    t0 = time.perf_counter()
    for _ in range(k):
        one()
    dt = (time.perf_counter() - t0) / k
    return {"value": grid.num_queries * len(F) / dt, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "ms_per_step": dt * 1e3}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="torus_128")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--precision", choices=["mixed", "kahan", "fp32", "fp16"], default="mixed",
                    help="forward arithmetic (mixed = Kahan FP32 + FP64 re-evaluation, the default)")
    ap.add_argument("--streams", type=int, choices=[1, 2], default=1,
                    help="1: one stream (default); 2: forward and adjoint on two streams")
    args = ap.parse_args(argv)
    args.warmup = max(3, args.warmup)  # at least 3 untimed warm-up steps, whatever was asked
    if args.impl == "reference":
        return run_reference(args)
    return run_native(args)


if __name__ == "__main__":
    sys.exit(main())
