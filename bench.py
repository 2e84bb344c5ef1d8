"""Benchmark of the winding-number hot path on B300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference] [--workload NAME]

One step = the whole hot path on one synthetic mesh and grid:
  face packing (dv_mesh_update_verts), forward winding numbers with compensated
  FP32 sums, near-surface / near-threshold selection, FP64 re-evaluation of the
  selected queries, occupancy (dv_voxelize_grid, mixed precision), and the
  adjoint dL/dV for an N(0,1) upstream (dv_winding_backward).
Metric: query x face pairs per second, counting each pair once for its forward
and backward evaluation (pairs = queries x faces per step); the forward and the
adjoint rates are reported beside it.

Default workload ``shsphere_256``: a sphere of radius 0.7 displaced by a seeded
spherical-harmonic field (degrees <= 8), as a frequency-101 geodesic mesh with
204 020 faces, on a 256^3 cell-centred grid over [-1,1]^3 (3.42e12 pairs per
step). ``torus_128`` (jittered open torus, 36 000 faces, 128^3) and the small
cases remain selectable with --workload.

Beside the timed steps, outside the timed region, the line carries
  * ``accuracy``: plain FP32, Kahan FP32 and mixed precision against the FP64
    oracle on a seeded sample of 100 000 voxel centres (max |dw| farther than
    1e-3 from the surface, occupancy mismatches outside ties);
  * ``served``: the served mixed stream (512 requests, Poisson 200 req/s, and
    again at 0.7 x the measured capacity) with p50/p99 latency and pairs/s;
  * ``cpu_baseline``: the oracle on the host's cores on a bounded sample.
The oracle runs in a separate process started before the first CUDA call: the
CPU baseline is timed while the GPU is idle, and the accuracy sample's oracle
values are computed while the GPU steps run.
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
# FP32 lane operations per pair (FMA = 1) of the direct formula: offsets, lengths, N, dots, D,
# arctangent and accumulation for the forward; about twice that algebra (no arctangent) for the
# adjoint. The kernels share distances and dots between consecutive faces and execute fewer, so
# a rate on this basis is an algorithmic-equivalent rate that can exceed the FP32 peak.
OPS_FWD = 59
OPS_BWD = 120
# FP32 lane operations the grid adjoint kernel executes per pair, counted from its code (FMA = 1;
# edge form: per point 3, per edge 9 per query): 36 for a face alone (3 points, 3 edges), 24 for a
# face of an edge-sharing pair (4 points and 4 edges per two faces). Used when no measured count
# (EXECUTED) matches the kernel's current source.
EXEC_BWD_SINGLE = 36.0
EXEC_BWD_PAIRED = 24.0

# Executed operations per unit, measured by ncu thread-instruction counters on the same mesh over
# a 64^3 grid: FFMA + FADD + FMUL + 2 x (FFMA2 + FADD2 + FMUL2) per query x face pair for the
# FP32 kernels, DFMA + DADD + DMUL per re-evaluated query x strip event for the FP64 pass. Keyed
# by (mesh, kernel); each entry records the SHA-256 of the kernel's source file at capture time
# and is ignored once that file changes.
EXECUTED = {
    # 8.255e11 FP32 lane ops / (262 144 x 204 020) pairs; profiles/hot_kernels_shsphere_64_ncu.md
    ("sh_sphere", "fwd_strip_kahan"): (15.44, "paper_2407_11272_b300/csrc/winding_fwd.cu",
                                       "c21070f8ec6075ccb701b639ef36e42e75799744f8df52c1773f722b409f7a49"),
    # 8.385e13 FP32 lane ops / (16 777 216 x 204 020) pairs, one full-size launch (edge form)
    ("sh_sphere", "bwd_grid"): (24.50, "paper_2407_11272_b300/csrc/winding_bwd.cu",
                                "6f0f6bd10313ca5aca21cd9b85b164b93a52b8b61bc2d9fca3480a979991b8f6"),
    # 3.351e9 FP64 ops / (480 flagged queries x 205 030 events)
    ("sh_sphere", "reeval_fp64"): (34.05, "paper_2407_11272_b300/csrc/winding_fp64.cu",
                                   "8c594e484ada6aa7cf91bbf908944d2813b8df3c27fe0c9620151088ab2747b9"),
}

# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum) from one ncu capture of
# the dominant kernel on the full workload, keyed by (workload, kernel), with the same source
# digest rule as EXECUTED.
TRAFFIC = {
    # 87 481 600 B read + 23 069 440 B written, one full-size launch (799 x 5 CTAs);
    # profiles/bwd_grid_shsphere_256_dram.md
    ("shsphere_256", "bwd_grid"): (110551040, "paper_2407_11272_b300/csrc/winding_bwd.cu",
                                   "6f0f6bd10313ca5aca21cd9b85b164b93a52b8b61bc2d9fca3480a979991b8f6"),
}

ACC_QUERIES = 100_000  # seeded voxel-centre sample of the accuracy block
ACC_SEED = 4

WORKLOADS = {
    "shsphere_256": dict(desc="SH-displaced geodesic sphere r=0.7 (l<=8, c~N(0,0.02^2), seed 3; 204020 faces), "
                              "256^3 grid on [-1,1]^3, fwd(mixed: Kahan FP32 + FP64 re-eval) + bwd",
                         n=256, mesh="sh_sphere"),
    "torus_128": dict(desc="jittered open torus R=0.6 r=0.25 200x100, 10% faces deleted (36000 faces), "
                           "128^3 grid on [-1,1]^3, fwd(mixed: Kahan FP32 + FP64 re-eval) + bwd",
                      n=128, mesh="torus"),
    "shsphere_64": dict(desc="the shsphere_256 mesh (204020 faces) on a 64^3 grid on [-1,1]^3, fwd(mixed) + bwd; "
                             "the small case for profiler captures", n=64, mesh="sh_sphere"),
    "torus_64": dict(desc="the torus_128 mesh (36000 faces) on a 64^3 grid on [-1,1]^3, fwd(mixed) + bwd; "
                          "the small case for profiler captures", n=64, mesh="torus"),
    "icosphere_32": dict(desc="icosphere k=3 r=0.8 (1280 faces), 32^3 grid on [-1,1]^3, fwd(mixed) + bwd", n=32,
                         mesh="icosphere"),
}
DEFAULT_WORKLOAD = "shsphere_256"


def _mesh_for(name):
    from paper_2407_11272_b300 import meshgen

    kind = WORKLOADS[name]["mesh"]
    if kind == "torus":
        return meshgen.jittered_torus()
    if kind == "sh_sphere":
        return meshgen.sh_sphere()
    return meshgen.icosphere(3, 0.8)


def _source_matches(src, digest):
    import hashlib

    path = os.path.join(ROOT, src)
    if not os.path.exists(path):
        return False
    with open(path, "rb") as fh:
        return hashlib.sha256(fh.read()).hexdigest() == digest


def _traffic(workload, kernel):
    """Captured DRAM bytes per launch of `kernel` on `workload`, or None if not captured or if the
    kernel's source changed after the capture."""
    ent = TRAFFIC.get((workload, kernel))
    if not ent or not _source_matches(ent[1], ent[2]):
        return None
    return ent[0]


def _executed(workload, kernel):
    """Measured executed operations per unit of `kernel` on `workload`'s mesh, or None."""
    ent = EXECUTED.get((WORKLOADS[workload]["mesh"], kernel))
    if not ent or not _source_matches(ent[1], ent[2]):
        return None
    return ent[0]


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


def _oracle_leg_main(conn, workload, acc_queries, budget_s):
    """Body of the spawned oracle process: on "go" the CPU baseline (the GPU side waits meanwhile),
    then the oracle's w and distance to the surface at the accuracy sample's voxel centres."""
    import oracle
    from paper_2407_11272_b300 import meshgen

    n = WORKLOADS[workload]["n"]
    V, F = _mesh_for(workload)
    oracle.build()
    if conn.recv() != "go":
        return
    conn.send(("baseline", _cpu_baseline(V, F, n, budget_s) if budget_s > 0 else None))
    if acc_queries <= 0:
        return
    idx = meshgen.query_subsample(n ** 3, acc_queries, seed=ACC_SEED)
    Q = oracle.grid_points([-1.0] * 3, [1.0] * 3, [n] * 3, idx)
    t0 = time.perf_counter()
    w64 = oracle.winding(V, F, Q)
    t1 = time.perf_counter()
    d = oracle.point_mesh_distance(V, F, Q)
    t2 = time.perf_counter()
    acc = {"idx": idx, "w64": w64, "d": d, "winding_s": t1 - t0, "distance_s": t2 - t1,
           "threads": oracle.max_threads(), "cells": n ** 3}
    # a closed mesh (every edge shared by exactly two faces): its occupancy on the whole grid from
    # signed ray crossings, which needs no solid angle
    und = np.sort(np.concatenate([F[:, [0, 1]], F[:, [1, 2]], F[:, [2, 0]]]), axis=1)
    _, cnt = np.unique(und, axis=0, return_counts=True)
    if np.all(cnt == 2):
        t3 = time.perf_counter()
        wr, amb = oracle.ray_winding_grid(V, F, [-1.0] * 3, [1.0] * 3, [n] * 3)
        acc["whole_grid"] = {"occ_bits": np.packbits(wr >= 1), "undecided_bits": np.packbits(amb),
                             "values": sorted(int(v) for v in np.unique(wr[~amb])), "seconds": time.perf_counter() - t3}
    conn.send(("accuracy", acc))


class OracleLeg:
    """The oracle's share of the bench in a process of its own (spawned, so it is started before
    and independent of any CUDA context): the CPU baseline, timed while the GPU is idle, then the
    accuracy sample's reference values, computed while the GPU steps run."""

    def __init__(self, workload, acc_queries, budget_s=12.0):
        import multiprocessing as mp

        ctx = mp.get_context("spawn")
        self.conn, child = ctx.Pipe()
        self.proc = ctx.Process(target=_oracle_leg_main, args=(child, workload, acc_queries, budget_s), daemon=True)
        self.proc.start()
        child.close()

    def baseline(self):
        self.conn.send("go")
        tag, val = self.conn.recv()
        assert tag == "baseline"
        return val

    def accuracy(self, timeout_s=1800.0):
        if not self.conn.poll(timeout_s):
            return None
        tag, val = self.conn.recv()
        assert tag == "accuracy"
        return val

    def close(self):
        if self.proc.is_alive():
            self.proc.terminate()
        self.proc.join(timeout=10)


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


def _kernel_rooflines(args, prof, pairs, nflagged, ne, F, nv, fp32_peak, fp64_peak):
    """Per hot kernel: the rate on the algorithmic basis (FP32 lane operations of the direct
    formula per pair; exceeds 1 by operation sharing) and on the executed basis (operations the
    kernel executes per unit, measured by ncu counters, else counted from the code), both against
    the peak of the pipe that bounds it."""
    out = {}
    for name, alg in (("fwd_strip_kahan", OPS_FWD), ("fwd_strip", OPS_FWD), ("bwd_grid", OPS_BWD)):
        if name not in prof:
            continue
        ms, cnt = prof[name]
        avg_s = ms / max(cnt, 1) * 1e-3
        rate = pairs / avg_s
        ent = {"ms_per_launch": avg_s * 1e3, "units": "query x face pairs", "units_per_launch": pairs,
               "pairs_per_s": rate, "peak": fp32_peak / 1e12, "peak_unit": "Tlane-op/s (FP32, FMA=1)",
               "alg_ops_per_pair": alg, "frac_alg_equivalent": alg * rate / fp32_peak}
        ex = _executed(args.workload, name)
        basis = ("ncu thread-instruction counters, one full-size launch" if name == "bwd_grid"
                 else "ncu thread-instruction counters on the same mesh at 64^3 (256^3 agrees)")
        if ex is None and name == "bwd_grid":
            pair_recs, singles = __import__("paper_2407_11272_b300.dv", fromlist=["dv"]).dv_build_face_pairs(F, nv)
            ex = (EXEC_BWD_PAIRED * 2 * len(pair_recs) + EXEC_BWD_SINGLE * len(singles)) / len(F)
            basis = (f"counted from the kernel's code ({EXEC_BWD_PAIRED:g} per paired face, "
                     f"{EXEC_BWD_SINGLE:g} per single face)")
        if ex is not None:
            ent.update(executed_ops_per_pair=ex, frac_executed=ex * rate / fp32_peak, executed_basis=basis)
        out[name] = ent
    if "reeval_fp64" in prof and nflagged:
        ms, cnt = prof["reeval_fp64"]
        avg_s = ms / max(cnt, 1) * 1e-3
        units = nflagged * ne
        ent = {"ms_per_launch": avg_s * 1e3, "units": "re-evaluated query x strip event",
               "units_per_launch": units, "units_per_s": units / avg_s, "peak": fp64_peak / 1e12,
               "peak_unit": "T DFMA-lane-op/s (FP64)"}
        ex = _executed(args.workload, "reeval_fp64")
        if ex is not None:
            ent.update(executed_ops_per_unit=ex, frac_executed=ex * units / avg_s / fp64_peak,
                       executed_basis="ncu thread-instruction counters on the same mesh at 64^3")
        out["reeval_fp64"] = ent
    return out


def _accuracy_gpu(mesh, grid, w, occ, idx, stream, dev):
    """Forward outputs at the accuracy sample in plain FP32, Kahan FP32 and mixed precision (each a
    whole-grid dv_voxelize_grid, timed with CUDA events), outside the timed region."""
    import torch

    from paper_2407_11272_b300 import dv

    idx_t = torch.from_numpy(idx).to(dev)
    out = {}
    for prec in ("fp32", "kahan", "mixed"):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        dv.dv_voxelize_grid(mesh, grid, out_w=w, out_occ=occ, precision=prec, stream=stream)
        b.record(stream)
        torch.cuda.synchronize(dev)
        # the whole grid's occupancy too, for closed meshes' ray-crossing check (2 MB as bits)
        out[prec] = (w[idx_t].cpu().numpy(), occ[idx_t].cpu().numpy(), a.elapsed_time(b),
                     np.packbits(occ.cpu().numpy().astype(bool)))
    return out


def _accuracy(gpu, ref, n_flagged, pairs):
    """Errors of each precision against the oracle at the sample: max and mean |dw| farther than
    1e-3 from the surface (the parity bar is 1e-4), max |dw| nearer, and occupancy mismatches
    among queries that are not ties (|w64 - 0.5| > 1e-9)."""
    w64, d = ref["w64"], ref["d"]
    far = d > 1e-3
    tie = np.abs(w64 - 0.5) <= 1e-9
    occ64 = w64 > 0.5
    out = {"queries": int(len(w64)), "seed": ACC_SEED, "n_far": int(far.sum()), "n_near": int((~far).sum()),
           "ties": int(tie.sum()),
           "oracle": f"FP64 winding + exact point-triangle distance, {ref['threads']} threads, "
                     f"{ref['winding_s']:.1f} s + {ref['distance_s']:.1f} s"}
    for prec, (wg, og, ms, _) in gpu.items():
        err = np.abs(wg.astype(np.float64) - w64)
        mism = (og.astype(bool) != occ64) & ~tie
        ent = {"fwd_ms": ms, "fwd_pairs_per_s": pairs / (ms * 1e-3),
               "max_abs_dw_far": float(err[far].max()) if far.any() else None,
               "mean_abs_dw_far": float(err[far].mean()) if far.any() else None,
               "max_abs_dw_near": float(err[~far].max()) if (~far).any() else None,
               "occ_mismatch": int(mism.sum()), "occ_mismatch_far": int((mism & far).sum()),
               "occ_mismatch_near": int((mism & ~far).sum())}
        ent["meets_1e-4_far"] = ent["max_abs_dw_far"] is None or ent["max_abs_dw_far"] <= 1e-4
        if prec == "mixed":
            ent["n_flagged_grid"] = int(n_flagged)
        out[prec] = ent
    wg = ref.get("whole_grid")
    if wg is not None:
        # every voxel of the grid: occupancy against the signed ray-crossing count of the closed mesh
        total = int(ref["cells"])
        amb = np.unpackbits(wg["undecided_bits"])[:total].astype(bool)
        ray = np.unpackbits(wg["occ_bits"])[:total].astype(bool)
        whole = {"cells": total, "undecided": int(amb.sum()), "ray_values": wg["values"],
                 "method": "signed ray crossings along +x per row (closed mesh), independent of Eq. 5",
                 "oracle_s": wg["seconds"]}
        for prec, (_, _, _, bits) in gpu.items():
            occ = np.unpackbits(bits)[:total].astype(bool)
            whole[f"occ_mismatch_{prec}"] = int(((occ != ray) & ~amb).sum())
        out["whole_grid"] = whole
    return out


def _served(dev):
    """The served mixed stream (512 requests, Poisson 200 req/s, seed 5), then the same stream at
    0.7 x the capacity that run shows (its offered load exceeds capacity), through serve.Server."""
    from paper_2407_11272_b300 import serve

    sv = serve.served_runs(capacity_run=False, device=dev)
    keep = ("p50_ms", "p99_ms", "mean_ms", "pairs_per_s", "requests_per_s", "makespan_s", "requests", "batches",
            "mean_batch", "batch_host_ms_mean", "batch_host_ms_p50", "batch_host_ms_max", "batch_host_s_total",
            "rate", "fraction")
    out = {"workload": sv["workload"], "mean_pairs_per_request": sv["mean_pairs_per_request"],
           "offered_pairs_per_s": sv["offered_pairs_per_s"], "capacity_from": sv["capacity_from"]}
    for k in ("at_rate", "sub_capacity"):
        out[k] = {x: sv[k][x] for x in keep if x in sv[k]}
    return out


def run_native(args):
    ws, rank, local = _dist_env()
    n = WORKLOADS[args.workload]["n"]
    leg = None
    if rank == 0 and not (args.no_cpu_baseline and args.no_accuracy):
        # before the first CUDA call: the oracle's process is spawned, not forked from a CUDA context
        leg = OracleLeg(args.workload, 0 if args.no_accuracy else ACC_QUERIES, 0.0 if args.no_cpu_baseline else 12.0)

    import torch

    from paper_2407_11272_b300 import build, dv, meshgen

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    build.build()
    V, F = _mesh_for(args.workload)
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

    torch.cuda.synchronize()
    cpu = leg.baseline() if leg is not None else None  # the oracle timed while the GPU is idle

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
    dv.dv_mesh_check(mesh)  # no bounded wait ran out during the timed steps

    # forward (near-surface flags, FP32 pass, split reduction, FP64 pass) and adjoint (face-parallel
    # kernel, vertex gather) rates from the per-kernel event times of the timed steps
    fwd_k = ("near_surface_grid", "fwd_strip_kahan", "fwd_strip", "split_reduce", "reeval_fp64")
    bwd_k = ("bwd_grid", "gather_dverts")
    fwd_ms = sum(prof[k][0] for k in fwd_k if k in prof) / args.steps
    bwd_ms = sum(prof[k][0] for k in bwd_k if k in prof) / args.steps

    # roofline of the dominant kernel: algorithmic FP32 lane operations per launch / measured duration
    peaks, peak_src = _peaks()
    sm_mhz = float(peaks.get("sm_max_mhz", 2032.0))
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    fp32_peak = sms * 128 * sm_mhz * 1e6  # lane-ops/s, FMA counted once
    fp64_peak = sms * 2 * sm_mhz * 1e6    # FP64 lanes: 1/64 of the FP32 lanes
    dom = max(prof.items(), key=lambda kv: kv[1][0]) if prof else ("none", (0.0, 1))
    dname, (dms, dn) = dom
    kr = _kernel_rooflines(args, prof, pairs, rep["n_flagged"], dv.dv_mesh_num_strip_events(mesh), F, len(V),
                           fp32_peak, fp64_peak)
    ops = {"fwd_strip_kahan": OPS_FWD, "fwd_strip": OPS_FWD, "bwd_grid": OPS_BWD}.get(dname, OPS_FWD)
    avg_s = dms / max(dn, 1) * 1e-3
    achieved = ops * pairs / avg_s if avg_s > 0 else 0.0
    roof = {"bound": "alu", "kernel": dname, "achieved": achieved / 1e12, "peak": fp32_peak / 1e12,
            "unit": "Tlane-op/s (FP32, FMA=1)", "frac": achieved / fp32_peak if fp32_peak else None,
            "frac_basis": f"algorithmic-equivalent: {ops} FP32 lane-ops per pair of the direct formula; above 1 "
                          "because the kernel shares distances and dots between faces",
            "traffic": _traffic(args.workload, dname), "ops_per_pair": ops,
            "peak_note": f"{sms} SMs x 128 FP32 lanes x {sm_mhz:.0f} MHz ({peak_src} sm_max_mhz)"}
    if dname in kr and "frac_executed" in kr[dname]:
        roof.update(executed_ops_per_pair=kr[dname]["executed_ops_per_pair"],
                    frac_executed=kr[dname]["frac_executed"], executed_basis=kr[dname]["executed_basis"])
    kernels = {k: {"ms_total": v[0], "launches": v[1], "share": v[0] / max(sum(x[0] for x in prof.values()), 1e-9)}
               for k, v in sorted(prof.items(), key=lambda kv: -kv[1][0])}
    bnd = _boundary_adjoint(mesh, g, grid, dV, prof, stream, dev)

    acc_gpu = None
    if leg is not None and not args.no_accuracy:
        acc_gpu = _accuracy_gpu(mesh, grid, w, occ, meshgen.query_subsample(nq, ACC_QUERIES, seed=ACC_SEED),
                                stream, dev)

    # end to end through the public API on every rank at once; the job time is the slowest rank's
    e2e = None
    if not args.no_e2e:
        e2e = _e2e(args, V, F, grid, dev, total_ms / args.steps)
        e2e_ms, e2e_value = aggregate_ranks(e2e["ms_per_step"], pairs, 1, ws, dev)
        e2e.update(value=e2e_value, ms_per_step=e2e_ms, h2d_bytes_per_step=ws * e2e["h2d_bytes_per_step"],
                   d2h_bytes_per_step=ws * e2e["d2h_bytes_per_step"])
    mesh.close()
    del flush, w, occ, g, dV
    torch.cuda.empty_cache()

    line = None
    if rank == 0:
        acc = None
        if acc_gpu is not None:
            ref = leg.accuracy()
            acc = _accuracy(acc_gpu, ref, rep["n_flagged"], pairs) if ref is not None else {"error": "oracle timed out"}
        if leg is not None:
            leg.close()
        served = None if args.no_served else _served(dev)
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
            "fwd_pairs_per_s": ws * pairs / (fwd_ms * 1e-3) if fwd_ms > 0 else None,
            "bwd_pairs_per_s": ws * pairs / (bwd_ms * 1e-3) if bwd_ms > 0 else None,
            "fwd_ms_per_step": fwd_ms, "bwd_ms_per_step": bwd_ms,
            "roofline": roof, "roofline_kernels": kr, "kernels": kernels, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": int(launches),
            "accuracy": acc,
            "served": served,
            "adjoint_boundary": bnd,
            "clocks": {"sm_mhz": ck["sm_mhz"], "sm_max_mhz": ck["sm_max_mhz"], "reasons": ck["reasons"],
                       "samples": ck["samples"]},
        }
        print(json.dumps(line))
    elif leg is not None:
        leg.close()
    if ws > 1:
        import torch.distributed as dist

        dist.barrier()
        dist.destroy_process_group()
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


def _e2e(args, V, F, grid, dev, step_ms):
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
    k = max(1, min(args.steps, 2 if step_ms > 2000 else 3))
    t0 = time.perf_counter()
    for _ in range(k):
        one()
    dt = (time.perf_counter() - t0) / k
    return {"value": grid.num_queries * len(F) / dt, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "ms_per_step": dt * 1e3, "steps": k}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1,
                    help="number of GPUs (ranks); N > 1 must be launched with torchrun --nproc-per-node N")
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default=DEFAULT_WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true", help="skip the 1e5-query accuracy block")
    ap.add_argument("--no-served", action="store_true", help="skip the served mixed stream")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--precision", choices=["mixed", "kahan", "fp32", "fp16"], default="mixed",
                    help="forward arithmetic (mixed = Kahan FP32 + FP64 re-evaluation, the default)")
    ap.add_argument("--streams", type=int, choices=[1, 2], default=1,
                    help="1: one stream (default); 2: forward and adjoint on two streams")
    args = ap.parse_args(argv)
    args.warmup = max(3, args.warmup)  # at least 3 untimed warm-up steps, whatever was asked
    ws = _dist_env()[0]
    if args.gpus != ws:
        print(f"bench.py: --gpus {args.gpus} but {ws} rank(s) were started (WORLD_SIZE={ws}); run N GPUs as "
              f"python -m torch.distributed.run --nproc-per-node {args.gpus} --master-addr 127.0.0.1 bench.py "
              f"--gpus {args.gpus}", file=sys.stderr)
        return 2
    if args.impl == "reference":
        return run_reference(args)
    return run_native(args)


if __name__ == "__main__":
    sys.exit(main())
