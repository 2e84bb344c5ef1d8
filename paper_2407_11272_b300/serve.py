"""Request server: continuous batching of voxelization and gradient requests on one GPU.

Requests (a mesh, a grid, optionally an upstream gradient for dL/dV) arrive over time. The
host loop
  * admits arrived requests in arrival order while their estimated device memory fits the
    budget (memory-admitted slots), uploads them and creates their resident meshes
    (``dv_mesh_create``) on an upload stream;
  * groups the admitted requests that are not yet running into a batch and launches the batch
    with ``dv_run_batch``: one CUDA graph with one parallel branch per request (forward in mixed
    precision, FP64 re-evaluation, occupancy, adjoint when asked), so the work of different
    requests overlaps on the device; several batches are in flight at once on their own
    streams, so requests that arrive while others run start as soon as memory allows;
  * retires finished batches (CUDA events), copies results to pinned host memory, frees the
    meshes in stream order and returns their memory to the budget.
Each request's result equals running it alone (same kernels and launch plans per request).

    python -m paper_2407_11272_b300.serve [--requests 512] [--rate 200] [--seed 5]

generates the served mixed stream (unions of 1-6 jittered ellipsoids, faces log-uniform in
[500, 100 000], grids uniform over {32, 64, 96, 128, 192}^3, 30 % with an N(0,1) upstream,
Poisson arrivals), serves it, measures capacity with all requests queued at t = 0, serves it
again at 0.7 x that capacity, and prints one JSON line with p50/p99 latency and pairs/s.
"""
from __future__ import annotations

import argparse
import collections
import json
import math
import time
from dataclasses import dataclass, field

import numpy as np

from . import meshgen

GRID_SIZES = (32, 64, 96, 128, 192)


@dataclass
class Request:
    rid: int
    verts: np.ndarray
    faces: np.ndarray
    n: int                     # grid resolution (cube over [-1, 1]^3)
    want_grad: bool
    arrival: float             # seconds after the start of serving
    upstream_seed: int = 0

    @property
    def queries(self) -> int:
        return self.n ** 3

    @property
    def pairs(self) -> int:
        """Query x face pairs evaluated (forward, plus the adjoint when asked)."""
        return self.queries * len(self.faces) * (2 if self.want_grad else 1)


@dataclass
class Result:
    rid: int
    occ: np.ndarray
    dverts: np.ndarray | None
    arrival: float
    admitted: float
    launched: float
    done: float
    batch: int

    @property
    def latency(self) -> float:
        return self.done - self.arrival


def make_workload(n_requests: int = 512, rate: float = 200.0, seed: int = 5, f_lo: float = 500, f_hi: float = 1e5,
                  grids=GRID_SIZES, grad_frac: float = 0.3, max_components: int = 6):
    """The served mixed stream: Poisson arrivals at ``rate`` req/s; each request a union of
    1..max_components jittered ellipsoids with a log-uniform face count in [f_lo, f_hi]."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(n_requests):
        t += rng.exponential(1.0 / rate) if rate > 0 else 0.0
        k = int(rng.integers(1, max_components + 1))
        F = int(round(math.exp(rng.uniform(math.log(f_lo), math.log(f_hi)))))
        n = int(rng.choice(grids))
        grad = bool(rng.random() < grad_frac)
        V, Fc = meshgen.ellipsoid_union(F, k, seed=int(rng.integers(1 << 31)))
        out.append(Request(i, V, Fc, n, grad, t, upstream_seed=int(rng.integers(1 << 31))))
    return out


def estimate_bytes(nv: int, nf: int, n: int, want_grad: bool) -> int:
    """Device memory a request holds while admitted: mesh records, adjacency, scratch, outputs."""
    nq = n ** 3
    mesh = nf * (12 + 48 + 96 + 12) + 4 * (nv + 1) + 16
    scratch = nq * (4 + 1 + 4) + min(8 * nq * 16, 64 << 20)  # w, near flags, flagged list, split partials
    outputs = nq * (4 + 1)
    grad = (4 * nq + 12 * nv + 36 * nf * 24) if want_grad else 0
    return int(mesh + scratch + outputs + grad)


class Admission:
    """Memory-admitted slots: FIFO admission while the estimated bytes fit the budget. A request
    larger than the whole budget is admitted only when nothing else is in flight."""

    def __init__(self, budget_bytes: int):
        self.budget = int(budget_bytes)
        self.used = 0
        self.count = 0

    def can_admit(self, nbytes: int) -> bool:
        if self.count == 0:
            return True
        return self.used + nbytes <= self.budget

    def admit(self, nbytes: int) -> None:
        self.used += int(nbytes)
        self.count += 1

    def release(self, nbytes: int) -> None:
        self.used -= int(nbytes)
        self.count -= 1
        assert self.used >= 0 and self.count >= 0


@dataclass
class _Active:
    req: Request
    nbytes: int
    admitted: float
    mesh: object = None
    grid: object = None
    occ: object = None
    up: object = None
    dverts: object = None
    host_occ: object = None
    host_dverts: object = None


@dataclass
class _Batch:
    bid: int
    items: list
    stream: object
    event: object
    launched: float


class Server:
    def __init__(self, device="cuda", mem_budget_bytes: int | None = None, max_batch: int = 16,
                 max_inflight: int = 3, precision: str = "mixed"):
        import torch

        from . import dv

        self.torch, self.dv = torch, dv
        self.dev = torch.device(device)
        if mem_budget_bytes is None:
            free, _ = torch.cuda.mem_get_info(self.dev)
            mem_budget_bytes = int(0.5 * free)
        self.admission = Admission(mem_budget_bytes)
        self.max_batch = max_batch
        self.max_inflight = max_inflight
        self.precision = precision
        self.upload = torch.cuda.Stream(device=self.dev)
        self.streams = [torch.cuda.Stream(device=self.dev) for _ in range(max_inflight)]

    # -- steps of the host loop -------------------------------------------------------------
    def _materialize(self, r: Request, now: float) -> _Active:
        torch, dv = self.torch, self.dv
        nbytes = estimate_bytes(len(r.verts), len(r.faces), r.n, r.want_grad)
        self.admission.admit(nbytes)
        a = _Active(r, nbytes, now)
        with torch.cuda.stream(self.upload):
            Vd = torch.from_numpy(r.verts).pin_memory().to(self.dev, non_blocking=True)
            Fd = torch.from_numpy(r.faces).pin_memory().to(self.dev, non_blocking=True)
            a.mesh = dv.dv_mesh_create(Vd, Fd, stream=self.upload)  # validates and packs; syncs the upload stream
            a.grid = dv.Grid.cube(r.n)
            if r.want_grad:
                g = meshgen.upstream_gradient(r.queries, seed=r.upstream_seed)
                a.up = torch.from_numpy(g).pin_memory().to(self.dev, non_blocking=True)
        return a

    def _launch(self, items: list, bid: int, now: float) -> _Batch:
        torch, dv = self.torch, self.dv
        busy = {id(b.stream) for b in self._inflight}
        stream = next(s for s in self.streams if id(s) not in busy)
        stream.wait_stream(self.upload)
        reqs = []
        with torch.cuda.stream(stream):
            for a in items:
                a.occ = torch.empty(a.req.queries, dtype=torch.uint8, device=self.dev)
                d = {"mesh": a.mesh, "grid": a.grid, "occ": a.occ}
                if a.req.want_grad:
                    a.up.record_stream(stream)
                    a.dverts = torch.empty((len(a.req.verts), 3), dtype=torch.float32, device=self.dev)
                    d.update(upstream=a.up, dverts=a.dverts)
                reqs.append(d)
            th = time.perf_counter()
            dv.dv_run_batch(reqs, precision=self.precision, stream=stream)
            self._batch_host_s.append(time.perf_counter() - th)  # scratch, capture, instantiate, launch
            for a in items:
                a.host_occ = torch.empty(a.req.queries, dtype=torch.uint8, pin_memory=True)
                a.host_occ.copy_(a.occ, non_blocking=True)
                if a.dverts is not None:
                    a.host_dverts = torch.empty(a.dverts.shape, dtype=torch.float32, pin_memory=True)
                    a.host_dverts.copy_(a.dverts, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(stream)
        return _Batch(bid, items, stream, ev, now)

    def _retire(self, b: _Batch, now: float, results: list) -> None:
        for a in b.items:
            results.append(Result(a.req.rid, a.host_occ.numpy().copy(),
                                  a.host_dverts.numpy().copy() if a.host_dverts is not None else None,
                                  a.req.arrival, a.admitted, b.launched, now, b.bid))
            a.mesh.close()  # stream-ordered free; the batch is complete
            self.admission.release(a.nbytes)

    # -- the loop ----------------------------------------------------------------------------
    def run(self, requests, realtime: bool = True, log=None):
        """Serve ``requests`` (arrival times relative to the start). With realtime=False every
        request is available at t = 0 (capacity measurement). Returns (results, stats)."""
        torch = self.torch
        pending = collections.deque(sorted(requests, key=lambda r: (r.arrival, r.rid)))
        admitted = collections.deque()
        self._inflight = []
        self._batch_host_s = []
        results, batch_sizes = [], []
        bid = 0
        torch.cuda.synchronize(self.dev)
        t0 = time.perf_counter()
        clock = lambda: time.perf_counter() - t0  # noqa: E731
        while pending or admitted or self._inflight:
            progressed = False
            for b in [b for b in self._inflight if b.event.query()]:
                self._inflight.remove(b)
                self._retire(b, clock(), results)
                progressed = True
            now = clock()
            while (pending and (not realtime or pending[0].arrival <= now)
                   and len(admitted) < 2 * self.max_batch):
                r = pending[0]
                if not self.admission.can_admit(estimate_bytes(len(r.verts), len(r.faces), r.n, r.want_grad)):
                    break
                pending.popleft()
                admitted.append(self._materialize(r, clock()))
                progressed = True
            if admitted and len(self._inflight) < self.max_inflight:
                items = [admitted.popleft() for _ in range(min(self.max_batch, len(admitted)))]
                self._inflight.append(self._launch(items, bid, clock()))
                batch_sizes.append(len(items))
                bid += 1
                progressed = True
            if not progressed:
                if self._inflight and not (pending and realtime):
                    self._inflight[0].event.synchronize()  # nothing can arrive: wait for the oldest batch
                elif self._inflight:
                    time.sleep(2e-4)  # poll: a request may arrive or a batch may finish
                elif pending and realtime:
                    time.sleep(max(0.0, min(pending[0].arrival - clock(), 0.01)))
        makespan = clock()
        lat = np.array([r.latency for r in results]) * 1e3
        by_id = {r.rid: r for r in requests}
        pairs = sum(by_id[r.rid].pairs for r in results)
        stats = {"requests": len(results), "makespan_s": makespan, "pairs_per_s": pairs / makespan,
                 "requests_per_s": len(results) / makespan,
                 "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                 "mean_ms": float(lat.mean()), "batches": bid,
                 "mean_batch": float(np.mean(batch_sizes)) if batch_sizes else 0.0}
        hs = np.array(self._batch_host_s) * 1e3
        if len(hs):
            # host time of dv_run_batch per batch: scratch reservation, graph capture, instantiation
            # and launch (the call returns before the GPU work ends)
            stats.update(batch_host_ms_mean=float(hs.mean()), batch_host_ms_p50=float(np.percentile(hs, 50)),
                         batch_host_ms_max=float(hs.max()), batch_host_s_total=float(hs.sum() * 1e-3))
        return results, stats


def served_runs(n_requests: int = 512, rate: float = 200.0, seed: int = 5, sub_capacity: float = 0.7,
                max_batch: int = 16, max_inflight: int = 3, capacity_run: bool = True, sweep=(), device="cuda"):
    """The served mixed stream at ``rate`` (arrivals in real time), optionally the same requests
    all queued at t = 0 (capacity), and the stream again at ``sub_capacity`` x the measured
    capacity (from the queued run, else from the run at ``rate`` when that rate exceeds it).
    Returns a dict of the runs' statistics (p50/p99 latency, pairs/s, requests/s, batches)."""
    t = time.perf_counter()
    reqs = make_workload(n_requests, rate, seed)
    gen_s = time.perf_counter() - t
    srv = Server(device=device, max_batch=max_batch, max_inflight=max_inflight)
    warm = make_workload(8, 0.0, seed=seed + 100, f_hi=5000, grids=(32,))
    srv.run(warm, realtime=False)
    cap = None
    if capacity_run:
        _, cap = srv.run(reqs, realtime=False)
    _, live = srv.run(reqs, realtime=True)
    mean_pairs = float(np.mean([r.pairs for r in reqs]))
    capacity = cap["pairs_per_s"] if cap else live["pairs_per_s"]
    sub_rate = sub_capacity * capacity / mean_pairs
    _, slow = srv.run(make_workload(n_requests, sub_rate, seed), realtime=True)
    out_sweep = []
    for frac in sweep:
        r = frac * capacity / mean_pairs
        _, st = srv.run(make_workload(n_requests, r, seed), realtime=True)
        out_sweep.append(dict(st, rate=r, fraction=frac))
    out = {"workload": f"{n_requests} requests, Poisson {rate} req/s (seed {seed}), ellipsoid unions "
                       "F log-uniform [500, 1e5], grids {32..192}^3, 30% with dL/dV",
           "generation_s": gen_s, "mean_pairs_per_request": mean_pairs, "offered_pairs_per_s": rate * mean_pairs,
           "capacity_from": "all queued at t=0" if cap else f"the run at {rate} req/s (offered load above capacity)",
           "at_rate": live, "sub_capacity": dict(slow, rate=sub_rate, fraction=sub_capacity)}
    if cap:
        out["capacity"] = cap
    if out_sweep:
        out["sweep"] = out_sweep
    return out


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--requests", type=int, default=512)
    ap.add_argument("--rate", type=float, default=200.0)
    ap.add_argument("--seed", type=int, default=5)
    ap.add_argument("--max-batch", type=int, default=16)
    ap.add_argument("--max-inflight", type=int, default=3)
    ap.add_argument("--sub-capacity", type=float, default=0.7)
    ap.add_argument("--sweep", type=str, default="",
                    help="extra comma-separated fractions of the measured capacity to offer as Poisson loads")
    a = ap.parse_args(argv)
    print(json.dumps(served_runs(a.requests, a.rate, a.seed, a.sub_capacity, a.max_batch, a.max_inflight,
                                 sweep=[float(x) for x in a.sweep.split(",") if x.strip()])))


if __name__ == "__main__":
    main()
