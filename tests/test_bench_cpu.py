"""bench.py's reference arm runs on the host (the oracle on this machine's cores) and prints one
JSON line with the contract's keys; the native arm needs a GPU and says so."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "icosphere_32", "--steps", "1",
                        "--warmup", "3"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["warmup"] >= 3
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]


def test_gpus_must_match_the_launched_ranks():
    # --gpus N without N ranks (no torchrun) is refused with an error naming the mismatch, for
    # both arms, before any work
    env = {k: v for k, v in os.environ.items() if k not in ("WORLD_SIZE", "RANK", "LOCAL_RANK")}
    for impl in ("native", "reference"):
        r = subprocess.run([sys.executable, "bench.py", "--impl", impl, "--gpus", "2", "--workload", "icosphere_32",
                            "--steps", "1"], cwd=ROOT, capture_output=True, text=True, timeout=300, env=env)
        assert r.returncode == 2, (impl, r.returncode, r.stderr[-500:])
        assert "--gpus 2" in r.stderr and "WORLD_SIZE=1" in r.stderr
        assert not [ln for ln in r.stdout.splitlines() if ln.startswith("{")]


def test_oracle_leg_runs_in_a_spawned_process():
    # the bench's oracle process (CPU baseline, then the accuracy sample's reference values) on a
    # tiny workload, without any GPU
    sys.path.insert(0, ROOT)
    import bench

    leg = bench.OracleLeg("icosphere_32", acc_queries=64, budget_s=0.5)
    try:
        cpu = leg.baseline()
        assert cpu["kind"] == "oracle" and cpu["value"] > 0 and cpu["cores"] >= 1
        ref = leg.accuracy(timeout_s=300)
        assert ref is not None and len(ref["idx"]) == 64 and len(ref["w64"]) == 64 and len(ref["d"]) == 64
        import numpy as np

        import oracle
        from paper_2407_11272_b300 import meshgen

        V, F = meshgen.icosphere(3, 0.8)
        Q = oracle.grid_points([-1.0] * 3, [1.0] * 3, [32] * 3, ref["idx"])
        assert np.array_equal(ref["w64"], oracle.winding(V, F, Q))
        wg = ref["whole_grid"]  # the icosphere is closed: the whole grid by ray crossings
        occ = np.unpackbits(wg["occ_bits"])[:ref["cells"]].astype(bool)
        assert ref["cells"] == 32 ** 3 and wg["values"] == [0, 1]
        w_all = oracle.winding(V, F, oracle.grid_queries([-1.0] * 3, [1.0] * 3, [32] * 3))
        und = np.unpackbits(wg["undecided_bits"])[:ref["cells"]].astype(bool)
        assert np.array_equal(occ[~und], (w_all > 0.5)[~und])
    finally:
        leg.close()
