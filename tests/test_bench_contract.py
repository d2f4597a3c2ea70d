"""The benchmark script's output: the reference arm (CPU) prints one JSON line
with the keys and kinds of values the benchmark contract names, the
all-cores oracle baseline splits the stations over worker processes, and a
short GPU-arm run carries the roofline, end-to-end, clock and launch keys."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for key in ("metric", "unit", "dtype", "data", "scaling"):
        assert isinstance(d[key], str) and d[key]
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["n_gpus"] == 1 and d["steps"] == 1 and d["warmup"] == 0
    assert d["higher_is_better"] is True and d["vs_baseline"] is None
    assert d["config"]["workload"] == "hetero-65536-8/16/32/64"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_all_cores_baseline_splits_the_stations():
    sys.path.insert(0, ROOT)
    import bench
    from paper_2507_01522_b300 import inputs as I
    w = I.heterogeneous(n_envs=96)
    res = bench.cpu_baseline_all_cores(w, 12, 3)
    assert res["kind"] == "oracle" and res["unit"] == "env-steps/s"
    assert 1 <= res["cores"] <= 96 and res["value"] > 0 and res["seconds"] >= 0
    assert "slices x 3 steps" in res["sample"]


@pytest.mark.gpu
def test_gpu_arm_json_line():
    """A short run of the GPU arm (4096 stations, one timed episode): the
    line carries the roofline, end-to-end, clock and launch-count keys."""
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--steps", "1", "--warmup", "1",
                          "--n-envs", "4096", "--no-serve", "--no-policy", "--no-variants", "--no-v2g",
                          "--no-cpu-baseline", "--no-configs"], cwd=ROOT, capture_output=True, text=True,
                         timeout=900)
    assert out.returncode == 0, out.stderr[-2000:]
    d = json.loads([l for l in out.stdout.splitlines() if l.startswith("{")][-1])
    assert d["value"] > 0 and d["n_gpus"] == 1 and d["higher_is_better"] is True
    rf = d["roofline"]
    assert rf["bound"] == "hbm" and rf["unit"] == "GB/s" and rf["achieved"] > 0 and rf["peak"] > 0
    assert abs(rf["frac"] - rf["achieved"] / rf["peak"]) < 1e-9
    # achieved = the plain form's algorithmic bytes of the launch's steps over the launch time
    assert abs(rf["achieved"] - rf["algorithmic_bytes_per_launch"] / (rf["launch_ms"] * 1e-3) / 1e9) < 1e-6 * rf["achieved"]
    e2e = d["e2e"]
    assert e2e["value"] > 0 and e2e["d2h_bytes_per_step"] > 0
    # levels in, two per byte, then the same levels as int8
    P, T = d["config"]["n_chargers"], d["config"]["horizon_steps"]
    assert e2e["h2d_bytes_per_step"] == (P + 1) // 2 * T
    assert d["e2e_int8_actions"]["h2d_bytes_per_step"] == P * T
    assert d["e2e_philox_actions"]["h2d_bytes_per_step"] == 0
    assert d["gpu_launches"] > 0 and d["plain"]["value"] > 0
    assert {"sm_mhz", "sm_max_mhz", "reasons"} <= set(d["clocks"])


def test_kernels_per_fused_launch():
    """The launch count the benchmark claims: one kernel per class range that
    holds stations (the 128-charger class alone; the 64-charger class alone
    in the V2G and extended forms without upper tree levels)."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_2507_01522_b300 import inputs as I
    w = I.heterogeneous(n_envs=256)
    assert bench.fused_kernels_per_launch(w) == 1
    assert bench.fused_kernels_per_launch(I.v2g_variant(w)) == 2
    cs = I.Workload(w.name, I.EnvParams(**{**w.params.__dict__, "cs_share_256": 128}), w.stations, w.exo, w.seed)
    assert bench.fused_kernels_per_launch(cs) == 2
    small = I.Workload(w.name, I.v2g_variant(w).params, w.stations.subset(
        [e for e in range(w.stations.n_envs) if w.stations.n_ports[e] <= 32]), w.exo, w.seed)
    assert bench.fused_kernels_per_launch(small) == 1
