#!/usr/bin/env python
"""Throughput of the batched charging-station step on B300.

One timed step = one full 288-step episode (24 h of 5-minute steps) of every
station of the heterogeneous batch (65536 stations, 25 % each of 8/16/32/64
chargers), random 11-level actions drawn in-kernel, run as a CUDA graph of
fused persistent-kernel launches (steps per launch and warps per block from
the library's autotuner).  The plain form (one thread per station, one launch
per step, same graph replay) is timed the same way beside it.

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle (the
plain FP64 C program the library is checked against) on a bounded sample of
the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "env-steps/s at 64K mixed-size envs vs plain form; p50/p99 serve step latency"
L2_FLUSH_BYTES = 512 << 20          # > 126 MB L2


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["b300", "reference"], default="b300")
    ap.add_argument("--n-envs", type=int, default=65536)
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-policy", action="store_true", help="skip the on-device policy rollout leg")
    ap.add_argument("--no-v2g", action="store_true", help="skip the vehicle-to-grid leg")
    ap.add_argument("--no-variants", action="store_true", help="skip the charge-sensitive and deeper-tree legs")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the uniform-station legs (16 x 16, and 4096 x 16 in two groups)")
    ap.add_argument("--policy-steps", type=int, default=128, help="rollout buffer length of the policy leg")
    ap.add_argument("--policy-only", action="store_true",
                    help="time only the policy rollout leg and print its JSON object (profiling aid)")
    ap.add_argument("--serve-envs", type=int, default=1 << 20, help="resident stations of the serving leg")
    ap.add_argument("--serve-actors", type=int, default=4096)
    ap.add_argument("--serve-think-us", type=float, default=0.0,
                    help="mean think time of a simulated actor (0: chosen for --serve-load of peak throughput)")
    ap.add_argument("--serve-load", type=float, default=0.7, help="offered load as a fraction of peak throughput")
    ap.add_argument("--serve-seconds", type=float, default=5.0)
    ap.add_argument("--shape", default="", help="K,W: fixed steps per launch and warps per block (skips the autotuner)")
    return ap.parse_args()


# ----------------------------------------------------------------------------
# helpers
# ----------------------------------------------------------------------------

class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int, period_ms: int = 20):
        self.index = index
        self.period_ms = period_ms
        self.p = None
        self.lines = []

    def _read(self):
        for line in self.p.stdout:
            self.lines.append(line)

    def __enter__(self):
        import threading
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-lms", str(self.period_ms)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                      text=True)
            self.reader = threading.Thread(target=self._read, daemon=True)
            self.reader.start()
            t0 = time.perf_counter()            # the timed region starts once the sampler runs
            while not self.lines and time.perf_counter() - t0 < 3.0 and self.p.poll() is None:
                time.sleep(0.005)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()
            self.reader.join(timeout=5)
            self.out = "".join(self.lines)

    def summary(self):
        rows = []
        for line in (self.out or "").strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                rows.append(f)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        sm = sorted(float(r[1]) for r in rows if r[1].replace(".", "").isdigit())
        mx = max(float(r[2]) for r in rows if r[2].replace(".", "").isdigit())
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx, "reasons": reasons,
                "samples": len(rows), "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit())}


def dist_init(backend: str = "nccl"):
    """Rank, world size and local rank from the torchrun environment; one
    process per GPU (nccl) or per CPU worker (gloo, used by the tests)."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws == 1:
        return 0, 1, 0
    import torch
    import torch.distributed as dist
    rank, local = int(os.environ["RANK"]), int(os.environ.get("LOCAL_RANK", "0"))
    if backend == "nccl":
        torch.cuda.set_device(local)
    if not dist.is_initialized():
        dist.init_process_group(backend)
    return rank, ws, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def _reduce(x, ws, op):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=op)
    return float(t.item())


def max_over_ranks(x, ws):
    import torch.distributed as dist
    return _reduce(x, ws, dist.ReduceOp.MAX) if ws > 1 else x


def whole_job_rate(units_local, seconds_local, ws):
    """Whole-job throughput: units summed over ranks / the slowest rank's time."""
    import torch.distributed as dist
    units = _reduce(float(units_local), ws, dist.ReduceOp.SUM) if ws > 1 else float(units_local)
    return units / max_over_ranks(seconds_local, ws)


def rank_seed(rank):
    """Philox key of a rank's batch: ranks simulate different stations."""
    return 1000 + rank


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "measured"
    except Exception:
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "sm_max_mhz": 2032.0}, "fallback"


# Algorithmic bytes per unit (the roofline of both forms): what one plain
# step must read and write per charger and per station, and the state bytes
# a fused launch loads and stores once for all its steps.
PLAIN_BYTES_PER_PORT_STEP = 34.0     # read trem,meta,soc,erem,cap,rbar (21) + write soc,erem,p,trem (13)
PLAIN_BYTES_PER_ENV_STEP = 97.0      # station fields read + written, reward + done
FUSED_STATE_BYTES_PER_PORT = 54.0    # per launch: state in (21) + out (21) + statics (12)
FUSED_STATE_BYTES_PER_ENV = 80.0
LANES_PER_SM = 128
POLICY_HIDDEN = 256


def policy_flops_per_env_step(D, N, L, H=POLICY_HIDDEN):
    """Multiply-adds x 2 of one MLP pass for one env (the algorithmic
    D -> H -> H -> N*L network; padding is not counted)."""
    return 2.0 * (D * H + H * H + H * N * L)


def policy_bytes_per_env_step(D, N):
    """HBM bytes the rollout must write per env-step: observation (FP32),
    levels (int8), reward (FP32), done (u8)."""
    return 4.0 * D + N + 4.0 + 1.0


def _record(name, sources, **want):
    """The fields of a committed ncu record (profiles/<name>: per-launch DRAM
    bytes, thread instructions, issue utilisation), if the kernel sources and
    the launch parameters are those the counters were taken on; else None."""
    import hashlib
    try:
        rec = dict(l.split() for l in open(os.path.join(ROOT, "profiles", name))
                   if l.strip() and not l.startswith("#"))
        src = b"".join(open(os.path.join(ROOT, "paper_2507_01522_b300", "csrc", f), "rb").read() for f in sources)
        if hashlib.sha256(src).hexdigest()[:16] != rec["source_sha256_16"]:
            return None
        if any(int(rec[k]) != int(v) for k, v in want.items()):
            return None
        return rec
    except Exception:
        return None


def _recorded(name, sources, **want):
    rec = _record(name, sources, **want)
    return None if rec is None else int(rec["dram_bytes_per_launch"])


FUSED_SOURCES = ("step_fused.cu", "chx_device.cuh", "chx_kernels.h")


def recorded_traffic(n_envs, K, W):
    """DRAM bytes per fused step launch (k_step_fused record)."""
    return _recorded("k_step_fused_traffic.txt", FUSED_SOURCES, n_envs=n_envs, steps_per_launch=K,
                     warps_per_block=W)


def recorded_issue(n_envs, K, W):
    """Thread instructions per launch and issue-slot utilisation of the fused
    kernel (k_step_fused record), or None."""
    rec = _record("k_step_fused_traffic.txt", FUSED_SOURCES, n_envs=n_envs, steps_per_launch=K,
                  warps_per_block=W)
    try:
        return float(rec["thread_inst_per_launch"]), float(rec["issue_active_pct"])
    except Exception:
        return None


ROLLOUT_SOURCES = ("policy.cu", "chx_tc.cuh", "chx_device.cuh", "chx_kernels.h")


def recorded_rollout_traffic(n_envs, T):
    """DRAM bytes per fused rollout launch (k_rollout record, scaled from the
    captured rollout length: every step writes the same buffers)."""
    try:
        rec = dict(l.split() for l in open(os.path.join(ROOT, "profiles", "k_rollout_traffic.txt"))
                   if l.strip() and not l.startswith("#"))
        per = _recorded("k_rollout_traffic.txt", ROLLOUT_SOURCES, n_envs=n_envs)
        if per is None:
            return None
        return int(per * T / int(rec["rollout_steps"]))
    except Exception:
        return None


def cpu_baseline(w, n_sample_envs, steps):
    """Time the CPU oracle, as it stands (single thread), on the first
    ``n_sample_envs`` stations of the workload for ``steps`` steps."""
    import numpy as np
    import oracle
    from paper_2507_01522_b300 import inputs as I
    ids = np.arange(n_sample_envs)
    sub = I.Workload(w.name, w.params, w.stations.subset(ids), w.exo, w.seed)
    o = oracle.Oracle(sub, streams=ids)
    t0 = time.perf_counter()
    for _ in range(steps):
        o.step(None)
    dt = time.perf_counter() - t0
    ports = int(sub.stations.total_ports)
    return dict(value=n_sample_envs * steps / dt, unit="env-steps/s", cores=1, kind="oracle",
                sample=f"first {n_sample_envs} of {w.stations.n_envs} stations ({ports} chargers) x {steps} steps, "
                       f"Philox actions, FP64, 1 thread", seconds=round(dt, 3),
                charger_steps_per_s=ports * steps / dt)


def _oracle_slice(job):
    """One worker of the all-cores CPU baseline: the oracle on its slice of
    the stations (their own Philox streams) for ``steps`` steps; returns the
    compute time."""
    import oracle
    sub, ids, steps = job
    o = oracle.Oracle(sub, streams=ids)
    t0 = time.perf_counter()
    for _ in range(steps):
        o.step(None)
    return time.perf_counter() - t0


def cpu_baseline_all_cores(w, n_per_core, steps):
    """The same oracle on every host core at once (processes, spawned: the
    benchmark has touched the GPU), each on its own slice of stations; the
    rate is all their env-steps over the slowest worker's compute time."""
    import multiprocessing as mp
    import numpy as np
    from paper_2507_01522_b300 import inputs as I
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    n_total = min(w.stations.n_envs, cores * n_per_core)
    bounds = [round(i * n_total / cores) for i in range(cores + 1)]
    jobs = []
    for i in range(cores):
        if bounds[i + 1] > bounds[i]:
            ids = np.arange(bounds[i], bounds[i + 1])
            jobs.append((I.Workload(w.name, w.params, w.stations.subset(ids), w.exo, w.seed), ids, steps))
    with mp.get_context("spawn").Pool(len(jobs)) as pool:
        times = pool.map(_oracle_slice, jobs)
    dt = max(times)
    return dict(value=n_total * steps / dt, unit="env-steps/s", cores=len(jobs), kind="oracle",
                sample=f"first {n_total} of {w.stations.n_envs} stations in {len(jobs)} slices x {steps} steps, "
                       f"one process per core, FP64", seconds=round(dt, 3))


def calibrate_sample(w, target_s, steps):
    import numpy as np
    import oracle
    from paper_2507_01522_b300 import inputs as I
    n = 256
    ids = np.arange(n)
    sub = I.Workload(w.name, w.params, w.stations.subset(ids), w.exo, w.seed)
    o = oracle.Oracle(sub, streams=ids)
    t0 = time.perf_counter()
    for _ in range(16):
        o.step(None)
    per_env_step = (time.perf_counter() - t0) / (n * 16)
    return int(max(64, min(w.stations.n_envs, target_s / (per_env_step * steps))))


# ----------------------------------------------------------------------------
# reference arm: the CPU oracle
# ----------------------------------------------------------------------------

def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2507_01522_b300 import inputs as I
    w = I.heterogeneous(n_envs=args.n_envs)
    T = w.params.ep_len
    n = calibrate_sample(w, 8.0, T)
    for _ in range(args.warmup):
        cpu_baseline(w, max(64, n // 8), 8)
    vals, secs = [], []
    for _ in range(args.steps):
        cb = cpu_baseline(w, n, T)
        vals.append(cb["value"])
        secs.append(cb["seconds"])
    v = sum(vals) / len(vals)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "env-steps/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(secs) / len(secs),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "n_envs": w.stations.n_envs, "horizon": T,
                       "sample_envs_per_step": n, "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": v, "unit": "env-steps/s", "cores": 1, "kind": "oracle",
                             "sample": cb["sample"]},
            "e2e": {"value": v, "unit": "env-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------
# the B300 arm
# ----------------------------------------------------------------------------

def fused_roofline(P, E, K, W, launch_ms, pk, pk_kind, dev):
    """Roofline of one fused launch (K steps of every station): the plain
    form's algorithmic bytes for the same steps over the fused launch time,
    against the measured HBM bandwidth (the fused form keeps the state on
    chip, so the fraction can exceed 1), with the SM issue utilisation and
    the lane-instruction rate from the committed ncu record beside it."""
    import torch
    hbm = pk["hbm_gbs"]
    plain_bytes = (PLAIN_BYTES_PER_PORT_STEP * P + PLAIN_BYTES_PER_ENV_STEP * E) * K
    fused_bytes = FUSED_STATE_BYTES_PER_PORT * P + FUSED_STATE_BYTES_PER_ENV * E + 5.0 * E * K
    gbs = plain_bytes / (launch_ms * 1e-3) / 1e9
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_mhz = pk.get("sm_max_mhz", 2032.0)
    lane_peak = sm_count * LANES_PER_SM * sm_mhz * 1e6
    rec = recorded_issue(E, K, W)
    alu = None
    if rec is not None:
        ti, issue = rec
        alu = {"achieved": ti / (launch_ms * 1e-3) / 1e12, "peak": lane_peak / 1e12, "unit": "T lane-instructions/s",
               "frac": ti / (launch_ms * 1e-3) / lane_peak, "thread_inst_per_launch": ti,
               "source": "smsp__thread_inst_executed.sum of the committed ncu record (profiles/k_step_fused_traffic.txt)",
               "peak_source": f"{sm_count} SMs x {LANES_PER_SM} lanes x {sm_mhz:.0f} MHz ({pk_kind} max clock)"}
    return {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
            "traffic": recorded_traffic(E, K, W), "kernel": "k_step_fused",
            "basis": "plain-form algorithmic bytes (34 B per charger-step + 97 B per station-step) of the "
                     "launch's K steps over the fused launch's CUDA-event time, of %s HBM bandwidth" % pk_kind,
            "algorithmic_bytes_per_launch": plain_bytes, "launch_ms": launch_ms, "steps_per_launch": K,
            "warps_per_block": W,
            "sm_issue_active": None if rec is None else rec[1] / 100.0,
            "fused_state_bytes_per_launch": fused_bytes,
            "fused_state_gbs": fused_bytes / (launch_ms * 1e-3) / 1e9,
            "alu": alu}


def run_b300(args):
    import numpy as np
    import torch
    from paper_2507_01522_b300 import chargax
    from paper_2507_01522_b300 import inputs as I

    rank, ws, local = dist_init()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = I.heterogeneous(n_envs=args.n_envs, seed=0)
    T = w.params.ep_len
    b = chargax.Batch(w, seed=rank_seed(rank))
    E, P = b.E, b.P
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    if args.shape:
        K, W = (int(x) for x in args.shape.split(","))
        b.set_launch(K, W)
    else:
        K, W = b.autotune(T)
    reward = torch.empty(E, T, device=dev)
    done = torch.empty(E, T, dtype=torch.uint8, device=dev)
    obs = torch.empty(b.obs_size, device=dev)
    launches_per_step = math.ceil(T / K)

    def timed(fn, n):
        times = []
        for _ in range(n):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            times.append((e0, e1))
        torch.cuda.synchronize()
        return [a.elapsed_time(c) for a, c in times]

    fused = lambda: b.rollout(T, reward=reward, done=done, obs=obs)
    for _ in range(args.warmup):
        fused()
    torch.cuda.synchronize()
    barrier(ws)
    torch.cuda.synchronize()
    with Clocks(local) as ck:
        ms = timed(fused, args.steps)
        torch.cuda.synchronize()
        barrier(ws)
    b.check()
    total_s = max_over_ranks(sum(ms) / 1e3, ws)
    ms_step = 1e3 * total_s / args.steps
    value = whole_job_rate(E * T * args.steps, sum(ms) / 1e3, ws)

    pk, pk_kind = peaks()
    roofline = fused_roofline(P, E, K, W, ms_step / launches_per_step, pk, pk_kind, dev)
    line = {"metric": METRIC, "value": value, "unit": "env-steps/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": w.name, "n_envs": E, "n_chargers": P, "horizon_steps": T,
                       "form": "fused persistent kernel, CUDA graph", "steps_per_launch": K, "warps_per_block": W,
                       "actions": "Philox uniform 11 levels in-kernel", "parallelism": f"replicas x{ws}",
                       "l2": f"flushed between timed steps ({L2_FLUSH_BYTES >> 20} MB write)"},
            "charger_steps_per_s": P * T * args.steps * ws / total_s,
            "roofline": roofline, "gpu_launches": launches_per_step * fused_kernels_per_launch(w) * args.steps}

    # plain form, same protocol: one launch per step, replayed as a graph
    if not args.no_plain:
        bp = chargax.Batch(w, seed=rank_seed(rank))
        rp = torch.empty(T, E, device=dev)
        dp = torch.empty(T, E, dtype=torch.uint8, device=dev)
        bp.step(reward=rp[0], done=dp[0])
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            for k in range(T):
                bp.step(reward=rp[k], done=dp[k])
        for _ in range(args.warmup):
            g.replay()
        torch.cuda.synchronize()
        barrier(ws)
        pms = timed(g.replay, args.steps)
        bp.check()
        ptotal = max_over_ranks(sum(pms) / 1e3, ws)
        pms_step = 1e3 * ptotal / args.steps
        plain_bytes = PLAIN_BYTES_PER_PORT_STEP * P + PLAIN_BYTES_PER_ENV_STEP * E
        gbs = plain_bytes / (pms_step * 1e-3 / T) / 1e9
        line["plain"] = {"value": E * T * args.steps * ws / ptotal, "unit": "env-steps/s", "ms_per_step": pms_step,
                         "launches_per_step": T,
                         "roofline": {"bound": "hbm", "achieved": gbs, "peak": pk["hbm_gbs"], "unit": "GB/s",
                                      "frac": gbs / pk["hbm_gbs"], "traffic": None, "kernel": "k_step_plain",
                                      "note": "one thread per station: memory-latency bound (state read and written every step)"}}
        line["fused_over_plain"] = line["value"] / line["plain"]["value"]
        line["gpu_launches"] += T * args.steps
        del bp

    # end to end through the C interface with host buffers: every step's
    # levels in (host actions, step-major), rewards, done flags and the final
    # observation out, copies inside the timed region
    if not args.no_e2e:
        n_act = b.P
        ha = torch.empty(T * n_act, dtype=torch.int8, pin_memory=True).numpy()
        ha[:] = I.random_actions(np.random.default_rng(rank), n_act, n_levels=w.params.n_levels,
                                 steps=T).T.reshape(-1)
        hr = torch.empty(E * T, dtype=torch.float32, pin_memory=True).numpy()
        hd = torch.empty(E * T, dtype=torch.uint8, pin_memory=True).numpy()
        ho = torch.empty(b.obs_size, dtype=torch.float32, pin_memory=True).numpy()

        def e2e_time(fn):
            fn()
            torch.cuda.synchronize()
            barrier(ws)
            et = []
            for _ in range(args.steps):
                flush.zero_()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                fn()
                et.append(time.perf_counter() - t0)
            return max_over_ranks(sum(et), ws)

        # the same levels packed two per byte (11 levels fit a nibble): the
        # copy in is what bounds this call, so it is the headline end-to-end form
        from paper_2507_01522_b300.chargax import pack_levels4
        h4 = torch.empty(T * ((n_act + 1) // 2), dtype=torch.uint8, pin_memory=True).numpy()
        h4[:] = pack_levels4(ha.reshape(T, n_act)).reshape(-1)
        etot = e2e_time(lambda: b.rollout_host_levels4(T, h4, hr, hd, ho))
        line["e2e"] = {"value": E * T * args.steps * ws / etot, "unit": "env-steps/s",
                       "h2d_bytes_per_step": int(h4.nbytes),
                       "d2h_bytes_per_step": int(hr.nbytes + hd.nbytes + ho.nbytes),
                       "ms_per_step": 1e3 * etot / args.steps,
                       "api": "chx_rollout_host_levels4 (pinned host levels in, step-major [T][chargers / 2], two "
                              "4-bit levels per byte; rewards, done flags step-major and the final observation "
                              "out; 12 launches, each one's levels copied in while the previous computes and its "
                              "outputs copied out while the next computes)"}
        line["gpu_launches"] += min(12, T) * args.steps
        itot = e2e_time(lambda: b.rollout_host_actions(T, ha, hr, hd, ho))
        line["e2e_int8_actions"] = {
            "value": E * T * args.steps * ws / itot, "unit": "env-steps/s", "h2d_bytes_per_step": int(ha.nbytes),
            "d2h_bytes_per_step": int(hr.nbytes + hd.nbytes + ho.nbytes), "ms_per_step": 1e3 * itot / args.steps,
            "api": "chx_rollout_host_actions (the same levels as one int8 per charger; 12 launches, each 0.85 "
                   "of the size of the one before; otherwise as e2e)"}
        line["gpu_launches"] += min(12, T) * args.steps
        ptot = e2e_time(lambda: b.rollout_host(T, hr, hd, ho))
        line["e2e_philox_actions"] = {
            "value": E * T * args.steps * ws / ptot, "unit": "env-steps/s", "h2d_bytes_per_step": 0,
            "d2h_bytes_per_step": int(hr.nbytes + hd.nbytes + ho.nbytes), "ms_per_step": 1e3 * ptot / args.steps,
            "api": "chx_rollout_host (levels drawn in the kernel; outputs as above; 4 launches of 5:4:2:1 "
                   "shares, each one's outputs copied while the next computes)"}
        line["gpu_launches"] += min(4, T) * args.steps
        del ha, h4, hr, hd, ho

    line["clocks"] = ck.summary()
    if not args.no_v2g:
        line["v2g"] = run_variant(args, rank, ws, timed, I.v2g_variant(w), line["value"], dev)
        line["gpu_launches"] += line["v2g"]["gpu_launches"]
    if not args.no_variants:
        wc = I.Workload(w.name + "-cs128", I.EnvParams(**{**w.params.__dict__, "cs_share_256": 128,
                                                          "soc_target": 0.8}), w.stations, w.exo, w.seed)
        line["charge_sensitive"] = run_variant(args, rank, ws, timed, wc, line["value"], dev)
        line["tree"] = run_variant(args, rank, ws, timed, I.tree_workload(args.n_envs, seed=0), line["value"], dev)
        line["gpu_launches"] += line["charge_sensitive"]["gpu_launches"] + line["tree"]["gpu_launches"]
    if not args.no_policy:
        del reward, done, obs
        pol = run_policy_rollout(args, rank, ws, dev, timed, pk)
        line["policy_rollout"] = pol
        line["gpu_launches"] += pol["gpu_launches"]
    if not args.no_configs:
        line["configs"] = {}
        for wc in (I.small_uniform(seed=0), I.fixed_station(seed=0)):
            leg = run_config_leg(args, rank, ws, timed, wc, pk, dev)
            line["configs"][wc.name] = leg
            line["gpu_launches"] += leg["gpu_launches"]
    if not args.no_serve:
        del b
        torch.cuda.empty_cache()
        # one server on rank 0 (its host threads would contend with other
        # ranks' servers on the shared host cores); the other ranks wait
        if rank == 0:
            line["serving"] = run_serving(args, rank)
            if ws > 1:
                line["serving"]["ranks"] = "rank 0 only (one GPU's server; the other ranks wait)"
        barrier(ws)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        n = calibrate_sample(w, 12.0, T)
        line["cpu_baseline"] = cpu_baseline(w, n, T)
        line["cpu_baseline"]["all_cores"] = cpu_baseline_all_cores(w, max(16, n // 2), T)
    if rank == 0:
        print(json.dumps(line), flush=True)
    barrier(ws)


def run_config_leg(args, rank, ws, timed, wc, pk, dev):
    """A uniform-station configuration (16 x 16 chargers, or 4096 x 16 in two
    groups of 8 at 80 kW), one 288-step episode per timed step with in-kernel
    random levels, plain form (one launch per step, graph replay) against the
    fused form (CUDA graph of fused launches, autotuned shape); both against
    the plain form's algorithmic HBM bytes."""
    import torch
    from paper_2507_01522_b300 import chargax
    T = wc.params.ep_len
    hbm = pk["hbm_gbs"]
    bf = chargax.Batch(wc, seed=rank_seed(rank))
    E, P = bf.E, bf.P
    plain_bytes_step = PLAIN_BYTES_PER_PORT_STEP * P + PLAIN_BYTES_PER_ENV_STEP * E
    if args.shape:
        K, W = (int(x) for x in args.shape.split(","))
        bf.set_launch(K, W)
    else:
        K, W = bf.autotune(T)
    reward = torch.empty(E, T, device=dev)
    done = torch.empty(E, T, dtype=torch.uint8, device=dev)
    fn = lambda: bf.rollout(T, reward=reward, done=done)
    for _ in range(args.warmup):
        fn()
    torch.cuda.synchronize()
    barrier(ws)
    ms = timed(fn, args.steps)
    bf.check()
    ftot = max_over_ranks(sum(ms) / 1e3, ws)
    fms = 1e3 * ftot / args.steps
    n_launch = math.ceil(T / K)
    fgbs = plain_bytes_step * T / (fms * 1e-3) / 1e9
    out = {"n_envs": E, "n_chargers": P, "horizon_steps": T, "actions": "Philox uniform 11 levels in-kernel",
           "fused": {"value": E * T * args.steps * ws / ftot, "unit": "env-steps/s", "ms_per_step": fms,
                     "steps_per_launch": K, "warps_per_block": W, "launches_per_step": n_launch,
                     "charger_steps_per_s": P * T * args.steps * ws / ftot,
                     "roofline": {"bound": "hbm", "achieved": fgbs, "peak": hbm, "unit": "GB/s", "frac": fgbs / hbm,
                                  "kernel": "k_step_fused", "traffic": None,
                                  "basis": "plain-form algorithmic bytes over the fused time"}}}
    del bf
    bp = chargax.Batch(wc, seed=rank_seed(rank))
    rp = torch.empty(T, E, device=dev)
    dp = torch.empty(T, E, dtype=torch.uint8, device=dev)
    bp.step(reward=rp[0], done=dp[0])
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        for k in range(T):
            bp.step(reward=rp[k], done=dp[k])
    for _ in range(args.warmup):
        g.replay()
    torch.cuda.synchronize()
    barrier(ws)
    pms = timed(g.replay, args.steps)
    bp.check()
    ptot = max_over_ranks(sum(pms) / 1e3, ws)
    pms_step = 1e3 * ptot / args.steps
    pgbs = plain_bytes_step * T / (pms_step * 1e-3) / 1e9
    out["plain"] = {"value": E * T * args.steps * ws / ptot, "unit": "env-steps/s", "ms_per_step": pms_step,
                    "launches_per_step": T, "charger_steps_per_s": P * T * args.steps * ws / ptot,
                    "roofline": {"bound": "hbm", "achieved": pgbs, "peak": hbm, "unit": "GB/s", "frac": pgbs / hbm,
                                 "kernel": "k_step_plain", "traffic": None,
                                 "basis": "34 B per charger-step + 97 B per station-step"}}
    out["fused_over_plain"] = out["fused"]["value"] / out["plain"]["value"]
    out["gpu_launches"] = (n_launch + T) * args.steps
    del bp, g
    return out


def fused_kernels_per_launch(w):
    """Kernels one fused launch of workload w runs: one per class range that
    holds stations.  The 128-charger class has an instance of its own, and so
    has the 64-charger class in the V2G and extended forms without upper
    tree levels; the other classes share one."""
    import numpy as np
    st = w.stations
    cls = set(int(c) for c in np.unique(np.searchsorted([8, 16, 32, 64, 128], np.asarray(st.n_ports))))
    n_upper = getattr(st, "n_upper", None)
    tree = n_upper is not None and int(np.sum(n_upper)) > 0
    p = w.params
    split = bool(p.v2g or p.action_delta or p.cs_share_256 > 0) and not tree
    ranges = ([(0, 2), (3, 3)] if split else [(0, 3)]) + [(4, 4)]
    return sum(any(lo <= c <= hi for c in cls) for lo, hi in ranges)


def run_variant(args, rank, ws, timed, wv, charge_only_value, dev):
    """A variant of the method on the same scale, fused form, the headline
    leg's timing protocol: vehicle-to-grid mode (signed levels, discharge
    taper, station battery, feed-in price, degradation), charge-sensitive
    users, or the deeper trees of Fig. charge-tree c."""
    import torch
    from paper_2507_01522_b300 import chargax

    T = wv.params.ep_len
    b = chargax.Batch(wv, seed=rank_seed(rank))
    if args.shape:
        K, W = (int(x) for x in args.shape.split(","))
        b.set_launch(K, W)
    else:
        K, W = b.autotune(T)
    reward = torch.empty(b.E, T, device=dev)
    done = torch.empty(b.E, T, dtype=torch.uint8, device=dev)
    obs = torch.empty(b.obs_size, device=dev)
    fn = lambda: b.rollout(T, reward=reward, done=done, obs=obs)
    for _ in range(args.warmup):
        fn()
    torch.cuda.synchronize()
    barrier(ws)
    ms = timed(fn, args.steps)
    b.check()
    total = max_over_ranks(sum(ms) / 1e3, ws)
    value = b.E * T * args.steps * ws / total
    out = {"value": value, "unit": "env-steps/s", "ms_per_step": 1e3 * total / args.steps, "workload": wv.name,
           "n_envs": b.E, "n_chargers": b.P, "n_levels": wv.params.n_levels, "steps_per_launch": K,
           "warps_per_block": W,
           "actions": f"Philox uniform {wv.params.n_levels} levels per charger" + (" and battery" if wv.params.v2g else "")
                      + ", in-kernel",
           "over_charge_only": value / charge_only_value,
           "gpu_launches": math.ceil(T / K) * fused_kernels_per_launch(wv) * args.steps}
    del b
    return out


def run_policy_rollout(args, rank, ws, dev, timed, pk):
    """On-device policy rollout: 16384 stations x 32 chargers, a buffer of
    args.policy_steps steps (observation FP32, levels int8, reward FP32,
    done), actions sampled from a randomly initialised BF16 MLP
    200 -> 256 -> 256 -> 32 x 11 on the tensor cores.  Both forms: fused
    (one kernel per rollout) and split (policy and step launches per step)."""
    import torch
    from paper_2507_01522_b300 import chargax
    from paper_2507_01522_b300 import inputs as I
    w = I.rollout_stations(seed=0)
    T = args.policy_steps
    b = chargax.Batch(w, seed=rank_seed(rank))
    E = b.E
    N = int(w.stations.n_ports[0])
    L = w.params.n_levels
    D = 8 + 6 * N
    pw = I.policy_weights(D, N, n_levels=L, seed=rank)
    b.policy_load(pw.w1, pw.b1, pw.w2, pw.b2, pw.w3, pw.b3)
    obs = torch.empty(T, E, D, device=dev)
    acts = torch.empty(T, E, N, dtype=torch.int8, device=dev)
    rew = torch.empty(T, E, device=dev)
    done = torch.empty(T, E, dtype=torch.uint8, device=dev)
    out = {"workload": w.name, "n_envs": E, "chargers_per_station": N, "rollout_steps": T,
           "policy": f"BF16 MLP {D}-{POLICY_HIDDEN}-{POLICY_HIDDEN}-{N}x{L}, FP32 accumulation, PPO initialisation",
           "unit": "env-steps/s", "buffers": "obs f32 [T][E][D], levels int8 [T][E][N], reward f32, done u8"}
    launches = 0
    for form, name in ((chargax.CHX_ROLLOUT_FUSED, "fused"), (chargax.CHX_ROLLOUT_SPLIT, "split")):
        fn = lambda: b.policy_rollout(T, obs, acts, rew, done, form=form)
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        barrier(ws)
        ms = timed(fn, args.steps)
        b.check()
        tot = max_over_ranks(sum(ms) / 1e3, ws)
        ms_roll = 1e3 * tot / args.steps
        flops = policy_flops_per_env_step(D, N, L) * E * T
        tf = flops / (ms_roll * 1e-3) / 1e12
        by = policy_bytes_per_env_step(D, N) * E * T
        gbs = by / (ms_roll * 1e-3) / 1e9
        n_launch = 1 if name == "fused" else 2 * T + 1
        launches += n_launch * args.steps
        out[name] = {"value": E * T * args.steps * ws / tot, "ms_per_rollout": ms_roll, "launches_per_rollout": n_launch,
                     "roofline": {"bound": "tensor", "achieved": tf, "peak": pk["bf16_tflops"], "unit": "TFLOP/s",
                                  "frac": tf / pk["bf16_tflops"],
                                  "traffic": recorded_rollout_traffic(E, T) if name == "fused" else None,
                                  "kernel": "k_rollout" if name == "fused" else "k_policy + k_step_fused",
                                  "flops_per_rollout": flops,
                                  "hbm_output_gbs": gbs, "hbm_output_frac": gbs / pk["hbm_gbs"]}}
    out["value"] = out["fused"]["value"]
    out["fused_over_split"] = out["fused"]["value"] / out["split"]["value"]
    out["gpu_launches"] = launches
    del b
    torch.cuda.empty_cache()
    return out


def run_serving(args, rank):
    """Serving leg: a pool of resident stations (8-128 chargers, log-uniform),
    closed-loop simulated actors each stepping its own stations, Philox
    actions; latency from submission to completion."""
    import numpy as np
    from paper_2507_01522_b300 import chargax
    from paper_2507_01522_b300 import inputs as I
    w = I.serving_pool(args.serve_envs, seed=rank)
    n = w.stations.n_ports
    cap = [int(np.sum(n <= 8))] + [int(np.sum((n > (4 << c)) & (n <= (8 << c)))) for c in range(1, 5)]
    t0 = time.perf_counter()
    srv = chargax.Server(w.params, w.exo, cap, hbm_budget_bytes=150e9, max_tick_envs=65536, n_streams=2)
    ids = srv.admit(w.stations, seed=2000 + rank)
    t_admit = time.perf_counter() - t0
    per = args.serve_envs // args.serve_actors
    # simulated actors' host threads: every host core but those of the
    # server's scheduler thread and this process
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 8)
    threads = max(2, min(16, cores - 4))
    # peak: every actor resubmits at once (no think time)
    peak = srv.simulate(ids, n_actors=args.serve_actors, envs_per_actor=per, mean_think_us=0.0,
                        duration_s=2.0, warmup_s=0.5, n_threads=threads, seed=rank)
    x_peak = peak["n_requests"] / peak["seconds"]
    # latency at a stated load: closed loop, think time Z with N / (Z + R) = load * peak
    think = args.serve_think_us or args.serve_actors / (args.serve_load * x_peak) * 1e6
    res = srv.simulate(ids, n_actors=args.serve_actors, envs_per_actor=per, mean_think_us=think,
                       duration_s=args.serve_seconds, warmup_s=1.0, n_threads=threads, seed=rank + 1)
    st = srv.stats()
    srv.stop()
    return {"workload": w.name, "resident_stations": int(st["resident"]), "chargers": int(w.stations.total_ports),
            "pool_bytes_admitted": st["used_bytes"], "hbm_budget_bytes": st["budget_bytes"],
            "actors": args.serve_actors, "envs_per_request": per, "mean_think_us": round(think, 1),
            "offered_load": "think time for %.0f %% of peak request rate" % (100 * args.serve_load)
            if not args.serve_think_us else "fixed think time",
            "peak": {"env_steps_per_s": peak["env_steps_per_s"], "requests_per_s": x_peak,
                     "p50_us": peak["p50_us"], "p99_us": peak["p99_us"],
                     "device_busy_frac": peak["device_busy_frac"]},
            "host_threads": threads, "admit_s": round(t_admit, 3),
            "p50_us": res["p50_us"], "p90_us": res["p90_us"], "p99_us": res["p99_us"], "max_us": res["max_us"],
            "env_steps_per_s": res["env_steps_per_s"], "requests": res["n_requests"],
            "mean_tick_envs": res["mean_tick_envs"], "device_busy_frac": res["device_busy_frac"],
            "seconds": res["seconds"],
            "host_ms": {k: round(st[k], 1) for k in ("host_submit_ms", "host_scan_ms", "host_pack_ms", "host_launch_ms",
                                                      "host_complete_ms", "elapsed_ms", "device_busy_ms")},
            "ticks": st["n_ticks"], "scans": st["n_scans"]}


def run_policy_only(args):
    import torch
    rank, ws, local = dist_init()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def timed(fn, n):
        times = []
        for _ in range(n):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            times.append((e0, e1))
        torch.cuda.synchronize()
        return [a.elapsed_time(c) for a, c in times]

    pk, _ = peaks()
    out = run_policy_rollout(args, rank, ws, dev, timed, pk)
    if rank == 0:
        print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.policy_only:
        run_policy_only(args)
    else:
        run_b300(args)


if __name__ == "__main__":
    main()
