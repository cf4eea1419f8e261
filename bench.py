#!/usr/bin/env python
"""Rendered env-steps/s of the simulate-then-render loop on one B300:
co-scheduled (sim of step t+1 on one SM partition while step t renders on
the other) versus serialized (sim then render on one stream, full GPU).

Workload: 1024 environments x 32 bodies (half spheres, half boxes), 8
substeps of dt = 1/240 s, one 128 x 128 RGB-D camera each (seeded synthetic
scene; the paper's ManiSkill scenes are not available), timed after 120
settling steps, every timed run of every mode from that same state.
Prints one JSON line (rank 0).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl vuda|reference]

Under torchrun each rank steps its own 1024 environments on its own GPU
(weak scaling, no data-path collective); throughput is summed over ranks
and the time is the maximum over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "rendered env-steps/s, co-scheduled vs serialized (1 B300); p50/p99 step latency"
WORKLOAD = "1024 envs x 32 bodies (sphere/box), 8 substeps, 128x128 RGB-D camera per env"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="vuda", choices=["vuda", "reference"])
    ap.add_argument("--envs", type=int, default=1024)
    ap.add_argument("--sim-sms", type=int, default=0, help="SMs of the sim partition (0: half)")
    ap.add_argument("--settle", type=int, default=120, help="untimed steps before measuring (bodies land)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serial-only", action="store_true", help="only the serialized loop (for profiling)")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving measurement")
    ap.add_argument("--serve-jobs", default="8,16,32,64", help="job counts of the serving grid")
    ap.add_argument("--serve-requests", type=int, default=10000)
    ap.add_argument("--configs", default="1,3,4", help="other workloads measured beside the headline one")
    ap.add_argument("--no-rollout", action="store_true", help="skip the RL-rollout measurement")
    return ap.parse_args()


class Clocks:
    """nvidia-smi sampling during the timed regions."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.on = False
        self._proc = None
        self._t = None

    def _run(self):
        # one nvidia-smi sampling every 100 ms; rows are kept while a timed region runs
        try:
            self._proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                           "--format=csv,noheader,nounits", "-lms", "100"],
                                          stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            for line in self._proc.stdout:
                if self.on and line.strip():
                    self.rows.append([x.strip() for x in line.split(",")])
        except Exception:
            pass

    def start(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()

    def stop(self):
        if self._proc is not None:
            self._proc.terminate()
            try:
                self._proc.wait(timeout=10)
            except Exception:
                pass
        if self._t:
            self._t.join(timeout=10)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4) if len(r) > 5 + k and r[5 + k] == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def dist_setup():
    """Rank, world size and local rank from the launcher's environment; for
    more than one rank a process group (NCCL with a GPU per rank, else gloo)."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch
        import torch.distributed as dist
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
            dist.init_process_group("nccl")
        else:
            dist.init_process_group("gloo")
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def allreduce_max(ws, x: float) -> float:
    """Maximum of x over the ranks (the job's time is its slowest rank's)."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def rank_scene(S, rank: int, envs: int):
    """The environments of one rank: environments [rank envs, (rank + 1) envs)
    of the benchmark scene (each environment's content depends only on its
    index, so N ranks together step the first N envs environments)."""
    return S.cfg2(envs, env_base=rank * envs)


def job_throughput(ws: int, envs: int, steps: int, seconds: float) -> float:
    """Whole-job env-steps/s: every rank's environments over the slowest
    rank's time."""
    return ws * envs * steps / seconds


def cpu_baseline(envs: int = 8, secs: float = 1.5):
    """The oracle as it stands, single-threaded, on a bounded sample of the
    workload: `envs` environments of the benchmark scene stepped and
    rendered for at least `secs` after the same settling."""
    import oracle
    from paper_2605_01352_b300 import scene as S
    sc = S.cfg2(envs)
    st, _, _ = oracle.sim_step(sc, 60)
    t = time.perf_counter()
    n = 0
    while n < 2 or time.perf_counter() - t < secs:
        st, _, _ = oracle.sim_step(sc, 1, state=st)
        oracle.render(sc, st["pos"], st["quat"], triid=False)
        n += 1
    dt = time.perf_counter() - t
    return {"value": envs * n / dt, "unit": "env-steps/s", "cores": 1, "kind": "oracle",
            "sample": "%d envs x %d steps of the benchmark scene (after 60 settling steps), sim + render, "
                      "single-threaded C oracle" % (envs, n)}


_BARRIER = None


def _oracle_init(barrier):
    global _BARRIER
    _BARRIER = barrier


def _oracle_worker(job):
    """One host core's share of the parallel oracle baseline: its own
    environments of the benchmark scene, settled, then stepped and rendered
    from a common start (a barrier across the workers) for at least `secs`."""
    envs, secs, base = job
    import oracle
    from paper_2605_01352_b300 import scene as S
    sc = S.cfg2(envs, env_base=base)
    st, _, _ = oracle.sim_step(sc, 60)
    if _BARRIER is not None:
        _BARRIER.wait()
    t0 = time.perf_counter()
    n = 0
    while n < 2 or time.perf_counter() - t0 < secs:
        st, _, _ = oracle.sim_step(sc, 1, state=st)
        oracle.render(sc, st["pos"], st["quat"], triid=False)
        n += 1
    return envs * n, time.perf_counter() - t0


def cpu_baseline_all_cores(envs: int = 2, secs: float = 1.5):
    """The oracle as it stands on every host core: one spawned process per
    core, each stepping and rendering its own environments; throughput = all
    env-steps / the longest worker's time (the workers start together)."""
    import multiprocessing as mp
    import oracle
    oracle.build()
    n = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    barrier = ctx.Barrier(n)
    with ctx.Pool(n, initializer=_oracle_init, initargs=(barrier,)) as pool:
        out = pool.map(_oracle_worker, [(envs, secs, k * envs) for k in range(n)], chunksize=1)
    work = sum(o[0] for o in out)
    span = max(o[1] for o in out)
    return {"value": work / span, "unit": "env-steps/s", "cores": n, "kind": "oracle",
            "sample": "%d processes x %d envs of the benchmark scene (after 60 settling steps), sim + render, "
                      "C oracle, %d env-steps in %.2f s" % (n, envs, work, span)}


def run_reference(args):
    """The oracle arm: the CPU oracle on the machine's host cores, timed over
    --steps steps (after --warmup), each a bounded sample of the workload."""
    ws, rank, _ = int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")), 0
    if rank != 0:
        return
    import oracle
    from paper_2605_01352_b300 import scene as S
    oracle.build()
    sample = 4
    sc = S.cfg2(sample)
    st, _, _ = oracle.sim_step(sc, 60)
    for _ in range(args.warmup):
        st, _, _ = oracle.sim_step(sc, 1, state=st)
        oracle.render(sc, st["pos"], st["quat"], triid=False)
    t = time.perf_counter()
    for _ in range(args.steps):
        st, _, _ = oracle.sim_step(sc, 1, state=st)
        oracle.render(sc, st["pos"], st["quat"], triid=False)
    dt = time.perf_counter() - t
    v = sample * args.steps / dt
    desc = "%d envs of the benchmark scene per step, sim + render, single-threaded C oracle" % sample
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "env-steps/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample_envs_per_step": sample},
        "cpu_baseline": {"value": v, "unit": "env-steps/s", "cores": 1, "kind": "oracle", "sample": desc},
        "e2e": {"value": v, "unit": "env-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def serving_bench(V, S, njobs: int, nreq: int, load: float = 0.8, burst: int = 16, nsat: int = 2000):
    """Serving workload (jobs of 16-1024 envs with 4-256 bodies and 64-256 px
    cameras), for continuous batching and for a serialized FIFO (one request
    at a time).  Capacity: the rate served under Poisson arrivals at twice the
    rate a burst of `burst` requests per job is served at (`nsat` requests; the
    queue grows and the server never idles).  Then `nreq` Poisson arrivals at
    `load` times the continuous-batching capacity, for both."""
    import torch
    jobs = S.cfg5_jobs(njobs)
    free, _ = torch.cuda.mem_get_info()
    budget = int(0.6 * free)

    def run(serialized: bool, rate_hz: float, nreq: int = nreq):
        srv = V.Server(hbm_budget_bytes=budget, max_inflight=1 if serialized else 2,
                       max_batch_jobs=1 if serialized else 0, serialized=serialized)
        ids = [srv.add_job(j) for j in jobs]
        envs = {i: j.num_envs for i, j in zip(ids, jobs)}
        for i in ids:                       # admit and warm up
            srv.submit(i)
        srv.wait_all(len(ids), timeout_s=600)
        if rate_hz <= 0:                    # capacity: a burst of requests from every job
            t = time.perf_counter()
            for _ in range(burst):
                for i in ids:
                    srv.submit(i)
            res = srv.wait_all(burst * len(ids), timeout_s=600)
            dt = time.perf_counter() - t
            srv.close()
            return len(res) / dt
        rng = np.random.default_rng(55)
        arrivals = np.cumsum(rng.exponential(1.0 / rate_hz, nreq))
        pick = rng.integers(0, len(ids), nreq)
        done = []
        t0 = time.perf_counter()
        k = 0
        while k < nreq:
            now = time.perf_counter() - t0
            while k < nreq and arrivals[k] <= now:
                srv.submit(ids[pick[k]])
                k += 1
            done += srv.poll()
            if k < nreq:
                time.sleep(max(0.0, min(arrivals[k] - (time.perf_counter() - t0), 0.001)))
        done += srv.wait_all(nreq - len(done), timeout_s=600)
        wall = time.perf_counter() - t0
        st = srv.stats()
        srv.close()
        lat = np.array([r["t_done_ms"] - r["t_submit_ms"] for r in done])
        es = sum(envs[r["job"]] for r in done)
        return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "requests_per_s": nreq / wall, "env_steps_per_s": es / wall, "mean_batch_jobs": st["mean_batch"],
                "peak_resident_bytes": st["peak_bytes"]}

    burst_cap = run(False, 0.0)
    burst_fifo = run(True, 0.0)
    cap = run(False, 2.0 * burst_cap, nsat)["requests_per_s"]
    cap_fifo = run(True, 2.0 * burst_fifo, nsat)["requests_per_s"]
    rate = load * cap
    cb = run(False, rate)
    fifo = run(True, rate)
    fifo_own = run(True, load * cap_fifo)
    return {"workload": "%d jobs of the serving recipe (16-1024 envs, 4-256 bodies, 64-256 px), %d Poisson requests "
                        "at %d%% of the continuous-batching capacity (the rate served under saturating Poisson "
                        "arrivals); HBM budget 60%% of free memory"
                        % (njobs, nreq, round(100 * load)),
            "jobs": njobs, "requests": nreq, "load": load,
            "capacity_requests_per_s": cap, "capacity_fifo_requests_per_s": cap_fifo,
            "burst_requests_per_s": burst_cap, "burst_fifo_requests_per_s": burst_fifo, "arrival_rate_hz": rate,
            "continuous_batching": cb, "serialized_fifo": fifo,
            "serialized_fifo_at_own_load": dict(fifo_own, arrival_rate_hz=load * cap_fifo)}


CONFIGS = {
    1: ("cfg1: 16 envs x 8 spheres, 4 substeps, one 64x64 RGB-D camera per env; plain serialized sim-then-render, "
        "100 steps", 100, 0),
    3: ("cfg3: 4096 envs x 64 convex hulls (500-2000 tris each), 8 substeps, two 128x128 RGB-D cameras per env; "
        "autotuned (tile size, bin limit, co-scheduling mode and split) and replayed from a CUDA graph", 16, 4),
    4: ("cfg4: 2048 envs with 4-256 bodies (log-uniform) and 64/128/256 px cameras; one persistent launch per phase "
        "(work lists by size class)", 40, 20),
}


def phase_roofline(env, sc, Ts: float, Tr: float, fp32_peak: float, hbm_peak: float, bytes_out: int) -> dict:
    """Both phases of one configuration against their bounds: the physics
    against the FP32 lanes (the method's operations counted per environment
    from its body and contact counts), the render against HBM (its output
    frames and the poses it reads)."""
    cc = env.contact_counts().astype(np.float64)
    nb = np.diff(sc.body_off).astype(np.float64)
    flops = float(sum(sim_flops(c, int(n), sc.params.substeps, sc.params.iterations) for c, n in zip(cc, nb)))
    sim_ach = flops / (Ts / 1000.0) / 1e12
    alg = bytes_out + env.B * 28
    ren_ach = alg / (Tr / 1000.0) / 1e9
    return {"sim": {"bound": "alu", "achieved": sim_ach, "peak": fp32_peak, "unit": "TFLOP/s",
                    "frac": sim_ach / fp32_peak, "algorithmic_flops_per_launch": flops, "launch_ms": Ts},
            "render": {"bound": "hbm", "achieved": ren_ach, "peak": hbm_peak, "unit": "GB/s",
                       "frac": ren_ach / hbm_peak, "algorithmic_bytes_per_launch": alg, "launch_ms": Tr}}


def oracle_sample(sc, secs: float = 1.0, max_envs: int = 8, settle: int = 0) -> dict:
    """The oracle as it stands, single-threaded, on a bounded sample of a
    configuration: its first environments (at most max_envs), stepped and
    rendered for at least `secs` (at least one step)."""
    import oracle
    sub = sc.subset(range(min(max_envs, sc.num_envs)))
    st = sub.state()
    if settle:
        st, _, _ = oracle.sim_step(sub, settle)
    t = time.perf_counter()
    n = 0
    while n < 1 or time.perf_counter() - t < secs:
        st, _, _ = oracle.sim_step(sub, 1, state=st)
        oracle.render(sub, st["pos"], st["quat"], triid=False)
        n += 1
    dt = time.perf_counter() - t
    return {"value": sub.num_envs * n / dt, "unit": "env-steps/s", "cores": 1, "kind": "oracle",
            "sample": "%d envs x %d steps of this configuration, sim + render, single-threaded C oracle"
                      % (sub.num_envs, n)}


def config_bench(V, S, k: int, fp32_peak: float, hbm_peak: float, warmup: int, cpu: bool) -> dict:
    """One of the other configurations: serialized and co-scheduled (cfg3:
    the autotuner's choice replayed from a CUDA graph; cfg4: persistent work
    lists) rendered env-steps/s, both phases' rooflines, and the oracle on a
    sample of the same workload."""
    import torch
    desc, steps, settle = CONFIGS[k]
    sc = {1: S.cfg1, 3: S.cfg3, 4: S.cfg4}[k]()
    env = V.Env(sc, persistent=(k == 4))
    ring = [env.alloc_frame(triid=False), env.alloc_frame(triid=False)]
    bytes_out = env.P * 7
    if settle:
        env.pipeline_run(settle, ring)
    env.pipeline_run(warmup, ring)
    torch.cuda.synchronize()
    start = env.get_state()   # every timed run (and the autotuner) steps from here

    def timed(n, runs=3):
        res = []
        for _ in range(runs):
            env.set_state(start)
            torch.cuda.synchronize()
            t = time.perf_counter()
            tm = env.pipeline_run(n, ring, timing=True)
            wall = time.perf_counter() - t
            dev = tm["total_ms"] / 1000.0
            res.append((dev if (dev == dev and dev > 0) else wall, tm))
        res.sort(key=lambda r: r[0])
        return res[len(res) // 2]

    t_ser, tm_ser = timed(steps)
    Ts, Tr = float(np.mean(tm_ser["sim_ms"])), float(np.mean(tm_ser["render_ms"]))
    out = {"workload": desc, "envs": sc.num_envs, "bodies": sc.num_bodies, "cameras": env.C, "pixels": int(env.P),
           "steps": steps, "warmup": warmup, "settle_steps": settle,
           "render_path": "tiled" if env.info().render_path == V.RENDER_TILED else "band",
           "serialized": {"value": sc.num_envs * steps / t_ser, "ms_per_step": 1000.0 * t_ser / steps},
           "phase_ms": {"sim": Ts, "render": Tr, "ideal_overlap": (Ts + Tr) / max(Ts, Tr)},
           "roofline": phase_roofline(env, sc, Ts, Tr, fp32_peak, hbm_peak, bytes_out)}
    if k == 3:
        env.set_state(start)
        tuned = env.autotune(ring, steps=2, use_cache=False)
        out["autotuned"] = tuned
        if tuned.get("graph_steps", 0) <= 0:
            try:
                env.pipeline_capture(8, ring, stream=None if env.cosched else torch.cuda.Stream())
            except Exception:
                pass
        t_co, _ = timed(steps)
        out["coscheduled"] = {"value": sc.num_envs * steps / t_co, "ms_per_step": 1000.0 * t_co / steps,
                              "mode": "autotuned choice (cosched_mode %d, graph steps %d)"
                                      % (tuned["cosched_mode"], tuned["graph_steps"])}
    elif k == 4 or k == 1:
        env.coschedule(V.COSCHED_STREAMS)
        env.pipeline_run(warmup, ring)
        t_co, _ = timed(steps)
        out["coscheduled"] = {"value": sc.num_envs * steps / t_co, "ms_per_step": 1000.0 * t_co / steps,
                              "mode": "two streams sharing all SMs" + (", persistent work lists" if k == 4 else "")}
    out["value"] = max(out["serialized"]["value"], out.get("coscheduled", {}).get("value", 0.0))
    out["speedup_vs_serialized"] = out["value"] / out["serialized"]["value"]
    out["status_flags"] = env.status()[1]
    env.close()
    if cpu:
        try:
            out["cpu_baseline"] = oracle_sample(sc, secs=1.0, max_envs={1: 16, 3: 1, 4: 8}[k])
        except Exception as ex:
            out["cpu_baseline"] = {"value": None, "error": repr(ex)}
    return out


def rollout_bench(V, S, E: int, steps: int, warmup: int, settle: int) -> dict:
    """RL rollout (vuda_rollout_run): the benchmark's environments split into
    two groups of trajectories, each step sim -> render -> MLP policy (hidden
    256 and 4096, randomly initialised, FP32) on one GPU; time-sliced (one
    stream) against the inter-trajectory schedule (one group's sim beside
    the other's render and policy) on shared SMs and on 50/50 green
    partitions.  Rendered env-steps/s of both groups together."""
    import torch
    from paper_2605_01352_b300.policy import MLPPolicy
    h = E // 2
    scenes = [S.cfg2(h, env_base=0), S.cfg2(E - h, env_base=h)]
    out = {"workload": "%d envs of the benchmark scene in two groups of %d, policy MLP on pooled 16x16 depth and "
                       "luminance (512 features) -> 3 forces per body" % (E, h), "steps": steps, "warmup": warmup}
    for hidden in (256, 4096):
        res = {}
        # green: the half split; green_88 / green_96: the sim partition one
        # and two 8-SM steps larger (the sim of both groups sets the step)
        for mode in ("serialized", "streams", "green", "green_88", "green_96"):
            envs = [V.Env(sc) for sc in scenes]
            rings = [[e.alloc_frame(triid=False), e.alloc_frame(triid=False)] for e in envs]
            forces = [torch.zeros((3, e.B), dtype=torch.float32, device="cuda") for e in envs]
            pols = [MLPPolicy(envs[g], sc, hidden, seed=3 + g) for g, sc in enumerate(scenes)]
            for e, r in zip(envs, rings):
                e.pipeline_run(settle, r)
            for g in range(2):     # one CUDA graph per group and frame slot
                pols[g].capture(rings[g], forces[g], torch.cuda.Stream())

            def policy(group, step, slot, stream):
                pols[group].act_captured(slot, stream)

            if mode == "streams":
                envs[0].coschedule(V.COSCHED_STREAMS)
            elif mode.startswith("green"):
                envs[0].coschedule(V.COSCHED_GREEN, int(mode[6:]) if mode != "green" else 0)
            cur = torch.cuda.current_stream()
            V.rollout_run(envs[0], envs[1], warmup, rings[0], rings[1], forces[0], forces[1], policy, stream=cur)
            torch.cuda.synchronize()
            t = time.perf_counter()
            V.rollout_run(envs[0], envs[1], steps, rings[0], rings[1], forces[0], forces[1], policy, stream=cur)
            torch.cuda.synchronize()
            wall = time.perf_counter() - t
            res[mode] = {"value": E * steps / wall, "ms_per_step": 1000.0 * wall / steps}
            if mode.startswith("green"):
                res[mode]["sim_sms"] = envs[0].cosched["sim_sms"]
            for e in envs:
                e.close()
        for mode in ("streams", "green", "green_88", "green_96"):
            res[mode]["speedup_vs_serialized"] = res[mode]["value"] / res["serialized"]["value"]
        out["hidden_%d" % hidden] = res
    out["timing"] = ("wall clock around vuda_rollout_run (host callbacks replay the policy's CUDA graph), after %d "
                     "warm-up steps" % warmup)
    return out


def physics_options_bench(V, S, E: int, settle: int) -> dict:
    """Physics step time on the settled benchmark batch with the options
    beyond the configured physics: the gyroscopic term of boxes and box-box
    edge-edge contacts (each off / on; the headline uses neither), and hull
    contacts on a batch of the same shape with hulls."""
    import dataclasses
    import torch
    out = {}
    s0 = torch.cuda.current_stream()
    for gyro, edges in ((0, 0), (1, 0), (0, 1), (1, 1)):
        sc = S.cfg2(E)
        sc = dataclasses.replace(sc, params=dataclasses.replace(sc.params, gyroscopic=gyro, edge_contacts=edges))
        env = V.Env(sc)
        ring = [env.alloc_frame(triid=False), env.alloc_frame(triid=False)]
        env.pipeline_run(settle, ring)
        for _ in range(3):
            env.sim_step(1, stream=s0)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s0)
        for _ in range(20):
            env.sim_step(1, stream=s0)
        b.record(s0)
        torch.cuda.synchronize()
        out["gyroscopic_%d_edge_contacts_%d" % (gyro, edges)] = {
            "sim_ms": a.elapsed_time(b) / 20, "contacts_mean": float(env.contact_counts().mean())}
        env.close()
    # hull contacts: the benchmark's batch shape with every third body a
    # convex hull of 8-48 faces (spheres and boxes between), simulated as
    # spheres of their radius (option off) and through their own faces (on)
    for hulls in (0, 1):
        sc = S.generate(E, 32, S.config_seed(2) ^ 0x4855, kinds="mixed_hulls", res=128, substeps=8,
                        hull_tris=(8, 48), n_hull_meshes=16)
        sc = dataclasses.replace(sc, params=dataclasses.replace(sc.params, hull_contacts=hulls))
        env = V.Env(sc)
        ring = [env.alloc_frame(triid=False), env.alloc_frame(triid=False)]
        env.pipeline_run(settle, ring)
        for _ in range(3):
            env.sim_step(1, stream=s0)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s0)
        for _ in range(20):
            env.sim_step(1, stream=s0)
        b.record(s0)
        torch.cuda.synchronize()
        out["mixed_hulls_hull_contacts_%d" % hulls] = {
            "sim_ms": a.elapsed_time(b) / 20, "contacts_mean": float(env.contact_counts().mean()),
            "workload": "%d envs x 32 bodies (sphere, box, hull of 8-48 faces in turn), 8 substeps, settled" % E}
        env.close()
    return out


def sim_flops(contacts: float, bodies: int, substeps: int, iterations: int) -> float:
    """Floating-point operations of one environment-step of the physics as
    the method defines them (each add, mul, div and sqrt counted once): per
    body and substep 116 (velocity, rotation, world inverse inertia,
    position and quaternion update); per candidate pair 12 (bounding-sphere
    test); about 40 per narrow-phase item (taken as 2.7 items per contact);
    per contact 160 to set up and 95 per Jacobi iteration; per body-contact
    list entry 6 and per body 27 per iteration for the sums and update."""
    n, c = bodies, contacts
    entries = 2.0 * c - n   # pair contacts appear in two bodies' lists
    per_sub = 116 * n + 12 * n * (n - 1) / 2 + 40 * 2.7 * c + 160 * c + iterations * (95 * c + 6 * entries + 27 * n)
    return per_sub * substeps


def csrc_sha() -> str:
    """Hash of every CUDA source of the library (a change anywhere
    invalidates the committed counters)."""
    d = os.path.join(ROOT, "paper_2605_01352_b300", "csrc")
    h = hashlib.sha256()
    for f in sorted(os.listdir(d)):
        if f.endswith((".cu", ".cuh")):
            h.update(f.encode())
            h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()


def kernel_counters(kernel: str) -> dict:
    """The committed ncu counters of `kernel` (DRAM bytes per launch, issue
    slots active, SM throughput), if they were taken on the current kernel
    sources; empty otherwise."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(path))
        if rec.get("csrc_sha256") != csrc_sha():
            return {}
        return dict(rec["kernels"][kernel])
    except Exception:
        return {}


def kernel_traffic(kernel: str):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if it
    was taken on the current kernel sources."""
    v = kernel_counters(kernel).get("bytes_per_launch")
    return float(v) if v is not None else None


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    ws, rank, local = dist_setup()
    from paper_2605_01352_b300 import build
    if rank == 0:
        build.build()
    barrier(ws)
    from paper_2605_01352_b300 import scene as S
    from paper_2605_01352_b300 import vuda as V

    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6400.0))
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"

    E = args.envs
    sc = rank_scene(S, rank, E)
    env = V.Env(sc)
    env_info_path = env.info().render_path
    launches_per_step = 3   # sim_kernel, then bin_kernel + tile_kernel (tiled) or shade_kernel + render_kernel (band)
    ring = [env.alloc_frame(triid=False), env.alloc_frame(triid=False)]
    P = env.P
    bytes_out = P * 7                                  # RGB8 + f32 depth
    bytes_pose = env.B * 28                            # pose slot read by the renderer
    bytes_state = env.B * (52 + 52 + 40 + 28)          # physics state in/out, params, pose out

    # settle: bodies land and piles form (untimed); every timed run below
    # starts from this settled state, so that the modes compare the same work
    # (piles keep settling, and a later run would step heavier contacts)
    env.pipeline_run(args.settle, ring)
    torch.cuda.synchronize()
    settled = env.get_state()
    clk = Clocks(local)
    clk.start()

    def timed(n, runs=5):
        """Median over `runs` timed runs of n steps from the settled state
        (device time of each run, max over ranks); the per-step timings and
        wall time of the median run."""
        res = []
        for _ in range(runs):
            env.set_state(settled)
            barrier(ws)
            torch.cuda.synchronize()
            clk.on = True
            t = time.perf_counter()
            tm = env.pipeline_run(n, ring, timing=True)
            wall = time.perf_counter() - t
            clk.on = False
            dev = tm["total_ms"] / 1000.0
            sec = dev if (dev == dev and dev > 0) else wall   # device time unless NaN
            res.append((allreduce_max(ws, sec), tm, wall))
        res.sort(key=lambda r: r[0])
        return res[len(res) // 2]

    # serialized: sim then render on one stream with the full GPU
    env.pipeline_run(args.warmup, ring)
    t_ser, tm_ser, _ = timed(args.steps)
    Ts = float(np.mean(tm_ser["sim_ms"]))
    Tr = float(np.mean(tm_ser["render_ms"]))

    if args.serial_only:
        clk.stop()
        if rank == 0:
            print(json.dumps({"serialized_env_steps_per_s": ws * E * args.steps / t_ser, "phase_ms":
                              {"sim": Ts, "render": Tr}}), flush=True)
        env.close()
        return
    def graph_timed(n, stream=None):
        """Steps replayed from a captured graph of 8 pipelined steps (median
        of 5 runs of n steps, rounded down to whole graphs, scaled to n)."""
        n8 = max(8, n - n % 8)
        env.pipeline_capture(8, ring, stream=stream)
        env.pipeline_run(8, ring, stream=stream)
        res = []
        for _ in range(5):
            env.set_state(settled)
            barrier(ws)
            torch.cuda.synchronize()
            clk.on = True
            t = time.perf_counter()
            tm = env.pipeline_run(n8, ring, stream=stream, timing=True)
            wall = time.perf_counter() - t
            clk.on = False
            dev = tm["total_ms"] / 1000.0
            res.append(allreduce_max(ws, dev if (dev == dev and dev > 0) else wall))
        env.pipeline_release_graph()
        return float(np.median(res)) * n / n8

    # serialized, replayed from a graph as well (launch gaps removed on both sides)
    t_serg = None
    try:
        t_serg = graph_timed(args.steps, stream=torch.cuda.Stream())
    except Exception as ex:  # report why, keep the main line
        t_serg = repr(ex)
    # co-scheduled: disjoint SM partitions (green contexts) at the fixed 50/50 split
    cos = env.coschedule(V.COSCHED_GREEN, args.sim_sms)
    env.pipeline_run(args.warmup, ring)
    t_gr, tm_gr, wall_gr = timed(args.steps)
    # the other half split the 8-SM granularity allows (72 sim / 76 render)
    green_alt = None
    try:
        cos_alt = env.coschedule(V.COSCHED_GREEN, cos["sim_sms"] - cos["sm_granularity"])
        env.pipeline_run(args.warmup, ring)
        t_ga = timed(args.steps)[0]
        green_alt = {"value": job_throughput(ws, E, args.steps, t_ga), "ms_per_step": 1000.0 * t_ga / args.steps,
                     "partition": cos_alt}
    except Exception as ex:  # report why, keep the main line
        green_alt = {"error": repr(ex)}
    # co-scheduled on two plain streams sharing all SMs, with each stream priority
    st_runs = {}
    for pname, prio in (("none", V.PRIORITY_NONE), ("sim_first", V.PRIORITY_SIM), ("render_first", V.PRIORITY_RENDER)):
        env.coschedule(V.COSCHED_STREAMS, priority=prio)
        env.pipeline_run(args.warmup, ring)
        st_runs[pname] = (prio,) + tuple(timed(args.steps))
    best_p = min(st_runs, key=lambda k: st_runs[k][1])
    prio_best, t_st, tm_st, wall_st = st_runs[best_p]
    # the better of green and streams, replayed from a captured CUDA graph of 8 pipelined steps
    best_mode = V.COSCHED_STREAMS if t_st <= t_gr else V.COSCHED_GREEN
    t_graph = None
    try:
        env.coschedule(best_mode, args.sim_sms, priority=prio_best if best_mode == V.COSCHED_STREAMS else 0)
        t_graph = graph_timed(args.steps)
    except Exception as ex:  # report why, keep the main line
        t_graph = repr(ex)
    best_name = ("streams_shared_sms_priority_" + best_p) if best_mode == V.COSCHED_STREAMS else "green_50_50"
    # headline: the fastest co-scheduled configuration measured above
    cands = [("green_50_50", t_gr, tm_gr, wall_gr), ("streams_shared_sms_priority_" + best_p, t_st, tm_st, wall_st)]
    if isinstance(t_graph, float):
        cands.append((best_name + "_graph8", t_graph, None, None))
    head = min(cands, key=lambda c: c[1])
    t_co, wall_co = head[1], head[3]
    tm_lat = head[2] if head[2] is not None else (tm_st if best_mode == V.COSCHED_STREAMS else tm_gr)
    lat = tm_lat["step_ms"]
    lat = lat[np.isfinite(lat)]
    # the autotuner's own choice (band height, co-scheduling mode and split, graph)
    try:
        env.set_state(settled)
        tuned = env.autotune(ring, steps=6, use_cache=False)
        tuned["env_steps_per_s"] = ws * E * 1000.0 / tuned["ms_per_step"]
    except Exception as ex:  # report why, keep the main line
        tuned = {"error": repr(ex)}
    env.coschedule(V.COSCHED_STREAMS, priority=prio_best)

    # end to end through the host-buffer loop: forces in, frames out
    e2e = None
    if not args.no_e2e:
        hf = torch.zeros((3, env.B), dtype=torch.float32).pin_memory()
        hr = torch.empty((2, P, 3), dtype=torch.uint8).pin_memory()
        hd = torch.empty((2, P), dtype=torch.float32).pin_memory()
        env.pipeline_run_host(args.warmup, ring, hr, hd, h_force=hf)
        env.set_state(settled)
        barrier(ws)
        torch.cuda.synchronize()
        t = time.perf_counter()
        env.pipeline_run_host(args.steps, ring, hr, hd, h_force=hf)
        t_e2e = allreduce_max(ws, time.perf_counter() - t)
        e2e = {"value": ws * E * args.steps / t_e2e, "unit": "env-steps/s",
               "h2d_bytes_per_step": int(hf.numel() * 4), "d2h_bytes_per_step": int(bytes_out),
               "path": "vuda_pipeline_run_host (co-scheduled), pinned host buffers, wall clock"}
        # the loop's ceiling: a plain pinned device -> host copy of one step's frame bytes
        dev_b = torch.empty(int(bytes_out), dtype=torch.uint8, device="cuda")
        host_b = torch.empty(int(bytes_out), dtype=torch.uint8).pin_memory()
        for _ in range(2):
            host_b.copy_(dev_b, non_blocking=True)
        torch.cuda.synchronize()
        t = time.perf_counter()
        for _ in range(10):
            host_b.copy_(dev_b, non_blocking=True)
        torch.cuda.synchronize()
        copy_gbs = 10 * bytes_out / (time.perf_counter() - t) / 1e9
        achieved_gbs = bytes_out * e2e["value"] / (ws * E) / 1e9
        e2e["d2h_roofline"] = {"bound": "d2h copy", "achieved_gbs": achieved_gbs, "peak_gbs": copy_gbs,
                               "frac": achieved_gbs / copy_gbs,
                               "peak_source": "measured here: pinned device -> host copy of one step's frame bytes"}
        del dev_b, host_b

    flags = env.status()[1]
    env_stats = {"contacts_mean": float(env.contact_counts().mean()), "bodies": 32,
                 "substeps": sc.params.substeps, "iterations": sc.params.iterations}
    env.close()
    if rank != 0:
        clk.stop()
        return
    sm_count = torch.cuda.get_device_properties(local).multi_processor_count
    fp32_peak = sm_count * 128 * float(peaks.get("sm_max_mhz", 2032.0)) * 1e6 / 1e12   # TFLOP/s, one op per lane
    # the other configurations, the RL rollout and the serving grid (one GPU)
    configs = {}
    if ws == 1:
        for k in [int(x) for x in args.configs.split(",") if x.strip()]:
            clk.on = True
            try:
                configs["cfg%d" % k] = config_bench(V, S, k, fp32_peak, hbm_peak, max(3, args.warmup),
                                                    not args.no_cpu_baseline)
            except Exception as ex:  # report why, keep the main line
                configs["cfg%d" % k] = {"error": repr(ex)}
            clk.on = False
    rollout = None
    if ws == 1 and not args.no_rollout:
        clk.on = True
        try:
            rollout = rollout_bench(V, S, E, min(args.steps, 50), max(3, args.warmup), args.settle)
        except Exception as ex:  # report why, keep the main line
            rollout = {"error": repr(ex)}
        clk.on = False
    options = None
    if ws == 1:
        clk.on = True
        try:
            options = physics_options_bench(V, S, E, args.settle)
        except Exception as ex:  # report why, keep the main line
            options = {"error": repr(ex)}
        clk.on = False
    serving = None
    if not args.no_serve and ws == 1:
        serving = []
        for nj in [int(x) for x in args.serve_jobs.split(",") if x.strip()]:
            clk.on = True
            try:
                serving.append(serving_bench(V, S, nj, args.serve_requests))
            except Exception as ex:  # report why, keep the main line
                serving.append({"jobs": nj, "error": repr(ex)})
            clk.on = False
        configs["cfg5"] = serving
    clk.stop()

    v_co = job_throughput(ws, E, args.steps, t_co)
    v_ser = job_throughput(ws, E, args.steps, t_ser)
    v_gr = job_throughput(ws, E, args.steps, t_gr)
    # physics: plain FP32 arithmetic (no FMA contraction), bound by the FP32 lanes
    flops = sim_flops(env_stats["contacts_mean"], env_stats["bodies"], env_stats["substeps"],
                      env_stats["iterations"]) * E
    ach = flops / (Ts / 1000.0) / 1e12
    roof_sim = {"kernel": "sim_kernel", "bound": "alu", "achieved": ach, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": ach / fp32_peak, "traffic": kernel_traffic("sim_kernel"),
                "algorithmic_flops_per_launch": flops, "launch_ms": Ts,
                "peak_source": "derived: SMs x 128 FP32 lanes x max SM clock (unfused ops; the path is built "
                               "without FMA contraction)",
                "hbm_bytes_per_launch": bytes_state, "hbm_achieved_gbs": bytes_state / (Ts / 1000.0) / 1e9,
                "ncu_issue_active_pct": kernel_counters("sim_kernel").get("issue_active_pct"),
                "ncu_sm_throughput_pct": kernel_counters("sim_kernel").get("sm_throughput_pct")}
    # renderer: the frame it must write and the poses it reads, over the render phase
    alg = bytes_out + bytes_pose
    ach_r = alg / (Tr / 1000.0) / 1e9
    roof_ren = {"kernel": "tile_kernel (+ bin_kernel: the render phase)" if env_info_path == V.RENDER_TILED
                else "render_kernel (+ shade_kernel: the render phase)", "bound": "hbm",
                "achieved": ach_r, "peak": hbm_peak, "unit": "GB/s", "frac": ach_r / hbm_peak,
                "traffic": kernel_traffic("tile_kernel" if env_info_path == V.RENDER_TILED else "render_kernel"),
                "algorithmic_bytes_per_launch": alg, "launch_ms": Tr,
                "ncu_issue_active_pct": kernel_counters("tile_kernel").get("issue_active_pct"),
                "ncu_sm_throughput_pct": kernel_counters("tile_kernel").get("sm_throughput_pct"),
                "peak_source": peak_src + " (MEASURED_PEAKS.json hbm_gbs)" if peak_src == "measured" else peak_src}
    roof = roof_sim if Ts >= Tr else roof_ren
    roof_other = roof_ren if Ts >= Tr else roof_sim
    cpu = cpu1 = None
    if not args.no_cpu_baseline and ws == 1:
        try:
            cpu1 = cpu_baseline()
            cpu = cpu_baseline_all_cores()
        except Exception as ex:  # the oracle is test infrastructure; report why it is missing
            cpu = {"value": None, "error": str(ex)}
    out = {
        "metric": METRIC, "value": v_co, "unit": "env-steps/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1000.0 * t_co / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "envs_per_gpu": E, "bodies_per_env": 32, "substeps": 8,
                   "iterations": 8, "camera": "128x128 RGB8 + f32 depth", "parallelism": "replicas" if ws > 1
                   else "single GPU", "render_path": "tiled" if env_info_path == V.RENDER_TILED else "band",
                   "l2": "per-step working set (frames 2 x %.0f MB) exceeds the 126 MB L2" % (bytes_out / 1e6),
                   "timed_from": "every timed run of every mode starts from the state %d steps after the drop"
                                 % args.settle},
        "coscheduled_mode": head[0],
        "serialized": {"value": v_ser, "ms_per_step": 1000.0 * t_ser / args.steps},
        "serialized_graph8": ({"value": job_throughput(ws, E, args.steps, t_serg),
                               "ms_per_step": 1000.0 * t_serg / args.steps}
                              if isinstance(t_serg, float) else {"error": t_serg}),
        "coscheduled_green_50_50": {"value": v_gr, "ms_per_step": 1000.0 * t_gr / args.steps, "partition": cos},
        "coscheduled_green_other_half_split": green_alt,
        "speedup_green_50_50_vs_serialized": v_gr / v_ser,
        "coscheduled_streams_shared_sms": {k: {"value": job_throughput(ws, E, args.steps, v[1]),
                                               "ms_per_step": 1000.0 * v[1] / args.steps}
                                           for k, v in st_runs.items()},
        "coscheduled_graph8": ({"value": job_throughput(ws, E, args.steps, t_graph),
                                "ms_per_step": 1000.0 * t_graph / args.steps, "mode": best_name}
                               if isinstance(t_graph, float) else {"error": t_graph}),
        "autotuned": tuned,
        "speedup_vs_serialized": v_co / v_ser,
        "speedup_vs_serialized_graph8": (v_co / job_throughput(ws, E, args.steps, t_serg)
                                         if isinstance(t_serg, float) else None),
        "phase_ms": {"sim": Ts, "render": Tr, "ideal_overlap": (Ts + Tr) / max(Ts, Tr)},
        "latency_ms": {"p50": float(np.percentile(lat, 50)) if lat.size else None,
                       "p99": float(np.percentile(lat, 99)) if lat.size else None},
        "e2e": e2e,
        "roofline": roof,
        "roofline_other_phase": roof_other,
        "cpu_baseline": cpu,
        "cpu_baseline_single_thread": cpu1,
        "serving": serving,
        "configs": configs,
        "rollout": rollout,
        "physics_options": options,
        "gpu_launches": launches_per_step * args.steps,
        "status_flags": flags,
        "clocks": clk.summary(),
        "wall_s_coscheduled": wall_co,
    }
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
