#!/usr/bin/env python
"""Throughput of the hot-electron PIC step on GB300: particle-steps/s and the
achieved fraction of the HBM roofline of the step kernel.

Workload (default): the large Fe(15 nm)/Au(300 nm) bilayer, 2e8 carriers
created by the pump pulse, capacity 4e8, dt = 0.5 fs, 60 energy bins,
densities every 50 steps, compaction every 50 steps.  Set-up (untimed) runs
the pulse window (t < 150 fs) and the launch-configuration autotuner, so that
the timed steps see the steady state.  One benchmark step = one
moment/compaction period of 50 time steps, i.e. one pass of every stage of
the step (flight, scattering, secondaries, deposit, compaction).  The
particle state (6.4 GB) is larger than L2, so no flush is needed between
steps.  At this capacity the buffer is full from the pulse on (the cascade
would hold more than 5 times the 2e8 primaries), so most secondaries are
dropped and counted; a second leg with the capacity raised to 2^30 slots
times the same kernels while secondaries are still placed.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

`--impl reference` times the CPU oracle on the host cores on a bounded sample
of the same workload (same metric and unit).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "particle-steps/s"
UNIT = "particle-steps/s"
HBM_FALLBACK_GBS = 6800.0
# Algorithmic bytes per unit, the count of the method's data movement:
# read the 16 B state and write z (4 B) per live carrier-step, write the
# other 12 B for a carrier with an event, 16 B per secondary placed.
B_STEP, B_EVENTFUL, B_CHANGED, B_SPAWN = 20, 12, 0, 16
# The stricter count of what the kernels must move: read z, mu, packed (12 B)
# + write z (4 B) per carrier-step (the id is never read: draws are keyed by
# slot), 8 B (mu, packed) per carrier whose record changed, 16 B per secondary
S_STEP, S_EVENTFUL, S_CHANGED, S_SPAWN = 16, 0, 8, 16


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--config", type=int, default=4)
    ap.add_argument("--scale", type=float, default=1.0)
    ap.add_argument("--period", type=int, default=0, help="time steps per benchmark step")
    ap.add_argument("--deterministic", action="store_true")
    ap.add_argument("--blocks-per-sm", type=int, default=0)
    ap.add_argument("--hist-mode", type=int, default=0)
    ap.add_argument("--ring", type=int, default=0)
    ap.add_argument("--graph", type=int, default=1, choices=(0, 1),
                    help="1: the main line replays whole periods from CUDA graphs (use_graph); "
                         "0: one launch per kernel")
    ap.add_argument("--event-pass", type=int, default=0, choices=(0, 1),
                    help="ordinary steps: 0 general step inside the streaming pass where it "
                         "applies, 1 separate event pass (the autotuner may change it)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--batched-scale", type=float, default=1.0)
    ap.add_argument("--batched-steps", type=int, default=0)
    ap.add_argument("--adjoint-scale", type=float, default=1.0)
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--autotune-steps", type=int, default=4)
    ap.add_argument("--no-unsaturated", action="store_true")
    ap.add_argument("--no-spin-valve", action="store_true")
    ap.add_argument("--spin-valve-scale", type=float, default=1.0)
    return ap.parse_args()


def workload(args):
    from paper_1807_04733_gb300 import workloads as W
    flags = W.FLAG_DETERMINISTIC if args.deterministic else 0
    wl = W.config(args.config, scale=args.scale, flags=flags)
    period = args.period if args.period else (wl.moment_every if wl.moment_every > 1 else 50)
    st = wl.stacks[0]
    pre = int(math.ceil(2 * st.t0 / wl.dt)) if st.n0 > 0 else 0
    return wl, period, pre


def config_dict(wl, period, pre, args):
    st = wl.stacks[0]
    mats = {0: "Fe", 1: "Au", 2: "Fe_AP"}
    return {
        "workload": wl.name,
        "stack": "/".join("%s(%dnm)" % (mats[m], c) for c, m in zip(st.layer_cells, st.layer_mat)),
        "n0": sum(s.n0 for s in wl.stacks),
        "capacity": sum(s.capacity for s in wl.stacks),
        "n_stacks": len(wl.stacks),
        "dt_fs": wl.dt, "n_e": wl.n_e, "dz_nm": wl.dz,
        "time_steps_per_step": period,
        "moment_every": wl.moment_every, "compact_every": wl.compact_every,
        "pre_roll_time_steps": pre,
        "build": "deterministic (no FMA)" if args.deterministic else "fast (FMA)",
        "l2": "inputs larger than L2 (16 B x capacity of particle state)",
        "launch": "whole periods replayed from CUDA graphs" if args.graph else "one launch per kernel",
    }


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback"


# ncu DRAM traffic of the step kernels, bytes per live carrier-step, from one
# steady-state capture of each on this workload scaled to 1/20, for the two
# forms of an ordinary step: "separate" (k_stream + k_event + k_place) and
# "fused" (k_stream with the general step inside + k_place); the traffic grows
# in proportion to the carriers advanced.  Valid only for the kernel source
# whose hash is given: reported as null once the kernels change.
NCU_TRAFFIC = {"separate": 16.76, "fused": 14.81, "src_sha": "59659cabec44282e"}


def kernel_sha():
    with open(os.path.join(ROOT, "paper_1807_04733_gb300", "csrc", "pic_step.cuh"), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


class Clocks:
    """nvidia-smi sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.p = None
        # the samples are read back at the end of the timed region
        self.path = os.path.join(tempfile.gettempdir(), "pic_bench_clocks_%d_%s.csv" % (os.getpid(), gpu_index))

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(5)
        except Exception:
            self.p.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i, v in enumerate(r)
                          if v.lower().startswith("active")})
        return {"sm_mhz": statistics.median(r[0] for r in rows),
                "sm_max_mhz": max(r[1] for r in rows), "reasons": reasons,
                "samples": len(rows)}


# ---------------------------------------------------------------------------
# oracle workers (CPU baseline and the reference arm): one process per core,
# each advancing its own replica of the workload
# ---------------------------------------------------------------------------
def _oracle_worker(conn, cfg_index, scale, seed, n_steps_max):
    from oracle.oracle import OracleSim
    from paper_1807_04733_gb300 import workloads as W
    wl = W.config(cfg_index, scale=scale, seed=seed)
    sim = OracleSim(wl, n_steps_max=n_steps_max)
    while True:
        cmd, n = conn.recv()
        if cmd == "stop":
            break
        t = time.perf_counter()
        rc = sim.step(n)
        _, _, led = sim.moments()
        conn.send((rc, led["particle_steps"], time.perf_counter() - t))


class OraclePool:
    def __init__(self, cfg_index, scale, workers, n_steps_max):
        ctx = mp.get_context("spawn")
        self.conns, self.procs = [], []
        for w in range(workers):
            a, b = ctx.Pipe()
            p = ctx.Process(target=_oracle_worker, args=(b, cfg_index, scale, 1000 + w, n_steps_max),
                            daemon=True)
            p.start()
            self.conns.append(a)
            self.procs.append(p)

    def step(self, n):
        """Advance every replica by n time steps; returns the particle-steps done."""
        for c in self.conns:
            c.send(("step", n))
        out = [c.recv() for c in self.conns]
        if any(rc != 0 for rc, _, _ in out):
            raise RuntimeError("oracle step failed")
        total = sum(ps for _, ps, _ in out)
        done = total - getattr(self, "_total", 0)
        self._total = total
        return done

    def close(self):
        for c in self.conns:
            c.send(("stop", 0))
        for p in self.procs:
            p.join(10)


def cpu_sample(args, wl, pre):
    """Oracle replicas of a scaled copy of the workload on the host cores."""
    cores = max(1, min(os.cpu_count() or 1, 64))
    # the large workload: 1.25e6 slots (20 MB of state) per replica, beyond
    # what the host cores' caches hold together
    scale = 3.125e-3 * args.scale if args.config == 4 else 1e-2 * args.scale
    n_each = max(1, int(round(wl.stacks[0].capacity * scale)))
    return cores, scale, n_each


def oracle_replicas(cfg_index, total_n0, pre, timed, cores=None, label=""):
    """The oracle on the host cores: one replica per core (its own seed), the
    workload scaled so that the replicas start total_n0 carriers together;
    pre untimed steps (the pulse window), then `timed` steps timed."""
    from paper_1807_04733_gb300 import workloads as W
    cores = cores or max(1, min(os.cpu_count() or 1, 64))
    full = W.config(cfg_index)
    scale = total_n0 / float(full.stacks[0].n0) / cores
    each = W.config(cfg_index, scale=scale)
    pool = OraclePool(cfg_index, scale, cores, pre + timed + 1)
    try:
        pool.step(pre)
        t = time.perf_counter()
        ps = pool.step(timed)
        dt = time.perf_counter() - t
    finally:
        pool.close()
    st = each.stacks[0]
    sample = ("%s: %d oracle replica(s), one per core, of %s scaled by %.4g (%d carriers, capacity %d, "
              "%.0f MB of particle state each): %d pulse steps untimed, %d steps timed"
              % (label, cores, full.name, scale, st.n0, st.capacity, st.capacity * 16 / 1e6, pre, timed))
    return {"value": ps / dt, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
            "particle_steps": ps, "seconds": dt}


def run_cpu_baselines():
    """The oracle as it stands, timed on the host: single-threaded on the
    Fe/Au bilayer in full (1e5 carriers, 500 steps of 1 fs), one replica per
    core on the spin valve (1e7 carriers in all, 100 steps after the pulse)
    and on the large bilayer (1e7 carriers in all, 50 steps after the pulse).
    Each replica's state is larger than the caches of its core."""
    out = {}
    out["single_thread_fe15_au100_full"] = oracle_replicas(0, 1e5, 0, 500, cores=1,
                                                           label="full workload, single thread")
    out["multicore_spin_valve_1e7_100_steps"] = oracle_replicas(1, 1e7, 300, 100,
                                                                label="1e7 carriers in all")
    out["multicore_large_1e7_50_steps"] = oracle_replicas(4, 1e7, 300, 50,
                                                          label="1e7 carriers in all")
    return out


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    wl, period, pre = workload(args)
    cores, scale, cap_each = cpu_sample(args, wl, pre)
    pool = OraclePool(args.config, scale, cores, pre + period * (args.warmup + args.steps) + 1)
    try:
        pool.step(pre)
        for _ in range(args.warmup):
            pool.step(period)
        t = time.perf_counter()
        ps = 0
        for _ in range(args.steps):
            ps += pool.step(period)
        dt = time.perf_counter() - t
    finally:
        pool.close()
    value = ps / dt
    sample = ("%d oracle replicas (one per core) of %s scaled by %g (capacity %d each), "
              "%d pre-roll steps, %d warm-up and %d timed steps of %d time steps"
              % (cores, wl.name, scale, cap_each, pre, args.warmup, args.steps, period))
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic", "config": config_dict(wl, period, pre, args), "impl": "reference",
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# adjoint leg: time(pic_grad) / time(pic_step) over the same run
# ---------------------------------------------------------------------------
def adjoint_leg(args):
    """The Fe(15 nm)/Au(100 nm) workload with 1e7 carriers (capacity 5e7, 800
    steps of 1 fs, densities every step): forward run, then the gradient of
    O1 + O2 with respect to the lifetime and transmittance tables, where O1 =
    sum over windows and cells 90..99 of (n_up - n_down) and O2 = sum over
    windows of (J_up - J_down) at face 15."""
    import torch
    from paper_1807_04733_gb300 import pic
    from paper_1807_04733_gb300 import workloads as W
    wl = W.config(3, scale=args.adjoint_scale)
    ctx = pic.Context(wl)
    stream = ctx.stream
    nc, n_out, _ = ctx.shape(0)
    gn = torch.zeros((1, n_out, 2, wl.n_e, nc), dtype=torch.float32, device="cuda")
    gJ = torch.zeros((1, n_out, 2, nc + 1), dtype=torch.float32, device="cuda")
    gn[0, :, 0, :, 90:100] = 1.0
    gn[0, :, 1, :, 90:100] = -1.0
    gJ[0, :, 0, 15] = 1.0
    gJ[0, :, 1, 15] = -1.0
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    torch.cuda.synchronize()
    pic.pic_profile(ctx.ctx, True)
    ev[0].record(stream)
    ctx.step(wl.n_steps)
    ev[1].record(stream)
    torch.cuda.synchronize()
    fwd_ms = ev[0].elapsed_time(ev[1])
    kf = pic.pic_profile_read(ctx.ctx)
    pic.pic_profile(ctx.ctx, False)
    led = ctx.ledger(0)
    times = []
    for i in range(2):          # the first call also allocates the replay buffers
        if i == 1:
            pic.pic_profile(ctx.ctx, True)
        ev[2].record(stream)
        g_tau, g_T = ctx.grad(gn, gJ)
        ev[3].record(stream)
        torch.cuda.synchronize()
        times.append(ev[2].elapsed_time(ev[3]))
    kt = pic.pic_profile_read(ctx.ctx)
    pic.pic_profile(ctx.ctx, False)
    grad_ms = times[-1]
    out = {"workload": "fe15_au100 (1e7 carriers, capacity 5e7, 800 x 1 fs, densities every step)"
                       if args.adjoint_scale == 1.0 else "fe15_au100 scaled by %g" % args.adjoint_scale,
           "observable": "O1 + O2 (spin density, cells 90..99; spin flux, face 15)",
           "forward_ms": fwd_ms, "grad_ms": grad_ms, "grad_ms_first_call": times[0],
           "ratio": grad_ms / fwd_ms, "particle_steps": led["particle_steps"],
           "forward_kernel_ms": {k: v[1] for k, v in kf.items() if not k.startswith("adjoint")},
           "grad_kernel_ms": {k: v[1] for k, v in kt.items() if k.startswith("adjoint")},
           "replay_launch_config": {k: v for k, v in ctx.launch_config().items() if "adj" in k},
           "grad_tau_abs_sum": float(g_tau.abs().sum()), "grad_T_abs_sum": float(g_T.abs().sum())}
    ctx.close()
    return out


# ---------------------------------------------------------------------------
# batched leg: one context for 64 stacks, graph-replayed steps, against 64
# one-stack contexts stepped one after another with single launches
# ---------------------------------------------------------------------------
def batched_leg(args):
    """64 Fe(15 nm)/Au(round U[20,200] nm) stacks, P and AP emitters
    alternating, N ~ logU[1e5, 1e7] per stack (sum ~1.4e8), capacity 4N,
    tables perturbed by +-20 % per stack, 1 fs steps, densities every step."""
    import torch
    from paper_1807_04733_gb300 import pic
    from paper_1807_04733_gb300 import workloads as W
    wl = W.config(2, scale=args.batched_scale)
    n = args.batched_steps or wl.n_steps
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]

    # launch configuration: tuned on a scratch context of the same stacks
    # after the pulse window, then used for the timed one
    tune = {}
    if not args.no_autotune:
        scratch = pic.Context(wl, n_steps_max=200 + 200 * 2)
        scratch.step(200)
        trials = scratch.autotune(2)
        cfg = scratch.launch_config()
        best = [t for t in trials if t["chosen"]][0]
        tune = {"trials": len(trials), "chosen": best}
        scratch.close()
        ctx = pic.Context(wl, use_graph=True, blocks_per_sm=best["blocks_per_sm"],
                          ring_stages=best["ring_stages"], hist_mode=best["hist_mode"],
                          consumer_warps=best["consumer_warps"])
    else:
        ctx = pic.Context(wl, use_graph=True)
    torch.cuda.synchronize()
    ev[0].record(ctx.stream)
    ctx.step(n)
    ev[1].record(ctx.stream)
    torch.cuda.synchronize()
    ms_b = ev[0].elapsed_time(ev[1])
    launches_b = ctx.launches
    ps_b = sum(ctx.ledger(s)["particle_steps"] for s in range(len(wl.stacks)))
    ctx.close()

    # the same stacks, each 50-step period one persistent cooperative launch
    # (replayed from a graph)
    pctx = pic.Context(wl, use_graph=2)
    torch.cuda.synchronize()
    ev[0].record(pctx.stream)
    pctx.step(n)
    ev[1].record(pctx.stream)
    torch.cuda.synchronize()
    ms_p = ev[0].elapsed_time(ev[1])
    launches_p = pctx.launches
    ps_p = sum(pctx.ledger(s)["particle_steps"] for s in range(len(wl.stacks)))
    pctx.close()

    singles = [pic.Context(wl.replace(stacks=[st])) for st in wl.stacks]
    torch.cuda.synchronize()
    ev[0].record(singles[0].stream)
    launches_s = 0
    for c in singles:
        c.step(n)
        launches_s += c.launches
    ev[1].record(singles[0].stream)
    torch.cuda.synchronize()
    ms_s = ev[0].elapsed_time(ev[1])
    ps_s = sum(c.ledger(0)["particle_steps"] for c in singles)
    for c in singles:
        c.close()
    return {"workload": "64 x Fe(15nm)/Au(20-200nm), sum n0 %d, %d x %g fs, densities every step"
                        % (sum(st.n0 for st in wl.stacks), n, wl.dt),
            "batched_graph_ms": ms_b, "sequential_plain_ms": ms_s, "speedup": ms_s / ms_b,
            "batched_particle_steps_per_s": ps_b / (ms_b * 1e-3),
            "sequential_particle_steps_per_s": ps_s / (ms_s * 1e-3),
            "batched_launches": launches_b, "sequential_launches": launches_s,
            "persistent_ms": ms_p, "persistent_speedup": ms_s / ms_p,
            "persistent_particle_steps_per_s": ps_p / (ms_p * 1e-3),
            "persistent_launches": launches_p,
            "autotune": tune}


# ---------------------------------------------------------------------------
# roofline of the step kernels and timed legs of other configurations
# ---------------------------------------------------------------------------
def roofline_of(delta, ktimes, ms, fused=False):
    """The step kernels: the streaming pass (k_stream), the event pass
    (k_event) and the placement of secondaries (k_place), or, fused (the
    ordinary steps of a context whose launch configuration has the general
    step inside the streaming pass), k_stream and k_place; one launch of each
    per time step, timed together with CUDA events on the context stream;
    "per launch" = per time step."""
    peak, peak_kind = measured_peak()
    n_k = ktimes["step"][0] + ktimes["step_moments"][0]
    k_ms = ktimes["step"][1] + ktimes["step_moments"][1] + ktimes["step_events"][1]
    if not n_k or not k_ms:
        return None
    alg = B_STEP * delta["particle_steps"] + B_EVENTFUL * delta["eventful"] + \
        B_CHANGED * delta["changed"] + B_SPAWN * delta["spawned"]
    strict = S_STEP * delta["particle_steps"] + S_EVENTFUL * delta["eventful"] + \
        S_CHANGED * delta["changed"] + S_SPAWN * delta["spawned"]
    achieved = (alg / n_k) / (k_ms / n_k * 1e-3) / 1e9
    achieved_s = (strict / n_k) / (k_ms / n_k * 1e-3) / 1e9
    traffic = None
    form = "fused" if fused else "separate"
    if NCU_TRAFFIC.get(form) and NCU_TRAFFIC.get("src_sha") == kernel_sha():
        traffic = NCU_TRAFFIC[form] * delta["particle_steps"] / n_k
    kernel = ("k_stream (general step inside) + k_place; density steps k_stream+k_event+k_place"
              if fused else "k_stream+k_event+k_place")
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": traffic, "kernel": kernel, "form": form,
            "peak_source": peak_kind,
            "byte_count": "per carrier-step 20 B (16 B read, z written) + 12 B per eventful "
                          "carrier + 16 B per placed secondary",
            "algorithmic_bytes_per_launch": alg / n_k,
            "strict": {"byte_count": "per carrier-step 16 B (z, mu, packed read, z written) + "
                                     "8 B per changed record + 16 B per placed secondary",
                       "bytes_per_launch": strict / n_k, "achieved": achieved_s,
                       "frac": achieved_s / peak},
            "avg_launch_ms": k_ms / n_k,
            "kernel_share_of_step_time": k_ms / ms if ms else 0}


def saturation(delta):
    tot = delta["spawned"] + delta["spawn_dropped"]
    return {"spawned": delta["spawned"], "spawn_dropped": delta["spawn_dropped"],
            "dropped_fraction": delta["spawn_dropped"] / tot if tot else 0.0}


def timed_leg(wl, pre, n_timed, chunk, capacity=None, autotune_steps=0):
    """A context of `wl`: `pre` untimed steps (the pulse window), the
    autotuner, then n_timed steps timed with CUDA events and per-kernel
    events; particle-steps/s over the timed steps and the step kernels'
    roofline."""
    import torch
    from paper_1807_04733_gb300 import pic
    n_max = pre + 200 * autotune_steps + n_timed + 1
    ctx = pic.Context(wl, n_steps_max=max(wl.n_steps, n_max), capacity=capacity)
    left = pre
    while left > 0:
        k = min(left, 100)
        ctx.step(k)
        left -= k
    tune = None
    if autotune_steps:
        trials = ctx.autotune(autotune_steps)
        tune = {"trials": len(trials), "chosen": [t for t in trials if t["chosen"]][0]}
    S = len(wl.stacks)
    led0 = [ctx.ledger(s) for s in range(S)]
    torch.cuda.synchronize()
    pic.pic_profile(ctx.ctx, True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(ctx.stream)
    left = n_timed
    while left > 0:
        k = min(left, chunk)
        ctx.step(k)
        left -= k
    e1.record(ctx.stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    kt = pic.pic_profile_read(ctx.ctx)
    pic.pic_profile(ctx.ctx, False)
    led1 = [ctx.ledger(s) for s in range(S)]
    delta = {k: sum(b[k] - a[k] for a, b in zip(led0, led1)) for k in led1[0]}
    lcfg = ctx.launch_config()
    out = {"value": delta["particle_steps"] / (ms * 1e-3), "unit": UNIT, "ms": ms,
           "time_steps": n_timed,
           "roofline": roofline_of(delta, kt, ms, fused=lcfg["grid_step_fused"] > 0),
           "saturation": saturation(delta), "ledger_delta": delta,
           "kernel_ms": {k: v[1] for k, v in kt.items() if v[0]},
           "launch_config": ctx.launch_config(), "autotune": tune}
    ctx.close()
    return out


def unsaturated_leg(args):
    """The large bilayer with its capacity raised to 2^30 slots (the most a
    stack holds; the cascade fills even these by about 750 time steps):
    after the pulse window, 300 time steps timed while every secondary is
    placed."""
    from paper_1807_04733_gb300 import workloads as W
    wl = W.config(4, scale=args.scale)
    cap = (1 << 30) - 1024
    pre = int(math.ceil(2 * wl.stacks[0].t0 / wl.dt))
    out = timed_leg(wl, pre, 300, 50, capacity=cap)
    out["workload"] = "%s with capacity %d, time steps %d..%d" % (wl.name, cap, pre, pre + 300)
    return out


def spin_valve_legs(args):
    """The Fe(10)/Au(50)/Fe(10) spin valve, parallel and antiparallel (1e7
    carriers, capacity 5e7, 0.5 fs, densities and fluxes every step): after
    the pulse window, 200 time steps timed, tuned by the autotuner."""
    from paper_1807_04733_gb300 import workloads as W
    out = {}
    for ap in (False, True):
        wl = W.spin_valve(ap, n0=int(1e7 * args.spin_valve_scale),
                          capacity=int(5e7 * args.spin_valve_scale))
        pre = int(math.ceil(2 * wl.stacks[0].t0 / wl.dt))
        leg = timed_leg(wl, pre, 200, 50, autotune_steps=0 if args.no_autotune else 2)
        leg["workload"] = "%s: n0 %d, capacity %d, time steps %d..%d" % (
            wl.name, wl.stacks[0].n0, wl.stacks[0].capacity, pre, pre + 200)
        out[wl.name] = leg
    return out


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def main():
    args = parse()
    if args.impl == "reference":
        return reference_arm(args)

    import torch
    from paper_1807_04733_gb300 import pic

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()

    wl, period, pre = workload(args)
    # replicas: every rank runs its own copy with its own seed (weak scaling)
    wl = wl.replace(seed=wl.seed + rank)
    tune_steps = 0 if args.no_autotune else args.autotune_steps
    total = pre + 200 * tune_steps + period * (args.warmup + 3 * args.steps) + 1
    ctx = pic.Context(wl, n_steps_max=max(wl.n_steps, total), blocks_per_sm=args.blocks_per_sm,
                      hist_mode=args.hist_mode, ring_stages=args.ring, event_pass=args.event_pass,
                      use_graph=bool(args.graph))
    stream = ctx.stream
    # set-up: the pulse window (inputs resident in HBM before timing)
    left = pre
    while left > 0:
        n = min(left, 100)
        ctx.step(n)
        left -= n
    # launch configuration: timed candidates on the running simulation
    tune = None
    if tune_steps:
        trials = ctx.autotune(tune_steps)
        tune = {"trials": len(trials), "chosen": [t for t in trials if t["chosen"]][0],
                "fastest_ns_per_particle_step": min(t["ns_per_particle_step"] for t in trials),
                "slowest_ns_per_particle_step": max(t["ns_per_particle_step"] for t in trials)}
    # whole periods from here on
    s_now = ctx.shape(0)[2]
    if s_now % period:
        ctx.step(period - s_now % period)
    for _ in range(args.warmup):
        ctx.step(period)
    led0 = [ctx.ledger(s) for s in range(len(wl.stacks))]

    # ---- device-timed region ----
    try:
        clk = Clocks("GPU-" + str(torch.cuda.get_device_properties(dev).uuid).replace("GPU-", ""))
    except Exception:
        clk = Clocks(str(dev))
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    clk.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    launches = 0
    for _ in range(args.steps):
        ctx.step(period)
        launches += ctx.launches
    e1.record(stream)
    torch.cuda.synchronize()
    clocks = clk.stop()
    ms = e0.elapsed_time(e1)
    led1 = [ctx.ledger(s) for s in range(len(wl.stacks))]
    if dist is not None:
        dist.barrier()
    delta = {k: sum(b[k] - a[k] for a, b in zip(led0, led1)) for k in led1[0]}
    ps = delta["particle_steps"]

    # ---- kernel breakdown: as many steps again, with CUDA events around
    # every launch (kept out of the timed region above) ----
    pic.pic_profile(ctx.ctx, True)
    ek0 = torch.cuda.Event(enable_timing=True)
    ek1 = torch.cuda.Event(enable_timing=True)
    ek0.record(stream)
    for _ in range(args.steps):
        ctx.step(period)
    ek1.record(stream)
    torch.cuda.synchronize()
    ms_k = ek0.elapsed_time(ek1)
    ktimes = pic.pic_profile_read(ctx.ctx)
    pic.pic_profile(ctx.ctx, False)
    led2 = [ctx.ledger(s) for s in range(len(wl.stacks))]
    delta_k = {k: sum(b[k] - a[k] for a, b in zip(led1, led2)) for k in led2[0]}

    # ---- end-to-end region: the C-ABI with host buffers, every step the
    # window just finished (densities and fluxes) and the ledger read back
    # into pinned host memory ----
    nc, no, _ = ctx.shape(0)
    n_host = torch.empty((2, wl.n_e, nc), dtype=torch.int32, pin_memory=True)
    J_host = torch.empty((2, nc + 1), dtype=torch.int32, pin_memory=True)
    torch.cuda.synchronize()
    t = time.perf_counter()
    ps_e2e = 0
    for _ in range(args.steps):
        ctx.step(period)
        w = ctx.shape(0)[2] // wl.moment_every - 1
        led = pic.pic_moment_window(ctx.ctx, 0, w, n_host.data_ptr(), J_host.data_ptr())
        ps_e2e = led["particle_steps"]
    e2e_s = time.perf_counter() - t
    ev_e2e = led["eventful"] - led2[0]["eventful"] if args.steps else 0
    ps_e2e -= led2[0]["particle_steps"]
    d2h = n_host.numel() * 4 + J_host.numel() * 4 + 13 * 8
    # the run's inputs (tables, excitation) are host buffers copied once by
    # pic_init / pic_excite; a step has no inputs of its own
    h2d_once = sum(t_.v.nbytes + t_.tau_in.nbytes + t_.tau_el.nbytes + t_.T.nbytes + t_.p0.nbytes
                   for t_ in ctx._tabs)

    # ---- reductions over ranks: the largest time, the sum of the units ----
    from paper_1807_04733_gb300 import shard
    ms_max, ps_all = shard.reduce_measurement(ms, float(ps), dist, "cuda")
    e2e_ms, ps_e2e_all = shard.reduce_measurement(e2e_s * 1e3, float(ps_e2e), dist, "cuda")

    roofline = roofline_of(delta_k, ktimes, ms_k, fused=ctx.launch_config()["grid_step_fused"] > 0)

    line = {
        "metric": METRIC, "value": ps_all / (ms_max * 1e-3), "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": config_dict(wl, period, pre, args),
        # the buffer is full in the timed window: most secondaries are
        # dropped and counted (the "unsaturated" leg places them all)
        "saturation": saturation(delta),
        "roofline": roofline,
        "e2e": {"value": ps_e2e_all / (e2e_ms * 1e-3), "unit": UNIT,
                "h2d_bytes_per_step": 0, "d2h_bytes_per_step": d2h,
                "h2d_bytes_once": h2d_once,
                # eventful carriers per carrier-step here (ledger_delta gives the
                # timed region's): the state relaxes as the run goes on
                "eventful_fraction": ev_e2e / ps_e2e if ps_e2e else None,
                "note": "pic_step then pic_moment_window into pinned host buffers every step; "
                        "the tables and the excitation are the run's only inputs, copied from "
                        "host buffers once (pic_init, pic_excite)"},
        "gpu_launches": launches,
        "clocks": clocks,
        "ledger_delta": delta,
        "kernel_ms": {k: v[1] for k, v in ktimes.items()},
        "kernel_launches": {k: v[0] for k, v in ktimes.items()},
        "launch_config": ctx.launch_config(),
        "autotune": tune,
    }
    ctx.close()
    if rank == 0 and world == 1 and not args.no_unsaturated and args.config == 4:
        line["unsaturated"] = unsaturated_leg(args)
    if rank == 0 and world == 1 and not args.no_spin_valve:
        line["spin_valve"] = spin_valve_legs(args)
    if rank == 0 and world == 1 and not args.no_adjoint:
        line["adjoint"] = adjoint_leg(args)
    if rank == 0 and world == 1 and not args.no_batched:
        line["batched"] = batched_leg(args)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        base = run_cpu_baselines()
        line["cpu_baseline"] = base["multicore_large_1e7_50_steps"]
        line["cpu_baselines"] = base
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
