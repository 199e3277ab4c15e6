"""Benchmark of the QuadSwarm forward-dynamics step on GB300.

One benchmark step = one 100 Hz control step of every drone of the plain
workload (8192 envs x 1 quadrotor, per-env randomisation, room contacts,
motor and sensor noise, goal-reaching reward), i.e. one qs_step call. The
metric is quadrotor-steps/s (the paper's "simulation samples per second",
Sec. IV). Inputs (the per-step command stream) are resident in device memory
before the timed region; L2 is flushed between timed steps and each step is
timed with CUDA events on the handle's stream.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl {gpu,reference}]

--impl reference times the FP64 CPU oracle (the only reference this build
has) on the host cores for the same workload and metric.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2306_09537_gb300 import workloads as W  # noqa: E402

METRIC = "quadrotor-steps/sec on 1 GB300 (plain vs batched vs fwd+adjoint), % of roofline"
# DRAM bytes (read + write) of one launch of the headline kernel on the plain
# 8192 x 1 step, from an ncu capture of this command (L2 flushed before the
# launch), and the SHA-256 of the library sources that capture was taken on:
# once the kernel sources change, the figure no longer describes the kernel
# and the roofline's traffic is reported as null until it is captured again.
HEADLINE_DRAM = {"bytes_per_launch": 1780395,
                 "sources_sha256": "d4a37949436b2a4969b4400bbbeba4aa2d0500f79455aff8a89730820f0e438b",
                 "source": "profiles/k_step_ws_plain_8192x1.md (ncu dram__bytes_read.sum + dram__bytes_write.sum)"}
UNIT = "quadrotor-steps/s"
WL = W.PLAIN
BENCH_FEATURES = WL.features + ("auto_reset",)
L2_FLUSH_BYTES = 256 << 20


def library_sources_sha256() -> str:
    """SHA-256 over the CUDA sources and the public header of the library."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2306_09537_gb300", "csrc")
    for f in sorted(os.listdir(csrc)) + ["../../include/qs.h"]:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(f.encode() + b"\0" + fh.read())
    return h.hexdigest()


def headline_traffic():
    """(bytes per launch or None, note) for the roofline's traffic field."""
    cur = library_sources_sha256()
    if HEADLINE_DRAM["sources_sha256"] == cur:
        return HEADLINE_DRAM["bytes_per_launch"], HEADLINE_DRAM["source"]
    return None, f"kernel sources changed since the ncu capture ({HEADLINE_DRAM['source']}); sources sha256 {cur[:16]}"


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the platform)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part")):
                    return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), float(p.get("sm_max_mhz", 2070.0)), "measured"
    except Exception:
        return 6800.0, 2070.0, "fallback"


# Algorithmic cost of one quadrotor-step of the per-call form (state in HBM
# between calls); see the design notes for the derivation.
def algorithmic_bytes(D, E, obs_dim):
    per_drone = 2 * 120 + 16 + 4 * obs_dim + 4 + 4          # state r+w, action, obs, reward, events
    per_env = 7 * 4 + 3 * 4 + 2 * 4 + 2 * 4 + 1               # params, goal, episode step r+w, tick r+w, done
    return D * per_drone + E * per_env


OPS_PER_QUAD_STEP_N1 = 1080  # FP32/INT32 lane operations, 2 substeps, N = 1 (derivation in the design notes)


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.lines = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def wait_samples(self, n, timeout=5.0):
        """Blocks until n more samples have arrived (or the timeout)."""
        if not self.proc:
            return
        target, t_end = len(self.lines) + n, time.perf_counter() + timeout
        while len(self.lines) < target and time.perf_counter() < t_end:
            time.sleep(0.01)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup():
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def rank_seed(rank: int) -> int:
    """Each rank simulates its own envs (weak scaling, no data exchange)."""
    return WL.seed + 1000 * rank


def max_over_ranks(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# --------------------------------------------------------------------------- CPU oracle legs
def oracle_run(steps, n_envs=None, threads=None, seed=None):
    """Runs the oracle on the bench workload; returns (quad-steps/s, cores, sample)."""
    from oracle import oracle as O
    flags = 0
    names = {"dr": O.F_DR, "motor_noise": O.F_MOTOR_NOISE, "obs_noise": O.F_OBS_NOISE, "collisions": O.F_COLLISIONS,
             "floor": O.F_FLOOR, "walls": O.F_WALLS, "auto_reset": O.F_AUTO_RESET}
    for f in BENCH_FEATURES:
        flags |= names[f]
    E = n_envs or WL.n_envs
    oc = O.default_config(n_envs=E, k_neighbors=WL.k_neighbors, flags=flags, seed=seed or WL.seed)
    oc.w[:] = [0.0] * 14
    O.set_config(oc, weights=WL.weights)
    o = O.Oracle(oc)
    o.reset(seed or WL.seed)
    period = min(steps, 100)
    acts = W.actions(WL.seed, period, o.D).astype(np.float64)
    cores = threads or os.cpu_count() or 1
    t0 = time.perf_counter()
    for t in range(steps):
        o.step(acts[t % period], n_threads=cores)
    dt = time.perf_counter() - t0
    return o.D * steps / dt, cores, f"{E} envs x {steps} control steps of the plain workload, binary64, {cores} threads"


def cpu_baseline_legs():
    """The oracle on all host cores (the whole 1000-step plain workload) and on
    one core (its first 200 steps), about 10-20 s of CPU work together, with
    the host's core count and CPU model."""
    v, cores, sample = oracle_run(1000)
    v1, _, sample1 = oracle_run(200, threads=1)
    return {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
            "single_thread": {"value": v1, "unit": UNIT, "cores": 1, "sample": sample1},
            "nproc": os.cpu_count(), "cpu_model": cpu_model()}


def run_reference(args, world, rank):
    if rank != 0:
        return
    # each bench step = one control step of all 8192 envs on the oracle
    from oracle import oracle as O  # noqa: F401
    oracle_run(max(1, args.warmup))
    v, cores, sample = oracle_run(args.steps)
    line = {"metric": METRIC, "value": v, "unit": UNIT, "impl": "reference", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": WL.n_envs / v * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WL.name, "n_envs": WL.n_envs, "swarm": 1, "k_neighbors": WL.k_neighbors,
                       "features": list(BENCH_FEATURES)},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                             "nproc": os.cpu_count(), "cpu_model": cpu_model()},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- GPU leg
def run_gpu(args, world, rank, local):
    import torch

    from paper_2306_09537_gb300 import qs
    from paper_2306_09537_gb300.env import QuadSwarmEnv
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(device=dev)
    seed = rank_seed(rank)
    with torch.cuda.stream(stream):
        env = QuadSwarmEnv(WL.n_envs, 1, WL.k_neighbors, BENCH_FEATURES, seed=seed, weights=WL.weights, device=dev,
                           stream=stream)
        env.reset(seed)
        steps, warm = args.steps, args.warmup
        period = min(steps + warm, 1000)
        acts = torch.from_numpy(W.actions(seed, period, env.D)).to(dev)
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
        n_classes = 1
        ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        # the clock samples (every 100 ms) span the warm-up, the timed region
        # and one sample after it, since a short timed region may fall between
        # two samples
        with ClockSampler(local) as clk:
            clk.wait_samples(1)
            # warm-up: the timed loop itself (flush, step) for at least W steps
            # and at least --warmup-seconds (0.5 s), so that clocks, the host
            # path and the GPU's front end are in their steady state when
            # timing starts
            t_warm, n_warm = time.perf_counter() + args.warmup_seconds, 0
            while n_warm < warm or time.perf_counter() < t_warm:
                flush.zero_()
                env.step(acts[n_warm % period])
                n_warm += 1
                if n_warm % 64 == 0:
                    stream.synchronize()
            stream.synchronize()
            barrier(world)
            torch.cuda.synchronize()
            t_wall = time.perf_counter()
            # a short device-side pause ahead of the first timed step lets the
            # host enqueue the timed steps before the GPU reaches them: each
            # event pair then times the GPU's step, never a GPU idling on the
            # host's launch of the next call
            if hasattr(torch.cuda, "_sleep"):
                torch.cuda._sleep(4_000_000)
            for t in range(steps):
                flush.zero_()
                ev0[t].record(stream)
                env.step(acts[(n_warm + t) % period])
                ev1[t].record(stream)
            stream.synchronize()
            t_wall = time.perf_counter() - t_wall
            barrier(world)
            torch.cuda.synchronize()
            clk.wait_samples(1)
        per = np.array([a.elapsed_time(b) for a, b in zip(ev0, ev1)])  # ms
        total_ms = max_over_ranks(float(per.sum()), world)
        env.sync()

        # end to end, synchronous host loop: each step's commands read by the
        # GPU from page-locked host memory (a ring of 64 command slots), the
        # step posted, its observation, reward and done written to page-locked
        # host memory and read there. Through the resident server
        # (qs_serve_step) and, for comparison, the per-call host-buffer step
        # (qs_step_host) on the same ring.
        ring = W.actions(seed + 1, 64, env.D)
        e2e_steps = min(steps, 500)
        if not args.no_e2e:
            # ranks align before serving: a collective enqueued behind the
            # resident launch would wait until the server retires
            barrier(world)
            check, e2e_local = 0.0, None
            try:
                srv = env.serve(slots=64)
            except qs.QSError as ex:  # no native atomics on host memory: the per-call form only
                if ex.status != qs.QS_ERR_UNSUPPORTED:
                    raise
                srv = None
            if srv is not None:
                srv.slots.copy_(torch.from_numpy(ring))
                r_np = srv.reward.numpy()
                for t in range(3):
                    qs.qs_serve_step(env.h, t % 64)
                t0 = time.perf_counter()
                for t in range(e2e_steps):
                    qs.qs_serve_step(env.h, t % 64)
                    check += float(r_np[0])
                e2e_local = time.perf_counter() - t0
                srv.close()
            a_host = torch.from_numpy(ring).pin_memory()
            obs_h = torch.empty(env.D, env.obs_dim).pin_memory()
            rew_h = torch.empty(env.D).pin_memory()
            done_h = torch.empty(env.E, dtype=torch.uint8).pin_memory()
            for t in range(3):
                qs.qs_step_host(env.h, a_host[t % 64], obs_h, rew_h, done_h)
            barrier(world)
            t0 = time.perf_counter()
            for t in range(e2e_steps):
                qs.qs_step_host(env.h, a_host[t % 64], obs_h, rew_h, done_h)
                check += float(rew_h[0])
            e2e_host_s = max_over_ranks(time.perf_counter() - t0, world)
            # every rank makes the same collective calls; the server's figure only if every rank served
            served = -max_over_ranks(-(1.0 if e2e_local is not None else 0.0), world) > 0.5
            e2e_srv = max_over_ranks(e2e_local if e2e_local is not None else 0.0, world)
            e2e_s = e2e_srv if served else e2e_host_s

    D, E, od = env.D, env.E, env.obs_dim
    value = world * D * steps / (total_ms * 1e-3)
    hbm, sm_max, src = peaks()
    launch_s = float(per.mean()) * 1e-3
    ab = algorithmic_bytes(D, E, od)
    ach_gbs = ab / launch_s / 1e9
    ops = OPS_PER_QUAD_STEP_N1 * D
    n_sm = torch.cuda.get_device_properties(torch.device("cuda", local)).multi_processor_count
    alu_peak = n_sm * 128 * sm_max * 1e6 / 1e9  # G lane-ops/s
    ach_gops = ops / launch_s / 1e9
    t_hbm, t_alu = ab / (hbm * 1e9), ops / (alu_peak * 1e9)
    if t_hbm >= t_alu:
        roof = {"bound": "hbm", "achieved": ach_gbs, "peak": hbm, "unit": "GB/s", "frac": ach_gbs / hbm,
                "peak_source": f"{src} MEASURED_PEAKS.json hbm_gbs" if src == "measured" else "fallback 6.8 TB/s"}
    else:
        roof = {"bound": "alu", "achieved": ach_gops, "peak": alu_peak, "unit": "Gop/s", "frac": ach_gops / alu_peak,
                "peak_source": f"{n_sm} SMs x 128 FP32/INT32 lanes x max SM clock"}
    traffic, traffic_src = headline_traffic()
    roof.update({"kernel": "qsk::k_step_ws<false>", "traffic": traffic, "traffic_source": traffic_src,
                 "algorithmic_bytes_per_launch": ab,
                 "algorithmic_ops_per_launch": ops,
                 "alt": {"hbm_frac": ach_gbs / hbm, "alu_frac": ach_gops / alu_peak}})
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps, "warmup": warm,
            "ms_per_step": total_ms / steps, "ms_per_step_median": float(np.median(per)),
            "ms_per_step_p90": float(np.quantile(per, 0.9)), "warmup_steps_run": n_warm,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": WL.name, "n_envs": WL.n_envs, "swarm": 1, "k_neighbors": WL.k_neighbors,
                       "features": list(BENCH_FEATURES), "form": "per-call qs_step, state in HBM",
                       "l2": "flushed between timed steps (256 MiB write)", "parallelism": f"replicas x{world}"},
            "e2e": None if args.no_e2e else {
                "value": world * D * e2e_steps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": D * 16,
                "d2h_bytes_per_step": D * od * 4 + D * 4 + E,
                "api": "qs_serve_step (resident server)" if served else "qs_step_host (no native host atomics)",
                "us_per_step": e2e_s / e2e_steps * 1e6,
                "qs_step_host": {"value": world * D * e2e_steps / e2e_host_s,
                                 "us_per_step": e2e_host_s / e2e_steps * 1e6}},
            "gpu_launches": steps * n_classes, "roofline": roof,
            "clocks": clk.summary(), "wall_s_timed": t_wall}
    env.close()
    return line


def _events_ms(fn, stream, reps=3, flush=None):
    import torch
    out = []
    for _ in range(reps):
        if flush is not None:
            flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        out.append(a.elapsed_time(b))
    return float(np.median(out))


def rollout_bytes(D, E, obs_dim):
    """Algorithmic bytes per quadrotor-step of the batched form (state stays on chip)."""
    return D * (16 + 4 * obs_dim + 4) + E * 1


def run_forms(dev, stream, seed):
    """The batched, swarm, uneven and env-count-sweep forms (extra keys)."""
    import torch

    from paper_2306_09537_gb300 import autotune, qs
    from paper_2306_09537_gb300.env import QuadSwarmEnv
    hbm, sm_max, _ = peaks()
    alu_peak = torch.cuda.get_device_properties(dev).multi_processor_count * 128 * sm_max * 1e6
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    forms = {}
    with torch.cuda.stream(stream):
        def make(wl, n_envs=None, feats=None, scenarios=()):
            sizes = wl.sizes() if n_envs is None else np.full(n_envs, wl.swarm, np.int32)
            env = QuadSwarmEnv(len(sizes), sizes if wl.swarm is None else wl.swarm, wl.k_neighbors,
                               feats or (wl.features + ("auto_reset",)), seed=seed, weights=wl.weights, device=dev,
                               stream=stream, scenarios=scenarios)
            env.reset(seed)
            return env

        def per_call(env, acts, steps):
            for t in range(3):
                env.step(acts[t % acts.shape[0]])
            tot = 0.0
            for t in range(steps):
                tot += _events_ms(lambda: env.step(acts[t % acts.shape[0]]), stream, reps=1, flush=flush)
            return tot / steps

        def rollout(env, acts, T, reps=3):
            obs = torch.empty(T, env.D, env.obs_dim, device=dev)
            rew = torch.empty(T, env.D, device=dev)
            done = torch.empty(T, env.E, dtype=torch.uint8, device=dev)
            env.rollout(acts[:T], obs, rew, done)  # capture + warm
            ms = _events_ms(lambda: env.rollout(acts[:T], obs, rew, done), stream, reps=reps, flush=flush) / T
            del obs, rew, done
            return ms

        # plain 8192 x 1: batched rollout of the 1000-step episode chunk
        env = make(W.PLAIN)
        tuned = autotune.tune(env, horizon=1000)
        acts = torch.from_numpy(W.actions(seed, 1000, env.D)).to(dev)
        ms = rollout(env, acts, 1000)
        forms["plain_rollout"] = {"value": env.D / ms * 1e3, "ms_per_step": ms, "T": 1000,
                                  "shape": list(tuned["rollout"]), "launches_per_rollout":
                                  -(-1000 // (tuned["rollout"][1] or 1000))}
        env.close()
        del acts

        # swarm 2048 x 8, K = 6: per-call and batched
        env = make(W.SWARM)
        tuned = autotune.tune(env, horizon=500)
        acts = torch.from_numpy(W.actions(seed, 500, env.D)).to(dev)
        ms_call = per_call(env, acts, 300)
        ms_roll = rollout(env, acts, 500)
        forms["swarm_call"] = {"value": env.D / ms_call * 1e3, "ms_per_step": ms_call}
        forms["swarm_rollout"] = {"value": env.D / ms_roll * 1e3, "ms_per_step": ms_roll, "T": 500,
                                  "shape": list(tuned["rollout"])}
        env.close()
        del acts

        # swarm 2048 x 8 with every training scenario (per-drone goals, Sec. III-D), and with downwash
        for name, kw in (("swarm_scenarios", dict(scenarios=tuple(qs.SCENARIOS))),
                         ("swarm_downwash", dict(feats=W.SWARM.features + ("auto_reset", "downwash")))):
            env = make(W.SWARM, **kw)
            tuned = autotune.tune(env, horizon=500)
            acts = torch.from_numpy(W.actions(seed, 500, env.D)).to(dev)
            ms_call = per_call(env, acts, 300)
            ms_roll = rollout(env, acts, 500)
            forms[name + "_call"] = {"value": env.D / ms_call * 1e3, "ms_per_step": ms_call}
            forms[name + "_rollout"] = {"value": env.D / ms_roll * 1e3, "ms_per_step": ms_roll, "T": 500,
                                        "shape": list(tuned["rollout"])}
            env.close()
            del acts

        # uneven swarms, 4096 envs, sizes {1..64}: the batched rollout, the per-call
        # step (one launch for every width class), and the baseline of per-size
        # launches: the same envs in one handle per width class, one launch each
        env = make(W.UNEVEN)
        tuned = autotune.tune(env, horizon=256)
        acts = torch.from_numpy(W.actions(seed, 256, env.D)).to(dev)
        ms_roll = rollout(env, acts, 256)
        ms_call = per_call(env, acts, 256)
        sizes = W.UNEVEN.sizes()
        wcls = np.array([1 if n == 1 else 1 << int(np.ceil(np.log2(n))) for n in sizes])
        parts = []
        for w in sorted(set(wcls.tolist())):
            sel = sizes[wcls == w]
            e = QuadSwarmEnv(len(sel), sel, W.UNEVEN.k_neighbors, W.UNEVEN.features + ("auto_reset",), seed=seed,
                             weights=W.UNEVEN.weights, device=dev, stream=stream)
            e.reset(seed)
            parts.append((e, torch.from_numpy(W.actions(seed, 1, e.D)).to(dev)[0]))

        def per_size():
            for e, a in parts:
                e.step(a)
        for _ in range(3):
            per_size()
        ms_ps = float(np.mean([_events_ms(per_size, stream, reps=1, flush=flush) for _ in range(100)]))
        for e, _ in parts:
            e.close()
        forms["uneven_batched"] = {"value": env.D / ms_roll * 1e3, "ms_per_step": ms_roll, "T": 256,
                                   "drones": env.D, "shape": list(tuned["rollout"])}
        forms["uneven_call"] = {"value": env.D / ms_call * 1e3, "ms_per_step": ms_call, "launches_per_step": 1}
        forms["uneven_per_size_launches"] = {"value": env.D / ms_ps * 1e3, "ms_per_step": ms_ps,
                                             "launches_per_step": len(parts)}
        forms["uneven_speedup_vs_per_size"] = ms_ps / ms_roll
        forms["uneven_call_speedup_vs_per_size"] = ms_ps / ms_call
        env.close()
        del acts

        # swarm size sweep at 32,768 drones, K = 6 (up to the paper's largest team,
        # N = 128): the O(N^2) pair pass per env; default launch shapes
        import dataclasses
        sweep = []
        for N in (8, 16, 32, 64, 128):
            env = make(dataclasses.replace(W.SWARM, n_envs=32768 // N, swarm=N))
            acts = torch.from_numpy(W.actions(seed, 200, env.D)).to(dev)
            ms_call = per_call(env, acts, 100)
            ms_roll = rollout(env, acts, 200)
            sweep.append({"swarm": N, "n_envs": env.E, "call": env.D / ms_call * 1e3, "rollout": env.D / ms_roll * 1e3,
                          "rollout_shape": list(qs.qs_get_rollout_shape(env.h))})
            env.close()
            del acts
        forms["swarm_size_sweep"] = sweep

        # differentiable rollout: 1024 x 8, T = 128, checkpoints every 16, smooth
        # contacts; and the same with the step's own (discrete) contacts
        wl = W.DIFF
        for name, feats in (("fwd_adjoint", wl.features),
                            ("fwd_adjoint_discrete", ("dr", "motor_noise", "floor", "walls", "collisions")),
                            ("fwd_adjoint_event_time",
                             ("dr", "motor_noise", "floor", "walls", "collisions", "event_time"))):
            env = QuadSwarmEnv(wl.n_envs, wl.swarm, wl.k_neighbors, feats, seed=seed, weights=wl.weights,
                               device=dev, stream=stream)
            env.reset(seed)
            T, C = wl.horizon, wl.ckpt_every
            x0 = env.get_state()["state"].contiguous()
            acts = torch.from_numpy(W.actions(seed, T, env.D, lo=0.05, hi=0.95)).to(dev)
            ws = torch.empty(qs.qs_diff_workspace_size(env.h, T, C), dtype=torch.uint8, device=dev)
            loss = torch.empty(env.D, device=dev)
            dl = torch.ones(env.D, device=dev)
            ga = torch.empty_like(acts)
            gx = torch.empty(env.D, 30, device=dev)

            def fwd():
                qs.qs_diff_forward(env.h, T, C, x0, acts, loss, ws)

            def fwd_bwd():
                fwd()
                qs.qs_diff_backward(env.h, T, C, acts, dl, ws, ga, gx)
            fwd_bwd()
            ms_f = _events_ms(fwd, stream, reps=3, flush=flush)
            ms_fb = _events_ms(fwd_bwd, stream, reps=3, flush=flush)
            forms[name] = {"value": env.D * T / ms_fb * 1e3, "ms_per_rollout": ms_fb, "T": T, "ckpt_every": C,
                           "drones": env.D, "forward_only_value": env.D * T / ms_f * 1e3,
                           "workspace_bytes": int(ws.numel()), "features": list(feats)}
            env.close()
            del acts, ws

        # drone-count sweep of the smooth fwd + adjoint (swarms of 8, T = 128,
        # checkpoints every 16): from latency-bound at 8,192 drones to full waves
        sweep = []
        for E in (1024, 8192, 32768):
            env = QuadSwarmEnv(E, wl.swarm, wl.k_neighbors, wl.features, seed=seed, weights=wl.weights,
                               device=dev, stream=stream)
            env.reset(seed)
            T, C = wl.horizon, wl.ckpt_every
            x0 = env.get_state()["state"].contiguous()
            acts = torch.from_numpy(W.actions(seed, T, env.D, lo=0.05, hi=0.95)).to(dev)
            ws = torch.empty(qs.qs_diff_workspace_size(env.h, T, C), dtype=torch.uint8, device=dev)
            loss = torch.empty(env.D, device=dev)
            dl = torch.ones(env.D, device=dev)
            ga = torch.empty_like(acts)
            gx = torch.empty(env.D, 30, device=dev)

            def fwd_bwd():
                qs.qs_diff_forward(env.h, T, C, x0, acts, loss, ws)
                qs.qs_diff_backward(env.h, T, C, acts, dl, ws, ga, gx)
            fwd_bwd()
            ms_fb = _events_ms(fwd_bwd, stream, reps=3, flush=flush)
            sweep.append({"drones": env.D, "value": env.D * T / ms_fb * 1e3, "ms_per_rollout": ms_fb,
                          "workspace_bytes": int(ws.numel())})
            env.close()
            del acts, ws, ga, gx
        forms["fwd_adjoint_sweep"] = sweep

        # env-count sweep of the batched plain form (1 drone per env)
        sweep = []
        for E in (8192, 65536, 262144, 1048576):
            env = make(W.PLAIN, n_envs=E)
            qs.qs_set_rollout_shape(env.h, 128, 0, True)
            T = 50
            acts = torch.from_numpy(W.actions(seed, T, env.D)).to(dev)
            ms = rollout(env, acts, T)
            s = ms * 1e-3
            ab = rollout_bytes(env.D, env.E, env.obs_dim)
            sweep.append({"n_envs": E, "value": env.D / s, "ms_per_step": ms,
                          "hbm_frac": ab / s / 1e9 / hbm,
                          "alu_frac": OPS_PER_QUAD_STEP_N1 * env.D / s / alu_peak})
            env.close()
            del acts
        forms["plain_rollout_sweep"] = sweep

        # env-count sweep of the per-call plain step (the headline form): from
        # latency-bound at 8192 drones to HBM-bound once the state outgrows L2
        sweep = []
        for E in (8192, 65536, 262144, 1048576):
            env = make(W.PLAIN, n_envs=E)
            acts = torch.from_numpy(W.actions(seed, 8, env.D)).to(dev)
            ms = per_call(env, acts, 20)
            s = ms * 1e-3
            ab = algorithmic_bytes(env.D, env.E, env.obs_dim)
            sweep.append({"n_envs": E, "value": env.D / s, "ms_per_step": ms, "hbm_frac": ab / s / 1e9 / hbm,
                          "alu_frac": OPS_PER_QUAD_STEP_N1 * env.D / s / alu_peak})
            env.close()
            del acts
        forms["plain_call_sweep"] = sweep
    return forms


def profile_case(name, local):
    """One small case of a form, for ncu captures (a few hundred MB on device)."""
    import torch

    from paper_2306_09537_gb300 import qs
    from paper_2306_09537_gb300.env import QuadSwarmEnv
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(stream):
        if name == "rollout":  # 65536 single-drone envs, 32-step rollouts
            env = QuadSwarmEnv(65536, 1, 0, BENCH_FEATURES, seed=2, weights=WL.weights, device=dev, stream=stream)
            env.reset(2)
            T = 32
            acts = torch.from_numpy(W.actions(2, T, env.D)).to(dev)
            obs = torch.empty(T, env.D, env.obs_dim, device=dev)
            rew = torch.empty(T, env.D, device=dev)
            for _ in range(3):
                env.rollout(acts, obs, rew, None)
        elif name in ("rollout_ws", "scenario_rollout"):
            # 8192 single-drone envs, or 2048 envs x 8 (K = 6) with every
            # scenario type: 100-step rollouts in the handle's default shape
            # (the warp-specialised rollout at these sizes)
            wl = W.PLAIN if name == "rollout_ws" else W.SWARM
            scn = () if name == "rollout_ws" else tuple(qs.SCENARIOS)
            env = QuadSwarmEnv(wl.n_envs, wl.swarm, wl.k_neighbors, wl.features + ("auto_reset",), seed=2,
                               weights=wl.weights, device=dev, stream=stream, scenarios=scn)
            env.reset(2)
            T = 100
            acts = torch.from_numpy(W.actions(2, T, env.D)).to(dev)
            obs = torch.empty(T, env.D, env.obs_dim, device=dev)
            rew = torch.empty(T, env.D, device=dev)
            for _ in range(3):
                env.rollout(acts, obs, rew, None)
        elif name == "call_large":  # per-call steps of 262,144 single-drone envs (HBM-bound form)
            env = QuadSwarmEnv(262144, 1, 0, BENCH_FEATURES, seed=2, weights=WL.weights, device=dev, stream=stream)
            env.reset(2)
            acts = torch.from_numpy(W.actions(2, 8, env.D)).to(dev)
            for t in range(8):
                env.step(acts[t])
        elif name == "swarm_call":  # 2048 envs x 8, K = 6, per-call steps
            wl = W.SWARM
            env = QuadSwarmEnv(wl.n_envs, wl.swarm, wl.k_neighbors, wl.features, seed=3, weights=wl.weights,
                               device=dev, stream=stream)
            env.reset(3)
            acts = torch.from_numpy(W.actions(3, 20, env.D)).to(dev)
            for t in range(20):
                env.step(acts[t])
        elif name in ("adjoint", "adjoint_discrete", "adjoint_event_time"):  # 1024 envs x 8, 32 steps, ckpt 16
            wl = W.DIFF
            feats = {"adjoint": wl.features, "adjoint_discrete": ("dr", "motor_noise", "floor", "walls", "collisions"),
                     "adjoint_event_time": ("dr", "motor_noise", "floor", "walls", "collisions", "event_time")}[name]
            env = QuadSwarmEnv(wl.n_envs, wl.swarm, 0, feats, seed=5, device=dev, stream=stream)
            env.reset(5)
            T, C = 32, 16
            x0 = env.get_state()["state"].contiguous()
            acts = torch.from_numpy(W.actions(5, T, env.D, lo=0.05, hi=0.95)).to(dev)
            ws = torch.empty(qs.qs_diff_workspace_size(env.h, T, C), dtype=torch.uint8, device=dev)
            loss = torch.empty(env.D, device=dev)
            ga = torch.empty_like(acts)
            gx = torch.empty(env.D, 30, device=dev)
            for _ in range(2):
                qs.qs_diff_forward(env.h, T, C, x0, acts, loss, ws)
                qs.qs_diff_backward(env.h, T, C, acts, torch.ones(env.D, device=dev), ws, ga, gx)
        env.sync()
        env.close()
    print(json.dumps({"profile_case": name, "ok": True}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--profile-case", choices=["rollout", "rollout_ws", "scenario_rollout", "call_large", "swarm_call",
                                               "adjoint", "adjoint_discrete", "adjoint_event_time"], default=None,
                    help="run one small case of a form (for ncu captures) and exit")
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--warmup-seconds", type=float, default=0.5,
                    help="least wall time of the headline's warm-up loop (0 for profiler runs: exactly W steps)")
    ap.add_argument("--impl", choices=["gpu", "reference"], default="gpu")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true",
                    help="skip the end-to-end loops (for profiler runs: a profiler that completes each launch before "
                         "returning would hold the resident server's launch until it retires, every step)")
    ap.add_argument("--no-forms", action="store_true", help="skip the batched / swarm / uneven / sweep forms")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.profile_case:
        profile_case(args.profile_case, int(os.environ.get("LOCAL_RANK", "0")))
        return
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    line = run_gpu(args, world, rank, local)
    if world == 1 and not args.no_forms:  # the extra forms run on a single GPU only
        import torch
        dev = torch.device("cuda", local)
        line["forms"] = run_forms(dev, torch.cuda.Stream(device=dev), WL.seed)
        f = line["forms"]
        # throughput of each form relative to the plain per-call GPU step (same binary32 accuracy)
        f["ratio_vs_plain_call"] = {k: f[k]["value"] / line["value"] for k in
                                    ("plain_rollout", "swarm_call", "swarm_rollout", "uneven_batched", "uneven_call",
                                     "fwd_adjoint", "fwd_adjoint_discrete", "fwd_adjoint_event_time")}
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline:  # the oracle's CPU baseline: rank 0 at N = 1 only
            line["cpu_baseline"] = cpu_baseline_legs()
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
