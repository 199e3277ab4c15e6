"""Autotuner of the launch shapes: CTA size per swarm-width class of the
per-call step, and CTA size / control steps per launch / graph use of the
batched rollout. Candidates are timed with CUDA events on a scratch twin of
the environment (same configuration, same seed), so tuning never advances the
caller's simulation; the best shapes are then applied to the caller's handle.
Each timed repetition starts from a cold L2 (a 256 MiB write before it), as a
step or rollout does when other work runs between calls, and a candidate is
ranked by its median over the repetitions: the ranking of close candidates
can differ between warm and cold timing (the uneven 4096-env rollout, one
session: persistent 64-thread CTAs 20.7 us per step warm and 19.2 us cold
against 20.3 and 20.4 us for the warp-specialised kernel). Results depend
only on the configuration and are cached per process."""
from __future__ import annotations

import numpy as np
import torch

from . import qs
from . import workloads as W

_CACHE: dict = {}


def _signature(env) -> tuple:
    c = env.cfg
    return (env.D, env.E, env.K, int(c.flags), int(c.scenarios), int(c.substeps), tuple(np.asarray(env.sizes).tolist())
            if env.sizes is not None else int(c.n_per_env))


L2_FLUSH_BYTES = 256 << 20


def _time(fn, stream, reps, flush):
    ts = []
    for _ in range(reps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        ts.append(a.elapsed_time(b))
    return float(np.median(ts))


def tune(env, steps: int = 32, horizon: int = 64, reps: int = 5, apply: bool = True) -> dict:
    """Returns {"step_blocks": {W: block}, "rollout": (block, fuse, graph), "timings": {...}}
    (step_blocks is empty for a handle with several width classes: its per-call
    step is the rollout launch, and the rollout shape covers it)."""
    from .env import QuadSwarmEnv
    key = _signature(env)
    if key in _CACHE:
        res = _CACHE[key]
    else:
        twin = QuadSwarmEnv(env.E, env.sizes if env.sizes is not None else int(env.cfg.n_per_env), env.K,
                            env.features, seed=int(env.cfg.seed), weights=env.weights, device=env.device,
                            stream=env.stream, scenarios=env.scenarios, **env.overrides)
        stream = twin.stream
        classes = sorted({int(2 ** np.ceil(np.log2(n))) if n > 1 else 1 for n in
                          (np.asarray(twin.sizes) if twin.sizes is not None else [int(twin.cfg.n_per_env)])})
        acts = torch.from_numpy(W.actions(int(twin.cfg.seed), max(steps, horizon), twin.D)).to(twin.device)
        timings = {"step": {}, "rollout": {}}
        step_blocks = {}
        with torch.cuda.stream(stream):
            flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=twin.device)
            # a handle with several width classes steps them all in one launch of
            # the rollout kernels, shaped below; only a single class has a
            # per-call kernel to shape
            for w in (classes if len(classes) == 1 else []):
                best = None
                for b in (qs.QS_BLOCK_WARP_SPECIALISED, 32, 64, 128, 256):
                    if b == qs.QS_BLOCK_WARP_SPECIALISED:
                        if w > 32:
                            continue
                    elif b % w or b < w:
                        continue
                    qs.qs_set_block(twin.h, w, b)

                    def run():
                        for t in range(steps):
                            twin.step(acts[t])
                    run()
                    ms = _time(run, stream, reps, flush) / steps
                    timings["step"][(w, b)] = ms
                    if best is None or ms < best[0]:
                        best = (ms, b)
                step_blocks[w] = best[1]
                qs.qs_set_block(twin.h, w, best[1])
            obs = torch.empty(horizon, twin.D, twin.obs_dim, device=twin.device)
            rew = torch.empty(horizon, twin.D, device=twin.device)
            best = None
            maxw = max(classes)
            for b in (qs.QS_BLOCK_WARP_SPECIALISED, 64, 128, 256):
                if b == qs.QS_BLOCK_WARP_SPECIALISED:
                    if maxw > 64:
                        continue
                elif b < maxw:
                    continue
                for fuse in (0, max(1, horizon // 8)):
                    for graph in (True, False):
                        qs.qs_set_rollout_shape(twin.h, b, fuse, graph)

                        def run():
                            twin.rollout(acts[:horizon], obs, rew, None)
                        run()
                        ms = _time(run, stream, reps, flush) / horizon
                        timings["rollout"][(b, fuse, graph)] = ms
                        if best is None or ms < best[0]:
                            best = (ms, (b, fuse, graph))
            del flush
        twin.close()
        res = {"step_blocks": step_blocks, "rollout": best[1], "timings": timings}
        _CACHE[key] = res
    if apply:
        for w, b in res["step_blocks"].items():
            qs.qs_set_block(env.h, w, b)
        qs.qs_set_rollout_shape(env.h, *res["rollout"])
    return res
