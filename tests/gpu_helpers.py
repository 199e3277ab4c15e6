"""Shared set-up of the GPU parity tests: the same seeded inputs go to the CUDA
path (through the C ABI) and to the FP64 oracle."""
import numpy as np
import torch

from oracle import oracle as O
from paper_2306_09537_gb300 import workloads as W

OR_FLAGS = {"dr": O.F_DR, "motor_noise": O.F_MOTOR_NOISE, "obs_noise": O.F_OBS_NOISE, "collisions": O.F_COLLISIONS,
            "floor": O.F_FLOOR, "walls": O.F_WALLS, "auto_reset": O.F_AUTO_RESET, "smooth": O.F_SMOOTH,
            "action_symmetric": O.F_ACTION_SYMMETRIC, "record_knn": O.F_RECORD_KNN,
            "downwash": O.F_DOWNWASH, "event_time": O.F_EVENT_TIME}
ALL_WEIGHTS = {n: 0.1 * (i + 1) * (-1) ** i for i, n in enumerate(O.W_NAMES)}
DEV = torch.device("cuda:0")


def pair(sizes, K, features, seed=1, weights=None, scenarios=(), **overrides):
    """(QuadSwarmEnv, Oracle) with the same configuration."""
    from paper_2306_09537_gb300.env import QuadSwarmEnv
    sizes = np.asarray(sizes, dtype=np.int32)
    E = len(sizes)
    env = QuadSwarmEnv(E, sizes, K, features, seed=seed, weights=weights, device=DEV, scenarios=scenarios,
                       **overrides)
    flags = 0
    for f in features:
        flags |= OR_FLAGS[f]
    oc = O.default_config(n_envs=E, k_neighbors=K, flags=flags, seed=seed, scenarios=O.scenario_mask(scenarios))
    if weights is not None:
        oc.w[:] = [0.0] * 14
        O.set_config(oc, weights=weights)
    o_over = {k: v for k, v in overrides.items()}
    O.set_config(oc, **o_over)
    o = O.Oracle(oc, sizes)
    return env, o


def nominal(env):
    p = env.cfg.params
    return [p.mass, p.ixx, p.iyy, p.izz, p.t2w, p.tau_m, p.arm]


def set_both(env, o, st, prm, goals, ep=0, tick=0):
    E = env.E
    epa = np.full(E, ep, dtype=np.int32)
    tka = np.full(E, tick, dtype=np.int32)
    env.set_state(torch.from_numpy(np.ascontiguousarray(st, np.float32)).to(DEV),
                  torch.from_numpy(np.ascontiguousarray(prm, np.float32)).to(DEV),
                  torch.from_numpy(np.ascontiguousarray(goals, np.float32)).to(DEV),
                  torch.from_numpy(epa).to(DEV), torch.from_numpy(tka).to(DEV))
    o.set_state(np.asarray(st, np.float64), np.asarray(prm, np.float64), np.asarray(goals, np.float64), epa,
                tka.astype(np.uint32))


def seeded_inputs(env, seed, sizes, spread=None, **kw):
    """Seeded binary32 state / params / goals of the paper's workload shapes."""
    D, E = env.D, env.E
    st = W.random_states(seed, D, **kw)
    if spread is not None:
        st[:, 0:3] = W.clustered_positions(seed, sizes, spread=spread)
    prm = W.random_params(seed, E, nominal(env))
    goals = W.random_goals(seed, E)
    return st, prm, goals


def gpu_state(env):
    s = env.get_state()
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in s.items()}


def env_of(sizes):
    return np.repeat(np.arange(len(sizes)), sizes)
