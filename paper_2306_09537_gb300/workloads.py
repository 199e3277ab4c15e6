"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module holds none of the method's arithmetic: it only describes the
workload shapes (paper Sec. IV: 100 Hz control, 200 Hz physics, 15 s episodes;
Sec. III-C/III-D: swarms sharing one goal, K nearest neighbours) and draws the
inputs a caller would feed the simulator -- per-rotor commands and, for the
uneven-swarm workload, the swarm sizes. Both the CUDA path and the oracle read
these arrays; random numbers that the method itself draws (domain
randomisation, noise, collision perturbations) are not made here: each side
draws them from its own Philox4x32-10 implementation.

The paper's workloads come from its scenario generators and from an RL
policy (Sec. III-D, III-F); there is no dataset. The stand-in here is a
seeded uniform [0,1]^4 command stream per drone per control step.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

# Named feature switches; each side maps them onto its own flag bits.
FEATURES = ("dr", "motor_noise", "obs_noise", "collisions", "floor", "walls", "auto_reset",
            "smooth", "action_symmetric", "record_knn", "downwash", "event_time")

UNEVEN_SIZES = (1, 2, 4, 8, 16, 32, 64)


@dataclass
class Workload:
    name: str
    n_envs: int
    swarm: int | None          # drones per env (uniform) or None for uneven sizes
    k_neighbors: int
    steps: int
    seed: int
    features: tuple = ()
    weights: dict = field(default_factory=dict)
    horizon: int = 0           # rollout length (batched / differentiable forms)
    ckpt_every: int = 0

    def sizes(self) -> np.ndarray:
        if self.swarm is not None:
            return np.full(self.n_envs, self.swarm, dtype=np.int32)
        return uneven_swarm_sizes(self.seed, self.n_envs)


GOAL_REACHING = {"pos": -1.0, "spin": -0.1, "hit_floor": -1.0, "hit_wall": -1.0, "hit_ceil": -1.0,
                 "hit_quad": -1.0}
PHYS = ("floor", "walls", "motor_noise", "obs_noise")

# 1 env x 1 drone, nominal parameters (no randomisation), 1000 control steps
TINY = Workload("tiny_1x1", 1, 1, 0, 1000, 1, PHYS, GOAL_REACHING)
# 8192 envs x 1 drone, +-20% randomisation, goal-reaching reward, room contacts
PLAIN = Workload("plain_8192x1", 8192, 1, 0, 1000, 2, PHYS + ("dr",), GOAL_REACHING)
# 2048 envs x 8 drones, K = 6, collisions with perturbation, one goal per env
SWARM = Workload("swarm_2048x8_k6", 2048, 8, 6, 1000, 3, PHYS + ("dr", "collisions"), GOAL_REACHING)
# 4096 envs with swarm sizes from {1..64} (P(N) ~ N^-0.38), 256-step rollouts, K = min(6, N-1)
UNEVEN = Workload("uneven_4096", 4096, None, 6, 256, 4, PHYS + ("dr", "collisions"), GOAL_REACHING,
                  horizon=256)
# 1024 envs x 8 drones, 128-step differentiable rollout with checkpoints every 16 steps
DIFF = Workload("diff_1024x8_t128", 1024, 8, 6, 128, 5, ("dr", "smooth", "motor_noise"), {},
                horizon=128, ckpt_every=16)

WORKLOADS = {w.name: w for w in (TINY, PLAIN, SWARM, UNEVEN, DIFF)}


def uneven_swarm_sizes(seed: int, n_envs: int) -> np.ndarray:
    """Swarm sizes from {1,2,4,8,16,32,64} with P(N) proportional to N^-0.38."""
    sizes = np.array(UNEVEN_SIZES, dtype=np.int64)
    p = sizes.astype(np.float64) ** -0.38
    p /= p.sum()
    rng = np.random.Generator(np.random.Philox(key=np.uint64(0xA5A5_0000 + seed)))
    return rng.choice(sizes, size=n_envs, p=p).astype(np.int32)


def actions(seed: int, steps: int, n_drones: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    """Seeded per-rotor commands, [steps][n_drones][4] float32, uniform in [lo, hi]."""
    rng = np.random.Generator(np.random.Philox(key=np.uint64(0x5EED_0000 + seed)))
    a = rng.random((steps, n_drones, 4), dtype=np.float32)
    return (lo + (hi - lo) * a).astype(np.float32)


def random_states(seed: int, n_drones: int, room=(5.0, 5.0, 10.0), vel=1.0, rate=1.0,
                  uf=(0.5, 0.9)) -> np.ndarray:
    """Seeded binary32 drone states [n][30] (x, v, R, w, uf, eps, fprev) for
    single-step tests. The rotation comes from the QR factorisation of a
    Gaussian matrix (sign-fixed to a rotation), so it is orthonormal up to
    binary32 rounding."""
    rng = np.random.Generator(np.random.Philox(key=np.uint64(0x57A7_0000 + seed)))
    s = np.zeros((n_drones, 30), dtype=np.float64)
    s[:, 0] = rng.uniform(-room[0], room[0], n_drones)
    s[:, 1] = rng.uniform(-room[1], room[1], n_drones)
    s[:, 2] = rng.uniform(0.0, room[2], n_drones)
    s[:, 3:6] = rng.uniform(-vel, vel, (n_drones, 3))
    g = rng.standard_normal((n_drones, 3, 3))
    q, r = np.linalg.qr(g)
    q = q * np.sign(np.diagonal(r, axis1=1, axis2=2))[:, None, :]
    det = np.linalg.det(q)
    q[det < 0, :, 0] *= -1.0
    s[:, 6:15] = q.reshape(n_drones, 9)
    s[:, 15:18] = rng.uniform(-rate, rate, (n_drones, 3))
    s[:, 18:22] = rng.uniform(uf[0], uf[1], (n_drones, 4))
    s[:, 22:26] = rng.normal(0.0, 1e-3, (n_drones, 4))
    s[:, 26:30] = rng.uniform(0.0, 1.0, (n_drones, 4))
    return s.astype(np.float32)


def random_params(seed: int, n_envs: int, nominal, lo=0.8, hi=1.2) -> np.ndarray:
    """Seeded binary32 per-env parameters [E][7] = nominal * U(lo, hi)."""
    rng = np.random.Generator(np.random.Philox(key=np.uint64(0x9A7A_0000 + seed)))
    nom = np.asarray(nominal, dtype=np.float64)
    return (nom[None, :] * rng.uniform(lo, hi, (n_envs, nom.size))).astype(np.float32)


def random_goals(seed: int, n_envs: int, room=(5.0, 5.0, 10.0)) -> np.ndarray:
    rng = np.random.Generator(np.random.Philox(key=np.uint64(0x60A1_0000 + seed)))
    g = np.stack([rng.uniform(-room[0], room[0], n_envs), rng.uniform(-room[1], room[1], n_envs),
                  rng.uniform(0.0, room[2], n_envs)], axis=1)
    return g.astype(np.float32)


def clustered_positions(seed: int, sizes, spread: float = 0.15, dup_frac: float = 0.0,
                        room=(5.0, 5.0, 10.0)) -> np.ndarray:
    """Binary32 positions [D][3]: each env's drones in a tight cluster (so that
    pairs collide and neighbour orders are contested); a fraction of drones
    copies another drone's position exactly (forced key ties)."""
    rng = np.random.Generator(np.random.Philox(key=np.uint64(0xC105_0000 + seed)))
    out = []
    for n in sizes:
        c = np.array([rng.uniform(-room[0] + 1, room[0] - 1), rng.uniform(-room[1] + 1, room[1] - 1),
                      rng.uniform(1.0, room[2] - 1.0)])
        p = c[None, :] + rng.uniform(-spread, spread, (int(n), 3))
        if dup_frac > 0 and n >= 2:
            for i in range(int(n)):
                if rng.random() < dup_frac:
                    p[i] = p[rng.integers(0, int(n))]
        out.append(p)
    return np.concatenate(out, axis=0).astype(np.float32)


def stacked_positions(seed: int, sizes, per_column: int = 3, offset: float = 0.04, gap=(0.1, 0.6),
                      pitch: float = 0.5, room=(5.0, 5.0, 10.0)) -> np.ndarray:
    """Binary32 positions [D][3] in vertical columns of up to `per_column`
    drones (formation flight with drones above one another): within a column
    each drone sits `gap` metres (uniform) above the previous one, offset
    horizontally by up to `offset` m per axis; columns stand `pitch` m apart
    on a grid around a random centre per env."""
    rng = np.random.Generator(np.random.Philox(key=np.uint64(0x57AC_0000 + seed)))
    out = []
    for n in sizes:
        n = int(n)
        ncol = (n + per_column - 1) // per_column
        side = int(np.ceil(np.sqrt(ncol)))
        span = (side - 1) * pitch
        c = np.array([rng.uniform(-room[0] + 1, room[0] - 1 - span), rng.uniform(-room[1] + 1, room[1] - 1 - span),
                      rng.uniform(1.0, room[2] - 1.0 - per_column * gap[1])])
        p = np.zeros((n, 3))
        for i in range(n):
            col, lvl = divmod(i, per_column)
            base = c + np.array([(col % side) * pitch, (col // side) * pitch, 0.0])
            if lvl == 0:
                p[i] = base
            else:
                p[i] = p[i - 1] + np.array([0.0, 0.0, rng.uniform(*gap)])
            p[i, 0:2] = base[0:2] + rng.uniform(-offset, offset, 2)
        out.append(p)
    return np.concatenate(out, axis=0).astype(np.float32)


def contact_swarm_states(seed: int, n_envs: int, n: int, spread: float = 0.08) -> np.ndarray:
    """Binary32 drone states [n_envs * n][30] of swarms placed to meet every
    contact within a few dozen steps: env e % 4 == 0 a cluster in mid-air
    (pairs collide), 1 a cluster just above the floor falling at 1.5 m/s,
    2 a cluster at the +x wall moving outward with the thrust axis pointing
    back into the room, 3 a cluster under the ceiling climbing with the thrust
    axis pointing down (so that drones leave the wall or ceiling after the hit
    instead of pressing on it); velocities and body rates otherwise as in
    random_states."""
    s = random_states(seed, n_envs * n, rate=0.5).astype(np.float64)
    rng = np.random.Generator(np.random.Philox(key=np.uint64(0xC0A7_0000 + seed)))
    for e in range(n_envs):
        sl = slice(e * n, (e + 1) * n)
        p = rng.uniform(-spread, spread, (n, 3))
        kind = e % 4
        if kind == 0:
            c = np.array([rng.uniform(-3.0, 3.0), rng.uniform(-3.0, 3.0), rng.uniform(3.0, 7.0)])
        elif kind == 1:
            c = np.array([rng.uniform(-3.0, 3.0), rng.uniform(-3.0, 3.0), spread + 0.03])
            s[sl, 5] = -1.5
        elif kind == 2:
            c = np.array([5.0 - spread - 0.03, rng.uniform(-3.0, 3.0), rng.uniform(3.0, 7.0)])
            s[sl, 3] = 1.5
            s[sl, 6:15] = np.array([0.0, 0.0, -1.0, 0.0, 1.0, 0.0, 1.0, 0.0, 0.0])  # body z along -x
        else:
            c = np.array([rng.uniform(-3.0, 3.0), rng.uniform(-3.0, 3.0), 10.0 - spread - 0.03])
            s[sl, 5] = 1.5
            s[sl, 6:15] = np.array([1.0, 0.0, 0.0, 0.0, -1.0, 0.0, 0.0, 0.0, -1.0])  # body z down
        s[sl, 0:3] = c[None, :] + p
    return s.astype(np.float32)
