"""Parity of the CUDA step (through the C ABI) with the FP64 oracle.

One step from identical inputs: neighbour indices, collision sets, event bits
and done are bit-exact, except for drones whose oracle step took a decision
within a relative margin of its threshold (there a binary32 and a binary64
run may legitimately branch apart; those drones are counted and must be
rare). Continuous outputs match within tolerances derived from binary32
rounding. Runs of 100 steps follow the lockstep-restart protocol of
tests/lockstep.py: positions within 1e-4 m and rotation entries within 1e-5,
or within the binary32 floor of the drone's own trajectory.
"""
import numpy as np
import pytest
import torch

import lockstep as L
from gpu_helpers import ALL_WEIGHTS, DEV, env_of, gpu_state, nominal, pair, seeded_inputs, set_both
from oracle import oracle as O
from paper_2306_09537_gb300 import workloads as W

pytestmark = pytest.mark.gpu

FULL = ("floor", "walls", "motor_noise", "obs_noise", "dr", "collisions", "record_knn")
MARGIN_1STEP = 1e-6  # ~17 binary32 ulps: one step from identical inputs cannot flip a wider decision


def one_step(sizes, K, features, seed, weights=ALL_WEIGHTS, spread=0.12, act_range=(0.0, 1.0), **kw):
    env, o = pair(sizes, K, features, seed=seed, weights=weights, **kw)
    st, prm, goals = seeded_inputs(env, seed, sizes, spread=spread if max(sizes) > 1 else None)
    set_both(env, o, st, prm, goals, ep=3, tick=11)
    acts = W.actions(seed, 1, env.D, lo=act_range[0], hi=act_range[1])[0]
    obs, rew, done = env.step(torch.from_numpy(acts).to(DEV))
    ev, knn = env.get_events(knn="record_knn" in features and K > 0)
    g = gpu_state(env)
    oobs, orew, odone = o.step(acts.astype(np.float64))
    oev, oknn, _ = o.get_events()
    margin, margin_knn = o.margins()
    os_ = o.get_state()
    return dict(env=env, o=o, obs=obs.cpu().numpy(), rew=rew.cpu().numpy(), done=done.cpu().numpy(),
                ev=ev.cpu().numpy().astype(np.uint32), knn=None if knn is None else knn.cpu().numpy().astype(np.int32),
                g=g, oobs=oobs, orew=orew, odone=odone, oev=oev, oknn=oknn, margin=margin, margin_knn=margin_knn,
                os=os_)


def velocity_tolerance(state, params, sizes, base=2e-5, eps_x=1e-6):
    """Per-env bound on the binary32 velocity error after a collision response:
    the contact normal (x_i - x_j)/d of a pair d apart carries a relative error
    of about eps_x / d, which scales the exchanged velocity |v_i| + |v_j|."""
    off = np.concatenate([[0], np.cumsum(sizes)])
    tol = np.full(len(sizes), base)
    for e in range(len(sizes)):
        a, b = off[e], off[e + 1]
        if b - a < 2:
            continue
        x, v = state[a:b, 0:3], state[a:b, 3:6]
        d = np.linalg.norm(x[:, None] - x[None], axis=2) + np.eye(b - a)
        sp = np.linalg.norm(v, axis=1)
        near = d < 2.0 * params[e, 6] * 1.001
        if near.any():
            tol[e] += (eps_x * (sp[:, None] + sp[None] + 1.0) / d)[near].max()
    return tol


def check_step(r, sizes, margin=MARGIN_1STEP, max_excluded=0.01):
    eo = env_of(sizes)
    bad_env = np.zeros(len(sizes), bool)
    np.logical_or.at(bad_env, eo, r["margin"] < margin)
    keep = ~bad_env[eo]
    assert keep.mean() >= 1.0 - max_excluded, f"too many near-threshold drones: {1 - keep.mean():.3%}"
    g, o = r["g"]["state"], r["os"]["state"]
    vtol = velocity_tolerance(o, r["os"]["params"], sizes)[eo][:, None]
    # continuous state: binary32 rounding of one step
    assert np.abs(g[keep, 0:3] - o[keep, 0:3]).max() < 2e-5
    assert (np.abs(g[keep, 3:6] - o[keep, 3:6]) <= vtol[keep]).all()
    assert np.abs(g[keep, 6:15] - o[keep, 6:15]).max() < 2e-6
    assert np.allclose(g[keep, 15:18], o[keep, 15:18], rtol=2e-5, atol=2e-5)
    assert np.allclose(g[keep, 18:30], o[keep, 18:30], rtol=1e-5, atol=1e-7)
    otol = np.broadcast_to(2e-5 + 0 * vtol, r["obs"].shape).copy()
    for k in range(r["obs"].shape[1]):
        if k in (3, 4, 5) or (k >= 18 and (k - 18) % 6 >= 3):  # velocity entries
            otol[:, k:k + 1] = 2 * vtol
    assert (np.abs(r["obs"][keep] - r["oobs"][keep]) <= otol[keep] + 2e-5 * np.abs(r["oobs"][keep])).all()
    rtol_ = 2e-5 + 2 * vtol[:, 0] * abs(ALL_WEIGHTS["vel"])
    assert (np.abs(r["rew"][keep] - r["orew"][keep]) <= rtol_[keep] + 2e-5 * np.abs(r["orew"][keep])).all()
    # discrete outputs: bit-exact
    assert np.array_equal(r["ev"][keep], r["oev"][keep])
    if r["knn"] is not None:
        kk = keep & (r["margin_knn"] >= margin)
        assert np.array_equal(r["knn"][kk], r["oknn"][kk])
    assert np.array_equal(r["done"], r["odone"])
    assert np.array_equal(r["g"]["ep_step"], r["os"]["ep_step"])
    assert np.array_equal(r["g"]["tick"].astype(np.uint32), r["os"]["tick"])
    return keep


# ----------------------------------------------------------------------------- reset
@pytest.mark.parametrize("sizes,K", [([1] * 2048, 0), ([8] * 256, 6), ([1, 2, 3, 5, 8, 13, 33, 64], 6)])
def test_reset_matches_oracle(sizes, K):
    env, o = pair(sizes, K, FULL, seed=21)
    obs = env.reset(21).clone()
    o.reset(21)
    g = gpu_state(env)
    s = o.get_state()
    assert np.allclose(g["params"], s["params"], rtol=2e-7, atol=0)
    assert np.abs(g["goals"] - s["goals"]).max() < 2e-6
    assert np.abs(g["state"][:, 0:6] - s["state"][:, 0:6]).max() < 2e-6
    assert np.abs(g["state"][:, 6:18] - s["state"][:, 6:18]).max() < 2e-6
    assert np.allclose(g["state"][:, 18:30], s["state"][:, 18:30], rtol=2e-7, atol=0)
    assert (g["ep_step"] == 0).all() and (g["tick"] == 0).all()
    oobs = o.observe()
    assert np.allclose(obs.cpu().numpy(), oobs, rtol=1e-5, atol=5e-6)


# ----------------------------------------------------------------------------- one step
@pytest.mark.parametrize("name,sizes,K,features", [
    ("single", [1] * 1000, 0, FULL),
    ("single_k6_padded", [1] * 300, 6, FULL),
    ("swarm8", [8] * 300, 6, FULL),
    ("uneven", [1, 2, 3, 4, 5, 7, 8, 9, 16, 17, 31, 32, 33, 48, 64] * 4, 6, FULL),
    ("large_swarms", [128, 100, 65, 128], 6, FULL),
    ("k_gt_n", [2, 3, 4] * 40, 8, FULL),
    ("symmetric_actions", [4] * 100, 3, FULL + ("action_symmetric",)),
    ("no_noise_no_dr", [8] * 100, 6, ("floor", "walls", "collisions", "record_knn")),
    # smooth contacts (the differentiable form) stepped by the general instance:
    # wall and floor penalties, and the pair penalty of swarms in every substep
    ("smooth_single", [1] * 300, 0, ("smooth", "dr", "motor_noise", "obs_noise")),
    ("smooth_swarm8", [8] * 200, 6, ("smooth", "dr", "motor_noise", "obs_noise", "collisions", "record_knn")),
    ("smooth_uneven", [1, 2, 3, 8, 17, 33, 64] * 4, 6, ("smooth", "dr", "motor_noise", "collisions", "record_knn")),
    # further feature combinations: each contact rule alone, neighbours without
    # collisions, and the smooth contacts with downwash (general instance)
    ("floor_only", [1] * 300, 0, ("floor", "dr", "motor_noise")),
    ("walls_only", [4] * 100, 3, ("walls", "dr", "collisions", "record_knn")),
    ("knn_without_collisions", [8] * 100, 6, ("floor", "walls", "obs_noise", "record_knn")),
    ("smooth_downwash", [8] * 100, 6, ("smooth", "dr", "motor_noise", "downwash", "collisions", "record_knn")),
])
def test_single_step_parity(name, sizes, K, features):
    # 100+ drones packed into 0.24 m would all touch; spread large swarms wider
    r = one_step(sizes, K, features, seed=sum(map(ord, name)) % 1000, spread=1.0 if max(sizes) > 64 else 0.12)
    check_step(r, sizes)


@pytest.mark.parametrize("symmetric", [False, True])
def test_single_step_parity_commands_out_of_range(symmetric):
    """Commands beyond the action map's range (Sec. III-A: clip to [0, 1], or
    the paper's (clip(a, -1, 1) + 1) / 2) are clipped the same way on both
    sides; the reward's action terms see the clipped commands."""
    feats = FULL + (("action_symmetric",) if symmetric else ())
    r = one_step([8] * 100, 6, feats, seed=77, act_range=(-1.5, 1.5))
    check_step(r, [8] * 100)


@pytest.mark.parametrize("substeps", [1, 3, 5])
@pytest.mark.parametrize("sizes,K", [([1] * 300, 0), ([8] * 100, 6), ([8] * 60, 0)])
def test_single_step_parity_substeps(substeps, sizes, K):
    """Physics substeps per control step other than the paper's two (the
    warp-specialised kernels draw the motor normals of up to four substeps
    ahead and the rest inline), and swarms without neighbour observations."""
    r = one_step(sizes, K, FULL, seed=40 + substeps, substeps=substeps)
    check_step(r, sizes)


@pytest.mark.parametrize("substeps", [1, 5])
def test_rollout_equals_steps_substeps(substeps):
    """Rollouts (warp-specialised and persistent) against per-call steps with
    1 and 5 physics substeps per control step."""
    from paper_2306_09537_gb300 import qs
    for sizes, shape in (([8] * 64, None), ([1, 2, 8, 33, 64, 5] * 6, None), ([1, 2, 8, 33, 64, 5] * 6,
                                                                              (qs.QS_BLOCK_WARP_SPECIALISED, 0, 1))):
        env, _ = pair(sizes, 6, FULL + ("auto_reset",), seed=14, episode_steps=7, substeps=substeps)
        env2, _ = pair(sizes, 6, FULL + ("auto_reset",), seed=14, episode_steps=7, substeps=substeps)
        if shape is not None:
            qs.qs_set_rollout_shape(env.h, *shape)
        T = 9
        acts = torch.from_numpy(W.actions(14, T, env.D)).to(DEV)
        obs = torch.empty(T, env.D, env.obs_dim, device=DEV)
        rew = torch.empty(T, env.D, device=DEV)
        env.rollout(acts, obs, rew, None)
        for t in range(T):
            o2, r2, _ = env2.step(acts[t])
            assert torch.equal(obs[t], o2) and torch.equal(rew[t], r2), (sizes[:3], shape, t)
        assert torch.equal(env.get_state()["state"], env2.get_state()["state"])


def test_single_step_contacts_exercised():
    """A room-contact-heavy state: many drones start at the floor, walls or
    ceiling, moving outward, so every contact branch is taken."""
    sizes = [1] * 2000
    env, o = pair(sizes, 0, FULL, seed=5, weights=ALL_WEIGHTS)
    st, prm, goals = seeded_inputs(env, 5, sizes, vel=3.0)
    rng = np.random.default_rng(5)
    n = env.D
    which = rng.integers(0, 4, n)
    st[which == 0, 2] = 0.0                               # on the floor
    st[which == 0, 3:6] = 0.0
    st[which == 1, 2] = rng.uniform(0, 0.01, (which == 1).sum())   # about to hit it
    st[which == 1, 5] = -2.0
    st[which == 2, 0] = 4.995                             # at a wall
    st[which == 2, 3] = 2.0
    st[which == 3, 2] = 9.995                             # at the ceiling
    st[which == 3, 5] = 2.0
    set_both(env, o, st, prm, goals)
    acts = W.actions(5, 1, n)[0]
    obs, rew, done = env.step(torch.from_numpy(acts).to(DEV))
    ev, _ = env.get_events()
    g = gpu_state(env)
    oobs, orew, _ = o.step(acts.astype(np.float64))
    oev, _, margin = o.get_events()
    keep = margin >= MARGIN_1STEP
    assert keep.mean() > 0.99
    ev = ev.cpu().numpy().astype(np.uint32)
    assert np.array_equal(ev[keep], oev[keep])
    for bit in (O.EV_HIT_FLOOR, O.EV_ON_FLOOR, O.EV_HIT_WALL, O.EV_HIT_CEIL):
        assert (oev & bit).sum() > 50
    s = o.get_state()["state"]
    assert np.abs(g["state"][keep, 0:6] - s[keep, 0:6]).max() < 2e-5
    assert np.abs(g["state"][keep, 6:15] - s[keep, 6:15]).max() < 2e-6
    assert np.allclose(rew.cpu().numpy()[keep], orew[keep], rtol=2e-5, atol=2e-5)


@pytest.mark.parametrize("sizes", [[8] * 200, [3, 5, 17, 33, 64, 128] * 3])
def test_downwash_parity(sizes):
    """Drones stacked in columns (Sec. III-B downwash): the warp-specialised
    step (swarms up to 32) and the general step (wider swarms) match the
    oracle, and the downwash term really changed the step."""
    feats = FULL + ("downwash",)
    env, o = pair(sizes, 6, feats, seed=8, weights=ALL_WEIGHTS)
    st, prm, goals = seeded_inputs(env, 8, sizes)
    st[:, 0:3] = W.stacked_positions(8, sizes)
    set_both(env, o, st, prm, goals, ep=3, tick=11)
    acts = W.actions(8, 1, env.D)[0]
    obs, rew, done = env.step(torch.from_numpy(acts).to(DEV))
    ev, knn = env.get_events(knn=True)
    r = dict(obs=obs.cpu().numpy(), rew=rew.cpu().numpy(), done=done.cpu().numpy(),
             ev=ev.cpu().numpy().astype(np.uint32), knn=knn.cpu().numpy().astype(np.int32), g=gpu_state(env))
    r["oobs"], r["orew"], r["odone"] = o.step(acts.astype(np.float64))
    r["oev"], r["oknn"], _ = o.get_events()
    r["margin"], r["margin_knn"] = o.margins()
    r["os"] = o.get_state()
    check_step(r, sizes)
    # the same step without downwash: most drones under another one must differ
    _, o2 = pair(sizes, 6, FULL, seed=8, weights=ALL_WEIGHTS)
    set_both(env, o2, st, prm, goals, ep=3, tick=11)
    o2.step(acts.astype(np.float64))
    dv = np.abs(o2.get_state()["state"][:, 3:6] - r["os"]["state"][:, 3:6]).max(axis=1)
    assert (dv > 1e-3).mean() > 0.2
    # and the GPU saw the same: its velocities follow the downwash run, not the plain one
    gv = r["g"]["state"][:, 3:6]
    hit = dv > 1e-3
    assert np.abs(gv[hit] - r["os"]["state"][hit, 3:6]).max() < 1e-3 < np.abs(gv[hit] - o2.get_state()["state"][hit, 3:6]).max()


# ----------------------------------------------------------------------------- exact discrete decisions
@pytest.mark.parametrize("dup", [0.0, 0.3])
def test_neighbours_and_collisions_bit_exact(dup):
    """Hovering drones at rest keep their binary32 positions through the step,
    so both sides decide on identical inputs: neighbour lists and collision
    sets must agree bit for bit, including forced ties (duplicate positions)."""
    sizes = [2, 3, 5, 7, 8, 9, 16, 31, 32, 33, 64, 128] * 6
    K = 6
    feats = ("collisions", "record_knn")
    env, o = pair(sizes, K, feats, seed=9, alpha_c=1.0)
    D, E = env.D, env.E
    st = np.zeros((D, 30), np.float32)
    st[:, 0:3] = W.clustered_positions(9, sizes, spread=0.08, dup_frac=dup)
    st[:, 6:15] = np.eye(3, dtype=np.float32).ravel()
    st[:, 18:22] = np.float32(np.sqrt(0.5))
    st[:, 26:30] = 0.5
    prm = np.tile(np.asarray(nominal(env), np.float32), (E, 1))
    goals = W.random_goals(9, E)
    set_both(env, o, st, prm, goals)
    acts = np.full((D, 4), 0.5, np.float32)
    env.step(torch.from_numpy(acts).to(DEV))
    ev, knn = env.get_events(knn=True)
    g = gpu_state(env)
    o.step(acts.astype(np.float64))
    oev, oknn, _ = o.get_events()
    assert np.array_equal(g["state"][:, 0:3], st[:, 0:3])  # positions untouched at binary32
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int32)
    bk, bh = O.pairs_f32(st[:, 0:3], prm[:, 6], off, K)
    knn = knn.cpu().numpy().astype(np.int32)
    ev = ev.cpu().numpy().astype(np.uint32)
    assert np.array_equal(knn, bk) and np.array_equal(knn, oknn)
    assert np.array_equal((ev & O.EV_HIT_QUAD) != 0, bh.astype(bool))
    assert np.array_equal(ev, oev)
    assert bh.mean() > 0.3  # the case really has collisions


# ----------------------------------------------------------------------------- free running
class GpuSide:
    """The CUDA path as the binary32 side of the lockstep protocol."""

    def __init__(self, env, K):
        self.env, self.K = env, K

    def step(self, a):
        self.env.step(torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(DEV))

    def state(self):
        g = gpu_state(self.env)
        return {"state": g["state"].astype(np.float64), "params": g["params"].astype(np.float64),
                "goals": g["goals"].astype(np.float64), "ep_step": g["ep_step"],
                "tick": g["tick"].astype(np.uint32)}

    def events(self):
        ev, knn = self.env.get_events(knn=self.K > 0)
        torch.cuda.synchronize()
        return ev.cpu().numpy().astype(np.uint32), (None if knn is None else knn.cpu().numpy().astype(np.int32))


@pytest.mark.parametrize("wl,n_envs,min_steps", [(W.TINY, 1, 100), (W.PLAIN, 8192, 90), (W.SWARM, 512, 50)])
def test_free_running_100_steps(wl, n_envs, min_steps):
    """100 free-running control steps from the GPU's own reset (the oracle
    starts from its binary32 state) under the lockstep protocol: envs whose
    oracle step takes a decision within 1e-5 (relative) of its threshold, or
    a collision decision the position discrepancy could flip, restart from
    the GPU's state; every drone stays compared. Bars, every step: neighbour
    lists and collision flags are the canonical decisions on the GPU's own
    positions; event bits equal the oracle's in every non-restarting env;
    neighbour lists equal the oracle's wherever the discrepancy cannot reorder
    them. After 100 steps: every position within 1e-4 m; every rotation entry
    within max(1e-5, 10 x the spread of the binary32-storage instruments),
    and no more drones above 1e-5 than those instruments show (the floor that
    tests/test_oracle_conditioning.py establishes on the CPU)."""
    sizes = [wl.swarm] * n_envs
    K = wl.k_neighbors
    feats = wl.features + (("record_knn",) if K > 0 else ())
    env, o = pair(sizes, K, feats, seed=wl.seed, weights=wl.weights)
    env.reset(wl.seed)

    def make(extra, salt):
        c = O.OrConfig.from_buffer_copy(o.cfg)
        c.flags |= extra
        c.round_salt = salt
        return O.Oracle(c, sizes)
    res = L.run(GpuSide(env, K), o, L.instruments(make, 3), W.actions(wl.seed, 100, env.D), wl.swarm, K)
    dx, dR, spread = res["dx"], res["dR"], res["envelope_R"]
    rate = (dR > 1e-5).mean()
    inst_rate = (res["inst_dR"] > 1e-5).mean(axis=1)
    print(f"\n{wl.name} x{n_envs}: restarted envs {res['restarted_envs']:.2%}, mean steps compared "
          f"{res['steps_compared'].mean():.1f}, neighbour lists compared exactly {res['knn_exact_frac']}, "
          f"position max {dx.max():.3g}, rotation max {dR.max():.3g}, drones above 1e-5: GPU {rate:.3%}, "
          f"instruments {np.round(inst_rate * 100, 3)} %")
    assert dx.max() <= 1e-4, f"position error {dx.max():.3g}"
    bar = np.maximum(1e-5, 10.0 * spread)
    assert (dR <= bar).all(), f"{(dR > bar).sum()} drones above the rotation bar, worst ratio {(dR / bar).max():.3g}"
    assert rate <= 1.5 * inst_rate.max() + 1.0 / env.D, (rate, inst_rate)
    assert res["steps_compared"].mean() >= min_steps


def test_plain_1000_steps_invariants():
    """Full plain workload, 1000 steps on the GPU: rotations stay orthonormal,
    states stay finite and inside the room, rates within the bound."""
    wl = W.PLAIN
    from paper_2306_09537_gb300.env import QuadSwarmEnv
    env = QuadSwarmEnv(wl.n_envs, 1, 0, wl.features, seed=wl.seed, weights=wl.weights, device=DEV)
    env.reset(wl.seed)
    acts = torch.from_numpy(W.actions(wl.seed, wl.steps, env.D)).to(DEV)
    for t in range(wl.steps):
        env.step(acts[t])
    env.sync()
    s = env.get_state()["state"].double().cpu().numpy()
    R = s[:, 6:15].reshape(-1, 3, 3)
    assert np.abs(R @ R.transpose(0, 2, 1) - np.eye(3)).max() < 1e-5
    assert np.abs(np.linalg.det(R) - 1).max() < 1e-5
    assert np.isfinite(s).all()
    assert np.abs(s[:, 0:2]).max() <= 5.0 and s[:, 2].min() >= 0.0 and s[:, 2].max() <= 10.0
    assert np.abs(s[:, 15:18]).max() <= 40.0 + 3.0


# ----------------------------------------------------------------------------- API behaviour
@pytest.mark.parametrize("pinned", ["all", "none", "actions_only", "outputs_only"])
def test_step_host_equals_step(pinned):
    """The host-buffer step: page-locked buffers are used by the kernel in
    place, other host memory goes through staging copies; any mix gives the
    device step's results."""
    from paper_2306_09537_gb300 import qs
    sizes = [8] * 64
    env, _ = pair(sizes, 6, FULL, seed=3)
    env2, _ = pair(sizes, 6, FULL, seed=3)
    acts = W.actions(3, 5, env.D)
    pin_out = pinned in ("all", "outputs_only")
    pin_in = pinned in ("all", "actions_only")

    def host(t):
        return t.pin_memory() if pin_out else t

    obs_h = host(torch.empty(env.D, env.obs_dim))
    rew_h = host(torch.empty(env.D))
    done_h = host(torch.empty(env.E, dtype=torch.uint8))
    for t in range(5):
        a_h = torch.from_numpy(acts[t].copy())
        if pin_in:
            a_h = a_h.pin_memory()
        qs.qs_step_host(env2.h, a_h, obs_h, rew_h if t != 2 else None, done_h)
        obs, rew, done = env.step(a_h.to(DEV))
        torch.cuda.synchronize()
        assert torch.equal(obs.cpu(), obs_h) and torch.equal(done.cpu(), done_h)
        if t != 2:
            assert torch.equal(rew.cpu(), rew_h)


def _rollout_vs_steps(sizes, K, T, shape=None, feats=FULL + ("auto_reset",), seed=4, episode_steps=7):
    from paper_2306_09537_gb300 import qs
    env, _ = pair(sizes, K, feats, seed=seed, episode_steps=episode_steps)
    env2, _ = pair(sizes, K, feats, seed=seed, episode_steps=episode_steps)
    if shape is not None:
        qs.qs_set_rollout_shape(env.h, *shape)
    acts = torch.from_numpy(W.actions(seed, T, env.D)).to(DEV)
    obs = torch.empty(T, env.D, env.obs_dim, device=DEV)
    rew = torch.empty(T, env.D, device=DEV)
    done = torch.empty(T, env.E, dtype=torch.uint8, device=DEV)
    env.rollout(acts, obs, rew, done)
    ro = (obs.clone(), rew.clone(), done.clone())
    ref_obs, ref_rew, ref_done = [], [], []
    for t in range(T):
        o2, r2, d2 = env2.step(acts[t])
        ref_obs.append(o2.clone())
        ref_rew.append(r2.clone())
        ref_done.append(d2.clone())
    s1, s2 = env.get_state(), env2.get_state()
    ev1, _ = env.get_events()
    ev2, _ = env2.get_events()
    return env, acts, ro, (torch.stack(ref_obs), torch.stack(ref_rew), torch.stack(ref_done)), (s1, s2), (ev1, ev2)


def test_rollout_equals_steps():
    """The persistent register-resident rollout (one launch for every swarm
    size, auto-reset crossing episode boundaries) reproduces T per-call steps."""
    sizes = [1, 2, 8, 64, 3, 33, 16, 5, 128] * 6
    _, _, ro, ref, (s1, s2), (ev1, ev2) = _rollout_vs_steps(sizes, 6, 12)
    for a, b in zip(ro, ref):
        assert torch.equal(a, b)
    for k in ("state", "params", "goals", "ep_step", "tick"):
        assert torch.equal(s1[k], s2[k]), k
    assert torch.equal(ev1, ev2)


@pytest.mark.parametrize("sizes,ws", [([8] * 64, False), ([1, 2, 8, 33, 64, 5] * 6, False),
                                      ([1, 2, 8, 33, 64, 5] * 6, True)])
def test_smooth_rollout_equals_steps(sizes, ws):
    """A smooth-contact handle (the general instance, with the pair penalty
    staged in every substep) gives the same bits in the rollout and in
    per-call steps, through the warp-specialised kernels (one or two dynamics
    warps per CTA) and the persistent one."""
    from paper_2306_09537_gb300 import qs
    feats = ("smooth", "dr", "motor_noise", "obs_noise", "collisions", "auto_reset")
    shape = (qs.QS_BLOCK_WARP_SPECIALISED, 0, 1) if ws else None
    _, acts, ro, ref, (s1, s2), (ev1, ev2) = _rollout_vs_steps(sizes, 6, 10, shape=shape, feats=feats, seed=9)
    for a, b in zip(ro, ref):
        assert torch.equal(a, b)
    for k in ("state", "params", "goals", "ep_step", "tick"):
        assert torch.equal(s1[k], s2[k]), k
    assert torch.equal(ev1, ev2)


@pytest.mark.parametrize("shape", [None, (1, 0, True), (1, 5, False), (1, 1, True), (64, 0, False)])
@pytest.mark.parametrize("extended", [False, True])
@pytest.mark.parametrize("widest", [32, 64])
def test_ws_rollout_equals_steps(shape, extended, widest):
    """Classes at most 64 wide: the warp-specialised persistent rollout (the
    default for such handles; noise and observation rows on as many noise
    warps as dynamics warps, one or two) reproduces per-call steps across
    auto-reset episodes, also with the scenario goals and downwash compiled
    in."""
    from paper_2306_09537_gb300 import qs
    sizes = [1, 2, 3, 5, 8, 13, 16, 31, 32] * 6 if widest == 32 else [1, 3, 8, 17, 33, 48, 64, 5, 32] * 4
    feats = FULL + ("auto_reset",) + (("downwash",) if extended else ())
    kw = dict(scenarios=("static", "swap", "pursuit_bezier", "swarm_vs_swarm")) if extended else {}
    env, _ = pair(sizes, 6, feats, seed=6, episode_steps=7, **kw)
    env2, _ = pair(sizes, 6, feats, seed=6, episode_steps=7, **kw)
    if shape is None:
        default_ws = widest == 32 and not extended
        assert (qs.qs_get_rollout_shape(env.h)[0] == qs.QS_BLOCK_WARP_SPECIALISED) == default_ws
        if not default_ws:
            qs.qs_set_rollout_shape(env.h, qs.QS_BLOCK_WARP_SPECIALISED, 0, 1)
    else:
        qs.qs_set_rollout_shape(env.h, *shape)
    T = 17
    acts = torch.from_numpy(W.actions(6, T, env.D)).to(DEV)
    obs = torch.empty(T, env.D, env.obs_dim, device=DEV)
    rew = torch.empty(T, env.D, device=DEV)
    done = torch.empty(T, env.E, dtype=torch.uint8, device=DEV)
    env.rollout(acts, obs, rew, done)
    for t in range(T):
        o2, r2, d2 = env2.step(acts[t])
        assert torch.equal(obs[t], o2) and torch.equal(rew[t], r2) and torch.equal(done[t], d2), t
    s1, s2 = env.get_state(), env2.get_state()
    for k in ("state", "params", "goals", "ep_step", "tick"):
        assert torch.equal(s1[k], s2[k]), k
    assert torch.equal(env.get_events()[0], env2.get_events()[0])
    if extended:
        assert torch.equal(env.get_scenario(), env2.get_scenario())


def test_ws_rollout_default_only_within_one_wave():
    """The warp-specialised rollout is the default only while its CTAs (one per
    32 drone lanes) fit one wave: a second wave would run the whole horizon
    again. 155,680 drones need 4,865 CTAs, more than 152 SMs x 32 resident
    CTAs could hold at any occupancy."""
    from paper_2306_09537_gb300 import qs
    from paper_2306_09537_gb300.env import QuadSwarmEnv
    for E, ws in ((4096, True), (152 * 32 * 32 + 32, False)):
        env = QuadSwarmEnv(E, 1, 0, ("floor", "walls", "motor_noise", "obs_noise", "dr"), seed=1, device=DEV)
        assert (qs.qs_get_rollout_shape(env.h)[0] == qs.QS_BLOCK_WARP_SPECIALISED) == ws, E
        env.close()


def test_per_call_default_shapes():
    """Per-call defaults: the warp-specialised step for narrow swarms while
    latency-bound; swarms of 17..32 only up to two CTAs per SM (here 4,096
    drones), beyond that one env per 32-thread CTA (32,768 drones); swarms of
    16 keep it at 32,768 drones."""
    from paper_2306_09537_gb300 import qs
    from paper_2306_09537_gb300.env import QuadSwarmEnv
    for E, N, expect in ((128, 32, qs.QS_BLOCK_WARP_SPECIALISED), (1024, 32, 32), (2048, 16, qs.QS_BLOCK_WARP_SPECIALISED)):
        env = QuadSwarmEnv(E, N, 6, ("floor", "walls", "collisions"), seed=1, device=DEV)
        assert qs.qs_get_block(env.h, N) == expect, (E, N)
        env.close()


def test_ws_rollout_needs_narrow_classes():
    from paper_2306_09537_gb300 import qs
    env, _ = pair([4, 65], 2, FULL, seed=1)
    assert qs.qs_get_rollout_shape(env.h)[0] != qs.QS_BLOCK_WARP_SPECIALISED
    with pytest.raises(qs.QSError):
        qs.qs_set_rollout_shape(env.h, qs.QS_BLOCK_WARP_SPECIALISED, 0, 1)


@pytest.mark.parametrize("shape", [(64, 0, True), (128, 5, True), (256, 3, False), (64, 1, False)])
def test_rollout_shape_does_not_change_results(shape):
    sizes = [1, 2, 8, 64, 4] * 5
    _, _, ro, ref, (s1, s2), _ = _rollout_vs_steps(sizes, 6, 9, shape=shape)
    for a, b in zip(ro, ref):
        assert torch.equal(a, b)
    assert torch.equal(s1["state"], s2["state"])


def test_rollout_graph_replay():
    """A second rollout with the same buffers replays the captured graph and
    continues the simulation exactly as per-call steps would."""
    from paper_2306_09537_gb300 import qs
    sizes = [8] * 40 + [1] * 64
    env, _ = pair(sizes, 6, FULL, seed=6)
    env2, _ = pair(sizes, 6, FULL, seed=6)
    T = 5
    acts = torch.from_numpy(W.actions(6, T, env.D)).to(DEV)
    obs = torch.empty(T, env.D, env.obs_dim, device=DEV)
    rew = torch.empty(T, env.D, device=DEV)
    for rep in range(3):
        env.rollout(acts, obs, rew, None)
        for t in range(T):
            o2, r2, _ = env2.step(acts[t])
            assert torch.equal(obs[t], o2) and torch.equal(rew[t], r2)
    assert qs.qs_get_rollout_shape(env.h)[2] is True
    assert torch.equal(env.get_state()["state"], env2.get_state()["state"])


@pytest.mark.parametrize("n", [1, 2, 3, 8, 20, 33, 64, 100])
def test_launch_shape_does_not_change_results(n):
    """The per-call kernel of a handle whose envs share one width class gives
    the same bits in every CTA shape (and warp-specialised where the class
    allows it)."""
    from paper_2306_09537_gb300 import qs
    WS = qs.QS_BLOCK_WARP_SPECIALISED
    wcls = 1 if n == 1 else int(2 ** np.ceil(np.log2(n)))
    sizes = [n] * max(4, 1536 // n)
    blocks = [b for b in (None, 32, 64, 128, 256, WS)
              if b is None or (b == WS and wcls <= 32) or (b != WS and b >= wcls and b % wcls == 0)]
    ref = None
    for block in blocks:
        env, _ = pair(sizes, 6, FULL, seed=8)
        if block:
            qs.qs_set_block(env.h, wcls, block)
            assert qs.qs_get_block(env.h, wcls) == block
        acts = torch.from_numpy(W.actions(8, 3, env.D)).to(DEV)
        for t in range(3):
            obs, rew, _ = env.step(acts[t])
        cur = (obs.clone(), rew.clone(), env.get_state()["state"])
        if ref is None:
            ref = cur
        else:
            assert all(torch.equal(a, b) for a, b in zip(ref, cur)), block


@pytest.mark.parametrize("sizes", [[1] * 100 + [8] * 40 + [3, 5, 2, 17, 32] * 7,
                                   [1] * 100 + [8] * 40 + [64] * 4 + [3, 5, 2] * 7 + [100, 128]])
def test_mixed_class_step_is_one_launch_in_any_rollout_shape(sizes):
    """A handle whose swarm sizes span several width classes steps them all in
    one launch of the rollout kernels (T = 1): the same bits through the
    persistent kernel in several CTA sizes and, where every class allows it,
    the warp-specialised one."""
    from paper_2306_09537_gb300 import qs
    WS = qs.QS_BLOCK_WARP_SPECIALISED
    shapes = [(128, 0, False), (256, 0, True)] + ([(WS, 0, False)] if max(sizes) <= 64 else [])
    ref = None
    for shape in shapes:
        env, _ = pair(sizes, 6, FULL + ("auto_reset",), seed=9, episode_steps=2)
        qs.qs_set_rollout_shape(env.h, *shape)
        acts = torch.from_numpy(W.actions(9, 4, env.D)).to(DEV)
        for t in range(4):  # across an auto-reset
            obs, rew, done = env.step(acts[t])
        cur = (obs.clone(), rew.clone(), done.clone(), env.get_state()["state"])
        if ref is None:
            ref = cur
        else:
            assert all(torch.equal(a, b) for a, b in zip(ref, cur)), shape


@pytest.mark.parametrize("n,K", [(1, 0), (8, 6), (48, 6)])
def test_uniform_geometry_matches_tile_tables(n, K):
    """With equal swarm sizes the kernels compute each tile, its envs and their
    first drones from the tile index; a handle whose last env differs in size
    reads them from the tile table, the permutation and the env offsets. The
    envs the two handles share give the same bits through every launch form:
    per-call (warp-specialised and general kernels) and rollouts
    (warp-specialised and persistent), across auto-resets."""
    from paper_2306_09537_gb300 import qs
    from paper_2306_09537_gb300.env import QuadSwarmEnv
    E = 3000 if n == 1 else 240
    last = 2 if n == 1 else n - 1
    feats = FULL + ("auto_reset",)
    sizes_b = np.array([n] * (E - 1) + [last], dtype=np.int32)
    Ds = (E - 1) * n
    st = W.random_states(9, E * n + 2)
    st[:Ds, 0:3] = W.clustered_positions(9, [n] * (E - 1), spread=0.12) if n > 1 else st[:Ds, 0:3]
    prm, goals = None, W.random_goals(9, E)
    envs = []
    for sizes in (n, sizes_b):
        env = QuadSwarmEnv(E, sizes, K, feats, seed=9, weights=ALL_WEIGHTS, device=DEV, episode_steps=4)
        if prm is None:
            prm = W.random_params(9, E, nominal(env))
        env.set_state(torch.from_numpy(np.ascontiguousarray(st[:env.D], np.float32)).to(DEV),
                      torch.from_numpy(prm.astype(np.float32)).to(DEV),
                      torch.from_numpy(goals.astype(np.float32)).to(DEV),
                      torch.zeros(E, dtype=torch.int32, device=DEV), torch.full((E,), 5, dtype=torch.int32, device=DEV))
        envs.append(env)
    a, b = envs
    wcls = 1 if n == 1 else int(2 ** np.ceil(np.log2(n)))

    def shared(env, obs, rew, done):
        return obs[..., :Ds, :], rew[..., :Ds], (None if done is None else done[..., :E - 1]), env.get_state()["state"][:Ds]

    T = 6
    acts = torch.from_numpy(W.actions(9, 4 * T, a.D + 2)).to(DEV)
    t = 0
    for block in (None, max(64, wcls)):  # per-call: default plan, then the general kernel
        if block:
            for env in envs:
                for w in ({1, 2} if env is b else {1}) if n == 1 else {wcls}:
                    qs.qs_set_block(env.h, w, block)
        for _ in range(T):
            ra = shared(a, *a.step(acts[t, :a.D].contiguous()))
            rb = shared(b, *b.step(acts[t, :b.D].contiguous()))
            assert all(torch.equal(x, y) for x, y in zip(ra, rb)), (block, t)
            t += 1
    shapes = ([(qs.QS_BLOCK_WARP_SPECIALISED, 0, False)] if wcls <= 64 else []) + [(max(128, wcls), 0, False)]
    for shape in shapes:
        outs = []
        for env in envs:
            qs.qs_set_rollout_shape(env.h, *shape)
            obs = torch.empty(T, env.D, env.obs_dim, device=DEV)
            rew = torch.empty(T, env.D, device=DEV)
            done = torch.empty(T, E, dtype=torch.uint8, device=DEV)
            env.rollout(acts[t:t + T, :env.D].contiguous(), obs, rew, done)
            outs.append(shared(env, obs, rew, done))
        assert all(torch.equal(x, y) for x, y in zip(*outs)), shape
        t += T
    for env in envs:
        env.close()


def test_auto_reset_matches_oracle():
    sizes = [4] * 50
    feats = FULL + ("auto_reset",)
    env, o = pair(sizes, 3, feats, seed=12, episode_steps=3)
    env.reset(12)
    o.reset(12)
    acts = W.actions(12, 4, env.D)
    for t in range(4):
        _, _, done = env.step(torch.from_numpy(acts[t]).to(DEV))
        _, _, odone = o.step(acts[t].astype(np.float64))
        assert np.array_equal(done.cpu().numpy(), odone)
    g = gpu_state(env)
    s = o.get_state()
    assert (g["ep_step"] == 1).all()
    assert np.allclose(g["params"], s["params"], rtol=2e-7)
    assert np.abs(g["goals"] - s["goals"]).max() < 2e-6


def test_misaligned_and_null_buffers_rejected():
    from paper_2306_09537_gb300 import qs
    env, _ = pair([1] * 8, 0, FULL, seed=1)
    buf = torch.zeros(8 * 4 + 1, device=DEV)
    with pytest.raises(qs.QSError) as ei:
        qs.qs_step(env.h, buf[1:])
    assert ei.value.status == qs.QS_ERR_ARG
    with pytest.raises(qs.QSError):
        qs.qs_step(env.h, None)
    with pytest.raises(qs.QSError):
        qs.qs_rollout(env.h, 0, buf[:32])


def test_nonfinite_state_reported_by_sync():
    """Failure detection without a GPU fault: a NaN planted in the state makes
    the step kernel raise the device status bit, which qs_sync reports."""
    from paper_2306_09537_gb300 import qs
    env, _ = pair([1] * 16, 0, FULL, seed=2)
    s = env.get_state()
    s["state"][3, 4] = float("nan")
    env.set_state(state=s["state"])
    env.step(torch.rand(16, 4, device=DEV))
    with pytest.raises(qs.QSError) as ei:
        env.sync()
    assert ei.value.status == qs.QS_ERR_STATE_NONFINITE
    env.reset(2)
    env.step(torch.rand(16, 4, device=DEV))
    env.sync()


# ----------------------------------------------------------------------------- full sizes
def _one_step_through(env, o, acts, path):
    """One control step of env through the per-call step or a one-step
    rollout in the given shape; returns the outputs as check_step wants."""
    from paper_2306_09537_gb300 import qs
    a = torch.from_numpy(acts).to(DEV)
    if path == "call":
        obs, rew, done = env.step(a)
    else:
        qs.qs_set_rollout_shape(env.h, *path)
        obs = torch.empty(1, env.D, env.obs_dim, device=DEV)
        rew = torch.empty(1, env.D, device=DEV)
        done = torch.empty(1, env.E, dtype=torch.uint8, device=DEV)
        env.rollout(a[None], obs, rew, done)
        obs, rew, done = obs[0], rew[0], done[0]
    ev, knn = env.get_events(knn=True)
    r = dict(obs=obs.cpu().numpy(), rew=rew.cpu().numpy(), done=done.cpu().numpy(),
             ev=ev.cpu().numpy().astype(np.uint32), knn=knn.cpu().numpy().astype(np.int32), g=gpu_state(env))
    r["oobs"], r["orew"], r["odone"] = o.step(acts.astype(np.float64), n_threads=8)
    r["oev"], r["oknn"], _ = o.get_events()
    r["margin"], r["margin_knn"] = o.margins()
    r["os"] = o.get_state()
    return r


@pytest.mark.parametrize("wl_name,path", [
    ("swarm_2048x8_k6", "call"), ("swarm_2048x8_k6", (1, 0, False)), ("swarm_2048x8_k6", (64, 0, True)),
    ("uneven_4096", "call"), ("uneven_4096", (64, 0, True)), ("uneven_4096", (128, 0, False)),
    ("uneven_4096", (1, 0, True)),  # warp-specialised rollout with two-warp pairs (swarms up to 64)
])
def test_full_size_one_step_parity(wl_name, path):
    """The swarm (2048 x 8, K = 6) and uneven (4096 envs, 40,408 drones)
    workloads at full size, from the method's reset state, through the per-call
    step and through one-step rollouts in the shapes the benchmark's autotuner
    chooses between: the one-step bars against the oracle."""
    wl = W.WORKLOADS[wl_name]
    sizes = wl.sizes()
    feats = FULL if "collisions" in wl.features else tuple(f for f in FULL if f != "collisions")
    env, o = pair(sizes, wl.k_neighbors, feats, seed=wl.seed, weights=ALL_WEIGHTS)
    o.reset(wl.seed)
    s0 = o.get_state()  # the oracle's own reset, rounded to binary32, goes to both sides
    set_both(env, o, s0["state"].astype(np.float32), s0["params"].astype(np.float32),
             s0["goals"].astype(np.float32), ep=3, tick=11)
    acts = W.actions(wl.seed, 1, env.D)[0]
    r = _one_step_through(env, o, acts, path)
    check_step(r, sizes)


def test_max_swarm_and_k_bit_exact_knn():
    """Swarms of the maximum size (128) with the maximum K (8) through the
    per-call step and the persistent rollout: neighbour lists bit-exact."""
    sizes = [128] * 24
    env, o = pair(sizes, 8, FULL, seed=17, weights=ALL_WEIGHTS)
    st, prm, goals = seeded_inputs(env, 17, sizes, spread=1.0)
    set_both(env, o, st, prm, goals, ep=3, tick=11)
    acts = W.actions(17, 1, env.D)[0]
    r = _one_step_through(env, o, acts, "call")
    check_step(r, sizes)
    set_both(env, o, st, prm, goals, ep=3, tick=11)
    r = _one_step_through(env, o, acts, (128, 0, True))
    check_step(r, sizes)
