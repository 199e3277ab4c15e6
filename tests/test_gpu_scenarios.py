"""Training scenarios (Sec. III-D) on the GPU against the FP64 oracle: the
scenario records drawn at a reset, every drone's goal over an episode (all
scenario types and formations, swarm sizes 1..128, across the switch step),
the observation and reward of steps that use those goals (warp-specialised,
general and persistent kernels), and records redrawn by auto-resets.

Records fed to both sides come from the oracle's own reset, rounded to
binary32. Integer fields (type, formations, switch step, seed) must agree
exactly; goals agree within the binary32 rounding of their formulas: 5e-6 m
for formations (offsets of a few metres), 3e-5 m for the Lissajous evader
(phase f tau T up to a few turns, times amplitudes up to 3.5 m) and 1e-5 m
for the Bezier evader.
"""
import numpy as np
import pytest
import torch

from gpu_helpers import ALL_WEIGHTS, DEV, env_of, gpu_state, pair, seeded_inputs, set_both
from oracle import oracle as O
from paper_2306_09537_gb300 import workloads as W

pytestmark = pytest.mark.gpu

ALL = tuple(O.SCN_NAMES)
SIZES = [1, 2, 3, 5, 8, 17, 33, 64, 100, 128] * 6
INT_FIELDS = [O.R_TYPE, O.R_F0, O.R_F1, O.R_TSW, O.R_SEED_LO, O.R_SEED_HI]
FEATS = ("floor", "walls", "motor_noise", "obs_noise", "dr", "collisions", "record_knn")


def goal_tolerance(rec):
    t = rec[:, O.R_TYPE].astype(int)
    tol = np.full(len(t), 5e-6)
    tol[t == O.SCN_NAMES.index("pursuit_lissajous")] = 3e-5
    tol[t == O.SCN_NAMES.index("pursuit_bezier")] = 1e-5
    return tol


def share_records(env, o):
    """The oracle's records, rounded to binary32, on both sides."""
    rec = o.get_scenario().astype(np.float32)
    o.set_scenario(rec.astype(np.float64))
    env.set_scenario(torch.from_numpy(rec).to(DEV))
    return rec


def set_ep(env, o, ep):
    ep = np.ascontiguousarray(ep, dtype=np.int32)
    env.set_state(ep_step=torch.from_numpy(ep).to(DEV))
    o.set_state(ep_step=ep)


@pytest.mark.parametrize("seed", [3, 11])
def test_reset_records_match_oracle(seed):
    env, o = pair(SIZES, 6, FEATS, seed=seed, scenarios=ALL)
    env.reset(seed)
    o.reset(seed)
    g = env.get_scenario().cpu().numpy()
    r = o.get_scenario()
    assert np.array_equal(g[:, INT_FIELDS], r[:, INT_FIELDS])
    assert np.allclose(g, r, rtol=1e-6, atol=1e-6)
    assert len(np.unique(r[:, O.R_TYPE])) == 8
    # only-single handles draw nothing
    env1, _ = pair([4] * 3, 2, FEATS, seed=seed, scenarios=("single",))
    env1.reset(seed)
    assert env1.get_scenario().abs().max().item() == 0.0


def test_goals_match_oracle_over_the_episode():
    env, o = pair(SIZES, 6, FEATS, seed=5, scenarios=ALL)
    env.reset(5)
    o.reset(5)
    rec = share_records(env, o)
    tsw = rec[:, O.R_TSW].astype(np.int32)
    tol = goal_tolerance(rec)[env_of(SIZES)]
    rng = np.random.default_rng(0)
    schedules = [np.zeros(len(SIZES)), tsw - 1, tsw, tsw + 1, np.full(len(SIZES), 1499)]
    schedules += [rng.integers(0, 1500, len(SIZES)) for _ in range(6)]
    for ep in schedules:
        set_ep(env, o, ep)
        g = env.get_goals().cpu().numpy()
        want = o.goals()
        err = np.abs(g - want).max(axis=1)
        assert (err <= tol).all(), (err.max(), np.argmax(err - tol))


@pytest.mark.parametrize("kind", ["swap", "swarm_vs_swarm", "dynamic", "pursuit_bezier"])
def test_step_parity_across_the_switch(kind):
    """One step from identical inputs whose episode step reaches the switch
    step exactly: observation rows (x - goal) and rewards match the oracle."""
    from test_gpu_step import check_step
    sizes = [2, 3, 8, 17, 32, 64, 128] * 4
    env, o = pair(sizes, 6, FEATS, seed=9, weights=ALL_WEIGHTS, scenarios=(kind,))
    env.reset(9)
    o.reset(9)
    rec = share_records(env, o)
    st, prm, goals = seeded_inputs(env, 9, sizes, spread=1.0)
    set_both(env, o, st, prm, goals, ep=0, tick=11)
    set_ep(env, o, rec[:, O.R_TSW].astype(np.int32) - 1)
    acts = W.actions(9, 1, env.D)[0]
    obs, rew, done = env.step(torch.from_numpy(acts).to(DEV))
    ev, knn = env.get_events(knn=True)
    r = dict(obs=obs.cpu().numpy(), rew=rew.cpu().numpy(), done=done.cpu().numpy(),
             ev=ev.cpu().numpy().astype(np.uint32), knn=knn.cpu().numpy().astype(np.int32), g=gpu_state(env))
    r["oobs"], r["orew"], r["odone"] = o.step(acts.astype(np.float64))
    r["oev"], r["oknn"], _ = o.get_events()
    r["margin"], r["margin_knn"] = o.margins()
    r["os"] = o.get_state()
    check_step(r, sizes)
    # the goals in the observation are the post-switch ones
    assert np.allclose(r["g"]["state"][:, 0:3] - r["obs"][:, 0:3], o.goals(), atol=2e-2)


def test_rollout_with_auto_reset_redraws_records():
    """A persistent rollout over several short episodes: records redrawn at
    every auto-reset equal the oracle's, the rollout equals per-step calls,
    and the goals at the end agree."""
    sizes = [1, 3, 8, 17, 64, 128] * 3
    feats = FEATS + ("auto_reset",)
    T, ep_len = 23, 7
    env, o = pair(sizes, 6, feats, seed=13, scenarios=ALL, episode_steps=ep_len)
    env2, _ = pair(sizes, 6, feats, seed=13, scenarios=ALL, episode_steps=ep_len)
    for e_ in (env, env2):
        e_.reset(13)
    o.reset(13)
    acts = torch.from_numpy(W.actions(13, T, env.D)).to(DEV)
    obs_r = torch.empty(T, env.D, env.obs_dim, device=DEV)
    rew_r = torch.empty(T, env.D, device=DEV)
    done_r = torch.empty(T, env.E, dtype=torch.uint8, device=DEV)
    env.rollout(acts, obs_r, rew_r, done_r)
    for t in range(T):
        ob, rw, dn = env2.step(acts[t])
        assert torch.equal(ob, obs_r[t]) and torch.equal(rw, rew_r[t]) and torch.equal(dn, done_r[t])
        o.step(acts[t].cpu().numpy().astype(np.float64), want_obs=False)
    g1, g2 = env.get_scenario().cpu().numpy(), env2.get_scenario().cpu().numpy()
    assert np.array_equal(g1, g2)
    r = o.get_scenario()
    assert np.array_equal(g1[:, INT_FIELDS], r[:, INT_FIELDS])
    assert np.allclose(g1, r, rtol=1e-6, atol=1e-6)
    assert torch.equal(env.get_goals(), env2.get_goals())
    assert np.array_equal(env.get_state()["ep_step"].cpu().numpy(), o.get_state()["ep_step"])
    # goals at the final step, on the oracle's own (binary32-rounded) records
    share_records(env, o)
    tol = goal_tolerance(r)[env_of(sizes)]
    assert (np.abs(env.get_goals().cpu().numpy() - o.goals()).max(axis=1) <= tol).all()


def test_diff_refuses_scenarios():
    from paper_2306_09537_gb300 import qs
    env, _ = pair([2] * 4, 1, ("smooth", "floor"), seed=1, scenarios=("static",))
    with pytest.raises(qs.QSError) as e:
        qs.qs_diff_forward(env.h, 4, 2, torch.zeros(8, 30, device=DEV), torch.zeros(4, 8, 4, device=DEV),
                           torch.zeros(8, device=DEV), torch.zeros(1 << 16, dtype=torch.uint8, device=DEV))
    assert e.value.status == qs.QS_ERR_UNSUPPORTED


@pytest.mark.parametrize("scenarios", [(), ALL])
def test_partial_reset_matches_oracle(scenarios):
    """qs_reset with an env mask after a few steps: the masked envs are
    redrawn from key `seed` at their current Philox counter (parameters, goal,
    scenario record, drones, episode step 0), the others keep their state and
    counters, and the observation of every env follows (sensor-noise substream
    1). Compared with the oracle's masked reset."""
    sizes = [1, 2, 3, 8, 17, 32, 64, 128] * 3
    env, o = pair(sizes, 6, FEATS, seed=31, scenarios=scenarios)
    env.reset(31)
    o.reset(31)
    if scenarios:
        share_records(env, o)
    st, prm, goals = seeded_inputs(env, 31, sizes, spread=1.0)
    set_both(env, o, st, prm, goals, ep=5, tick=9)
    for t in range(3):
        a = W.actions(31 + t, 1, env.D)[0]
        env.step(torch.from_numpy(a).to(DEV))
        o.step(a.astype(np.float64), want_obs=False)
    mask = (np.arange(len(sizes)) % 3 != 1).astype(np.uint8)
    obs = env.reset(77, torch.from_numpy(mask).to(DEV)).clone()
    o.reset(77, mask)
    g, s = gpu_state(env), o.get_state()
    redrawn = mask.astype(bool)
    eo = env_of(sizes)
    dr = redrawn[eo]
    # redrawn envs: the draw of a reset (binary32 vs binary64 arithmetic)
    assert np.allclose(g["params"][redrawn], s["params"][redrawn], rtol=2e-7, atol=0)
    assert np.abs(g["goals"][redrawn] - s["goals"][redrawn]).max() < 2e-6
    assert np.abs(g["state"][dr, 0:18] - s["state"][dr, 0:18]).max() < 2e-6
    assert np.allclose(g["state"][dr, 18:30], s["state"][dr, 18:30], rtol=2e-7, atol=0)
    assert (g["ep_step"][redrawn] == 0).all()
    # counters: a masked reset keeps every env's Philox counter
    assert np.array_equal(g["tick"].astype(np.uint32), s["tick"])
    assert np.array_equal(g["ep_step"], s["ep_step"])
    if scenarios:
        gr, orr = env.get_scenario().cpu().numpy(), o.get_scenario()
        assert np.array_equal(gr[redrawn][:, INT_FIELDS], orr[redrawn][:, INT_FIELDS])
        assert np.allclose(gr[redrawn], orr[redrawn], rtol=1e-6, atol=1e-6)
        assert np.array_equal(gr[~redrawn], orr[~redrawn].astype(np.float32))
    # the reset observation of the redrawn envs (the others' drift is chaotic)
    oobs = o.observe()
    assert np.allclose(obs.cpu().numpy()[dr], oobs[dr], rtol=1e-5, atol=2e-5)
