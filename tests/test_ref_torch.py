"""Pins of the torch-autograd FP64 reference of the smooth step (CPU): its
forward equals the C oracle's smooth form, and its autograd gradient equals
central finite differences of the C oracle."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from oracle.ref_step_torch import smooth_rollout_loss
from paper_2306_09537_gb300 import workloads as W

SIZES = [3, 2]
T = 6


def setup_case(seed=3):
    E, D = len(SIZES), sum(SIZES)
    c = O.default_config(n_envs=E, k_neighbors=0, flags=O.F_SMOOTH, seed=seed)
    nominal = [c.mass, c.ixx, c.iyy, c.izz, c.t2w, c.tau_m, c.arm]
    st = W.random_states(seed, D).astype(np.float64)
    st[:, 0:3] = W.clustered_positions(seed, SIZES, spread=0.05).astype(np.float64)
    st[0, 0] = 4.98  # one drone pressing a wall, one near the floor
    st[3, 2] = 0.01
    prm = W.random_params(seed, E, nominal).astype(np.float64)
    goals = W.random_goals(seed, E).astype(np.float64)
    acts = W.actions(seed, T, D, lo=0.05, hi=0.95).astype(np.float64)
    cfg = {k: getattr(c, k) for k in ("dt", "gravity", "alpha_ns_frac", "alpha_nd", "smooth_kc", "smooth_beta",
                                      "kappa", "room_hx", "room_hy", "room_h", "omega_max", "substeps")}
    return c, st, prm, goals, acts, cfg


def oracle_loss(c, st, prm, goals, acts):
    o = O.Oracle(c, SIZES)
    o.set_state(st, prm, goals, np.zeros(len(SIZES), np.int32), np.zeros(len(SIZES), np.uint32))
    loss = np.zeros(o.D)
    for t in range(acts.shape[0]):
        o.step(acts[t], want_obs=False, want_loss=True, loss=loss)
    return loss


def test_reference_forward_equals_oracle():
    c, st, prm, goals, acts, cfg = setup_case()
    want = oracle_loss(c, st, prm, goals, acts)
    got = smooth_rollout_loss(torch.tensor(st), torch.tensor(acts), torch.tensor(prm), torch.tensor(goals), SIZES,
                              cfg).numpy()
    assert np.allclose(got, want, rtol=1e-11, atol=1e-12)


def test_reference_gradient_equals_oracle_finite_differences():
    c, st, prm, goals, acts, cfg = setup_case()
    x0 = torch.tensor(st, requires_grad=True)
    a = torch.tensor(acts, requires_grad=True)
    L = smooth_rollout_loss(x0, a, torch.tensor(prm), torch.tensor(goals), SIZES, cfg).sum()
    L.backward()
    rng = np.random.default_rng(0)
    h = 1e-6
    checks = [("x", int(d), int(k)) for d, k in zip(rng.integers(0, 5, 12), rng.integers(0, 26, 12))]
    checks += [("a", int(t), int(i)) for t, i in zip(rng.integers(0, T, 12), rng.integers(0, 20, 12))]
    for kind, p, q in checks:
        sp, sm_, ap, am = st.copy(), st.copy(), acts.copy(), acts.copy()
        if kind == "x":
            sp[p, q] += h
            sm_[p, q] -= h
            g = x0.grad[p, q].item()
        else:
            ap[p].reshape(-1)[q] += h
            am[p].reshape(-1)[q] -= h
            g = a.grad[p].reshape(-1)[q].item()
        fd = (oracle_loss(c, sp, prm, goals, ap).sum() - oracle_loss(c, sm_, prm, goals, am).sum()) / (2 * h)
        assert abs(g - fd) <= 1e-5 * max(1.0, abs(fd)), (kind, p, q, g, fd)


# ----------------------------------------------------------------------------- discrete contacts
DSIZES = [3, 4]
DT = 12


def discrete_case(seed=28, event_time=False):
    """Env 0: one drone falls onto the floor (hit, then resting with
    friction), one flies into the +x wall, one catches up with it and
    collides; env 1: four drones packed closely enough to collide."""
    from oracle.ref_step_torch import discrete_rollout_loss  # noqa: F401
    E, D = len(DSIZES), sum(DSIZES)
    flags = O.F_FLOOR | O.F_WALLS | O.F_COLLISIONS | (O.F_EVENT_TIME if event_time else 0)
    c = O.default_config(n_envs=E, k_neighbors=0, flags=flags, seed=seed)
    O.set_config(c, coll_sigma_v=0.0, coll_sigma_w=0.0)
    nominal = [c.mass, c.ixx, c.iyy, c.izz, c.t2w, c.tau_m, c.arm]
    st = W.random_states(seed, D, rate=0.5).astype(np.float64)
    st[0, 0:6] = [0.0, 0.0, 0.02, 0.3, -0.2, -1.5]
    st[1, 0:6] = [4.965, 1.0, 5.0, 1.0, 0.0, 0.0]
    st[2, 0:6] = [4.852, 1.0, 5.0, 2.6, 0.0, 0.0]
    st[3:7, 0:3] = W.clustered_positions(seed, [4], spread=0.05).astype(np.float64) + [0.0, 0.0, 3.0]
    prm = W.random_params(seed, E, nominal).astype(np.float64)
    goals = W.random_goals(seed, E).astype(np.float64)
    acts = W.actions(seed, DT, D, lo=0.2, hi=0.8).astype(np.float64)
    cfg = {k: getattr(c, k) for k in ("dt", "gravity", "kappa", "room_hx", "room_hy", "room_h", "omega_max",
                                      "substeps", "mu", "alpha_c")}
    cfg.update(floor=True, walls=True, collisions=True, event_time=event_time)
    return c, st, prm, goals, acts, cfg


def oracle_run_discrete(c, st, prm, goals, acts):
    o = O.Oracle(c, DSIZES)
    o.set_state(st, prm, goals, np.zeros(len(DSIZES), np.int32), np.zeros(len(DSIZES), np.uint32))
    loss = np.zeros(o.D)
    evs, margin = [], np.inf
    for t in range(acts.shape[0]):
        o.step(acts[t], want_obs=False, want_loss=True, loss=loss)
        ev, _, mg = o.get_events()
        evs.append(ev.copy())
        margin = min(margin, mg.min())
        o.clear_margin()
    return loss, np.array(evs), margin


@pytest.mark.parametrize("event_time", [False, True])
def test_discrete_reference_forward_and_events_equal_oracle(event_time):
    from oracle.ref_step_torch import discrete_rollout_loss
    c, st, prm, goals, acts, cfg = discrete_case(event_time=event_time)
    want, oev, margin = oracle_run_discrete(c, st, prm, goals, acts)
    evs = []
    got = discrete_rollout_loss(torch.tensor(st), torch.tensor(acts), torch.tensor(prm), torch.tensor(goals),
                                DSIZES, cfg, events=evs).numpy()
    assert margin > 1e-6  # no decision within binary64 rounding of its threshold
    assert np.array_equal(np.array(evs).astype(np.uint32), oev)
    seen = int(np.bitwise_or.reduce(oev.ravel()))
    for bit in (O.EV_HIT_FLOOR, O.EV_ON_FLOOR, O.EV_HIT_WALL, O.EV_HIT_QUAD):
        assert seen & bit, bit
    assert np.allclose(got, want, rtol=1e-11, atol=1e-12)


@pytest.mark.parametrize("event_time", [False, True])
def test_discrete_reference_gradient_equals_oracle_finite_differences(event_time):
    """Every command and initial-state entry: autograd of the reference
    against central differences of the C oracle (h = 1e-6), where the
    differences at h and 2h agree (a perturbation that flips a contact
    decision makes the loss jump; such coordinates are left out)."""
    from oracle.ref_step_torch import discrete_rollout_loss
    c, st, prm, goals, acts, cfg = discrete_case(event_time=event_time)
    x0 = torch.tensor(st, requires_grad=True)
    a = torch.tensor(acts, requires_grad=True)
    discrete_rollout_loss(x0, a, torch.tensor(prm), torch.tensor(goals), DSIZES, cfg).sum().backward()

    def fd(sp, ap, h):
        def L(s_, a_):
            return oracle_run_discrete(c, s_, prm, goals, a_)[0].sum()
        return (L(*sp(h)) - L(*sp(-h))) / (2 * h) if ap is None else (L(*ap(h)) - L(*ap(-h))) / (2 * h)

    got, ref, ok = [], [], []
    for d in range(sum(DSIZES)):
        for k in range(26):
            def sp(h, d=d, k=k):
                s2 = st.copy()
                s2[d, k] += h
                return s2, acts
            f1, f2 = fd(sp, None, 1e-6), fd(sp, None, 2e-6)
            got.append(x0.grad[d, k].item()), ref.append(f1), ok.append(abs(f1 - f2) <= 1e-4 * (1 + abs(f1)))
    rng = np.random.default_rng(1)
    for t, d, r in zip(rng.integers(0, DT, 40), rng.integers(0, sum(DSIZES), 40), rng.integers(0, 4, 40)):
        def ap(h, t=t, d=d, r=r):
            a2 = acts.copy()
            a2[t, d, r] += h
            return st, a2
        f1, f2 = fd(None, ap, 1e-6), fd(None, ap, 2e-6)
        got.append(a.grad[t, d, r].item()), ref.append(f1), ok.append(abs(f1 - f2) <= 1e-4 * (1 + abs(f1)))
    got, ref, ok = np.array(got), np.array(ref), np.array(ok)
    assert ok.mean() >= 0.95
    scale = np.abs(ref[ok]).max()
    assert np.all(np.abs(got[ok] - ref[ok]) <= 1e-5 * np.abs(ref[ok]) + 1e-7 * scale), \
        np.abs(got[ok] - ref[ok]).max() / scale


def test_event_time_contacts_move_the_map():
    """The event-time contacts change the step where a contact happens: the
    falling drone's horizontal position after its floor hit and the
    wall-hitting and colliding drones' positions differ from the sampled
    contacts, and the gradients of the loss with respect to the falling
    drone's initial height and vertical speed gain the crossing-time term
    (the sampled floor reset passes nothing through it)."""
    from oracle.ref_step_torch import discrete_rollout_loss
    out = {}
    for et in (False, True):
        c, st, prm, goals, acts, cfg = discrete_case(event_time=et)
        x0 = torch.tensor(st, requires_grad=True)
        L = discrete_rollout_loss(x0, torch.tensor(acts), torch.tensor(prm), torch.tensor(goals), DSIZES, cfg)
        L.sum().backward()
        out[et] = (L.detach().numpy(), x0.grad.numpy().copy())
    dl = np.abs(out[True][0] - out[False][0])
    assert (dl[:3] > 1e-6).all()             # every contact of env 0 moved the trajectory
    g0, g1 = out[False][1], out[True][1]
    for k in (2, 5):  # z0 and v_z0 of the drone that lands
        assert abs(g1[0, k] - g0[0, k]) > 1e-2 * max(abs(g0[0, k]), 1e-3), (k, g0[0, k], g1[0, k])


def test_event_time_gradient_conditioning():
    """The crossing-time terms make the event-time gradient worse conditioned
    than the sampled one: on a colliding swarm of 8 (contact_swarm_states,
    seed 56, env 7: its step 24 holds a shallow pair contact) over 25 steps,
    perturbing the initial state by relative amounts of binary32 rounding
    (1e-7) moves the event-time gradient several times more than the sampled
    one. This is the measured reason for the GPU test's wider bar on the
    event-time adjoint (1e-3 relative instead of 1e-4), which still leaves
    an order of magnitude above the spread measured here."""
    from oracle.ref_step_torch import discrete_rollout_loss
    seed, E, N, T = 56, 8, 8, 25
    c = O.default_config(n_envs=1, k_neighbors=0, flags=O.F_COLLISIONS, seed=seed)
    nominal = [c.mass, c.ixx, c.iyy, c.izz, c.t2w, c.tau_m, c.arm]
    st = W.contact_swarm_states(seed, E, N).astype(np.float64)[56:64]
    prm = W.random_params(seed, E, nominal).astype(np.float64)[7:8]
    goals = W.random_goals(seed, E).astype(np.float64)[7:8]
    acts = W.actions(seed, 32, E * N, lo=0.2, hi=0.8).astype(np.float64)[:T, 56:64]
    cfg = {k: getattr(c, k) for k in ("dt", "gravity", "kappa", "room_hx", "room_hy", "room_h", "omega_max",
                                      "substeps", "mu", "alpha_c")}
    cfg.update(coll_sigma=0.0, floor=False, walls=False, collisions=True)
    rng = np.random.default_rng(0)
    pert = [rng.uniform(-1.0, 1.0, st.shape) * 1e-7 for _ in range(3)]
    spread = {}
    for et in (False, True):
        cfg["event_time"] = et
        gs = []
        for k in range(4):
            x0 = torch.tensor(st * (1.0 + (pert[k - 1] if k else 0.0)), requires_grad=True)
            discrete_rollout_loss(x0, torch.tensor(acts), torch.tensor(prm), torch.tensor(goals), [N],
                                  cfg).sum().backward()
            gs.append(x0.grad.numpy()[:, :26].copy())
        scale = np.abs(gs[0]).max()
        spread[et] = max(np.abs(g - gs[0]).max() for g in gs[1:]) / scale
    assert spread[True] > 3.0 * spread[False], spread
    assert spread[True] < 1e-4, spread  # the GPU bar (1e-3 relative, 1e-4 of the largest) is 10x wider
