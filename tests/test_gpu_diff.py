"""The differentiable rollout on the GPU: forward loss against the FP64 oracle,
hand-written adjoint against central finite differences of the oracle and
against torch.autograd through the FP64 torch reference, independence of the
checkpoint interval, and the autograd.Function wrapper."""
import numpy as np
import pytest
import torch

from gpu_helpers import DEV, nominal, pair
from oracle import oracle as O
from oracle.ref_step_torch import discrete_rollout_loss, smooth_rollout_loss
from paper_2306_09537_gb300 import qs
from paper_2306_09537_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def setup(sizes, T, seed, features=("smooth",), spread=0.06):
    env, o = pair(sizes, 0, features, seed=seed)
    E, D = env.E, env.D
    st = W.random_states(seed, D, rate=1.0)
    st[:, 0:3] = W.clustered_positions(seed, sizes, spread=spread)
    prm = W.random_params(seed, E, nominal(env))
    goals = W.random_goals(seed, E)
    z = np.zeros(E, np.int32)
    env.set_state(params=torch.from_numpy(prm).to(DEV), goals=torch.from_numpy(goals).to(DEV),
                  ep_step=torch.from_numpy(z).to(DEV), tick=torch.from_numpy(z).to(DEV))
    acts = W.actions(seed, T, D, lo=0.05, hi=0.95)
    return env, o, st, prm, goals, acts


def gpu_grads(env, st, acts, C):
    T, D = acts.shape[0], env.D
    x0 = torch.from_numpy(st).to(DEV)
    a = torch.from_numpy(acts).to(DEV)
    ws = torch.empty(qs.qs_diff_workspace_size(env.h, T, C), dtype=torch.uint8, device=DEV)
    loss = torch.empty(D, device=DEV)
    qs.qs_diff_forward(env.h, T, C, x0, a, loss, ws)
    ga = torch.empty_like(a)
    gx = torch.empty(D, 30, device=DEV)
    qs.qs_diff_backward(env.h, T, C, a, torch.ones(D, device=DEV), ws, ga, gx)
    env.sync()
    return loss.cpu().numpy(), ga.cpu().numpy().astype(np.float64), gx.cpu().numpy().astype(np.float64)


def oracle_total(o, st, prm, goals, acts):
    E = len(prm)
    o.set_state(st, prm, goals, np.zeros(E, np.int32), np.zeros(E, np.uint32))
    loss = np.zeros(o.D)
    for t in range(acts.shape[0]):
        o.step(acts[t], want_obs=False, want_loss=True, loss=loss)
    return loss


def test_forward_loss_matches_oracle():
    sizes = [8] * 64
    env, o, st, prm, goals, acts = setup(sizes, 32, 11, features=("smooth", "motor_noise", "dr"))
    loss, _, _ = gpu_grads(env, st, acts, 8)
    want = oracle_total(o, st.astype(np.float64), prm.astype(np.float64), goals.astype(np.float64),
                        acts.astype(np.float64))
    assert np.allclose(loss, want, rtol=1e-4, atol=1e-4)


def test_adjoint_matches_oracle_finite_differences():
    """1 env x 2 drones x 16 steps, motor noise on, checkpoints every 4 steps:
    every command and every initial-state entry against central differences
    (h = 1e-6) of the FP64 oracle; tolerance 1e-3 relative or 1e-5 of the
    largest gradient entry."""
    sizes = [2]
    T, C = 16, 4
    env, o, st, prm, goals, acts = setup(sizes, T, 21, features=("smooth", "motor_noise"), spread=0.04)
    _, ga, gx = gpu_grads(env, st, acts, C)
    st64, prm64, g64, a64 = (v.astype(np.float64) for v in (st, prm, goals, acts))
    h = 1e-6
    fd_a = np.zeros_like(a64)
    for t in range(T):
        for d in range(2):
            for r in range(4):
                ap, am = a64.copy(), a64.copy()
                ap[t, d, r] += h
                am[t, d, r] -= h
                fd_a[t, d, r] = (oracle_total(o, st64, prm64, g64, ap).sum() -
                                 oracle_total(o, st64, prm64, g64, am).sum()) / (2 * h)
    fd_x = np.zeros((2, 30))
    for d in range(2):
        for k in range(26):
            sp, sm_ = st64.copy(), st64.copy()
            sp[d, k] += h
            sm_[d, k] -= h
            fd_x[d, k] = (oracle_total(o, sp, prm64, g64, a64).sum() -
                          oracle_total(o, sm_, prm64, g64, a64).sum()) / (2 * h)
    for g, fd in ((ga, fd_a), (gx[:, :26], fd_x[:, :26])):
        scale = np.abs(fd).max()
        assert np.all(np.abs(g - fd) <= 1e-3 * np.abs(fd) + 1e-5 * scale), np.abs(g - fd).max() / scale
    assert np.all(gx[:, 26:] == 0)


def close_to_reference(g, ref, rel=1e-4, frac=1e-5):
    """Every entry within rel of itself or frac of the largest reference entry
    (binary32 arithmetic over the rollout against binary64)."""
    scale = np.abs(ref).max()
    err = np.abs(g - ref)
    tol = rel * np.abs(ref) + frac * scale
    ok = err <= tol
    i = np.unravel_index(np.argmax(err / tol), err.shape)
    return bool(ok.all()), f"worst err/tol {float((err / tol)[i]):.3g} at {i}: got {g[i]:.6g}, reference {ref[i]:.6g}, " \
                           f"{int((~ok).sum())} of {ok.size} entries out"


def test_adjoint_matches_torch_autograd_reference():
    """8 envs x 8 drones x 32 steps (pairs interacting), checkpoints every 8:
    within 1e-4 relative (or 1e-5 of the largest entry)."""
    sizes = [8] * 8
    T, C = 32, 8
    env, o, st, prm, goals, acts = setup(sizes, T, 5, features=("smooth",))
    _, ga, gx = gpu_grads(env, st, acts, C)
    p = env.cfg.params
    cfg = {"dt": env.cfg.dt, "gravity": p.gravity, "alpha_ns_frac": p.alpha_ns_frac, "alpha_nd": p.alpha_nd,
           "smooth_kc": p.smooth_kc, "smooth_beta": p.smooth_beta, "kappa": p.kappa, "room_hx": p.room_hx,
           "room_hy": p.room_hy, "room_h": p.room_h, "omega_max": p.omega_max, "substeps": env.cfg.substeps}
    cfg = {k: float(v) if k != "substeps" else int(v) for k, v in cfg.items()}
    x0 = torch.tensor(st.astype(np.float64), requires_grad=True)
    a = torch.tensor(acts.astype(np.float64), requires_grad=True)
    L = smooth_rollout_loss(x0, a, torch.tensor(prm.astype(np.float64)), torch.tensor(goals.astype(np.float64)),
                            sizes, cfg).sum()
    L.backward()
    for g, ref in ((ga, a.grad.numpy()), (gx[:, :26], x0.grad.numpy()[:, :26])):
        ok, worst = close_to_reference(g, ref)
        assert ok, worst


@pytest.mark.parametrize("features", [("smooth",), ("floor", "walls", "collisions")])
def test_wide_swarms_adjoint(features):
    """Swarms of 128 and 64 drones (the adjoint's two warp groups then span
    several warps each and meet at named barriers) next to a small one:
    forward loss against the FP64 oracle, gradients independent of the
    checkpoint interval (one segment, or several pipelined), and, for the
    smooth contacts, against torch.autograd through the FP64 reference."""
    sizes = [128, 64, 3]
    T = 12
    env, o, st, prm, goals, acts = setup(sizes, T, 31, features=features, spread=0.3)
    loss, ga, gx = gpu_grads(env, st, acts, 3)
    want = oracle_total(o, st.astype(np.float64), prm.astype(np.float64), goals.astype(np.float64),
                        acts.astype(np.float64))
    assert np.allclose(loss, want, rtol=1e-4, atol=1e-4)
    _, ga1, gx1 = gpu_grads(env, st, acts, T)
    assert np.array_equal(ga, ga1) and np.array_equal(gx, gx1)
    if "smooth" in features:
        p = env.cfg.params
        cfg = {"dt": env.cfg.dt, "gravity": p.gravity, "alpha_ns_frac": p.alpha_ns_frac, "alpha_nd": p.alpha_nd,
               "smooth_kc": p.smooth_kc, "smooth_beta": p.smooth_beta, "kappa": p.kappa, "room_hx": p.room_hx,
               "room_hy": p.room_hy, "room_h": p.room_h, "omega_max": p.omega_max, "substeps": env.cfg.substeps}
        cfg = {k: float(v) if k != "substeps" else int(v) for k, v in cfg.items()}
        x0 = torch.tensor(st.astype(np.float64), requires_grad=True)
        a = torch.tensor(acts.astype(np.float64), requires_grad=True)
        L = smooth_rollout_loss(x0, a, torch.tensor(prm.astype(np.float64)), torch.tensor(goals.astype(np.float64)),
                                sizes, cfg).sum()
        L.backward()
        for g, ref in ((ga, a.grad.numpy()), (gx[:, :26], x0.grad.numpy()[:, :26])):
            ok, worst = close_to_reference(g, ref)
            assert ok, worst


@pytest.mark.parametrize("features", [("smooth", "motor_noise", "dr"),
                                      ("floor", "walls", "collisions", "motor_noise", "dr")])
def test_diff_forward_runs_the_steps_dynamics(features):
    """The differentiable forward steps the step's own dynamics: its state
    checkpoint after C control steps equals, bit for bit, the state a rollout
    reaches from the same initial state, parameters, goals and commands
    (position, velocity, attitude, body rates, motor speeds, motor noise; the
    previous-command entries, which only the step's reward reads, excluded)."""
    from paper_2306_09537_gb300 import qs as Q
    sizes = [8] * 16 + [3, 1, 17, 32]
    T, C = 8, 4
    env, _, st, prm, goals, acts = setup(sizes, T, 31, features=features)
    x0 = torch.from_numpy(st).to(DEV)
    a = torch.from_numpy(acts).to(DEV)
    ws = torch.empty(Q.qs_diff_workspace_size(env.h, T, C), dtype=torch.uint8, device=DEV)
    loss = torch.empty(env.D, device=DEV)
    Q.qs_diff_forward(env.h, T, C, x0, a, loss, ws)
    env.sync()
    nplane, D = 9, env.D  # checkpoints lead the workspace: [T / C][9 float4 planes][D]
    ck = ws.view(torch.float32)[: (T // C) * nplane * D * 4].reshape(T // C, nplane, D, 4)
    ck1 = ck[1].permute(1, 0, 2).reshape(D, nplane * 4).cpu().numpy()
    env2, _ = pair(sizes, 0, features, seed=31)
    z = torch.zeros(env2.E, dtype=torch.int32, device=DEV)
    env2.set_state(x0, torch.from_numpy(prm).to(DEV), torch.from_numpy(goals).to(DEV), z, z)
    env2.rollout(a[:C].contiguous(), None, None, None)
    s2 = env2.get_state()["state"].cpu().numpy()
    assert np.array_equal(ck1[:, 0:26], s2[:, 0:26])


def test_checkpoint_interval_does_not_change_gradients():
    sizes = [8] * 16 + [3] * 8
    T = 24
    env, o, st, prm, goals, acts = setup(sizes, T, 9, features=("smooth", "motor_noise"))
    ref = gpu_grads(env, st, acts, T)
    for C in (1, 5, 8):
        got = gpu_grads(env, st, acts, C)
        for x, y in zip(got, ref):
            assert np.array_equal(x, y)


def test_rollout_fn_autograd():
    from paper_2306_09537_gb300.env import RolloutFn
    sizes = [8] * 32
    T = 20
    env, o, st, prm, goals, acts = setup(sizes, T, 13, features=("smooth", "motor_noise"))
    a = torch.from_numpy(acts).to(DEV).requires_grad_(True)
    x0 = torch.from_numpy(st).to(DEV).requires_grad_(True)
    loss = RolloutFn.apply(a, x0, env, 8)
    (2.0 * loss.sum()).backward()
    _, ga, gx = gpu_grads(env, st, acts, 8)
    assert np.allclose(a.grad.cpu().numpy(), 2.0 * ga, rtol=0, atol=0)
    assert np.allclose(x0.grad.cpu().numpy(), 2.0 * gx, rtol=0, atol=0)


def test_diff_rejects_bad_horizons():
    env, _ = pair([1] * 4, 0, ("floor",), seed=1)
    with pytest.raises(qs.QSError):
        qs.qs_diff_forward(env.h, 0, 2, torch.zeros(4, 30, device=DEV), torch.zeros(1, 4, 4, device=DEV),
                           torch.zeros(4, device=DEV), torch.zeros(1 << 16, dtype=torch.uint8, device=DEV))


def test_diff_rejects_downwash():
    """The smooth form has no downwash term: a handle with downwash on is refused."""
    env, _ = pair([2] * 4, 1, ("smooth", "floor", "downwash"), seed=1)
    with pytest.raises(qs.QSError) as e:
        qs.qs_diff_forward(env.h, 4, 2, torch.zeros(8, 30, device=DEV), torch.zeros(4, 8, 4, device=DEV),
                           torch.zeros(8, device=DEV), torch.zeros(1 << 16, dtype=torch.uint8, device=DEV))
    assert e.value.status == qs.QS_ERR_UNSUPPORTED


# ----------------------------------------------------------------------------- discrete contacts
DISCRETE = ("floor", "walls", "collisions", "motor_noise")


def discrete_case(seed, features=DISCRETE):
    """1 env x 3 drones whose 12 steps take every contact branch: drone 0 falls
    onto the floor (hit, then resting with friction), drone 1 flies into the
    +x wall, drone 2 catches up with drone 1 and collides with it."""
    env, o = pair([3], 0, features, seed=seed)
    st = W.random_states(seed, 3, rate=0.5)
    st[0, 0:6] = [0.0, 0.0, 0.02, 0.3, -0.2, -1.5]
    st[1, 0:6] = [4.965, 1.0, 5.0, 1.0, 0.0, 0.0]
    st[2, 0:6] = [4.852, 1.0, 5.0, 2.6, 0.0, 0.0]
    prm = W.random_params(seed, 1, nominal(env))
    goals = np.array([[1.0, -1.0, 3.0]], np.float32)
    z = np.zeros(1, np.int32)
    env.set_state(params=torch.from_numpy(prm).to(DEV), goals=torch.from_numpy(goals).to(DEV),
                  ep_step=torch.from_numpy(z).to(DEV), tick=torch.from_numpy(z).to(DEV))
    acts = W.actions(seed, 12, 3, lo=0.2, hi=0.8)
    return env, o, st, prm, goals, acts


@pytest.mark.parametrize("features", [DISCRETE, DISCRETE + ("event_time",)])
def test_discrete_case_takes_every_branch(features):
    """The oracle run of the case hits the floor, rests on it, hits a wall and
    collides, with every decision well away from its threshold."""
    env, o, st, prm, goals, acts = discrete_case(5, features)
    o.set_state(st.astype(np.float64), prm.astype(np.float64), goals.astype(np.float64), np.zeros(1, np.int32),
                np.zeros(1, np.uint32))
    seen = 0
    for t in range(acts.shape[0]):
        o.step(acts[t].astype(np.float64), want_obs=False)
        ev, _, _ = o.get_events()
        seen |= int(np.bitwise_or.reduce(ev))
    for bit in (O.EV_HIT_FLOOR, O.EV_ON_FLOOR, O.EV_HIT_WALL, O.EV_HIT_QUAD):
        assert seen & bit, bit
    margin, _ = o.margins()
    assert margin.min() > 1e-5


@pytest.mark.parametrize("features", [DISCRETE, DISCRETE + ("event_time",)])
def test_discrete_forward_loss_matches_oracle(features):
    env, o, st, prm, goals, acts = discrete_case(5, features)
    loss, _, _ = gpu_grads(env, st, acts, 4)
    want = oracle_total(o, st.astype(np.float64), prm.astype(np.float64), goals.astype(np.float64),
                        acts.astype(np.float64))
    assert np.allclose(loss, want, rtol=1e-4, atol=1e-4)


@pytest.mark.parametrize("features", [DISCRETE, DISCRETE + ("event_time",)])
def test_discrete_adjoint_matches_oracle_finite_differences(features):
    """Every command and every initial-state entry of the discrete-contact case
    (sampled contacts, and event-time contacts) against central differences
    of the FP64 oracle (h = 1e-6; a coordinate whose differences at h and 2h
    disagree, i.e. whose perturbation flips a contact decision, is left out;
    at most 5% may be): 1e-3 relative or 1e-4 of the largest entry."""
    T, C = 12, 4
    env, o, st, prm, goals, acts = discrete_case(5, features)
    _, ga, gx = gpu_grads(env, st, acts, C)
    st64, prm64, g64, a64 = (v.astype(np.float64) for v in (st, prm, goals, acts))

    def fd(perturb, h):
        p_, m_ = perturb(h), perturb(-h)
        return (oracle_total(o, *p_).sum() - oracle_total(o, *m_).sum()) / (2 * h)

    got, ref, ok = [], [], []
    for t in range(T):
        for d in range(3):
            for r in range(4):
                def pa(h, t=t, d=d, r=r):
                    a2 = a64.copy()
                    a2[t, d, r] += h
                    return st64, prm64, g64, a2
                f1, f2 = fd(pa, 1e-6), fd(pa, 2e-6)
                got.append(ga[t, d, r]), ref.append(f1), ok.append(abs(f1 - f2) <= 1e-4 * (1 + abs(f1)))
    for d in range(3):
        for k in range(26):
            def px(h, d=d, k=k):
                s2 = st64.copy()
                s2[d, k] += h
                return s2, prm64, g64, a64
            f1, f2 = fd(px, 1e-6), fd(px, 2e-6)
            got.append(gx[d, k]), ref.append(f1), ok.append(abs(f1 - f2) <= 1e-4 * (1 + abs(f1)))
    got, ref, ok = np.array(got), np.array(ref), np.array(ok)
    assert ok.mean() >= 0.95
    scale = np.abs(ref[ok]).max()
    err = np.abs(got[ok] - ref[ok])
    assert np.all(err <= 1e-3 * np.abs(ref[ok]) + 1e-4 * scale), err.max() / scale
    assert np.all(gx[:, 26:] == 0)
    # the gradient through the floor-hit reset: the fallen drone's initial
    # height and vertical speed no longer reach its later positions
    assert np.abs(ref).max() > 0


def test_rollout_fn_discrete_contacts():
    """RolloutFn on a handle with the discrete contacts: torch.autograd
    gradients equal the library's forward/backward entry points."""
    from paper_2306_09537_gb300.env import RolloutFn
    env, o, st, prm, goals, acts = discrete_case(5)
    T = acts.shape[0]
    a = torch.from_numpy(acts).to(DEV).requires_grad_(True)
    x0 = torch.from_numpy(st).to(DEV).requires_grad_(True)
    loss = RolloutFn.apply(a, x0, env, 4)
    loss.sum().backward()
    l_ref, ga, gx = gpu_grads(env, st, acts, 4)
    assert np.allclose(loss.detach().cpu().numpy(), l_ref, rtol=0, atol=0)
    assert np.array_equal(a.grad.cpu().numpy().astype(np.float64), ga)
    assert np.array_equal(x0.grad.cpu().numpy().astype(np.float64), gx)


@pytest.mark.parametrize("event_time", [False, True])
def test_discrete_adjoint_matches_torch_autograd_reference(event_time):
    """8 envs x 8 drones x 32 steps that take every contact (mid-air collisions,
    floor hits and resting friction, walls, ceiling; contact_swarm_states),
    checkpoints every 8, contact perturbations and motor noise off: the
    discrete-contact adjoint against torch.autograd of the FP64 reference
    with the same contact rules (each decision held fixed, R27), within 1e-4
    relative (or 1e-5 of the largest entry); with the event-time contacts
    within 1e-3 (or 1e-4). The oracle's run of the case keeps every decision
    at least 1e-5 (relative) from its threshold, so the binary32 forward takes
    the reference's branches."""
    sizes, T, C, seed = [8] * 8, 32, 8, 56
    feats = ("floor", "walls", "collisions") + (("event_time",) if event_time else ())
    env, o = pair(sizes, 0, feats, seed=seed, coll_sigma_v=0.0, coll_sigma_w=0.0)
    E, D = env.E, env.D
    st = W.contact_swarm_states(seed, E, 8)
    prm = W.random_params(seed, E, nominal(env))
    goals = W.random_goals(seed, E)
    z = np.zeros(E, np.int32)
    env.set_state(params=torch.from_numpy(prm).to(DEV), goals=torch.from_numpy(goals).to(DEV),
                  ep_step=torch.from_numpy(z).to(DEV), tick=torch.from_numpy(z).to(DEV))
    acts = W.actions(seed, T, D, lo=0.2, hi=0.8)
    st64, prm64, g64, a64 = (v.astype(np.float64) for v in (st, prm, goals, acts))
    o.set_state(st64, prm64, g64, z, z.astype(np.uint32))
    seen, margin = 0, np.inf
    for t in range(T):
        o.step(a64[t], want_obs=False)
        ev, _, m = o.get_events()
        seen |= int(np.bitwise_or.reduce(ev))
        margin = min(margin, m.min())
        o.clear_margin()
    assert margin >= 1e-5
    for bit in (O.EV_HIT_FLOOR, O.EV_ON_FLOOR, O.EV_HIT_WALL, O.EV_HIT_CEIL, O.EV_HIT_QUAD):
        assert seen & bit, bit
    loss, ga, gx = gpu_grads(env, st, acts, C)
    p = env.cfg.params
    cfg = {"dt": env.cfg.dt, "gravity": p.gravity, "kappa": p.kappa, "room_hx": p.room_hx, "room_hy": p.room_hy,
           "room_h": p.room_h, "omega_max": p.omega_max, "mu": p.mu, "alpha_c": p.alpha_c}
    cfg = {k: float(v) for k, v in cfg.items()}
    cfg.update(substeps=int(env.cfg.substeps), floor=True, walls=True, collisions=True, event_time=event_time)
    x0 = torch.tensor(st64, requires_grad=True)
    a = torch.tensor(a64, requires_grad=True)
    L = discrete_rollout_loss(x0, a, torch.tensor(prm64), torch.tensor(g64), sizes, cfg)
    assert np.allclose(loss, L.detach().numpy(), rtol=1e-4, atol=1e-4)
    L.sum().backward()
    # the crossing-time derivatives are worse conditioned (a shallow pair
    # overlap makes the contact time sensitive to the positions, and its
    # derivatives carry 1 / (approach speed)): perturbing the initial state
    # by binary32 rounding moves the event-time gradient about 10x more than
    # the sampled one (tests/test_ref_torch.py), hence a 10x wider bar
    rel, frac = (1e-3, 1e-4) if event_time else (1e-4, 1e-5)
    for g, ref in ((ga, a.grad.numpy()), (gx[:, :26], x0.grad.numpy()[:, :26])):
        ok, worst = close_to_reference(g, ref, rel, frac)
        assert ok, worst
    assert np.all(gx[:, 26:] == 0)
    # one checkpoint segment or several pipelined: the same bits
    _, ga1, gx1 = gpu_grads(env, st, acts, T)
    assert np.array_equal(ga, ga1) and np.array_equal(gx, gx1)


def test_event_time_changes_the_gradient_and_is_refused_elsewhere():
    """Event-time contacts move the trajectory and the gradient where contacts
    happen (the crossing-time terms), and a handle with them runs only the
    differentiable rollout: the step, rollout and server entry points and the
    smooth form refuse it."""
    g = {}
    for et in (False, True):
        env, o, st, prm, goals, acts = discrete_case(5, DISCRETE + (("event_time",) if et else ()))
        g[et] = gpu_grads(env, st, acts, 4)
    assert np.abs(g[True][0] - g[False][0]).max() > 1e-4
    assert np.abs(g[True][2] - g[False][2]).max() > 1e-3 * np.abs(g[False][2]).max()
    env, _ = pair([3], 0, DISCRETE + ("event_time",), seed=5)
    a = torch.zeros(env.D, 4, device=DEV)
    with pytest.raises(qs.QSError) as e:
        env.step(a)
    assert e.value.status == qs.QS_ERR_UNSUPPORTED
    with pytest.raises(qs.QSError) as e:
        env.rollout(a[None].contiguous())
    assert e.value.status == qs.QS_ERR_UNSUPPORTED
    env2, _ = pair([3], 0, ("smooth", "event_time"), seed=5)
    with pytest.raises(qs.QSError) as e:
        qs.qs_diff_forward(env2.h, 4, 2, torch.zeros(3, 30, device=DEV), torch.zeros(4, 3, 4, device=DEV),
                           torch.zeros(3, device=DEV), torch.zeros(1 << 16, dtype=torch.uint8, device=DEV))
    assert e.value.status == qs.QS_ERR_UNSUPPORTED
