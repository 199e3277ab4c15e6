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
