"""Guard bands around every output buffer (a stand-in for a memory checker):
each output is a view into a larger allocation whose bytes before and after
the view hold a sentinel; every entry point that writes must leave both bands
untouched. Mixed swarm sizes put every width class (1 .. 128) and every step
kernel (warp-specialised, one thread per drone, persistent and
warp-specialised rollouts, the resident server, the adjoint) on the test."""
import numpy as np
import pytest
import torch

from gpu_helpers import ALL_WEIGHTS, DEV
from paper_2306_09537_gb300 import qs
from paper_2306_09537_gb300 import workloads as W
from paper_2306_09537_gb300.env import QuadSwarmEnv

pytestmark = pytest.mark.gpu

G = 256  # guard elements on each side (keeps every view 16-byte aligned)
SENTINEL = {torch.float32: 7.125e30, torch.int32: -123456789, torch.int16: -12345, torch.uint8: 0xA5}
FEATS = ("floor", "walls", "motor_noise", "obs_noise", "dr", "collisions", "auto_reset", "record_knn")


class Guarded:
    """An output tensor of `shape` with G sentinel elements on either side."""

    def __init__(self, shape, dtype=torch.float32, device=DEV, pinned=False):
        n = int(np.prod(shape))
        base = torch.full((n + 2 * G,), SENTINEL[dtype], dtype=dtype)
        self.base = base.pin_memory() if pinned else base.to(device)
        self.view = self.base[G:G + n].view(*shape)

    def intact(self):
        torch.cuda.synchronize()
        b = self.base.cpu()
        s = SENTINEL[b.dtype]
        return bool((b[:G] == s).all()) and bool((b[-G:] == s).all())


def _env(sizes, K, stream=None, **kw):
    return QuadSwarmEnv(len(sizes), np.asarray(sizes, np.int32), K, FEATS, seed=3, weights=ALL_WEIGHTS, device=DEV,
                        stream=stream, episode_steps=4, **kw)


@pytest.mark.parametrize("sizes", [[1, 2, 3, 5, 8, 13, 31, 33, 64, 100, 128] * 3, [1] * 700, [8] * 96 + [5, 3]])
def test_step_rollout_and_accessors_stay_inside_their_buffers(sizes):
    env = _env(sizes, 6)
    D, E, od = env.D, env.E, env.obs_dim
    acts = torch.from_numpy(W.actions(3, 6, D)).to(DEV)
    obs, rew, done = Guarded((D, od)), Guarded((D,)), Guarded((E,), torch.uint8)
    qs.qs_reset(env.h, 5, None, obs.view)
    for t in range(6):  # crosses an auto-reset (episodes of 4 steps)
        qs.qs_step(env.h, acts[t], obs.view, rew.view, done.view)
    assert obs.intact() and rew.intact() and done.intact()
    T = 5
    shapes = [(128, 0, True), (256, 2, False)]
    if max(sizes) <= 64:
        shapes.append((qs.QS_BLOCK_WARP_SPECIALISED, 0, False))
    for shape in shapes:
        qs.qs_set_rollout_shape(env.h, *shape)
        o, r, d = Guarded((T, D, od)), Guarded((T, D)), Guarded((T, E), torch.uint8)
        ra = torch.from_numpy(W.actions(4, T, D)).to(DEV)
        qs.qs_rollout(env.h, T, ra, o.view, r.view, d.view)
        assert o.intact() and r.intact() and d.intact(), shape
    st, prm, gl = Guarded((D, qs.QS_STATE_DIM)), Guarded((E, qs.QS_PARAM_DIM)), Guarded((E, 3))
    ep, tk = Guarded((E,), torch.int32), Guarded((E,), torch.int32)
    qs.qs_get_state(env.h, st.view, prm.view, gl.view, ep.view, tk.view)
    ev, knn = Guarded((D,), torch.int32), Guarded((D, 6), torch.int16)
    qs.qs_get_events(env.h, ev.view, knn.view)
    goals = Guarded((D, 3))
    qs.qs_get_goals(env.h, goals.view)
    rec = Guarded((E, qs.QS_NSCN))
    qs.qs_get_scenario(env.h, rec.view)
    for g in (st, prm, gl, ep, tk, ev, knn, goals, rec):
        assert g.intact()


def test_server_stays_inside_its_host_buffers():
    sizes = [1, 3, 8, 17, 33, 48, 64, 5] * 4
    env = _env(sizes, 6, stream=torch.cuda.Stream())
    D, E, od = env.D, env.E, env.obs_dim
    S = 3
    slots = Guarded((S, D, 4), pinned=True)
    slots.view.copy_(torch.from_numpy(W.actions(6, S, D)))
    obs, rew = Guarded((D, od), pinned=True), Guarded((D,), pinned=True)
    done = Guarded((E,), torch.uint8, pinned=True)
    try:
        qs.qs_serve_begin(env.h, slots.view, obs.view, rew.view, done.view, 1000, S)
    except qs.QSError as ex:
        if ex.status == qs.QS_ERR_UNSUPPORTED and "native atomics" in str(ex):
            pytest.skip("no native atomics on host memory")
        raise
    for t in range(7):
        qs.qs_serve_step(env.h, t % S)
    qs.qs_serve_end(env.h)
    assert obs.intact() and rew.intact() and done.intact()


def test_adjoint_stays_inside_its_buffers():
    for features in (("dr", "smooth", "motor_noise"), ("dr", "motor_noise", "floor", "walls", "collisions")):
        env = QuadSwarmEnv(40, np.array([8] * 20 + [3] * 20, np.int32), 0, features, seed=2, device=DEV)
        D, T, C = env.D, 6, 4
        x0 = env.get_state()["state"].contiguous()
        acts = torch.from_numpy(W.actions(2, T, D, lo=0.05, hi=0.95)).to(DEV)
        ws = Guarded((qs.qs_diff_workspace_size(env.h, T, C),), torch.uint8)
        loss, ga, gx = Guarded((D,)), Guarded((T, D, 4)), Guarded((D, qs.QS_STATE_DIM))
        qs.qs_diff_forward(env.h, T, C, x0, acts, loss.view, ws.view)
        qs.qs_diff_backward(env.h, T, C, acts, torch.ones(D, device=DEV), ws.view, ga.view, gx.view)
        for g in (ws, loss, ga, gx):
            assert g.intact(), features
