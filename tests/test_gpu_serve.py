"""The resident step server (qs_serve_begin / qs_serve_step / qs_serve_end):
the same bits as per-call steps through every swarm layout, across
auto-resets, idle retirement and the hand-back to per-call stepping."""
import time

import numpy as np
import pytest
import torch

from gpu_helpers import ALL_WEIGHTS, DEV, nominal
from paper_2306_09537_gb300 import qs
from paper_2306_09537_gb300 import workloads as W
from paper_2306_09537_gb300.env import QuadSwarmEnv

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True, scope="module")
def _host_link_supports_serving():
    """The server needs native atomics on page-locked host memory (a coherent
    host link such as NVLink-C2C); elsewhere qs_serve_begin refuses with
    QS_ERR_UNSUPPORTED and these tests do not apply."""
    env = QuadSwarmEnv(4, 1, 0, ("floor",), seed=1, device=DEV, stream=torch.cuda.Stream())
    try:
        qs.qs_serve_begin(env.h, torch.zeros(env.D, 4).pin_memory())
        qs.qs_serve_end(env.h)
    except qs.QSError as ex:
        if ex.status == qs.QS_ERR_UNSUPPORTED and "native atomics" in str(ex):
            pytest.skip("no native atomics on host memory")
        raise
    finally:
        env.close()

FEATS = ("floor", "walls", "motor_noise", "obs_noise", "dr", "collisions", "auto_reset")


def twins(sizes, K, feats=FEATS, scenarios=(), seed=7, **kw):
    """Two handles in the same seeded state (clustered swarms, so that pairs
    collide)."""
    envs = []
    for stream in (torch.cuda.Stream(), None):  # the server needs a non-blocking stream of its own
        env = QuadSwarmEnv(len(sizes), np.asarray(sizes, np.int32), K, feats, seed=seed, weights=ALL_WEIGHTS,
                           device=DEV, stream=stream, scenarios=scenarios, episode_steps=5, **kw)
        envs.append(env)
    a = envs[0]
    st = W.random_states(seed, a.D)
    if max(sizes) > 1:
        st[:, 0:3] = W.clustered_positions(seed, sizes, spread=0.12)
    prm = W.random_params(seed, a.E, nominal(a))
    goals = W.random_goals(seed, a.E)
    inputs = (torch.from_numpy(st.astype(np.float32)).to(DEV), torch.from_numpy(prm.astype(np.float32)).to(DEV),
              torch.from_numpy(goals.astype(np.float32)).to(DEV), torch.zeros(a.E, dtype=torch.int32, device=DEV),
              torch.full((a.E,), 3, dtype=torch.int32, device=DEV))
    torch.cuda.synchronize()  # the inputs come from the current stream, the server handle runs on its own
    for env in envs:
        env.set_state(*inputs)
    torch.cuda.synchronize()
    return envs


def state_of(env):
    s = env.get_state()
    ev = env.get_events()[0]
    env.stream.synchronize()
    return s, ev


def serve_vs_steps(sizes, K, T, scenarios=(), feats=FEATS, pause_at=None, idle_ms=1000, **kw):
    a, b = twins(sizes, K, feats, scenarios, **kw)
    acts = W.actions(11, T, a.D)
    srv = a.serve(idle_ms=idle_ms)
    for t in range(T):
        if pause_at is not None and t == pause_at:
            time.sleep(0.2)  # several idle periods: the server retires and is started again
        srv.actions.copy_(torch.from_numpy(acts[t]))
        o1, r1, d1 = srv.step()
        o2, r2, d2 = b.step(torch.from_numpy(acts[t]).to(DEV))
        assert torch.equal(o1, o2.cpu()), t
        assert torch.equal(r1, r2.cpu()), t
        assert torch.equal(d1, d2.cpu()), t
    srv.close()
    (s1, ev1), (s2, ev2) = state_of(a), state_of(b)
    for k in ("state", "params", "goals", "ep_step", "tick"):
        assert torch.equal(s1[k], s2[k]), k
    assert torch.equal(ev1, ev2)
    return a, b


def test_serve_equals_steps_single_drones():
    serve_vs_steps([1] * 3000, 0, 12)


def test_serve_equals_steps_swarms():
    serve_vs_steps([8] * 256, 6, 12)


def test_serve_equals_steps_uneven_with_scenarios_and_downwash():
    """Two dynamics warps per CTA (swarms up to 64) and the extended instance."""
    sizes = [1, 3, 8, 17, 33, 48, 64, 5, 32] * 4
    serve_vs_steps(sizes, 6, 11, scenarios=("static", "swap", "pursuit_bezier", "swarm_vs_swarm"),
                   feats=FEATS + ("downwash",))


def test_serve_equals_steps_smooth_swarms():
    """Smooth contacts (the general instance, the pair penalty staged before
    every substep by one or two dynamics warps)."""
    serve_vs_steps([8, 33, 64, 2, 17] * 8, 6, 10, feats=("smooth", "motor_noise", "obs_noise", "dr", "collisions",
                                                        "auto_reset"))


def test_serve_command_slots():
    """Commands written ahead into slots, stepped in a shuffled slot order."""
    a, b = twins([8] * 128, 6)
    S, T = 5, 12
    acts = W.actions(13, T, a.D)
    order = np.random.default_rng(1).integers(0, S, T)
    with a.serve(slots=S) as srv:
        for t in range(T):
            srv.slots[order[t]].copy_(torch.from_numpy(acts[t]))
            o1, r1, d1 = srv.step(int(order[t]))
            o2, r2, d2 = b.step(torch.from_numpy(acts[t]).to(DEV))
            assert torch.equal(o1, o2.cpu()) and torch.equal(r1, r2.cpu()) and torch.equal(d1, d2.cpu()), t
        for bad in (-1, S):
            with pytest.raises(qs.QSError):
                srv.step(bad)
        srv.step(0)  # still serving after the refusals
    with pytest.raises(qs.QSError):
        qs.qs_serve_begin(a.h, srv.slots, n_slots=0)


def test_serve_retires_when_idle_and_restarts():
    serve_vs_steps([8] * 64, 6, 8, pause_at=4, idle_ms=20)


def test_serve_hands_back_to_per_call_steps():
    """After qs_serve_end the drones continue with qs_step and qs_rollout as if
    every step had been a qs_step."""
    a, b = serve_vs_steps([4] * 100, 3, 6)
    acts = torch.from_numpy(W.actions(12, 4, a.D)).to(DEV)
    torch.cuda.synchronize()
    for t in range(4):
        o1, r1, _ = a.step(acts[t])
        a.stream.synchronize()
        o1, r1 = o1.clone(), r1.clone()
        o2, r2, _ = b.step(acts[t])
        assert torch.equal(o1, o2) and torch.equal(r1, r2)
    a2 = a.serve()  # a second session on the same handle
    a2.actions.copy_(acts[0].cpu())
    a2.step()
    a2.close()
    b.step(acts[0])
    assert torch.equal(state_of(a)[0]["state"], state_of(b)[0]["state"])


def test_serve_refuses_other_calls_while_serving():
    env = QuadSwarmEnv(64, 1, 0, FEATS, seed=3, device=DEV, stream=torch.cuda.Stream())
    act = torch.rand(env.D, 4, device=DEV)
    torch.cuda.synchronize()
    with env.serve() as srv:
        srv.actions.uniform_()
        srv.step()
        for call in (lambda: env.step(act), lambda: env.get_state(), lambda: env.reset(1), lambda: env.sync(),
                     lambda: qs.qs_serve_begin(env.h, srv.actions)):
            with pytest.raises(qs.QSError):
                call()
        srv.step()  # still serving after the refusals
    env.step(act)
    env.sync()


def test_serve_rejects_unsupported_handles_and_buffers():
    legacy = QuadSwarmEnv(16, 1, 0, FEATS, seed=3, device=DEV, stream=torch.cuda.default_stream(DEV))
    with pytest.raises(qs.QSError) as ex:
        qs.qs_serve_begin(legacy.h, torch.zeros(legacy.D, 4).pin_memory())
    assert ex.value.status == qs.QS_ERR_UNSUPPORTED
    env = QuadSwarmEnv(16, 1, 0, FEATS, seed=3, device=DEV, stream=torch.cuda.Stream())
    with pytest.raises(qs.QSError):
        qs.qs_serve_begin(env.h, torch.zeros(env.D, 4, device=DEV))  # device memory
    with pytest.raises(qs.QSError):
        qs.qs_serve_begin(env.h, torch.zeros(env.D, 4))  # pageable host memory
    for idle in (0, 60001):  # a resident launch may not wait longer than a minute on a shared GPU
        with pytest.raises(qs.QSError) as ex:
            qs.qs_serve_begin(env.h, torch.zeros(env.D, 4).pin_memory(), idle_ms=idle)
        assert ex.value.status == qs.QS_ERR_ARG
    with pytest.raises(qs.QSError):
        qs.qs_serve_step(env.h)  # not serving
    qs.qs_serve_end(env.h)  # not serving: nothing to end
    wide = QuadSwarmEnv(2, np.array([65, 3], np.int32), 2, FEATS, seed=3, device=DEV, stream=torch.cuda.Stream())
    with pytest.raises(qs.QSError) as ex:
        qs.qs_serve_begin(wide.h, torch.zeros(wide.D, 4).pin_memory())
    assert ex.value.status == qs.QS_ERR_UNSUPPORTED
