"""The allocation-free differentiable rollout (qs_diff_grad_static).

Callers that cannot allocate device memory when they need a gradient (code
inside a CUDA graph capture, real-time loops that must not call cudaMalloc,
plugins whose host framework owns the memory budget) use this entry point: its
workspace is a fixed array in the library's device image. Two calls in a row,
with different commands, must each reproduce the workspace-based entry points
(qs_diff_forward + qs_diff_backward) bit for bit; a rollout too large for the array is
refused without work."""
import numpy as np
import pytest
import torch

from gpu_helpers import DEV, nominal, pair
from paper_2306_09537_gb300 import qs
from paper_2306_09537_gb300 import workloads as W

pytestmark = pytest.mark.gpu

SIZES = [8] * 48 + [3] * 16
T, C = 24, 8


def make_env():
    env, _ = pair(SIZES, 0, ("smooth", "motor_noise", "dr"), seed=17)
    prm = W.random_params(17, env.E, nominal(env))
    goals = W.random_goals(17, env.E)
    env.set_state(params=torch.from_numpy(prm).to(DEV), goals=torch.from_numpy(goals).to(DEV))
    st = W.random_states(17, env.D)
    st[:, 0:3] = W.clustered_positions(17, SIZES, spread=0.06)
    return env, torch.from_numpy(st).to(DEV)


def with_workspace(env, x0, acts, dloss):
    ws = torch.empty(qs.qs_diff_workspace_size(env.h, T, C), dtype=torch.uint8, device=DEV)
    loss = torch.empty(env.D, device=DEV)
    ga = torch.empty_like(acts)
    gx = torch.empty(env.D, 30, device=DEV)
    qs.qs_diff_forward(env.h, T, C, x0, acts, loss, ws)
    qs.qs_diff_backward(env.h, T, C, acts, dloss, ws, ga, gx)
    env.sync()
    return loss.cpu().numpy(), ga.cpu().numpy(), gx.cpu().numpy()


def static(env, x0, acts, dloss):
    loss = torch.full((env.D,), float("nan"), device=DEV)
    ga = torch.full_like(acts, float("nan"))
    gx = torch.full((env.D, 30), float("nan"), device=DEV)
    qs.qs_diff_grad_static(env.h, T, C, x0, acts, dloss, loss, ga, gx)
    env.sync()
    return loss.cpu().numpy(), ga.cpu().numpy(), gx.cpu().numpy()


def test_static_workspace_matches_caller_workspace_twice():
    env, x0 = make_env()
    dloss = torch.linspace(0.5, 1.5, env.D, device=DEV)
    runs = []
    for seed in (3, 4):  # two calls in a row, different commands
        acts = torch.from_numpy(W.actions(seed, T, env.D, lo=0.05, hi=0.95)).to(DEV)
        runs.append((with_workspace(env, x0, acts, dloss), static(env, x0, acts, dloss)))
    for ref, got in runs:
        for r, g in zip(ref, got):
            assert np.isfinite(g).all()
            assert np.array_equal(g, r)  # the same kernels on another workspace: bit for bit
    # the two calls really differed, so stale contents would have shown
    assert not np.allclose(runs[0][1][1], runs[1][1][1])


def test_static_workspace_refuses_oversize_rollout():
    env, x0 = make_env()
    big_T = 4096
    need = qs.qs_diff_workspace_size(env.h, big_T, big_T)
    assert need > qs.QS_DIFF_STATIC_BYTES
    acts = torch.zeros(big_T, env.D, 4, device=DEV)
    out = torch.zeros(env.D, device=DEV)
    with pytest.raises(qs.QSError) as ei:
        qs.qs_diff_grad_static(env.h, big_T, big_T, x0, acts, out, out, acts, torch.zeros(env.D, 30, device=DEV))
    assert ei.value.status == qs.QS_ERR_UNSUPPORTED
    assert "static" in str(ei.value)
