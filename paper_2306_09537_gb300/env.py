"""QuadSwarmEnv: the Gym-style multi-agent environment of the paper (Sec. III,
Table I "Gym Wrapper") over the C ABI, with torch tensors for device memory
and the current torch CUDA stream for ordering."""
from __future__ import annotations

import numpy as np
import torch

from . import qs


class QuadSwarmEnv:
    """E environments of N_e quadrotors each; one ``step`` is one 100 Hz control
    step of all of them, computed by libquadswarm_gpu.so on the current device."""

    def __init__(self, n_envs: int, swarm=1, k_neighbors: int = 0, features=(), seed: int = 1, weights=None,
                 device="cuda", stream=None, scenarios=(), **overrides):
        self.device = torch.device(device)
        if self.device.type != "cuda":
            raise ValueError("QuadSwarmEnv runs on a CUDA device only")
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        sizes = None
        if swarm is None or not np.isscalar(swarm):
            sizes = np.ascontiguousarray(swarm, dtype=np.int32)
            swarm = 1
        self.sizes, self.features, self.weights, self.overrides = sizes, tuple(features), weights, dict(overrides)
        self.scenarios = tuple(scenarios)
        self.cfg = qs.make_config(n_envs, swarm, k_neighbors, features, seed, weights, scenarios=scenarios,
                                  **overrides)
        with torch.cuda.device(self.device):
            self.h = qs.qs_create(self.cfg, self.stream.cuda_stream, swarm_sizes=sizes)
        self.D, self.E, self.obs_dim = qs.qs_get_dims(self.h)
        self.K = int(k_neighbors)
        kw = dict(device=self.device)
        self.obs = torch.empty(self.D, self.obs_dim, dtype=torch.float32, **kw)
        self.reward = torch.empty(self.D, dtype=torch.float32, **kw)
        self.done = torch.empty(self.E, dtype=torch.uint8, **kw)

    def close(self):
        if getattr(self, "h", None):
            qs.qs_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def reset(self, seed: int, env_mask=None) -> torch.Tensor:
        qs.qs_reset(self.h, seed, env_mask, self.obs)
        return self.obs

    def step(self, actions: torch.Tensor):
        assert actions.shape == (self.D, 4) and actions.dtype == torch.float32 and actions.is_cuda
        qs.qs_step(self.h, actions.contiguous(), self.obs, self.reward, self.done)
        return self.obs, self.reward, self.done

    def rollout(self, actions: torch.Tensor, obs=None, reward=None, done=None):
        T = actions.shape[0]
        assert actions.shape == (T, self.D, 4)
        qs.qs_rollout(self.h, T, actions.contiguous(), obs, reward, done)
        return obs, reward, done

    def get_state(self):
        kw = dict(device=self.device)
        out = {"state": torch.empty(self.D, qs.QS_STATE_DIM, **kw), "params": torch.empty(self.E, qs.QS_PARAM_DIM, **kw),
               "goals": torch.empty(self.E, 3, **kw), "ep_step": torch.empty(self.E, dtype=torch.int32, **kw),
               "tick": torch.empty(self.E, dtype=torch.int32, **kw)}
        qs.qs_get_state(self.h, out["state"], out["params"], out["goals"], out["ep_step"], out["tick"])
        return out

    def set_state(self, state=None, params=None, goals=None, ep_step=None, tick=None):
        qs.qs_set_state(self.h, state, params, goals, ep_step, tick)

    def get_events(self, knn: bool = False):
        ev = torch.empty(self.D, dtype=torch.int32, device=self.device)
        nb = torch.empty(self.D, max(self.K, 1), dtype=torch.int16, device=self.device) if knn else None
        qs.qs_get_events(self.h, ev, nb)
        return ev, (nb[:, :self.K] if nb is not None else None)

    def get_scenario(self) -> torch.Tensor:
        """Scenario records [E][QS_NSCN] (Sec. III-D)."""
        out = torch.empty(self.E, qs.QS_NSCN, device=self.device)
        qs.qs_get_scenario(self.h, out)
        return out

    def set_scenario(self, records: torch.Tensor):
        qs.qs_set_scenario(self.h, records.contiguous())

    def get_goals(self) -> torch.Tensor:
        """Goal [D][3] of every drone at its env's current control step."""
        out = torch.empty(self.D, 3, device=self.device)
        qs.qs_get_goals(self.h, out)
        return out

    def sync(self):
        qs.qs_sync(self.h)

    def serve(self, idle_ms: int = 1000, slots: int = 1) -> "Server":
        """Resident stepping with page-locked host buffers (see qs_serve_begin):

            with env.serve() as srv:
                srv.actions[:] = a          # host tensor [D][4] (command slot 0)
                srv.step()                  # returns when obs / reward / done are in host memory
                use(srv.obs, srv.reward, srv.done)

        With slots > 1, srv.slots [slots][D][4] holds commands written ahead and
        srv.step(slot) steps with slot `slot`."""
        return Server(self, idle_ms, slots)


class Server:
    """Page-locked host buffers and a resident step server of one env handle."""

    def __init__(self, env: QuadSwarmEnv, idle_ms: int = 1000, slots: int = 1):
        self.env = env
        self.slots = torch.zeros(slots, env.D, 4).pin_memory()
        self.actions = self.slots[0]
        self.obs = torch.zeros(env.D, env.obs_dim).pin_memory()
        self.reward = torch.zeros(env.D).pin_memory()
        self.done = torch.zeros(env.E, dtype=torch.uint8).pin_memory()
        qs.qs_serve_begin(env.h, self.slots, self.obs, self.reward, self.done, idle_ms, slots)
        self.active = True

    def step(self, slot: int = 0):
        qs.qs_serve_step(self.env.h, slot)
        return self.obs, self.reward, self.done

    def close(self):
        if self.active:
            self.active = False
            if self.env.h:  # a destroyed handle ended its server already
                qs.qs_serve_end(self.env.h)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class RolloutFn(torch.autograd.Function):
    """Differentiable rollout of the step (smooth contacts when the env has the
    "smooth" feature, else the contacts as the step runs them, differentiated
    along the branch each contact decision took): loss[d] = sum_t |x_d(t) - goal|^2 +
    1e-3 |f^_d(t)|^2 for commands actions [T][D][4] from initial states
    x0 [D][30]. The forward pass stores a checkpoint every `ckpt_every` steps
    in a workspace it allocates from torch; backward recomputes each segment
    and runs the library's hand-written adjoint kernel.

        loss = RolloutFn.apply(actions, x0, env, ckpt_every)"""

    @staticmethod
    def forward(ctx, actions, x0, env, ckpt_every=16):
        T = actions.shape[0]
        assert actions.shape == (T, env.D, 4) and x0.shape == (env.D, qs.QS_STATE_DIM)
        actions = actions.detach().contiguous()
        x0 = x0.detach().contiguous()
        ws = torch.empty(qs.qs_diff_workspace_size(env.h, T, ckpt_every), dtype=torch.uint8, device=env.device)
        loss = torch.empty(env.D, dtype=torch.float32, device=env.device)
        qs.qs_diff_forward(env.h, T, ckpt_every, x0, actions, loss, ws)
        ctx.save_for_backward(actions)
        ctx.env, ctx.ws, ctx.ckpt_every = env, ws, ckpt_every
        return loss

    @staticmethod
    def backward(ctx, dloss):
        (actions,) = ctx.saved_tensors
        env = ctx.env
        grad_a = torch.empty_like(actions)
        grad_x0 = torch.empty(env.D, qs.QS_STATE_DIM, dtype=torch.float32, device=env.device)
        qs.qs_diff_backward(env.h, actions.shape[0], ctx.ckpt_every, actions, dloss.contiguous(), ctx.ws, grad_a,
                            grad_x0)
        return grad_a, grad_x0, None, None
