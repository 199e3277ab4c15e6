"""Plain PyTorch (CPU, float64) restatement of the smooth-contact control step,
differentiated by torch.autograd: the reference for gradients of the
differentiable rollout.

Test infrastructure, like the rest of oracle/. It follows the same equations
as qs_oracle.c's smooth form (Sec. III-A dynamics, motor lag and noise; the
floor, walls, ceiling and quad-quad contacts of Sec. III-B as softplus
penalties) written with tensor ops over all drones at once; the polar factor
of the integrated rotation is Newton's iteration X <- (X + X^-T)/2 with a
fixed number of steps (converged in binary64 for the near-orthogonal inputs
of one substep). It shares no code with the CUDA path; tests pin it to the C
oracle (forward) and to finite differences of the C oracle (gradient).
"""
from __future__ import annotations

import math

import torch


def skew(w):
    z = torch.zeros_like(w[..., 0])
    return torch.stack([torch.stack([z, -w[..., 2], w[..., 1]], -1),
                        torch.stack([w[..., 2], z, -w[..., 0]], -1),
                        torch.stack([-w[..., 1], w[..., 0], z], -1)], -2)


def polar(m, iters=8):
    x = m
    for _ in range(iters):
        x = 0.5 * (x + torch.linalg.inv(x).transpose(-1, -2))
    return x


def softplus_b(u, beta):
    return torch.nn.functional.softplus(beta * u) / beta


def smooth_rollout_loss(x0, actions, params, goals, sizes, cfg, motor_normals=None):
    """Per-drone loss sum_t |x(t) - g|^2 + 1e-3 |f^(t)|^2 of T smooth steps.

    x0 [D,30], actions [T,D,4], params [E,7] (m, Ixx, Iyy, Izz, t2w, tau_m, arm),
    goals [E,3], sizes [E]; cfg: dict of the model constants; motor_normals
    [T, substeps, D, 4] (None: no motor noise)."""
    dt, g = cfg["dt"], cfg["gravity"]
    sizes = [int(n) for n in sizes]
    env_of = torch.repeat_interleave(torch.arange(len(sizes)), torch.tensor(sizes))
    P = params[env_of]
    m, I, t2w, tau_m, arm = P[:, 0], P[:, 1:4], P[:, 4], P[:, 5], P[:, 6]
    G = goals[env_of]
    fmax = 0.25 * m * g * t2w
    alag = 1.0 - torch.exp(-dt / tau_m)
    ans = cfg["alpha_ns_frac"] * m * g / 4.0
    kcg = cfg["smooth_kc"] * g
    beta = cfg["smooth_beta"]
    # pairs (i, j), i != j, of every env
    ii, jj = [], []
    off = 0
    for n in sizes:
        for a in range(n):
            for b in range(n):
                if a != b:
                    ii.append(off + a)
                    jj.append(off + b)
        off += n
    ii, jj = torch.tensor(ii, dtype=torch.long), torch.tensor(jj, dtype=torch.long)

    x, v = x0[:, 0:3], x0[:, 3:6]
    R = x0[:, 6:15].reshape(-1, 3, 3)
    w, uf, eps = x0[:, 15:18], x0[:, 18:22], x0[:, 22:26]
    sa = arm / math.sqrt(2.0)
    loss = torch.zeros(x0.shape[0], dtype=x0.dtype)
    for t in range(actions.shape[0]):
        fh = torch.clamp(actions[t], 0.0, 1.0)
        u = torch.sqrt(fh)
        for s in range(cfg["substeps"]):
            # pair penalty from positions at the substep start
            pacc = torch.zeros_like(x)
            if ii.numel():
                r = x[ii] - x[jj]
                d = torch.sqrt((r * r).sum(-1))
                mag = kcg * softplus_b(2.0 * arm[ii] - d, beta) / d
                pacc = pacc.index_add(0, ii, mag[:, None] * r)
            uf = uf + alag[:, None] * (u - uf)
            if motor_normals is not None:
                eps = cfg["alpha_nd"] * eps + ans[:, None] * motor_normals[t, s]
            f = fmax[:, None] * uf * uf + eps
            T = f.sum(-1)
            tau = torch.stack([sa * (f[:, 0] + f[:, 1] - f[:, 2] - f[:, 3]),
                               sa * (-f[:, 0] + f[:, 1] + f[:, 2] - f[:, 3]),
                               cfg["kappa"] * (-f[:, 0] + f[:, 1] - f[:, 2] + f[:, 3])], -1)
            acc = T[:, None] * R[:, :, 2] / m[:, None]
            acc = acc + torch.tensor([0.0, 0.0, -g], dtype=x.dtype)
            wall = torch.stack([
                kcg * (softplus_b(-cfg["room_hx"] - x[:, 0], beta) - softplus_b(x[:, 0] - cfg["room_hx"], beta)),
                kcg * (softplus_b(-cfg["room_hy"] - x[:, 1], beta) - softplus_b(x[:, 1] - cfg["room_hy"], beta)),
                kcg * (softplus_b(-x[:, 2], beta) - softplus_b(x[:, 2] - cfg["room_h"], beta))], -1)
            acc = acc + wall + pacc
            Iw = I * w
            wdot = (tau - torch.cross(w, Iw, dim=-1)) / I
            v = v + acc * dt
            x = x + v * dt
            w = torch.clamp(w + wdot * dt, -cfg["omega_max"], cfg["omega_max"])
            R = polar(R + dt * R @ skew(w))
        loss = loss + ((x - G) ** 2).sum(-1) + 1e-3 * (fh * fh).sum(-1)
    return loss
