"""Plain PyTorch (CPU, float64) restatements of the control step,
differentiated by torch.autograd: the references for gradients of the
differentiable rollout.

Test infrastructure, like the rest of oracle/. Two forms, both written with
tensor ops over all drones at once:

* smooth_rollout_loss: the smooth-contact form (Sec. III-A dynamics, motor lag
  and noise; the floor, walls, ceiling and quad-quad contacts of Sec. III-B as
  softplus penalties);
* discrete_rollout_loss: the step with the paper's own contact rules (floor
  hit and resting friction, walls and ceiling, quad-quad collisions with the
  Jacobi response), each decision taken on the reference's own binary64
  values (the pair set on their binary32 rounding, as the step defines it)
  and held fixed while autograd differentiates the branch taken: the
  derivative of the piecewise-smooth map along the branches of the run.
  Contact perturbations and motor noise are left out (their draws are
  additive and drop out of the gradient; the comparisons set them to zero).
  With cfg["event_time"] the contacts are resolved at their crossing time
  (qs_oracle.h, OR_F_EVENT_TIME); autograd then differentiates through the
  crossing times too.

The polar factor of the integrated rotation is Newton's iteration
X <- (X + X^-T)/2 with a fixed number of steps (converged in binary64 for the
near-orthogonal inputs of one substep). Nothing here is shared with the CUDA
path; tests pin both forms to the C oracle (forward, events) and to finite
differences of the C oracle (gradient).
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


def _safe_norm(a):
    """Euclidean norm over the last axis; 1 where the vector is zero."""
    q = (a * a).sum(-1)
    return torch.sqrt(torch.where(q > 0.0, q, torch.ones_like(q)))


def _pair_lists(sizes):
    """Ordered pairs (i, j), i != j, of drones in the same env."""
    ii, jj = [], []
    off = 0
    for n in sizes:
        for a in range(n):
            for b in range(n):
                if a != b:
                    ii.append(off + a)
                    jj.append(off + b)
        off += n
    return torch.tensor(ii, dtype=torch.long), torch.tensor(jj, dtype=torch.long)


def _collide(x, arm, ii, jj):
    """Collision decision of each ordered pair: the binary32 key
    |x_j - x_i|^2 (differences, squares and sums each rounded to binary32,
    in the order x, y, z) against the binary32 threshold (l_i + l_j)^2."""
    import numpy as np
    xf = x.detach().numpy().astype(np.float32)
    lf = arm.detach().numpy().astype(np.float32)
    d = xf[jj.numpy()] - xf[ii.numpy()]
    sq = d * d
    key = (sq[:, 0] + sq[:, 1]) + sq[:, 2]
    thr = lf[ii.numpy()] + lf[jj.numpy()]
    thr = thr * thr
    return torch.from_numpy(key < thr)


def discrete_rollout_loss(x0, actions, params, goals, sizes, cfg, events=None):
    """Per-drone loss sum_t |x(t) - g|^2 + 1e-3 |f^(t)|^2 of T steps with the
    discrete contacts (flags: cfg["floor"], cfg["walls"], cfg["collisions"]),
    no motor noise and no contact perturbations. Same arguments as
    smooth_rollout_loss plus cfg["mu"], cfg["alpha_c"]; ``events``, if a
    list, receives each step's event bits (hit floor 1, on floor 2, wall 4,
    ceiling 8, quad 16) per drone. cfg["event_time"] (default False): the
    contacts at their crossing times (floor: tau = -z0 / v_z; walls and
    ceiling: the earliest boundary crossing of the substep's straight path;
    pairs: the contact distance on the pair's relative motion run back from
    the end of the step, at most the step's duration)."""
    dt, g = cfg["dt"], cfg["gravity"]
    et = bool(cfg.get("event_time", False))
    Tc = cfg["substeps"] * dt
    sizes = [int(n) for n in sizes]
    env_of = torch.repeat_interleave(torch.arange(len(sizes)), torch.tensor(sizes))
    P = params[env_of]
    m, I, t2w, tau_m, arm = P[:, 0], P[:, 1:4], P[:, 4], P[:, 5], P[:, 6]
    G = goals[env_of]
    fmax = 0.25 * m * g * t2w
    alag = 1.0 - torch.exp(-dt / tau_m)
    mu, ac, wmax = cfg["mu"], cfg["alpha_c"], cfg["omega_max"]
    lim = torch.tensor([cfg["room_hx"], cfg["room_hy"]], dtype=x0.dtype)
    ii, jj = _pair_lists(sizes)
    D = x0.shape[0]
    zero = torch.zeros(D, dtype=x0.dtype)

    x, v = x0[:, 0:3], x0[:, 3:6]
    R = x0[:, 6:15].reshape(-1, 3, 3)
    w, uf, eps = x0[:, 15:18], x0[:, 18:22], x0[:, 22:26]
    sa = arm / math.sqrt(2.0)
    loss = torch.zeros(D, dtype=x0.dtype)
    for t in range(actions.shape[0]):
        ev = torch.zeros(D, dtype=torch.int64)
        fh = torch.clamp(actions[t], 0.0, 1.0)
        u = torch.sqrt(fh)
        for s in range(cfg["substeps"]):
            # S1-S3: lag, thrust, wrench
            uf = alag[:, None] * (u - uf) + uf
            f = fmax[:, None] * uf * uf + eps
            T = f.sum(-1)
            tau = torch.stack([sa * (f[:, 0] + f[:, 1] - f[:, 2] - f[:, 3]),
                               sa * (-f[:, 0] + f[:, 1] + f[:, 2] - f[:, 3]),
                               cfg["kappa"] * (-f[:, 0] + f[:, 1] - f[:, 2] + f[:, 3])], -1)
            F = T[:, None] * R[:, :, 2]
            acc = F / m[:, None] - torch.tensor([0.0, 0.0, g], dtype=x.dtype)
            # S4 with the floor: thrust too weak to lift a drone at z <= 0
            on = torch.zeros(D, dtype=torch.bool)
            moving = torch.zeros(D, dtype=torch.bool)
            if cfg["floor"]:
                on = (x[:, 2] <= 0.0) & (F[:, 2] < m * g)
                ffric = mu * (m * g - F[:, 2])
                rest = (v[:, 0] == 0.0) & (v[:, 1] == 0.0)
                moving = on & ~rest
                # norms of zero vectors are taken as 1 in the branch not used, so
                # that no infinite derivative enters the graph
                nf = _safe_norm(F[:, 0:2])
                keep = torch.where(nf > ffric, (nf - ffric) / nf, zero)
                nv = _safe_norm(v[:, 0:2])
                f_static = F[:, 0:2] * keep[:, None]
                f_slide = F[:, 0:2] - ffric[:, None] * v[:, 0:2] / nv[:, None]
                fxy = torch.where(rest[:, None], f_static, f_slide)
                acc_on = torch.cat([fxy / m[:, None], zero[:, None]], -1)
                acc = torch.where(on[:, None], acc_on, acc)
                v = torch.where(on[:, None], torch.cat([v[:, 0:2], zero[:, None]], -1), v)
                ev = ev | torch.where(on, 2, 0)
            # S5: Euler's equation; S6: semi-implicit Euler and the polar factor
            wdot = (tau - torch.cross(w, I * w, dim=-1)) / I
            vold = v[:, 0:2]
            xs0 = x  # substep start (event-time contacts)
            v = v + acc * dt
            if cfg["floor"]:
                stop = moving & ((v[:, 0:2] * vold).sum(-1) < 0.0)
                v = torch.where(stop[:, None], torch.cat([zero[:, None], zero[:, None], v[:, 2:3]], -1), v)
            x = x + v * dt
            w = torch.clamp(w + wdot * dt, -wmax, wmax)
            R = polar(R + dt * R @ skew(w))
            # S7: floor hit: z, v, w to zero, upright keeping the body x-axis heading
            if cfg["floor"]:
                hit = (x[:, 2] <= 0.0) & (v[:, 2] < 0.0)
                hyp = _safe_norm(R[:, 0:2, 0])
                cs, sn = R[:, 0, 0] / hyp, R[:, 1, 0] / hyp
                o, z = torch.ones_like(cs), torch.zeros_like(cs)
                Rz = torch.stack([torch.stack([cs, -sn, z], -1), torch.stack([sn, cs, z], -1),
                                  torch.stack([z, z, o], -1)], -2)
                R = torch.where(hit[:, None, None], Rz, R)
                if et:
                    vz = torch.where(hit, v[:, 2], -torch.ones_like(zero))
                    tau = torch.clamp(-xs0[:, 2] / vz, 0.0, dt)
                    xy = xs0[:, 0:2] + v[:, 0:2] * tau[:, None]
                    x = torch.where(hit[:, None], torch.cat([xy, x[:, 2:3]], -1), x)
                x = torch.where(hit[:, None], torch.cat([x[:, 0:2], zero[:, None]], -1), x)
                v = torch.where(hit[:, None], torch.zeros_like(v), v)
                w = torch.where(hit[:, None], torch.zeros_like(w), w)
                ev = ev | torch.where(hit, 1, 0)
            # S8: walls and ceiling: back onto the boundary; an outward normal
            # velocity is removed, then the decay alpha_c
            if cfg["walls"]:
                xs, vs, clamped = [], [], []
                v1 = v
                tau = torch.full_like(zero, dt)
                hit_wall = torch.zeros(D, dtype=torch.bool)
                for k in range(2):
                    over, under = x[:, k] > lim[k], x[:, k] < -lim[k]
                    out = (over & (v[:, k] > 0.0)) | (under & (v[:, k] < 0.0))
                    hit_wall = hit_wall | out
                    if et:
                        bound = torch.where(over, lim[k] + 0.0 * x[:, k], -lim[k] + 0.0 * x[:, k])
                        vk = torch.where(out, v[:, k], torch.ones_like(zero))
                        tau = torch.where(out, torch.minimum(tau, (bound - xs0[:, k]) / vk), tau)
                    xs.append(torch.where(over, lim[k] + 0.0 * x[:, k], torch.where(under, -lim[k] + 0.0 * x[:, k],
                                                                                     x[:, k])))
                    vs.append(torch.where(out, zero, v[:, k]))
                    clamped.append(over | under)
                over = x[:, 2] > cfg["room_h"]
                hit_ceil = over & (v[:, 2] > 0.0)
                if et:
                    vk = torch.where(hit_ceil, v[:, 2], torch.ones_like(zero))
                    tau = torch.where(hit_ceil, torch.minimum(tau, (cfg["room_h"] - xs0[:, 2]) / vk), tau)
                xs.append(torch.where(over, cfg["room_h"] + 0.0 * x[:, 2], x[:, 2]))
                vs.append(torch.where(hit_ceil, zero, v[:, 2]))
                clamped.append(over)
                x, v = torch.stack(xs, -1), torch.stack(vs, -1)
                resp = hit_wall | hit_ceil
                v = torch.where(resp[:, None], ac * v, v)
                if et:
                    tau = torch.clamp(tau, min=0.0)
                    xe = xs0 + v1 * tau[:, None] + v * (dt - tau)[:, None]
                    free = resp[:, None] & ~torch.stack(clamped, -1)
                    x = torch.where(free, xe, x)
                ev = ev | torch.where(hit_wall, 4, 0) | torch.where(hit_ceil, 8, 0)
        # S9, S10: the pair set on the positions after the substeps and the
        # Jacobi response from the pre-collision velocities
        if cfg["collisions"] and ii.numel():
            coll = _collide(x, arm, ii, jj)
            hitq = torch.zeros(D, dtype=torch.bool).index_fill(0, ii[coll], True)
            ev = ev | torch.where(hitq, 16, 0)
            r = x[ii] - x[jj]
            dvv = v[ii] - v[jj]
            app = (dvv * r).sum(-1)
            sel = coll & (app < 0.0).detach()
            dist = _safe_norm(r)
            n = torch.where(((r * r).sum(-1) > 0.0)[:, None], r / dist[:, None],
                            torch.tensor([0.0, 0.0, 1.0], dtype=x.dtype).expand_as(r))
            vn = ((v[jj] - v[ii]) * n).sum(-1)
            contrib = torch.where(sel[:, None], vn[:, None] * n, torch.zeros_like(n))
            dv = torch.zeros_like(v).index_add(0, ii, contrib)
            responded = torch.zeros(D, dtype=torch.bool).index_fill(0, ii[sel], True)
            vpre = v
            v = torch.where(responded[:, None], ac * (v + dv), v)
            if et:
                # contact time sigma of each pair: |r - (v_i - v_j) sigma| = 2 l
                rho2 = (2.0 * arm[ii]) ** 2
                a_ = (dvv * dvv).sum(-1)
                c0 = (r * r).sum(-1) - rho2
                disc = torch.where(sel, app * app - a_ * c0, torch.ones_like(app))
                den = torch.where(sel, torch.sqrt(disc) - app, torch.ones_like(app))
                sig = torch.clamp(torch.where(sel, -c0 / den, torch.zeros_like(app)), 0.0, Tc)
                dx_et = torch.zeros_like(x).index_add(0, ii, contrib * sig[:, None])
                smax = torch.zeros_like(zero).scatter_reduce(0, ii, torch.where(sel, sig, torch.zeros_like(sig)),
                                                             reduce="amax", include_self=True)
                Dv = v - vpre - ac * dv
                x = torch.where(responded[:, None], x + ac * dx_et + Dv * smax[:, None], x)
        if events is not None:
            events.append(ev.numpy().copy())
        loss = loss + ((x - G) ** 2).sum(-1) + 1e-3 * (fh * fh).sum(-1)
    return loss
