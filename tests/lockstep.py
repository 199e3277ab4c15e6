"""Free-running parity with lockstep restarts (the protocol for runs of many
control steps).

A binary32 run (the CUDA path, or in the CPU floor test an FP64 run that
stores its state in binary32) and the FP64 oracle advance side by side from
the same binary32 state. After every control step:

* the discrete outputs of the binary32 side are its own canonical decisions:
  neighbour lists and collision flags equal the canonical binary32 pair keys
  (Sec. III-B, III-C) evaluated on its own positions, every drone, every step;
* against the oracle, event bits must be identical for every env whose
  oracle step took no decision within a relative margin of its threshold and
  no collision decision that the current position discrepancy could flip;
  neighbour lists must be identical for every drone of those envs whose
  ranking the discrepancy cannot change;
* an env that did take such a decision restarts from lockstep: the binary32
  side's state of that env is copied into the oracle (and into the
  conditioning instruments), since from there the two may legitimately
  branch apart. Restarts are counted; every drone stays in the comparison.

The conditioning instruments are FP64 oracle runs that round their state to
binary32 after every substep (to nearest, and stochastically under two salts).
Their deviation from the oracle measures how strongly each trajectory
amplifies perturbations of binary32 size: tumbling drones spinning near the
intermediate principal axis of inertia grow such perturbations exponentially
(Euler's equation, Sec. III-A), so after 100 steps a few percent of drones
leave 1e-5 in a rotation entry in any run that stores its state in binary32.
"""
from __future__ import annotations

import numpy as np

from oracle import oracle as O


def _ulp32(x):
    return np.spacing(np.abs(np.asarray(x, np.float64)).astype(np.float32)).astype(np.float64)


def robust_pair_decisions(xs, xo, arm, N, K):
    """Per drone of swarms of N: (collision decisions robust, ranking robust).

    xs: positions of the binary32 side, xo: the oracle's (binary64, its keys
    use their binary32 rounding); arm: per-env arm length. A decision is robust
    when the key |x_j - x_i|^2 cannot cross the threshold (or the neighbouring
    ranked key) under the observed position discrepancy: with
    delta_i = |xs_i - xo_i| + rounding of xo_i, |dk_ij| <= 2 d_ij (delta_i +
    delta_j) + (delta_i + delta_j)^2 plus a few binary32 ulps of the key."""
    D = xs.shape[0]
    E = D // N
    if N < 2:
        return np.ones(D, bool), np.ones(D, bool)
    xs = xs.reshape(E, N, 3)
    xo = xo.reshape(E, N, 3)
    delta = np.linalg.norm(xs - xo, axis=2) + np.sqrt(3.0) * _ulp32(xo).max(axis=2)
    diff = xo[:, None, :, :] - xo[:, :, None, :]
    k = (diff * diff).sum(-1)
    d = np.sqrt(k)
    dd = delta[:, :, None] + delta[:, None, :]
    bound = 2.0 * d * dd + dd * dd + 4.0 * _ulp32(k) + 1e-30
    thr = np.float32(2.0) * np.asarray(arm, np.float32)
    thr = (thr * thr).astype(np.float64)[:, None, None]
    eye = np.eye(N, dtype=bool)[None]
    hit_ok = ((np.abs(k - thr) > bound + _ulp32(thr)) | eye).all(axis=2)
    keff = min(K, N - 1)
    knn_ok = np.ones((E, N), bool)
    if keff > 0:
        kk = np.where(eye, np.inf, k)
        bb = np.where(eye, 0.0, bound)
        order = np.argsort(kk, axis=2, kind="stable")
        ks = np.take_along_axis(kk, order, axis=2)
        bs = np.take_along_axis(bb, order, axis=2)
        last = min(keff, N - 2)  # the boundary after rank keff-1 matters only if another drone follows
        for r in range(last + 1):
            knn_ok &= (ks[:, :, r + 1] - ks[:, :, r]) > bs[:, :, r] + bs[:, :, r + 1]
    return hit_ok.reshape(D), knn_ok.reshape(D)


def instruments(make_oracle, n_sr=2):
    """Conditioning instruments: oracle runs storing their state in binary32
    after each substep, to nearest and stochastically (n_sr salts)."""
    out = [make_oracle(O.F_ROUND32, 0)]
    for s in range(n_sr):
        out.append(make_oracle(O.F_ROUND32 | O.F_ROUND32_SR, s + 1))
    return out


def run(side, oracle, insts, acts, N, K, margin_thr=1e-5, cond_thr=0.1, check_own=True):
    """Advance the binary32 side, the oracle and the instruments in lockstep
    for len(acts) control steps (all from the side's current state), with
    restarts as described above. ``side`` provides step(a), state() -> dict of
    numpy arrays (state [D][30], params [E][7]) and events() -> (ev [D] uint32,
    knn [D][K] int32 or None). Returns the per-drone results at the end."""
    s0 = side.state()
    for o in [oracle] + insts:
        o.set_state(s0["state"], s0["params"], s0["goals"], s0["ep_step"], s0["tick"])
        o.clear_margin()
    D, E = s0["state"].shape[0], s0["params"].shape[0]
    eo = np.repeat(np.arange(E), N)
    arm = s0["params"][:, 6]
    off = np.arange(E + 1, dtype=np.int32) * N
    restarted = np.zeros(E, bool)
    last_restart = np.zeros(D, int)
    n_ev = n_knn = n_knn_exact = n_stable = 0
    for t, a in enumerate(acts):
        a64 = np.asarray(a, np.float64)
        side.step(a)
        oracle.step(a64)
        for o in insts:
            o.step(a64)
        ss = side.state()
        ev, knn = side.events()
        oev, oknn, margin = oracle.get_events()
        cond = oracle.last_cond
        xs, xo = ss["state"][:, 0:3], oracle.get_state()["state"][:, 0:3]
        if check_own and (K > 0 or N > 1):
            # the side's own decisions are the canonical ones on its own positions
            bk, bh = O.pairs_f32(xs.astype(np.float32), arm.astype(np.float32), off, K)
            assert np.array_equal((ev & O.EV_HIT_QUAD) != 0, bh.astype(bool)), f"step {t}: collision flags"
            if knn is not None and K > 0:
                assert np.array_equal(knn, bk), f"step {t}: neighbour lists"
        hit_ok, knn_ok = robust_pair_decisions(xs, xo, arm, N, K)
        unstable = np.zeros(E, bool)
        np.logical_or.at(unstable, eo, (margin < margin_thr) | (cond < cond_thr) | ~hit_ok)
        stable = ~unstable[eo]
        bad = stable & (ev != oev)
        assert not bad.any(), f"step {t}: event bits differ for {bad.sum()} drones, e.g. {np.flatnonzero(bad)[:5]}"
        n_ev += stable.sum()
        n_stable += stable.sum()
        if knn is not None and K > 0:
            sel = stable & knn_ok
            badk = sel & (knn != oknn[:, :K]).any(axis=1)
            assert not badk.any(), f"step {t}: neighbour lists differ for {badk.sum()} drones"
            n_knn += D
            n_knn_exact += sel.sum()
        if unstable.any():
            rows = unstable[eo]
            for o in [oracle] + insts:
                st = o.get_state()["state"]
                st[rows] = ss["state"][rows]
                o.set_state(st)
            restarted |= unstable
            last_restart[rows] = t + 1
        oracle.clear_margin()
    so = oracle.get_state()["state"]
    ss = side.state()["state"]
    dx = np.abs(ss[:, 0:3] - so[:, 0:3]).max(1)
    dR = np.abs(ss[:, 6:15] - so[:, 6:15]).max(1)
    inst_dR = np.array([np.abs(o.get_state()["state"][:, 6:15] - so[:, 6:15]).max(1) for o in insts])
    inst_dx = np.array([np.abs(o.get_state()["state"][:, 0:3] - so[:, 0:3]).max(1) for o in insts])
    return dict(dx=dx, dR=dR, inst_dR=inst_dR, inst_dx=inst_dx, envelope_R=inst_dR.max(0),
                restarted_envs=restarted.mean(), steps_compared=len(acts) - last_restart,
                event_comparisons=int(n_ev), knn_exact_frac=(n_knn_exact / n_knn if n_knn else None))


class OracleSide:
    """An oracle run playing the binary32 side (the CPU floor test)."""

    def __init__(self, o, K):
        self.o, self.K = o, K

    def step(self, a):
        self.o.step(np.asarray(a, np.float64))

    def state(self):
        return self.o.get_state()

    def events(self):
        ev, knn, _ = self.o.get_events()
        return ev, (knn[:, :self.K].astype(np.int32) if self.K > 0 else None)
