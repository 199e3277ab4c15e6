"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a closed
form, an invariant, a published known-answer vector, a special case or a
brute force on tiny inputs. Paper sections are cited per test.
"""
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2306_09537_gb300 import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))


def make(n_envs=1, sizes=None, flags=0, K=0, **kw):
    c = O.default_config(n_envs=n_envs, k_neighbors=K, flags=flags, seed=1)
    O.set_config(c, **kw)
    return c, O.Oracle(c, sizes)


def nominal(c):
    return np.array([c.mass, c.ixx, c.iyy, c.izz, c.t2w, c.tau_m, c.arm])


def base_state(n=1, x=(0.0, 0.0, 5.0), uf=math.sqrt(0.5), fprev=0.5):
    s = np.zeros((n, 30))
    s[:, 0:3] = x
    s[:, 6:15] = np.eye(3).ravel()
    s[:, 18:22] = uf
    s[:, 26:30] = fprev
    return s


def rz(psi):
    c, s = math.cos(psi), math.sin(psi)
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


def rx(a):
    c, s = math.cos(a), math.sin(a)
    return np.array([[1.0, 0.0, 0.0], [0.0, c, -s], [0.0, s, c]])


# --------------------------------------------------------------------------- P11 Philox
def test_philox_known_answers():
    """Random123 known-answer vectors for Philox4x32-10 (Salmon et al., SC'11)."""
    rows = [l.split() for l in open(os.path.join(HERE, "golden", "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(t, 16) for t in r]
        out = O.philox4x32_10(v[0:4], v[4:6])
        assert [int(x) for x in out] == v[6:10]


def test_uniform_map_exact_and_open():
    assert O.uniform(0) == 2.0 ** -24
    assert O.uniform(0xFFFFFFFF) == 1.0 - 2.0 ** -24
    # binary32-exact: (2k+1) 2^-24 with k < 2^23 has at most 24 significant bits
    for r in (1 << 9, 12345 << 9, 0x80000000, 0xDEADBEEF):
        u = O.uniform(r)
        assert float(np.float32(u)) == u


def test_philox_uniform_moments():
    n = 20000
    u = np.array([O.uniform(int(x)) for i in range(n // 4)
                  for x in O.philox4x32_10([i, 7, 3 << 16, 0], [11, 0])])
    assert abs(u.mean() - 0.5) < 4 * math.sqrt(1 / 12 / n)
    assert abs(u.var() - 1 / 12) < 4 * math.sqrt(1 / 180 / n)


# --------------------------------------------------------------------------- polar factor
def test_polar_factor_definition():
    """or_polar returns the unique rotation R with M = R H, H symmetric positive definite."""
    rng = np.random.default_rng(0)
    for _ in range(50):
        q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
        if np.linalg.det(q) < 0:
            q[:, 0] *= -1
        a = rng.standard_normal((3, 3))
        h = a @ a.T + 0.5 * np.eye(3)
        m = q @ h
        r = O.polar(m)
        assert np.abs(r @ r.T - np.eye(3)).max() < 1e-13
        assert abs(np.linalg.det(r) - 1.0) < 1e-13
        hh = r.T @ m
        assert np.abs(hh - hh.T).max() < 1e-12
        assert np.linalg.eigvalsh(0.5 * (hh + hh.T)).min() > 0
        assert np.abs(r - q).max() < 1e-11
    # a scaled rotation maps back to the rotation; a rotation is a fixed point
    q = rz(0.3) @ rx(-1.1)
    assert np.abs(O.polar(2.5 * q) - q).max() < 1e-14
    assert np.abs(O.polar(q) - q).max() < 1e-15


# --------------------------------------------------------------------------- P1 hover
def test_p1_hover_equilibrium():
    """Sec. III-A: with thrust f_max * u^2 = m g / 4 per rotor (t2w = 2, command 0.5),
    R = I and zero rates, gravity and thrust cancel: the state does not move."""
    c, o = make(flags=O.F_FLOOR | O.F_WALLS)
    st = base_state(x=(1.0, -2.0, 5.0))
    o.set_state(st, nominal(c)[None], np.zeros((1, 3)), np.zeros(1, np.int32), 0)
    for _ in range(1000):
        o.step(np.full((1, 4), 0.5))
    s = o.get_state()["state"]
    assert np.abs(s - st).max() < 1e-12


# --------------------------------------------------------------------------- P2 free fall
def test_p2_free_fall_discrete_closed_form():
    """Zero thrust: a = g exactly; semi-implicit Euler gives v_n = v0 - n g dt and
    z_n = z0 + n v0 dt - g dt^2 n(n+1)/2 after n substeps (Sec. III-A)."""
    c, o = make(flags=0)
    st = base_state(x=(0.5, -0.25, 500.0), uf=0.0, fprev=0.0)
    st[0, 3:6] = (0.3, -0.2, 1.0)
    o.set_state(st, nominal(c)[None], np.zeros((1, 3)), np.zeros(1, np.int32), 0)
    dt, g = c.dt, c.gravity
    for t in range(1, 201):
        o.step(np.zeros((1, 4)))
        if t % 40 == 0:
            n = 2 * t
            s = o.get_state()["state"][0]
            assert abs(s[5] - (1.0 - n * g * dt)) < 1e-10
            assert abs(s[2] - (500.0 + n * 1.0 * dt - g * dt * dt * n * (n + 1) / 2)) < 1e-9
            assert abs(s[0] - (0.5 + n * 0.3 * dt)) < 1e-12
            assert abs(s[1] - (-0.25 - n * 0.2 * dt)) < 1e-12
    # the continuous free fall is matched to first order in dt
    tt = 400 * dt
    assert abs(s[2] - (500.0 + tt - 0.5 * g * tt * tt)) < g * tt * dt


# --------------------------------------------------------------------------- P3 pure yaw
def test_p3_pure_yaw_response():
    """Commands (a, b, a, b): roll/pitch torques cancel, the yaw torque is
    2 kappa (f_b - f_a) (Sec. III-A tau_p), the lag follows its closed form,
    and the heading advances by atan(dt w_z) per substep (the polar factor of
    I + dt [w]x)."""
    c, o = make(flags=0)
    st = base_state(uf=0.6)
    o.set_state(st, nominal(c)[None], np.zeros((1, 3)), np.zeros(1, np.int32), 0)
    a, b = 0.3, 0.7
    act = np.array([[a, b, a, b]])
    dt = c.dt
    alpha = 1.0 - math.exp(-dt / c.tau_m)
    fmax = 0.25 * c.mass * c.gravity * c.t2w
    wz, psi = 0.0, 0.0
    for t in range(1, 51):
        o.step(act)
        for sub in (1, 2):
            k = 2 * (t - 1) + sub
            ufa = math.sqrt(a) + (0.6 - math.sqrt(a)) * (1 - alpha) ** k
            ufb = math.sqrt(b) + (0.6 - math.sqrt(b)) * (1 - alpha) ** k
            tz = 2 * c.kappa * (fmax * ufb ** 2 - fmax * ufa ** 2)
            wz += dt * tz / c.izz
            psi += math.atan(dt * wz)
        s = o.get_state()["state"][0]
        assert abs(s[17] - wz) < 1e-9 * max(1.0, abs(wz))
        assert np.abs(s[15:17]).max() < 1e-9
        assert np.abs(s[6:15].reshape(3, 3) - rz(psi)).max() < 1e-9
    assert abs(wz) > 1.0  # the test exercised a real rotation


# --------------------------------------------------------------------------- P4 motor lag
def test_p4_motor_lag_settling():
    """Sec. III-A: first-order lag whose 2% settling time is tau_m ln 50."""
    c, o = make(flags=0, substeps=1)
    st = base_state(uf=0.0, x=(0, 0, 900.0))
    o.set_state(st, nominal(c)[None], np.zeros((1, 3)), np.zeros(1, np.int32), 0)
    alpha = 1.0 - math.exp(-c.dt / c.tau_m)
    kstar = math.ceil(math.log(50.0) / -math.log(1.0 - alpha))
    hist = []
    for k in range(1, kstar + 3):
        o.step(np.ones((1, 4)))
        uf = o.get_state()["state"][0, 18]
        hist.append(uf)
        assert abs(uf - (1.0 - (1.0 - alpha) ** k)) < 1e-14
    assert hist[kstar - 1] >= 0.98 and hist[kstar - 2] < 0.98
    assert abs(kstar * c.dt - c.tau_m * math.log(50.0)) <= c.dt


# --------------------------------------------------------------------------- P5 motor noise
def test_p5_motor_noise_ar1_statistics():
    """Sec. III-A motor noise eps <- a_nd eps + a_ns N(0,1): stationary variance
    a_ns^2 / (1 - a_nd^2), lag-1 autocorrelation a_nd, zero mean."""
    E = 2000
    c, o = make(n_envs=E, flags=O.F_MOTOR_NOISE, substeps=1)
    st = base_state(E, x=(0, 0, 900.0))
    o.set_state(st, np.tile(nominal(c), (E, 1)), np.zeros((E, 3)), np.zeros(E, np.int32), 0)
    act = np.full((E, 4), 0.5)
    for _ in range(120):
        o.step(act)
    e0 = o.get_state()["state"][:, 22:26].ravel().copy()
    o.step(act)
    e1 = o.get_state()["state"][:, 22:26].ravel()
    ans = c.alpha_ns_frac * c.mass * c.gravity / 4
    var = ans ** 2 / (1 - c.alpha_nd ** 2)
    n = e0.size
    assert abs(e0.mean()) < 4 * math.sqrt(var / n)
    assert abs(e0.var() / var - 1) < 4 * math.sqrt(2 / n)
    rho = np.corrcoef(e0, e1)[0, 1]
    assert abs(rho - c.alpha_nd) < 4 * (1 - c.alpha_nd ** 2) / math.sqrt(n)


# --------------------------------------------------------------------------- P6 torque-free
def _torque_free(w0, substeps, steps=100):
    c, o = make(flags=0, substeps=substeps, dt=0.01 / substeps)
    st = base_state(uf=0.0, fprev=0.0, x=(0, 0, 900.0))
    st[0, 6:15] = (rz(0.4) @ rx(0.3)).ravel()
    st[0, 15:18] = w0
    o.set_state(st, nominal(c)[None], np.zeros((1, 3)), np.zeros(1, np.int32), 0)
    inertia = np.diag([c.ixx, c.iyy, c.izz])
    L0 = st[0, 6:15].reshape(3, 3) @ inertia @ np.asarray(w0)
    drift = 0.0
    for _ in range(steps):
        o.step(np.zeros((1, 4)))
        s = o.get_state()["state"][0]
        L = s[6:15].reshape(3, 3) @ inertia @ s[15:18]
        drift = max(drift, np.linalg.norm(L - L0) / np.linalg.norm(L0))
    return s, drift


def test_p6_torque_free_rotation():
    """Torque-free rigid body (Sec. III-A Euler equation with tau = 0): rotation
    about a principal axis keeps w constant; in general the world-frame angular
    momentum R I w is conserved up to the integrator's first-order error, which
    halves when dt halves. A wrong sign in w x (I w) or in dR/dt breaks this."""
    s, drift = _torque_free((0.0, 0.0, 3.0), 2)
    assert np.abs(s[15:18] - (0.0, 0.0, 3.0)).max() == 0.0
    assert drift < 1e-12
    w0 = (1.5, -0.7, 2.0)
    _, d1 = _torque_free(w0, 2)
    _, d2 = _torque_free(w0, 4)
    assert d1 < 2e-2
    assert 1.6 < d1 / d2 < 2.5


# --------------------------------------------------------------------------- P7 orthonormality
def test_p7_rotation_stays_orthonormal():
    E = 64
    c, o = make(n_envs=E, flags=O.F_MOTOR_NOISE)
    st = W.random_states(3, E, rate=10.0).astype(np.float64)
    st[:, 2] += 500.0
    o.set_state(st, np.tile(nominal(c), (E, 1)), np.zeros((E, 3)), np.zeros(E, np.int32), 0)
    acts = W.actions(3, 100, E)
    for t in range(100):
        o.step(acts[t])
        R = o.get_state()["state"][:, 6:15].reshape(E, 3, 3)
        assert np.abs(R @ R.transpose(0, 2, 1) - np.eye(3)).max() < 1e-12
        assert np.abs(np.linalg.det(R) - 1.0).max() < 1e-12


# --------------------------------------------------------------------------- P8 collisions
def test_p8_head_on_collision_swaps_normal_velocity():
    """Sec. III-B quad-quad rule with alpha = 1 and no noise: v1 + ((v2-v1).n) n
    swaps the normal components (equal masses): momentum and energy are
    conserved and the tangential components are kept."""
    c, o = make(n_envs=1, sizes=[2], flags=O.F_COLLISIONS, alpha_c=1.0, coll_sigma_v=0.0,
                coll_sigma_w=0.0)
    st = base_state(2)
    st[0, 0:3] = (0.0, 0.0, 5.0)
    st[1, 0:3] = (0.05, 0.0, 5.0)
    st[0, 3:6] = (1.0, 0.0, 0.0)
    st[1, 3:6] = (-1.0, 0.0, 0.0)
    o.set_state(st, nominal(c)[None], np.zeros((1, 3)), np.zeros(1, np.int32), 0)
    o.step(np.full((2, 4), 0.5))
    s = o.get_state()["state"]
    ev, _, _ = o.get_events()
    assert (ev & O.EV_HIT_QUAD).all()
    assert np.abs(s[0, 3:6] - (-1.0, 0.0, 0.0)).max() < 1e-12
    assert np.abs(s[1, 3:6] - (1.0, 0.0, 0.0)).max() < 1e-12

    rng = np.random.default_rng(5)
    for _ in range(20):
        n = rng.standard_normal(3)
        n /= np.linalg.norm(n)
        c, o = make(n_envs=1, sizes=[2], flags=O.F_COLLISIONS, alpha_c=1.0, coll_sigma_v=0.0,
                    coll_sigma_w=0.0)
        st = base_state(2)
        st[1, 0:3] = st[0, 0:3] + 0.06 * n
        v1, v2 = 0.5 * n + rng.uniform(-0.3, 0.3, 3), -0.5 * n + rng.uniform(-0.3, 0.3, 3)
        st[0, 3:6], st[1, 3:6] = v1, v2
        o.set_state(st, nominal(c)[None], np.zeros((1, 3)), np.zeros(1, np.int32), 0)
        before = o.get_state()["state"]
        o.step(np.full((2, 4), 0.5))
        # substeps move the drones (hover: no acceleration), then the response
        after = o.get_state()["state"]
        vb, va = before[:, 3:6], after[:, 3:6]
        assert np.abs(va.sum(0) - vb.sum(0)).max() < 1e-12
        assert abs((va ** 2).sum() - (vb ** 2).sum()) < 1e-12
        nn = after[0, 0:3] - after[1, 0:3]
        nn /= np.linalg.norm(nn)
        for i, j in ((0, 1), (1, 0)):
            assert abs(va[i] @ nn - vb[j] @ nn) < 1e-12
            assert np.abs((va[i] - (va[i] @ nn) * nn) - (vb[i] - (vb[i] @ nn) * nn)).max() < 1e-12


def test_separating_pair_only_flags():
    """Overlapping but separating drones are flagged and keep their velocities."""
    c, o = make(n_envs=1, sizes=[2], flags=O.F_COLLISIONS, alpha_c=0.5)
    st = base_state(2)
    st[1, 0:3] = (0.04, 0.0, 5.0)
    st[0, 3:6] = (-0.2, 0.0, 0.0)
    st[1, 3:6] = (0.2, 0.0, 0.0)
    o.set_state(st, nominal(c)[None], np.zeros((1, 3)), np.zeros(1, np.int32), 0)
    o.step(np.full((2, 4), 0.5))
    ev, _, _ = o.get_events()
    assert (ev & O.EV_HIT_QUAD).all()
    s = o.get_state()["state"]
    assert np.abs(s[:, 3:6] - st[:, 3:6]).max() < 1e-12


# --------------------------------------------------------------------------- P9 room contacts
def test_p9_wall_removes_normal_velocity():
    """Sec. III-B wall rule: the quad-quad rule with a static partner removes the
    normal component, keeps alpha_c times the tangential one; position clamped."""
    c, o = make(flags=O.F_WALLS, alpha_c=0.8, coll_sigma_v=0.0, coll_sigma_w=0.0)
    st = base_state(x=(4.999, 0.0, 5.0))
    st[0, 3:6] = (1.0, 0.5, 0.0)
    o.set_state(st, nominal(c)[None], np.zeros((1, 3)), np.zeros(1, np.int32), 0)
    o.step(np.full((1, 4), 0.5))
    s = o.get_state()["state"][0]
    ev, _, _ = o.get_events()
    assert ev[0] & O.EV_HIT_WALL and not ev[0] & O.EV_HIT_CEIL
    assert s[0] == 5.0
    assert abs(s[3]) < 1e-12 and abs(s[4] - 0.4) < 1e-12
    # ceiling
    c, o = make(flags=O.F_WALLS, alpha_c=0.8, coll_sigma_v=0.0, coll_sigma_w=0.0)
    st = base_state(x=(0.0, 0.0, 9.999))
    st[0, 3:6] = (0.0, 0.0, 1.0)
    o.set_state(st, nominal(c)[None], np.zeros((1, 3)), np.zeros(1, np.int32), 0)
    o.step(np.full((1, 4), 0.5))
    s = o.get_state()["state"][0]
    ev, _, _ = o.get_events()
    assert ev[0] & O.EV_HIT_CEIL and s[2] == 10.0 and abs(s[5]) < 1e-12


def test_p9_floor_hit_resets_momenta_keeps_heading():
    """Sec. III-B ground: on hitting the floor v, w -> 0, body z-axis upright."""
    c, o = make(flags=O.F_FLOOR)
    st = base_state(x=(0.3, 0.1, 0.001))
    R0 = rz(0.9) @ rx(0.2)
    st[0, 6:15] = R0.ravel()
    st[0, 3:6] = (0.3, 0.2, -1.0)
    st[0, 15:18] = (0.1, -0.2, 0.3)
    o.set_state(st, nominal(c)[None], np.zeros((1, 3)), np.zeros(1, np.int32), 0)
    o.step(np.full((1, 4), 0.3))  # below hover: the drone then rests on the floor
    s = o.get_state()["state"][0]
    ev, _, _ = o.get_events()
    assert ev[0] & O.EV_HIT_FLOOR and ev[0] & O.EV_ON_FLOOR
    assert s[2] == 0.0 and np.all(s[3:6] == 0.0) and np.all(s[15:18] == 0.0)
    R = s[6:15].reshape(3, 3)
    assert R[2, 2] == 1.0 and R[0, 2] == 0.0 and R[1, 2] == 0.0 and R[2, 0] == 0.0
    psi = math.atan2(R[1, 0], R[0, 0])
    assert abs(psi - math.atan2(R0[1, 0], R0[0, 0])) < 0.01
    assert np.abs(R - rz(psi)).max() < 1e-14


def test_p9_static_and_sliding_friction():
    """Sec. III-B ground: at rest with |F_xy| <= mu (m g - F_z) nothing moves;
    otherwise the drone accelerates by (|F_xy| - mu (m g - F_z)) / m."""
    c, o = make(flags=O.F_FLOOR)
    st = base_state(x=(1.0, 2.0, 0.0), uf=math.sqrt(0.4), fprev=0.4)
    st[0, 6:15] = rx(0.05).ravel()
    o.set_state(st, nominal(c)[None], np.zeros((1, 3)), np.zeros(1, np.int32), 0)
    for _ in range(10):
        o.step(np.full((1, 4), 0.4))
    s = o.get_state()["state"][0]
    ev, _, _ = o.get_events()
    assert ev[0] & O.EV_ON_FLOOR
    assert s[0] == 1.0 and s[1] == 2.0 and s[2] == 0.0 and np.all(s[3:6] == 0.0)

    c, o = make(flags=O.F_FLOOR, substeps=1)
    st = base_state(x=(1.0, 2.0, 0.0), uf=math.sqrt(0.4), fprev=0.4)
    st[0, 6:15] = rx(0.3).ravel()
    o.set_state(st, nominal(c)[None], np.zeros((1, 3)), np.zeros(1, np.int32), 0)
    o.step(np.full((1, 4), 0.4))
    s = o.get_state()["state"][0]
    m, g = c.mass, c.gravity
    T = 0.8 * m * g
    Fxy, Fz = T * math.sin(0.3), T * math.cos(0.3)
    a = (Fxy - c.mu * (m * g - Fz)) / m
    # F = R (0,0,T) with R = Rx(0.3): F_y = -T sin(0.3)
    assert abs(s[4] - (-a * c.dt)) < 1e-12 and abs(s[3]) < 1e-15 and s[5] == 0.0


# --------------------------------------------------------------------------- P10 KNN + collisions
def _brute_pairs(pos, arm, off, K):
    D = int(off[-1])
    knn = -np.ones((D, K), dtype=np.int32)
    hit = np.zeros(D, dtype=np.uint8)
    for e in range(len(off) - 1):
        a, b = off[e], off[e + 1]
        n = b - a
        r = np.float32(arm[e]) + np.float32(arm[e])
        thr = np.float32(r * r)
        for i in range(n):
            keys, idx = [], []
            for j in range(n):
                if j == i:
                    continue
                d = (pos[a + j] - pos[a + i]).astype(np.float32)
                sq = d * d
                k = np.float32(np.float32(sq[0] + sq[1]) + sq[2])
                keys.append(k)
                idx.append(j)
                if k < thr:
                    hit[a + i] = 1
            order = np.lexsort((np.array(idx), np.array(keys, dtype=np.float32)))
            for q in range(min(K, n - 1)):
                knn[a + i, q] = idx[order[q]]
    return knn, hit


def test_p10_knn_and_collision_sets_brute_force():
    """Sec. II-B / III-C: the K nearest by (binary32 key, index) with ties broken
    by the lower index; collision iff key < (l_i + l_j)^2. Brute force on
    tiny swarms with forced duplicate positions and N - 1 < K."""
    rng = np.random.default_rng(11)
    for trial in range(300):
        sizes = rng.integers(1, 9, size=rng.integers(1, 5))
        pos = W.clustered_positions(trial, sizes, spread=0.1, dup_frac=0.3)
        arm = rng.uniform(0.03, 0.06, len(sizes)).astype(np.float32)
        off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int32)
        K = int(rng.integers(0, 7))
        knn, hit = O.pairs_f32(pos, arm, off, K)
        bk, bh = _brute_pairs(pos, arm, off, K)
        assert np.array_equal(knn, bk)
        assert np.array_equal(hit, bh)


def test_knn_is_euclidean_nearest_when_untied():
    """With well separated distances the canonical order is the Euclidean order."""
    rng = np.random.default_rng(2)
    for _ in range(200):
        n = int(rng.integers(2, 12))
        pos = rng.uniform(-3, 3, (n, 3)).astype(np.float32)
        d = np.linalg.norm(pos[:, None, :].astype(np.float64) - pos[None, :, :], axis=2)
        K = min(6, n - 1)
        knn, _ = O.pairs_f32(pos, np.array([0.046], np.float32), np.array([0, n], np.int32), K)
        for i in range(n):
            di = np.delete(d[i], i)
            ji = np.delete(np.arange(n), i)
            srt = np.sort(di)
            if srt.size > 1 and np.min(np.diff(srt)) < 1e-4 * srt[-1]:
                continue
            assert list(knn[i]) == list(ji[np.argsort(di)][:K])


def test_step_knn_matches_pair_function_on_parked_swarm():
    """Drones hovering at rest keep their binary32 positions over a step, so the
    step's neighbour lists equal the stand-alone pair pass on those positions."""
    sizes = [8, 3, 5, 1]
    E = len(sizes)
    c, o = make(n_envs=E, sizes=sizes, K=6, flags=O.F_COLLISIONS | O.F_RECORD_KNN, alpha_c=1.0)
    pos = W.clustered_positions(4, sizes, spread=0.08, dup_frac=0.25)
    st = base_state(sum(sizes))
    st[:, 0:3] = pos
    o.set_state(st, np.tile(nominal(c), (E, 1)), np.zeros((E, 3)), np.zeros(E, np.int32), 0)
    o.step(np.full((sum(sizes), 4), 0.5))
    ev, knn, _ = o.get_events()
    s = o.get_state()["state"]
    assert np.array_equal(s[:, 0:3].astype(np.float32), pos)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int32)
    bk, bh = _brute_pairs(pos, np.full(E, np.float32(c.arm)), off, 6)
    assert np.array_equal(knn, bk)
    assert np.array_equal((ev & O.EV_HIT_QUAD) != 0, bh.astype(bool))


# --------------------------------------------------------------------------- P12 DR + reset
def test_p12_domain_randomisation():
    E = 4000
    c, o = make(n_envs=E, flags=O.F_DR)
    o.reset(123)
    prm = o.get_state()["params"]
    nom = nominal(c)
    ratio = prm / nom
    assert ratio.min() >= 0.8 and ratio.max() <= 1.2
    assert np.all(np.abs(ratio.mean(0) - 1.0) < 4 * 0.4 / math.sqrt(12 * E))
    o2 = O.Oracle(c)
    o2.reset(123)
    assert np.array_equal(o2.get_state()["params"], prm)
    o2.reset(124)
    assert not np.array_equal(o2.get_state()["params"], prm)
    c0, o0 = make(n_envs=3, flags=0)
    o0.reset(5)
    assert np.array_equal(o0.get_state()["params"], np.tile(nom, (3, 1)))


def test_reset_initial_state_distribution():
    """Initial state: position uniform in the room, v and w uniform in [-1,1],
    orientation uniform on SO(3) (E[R] = 0, E[R_ij^2] = 1/3), hover motors."""
    E = 5000
    c, o = make(n_envs=E, flags=O.F_DR)
    o.reset(9)
    s = o.get_state()
    st, prm, goal = s["state"], s["params"], s["goals"]
    assert st[:, 0].min() >= -5 and st[:, 0].max() <= 5 and st[:, 2].min() >= 0 and st[:, 2].max() <= 10
    assert np.abs(st[:, 3:6]).max() <= 1 and np.abs(st[:, 15:18]).max() <= 1
    R = st[:, 6:15].reshape(E, 3, 3)
    assert np.abs(R @ R.transpose(0, 2, 1) - np.eye(3)).max() < 1e-12
    assert np.abs(np.linalg.det(R) - 1).max() < 1e-12
    assert np.abs(R.mean(0)).max() < 4 * math.sqrt(1 / 3 / E)
    assert np.abs((R ** 2).mean(0) - 1 / 3).max() < 4 * math.sqrt(4 / 45 / E)
    assert np.allclose(st[:, 18], np.sqrt(1 / prm[:, 4])) and np.allclose(st[:, 26], 1 / prm[:, 4])
    assert np.all(st[:, 22:26] == 0)
    assert goal[:, 2].min() >= 0 and goal[:, 2].max() <= 10 and np.abs(goal[:, :2]).max() <= 5


# --------------------------------------------------------------------------- observations, reward, done
def test_observation_layout_and_sensor_noise():
    """Sec. III-C: [x - g, v, R, w, (x_j - x_i, v_j - v_i) for the K nearest];
    sensor noise U(-s,s) on x and v, N(0, s^2) on w."""
    sizes = [4] * 500
    E = len(sizes)
    c, o = make(n_envs=E, sizes=sizes, K=2, flags=O.F_RECORD_KNN)
    o.reset(31)
    acts = W.actions(31, 1, sum(sizes))[0]
    obs, _, _ = o.step(acts)
    s = o.get_state()
    st, goal = s["state"], s["goals"]
    _, knn, _ = o.get_events()
    env_of = np.repeat(np.arange(E), 4)
    assert np.allclose(obs[:, 0:3], st[:, 0:3] - goal[env_of], atol=1e-14)
    assert np.allclose(obs[:, 3:6], st[:, 3:6]) and np.allclose(obs[:, 6:15], st[:, 6:15])
    assert np.allclose(obs[:, 15:18], st[:, 15:18])
    base = env_of * 4
    for k in range(2):
        j = base + knn[:, k]
        assert np.allclose(obs[:, 18 + 6 * k:21 + 6 * k], st[j, 0:3] - st[:, 0:3], atol=1e-14)
        assert np.allclose(obs[:, 21 + 6 * k:24 + 6 * k], st[j, 3:6] - st[:, 3:6], atol=1e-14)

    c2, o2 = make(n_envs=E, sizes=sizes, K=2, flags=O.F_RECORD_KNN | O.F_OBS_NOISE)
    o2.reset(31)
    obs2, _, _ = o2.step(acts)
    nx, nv, nw = (obs2 - obs)[:, 0:3], (obs2 - obs)[:, 3:6], (obs2 - obs)[:, 15:18]
    assert np.abs(obs2[:, 6:15] - obs[:, 6:15]).max() == 0 and np.abs(obs2[:, 18:] - obs[:, 18:]).max() == 0
    for noise, sig in ((nx, 5e-3), (nv, 1e-2)):
        assert np.abs(noise).max() <= sig
        assert abs(noise.var() / (sig ** 2 / 3) - 1) < 0.05
    assert abs(nw.std() / 1.75e-4 - 1) < 0.05


def test_reward_special_case_identity_pose():
    """Sec. III-E at the goal, at rest, R = I, command f^ = f^_prev = 0.5 on all
    rotors: distance, speed, spin and command-change terms vanish; R22 = 1,
    (tr R - 1)/2 = 1, R00 = 1, |f^| = 1."""
    weights = {"pos": -3.0, "vel": -5.0, "ori": 0.7, "spin": -11.0, "act": 0.13, "dact": -17.0,
               "rot": 0.19, "yaw": 0.23}
    c, o = make(flags=0, weights=weights)
    st = base_state(x=(1.0, 2.0, 3.0))
    o.set_state(st, nominal(c)[None], np.array([[1.0, 2.0, 3.0]]), np.zeros(1, np.int32), 0)
    _, r, _ = o.step(np.full((1, 4), 0.5))
    assert abs(r[0] - (0.7 + 0.13 + 0.19 + 0.23)) < 1e-9


def test_done_and_auto_reset():
    """Episodes end after episode_steps control steps (15 s at 100 Hz, Sec. IV)."""
    c, o = make(n_envs=2, flags=O.F_AUTO_RESET, episode_steps=5)
    o.reset(3)
    st0 = o.get_state()["state"].copy()
    for t in range(1, 6):
        _, _, d = o.step(np.full((2, 4), 0.5))
        assert d.tolist() == ([1, 1] if t == 5 else [0, 0])
    s = o.get_state()
    assert s["ep_step"].tolist() == [0, 0]
    assert not np.allclose(s["state"], st0)


# --------------------------------------------------------------------------- smooth contacts
def test_smooth_floor_equilibrium():
    """Softplus floor penalty k_c sp_beta(-z)/m balances gravity at
    sp_beta(-z*) = 1 / smooth_kc, i.e. z* = -log(exp(beta / kc) - 1) / beta."""
    c, o = make(flags=O.F_SMOOTH)
    beta, kc = c.smooth_beta, c.smooth_kc
    zs = -math.log(math.expm1(beta / kc)) / beta
    st = base_state(x=(0.0, 0.0, zs), uf=0.0, fprev=0.0)
    o.set_state(st, nominal(c)[None], np.zeros((1, 3)), np.zeros(1, np.int32), 0)
    for _ in range(20):
        o.step(np.zeros((1, 4)))
    s = o.get_state()["state"][0]
    assert abs(s[2] - zs) < 1e-12 and np.abs(s[3:6]).max() < 1e-12


def test_smooth_pair_forces_cancel():
    """Equal and opposite pair penalties: total velocity changes by gravity only."""
    c, o = make(n_envs=1, sizes=[3], flags=O.F_SMOOTH)
    st = base_state(3, uf=0.0, fprev=0.0)
    st[:, 0:3] = [[0.0, 0.0, 5.0], [0.05, 0.01, 5.02], [-0.03, 0.04, 4.99]]
    st[:, 3:6] = [[0.1, 0.0, 0.0], [0.0, -0.2, 0.1], [0.0, 0.0, 0.3]]
    o.set_state(st, nominal(c)[None], np.zeros((1, 3)), np.zeros(1, np.int32), 0)
    for t in range(1, 6):
        o.step(np.zeros((3, 4)))
    s = o.get_state()["state"]
    expect = st[:, 3:6].sum(0) + np.array([0, 0, -3 * c.gravity * 10 * c.dt])
    assert np.abs(s[:, 3:6].sum(0) - expect).max() < 1e-11
    assert np.abs(s[:, 3:6] - st[:, 3:6]).max() > 0.1  # the penalty acted


def test_body_rate_bound():
    """Body rates saturate at omega_max per axis (reading; the paper is silent)."""
    c, o = make(flags=0)
    st = base_state(uf=0.0, fprev=0.0, x=(0, 0, 900.0))
    st[0, 15:18] = (0.0, 0.0, 60.0)
    o.set_state(st, nominal(c)[None], np.zeros((1, 3)), np.zeros(1, np.int32), 0)
    o.step(np.zeros((1, 4)))
    s = o.get_state()["state"][0]
    assert s[17] == c.omega_max == 40.0 and s[15] == 0.0 and s[16] == 0.0
    R = s[6:15].reshape(3, 3)
    assert abs(math.atan2(R[1, 0], R[0, 0]) - 2 * math.atan(c.dt * 40.0)) < 1e-12


# --------------------------------------------------------------------------- downwash
def _downwash_case(above, sig=0.0):
    """Drone 0 hovering at (0,0,5); drones in `above` at the given offsets."""
    n = 1 + len(above)
    c, o = make(n_envs=1, sizes=[n], flags=O.F_DOWNWASH, dw_sigma_a=sig, dw_sigma_w=sig)
    st = base_state(n)
    for k, off in enumerate(above):
        st[1 + k, 0:3] = np.array([0.0, 0.0, 5.0]) + np.asarray(off)
    o.set_state(st, nominal(c)[None], np.zeros((1, 3)), np.zeros(1, np.int32), 0)
    o.step(np.full((n, 4), 0.5))
    return c, o.get_state()["state"]


def test_downwash_closed_form():
    """Sec. III-B downwash on the lower drone: k1 (k2 dz + b1) for a drone
    overlapping it from above within the height window, acting for one control
    step; none on the upper drone, none outside the window; contributions add."""
    for dz in (0.1, 0.25, 0.4):
        c, s = _downwash_case([(0.01, -0.02, dz)])
        Tc = c.substeps * c.dt
        want = -Tc * c.dw_k1 * (c.dw_k2 * dz + c.dw_b1)
        assert abs(s[0, 5] - want) < 1e-12 and np.abs(s[0, 3:5]).max() < 1e-12
        assert np.abs(s[1, 3:6]).max() < 1e-12
        assert np.abs(s[:, 15:18]).max() < 1e-12
    assert abs(_downwash_case([(0.0, 0.0, 0.25)])[1][0, 5] - 0.5 * _downwash_case([(0.0, 0.0, 0.0001)])[1][0, 5]) < 1e-5
    for off in ((0.2, 0.0, 0.2), (0.0, 0.0, 0.6), (0.0, 0.0, -0.2)):  # beside, too high, below
        _, s = _downwash_case([off])
        assert np.abs(s[0, 3:6]).max() < 1e-12
    c, s2 = _downwash_case([(0.0, 0.01, 0.1), (0.01, 0.0, 0.3)])
    Tc = c.substeps * c.dt
    want = -Tc * c.dw_k1 * ((c.dw_k2 * 0.1 + c.dw_b1) + (c.dw_k2 * 0.3 + c.dw_b1))
    assert abs(s2[0, 5] - want) < 1e-12


def test_downwash_noise_moments():
    """The downwash disturbances eps_d and eps_wd (Sec. III-B) are zero-mean
    Gaussian with the configured scales, act for one control step, and reach
    only the drone underneath."""
    E = 4000
    c, o = make(n_envs=E, sizes=[2] * E, flags=O.F_DOWNWASH)
    st = base_state(2 * E)
    st[1::2, 2] += 0.2
    o.set_state(st, np.tile(nominal(c), (E, 1)), np.zeros((E, 3)), np.zeros(E, np.int32), 0)
    o.step(np.full((2 * E, 4), 0.5))
    s = o.get_state()["state"]
    Tc = c.substeps * c.dt
    lower, upper = s[0::2], s[1::2]
    dv = lower[:, 3:6] - np.array([0.0, 0.0, -Tc * c.dw_k1 * (c.dw_k2 * 0.2 + c.dw_b1)])
    for k in range(3):
        assert abs(dv[:, k].mean()) < 4 * Tc * c.dw_sigma_a / math.sqrt(E)
        assert abs(dv[:, k].std() / (Tc * c.dw_sigma_a) - 1.0) < 0.05
        assert abs(lower[:, 15 + k].std() / (Tc * c.dw_sigma_w) - 1.0) < 0.05
    assert abs(np.corrcoef(dv[:, 0], lower[:, 15])[0, 1]) < 0.06
    assert np.abs(upper[:, 3:6]).max() < 1e-12 and np.abs(upper[:, 15:18]).max() < 1e-12
