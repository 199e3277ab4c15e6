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


def ry(a):
    c, s = math.cos(a), math.sin(a)
    return np.array([[c, 0.0, s], [0.0, 1.0, 0.0], [-s, 0.0, c]])


@pytest.mark.parametrize("axis", ["roll", "pitch"])
def test_p3_roll_and_pitch_from_the_rotor_layout(axis):
    """Sec. III-A: the thrust torque is the sum of p_r x (0, 0, f_r) over rotors
    at p_r = l (cos t_r, sin t_r, 0), t_r = 45 + 90 r degrees (X layout). Commands
    (a, a, b, b) give a pure roll torque, (a, b, b, a) a pure pitch torque (the
    other thrust torque and the yaw torque cancel); with the motors at their lag
    fixed point the torque is constant, the rotation stays about one principal
    axis (no gyroscopic term), so after n substeps w = n dt tau / I exactly and
    the attitude is the rotation about that axis by the sum of atan(dt w)."""
    c, o = make(flags=0)
    a, b = 0.55, 0.45
    f_hat = np.array([a, a, b, b]) if axis == "roll" else np.array([a, b, b, a])
    st = base_state()
    st[0, 18:22] = np.sqrt(f_hat)   # u_f = sqrt(f^): the lag leaves it unchanged
    st[0, 26:30] = f_hat
    o.set_state(st, nominal(c)[None], np.zeros((1, 3)), np.zeros(1, np.int32), 0)
    fmax = 0.25 * c.mass * c.gravity * c.t2w
    f = fmax * f_hat
    tau = np.zeros(3)
    for r in range(4):
        t = math.radians(45.0 + 90.0 * r)
        tau += np.cross(c.arm * np.array([math.cos(t), math.sin(t), 0.0]), np.array([0.0, 0.0, f[r]]))
    k, inertia, rot = (0, c.ixx, rx) if axis == "roll" else (1, c.iyy, ry)
    assert abs(tau[1 - k]) < 1e-18 and tau[2] == 0.0 and abs(tau[k]) > 1e-4
    # rotors at +y (roll) or +x (pitch) push harder: roll rate positive, pitch rate negative
    assert (tau[k] > 0) == (axis == "roll")
    dt, w, ang = c.dt, 0.0, 0.0
    for t in range(1, 11):
        o.step(f_hat[None])
        for sub in range(2):
            w += dt * tau[k] / inertia
            ang += math.atan(dt * w)
        s = o.get_state()["state"][0]
        assert abs(s[15 + k] - w) < 1e-9 * max(1.0, abs(w)), t
        assert abs(s[15 + (1 - k)]) < 1e-12 and abs(s[17]) < 1e-12
        assert np.abs(s[6:15].reshape(3, 3) - rot(ang)).max() < 1e-9, t
    assert abs(w) > 1.0


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


def _gaussian(x, sigma):
    """Sample x of N(0, sigma^2): mean, variance and kurtosis within 4 standard
    errors."""
    n = x.size
    m, v = x.mean(), x.var()
    kurt = ((x - m) ** 4).mean() / v ** 2
    return abs(m) < 4 * sigma / math.sqrt(n) and abs(v / sigma ** 2 - 1) < 4 * math.sqrt(2 / n) \
        and abs(kurt - 3) < 4 * math.sqrt(24 / n)


@pytest.mark.parametrize("contact", ["quad", "wall"])
def test_contact_perturbations_are_gaussian(contact):
    """Sec. III-B: a responding drone gets v <- alpha (v + v~ + eps_v) and
    w <- w + eps_w with Gaussian eps. With alpha = 1 and the contact the last
    event of the step (the pair response follows both substeps; the wall is
    crossed in the second substep), the difference to the same step without
    perturbation is eps itself: each component N(0, sigma^2), uncorrelated."""
    n_env, sv, sw = 4000, 0.2, 0.5
    runs = []
    for sig_v, sig_w in ((sv, sw), (0.0, 0.0)):
        if contact == "quad":
            c, o = make(n_envs=n_env, sizes=[2] * n_env, flags=O.F_COLLISIONS, alpha_c=1.0, coll_sigma_v=sig_v,
                        coll_sigma_w=sig_w)
            st = base_state(2 * n_env)
            st[1::2, 0] = 0.05
            st[0::2, 3], st[1::2, 3] = 1.0, -1.0
            goals = np.zeros((n_env, 3))
        else:
            c, o = make(n_envs=n_env, flags=O.F_WALLS, alpha_c=1.0, coll_sigma_v=sig_v, coll_sigma_w=sig_w)
            st = base_state(n_env, x=(5.0 - 1.5 * c.dt, 0.0, 5.0))
            st[:, 3:6] = (1.0, 0.5, 0.0)
            goals = np.zeros((n_env, 3))
        o.set_state(st, np.tile(nominal(c), (n_env, 1)), goals, np.zeros(n_env, np.int32), 0)
        o.step(np.full((st.shape[0], 4), 0.5))
        ev, _, _ = o.get_events()
        assert (ev & (O.EV_HIT_QUAD if contact == "quad" else O.EV_HIT_WALL)).all()
        runs.append(o.get_state()["state"])
    dv = runs[0][:, 3:6] - runs[1][:, 3:6]
    dw = runs[0][:, 15:18] - runs[1][:, 15:18]
    for k in range(3):
        assert _gaussian(dv[:, k], sv), ("v", k, dv[:, k].mean(), dv[:, k].std())
        assert _gaussian(dw[:, k], sw), ("w", k, dw[:, k].mean(), dw[:, k].std())
    corr = np.corrcoef(np.hstack([dv, dw]).T)
    assert np.abs(corr - np.eye(6)).max() < 4 / math.sqrt(dv.shape[0])


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


def test_event_time_floor_and_wall_crossing_closed_form():
    """Event-time contacts (beyond the paper; the differentiable model's
    variant): motors off, upright, one substep. Floor: the drone crosses
    z = 0 at tau = -z0 / v1_z on the straight path x0 + v1 s (v1 = v0 + g dt,
    semi-implicit Euler) and stops there, so x_xy = x0_xy + v1_xy tau
    instead of x0_xy + v1_xy dt. Wall: the first crossing of x = 5 at
    tau = (5 - x0) / v1_x; after it the tangential coordinates move with
    alpha_c v1 (no perturbation), the normal one stays on the wall."""
    dt = 0.005
    c, o = make(flags=O.F_FLOOR | O.F_EVENT_TIME, substeps=1, dt=dt)
    st = base_state(x=(0.3, 0.1, 0.004), uf=0.0, fprev=0.0)
    st[0, 3:6] = (1.0, 0.5, -1.0)
    o.set_state(st, nominal(c)[None], np.zeros((1, 3)), np.zeros(1, np.int32), 0)
    o.step(np.zeros((1, 4)))
    s = o.get_state()["state"][0]
    v1z = -1.0 - c.gravity * dt
    tau = -0.004 / v1z
    assert s[2] == 0.0 and np.all(s[3:6] == 0.0)
    assert abs(s[0] - (0.3 + 1.0 * tau)) < 1e-15 and abs(s[1] - (0.1 + 0.5 * tau)) < 1e-15
    assert tau < dt and abs(s[0] - (0.3 + 1.0 * dt)) > 1e-4  # the sampled reset would have gone the whole dt

    c, o = make(flags=O.F_WALLS | O.F_EVENT_TIME, substeps=1, dt=dt, coll_sigma_v=0.0, coll_sigma_w=0.0)
    st = base_state(x=(4.995, 1.0, 5.0), uf=0.0, fprev=0.0)
    st[0, 3:6] = (2.0, 0.4, 0.3)
    o.set_state(st, nominal(c)[None], np.zeros((1, 3)), np.zeros(1, np.int32), 0)
    o.step(np.zeros((1, 4)))
    s = o.get_state()["state"][0]
    ev, _, _ = o.get_events()
    assert ev[0] & O.EV_HIT_WALL
    v1 = np.array([2.0, 0.4, 0.3 - c.gravity * dt])
    tau = (5.0 - 4.995) / v1[0]
    ac = c.alpha_c
    assert s[0] == 5.0 and s[3] == 0.0
    assert abs(s[1] - (1.0 + v1[1] * tau + ac * v1[1] * (dt - tau))) < 1e-15
    assert abs(s[2] - (5.0 + v1[2] * tau + ac * v1[2] * (dt - tau))) < 1e-15
    assert abs(s[4] - ac * v1[1]) < 1e-15 and abs(s[5] - ac * v1[2]) < 1e-15


def test_event_time_pair_contact_time_closed_form():
    """Event-time pair contact: two drones on a line, approaching head-on
    with closing speed u, overlapping by delta at the end of the step: the
    contact happened sigma = delta / u before the end (within the step), and
    with alpha_c = 1 and no perturbation each drone flies its exchanged
    velocity for sigma, so the positions move by (v_i' - v_i) sigma."""
    dt = 0.005
    c, o = make(n_envs=1, sizes=[2], flags=O.F_COLLISIONS | O.F_EVENT_TIME, substeps=1, dt=dt, alpha_c=1.0,
                coll_sigma_v=0.0, coll_sigma_w=0.0)
    arm = c.arm
    st = base_state(n=2, x=(0.0, 0.0, 5.0), uf=0.0, fprev=0.0)
    u = 3.0
    delta = 0.004
    # positions at the end of the substep are x0 + v1 dt (free flight, x and y unaffected by gravity)
    gap = 2.0 * arm - delta
    st[0, 0], st[1, 0] = -gap / 2 - 1.5 * dt, gap / 2 + 1.5 * dt
    st[0, 3], st[1, 3] = 1.5, -1.5
    o.set_state(st, np.tile(nominal(c), (1, 1)), np.zeros((1, 3)), np.zeros(1, np.int32), 0)
    o.step(np.zeros((2, 4)))
    s = o.get_state()["state"]
    sigma = delta / u
    # exchanged velocities: -1.5 and +1.5; displacement (v' - v) sigma = -3 sigma and +3 sigma
    assert abs(s[0, 3] + 1.5) < 1e-12 and abs(s[1, 3] - 1.5) < 1e-12
    assert abs(s[0, 0] - (-gap / 2 - 3.0 * sigma)) < 1e-12
    assert abs(s[1, 0] - (gap / 2 + 3.0 * sigma)) < 1e-12


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


@pytest.mark.parametrize("term", ["pos", "vel", "ori", "spin", "act", "dact", "rot", "yaw"])
def test_reward_terms_one_at_a_time(term):
    """Sec. III-E, one weight at a time on a generic state: each state term is
    its weight times the quantity the paper names (unsquared norms; the
    command terms on f^ and f^ - f^_prev), evaluated on the state after the
    step and checked against numpy's norms of that state."""
    weights = {n: 0.0 for n in O.W_NAMES}
    weights[term] = -1.7
    c, o = make(flags=0, weights=weights)
    st = base_state(x=(1.0, -2.0, 4.0))
    st[0, 3:6] = (0.3, -0.8, 0.5)
    st[0, 6:15] = (rz(0.4) @ rx(0.3)).ravel()
    st[0, 15:18] = (1.5, -2.0, 3.0)
    f_prev = np.array([0.4, 0.9, 0.5, 0.7])
    st[0, 26:30] = f_prev
    goal = np.array([[0.5, 0.5, 3.0]])
    o.set_state(st, nominal(c)[None], goal, np.zeros(1, np.int32), 0)
    f_hat = np.array([0.1, 0.5, 0.5, 0.7])
    _, r, _ = o.step(f_hat[None])
    s = o.get_state()["state"][0]
    x, v, R, w = s[0:3], s[3:6], s[6:15].reshape(3, 3), s[15:18]
    q = {"pos": np.linalg.norm(x - goal[0]), "vel": np.linalg.norm(v), "ori": R[2, 2], "spin": np.linalg.norm(w),
         "act": np.linalg.norm(f_hat), "dact": np.linalg.norm(f_hat - f_prev), "rot": 0.5 * (np.trace(R) - 1.0),
         "yaw": R[0, 0]}[term]
    assert np.abs(s[6:15]).min() > 1e-3 or term not in ("ori", "rot", "yaw")
    assert abs(r[0] - (-1.7) * q) < 1e-12 * max(1.0, abs(q)), (term, r[0], q)


def test_reward_proximity_term():
    """Sec. III-E proximity term: each neighbour within alpha_prox = 4 l adds
    max(1 - d / alpha_prox, 0) (linear in the distance d). Two identical drones
    0.1 m apart at hover keep their separation over the step, so each one's
    reward is w_near (1 - 0.1 / alpha_prox); at 0.3 m (beyond alpha_prox) it is 0."""
    weights = {n: 0.0 for n in O.W_NAMES}
    weights["near"] = -2.0
    for sep in (0.1, 0.3):
        c, o = make(n_envs=1, sizes=[2], K=1, flags=0, weights=weights)
        st = base_state(n=2)
        st[1, 0] = sep
        o.set_state(st, nominal(c)[None], np.array([[0.0, 0.0, 5.0]]), np.zeros(1, np.int32), 0)
        _, r, _ = o.step(np.full((2, 4), 0.5))
        s = o.get_state()["state"]
        assert abs((s[1, 0] - s[0, 0]) - sep) < 1e-12
        alpha_prox = 4.0 * c.arm
        expect = -2.0 * max(1.0 - sep / alpha_prox, 0.0)
        assert np.abs(r - expect).max() < 1e-12, (sep, r, expect)
    assert 0.1 < 4.0 * c.arm < 0.3


def test_symmetric_action_map():
    """Sec. III-A as printed: f^ = (clip(a, -1, 1) + 1) / 2. Commands (-1, 0, 1, 3)
    give f^ = (0, 1/2, 1, 1), |f^| = 3/2 (read through the command-norm reward
    term alone); commands 0 give the hover command 1/2 (t2w = 2), so a hovering
    drone stays exactly where it is."""
    weights = {n: 0.0 for n in O.W_NAMES}
    weights["act"] = 1.0
    c, o = make(flags=O.F_ACTION_SYMMETRIC, weights=weights)
    o.set_state(base_state(), nominal(c)[None], np.zeros((1, 3)), np.zeros(1, np.int32), 0)
    _, r, _ = o.step(np.array([[-1.0, 0.0, 1.0, 3.0]]))
    assert abs(r[0] - 1.5) < 1e-15
    c, o = make(flags=O.F_ACTION_SYMMETRIC)
    st = base_state()
    o.set_state(st, nominal(c)[None], np.zeros((1, 3)), np.zeros(1, np.int32), 0)
    for _ in range(10):
        o.step(np.zeros((1, 4)))
    s = o.get_state()["state"][0]
    assert np.abs(s[0:6] - st[0, 0:6]).max() < 1e-12 and np.abs(s[15:18]).max() < 1e-12


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


def _sp(u, beta):
    """softplus_beta(u) = log(1 + exp(beta u)) / beta"""
    return np.logaddexp(0.0, beta * u) / beta


@pytest.mark.parametrize("face", ["ceiling", "+x", "-x", "+y", "-y"])
def test_smooth_boundaries_push_inward(face):
    """Smooth contacts (the differentiable form): a boundary pushes with
    k_c sp_beta(u) / m = smooth_kc g sp_beta(u) along its inward normal, u the
    penetration, in every substep. A hovering drone 2 mm past the face: after
    the control step its outward velocity is -dt k (sp(u0) + sp(u1)) with u1
    the penetration after the first (semi-implicit) substep; the other
    components stay 0."""
    c, o = make(flags=O.F_SMOOTH)
    H, hx, hy = c.room_h, c.room_hx, c.room_hy
    axis, sign, lim = {"ceiling": (2, 1, H), "+x": (0, 1, hx), "-x": (0, -1, hx), "+y": (1, 1, hy),
                       "-y": (1, -1, hy)}[face]
    x0 = np.array([0.0, 0.0, 5.0])
    x0[axis] = sign * (lim + 0.002)
    o.set_state(base_state(x=tuple(x0)), nominal(c)[None], np.zeros((1, 3)), np.zeros(1, np.int32), 0)
    o.step(np.full((1, 4), 0.5))
    s = o.get_state()["state"][0]
    k, dt, beta = c.smooth_kc * c.gravity, c.dt, c.smooth_beta
    u0 = 0.002
    v1 = -dt * k * _sp(u0, beta)                 # outward component after substep 1
    u1 = u0 + v1 * dt
    v2 = v1 - dt * k * _sp(u1, beta)
    v = s[3:6]
    assert abs(sign * v[axis] - v2) < 1e-12 * max(1.0, abs(v2)), (v, v2)
    assert np.abs(np.delete(v, axis)).max() < 1e-12
    assert v2 < -0.005  # pushed inward


def test_smooth_pair_repels_along_the_line_of_centres():
    """Smooth pair term: k_c sp_beta(2 l - d) / m along n_ij = (x_i - x_j) / d,
    evaluated in every substep on the positions at its start: two hovering
    drones 1.5 l apart along a skew direction move apart along it, each by
    dt k (sp(2 l - d0) + sp(2 l - d1)) with d1 = d0 + 2 v1 dt after the first
    (semi-implicit) substep."""
    c, o = make(n_envs=1, sizes=[2], flags=O.F_SMOOTH)
    n = np.array([0.6, -0.48, 0.64])
    n /= np.linalg.norm(n)
    d = 1.5 * c.arm
    st = base_state(2)
    st[1, 0:3] = st[0, 0:3] + d * n
    o.set_state(st, nominal(c)[None], np.zeros((1, 3)), np.zeros(1, np.int32), 0)
    o.step(np.full((2, 4), 0.5))
    v = o.get_state()["state"][:, 3:6]
    k, dt = c.smooth_kc * c.gravity, c.dt
    v1 = dt * k * _sp(2 * c.arm - d, c.smooth_beta)
    d1 = d + 2 * v1 * dt
    gain = v1 + dt * k * _sp(2 * c.arm - d1, c.smooth_beta)
    assert np.abs(v[0] - (-gain * n)).max() < 1e-12 and np.abs(v[1] - gain * n).max() < 1e-12
    assert gain > 0.01


def test_diff_loss_definition():
    """The differentiable rollout's loss: per drone and step ||x - g||^2 on the
    position after the step plus 1e-3 ||f^||^2, summed over the steps."""
    c, o = make(n_envs=1, sizes=[3], flags=O.F_SMOOTH)
    st = base_state(3)
    st[:, 0:3] = [[0.0, 0.0, 5.0], [1.0, -1.0, 4.0], [-2.0, 0.5, 6.0]]
    goal = np.array([[0.5, 0.25, 5.5]])
    o.set_state(st, nominal(c)[None], goal, np.zeros(1, np.int32), 0)
    acts = [np.array([[0.2, 0.4, 0.6, 0.8]] * 3), np.array([[0.9, 0.1, 0.3, 0.7]] * 3)]
    total = np.zeros(3)
    expect = np.zeros(3)
    for a in acts:
        _, _, _, l = o.step(a, want_loss=True)
        total += l
        x = o.get_state()["state"][:, 0:3]
        expect += ((x - goal[0]) ** 2).sum(1) + 1e-3 * (a ** 2).sum(1)
    assert np.abs(total - expect).max() < 1e-12


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


# --------------------------------------------------------------------------- scenarios (Sec. III-D)
FORM_SIZES = [1, 2, 3, 5, 8, 17, 64, 100, 128]


def _offsets(form, n, s=0.5, rmax=4.0):
    return np.array([O.formation_offset(form, k, n, s, rmax) for k in range(n)])


def _min_dist(p):
    d = np.linalg.norm(p[:, None] - p[None], axis=2) + np.eye(len(p)) * 1e9
    return d.min()


def test_formation_circle_and_cylinder():
    s = 0.5
    for n in FORM_SIZES:
        p = _offsets("circle", n, s)
        r = np.hypot(p[:, 0], p[:, 1])
        want_r = min(s * n / (2 * math.pi), 4.0)
        assert np.allclose(r, want_r, rtol=1e-12) and np.abs(p[:, 2]).max() == 0.0
        if n >= 2:  # evenly spaced: neighbouring goals a chord 2 r sin(pi/n) apart, arc s when uncapped
            ang = np.sort(np.mod(np.arctan2(p[:, 1], p[:, 0]), 2 * math.pi))
            gaps = np.diff(np.concatenate([ang, [ang[0] + 2 * math.pi]]))
            assert np.allclose(gaps, 2 * math.pi / n, atol=1e-12)
            if want_r < 4.0:
                assert abs(want_r * 2 * math.pi / n - s) < 1e-12
        p = _offsets("cylinder", n, s)
        L = next(L for L in range(1, 20) if 4 * L * L >= n)
        m = -(-n // L)
        r = np.hypot(p[:, 0], p[:, 1])
        assert np.allclose(r, min(s * m / (2 * math.pi), 4.0), rtol=1e-12)
        levels = np.unique(np.round(p[:, 2] / s, 9))
        assert np.allclose(np.diff(levels), 1.0) and abs(levels.mean()) < 1e-9  # rings s apart, centred
        assert max(np.sum(np.isclose(p[:, 2], z * s)) for z in levels) <= m
        if n >= 2:
            assert _min_dist(p) > 1e-6  # distinct goals


def test_formation_grid_and_cube():
    s = 0.5
    for n in FORM_SIZES:
        for form, dim in (("grid", 2), ("cube", 3)):
            p = _offsets(form, n, s)
            q = p / s
            m = next(m for m in range(1, 20) if m ** dim >= n)
            # every coordinate on the half-spacing lattice, goals distinct, nearest neighbours s apart
            assert np.allclose(2 * q, np.round(2 * q), atol=1e-12)
            if dim == 2:
                assert np.abs(p[:, 2]).max() == 0.0
            if n >= 2:
                assert abs(_min_dist(p) - s) < 1e-12
            assert len({tuple(np.round(r, 9)) for r in q}) == n
            ext = q.max(axis=0) - q.min(axis=0)
            assert ext[:dim].max() <= m - 1 + 1e-12
            if n == m ** dim:  # a full grid is centred
                assert np.abs(p.mean(axis=0)).max() < 1e-12


def test_formation_sphere_fibonacci():
    s = 0.5
    golden = (3 - math.sqrt(5)) / 2  # turns
    for n in FORM_SIZES:
        p = _offsets("sphere", n, s)
        r = s * math.sqrt(n / (4 * math.pi))
        assert np.allclose(np.linalg.norm(p, axis=1), r, rtol=1e-12)
        assert abs(4 * math.pi * r * r / n - s * s) < 1e-12       # area s^2 per goal
        z = p[:, 2] / r
        assert np.allclose(np.diff(z), -2.0 / n, atol=1e-12) and abs(z.mean()) < 1e-12
        if n >= 2:
            az = np.arctan2(p[:, 1], p[:, 0]) / (2 * math.pi)
            step = np.mod(np.diff(az) - golden + 0.5, 1.0) - 0.5   # azimuth advances by the golden angle
            ok = np.abs(z[:-1]) < 1 - 1e-9
            assert np.abs(step[ok[:len(step)]]).max() < 1e-8
            assert _min_dist(p) > 0.3 * s
    p = _offsets("sphere", 128, s)
    assert np.linalg.norm(p.mean(axis=0)) < 0.02 * s * math.sqrt(128 / (4 * math.pi))


def _scn_oracle(sizes, mask, seed=7, episode_steps=1500, **kw):
    c, o = make(n_envs=len(sizes), sizes=sizes, scenarios=mask, episode_steps=episode_steps, **kw)
    o.reset(seed)
    return c, o


def test_scenario_draw_distribution():
    E = 24000
    c, o = _scn_oracle([1] * E, 0xFF)
    rec = o.get_scenario()
    t = rec[:, O.R_TYPE].astype(int)
    cnt = np.bincount(t, minlength=8)
    assert (np.abs(cnt - E / 8) < 5 * math.sqrt(E / 8)).all()
    for col in (O.R_F0, O.R_F1):
        cf = np.bincount(rec[:, col].astype(int), minlength=5)
        assert len(cf) == 5 and (np.abs(cf - E / 5) < 5 * math.sqrt(E / 5)).all()
    tsw = rec[:, O.R_TSW]
    assert tsw.min() >= 375 and tsw.max() <= 1125 and np.all(tsw == np.round(tsw))
    assert abs(tsw.mean() - 750) < 5 * 217 / math.sqrt(E)
    form = t != O.SCN_NAMES.index("pursuit_lissajous")
    for q in (O.R_C0, O.R_C1):
        cc = rec[form & (t != 0), q:q + 3]
        assert cc[:, 0].min() >= -3.5 and cc[:, 0].max() <= 3.5 and cc[:, 2].min() >= 1.5 and cc[:, 2].max() <= 8.5
        assert abs(cc[:, 0].mean()) < 0.05 and abs(cc[:, 2].mean() - 5.0) < 0.05
    li = t == O.SCN_NAMES.index("pursuit_lissajous")
    A = rec[li, O.R_C1:O.R_C1 + 3]
    assert (A >= 0.5 * np.array([3.5, 3.5, 3.5]) - 1e-12).all() and (A <= 3.5 + 1e-12).all()
    f = rec[li, O.R_FREQ:O.R_FREQ + 3]
    assert f.min() >= 0.05 and f.max() <= 0.15
    seeds = rec[:, O.R_SEED_LO] + 65536 * rec[:, O.R_SEED_HI]
    assert len(np.unique(seeds[t != 0])) > 0.99 * (t != 0).sum()
    # a subset of scenarios draws only from that subset; the single goal alone draws no record
    _, o2 = _scn_oracle([1] * 2000, O.scenario_mask(["static", "swap"]))
    assert set(np.unique(o2.get_scenario()[:, O.R_TYPE]).astype(int)) == {1, 3}
    _, o3 = _scn_oracle([1] * 10, O.scenario_mask(["single"]))
    assert np.abs(o3.get_scenario()).max() == 0.0


def _with_record(sizes, rec, ep):
    """Oracle whose envs all carry scenario record `rec`, at control step ep."""
    E = len(sizes)
    c, o = _scn_oracle(sizes, 0xFF)
    o.set_scenario(np.tile(rec, (E, 1)))
    s = o.get_state()
    o.set_state(ep_step=np.full(E, ep, np.int32))
    return c, o


def _record(kind, f0=0, f1=1, tsw=10, seed=12345, c0=(0.5, -1.0, 4.0), c1=(-2.0, 1.5, 6.0), freq=(0.1, 0.13, 0.07),
            phase=(0.1, 0.6, 0.3)):
    r = np.zeros(O.NSCN)
    r[O.R_TYPE] = O.SCN_NAMES.index(kind)
    r[O.R_F0], r[O.R_F1], r[O.R_TSW] = f0, f1, tsw
    r[O.R_SEED_LO], r[O.R_SEED_HI] = seed & 0xFFFF, seed >> 16
    r[O.R_C0:O.R_C0 + 3] = c0
    r[O.R_C1:O.R_C1 + 3] = c1
    r[O.R_FREQ:O.R_FREQ + 3] = freq
    r[O.R_PHASE:O.R_PHASE + 3] = phase
    return r


def _goals_at(c, o, ep):
    o.set_state(ep_step=np.full(o.E, ep, np.int32))
    return o.goals()


def test_scenario_static_dynamic_swarm_vs_swarm():
    n = 9
    c, o = _with_record([n], _record("static", f0=2), 0)
    want = np.array([0.5, -1.0, 4.0]) + _offsets("sphere", n)
    for ep in (0, 9, 10, 700):
        assert np.allclose(_goals_at(c, o, ep), want, atol=1e-12)
    c, o = _with_record([n], _record("dynamic", f0=0, f1=4, tsw=10), 0)
    assert np.allclose(_goals_at(c, o, 9), np.array([0.5, -1.0, 4.0]) + _offsets("circle", n), atol=1e-12)
    assert np.allclose(_goals_at(c, o, 10), np.array([-2.0, 1.5, 6.0]) + _offsets("cube", n), atol=1e-12)
    # swarm vs swarm: 5 + 4 drones; each group a formation of its own size; centres swap at the switch
    c, o = _with_record([n], _record("swarm_vs_swarm", f0=1, f1=3, tsw=10), 0)
    g = _goals_at(c, o, 9)
    assert np.allclose(g[:5], np.array([0.5, -1.0, 4.0]) + _offsets("grid", 5), atol=1e-12)
    assert np.allclose(g[5:], np.array([-2.0, 1.5, 6.0]) + _offsets("grid", 4), atol=1e-12)
    g = _goals_at(c, o, 10)
    assert np.allclose(g[:5], np.array([-2.0, 1.5, 6.0]) + _offsets("cylinder", 5), atol=1e-12)
    assert np.allclose(g[5:], np.array([0.5, -1.0, 4.0]) + _offsets("cylinder", 4), atol=1e-12)


def test_scenario_swap_is_a_permutation():
    for n in (2, 3, 8, 17, 64):
        perms = []
        for seed in (1, 2, 3):
            c, o = _with_record([n], _record("swap", f0=1, tsw=10, seed=seed), 0)
            before = _goals_at(c, o, 9)
            after = _goals_at(c, o, 10)
            assert np.allclose(before, np.array([0.5, -1.0, 4.0]) + _offsets("grid", n), atol=1e-12)
            # the same set of goals, reassigned one to one
            idx = [int(np.argmin(np.linalg.norm(before - a, axis=1))) for a in after]
            assert sorted(idx) == list(range(n))
            assert np.allclose(after, before[idx], atol=1e-12)
            assert np.allclose(_goals_at(c, o, 500), after, atol=0)  # fixed for the rest of the episode
            perms.append(tuple(idx))
        if n >= 8:
            assert len(set(perms)) == 3 and all(p != tuple(range(n)) for p in perms)


def test_scenario_shrink_expand():
    n, P = 8, 400
    c, o = _with_record([n], _record("shrink_expand", f0=4), 0)
    base = _offsets("cube", n)
    c0 = np.array([0.5, -1.0, 4.0])
    for ep, lam in ((0, 1.0), (P // 4, 0.75), (P // 2, 0.5), (P, 1.0), (3 * P // 2, 0.5)):
        assert np.allclose(_goals_at(c, o, ep) - c0, lam * base, atol=1e-12), ep


def test_scenario_lissajous_is_sinusoidal():
    """Each axis of the evader follows c + A sin(w tau + phi): it satisfies the
    three-term recurrence y(t+1) + y(t-1) = 2 cos(w) y(t) of a pure sinusoid
    with w = 2 pi f T, stays within c +- A, and starts at c + A sin(2 pi phase)."""
    c, o = _with_record([3], _record("pursuit_lissajous", c1=(2.0, 3.0, 1.5)), 0)
    T = c.substeps * c.dt
    cen, A = np.array([0.5, -1.0, 4.0]), np.array([2.0, 3.0, 1.5])
    f, ph = np.array([0.1, 0.13, 0.07]), np.array([0.1, 0.6, 0.3])
    ys = np.array([_goals_at(c, o, t)[0] - cen for t in range(0, 1500, 7)])
    g3 = _goals_at(c, o, 0)
    assert np.allclose(g3, g3[0], atol=0)  # all drones chase the one evader
    assert np.allclose(g3[0], cen + A * np.sin(2 * math.pi * ph), atol=1e-12)
    for t in (1, 50, 777, 1400):
        y0, y1, y2 = (_goals_at(c, o, t + k)[0] - cen for k in (-1, 0, 1))
        assert np.allclose(y0 + y2, 2 * np.cos(2 * math.pi * f * T) * y1, atol=1e-12)
    assert (np.abs(ys) <= A + 1e-12).all() and (np.abs(ys).max(axis=0) > 0.9 * A).all()


def test_scenario_bezier_through_waypoints_c1():
    """The evader passes the waypoints at segment boundaries and its path is C1
    there, with Catmull-Rom tangents: the step after a knot W_q is about
    (W_{q+1} - W_{q-1}) / (2S), the same on either side."""
    S = 300
    c, o = _with_record([2], _record("pursuit_bezier"), 0)
    knots = np.array([_goals_at(c, o, q * S)[0] for q in range(5)])
    assert (np.abs(knots[:, :2]) <= 3.5).all() and (knots[:, 2] >= 1.5).all() and (knots[:, 2] <= 8.5).all()
    for q in (1, 2, 3):
        left = knots[q] - _goals_at(c, o, q * S - 1)[0]
        right = _goals_at(c, o, q * S + 1)[0] - knots[q]
        tangent = (knots[q + 1] - knots[q - 1]) / (2 * S)
        assert np.allclose(left, tangent, atol=20.0 / S ** 2) and np.allclose(right, tangent, atol=20.0 / S ** 2)
    mid = _goals_at(c, o, S // 2)[0]
    assert np.linalg.norm(mid - knots[0]) > 1e-3 and np.linalg.norm(mid - knots[1]) > 1e-3


def test_scenario_goal_used_by_the_step():
    """The observation and the position reward of a step use the goal at the
    step's end (tau = steps done), which is what or_goals reports after it."""
    sizes = [8, 5]
    c, o = _scn_oracle(sizes, O.scenario_mask(["dynamic"]), w=[0.0] * 13 + [0.0])
    rec = np.array([_record("dynamic", f0=0, f1=1, tsw=4)] * 2)
    o.set_scenario(rec)
    o.set_state(ep_step=np.full(2, 3, np.int32))
    st = o.get_state()["state"]
    obs, rew, _ = o.step(np.full((13, 4), 0.5))
    g = o.goals()                      # tau = 4: after the switch
    x = o.get_state()["state"][:, 0:3]
    assert np.allclose(obs[:, 0:3], x - g, atol=1e-12)
    assert np.allclose(g, np.concatenate([np.array([-2.0, 1.5, 6.0]) + _offsets("grid", n) for n in sizes]))
    assert np.abs(rew).max() == 0.0
    _, o2 = _scn_oracle(sizes, O.scenario_mask(["dynamic"]), w=[-1.0] + [0.0] * 13)
    o2.set_scenario(rec)
    o2.set_state(state=st, ep_step=np.full(2, 3, np.int32))
    _, rew2, _ = o2.step(np.full((13, 4), 0.5))
    assert np.allclose(rew2, -np.linalg.norm(x - g, axis=1), atol=1e-12)
