"""Closed forms checked on the CUDA path directly (the oracle is pinned to the
same ones in test_oracle_pins.py): hover equilibrium and the discrete free
fall of semi-implicit Euler, through the per-call step and the rollout."""
import numpy as np
import pytest
import torch

from gpu_helpers import DEV, nominal
from paper_2306_09537_gb300.env import QuadSwarmEnv

pytestmark = pytest.mark.gpu

E = 256


def _env(z0):
    """Drones at rest, upright, nominal parameters (t2w = 2: hover command 1/2),
    motors at hover speed sqrt(1/2), no noise, floor or walls."""
    env = QuadSwarmEnv(E, 1, 0, (), seed=1, device=DEV)
    st = np.zeros((E, 30), np.float32)
    st[:, 0] = np.linspace(-3, 3, E)
    st[:, 1] = np.linspace(2, -2, E)
    st[:, 2] = z0
    st[:, 6:15] = np.eye(3, dtype=np.float32).ravel()
    prm = np.tile(np.array(nominal(env), np.float32), (E, 1))
    assert prm[0, 4] == 2.0  # t2w
    return env, st, prm


def _set(env, st, prm):
    env.set_state(torch.from_numpy(st).to(DEV), torch.from_numpy(prm).to(DEV), torch.zeros(E, 3, device=DEV),
                  torch.zeros(E, dtype=torch.int32, device=DEV), torch.zeros(E, dtype=torch.int32, device=DEV))


@pytest.mark.parametrize("form", ["step", "rollout"])
def test_hover_equilibrium(form):
    """Thrust m g on every rotor set: no torque, so the rotation stays exactly
    the identity and the body rates exactly zero; the position drifts only by
    the binary32 rounding of the thrust balance (|T / m - g| ~ 1e-6 m/s^2,
    under 1e-5 m over 10 s)."""
    env, st, prm = _env(5.0)
    st[:, 18:22] = np.sqrt(np.float32(0.5))  # u_f at hover
    st[:, 26:30] = 0.5                       # previous command
    _set(env, st, prm)
    T = 1000
    acts = torch.full((T, env.D, 4), 0.5, device=DEV)
    if form == "step":
        for t in range(T):
            env.step(acts[t])
    else:
        env.rollout(acts, torch.empty(T, env.D, env.obs_dim, device=DEV), None, None)
    s = env.get_state()["state"].cpu().numpy()
    assert np.array_equal(s[:, 6:15], st[:, 6:15])       # R = I
    assert np.all(s[:, 15:18] == 0)                      # body rates
    assert np.abs(s[:, 0:3] - st[:, 0:3]).max() <= 1e-5  # position
    assert np.abs(s[:, 3:6]).max() <= 1e-5               # velocity


@pytest.mark.parametrize("form", ["step", "rollout"])
def test_free_fall_semi_implicit_euler(form):
    """Motors off: a = g exactly each substep, so after n substeps of dt
    v_n = -g n dt and z_n = z_0 - g dt^2 n (n + 1) / 2 (semi-implicit Euler;
    explicit Euler would give n (n - 1) / 2, 2.5 cm apart after 1 s), within
    binary32 accumulation; x and y stay exactly put."""
    env, st, prm = _env(9.0)
    _set(env, st, prm)
    T = 100
    acts = torch.zeros(T, env.D, 4, device=DEV)
    if form == "step":
        for t in range(T):
            env.step(acts[t])
    else:
        env.rollout(acts, torch.empty(T, env.D, env.obs_dim, device=DEV), None, None)
    s = env.get_state()["state"].cpu().numpy()
    dt, g, n = float(env.cfg.dt), float(env.cfg.params.gravity), T * int(env.cfg.substeps)
    z = 9.0 - g * dt * dt * n * (n + 1) / 2
    assert np.abs(s[:, 2] - z).max() <= 2e-4
    assert np.abs(s[:, 5] - (-g * n * dt)).max() <= 2e-5
    assert np.array_equal(s[:, 0:2], st[:, 0:2]) and np.all(s[:, 3:5] == 0)
    assert abs(z - (9.0 - g * dt * dt * n * (n - 1) / 2)) > 0.02  # the two integrators are told apart


def test_head_on_collision_swaps_normal_velocities():
    """Two equal drones closing head-on along x, alpha_c = 1 and no
    perturbation: after the step's collision pass their x velocities are
    swapped (so momentum and kinetic energy are conserved), both are flagged,
    and the tangential components are untouched."""
    env = QuadSwarmEnv(1, 2, 1, ("collisions",), seed=1, device=DEV, alpha_c=1.0, coll_sigma_v=0.0, coll_sigma_w=0.0)
    st = np.zeros((2, 30), np.float32)
    st[:, 2] = 5.0
    st[0, 0], st[1, 0] = -0.03, 0.03          # 6 cm apart: inside 2 x arm (9.2 cm)
    st[0, 3], st[1, 3] = 1.0, -0.5            # closing at 1.5 m/s
    st[:, 4] = 0.25                           # a common tangential velocity
    st[:, 6:15] = np.eye(3, dtype=np.float32).ravel()
    st[:, 18:22] = np.sqrt(np.float32(0.5))
    st[:, 26:30] = 0.5
    prm = np.tile(np.array(nominal(env), np.float32), (1, 1))
    env.set_state(torch.from_numpy(st).to(DEV), torch.from_numpy(prm).to(DEV), torch.zeros(1, 3, device=DEV),
                  torch.zeros(1, dtype=torch.int32, device=DEV), torch.zeros(1, dtype=torch.int32, device=DEV))
    env.step(torch.full((2, 4), 0.5, device=DEV))
    s = env.get_state()["state"].cpu().numpy()
    ev, _ = env.get_events()
    assert abs(s[0, 3] - (-0.5)) <= 1e-5 and abs(s[1, 3] - 1.0) <= 1e-5
    assert abs((s[0, 3] + s[1, 3]) - 0.5) <= 1e-5                              # momentum
    assert abs((s[0, 3] ** 2 + s[1, 3] ** 2) - (1.0 + 0.25)) <= 2e-5            # kinetic energy along x
    assert np.allclose(s[:, 4], 0.25, atol=1e-6) and np.abs(s[:, 5]).max() <= 1e-5
    assert np.all((ev.cpu().numpy() & 16) != 0)                                 # hit_quad on both


def test_motor_lag_step_response():
    """From rest, command 1 on every rotor: the normalised rotor speed after n
    substeps is 1 - (1 - alpha)^n with alpha = 1 - exp(-dt / tau_m), reaching
    98% after ceil(ln 50 / -ln(1 - alpha)) substeps (2% settling, tau_m ln 50)."""
    env, st, prm = _env(5.0)
    _set(env, st, prm)
    dt, tau = float(env.cfg.dt), float(prm[0, 5])
    alpha = 1.0 - np.exp(-dt / tau)
    n98 = int(np.ceil(np.log(50.0) / -np.log(1.0 - alpha)))
    S = int(env.cfg.substeps)
    for t in range(1, (n98 + S - 1) // S + 2):
        env.step(torch.ones(env.D, 4, device=DEV))
        uf = env.get_state()["state"][:, 18:22].cpu().numpy()
        n = t * S
        assert np.abs(uf - (1.0 - (1.0 - alpha) ** n)).max() <= 2e-6, t
        assert (uf.min() >= 0.98) == (n >= n98), t


def test_torque_free_spin_about_a_principal_axis():
    """Motors off and a body rate about the z axis: w x (I w) vanishes, so the
    body rate stays exactly constant, and the rotation advances by
    atan(dt w_z) per substep about z (the polar factor of I + dt [w]x)."""
    env, st, prm = _env(9.0)
    wz = 3.0
    st[:, 17] = wz
    _set(env, st, prm)
    T = 50
    for t in range(T):
        env.step(torch.zeros(env.D, 4, device=DEV))
    s = env.get_state()["state"].cpu().numpy()
    dt, n = float(env.cfg.dt), T * int(env.cfg.substeps)
    psi = n * np.arctan(dt * wz)
    Rz = np.array([[np.cos(psi), -np.sin(psi), 0.0], [np.sin(psi), np.cos(psi), 0.0], [0.0, 0.0, 1.0]])
    assert np.all(s[:, 15] == 0) and np.all(s[:, 16] == 0) and np.all(s[:, 17] == np.float32(wz))
    assert np.abs(s[:, 6:15] - Rz.ravel()).max() <= 2e-5


def test_wall_removes_the_normal_velocity():
    """A drone past the x wall and moving outward (alpha_c = 1, no
    perturbation): put back on the wall, its normal velocity removed, the
    tangential one kept; flagged hit_wall."""
    env = QuadSwarmEnv(E, 1, 0, ("walls",), seed=1, device=DEV, alpha_c=1.0, coll_sigma_v=0.0, coll_sigma_w=0.0)
    _, st, prm = _env(5.0)
    hx = float(env.cfg.params.room_hx)
    st[:, 0] = hx - 0.001
    st[:, 3] = 2.0                 # outward: crosses the wall within the step
    st[:, 4] = np.linspace(-1, 1, E)
    st[:, 18:22] = np.sqrt(np.float32(0.5))
    st[:, 26:30] = 0.5
    _set(env, st, prm)
    env.step(torch.full((E, 4), 0.5, device=DEV))
    s = env.get_state()["state"].cpu().numpy()
    ev, _ = env.get_events()
    assert np.all(s[:, 0] == np.float32(hx)) and np.all(s[:, 3] == 0)
    assert np.abs(s[:, 4] - st[:, 4]).max() <= 1e-6
    assert np.all((ev.cpu().numpy() & 4) != 0)  # hit_wall


def test_floor_hit_rests_upright_keeping_the_heading():
    """A tilted, rolling drone falling through the floor: height, velocity and
    body rates zero, the rotation upright about z with the heading of the body
    x axis kept; flagged hit_floor."""
    env = QuadSwarmEnv(E, 1, 0, ("floor",), seed=1, device=DEV)
    _, st, prm = _env(0.005)
    yaw = np.linspace(-3.0, 3.0, E)
    tilt = 0.3
    for i, psi in enumerate(yaw):
        Rz = np.array([[np.cos(psi), -np.sin(psi), 0], [np.sin(psi), np.cos(psi), 0], [0, 0, 1.0]])
        Rx = np.array([[1.0, 0, 0], [0, np.cos(tilt), -np.sin(tilt)], [0, np.sin(tilt), np.cos(tilt)]])
        st[i, 6:15] = (Rz @ Rx).ravel()
    st[:, 5] = -2.0
    st[:, 15:18] = (1.0, 0.0, 0.0)  # a roll rate: turns about the body x axis, whose heading is kept
    _set(env, st, prm)
    env.step(torch.zeros(E, 4, device=DEV))
    s = env.get_state()["state"].cpu().numpy()
    ev, _ = env.get_events()
    assert np.all(s[:, 2] == 0) and np.all(s[:, 3:6] == 0) and np.all(s[:, 15:18] == 0)
    R = s[:, 6:15].reshape(E, 3, 3)
    assert np.abs(R[:, 2, :] - [0, 0, 1]).max() == 0 and np.abs(R[:, :, 2] - [0, 0, 1]).max() == 0
    heading = np.arctan2(R[:, 1, 0], R[:, 0, 0])
    assert np.abs(np.angle(np.exp(1j * (heading - yaw)))).max() <= 1e-5
    assert np.all((ev.cpu().numpy() & 1) != 0)  # hit_floor


@pytest.mark.parametrize("form", ["step", "rollout"])
def test_reward_action_term_square_root_error(form):
    """With only the action weight set, the reward is the norm of the
    normalised command (Sec. III-E); with one non-zero rotor command f per
    drone that is sqrt(fl32(f^2)), which the step evaluates with the hardware
    square-root approximation (as it does the rotor-speed command sqrt(f) and
    the Box-Muller radius). Against the binary64 root of the same binary32
    input its relative error stays within two units in the last place
    (2^-22) over the command range, and the root of zero is zero."""
    n = 65536
    env = QuadSwarmEnv(n, 1, 0, (), seed=4, weights={"act": 1.0}, device=DEV)
    env.reset(4)
    rng = np.random.default_rng(4)
    f = rng.uniform(0.0, 1.0, n).astype(np.float32)
    f[:8] = [0.0, 1.0, 0.5, 0.25, 1e-6, 2.0 ** -20, 0.75, np.nextafter(np.float32(1), np.float32(0))]
    acts = np.zeros((n, 4), np.float32)
    acts[:, 0] = f
    a = torch.from_numpy(acts).to(DEV)
    if form == "step":
        env.step(a)
        r = env.reward.cpu().numpy().astype(np.float64)
    else:
        rew = torch.empty(1, n, device=DEV)
        env.rollout(a[None], None, rew, None)
        r = rew[0].cpu().numpy().astype(np.float64)
    x = (f * f).astype(np.float64)  # fl32(f^2), correctly rounded by numpy
    want = np.sqrt(x)
    assert r[0] == 0.0
    rel = np.abs(r[1:] - want[1:]) / want[1:]
    print(f"max relative error {rel.max():.3e} = 2^{np.log2(rel.max()):.2f}")
    assert rel.max() <= 2.0 ** -22


def test_normals_within_the_binary32_transform_bound():
    """The body-rate sensor noise is sigma_w times Box-Muller normals (R18).
    Drones hovering with zero body rates and equal rotor commands feel no
    torque and keep their body rates exactly zero through a step, so the
    observed body rates are the noise alone. Each of the 3 x 8192 normals is
    compared with the exact transform of the same two uniforms, formed here in
    binary64 from the oracle's Philox stream (first checked against the
    oracle's own step, which pins this test's reading of the stream layout),
    within the error of the binary32 transform: with y = -2 ln u0 the radius
    rho = sqrt(y) and dy = 2 x 2^-21.41 max(1, y / 2) the error of a
    logarithm that is good to 2^-21.41 absolute on [0.5, 2] and 3 units in the
    last place elsewhere, |n - n_exact| <= min(dy / (2 rho), sqrt(dy)) +
    1e-6 (rho + 1) (the sine and cosine to 2^-21.41 absolute, the square root
    and the products to a few units in the last place)."""
    from gpu_helpers import pair, set_both
    from oracle import oracle as O
    E, seed, tick = 8192, 11, 3
    env, o = pair(np.ones(E, np.int32), 0, ("obs_noise",), seed=seed)
    st = np.zeros((E, 30), np.float32)
    st[:, 0] = np.linspace(-3, 3, E)
    st[:, 1] = np.linspace(2, -2, E)
    st[:, 2] = 5.0
    st[:, 6:15] = np.eye(3, dtype=np.float32).ravel()
    st[:, 18:22] = np.sqrt(np.float32(0.5))
    st[:, 26:30] = 0.5
    prm = np.tile(np.array(nominal(env), np.float32), (E, 1))
    set_both(env, o, st, prm, np.zeros((E, 3), np.float32), tick=tick)
    env.step(torch.full((E, 4), 0.5, device=DEV))
    obs = env.obs.cpu().numpy().astype(np.float64)
    o_obs = o.step(np.full((E, 4), 0.5))[0]
    s = env.get_state()["state"].cpu().numpy()
    assert np.all(s[:, 15:18] == 0)  # the body rates stayed exactly zero
    n_gpu = obs[:, 15:18] / float(np.float32(env.cfg.params.obs_sigma_w))
    n_or = o_obs[:, 15:18] / float(o.cfg.obs_sigma_w)

    # the transform of the stream's uniforms: blocks 1 and 2 of the OBS tag
    # (4), substream 0, at counter (tick, drone); words z, w of block 1 feed
    # the first pair, words x, y of block 2 the third normal
    key = np.array([seed & 0xffffffff, seed >> 32], np.uint32)
    d = np.arange(E, dtype=np.uint32)

    def block(blk):
        ctr = np.stack([np.full(E, tick, np.uint32), d, np.full(E, (4 << 16) | blk, np.uint32),
                        np.zeros(E, np.uint32)], axis=1)
        return O.philox4x32_10_batch(ctr, key)

    def u(r):
        return ((r.astype(np.float64) // 512) + 0.5) / 8388608.0
    b1, b2 = block(1), block(2)
    y01, y2 = -2.0 * np.log(u(b1[:, 2])), -2.0 * np.log(u(b2[:, 0]))
    th01, th2 = 2.0 * np.pi * u(b1[:, 3]), 2.0 * np.pi * u(b2[:, 1])
    exact = np.stack([np.sqrt(y01) * np.cos(th01), np.sqrt(y01) * np.sin(th01), np.sqrt(y2) * np.cos(th2)], axis=1)
    y = np.stack([y01, y01, y2], axis=1)
    assert np.abs(n_or - exact).max() <= 1e-9  # the oracle draws exactly these normals
    rho = np.sqrt(y)
    dy = 2.0 * 2.0 ** -21.41 * np.maximum(1.0, y / 2.0)
    bound = np.minimum(dy / (2.0 * np.maximum(rho, 1e-30)), np.sqrt(dy)) + 1e-6 * (rho + 1.0)
    err = np.abs(n_gpu - exact)
    assert np.all(err <= bound), float((err / bound).max())
