"""ctypes binding of the FP64 CPU oracle (``qs_oracle.c``).

Test infrastructure: only the tests, ``__graft_entry__.smoke()`` and the CPU
baseline legs of ``bench.py`` load this module. It shares no code with the CUDA
library (paper Sec. III-A .. III-E; the readings it takes are stated in
``qs_oracle.c`` at the point of use).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

# configuration flags (same bit meaning as the oracle header)
F_DR, F_MOTOR_NOISE, F_OBS_NOISE, F_COLLISIONS = 1 << 0, 1 << 1, 1 << 2, 1 << 3
F_FLOOR, F_WALLS, F_AUTO_RESET, F_SMOOTH = 1 << 4, 1 << 5, 1 << 6, 1 << 7
F_ACTION_SYMMETRIC, F_RECORD_KNN, F_DOWNWASH = 1 << 8, 1 << 9, 1 << 10
F_ROUND32, F_ROUND32_SR = 1 << 11, 1 << 12  # conditioning instruments (see qs_oracle.h)
F_EVENT_TIME = 1 << 13  # contacts resolved at their crossing time (see qs_oracle.h)
EV_HIT_FLOOR, EV_ON_FLOOR, EV_HIT_WALL, EV_HIT_CEIL, EV_HIT_QUAD = 1, 2, 4, 8, 16
NST, NPRM = 30, 7
W_NAMES = ["pos", "vel", "ori", "spin", "act", "dact", "rot", "yaw", "hit_floor", "on_floor",
           "hit_wall", "hit_ceil", "hit_quad", "near"]
TAG_RESET_ENV, TAG_RESET_DRONE, TAG_MOTOR, TAG_OBS, TAG_COLL, TAG_WALL = 1, 2, 3, 4, 5, 6
TAG_SCN, TAG_AUTO_SCN, TAG_WAYPOINT, TAG_SWAP = 10, 11, 12, 13
# training scenarios (Sec. III-D) and goal formations
SCN_NAMES = ["single", "static", "dynamic", "swap", "shrink_expand", "swarm_vs_swarm", "pursuit_lissajous",
             "pursuit_bezier"]
FORM_NAMES = ["circle", "grid", "sphere", "cylinder", "cube"]
NSCN = 18
R_TYPE, R_F0, R_F1, R_TSW, R_SEED_LO, R_C0, R_C1, R_FREQ, R_PHASE, R_SEED_HI = 0, 1, 2, 3, 4, 5, 8, 11, 14, 17


def scenario_mask(names) -> int:
    """Bit mask of the named scenarios (SCN_NAMES)."""
    m = 0
    for n in names:
        m |= 1 << SCN_NAMES.index(n)
    return m


class OrConfig(C.Structure):
    _fields_ = [
        ("n_envs", C.c_int32), ("k_neighbors", C.c_int32), ("substeps", C.c_int32),
        ("episode_steps", C.c_int32), ("dt", C.c_double), ("seed", C.c_uint64),
        ("flags", C.c_uint32), ("scenarios", C.c_uint32),
        ("mass", C.c_double), ("arm", C.c_double), ("ixx", C.c_double), ("iyy", C.c_double),
        ("izz", C.c_double), ("t2w", C.c_double), ("kappa", C.c_double), ("tau_m", C.c_double),
        ("gravity", C.c_double), ("mu", C.c_double),
        ("alpha_nd", C.c_double), ("alpha_ns_frac", C.c_double), ("alpha_c", C.c_double),
        ("coll_sigma_v", C.c_double), ("coll_sigma_w", C.c_double),
        ("obs_sigma_x", C.c_double), ("obs_sigma_v", C.c_double), ("obs_sigma_w", C.c_double),
        ("room_hx", C.c_double), ("room_hy", C.c_double), ("room_h", C.c_double),
        ("dr_lo", C.c_double), ("dr_hi", C.c_double),
        ("smooth_beta", C.c_double), ("smooth_kc", C.c_double), ("prox_factor", C.c_double),
        ("omega_max", C.c_double),
        ("dw_k1", C.c_double), ("dw_k2", C.c_double), ("dw_b1", C.c_double), ("dw_height", C.c_double),
        ("dw_sigma_a", C.c_double), ("dw_sigma_w", C.c_double),
        ("form_spacing", C.c_double), ("form_rmax", C.c_double), ("scn_margin", C.c_double),
        ("se_min", C.c_double), ("se_period", C.c_double), ("liss_f", C.c_double), ("bez_seg", C.c_double),
        ("w", C.c_double * 14),
        ("round_salt", C.c_uint64),
    ]


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` with gcc (binary64, no FP contraction)."""
    src = os.path.join(_HERE, "qs_oracle.c")
    hdr = os.path.join(_HERE, "qs_oracle.h")
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(src), os.path.getmtime(hdr))):
        return _LIB_PATH
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-D_GNU_SOURCE", "-O2", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-Wall", "-pthread", "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True, cwd=_HERE)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    """The loaded oracle library. ``QS_ORACLE_LIB`` names another build of the
    same source to load instead: the mutation test points it at copies with a
    planted mistake, to check that the pins reject each one."""
    global _lib
    with _lock:
        if _lib is None:
            path = os.environ.get("QS_ORACLE_LIB") or build()
            L = C.CDLL(path)
            P = C.POINTER
            L.or_philox4x32_10.argtypes = [P(C.c_uint32), P(C.c_uint32), P(C.c_uint32)]
            L.or_philox4x32_10_n.argtypes = [P(C.c_uint32), P(C.c_uint32), P(C.c_uint32), C.c_size_t]
            L.or_uniform.argtypes = [C.c_uint32]
            L.or_uniform.restype = C.c_double
            L.or_polar.argtypes = [P(C.c_double), P(C.c_double)]
            L.or_pair_key.argtypes = [P(C.c_float), P(C.c_float)]
            L.or_pair_key.restype = C.c_float
            L.or_default_config.argtypes = [P(OrConfig)]
            L.or_create.argtypes = [P(OrConfig), P(C.c_int32)]
            L.or_create.restype = C.c_void_p
            L.or_destroy.argtypes = [C.c_void_p]
            L.or_n_drones.argtypes = [C.c_void_p]
            L.or_n_drones.restype = C.c_int
            L.or_reset.argtypes = [C.c_void_p, C.c_uint64, P(C.c_uint8)]
            L.or_step.argtypes = [C.c_void_p, P(C.c_double), P(C.c_double), P(C.c_double),
                                  P(C.c_uint8), P(C.c_double), C.c_int]
            L.or_get_state.argtypes = [C.c_void_p, P(C.c_double), P(C.c_double), P(C.c_double),
                                       P(C.c_int32), P(C.c_uint32)]
            L.or_set_state.argtypes = [C.c_void_p, P(C.c_double), P(C.c_double), P(C.c_double),
                                       P(C.c_int32), P(C.c_uint32)]
            L.or_get_events.argtypes = [C.c_void_p, P(C.c_uint32), P(C.c_int32), P(C.c_double), P(C.c_double),
                                        P(C.c_double)]
            L.or_clear_margin.argtypes = [C.c_void_p]
            L.or_observe.argtypes = [C.c_void_p, P(C.c_double)]
            L.or_get_scenario.argtypes = [C.c_void_p, P(C.c_double)]
            L.or_set_scenario.argtypes = [C.c_void_p, P(C.c_double)]
            L.or_goals.argtypes = [C.c_void_p, P(C.c_double)]
            L.or_formation_offset.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, P(C.c_double)]
            L.or_pairs_f32.argtypes = [P(C.c_float), P(C.c_float), P(C.c_int32), C.c_int, C.c_int,
                                       P(C.c_int32), P(C.c_uint8)]
            _lib = L
    return _lib


def _ptr(a, ctype):
    if a is None:
        return None
    return a.ctypes.data_as(C.POINTER(ctype))


def philox4x32_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().or_philox4x32_10(_ptr(c, C.c_uint32), _ptr(k, C.c_uint32), _ptr(out, C.c_uint32))
    return out


def philox4x32_10_batch(ctr, key) -> np.ndarray:
    """Philox4x32-10 of every row of ctr [n][4] under key [2]: [n][4] uint32."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros_like(c)
    lib().or_philox4x32_10_n(_ptr(c, C.c_uint32), _ptr(k, C.c_uint32), _ptr(out, C.c_uint32), c.shape[0])
    return out


def uniform(r: int) -> float:
    return lib().or_uniform(int(r))


def polar(m) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(m, dtype=np.float64).reshape(9))
    out = np.zeros(9)
    lib().or_polar(_ptr(a, C.c_double), _ptr(out, C.c_double))
    return out.reshape(3, 3)


def pair_key(xi, xj) -> np.float32:
    a = np.ascontiguousarray(xi, dtype=np.float32)
    b = np.ascontiguousarray(xj, dtype=np.float32)
    return np.float32(lib().or_pair_key(_ptr(a, C.c_float), _ptr(b, C.c_float)))


def pairs_f32(pos, arm, env_off, K):
    """Canonical KNN indices [D][K] (-1 padded) and hit flags [D] on binary32 inputs."""
    pos = np.ascontiguousarray(pos, dtype=np.float32)
    arm = np.ascontiguousarray(arm, dtype=np.float32)
    off = np.ascontiguousarray(env_off, dtype=np.int32)
    D = int(off[-1])
    knn = np.zeros((D, max(K, 1)), dtype=np.int32)
    hit = np.zeros(D, dtype=np.uint8)
    lib().or_pairs_f32(_ptr(pos, C.c_float), _ptr(arm, C.c_float), _ptr(off, C.c_int32),
                       len(off) - 1, int(K), _ptr(knn, C.c_int32), _ptr(hit, C.c_uint8))
    return knn[:, :K], hit


def formation_offset(form, k: int, n: int, s: float, rmax: float) -> np.ndarray:
    """Offset of goal slot k of an n-goal formation (FORM_NAMES or index)."""
    f = FORM_NAMES.index(form) if isinstance(form, str) else int(form)
    out = np.zeros(3)
    lib().or_formation_offset(f, int(k), int(n), float(s), float(rmax), _ptr(out, C.c_double))
    return out


def default_config(**kw) -> OrConfig:
    c = OrConfig()
    lib().or_default_config(C.byref(c))
    set_config(c, **kw)
    return c


def set_config(c: OrConfig, **kw) -> OrConfig:
    for k, v in kw.items():
        if k == "weights":
            for name, val in v.items():
                c.w[W_NAMES.index(name)] = float(val)
        elif k == "w":
            for i, val in enumerate(v):
                c.w[i] = float(val)
        else:
            setattr(c, k, v)
    return c


class Oracle:
    """One oracle instance: ``n_envs`` environments with the given swarm sizes."""

    def __init__(self, cfg: OrConfig, swarm_sizes=None):
        L = lib()
        self.cfg = cfg
        E = cfg.n_envs
        sizes = np.ones(E, dtype=np.int32) if swarm_sizes is None else np.ascontiguousarray(
            swarm_sizes, dtype=np.int32)
        assert sizes.shape == (E,)
        self.sizes = sizes
        self.env_off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int32)
        self.h = L.or_create(C.byref(cfg), _ptr(sizes, C.c_int32))
        if not self.h:
            raise ValueError("oracle: invalid configuration")
        self.D = int(L.or_n_drones(self.h))
        self.E = E
        self.K = int(cfg.k_neighbors)
        self.obs_dim = 18 + 6 * self.K

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            lib().or_destroy(h)
            self.h = None

    def reset(self, seed: int, mask=None):
        m = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
        lib().or_reset(self.h, C.c_uint64(int(seed)), _ptr(m, C.c_uint8))

    def step(self, actions, n_threads: int = 1, want_obs=True, want_loss=False, loss=None):
        a = np.ascontiguousarray(actions, dtype=np.float64).reshape(self.D, 4)
        obs = np.zeros((self.D, self.obs_dim)) if want_obs else None
        rew = np.zeros(self.D)
        done = np.zeros(self.E, dtype=np.uint8)
        if want_loss and loss is None:
            loss = np.zeros(self.D)
        lib().or_step(self.h, _ptr(a, C.c_double), _ptr(obs, C.c_double), _ptr(rew, C.c_double),
                      _ptr(done, C.c_uint8), _ptr(loss, C.c_double) if want_loss else None,
                      int(n_threads))
        if want_loss:
            return obs, rew, done, loss
        return obs, rew, done

    def get_state(self):
        st = np.zeros((self.D, NST))
        prm = np.zeros((self.E, NPRM))
        goal = np.zeros((self.E, 3))
        ep = np.zeros(self.E, dtype=np.int32)
        tick = np.zeros(self.E, dtype=np.uint32)
        lib().or_get_state(self.h, _ptr(st, C.c_double), _ptr(prm, C.c_double),
                           _ptr(goal, C.c_double), _ptr(ep, C.c_int32), _ptr(tick, C.c_uint32))
        return {"state": st, "params": prm, "goals": goal, "ep_step": ep, "tick": tick}

    def set_state(self, state=None, params=None, goals=None, ep_step=None, tick=None):
        st = None if state is None else np.ascontiguousarray(state, dtype=np.float64).reshape(self.D, NST)
        prm = None if params is None else np.ascontiguousarray(params, dtype=np.float64).reshape(self.E, NPRM)
        goal = None if goals is None else np.ascontiguousarray(goals, dtype=np.float64).reshape(self.E, 3)
        ep = None if ep_step is None else np.ascontiguousarray(np.broadcast_to(ep_step, (self.E,)), dtype=np.int32)
        tk = None if tick is None else np.ascontiguousarray(np.broadcast_to(tick, (self.E,)), dtype=np.uint32)
        lib().or_set_state(self.h, _ptr(st, C.c_double), _ptr(prm, C.c_double), _ptr(goal, C.c_double),
                           _ptr(ep, C.c_int32), _ptr(tk, C.c_uint32))

    def get_scenario(self) -> np.ndarray:
        rec = np.zeros((self.E, NSCN))
        lib().or_get_scenario(self.h, _ptr(rec, C.c_double))
        return rec

    def set_scenario(self, rec):
        r = np.ascontiguousarray(rec, dtype=np.float64).reshape(self.E, NSCN)
        lib().or_set_scenario(self.h, _ptr(r, C.c_double))

    def goals(self) -> np.ndarray:
        """Per-drone goals [D][3] at each env's current control step."""
        g = np.zeros((self.D, 3))
        lib().or_goals(self.h, _ptr(g, C.c_double))
        return g

    def observe(self):
        obs = np.zeros((self.D, self.obs_dim))
        lib().or_observe(self.h, _ptr(obs, C.c_double))
        return obs

    def get_events(self):
        ev = np.zeros(self.D, dtype=np.uint32)
        knn = np.zeros((self.D, max(self.K, 1)), dtype=np.int32)
        margin = np.zeros(self.D)
        margin_knn = np.zeros(self.D)
        cond = np.zeros(self.D)
        lib().or_get_events(self.h, _ptr(ev, C.c_uint32), _ptr(knn, C.c_int32), _ptr(margin, C.c_double),
                            _ptr(margin_knn, C.c_double), _ptr(cond, C.c_double))
        self.last_margin_knn = margin_knn
        self.last_cond = cond
        return ev, knn[:, :self.K], margin

    def margins(self):
        """(dynamics margin since the last reset/clear, neighbour-order margin of the last step)."""
        _, _, m = self.get_events()
        return m, self.last_margin_knn

    def conditioning(self):
        """Smallest heading-extraction length of any floor reset since the last reset/clear."""
        self.get_events()
        return self.last_cond

    def clear_margin(self):
        lib().or_clear_margin(self.h)
