"""Thin ctypes binding of the C ABI in include/qs.h (argument marshalling only).

Every function here has the name of the C entry point it calls and converts
torch tensors (device memory owned by the caller) or numpy arrays (host
memory) into plain pointers; all computation happens in libquadswarm_gpu.so.
Importing this module loads the library and raises if it is missing: there is
no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

from . import build as _build

(QS_OK, QS_ERR_ARG, QS_ERR_CUDA, QS_ERR_OOM, QS_ERR_STATE_NONFINITE, QS_ERR_TIMEOUT, QS_ERR_UNSUPPORTED,
 QS_ERR_INDEX) = range(8)
STATUS_NAMES = ["QS_OK", "QS_ERR_ARG", "QS_ERR_CUDA", "QS_ERR_OOM", "QS_ERR_STATE_NONFINITE", "QS_ERR_TIMEOUT",
                "QS_ERR_UNSUPPORTED", "QS_ERR_INDEX"]
QS_BUILD_DEBUG_CHECKS = 1
QS_MAX_SWARM, QS_MAX_K, QS_STATE_DIM, QS_PARAM_DIM = 128, 8, 30, 7
QS_BLOCK_WARP_SPECIALISED = 1

F_DR, F_MOTOR_NOISE, F_OBS_NOISE, F_COLLISIONS = 1 << 0, 1 << 1, 1 << 2, 1 << 3
F_FLOOR, F_WALLS, F_AUTO_RESET, F_SMOOTH = 1 << 4, 1 << 5, 1 << 6, 1 << 7
F_ACTION_SYMMETRIC, F_RECORD_KNN, F_DOWNWASH, F_EVENT_TIME = 1 << 8, 1 << 9, 1 << 10, 1 << 11
FEATURE_FLAGS = {"dr": F_DR, "motor_noise": F_MOTOR_NOISE, "obs_noise": F_OBS_NOISE, "collisions": F_COLLISIONS,
                 "floor": F_FLOOR, "walls": F_WALLS, "auto_reset": F_AUTO_RESET, "smooth": F_SMOOTH,
                 "action_symmetric": F_ACTION_SYMMETRIC, "record_knn": F_RECORD_KNN, "downwash": F_DOWNWASH,
                 "event_time": F_EVENT_TIME}
EV_HIT_FLOOR, EV_ON_FLOOR, EV_HIT_WALL, EV_HIT_CEIL, EV_HIT_QUAD = 1, 2, 4, 8, 16
W_NAMES = ["pos", "vel", "ori", "spin", "act", "dact", "rot", "yaw", "hit_floor", "on_floor", "hit_wall", "hit_ceil",
           "hit_quad", "near"]

EXPORTS = ["qs_config_default", "qs_create", "qs_destroy", "qs_get_dims", "qs_reset", "qs_step", "qs_step_host",
           "qs_rollout", "qs_set_rollout_shape", "qs_get_rollout_shape", "qs_diff_workspace_size",
           "qs_diff_forward", "qs_diff_backward", "qs_diff_grad_static", "qs_get_state", "qs_set_state",
           "qs_get_events", "qs_get_scenario", "qs_set_scenario", "qs_get_goals", "qs_sync", "qs_set_block",
           "qs_get_block", "qs_serve_begin", "qs_serve_step", "qs_serve_end", "qs_philox4x32_10", "qs_last_error",
           "qs_build_flags", "qs_debug_check_selftest"]
# training scenarios (Sec. III-D) and goal formations, in the order of QS_SCN_* / QS_FORM_*
SCENARIOS = ["single", "static", "dynamic", "swap", "shrink_expand", "swarm_vs_swarm", "pursuit_lissajous",
             "pursuit_bezier"]
FORMATIONS = ["circle", "grid", "sphere", "cylinder", "cube"]
QS_NSCN = 18


def scenario_mask(names) -> int:
    """Bit mask (qs_config.scenarios) of the named scenarios."""
    m = 0
    for n in names:
        m |= 1 << SCENARIOS.index(n)
    return m
QS_DIFF_STATIC_BYTES = 64 << 20
QS_SERVE_IDLE_MS_MAX = 60000  # longest idle wait of the resident server


class qs_params(C.Structure):
    _fields_ = [(n, C.c_float) for n in (
        "mass", "arm", "ixx", "iyy", "izz", "t2w", "kappa", "tau_m", "gravity", "mu",
        "alpha_nd", "alpha_ns_frac", "alpha_c", "coll_sigma_v", "coll_sigma_w",
        "obs_sigma_x", "obs_sigma_v", "obs_sigma_w", "room_hx", "room_hy", "room_h",
        "dr_lo", "dr_hi", "smooth_beta", "smooth_kc", "prox_factor", "omega_max",
        "dw_k1", "dw_k2", "dw_b1", "dw_height", "dw_sigma_a", "dw_sigma_w",
        "form_spacing", "form_rmax", "scn_margin", "se_min", "se_period", "liss_f", "bez_seg")] + [("w", C.c_float * 14)]


class qs_config(C.Structure):
    _fields_ = [("size", C.c_uint32), ("n_envs", C.c_int32), ("swarm_sizes", C.POINTER(C.c_int32)),
                ("n_per_env", C.c_int32), ("k_neighbors", C.c_int32), ("substeps", C.c_int32), ("dt", C.c_float),
                ("episode_steps", C.c_int32), ("seed", C.c_uint64), ("flags", C.c_uint32), ("scenarios", C.c_uint32),
                ("params", qs_params)]


class QSError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status}: {msg}")
        self.status = status


def library_path() -> str:
    return os.environ.get("QS_LIBRARY") or _build.LIB


def _load():
    # QS_LIBRARY names another build of the same sources to load (the debug
    # build with device index checks, _build.LIB_DEBUG)
    path = library_path()
    if not os.path.exists(path):
        raise ImportError(f"libquadswarm_gpu.so is not built ({path}); run __graft_entry__.build() or "
                          "python -m paper_2306_09537_gb300.build")
    L = C.CDLL(path)
    P, V = C.POINTER, C.c_void_p
    L.qs_config_default.argtypes = [P(qs_config)]
    L.qs_config_default.restype = None
    L.qs_create.argtypes = [P(qs_config), V, P(V)]
    L.qs_destroy.argtypes = [V]
    L.qs_get_dims.argtypes = [V, P(C.c_int32), P(C.c_int32), P(C.c_int32)]
    L.qs_reset.argtypes = [V, C.c_uint64, V, V]
    L.qs_step.argtypes = [V, V, V, V, V]
    L.qs_step_host.argtypes = [V, V, V, V, V]
    L.qs_rollout.argtypes = [V, C.c_int32, V, V, V, V]
    L.qs_set_rollout_shape.argtypes = [V, C.c_int32, C.c_int32, C.c_int32]
    L.qs_get_rollout_shape.argtypes = [V, P(C.c_int32), P(C.c_int32), P(C.c_int32)]
    L.qs_diff_workspace_size.argtypes = [V, C.c_int32, C.c_int32, P(C.c_size_t)]
    L.qs_diff_forward.argtypes = [V, C.c_int32, C.c_int32, V, V, V, V]
    L.qs_diff_backward.argtypes = [V, C.c_int32, C.c_int32, V, V, V, V, V]
    L.qs_diff_grad_static.argtypes = [V, C.c_int32, C.c_int32, V, V, V, V, V, V]
    L.qs_get_state.argtypes = [V, V, V, V, V, V]
    L.qs_set_state.argtypes = [V, V, V, V, V, V]
    L.qs_get_events.argtypes = [V, V, V]
    L.qs_get_scenario.argtypes = [V, V]
    L.qs_set_scenario.argtypes = [V, V]
    L.qs_get_goals.argtypes = [V, V]
    L.qs_sync.argtypes = [V]
    L.qs_serve_begin.argtypes = [V, V, C.c_int32, V, V, V, C.c_int32]
    L.qs_serve_step.argtypes = [V, C.c_int32]
    L.qs_serve_end.argtypes = [V]
    L.qs_philox4x32_10.argtypes = [V, C.c_uint32, C.c_uint32, C.c_int32, V, C.c_int64, V]
    L.qs_set_block.argtypes = [V, C.c_int32, C.c_int32]
    L.qs_get_block.argtypes = [V, C.c_int32, P(C.c_int32)]
    L.qs_last_error.argtypes = [V]
    L.qs_last_error.restype = C.c_char_p
    L.qs_build_flags.argtypes = []
    L.qs_debug_check_selftest.argtypes = [V, C.c_int32]
    for n in EXPORTS:
        if n not in ("qs_config_default", "qs_last_error"):
            getattr(L, n).restype = C.c_int
    return L


_L = _load()


def lib():
    return _L


def _p(t):
    """Pointer of a torch tensor / numpy array / None (no copies are made)."""
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        if not t.is_contiguous():
            raise ValueError("tensors passed to the C ABI must be contiguous")
        return C.c_void_p(t.data_ptr())
    if hasattr(t, "ctypes"):
        if not t.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays passed to the C ABI must be C-contiguous")
        return C.c_void_p(t.ctypes.data)
    raise TypeError(f"cannot pass {type(t)} to the C ABI")


def _check(status, h=None):
    if status != QS_OK:
        raise QSError(status, qs_last_error(h))
    return status


def qs_last_error(h=None) -> str:
    return _L.qs_last_error(h).decode()


def qs_config_default() -> qs_config:
    cfg = qs_config()
    _L.qs_config_default(C.byref(cfg))
    return cfg


def qs_create(cfg: qs_config, stream: int = 0, swarm_sizes=None):
    """Returns an opaque handle; `stream` is a cudaStream_t as an int."""
    keep = None
    if swarm_sizes is not None:
        import numpy as np
        keep = np.ascontiguousarray(swarm_sizes, dtype=np.int32)
        cfg.swarm_sizes = keep.ctypes.data_as(C.POINTER(C.c_int32))
    h = C.c_void_p()
    st = _L.qs_create(C.byref(cfg), C.c_void_p(stream), C.byref(h))
    cfg.swarm_sizes = None
    del keep
    _check(st)
    return h


def qs_destroy(h):
    return _check(_L.qs_destroy(h))


def qs_get_dims(h):
    d, e, o = C.c_int32(), C.c_int32(), C.c_int32()
    _check(_L.qs_get_dims(h, C.byref(d), C.byref(e), C.byref(o)), h)
    return d.value, e.value, o.value


def qs_reset(h, seed: int, env_mask=None, obs=None):
    return _check(_L.qs_reset(h, C.c_uint64(int(seed)), _p(env_mask), _p(obs)), h)


def qs_step(h, actions, obs=None, reward=None, done=None):
    return _check(_L.qs_step(h, _p(actions), _p(obs), _p(reward), _p(done)), h)


def qs_step_host(h, actions, obs=None, reward=None, done=None):
    return _check(_L.qs_step_host(h, _p(actions), _p(obs), _p(reward), _p(done)), h)


def qs_rollout(h, T: int, actions, obs=None, reward=None, done=None):
    return _check(_L.qs_rollout(h, int(T), _p(actions), _p(obs), _p(reward), _p(done)), h)


def qs_set_rollout_shape(h, block: int, fuse: int = 0, use_graph: bool = True):
    return _check(_L.qs_set_rollout_shape(h, int(block), int(fuse), int(bool(use_graph))), h)


def qs_get_rollout_shape(h):
    b, f, g = C.c_int32(), C.c_int32(), C.c_int32()
    _check(_L.qs_get_rollout_shape(h, C.byref(b), C.byref(f), C.byref(g)), h)
    return b.value, f.value, bool(g.value)


def qs_diff_workspace_size(h, T: int, ckpt_every: int) -> int:
    b = C.c_size_t()
    _check(_L.qs_diff_workspace_size(h, int(T), int(ckpt_every), C.byref(b)), h)
    return b.value


def qs_diff_forward(h, T: int, ckpt_every: int, x0, actions, loss, workspace):
    return _check(_L.qs_diff_forward(h, int(T), int(ckpt_every), _p(x0), _p(actions), _p(loss), _p(workspace)), h)


def qs_diff_backward(h, T: int, ckpt_every: int, actions, dloss, workspace, grad_actions, grad_x0):
    return _check(_L.qs_diff_backward(h, int(T), int(ckpt_every), _p(actions), _p(dloss), _p(workspace),
                                      _p(grad_actions), _p(grad_x0)), h)


def qs_diff_grad_static(h, T: int, ckpt_every: int, x0, actions, dloss, loss, grad_actions, grad_x0):
    """Forward + adjoint without a workspace argument: the library's fixed
    device array (QS_DIFF_STATIC_BYTES) holds the checkpoints, for callers
    that cannot allocate device memory at that point."""
    return _check(_L.qs_diff_grad_static(h, int(T), int(ckpt_every), _p(x0), _p(actions), _p(dloss), _p(loss),
                                         _p(grad_actions), _p(grad_x0)), h)


def qs_get_state(h, state=None, params=None, goals=None, ep_step=None, tick=None):
    return _check(_L.qs_get_state(h, _p(state), _p(params), _p(goals), _p(ep_step), _p(tick)), h)


def qs_set_state(h, state=None, params=None, goals=None, ep_step=None, tick=None):
    return _check(_L.qs_set_state(h, _p(state), _p(params), _p(goals), _p(ep_step), _p(tick)), h)


def qs_get_events(h, events=None, knn=None):
    return _check(_L.qs_get_events(h, _p(events), _p(knn)), h)


def qs_get_scenario(h, records):
    return _check(_L.qs_get_scenario(h, _p(records)), h)


def qs_set_scenario(h, records):
    return _check(_L.qs_set_scenario(h, _p(records)), h)


def qs_get_goals(h, goals):
    return _check(_L.qs_get_goals(h, _p(goals)), h)


def qs_sync(h):
    return _check(_L.qs_sync(h), h)


def qs_serve_begin(h, actions, obs=None, reward=None, done=None, idle_ms: int = 1000, n_slots: int = 1):
    return _check(_L.qs_serve_begin(h, _p(actions), int(n_slots), _p(obs), _p(reward), _p(done), int(idle_ms)), h)


def qs_serve_step(h, slot: int = 0):
    return _check(_L.qs_serve_step(h, int(slot)), h)


def qs_serve_end(h):
    return _check(_L.qs_serve_end(h), h)


def qs_philox4x32_10(ctr, key0: int, key1: int, out, variant: int = 0, stream=None):
    """out [n][4] = the library's Philox4x32-10 of ctr [n][3] (uint32 tensors on the device)."""
    n = ctr.shape[0]
    return _check(_L.qs_philox4x32_10(_p(ctr), C.c_uint32(int(key0)), C.c_uint32(int(key1)), int(variant), _p(out),
                                      int(n), stream))


def qs_build_flags() -> int:
    """Bits of the loaded build (QS_BUILD_DEBUG_CHECKS: device index checks)."""
    return int(_L.qs_build_flags())


def qs_debug_check_selftest(h, index: int):
    return _check(_L.qs_debug_check_selftest(h, int(index)), h)


def qs_set_block(h, width: int, block: int):
    return _check(_L.qs_set_block(h, int(width), int(block)), h)


def qs_get_block(h, width: int) -> int:
    b = C.c_int32()
    _check(_L.qs_get_block(h, int(width), C.byref(b)), h)
    return b.value


def make_config(n_envs=1, swarm=1, k_neighbors=0, features=(), seed=1, weights=None, scenarios=(),
                **overrides) -> qs_config:
    """qs_config from the library defaults, feature names, scenario names and overrides."""
    cfg = qs_config_default()
    cfg.scenarios = scenario_mask(scenarios)
    cfg.n_envs = int(n_envs)
    cfg.n_per_env = int(swarm) if swarm is not None else 1
    cfg.k_neighbors = int(k_neighbors)
    cfg.seed = int(seed)
    flags = 0
    for f in features:
        flags |= FEATURE_FLAGS[f]
    cfg.flags = flags
    if weights is not None:
        for i in range(14):
            cfg.params.w[i] = 0.0
        for name, val in weights.items():
            cfg.params.w[W_NAMES.index(name)] = float(val)
    for k, v in overrides.items():
        if hasattr(cfg.params, k):
            setattr(cfg.params, k, v)
        else:
            setattr(cfg, k, v)
    return cfg
