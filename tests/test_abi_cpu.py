"""C-ABI checks that need no GPU: the library builds and loads, exports every
function include/qs.h declares, validates arguments before touching the
device, and its default constants equal the oracle's (both are the readings
of the paper's unstated constants)."""
import ctypes as C
import math
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def qs():
    import __graft_entry__ as g
    g.build()
    from paper_2306_09537_gb300 import qs as q
    return q


def declared_functions():
    src = open(os.path.join(ROOT, "include", "qs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(qs_[a-z0-9_]+)\s*\(", src)))


def test_exports_every_declared_symbol(qs):
    names = declared_functions()
    assert len(names) >= 15
    lib = C.CDLL(qs.library_path())
    for n in names:
        assert hasattr(lib, n), f"{n} declared in include/qs.h but not exported"
    assert sorted(qs.EXPORTS) == names


def test_config_size_and_defaults_match_oracle(qs):
    from oracle import oracle as O
    cfg = qs.qs_config_default()
    assert cfg.size == C.sizeof(qs.qs_config)
    oc = O.default_config()
    p = cfg.params
    for name in ("mass", "arm", "ixx", "iyy", "izz", "t2w", "kappa", "tau_m", "gravity", "mu", "alpha_nd",
                 "alpha_ns_frac", "alpha_c", "coll_sigma_v", "coll_sigma_w", "obs_sigma_x", "obs_sigma_v",
                 "obs_sigma_w", "room_hx", "room_hy", "room_h", "dr_lo", "dr_hi", "smooth_beta", "smooth_kc",
                 "prox_factor", "omega_max", "dw_k1", "dw_k2", "dw_b1", "dw_height", "dw_sigma_a", "dw_sigma_w",
                 "form_spacing", "form_rmax", "scn_margin", "se_min", "se_period", "liss_f", "bez_seg"):
        assert getattr(p, name) == np.float32(getattr(oc, name)), name
    for i in range(14):
        assert p.w[i] == np.float32(oc.w[i])
    assert cfg.substeps == oc.substeps and math.isclose(cfg.dt, oc.dt, rel_tol=1e-7)
    assert cfg.episode_steps == oc.episode_steps and cfg.k_neighbors == oc.k_neighbors
    assert cfg.flags == oc.flags and cfg.scenarios == oc.scenarios == 0


@pytest.mark.parametrize("field,value,status", [
    ("n_envs", 0, 1), ("k_neighbors", -1, 1), ("k_neighbors", 9, 6), ("substeps", 0, 1), ("dt", 0.0, 1),
    ("episode_steps", 0, 1), ("n_per_env", 0, 1), ("n_per_env", 129, 6), ("size", 4, 1)])
def test_create_rejects_bad_config_without_device(qs, field, value, status):
    cfg = qs.qs_config_default()
    setattr(cfg, field, value)
    h = C.c_void_p()
    assert qs.lib().qs_create(C.byref(cfg), None, C.byref(h)) == status
    assert h.value is None
    assert qs.qs_last_error(None)


def test_create_rejects_bad_params(qs):
    cfg = qs.qs_config_default()
    cfg.params.mass = -1.0
    h = C.c_void_p()
    assert qs.lib().qs_create(C.byref(cfg), None, C.byref(h)) == qs.QS_ERR_ARG


def test_null_handle_calls_fail_cleanly(qs):
    L = qs.lib()
    assert L.qs_destroy(None) == qs.QS_ERR_ARG
    assert L.qs_step(None, None, None, None, None) == qs.QS_ERR_ARG
    assert L.qs_reset(None, 1, None, None) == qs.QS_ERR_ARG
    assert L.qs_sync(None) == qs.QS_ERR_ARG
    assert L.qs_rollout(None, 1, None, None, None, None) == qs.QS_ERR_ARG
    assert L.qs_get_dims(None, None, None, None) == qs.QS_ERR_ARG
    assert L.qs_serve_begin(None, None, 1, None, None, None, 1000) == qs.QS_ERR_ARG
    assert L.qs_serve_step(None, 0) == qs.QS_ERR_ARG
    assert L.qs_serve_end(None) == qs.QS_ERR_ARG
    assert "NULL" in qs.qs_last_error(None)


def test_debug_build_loads_with_every_symbol_and_its_flag(qs):
    """The debug build (device index checks) exports the same ABI and says so;
    the release build reports no checks."""
    from paper_2306_09537_gb300 import build as b
    dbg = C.CDLL(b.LIB_DEBUG)
    for n in declared_functions():
        assert hasattr(dbg, n), f"{n} missing from the debug build"
    dbg.qs_build_flags.restype = C.c_int32
    assert dbg.qs_build_flags() == qs.QS_BUILD_DEBUG_CHECKS
    assert qs.qs_build_flags() == 0
