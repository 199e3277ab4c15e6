"""The debug build with device index checks (libquadswarm_gpu_debug.so,
QS_DEBUG_CHECKS): the bounds substitute beside the guard bands of
tests/test_gpu_bounds.py, since compute-sanitizer is closed on this machine.

Every kernel family runs in the debug build on shapes that exercise its
launch geometry (every swarm-width class, warp-specialised and persistent
forms, scenarios, downwash, masked resets, the differentiable rollout with
every contact model): no index check fails (qs_sync would return
QS_ERR_INDEX) and every output equals the release build's bit for bit. A
check that fails is reported: the self-test entry point checks an index
equal to the drone count, which the kernel skips and qs_sync reports."""
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

from gpu_helpers import DEV, pair
from paper_2306_09537_gb300 import build as B
from paper_2306_09537_gb300 import qs

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


def run_with(lib, out):
    env = dict(os.environ, QS_LIBRARY=lib)
    r = subprocess.run([sys.executable, os.path.join(HERE, "debug_checks_run.py"), out], env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    return np.load(out)


def test_debug_build_checks_pass_and_match_release(tmp_path):
    B.build(with_debug=True)
    dbg = run_with(B.LIB_DEBUG, str(tmp_path / "debug.npz"))
    rel = run_with(B.LIB, str(tmp_path / "release.npz"))
    assert int(dbg["flags"][0]) == qs.QS_BUILD_DEBUG_CHECKS and int(rel["flags"][0]) == 0
    assert sorted(dbg.files) == sorted(rel.files)
    for k in dbg.files:
        if k != "flags":
            assert np.array_equal(dbg[k], rel[k], equal_nan=True), k


def test_failed_check_is_reported_without_access():
    code = r'''
import sys, torch
sys.path.insert(0, sys.argv[1]); sys.path.insert(0, sys.argv[1] + "/tests")
from gpu_helpers import pair
from paper_2306_09537_gb300 import qs
env, _ = pair([3, 5], 0, ("floor",), seed=1)
env.reset(1)
qs.qs_debug_check_selftest(env.h, env.D - 1)   # in range: passes
env.sync()
qs.qs_debug_check_selftest(env.h, env.D)       # one past the end: checked, skipped, reported
try:
    env.sync()
except qs.QSError as e:
    assert e.status == qs.QS_ERR_INDEX, e.status
    print("reported")
'''
    env = dict(os.environ, QS_LIBRARY=B.LIB_DEBUG)
    r = subprocess.run([sys.executable, "-c", code, os.path.dirname(HERE)], env=env, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0 and "reported" in r.stdout, r.stdout[-2000:] + r.stderr[-2000:]


def test_release_build_has_no_selftest():
    env, _ = pair([3], 0, ("floor",), seed=1)
    with pytest.raises(qs.QSError) as e:
        qs.qs_debug_check_selftest(env.h, 0)
    assert e.value.status == qs.QS_ERR_UNSUPPORTED
