"""The oracle's pins reject plausible mistakes: each case below plants one
mistake in a copy of the oracle's source (a wrong sign, a dropped term, a
transposed operand, a wrong index), builds it, and runs the pin suite
(tests/test_oracle_pins.py and the principal-axis pins of
tests/test_oracle_conditioning.py) against that build; some pin must fail. A mistake
no pin catches would pass straight into the GPU parity bars."""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE = os.path.join(ROOT, "oracle")
OUT = os.path.join(ORACLE, "_build", "mutants")

# name: [(text in qs_oracle.c, replacement)], each text present exactly once
MUTANTS = {
    # S3 wrench
    "yaw spin signs flipped": [("const double spin[4] = {-1.0, 1.0, -1.0, 1.0};",
                                "const double spin[4] = {1.0, -1.0, 1.0, -1.0};")],
    "pitch torque sign": [("tau[1] += -px * f[r];", "tau[1] += px * f[r];")],
    "roll torque sign": [("tau[0] += py * f[r];", "tau[0] += -py * f[r];")],
    # S1 motor lag
    "lag coefficient exp(-dt/tau) instead of 1 - exp(-dt/tau)": [
        ("const double alpha_lag = 1.0 - exp(-dt / tau_m);", "const double alpha_lag = exp(-dt / tau_m);")],
    # S4 linear dynamics
    "gravity sign": [("F[2] / m - g}", "F[2] / m + g}")],
    "thrust along a row of R instead of its third column": [
        ("double F[3] = {R[2] * T, R[5] * T, R[8] * T};", "double F[3] = {R[6] * T, R[7] * T, R[8] * T};")],
    # S5 angular dynamics
    "gyroscopic term dropped": [
        ("double wdot[3] = {(tau[0] - gyro[0]) / ixx, (tau[1] - gyro[1]) / iyy, (tau[2] - gyro[2]) / izz};",
         "double wdot[3] = {tau[0] / ixx, tau[1] / iyy, tau[2] / izz};")],
    "gyroscopic term with the x and y inertias swapped": [
        ("double Iw[3] = {ixx * w[0], iyy * w[1], izz * w[2]};", "double Iw[3] = {iyy * w[0], ixx * w[1], izz * w[2]};")],
    "gyroscopic term sign": [("(tau[0] - gyro[0]) / ixx, (tau[1] - gyro[1]) / iyy, (tau[2] - gyro[2]) / izz",
                              "(tau[0] + gyro[0]) / ixx, (tau[1] + gyro[1]) / iyy, (tau[2] + gyro[2]) / izz")],
    # S6 integration
    "explicit instead of semi-implicit Euler": [
        ("for (int k = 0; k < 3; ++k) x[k] += v[k] * dt;",
         "for (int k = 0; k < 3; ++k) x[k] += (v[k] - acc[k] * dt) * dt;")],
    "rotation advanced the wrong way": [("M[3 * i + 0] = r0 + dt *", "M[3 * i + 0] = r0 - dt *"),
                                        ("M[3 * i + 1] = r1 + dt *", "M[3 * i + 1] = r1 - dt *"),
                                        ("M[3 * i + 2] = r2 + dt *", "M[3 * i + 2] = r2 - dt *")],
    # S7, S8 contacts
    "floor hit heading sign": [("if (hyp >= 1e-6) { cs = R[0] / hyp; sn = R[3] / hyp; }",
                                "if (hyp >= 1e-6) { cs = R[0] / hyp; sn = -R[3] / hyp; }")],
    "wall reflects instead of removing the normal velocity": [
        ("if (v[k] > 0.0) { v[k] = 0.0; hit_wall = 1;", "if (v[k] > 0.0) { v[k] = -v[k]; hit_wall = 1;")],
    # S10 collision response
    "collision response sign": [
        ("(vj[0] - vi[0]) * n[0] + (vj[1] - vi[1]) * n[1] + (vj[2] - vi[2]) * n[2]",
         "(vi[0] - vj[0]) * n[0] + (vi[1] - vj[1]) * n[1] + (vi[2] - vj[2]) * n[2]")],
    # S11 neighbours
    "neighbour ties to the higher index": [("return x->j < y->j ? -1 : (x->j > y->j ? 1 : 0);",
                                            "return x->j > y->j ? -1 : (x->j < y->j ? 1 : 0);")],
    # S12 observation
    "goal-relative position sign": [("o[k] = x[k] - goal[k] + ex[k];", "o[k] = goal[k] - x[k] + ex[k];")],
    "neighbour-relative position sign": [("on[q] = sj[OR_S_X + q] - x[q];", "on[q] = x[q] - sj[OR_S_X + q];")],
    "rotation observed transposed": [("for (int k = 0; k < 9; ++k) o[6 + k] = R[k];",
                                      "for (int k = 0; k < 9; ++k) o[6 + k] = R[3 * (k % 3) + k / 3];")],
    "position noise U(0, s) instead of U(-s, s)": [("ex[0] = (2.0 * u0[0] - 1.0) * c->obs_sigma_x;",
                                                    "ex[0] = u0[0] * c->obs_sigma_x;")],
    # S13 reward
    "spin norm missing a component": [("r += W[OR_W_SPIN] * sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);",
                                       "r += W[OR_W_SPIN] * sqrt(w[0] * w[0] + w[1] * w[1]);")],
    "orientation term on the wrong entry of R": [("r += W[OR_W_ORI] * R[8];", "r += W[OR_W_ORI] * R[4];")],
    "command change with swapped rotors": [("fh[0] - fprev[0], fh[1] - fprev[1]", "fh[0] - fprev[1], fh[1] - fprev[0]")],
    "proximity term on the squared distance": [("near += fmax(1.0 - dd / alpha_prox, 0.0);",
                                                "near += fmax(1.0 - dd * dd / alpha_prox, 0.0);")],
    # S0 randomisation and the random streams
    "randomisation range halved": [("c->dr_lo + (c->dr_hi - c->dr_lo) * u[k]",
                                    "c->dr_lo + (c->dr_hi - c->dr_lo) * 0.5 * u[k]")],
    "uniform from the wrong bits": [("((double)(r >> 9) + 0.5) * (1.0 / 8388608.0)",
                                     "((double)(r >> 8) + 0.5) * (1.0 / 16777216.0)")],
    "Box-Muller angle pi u instead of 2 pi u": [("double ang = 2.0 * M_PI * u1;", "double ang = M_PI * u1;")],
    "initial velocity range [0, 2] instead of [-1, 1]": [("s[OR_S_V + 1] = -1.0 + 2.0 * u[4];",
                                                          "s[OR_S_V + 1] = 2.0 * u[4];")],
    "initial rotation from a wrong quaternion formula": [("R[1] = 2.0 * (qx * qy - qz * qw);",
                                                          "R[1] = 2.0 * (qx * qy + qz * qw);")],
    # S1, S2 motors
    "thrust linear in the rotor speed": [("f[r] = fmax * uf[r] * uf[r] + eps[r];", "f[r] = fmax * uf[r] + eps[r];")],
    "motor noise without its AR(1) memory": [("eps[r] = c->alpha_nd * eps[r] + alpha_ns * n[r];",
                                              "eps[r] = alpha_ns * n[r];")],
    # S6, S7, S8 again
    "no re-orthonormalisation": [("double nx = 0.5 * (x[k] + it[k]);", "double nx = x[k];")],
    "friction on m g instead of m g - F_z": [("double ffric = c->mu * (m * g - F[2]);",
                                              "double ffric = c->mu * m * g;")],
    "ceiling reflects": [("if (v[2] > 0.0) { v[2] = 0.0; hit_ceil = 1;",
                          "if (v[2] > 0.0) { v[2] = -v[2]; hit_ceil = 1;")],
    "wall body-rate perturbation dropped": [("w[k] = w[k] + c->coll_sigma_w * n[3 + k];", "w[k] = w[k];")],
    "smooth floor pulls down": [("acc[2] += kc * softplus_b(-x[2], beta);", "acc[2] -= kc * softplus_b(-x[2], beta);")],
    # S9, S10 again
    "collision radius l instead of 2 l": [("volatile float r = li + lj;", "volatile float r = li;")],
    "collision body-rate perturbation dropped": [("wi[k] = wi[k] + c->coll_sigma_w * nn[3 + k];", "wi[k] = wi[k];")],
    # S10b downwash
    "downwash pushes up": [("az[i] -= c->dw_k1 * (c->dw_k2 * dz + c->dw_b1);",
                            "az[i] += c->dw_k1 * (c->dw_k2 * dz + c->dw_b1);")],
    "downwash from the drone below": [("if (rxy2 < r * r && dz > 0.0 && dz < c->dw_height) {",
                                       "if (rxy2 < r * r && dz < 0.0 && -dz < c->dw_height) {")],
    # S13 done
    "episode ends a step late": [("int is_done = h->ep_t[e] >= c->episode_steps;",
                                  "int is_done = h->ep_t[e] > c->episode_steps;")],
    "body rates unbounded above": [("if (w[k] > c->omega_max) w[k] = c->omega_max;", "if (0) w[k] = c->omega_max;")],
    "velocity noise U(0, s) instead of U(-s, s)": [("evv[1] = (2.0 * u1[0] - 1.0) * c->obs_sigma_v;",
                                                    "evv[1] = u1[0] * c->obs_sigma_v;")],
    "body-rate noise missing on one axis": [
        ("ew[0] = n0 * c->obs_sigma_w; ew[1] = n1 * c->obs_sigma_w; ew[2] = n2 * c->obs_sigma_w;",
         "ew[0] = n0 * c->obs_sigma_w; ew[1] = n1 * c->obs_sigma_w; ew[2] = 0.0;")],
    # Sec. III-D scenario goals
    "circle radius s n / pi": [("double r = fmin(s * n / (2.0 * M_PI), rmax), th = 2.0 * M_PI * k / n;",
                                "double r = fmin(s * n / M_PI, rmax), th = 2.0 * M_PI * k / n;")],
    "grid not centred": [("out[0] = s * ((k % m) - 0.5 * (m - 1));\n        out[1] = s * ((k / m) - 0.5 * (rows - 1));",
                          "out[0] = s * (k % m);\n        out[1] = s * ((k / m) - 0.5 * (rows - 1));")],
    "sphere heights off by half a step": [("double z = 1.0 - (2.0 * k + 1.0) / n, rho = sqrt(1.0 - z * z);",
                                           "double z = 1.0 - (2.0 * k) / n, rho = sqrt(1.0 - z * z);")],
    "cylinder rings not centred": [("out[2] = s * ((k / m) - 0.5 * (used - 1));", "out[2] = s * (k / m);")],
    "cube layers twice as far apart": [("out[2] = s * ((k / (m * m)) - 0.5 * (layers - 1));",
                                        "out[2] = 2.0 * s * ((k / (m * m)) - 0.5 * (layers - 1));")],
    # smooth contacts and the loss of the differentiable rollout
    "softplus without the 1/beta": [("return (fmax(z, 0.0) + log1p(exp(-fabs(z)))) / beta;",
                                     "return (fmax(z, 0.0) + log1p(exp(-fabs(z))));")],
    "smooth pair pulls together": [
        ("out[0] += mag * dx / dist; out[1] += mag * dy / dist; out[2] += mag * dz / dist;",
         "out[0] -= mag * dx / dist; out[1] -= mag * dy / dist; out[2] -= mag * dz / dist;")],
    "smooth pair radius l instead of 2 l": [
        ("double mag = kc * softplus_b(2.0 * p[OR_P_ARM] - dist, c->smooth_beta);",
         "double mag = kc * softplus_b(p[OR_P_ARM] - dist, c->smooth_beta);")],
    "smooth ceiling pulls out": [("acc[2] -= kc * softplus_b(x[2] - c->room_h, beta);",
                                  "acc[2] += kc * softplus_b(x[2] - c->room_h, beta);")],
    "smooth wall pulls out": [("acc[0] -= kc * softplus_b(x[0] - c->room_hx, beta);",
                               "acc[0] += kc * softplus_b(x[0] - c->room_hx, beta);")],
    "loss command weight 1e-2": [("for (int r = 0; r < 4; ++r) l += 1e-3 * fh[r] * fh[r];",
                                  "for (int r = 0; r < 4; ++r) l += 1e-2 * fh[r] * fh[r];")],
    "loss on unsquared distances": [("for (int k = 0; k < 3; ++k) l += (x[k] - goal[k]) * (x[k] - goal[k]);",
                                     "for (int k = 0; k < 3; ++k) l += fabs(x[k] - goal[k]);")],
    "switch one step late": [("const int sw = tau >= (int)rec[OR_R_TSW];", "const int sw = tau > (int)rec[OR_R_TSW];")],
    "shrink factor starting contracted": [
        ("lam = 1.0 - (1.0 - c->se_min) * 0.5 * (1.0 - cos(2.0 * M_PI * tau / c->se_period));",
         "lam = 1.0 - (1.0 - c->se_min) * 0.5 * (1.0 + cos(2.0 * M_PI * tau / c->se_period));")],
    "dynamic goals keep the first centre": [
        ("for (int k = 0; k < 3; ++k) g[k] = (sw ? c1[k] : c0[k]) + off[k];",
         "for (int k = 0; k < 3; ++k) g[k] = c0[k] + off[k];")],
    "swarm vs swarm groups never exchange": [("const double* cc = (grp ^ sw) ? c1 : c0;",
                                              "const double* cc = grp ? c1 : c0;")],
    "swap never swaps": [("const int slot = sw ? swap_slot(h, rec_seed(rec), i, N) : i;", "const int slot = i;")],
    "Lissajous cosine": [("g[k] = c0[k] + c1[k] * sin(2.0 * M_PI * (p - floor(p)));",
                          "g[k] = c0[k] + c1[k] * cos(2.0 * M_PI * (p - floor(p)));")],
    "Lissajous time in substeps": [("const double T = c->substeps * c->dt;", "const double T = c->dt;")],
    "Bezier control point off the Catmull-Rom tangent": [("double p1 = w0[k] + (w1[k] - wm[k]) / 6.0,",
                                                          "double p1 = w0[k] + (w1[k] - wm[k]) / 3.0,")],
    "downwash body-rate noise dropped": [("wi[k] += Tc * c->dw_sigma_w * nn[3 + k];", "wi[k] += 0.0;")],
    "reset rotor speed at the hover command instead of its root": [("s[OR_S_UF + r] = sqrt(hov);",
                                                                     "s[OR_S_UF + r] = hov;")],
    "symmetric action map without the half": [("fh = 0.5 * (a + 1.0);", "fh = a + 1.0;")],
    "commands clipped at 0.9": [("fh = a_in[r] < 0.0 ? 0.0 : (a_in[r] > 1.0 ? 1.0 : a_in[r]);",
                                 "fh = a_in[r] < 0.0 ? 0.0 : (a_in[r] > 0.9 ? 0.9 : a_in[r]);")],
    "lag toward the command instead of its root": [("double u = sqrt(fh);", "double u = fh;")],
    "golden angle replaced by its complement": [
        ("return (uint32_t)floor(4294967296.0 * (3.0 - sqrt(5.0)) / 2.0);",
         "return (uint32_t)floor(4294967296.0 * (sqrt(5.0) - 1.0) / 4.0);")],
}


def _build(name, edits, src):
    for old, new in edits:
        assert src.count(old) == 1, (name, old)
        src = src.replace(old, new)
    stem = "".join(ch if ch.isalnum() else "_" for ch in name)
    cpath, so = os.path.join(OUT, stem + ".c"), os.path.join(OUT, stem + ".so")
    with open(cpath, "w") as f:
        f.write(src)
    subprocess.run(["gcc", "-std=c11", "-D_GNU_SOURCE", "-O2", "-fPIC", "-shared", "-ffp-contract=off",
                    "-fno-fast-math", "-pthread", "-I", ORACLE, "-o", so, cpath, "-lm"], check=True)
    return so


PIN_TESTS = [os.path.join(ROOT, "tests", "test_oracle_pins.py"),
             os.path.join(ROOT, "tests", "test_oracle_conditioning.py") + "::test_intermediate_axis_instability_rate",
             os.path.join(ROOT, "tests", "test_oracle_conditioning.py") + "::test_major_and_minor_axis_spin_is_stable"]


def _caught(name, edits, src):
    """True when a pin fails on the mutant (pytest exit code 1 with a failed
    test); any other outcome of the run (a collection or usage error, a crash)
    is a fault of the harness and raises."""
    so = _build(name, edits, src)
    env = dict(os.environ, QS_ORACLE_LIB=so)
    r = subprocess.run([sys.executable, "-m", "pytest", *PIN_TESTS, "-x", "-q", "-p", "no:cacheprovider",
                        "-m", "not gpu"], cwd=ROOT, env=env, capture_output=True, text=True)
    if r.returncode == 0:
        return False
    if r.returncode == 1 and " failed" in r.stdout:
        return True
    raise RuntimeError(f"mutant {name!r}: pytest exited {r.returncode} without a failed pin:\n"
                       f"{r.stdout[-2000:]}\n{r.stderr[-2000:]}")


def test_pins_reject_every_planted_mistake():
    if shutil.which("gcc") is None:
        pytest.skip("gcc is needed to build the mutated oracles")
    os.makedirs(OUT, exist_ok=True)
    with open(os.path.join(ORACLE, "qs_oracle.c")) as f:
        src = f.read()
    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        futs = {name: ex.submit(_caught, name, edits, src) for name, edits in MUTANTS.items()}
        survivors = [name for name, fut in futs.items() if not fut.result()]
    assert not survivors, f"mistakes no pin catches: {survivors}"
