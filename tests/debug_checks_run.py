"""Workload run by tests/test_gpu_debug_checks.py in a process of its own,
with whichever library QS_LIBRARY names: every kernel family on shapes that
exercise its launch geometry, a qs_sync after each, and the outputs saved for
a bitwise comparison between builds. Usage: debug_checks_run.py OUT.npz"""
import os
import sys

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

from paper_2306_09537_gb300 import qs  # noqa: E402
from paper_2306_09537_gb300 import workloads as W  # noqa: E402
from paper_2306_09537_gb300.env import QuadSwarmEnv  # noqa: E402

DEV = torch.device("cuda:0")
FULL = ("floor", "walls", "motor_noise", "obs_noise", "dr", "collisions", "record_knn", "auto_reset")


def main(out_path):
    out = {"flags": np.array([qs.qs_build_flags()])}
    stream = torch.cuda.Stream(device=DEV)
    with torch.cuda.stream(stream):
        cases = [
            ("plain", [1] * 3000, 0, FULL, ()),                                  # warp-specialised, uniform geometry
            ("uneven", [1, 2, 3, 5, 8, 13, 17, 31, 33, 64, 100, 128] * 6, 6, FULL, ()),  # every width class
            ("swarm_ws", [8] * 300, 6, FULL, ()),
            ("swarm64", [64, 40, 33] * 8, 6, FULL + ("downwash",), ()),
            ("scenarios", [8, 5, 16, 1] * 40, 6, FULL, tuple(qs.SCENARIOS)),
            # smooth contacts stepped by the general instance (pair penalty staged per substep)
            ("smooth_step", [1, 2, 8, 33, 64] * 8, 6, ("smooth", "motor_noise", "obs_noise", "dr", "collisions",
                                                     "record_knn", "auto_reset"), ()),
        ]
        for name, sizes, K, feats, scn in cases:
            env = QuadSwarmEnv(len(sizes), np.asarray(sizes, np.int32), K, feats, seed=11, device=DEV,
                               stream=stream, scenarios=scn)
            obs0 = env.reset(11).clone()
            acts = torch.from_numpy(W.actions(11, 12, env.D)).to(DEV)
            for t in range(6):
                env.step(acts[t])
            obs, rew, done = env.obs.clone(), env.reward.clone(), env.done.clone()
            T = 6
            ro = torch.empty(T, env.D, env.obs_dim, device=DEV)
            rr = torch.empty(T, env.D, device=DEV)
            rd = torch.empty(T, env.E, dtype=torch.uint8, device=DEV)
            env.rollout(acts[6:12].contiguous(), ro, rr, rd)
            ev, knn = env.get_events(knn=K > 0)
            st = env.get_state()
            goals = env.get_goals()
            mask = torch.zeros(env.E, dtype=torch.uint8, device=DEV)
            mask[::3] = 1
            env.reset(12, env_mask=mask)
            env.sync()  # raises QS_ERR_INDEX if any check failed
            for k, v in (("obs0", obs0), ("obs", obs), ("rew", rew), ("done", done), ("ro", ro), ("rr", rr),
                         ("rd", rd), ("ev", ev), ("state", st["state"]), ("goals", goals),
                         ("after_mask", env.get_state()["state"])):
                out[f"{name}_{k}"] = v.cpu().numpy()
            if knn is not None:
                out[f"{name}_knn"] = knn.cpu().numpy()
            env.close()
        # the differentiable rollout, every contact model
        for name, feats in (("smooth", ("smooth", "motor_noise", "dr")),
                            ("discrete", ("floor", "walls", "collisions", "motor_noise", "dr")),
                            ("event_time", ("floor", "walls", "collisions", "motor_noise", "dr", "event_time"))):
            sizes = np.asarray([8] * 12 + [3, 1, 17, 32], np.int32)
            env = QuadSwarmEnv(len(sizes), sizes, 0, feats, seed=13, device=DEV, stream=stream)
            env.reset(13)
            T, C = 12, 4
            x0 = env.get_state()["state"].contiguous()
            a = torch.from_numpy(W.actions(13, T, env.D, lo=0.05, hi=0.95)).to(DEV)
            ws = torch.empty(qs.qs_diff_workspace_size(env.h, T, C), dtype=torch.uint8, device=DEV)
            loss = torch.empty(env.D, device=DEV)
            ga = torch.empty_like(a)
            gx = torch.empty(env.D, 30, device=DEV)
            qs.qs_diff_forward(env.h, T, C, x0, a, loss, ws)
            qs.qs_diff_backward(env.h, T, C, a, torch.ones(env.D, device=DEV), ws, ga, gx)
            env.sync()
            out[f"diff_{name}_loss"] = loss.cpu().numpy()
            out[f"diff_{name}_ga"] = ga.cpu().numpy()
            out[f"diff_{name}_gx"] = gx.cpu().numpy()
            env.close()
    np.savez(out_path, **out)
    print("ok")


if __name__ == "__main__":
    main(sys.argv[1])
