"""Shared set-up of the GPU parity tests: workloads are drawn with the oracle's
clearance and FK callbacks (no oracle input ever comes from the CUDA path), then
both sides receive the same float32 arrays."""
import numpy as np
import torch

import oracle
from paper_2410_16727_gb300 import api, binding as B, inputs as I


def oracle_workload(name, n_scenes=None, **kw):
    spec = I.WORKLOADS[name]
    cub, grids = I.make_scenes(spec, n_scenes=n_scenes)
    T = kw.get("T", spec.T)
    orc = oracle.Oracle(I.make_robot(), I.CostParams(), grids, cub, T=T)
    wl = I.build_workload(spec, cub, grids, orc.clearance, orc.flange_pose, **kw)
    return wl, orc


def gpu_side(wl, opt=None):
    planner = api.Planner(wl.robot, wl.cost, opt or wl.opt)
    planner.set_scenes(wl.cuboids, wl.grids)
    batch = planner.batch(wl.q_start, wl.goal, wl.scene_of_problem, wl.S, wl.T)
    return planner, batch


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


def to_np(t):
    return t.detach().cpu().numpy()
