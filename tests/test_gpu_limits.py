"""GPU parity at the interface's limits against the FP64 oracle: the largest
L-BFGS history (m = 8) and the smallest (m = 1) in the fused plan, the largest
sphere table (64 spheres: the self-collision masks use every bit), and the swept
check with four waypoints per lane (T = 128)."""
import dataclasses

import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import rel_l2, to_np
from oracle.oracle import esdf_lookup
from paper_2410_16727_gb300 import api, binding as B, inputs as I

pytestmark = pytest.mark.gpu


def _cuda(a):
    return torch.as_tensor(np.ascontiguousarray(a, np.float32)).cuda()


def _robot64():
    r = I.make_robot()
    rng = np.random.default_rng(64)
    extra = 64 - len(r.sph_r)
    fr = np.concatenate([r.sph_frame, rng.integers(1, 9, extra).astype(np.int32)])
    o = np.concatenate([r.sph_o, rng.normal(0.0, 0.05, (extra, 3)).astype(np.float32)])
    rad = np.concatenate([r.sph_r, rng.uniform(0.03, 0.06, extra).astype(np.float32)])
    order = np.argsort(fr, kind="stable")
    return dataclasses.replace(r, sph_frame=fr[order], sph_o=o[order], sph_r=rad[order])


def _on_cell_face(orc, wl, p, x, robot, tol=2e-5):
    """Some sphere of trajectory x with an active collision hinge has its centre
    (FP64, the oracle's chain) within tol voxels of a cell face: there the
    trilinear gradient's normal component jumps, and FP32 rounding of the
    position (about 5e-6 voxels here) may pick the neighbouring cell."""
    sc = int(wl.scene_of_problem[p])
    g = wl.grids[sc]
    c = orc.sphere_centres(x.astype(np.float64)).reshape(-1, 3)
    phi, _ = esdf_lookup(orc.phis[sc], g, c)
    active = (np.tile(robot.sph_r.astype(np.float64), x.shape[0]) + 0.01 - phi) > 0
    u = (c - np.asarray(g.origin, np.float64)) / g.res - 0.5
    return bool(((np.abs(u - np.round(u)) < tol).any(axis=1) & active).any())


def _setup(robot, cost, T, S, n_problems=4, opt=None):
    spec = I.WORKLOADS["tiny"]
    cub, grids = I.make_scenes(spec, n_scenes=2)
    orc = oracle.Oracle(robot, cost, grids, cub, T=T)
    wl = I.build_workload(spec, cub, grids, orc.clearance, orc.flange_pose, n_problems=n_problems, S=S, T=T,
                          robot=robot)
    wl = dataclasses.replace(wl, cost=cost)
    planner = api.Planner(robot, cost, opt or wl.opt)
    planner.set_scenes(cub, grids)
    batch = planner.batch(wl.q_start, wl.goal, wl.scene_of_problem, S, T)
    return wl, orc, planner, batch


@pytest.mark.parametrize("m", [1, 8])
def test_history_length_limits_follow_oracle(gpu_lib, m):
    opt = I.OptParams(iters=12, m=m)
    wl, orc, planner, batch = _setup(I.make_robot(), I.CostParams(), 32, 16, opt=opt)
    out = planner.plan(batch, wl.seeds)
    ref = orc.plan(wl.scene_of_problem, wl.q_start, wl.goal, wl.seeds, opt)
    rel = np.abs(to_np(out["cost"]) - ref["cost"]) / np.maximum(ref["cost"], 1e-6)
    assert np.quantile(rel, 0.95) <= 1e-3 and rel.max() <= 1e-2, (np.quantile(rel, 0.95), rel.max())


@pytest.mark.parametrize("T,w_self", [(32, 0.0), (64, 0.0), (32, 100.0)])
def test_64_spheres_cost_and_gradient(gpu_lib, T, w_self):
    robot = _robot64()
    cost = dataclasses.replace(I.CostParams(), w_self=w_self)
    wl, orc, planner, batch = _setup(robot, cost, T, 8)
    h = B.Robot(robot)
    assert h.n_spheres == 64
    if w_self > 0:
        assert np.array_equal(h.self_pairs(), orc.self_mask)
    rng = np.random.default_rng(T)
    x = np.stack([I.random_trajectories(rng, wl.q_start[p], 8, T, robot.limits, spread=1.5)
                  for p in range(wl.P)]).astype(np.float32)
    c, g = B.cost_grad(planner.robot, batch.desc, batch.pr, _cuda(x))
    c, g = to_np(c), to_np(g)
    skipped = 0
    for p in range(wl.P):
        wc, wg = orc.cost(int(wl.scene_of_problem[p]), wl.q_start[p], wl.goal[p], x[p])
        for s in range(8):
            assert abs(c[p, s] - wc[s]) <= 1e-4 * max(abs(wc[s]), 1e-6), (p, s)
            if _on_cell_face(orc, wl, p, x[p, s], robot):
                skipped += 1
                continue
            assert rel_l2(g[p, s], wg[s]) <= 1e-3, (p, s)
    assert skipped <= 2, skipped
    # the sphere centres of the 64-sphere table, in the caller's order
    q = wl.seeds[0, :2].reshape(-1, 7)
    _, sph = B.fk(planner.robot, _cuda(q), spheres=True)
    assert np.abs(to_np(sph) - orc.sphere_centres(q)).max() <= 1e-5


def test_sweep_four_waypoints_per_lane(gpu_lib):
    cost = dataclasses.replace(I.CostParams(), n_sweep=2)
    T = 128
    wl, orc, planner, batch = _setup(I.make_robot(), cost, T, 4, n_problems=2)
    rng = np.random.default_rng(128)
    x = np.stack([I.random_trajectories(rng, wl.q_start[p], 4, T, wl.robot.limits, spread=1.5)
                  for p in range(wl.P)]).astype(np.float32)
    c, g = B.cost_grad(planner.robot, batch.desc, batch.pr, _cuda(x))
    c, g = to_np(c), to_np(g)
    for p in range(wl.P):
        wc, wg = orc.cost(int(wl.scene_of_problem[p]), wl.q_start[p], wl.goal[p], x[p])
        for s in range(4):
            assert abs(c[p, s] - wc[s]) <= 1e-4 * max(abs(wc[s]), 1e-6), (p, s)
            assert rel_l2(g[p, s], wg[s]) <= 1e-3, (p, s)
    opt = I.OptParams(iters=3)
    planner2 = api.Planner(wl.robot, cost, opt)
    planner2.set_scenes(wl.cuboids, wl.grids)
    out = planner2.plan(planner2.batch(wl.q_start, wl.goal, wl.scene_of_problem, 4, T), wl.seeds)
    ref = orc.plan(wl.scene_of_problem, wl.q_start, wl.goal, wl.seeds, opt)
    rel = np.abs(to_np(out["cost"]) - ref["cost"]) / np.maximum(ref["cost"], 1e-6)
    assert rel.max() <= 1e-3, rel.max()
