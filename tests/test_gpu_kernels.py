"""GPU parity of the ESDF, FK, cost, adjoint and evaluation kernels against the
FP64 oracle, through the C ABI.

Tolerances (from the method's acceptance bar): ESDF values and sphere centres
1e-5 m; per-trajectory cost 1e-4 relative; gradient 1e-3 relative L2 per
trajectory."""
import math

import numpy as np
import pytest
import torch

import oracle
from gpu_helpers import gpu_side, oracle_workload, rel_l2, to_np
from paper_2410_16727_gb300 import api, binding as B, inputs as I

pytestmark = pytest.mark.gpu

TOL_M = 1e-5
TOL_COST = 1e-4
TOL_GRAD = 1e-3


def _cuda(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a)).to("cuda", dtype)


# ------------------------------------------------------------------ ESDF

@pytest.mark.parametrize("seed,n,nb", [(0, (8, 8, 8), 1), (1, (12, 10, 9), 2), (2, (16, 16, 16), 3),
                                       (3, (9, 13, 16), 3), (4, (33, 2, 5), 4)])
def test_esdf_small_grids(gpu_lib, seed, n, nb):
    rng = np.random.default_rng(seed)
    grid = I.Grid((-0.1, -0.05, 0.0), 0.037, n)
    ext = np.array(n) * grid.res
    boxes = np.array([[*(np.asarray(grid.origin) + rng.uniform(0.2, 0.8, 3) * ext), *rng.uniform(0.02, 0.12, 3)]
                      for _ in range(nb)], np.float32)
    got = to_np(B.scene_build_esdf(_cuda(boxes), grid))
    want = oracle.esdf_build(boxes, grid)
    assert np.abs(got - want).max() <= TOL_M


def test_esdf_empty_scene_is_far(gpu_lib):
    grid = I.Grid((0.0, 0.0, 0.0), 0.1, (4, 5, 6))
    got = to_np(B.scene_build_esdf(torch.zeros((0, 6), device="cuda"), grid))
    assert (got == B.ESDF_FAR).all()


def test_esdf_tiny_workload_full_grid(gpu_lib):
    cub, grids = I.make_scenes(I.WORKLOADS["tiny"])
    got = to_np(B.scene_build_esdf(_cuda(cub[0]), grids[0]))
    want = oracle.esdf_build(cub[0], grids[0])
    assert np.abs(got - want).max() <= TOL_M


def test_esdf_batch_matches_single_builds(gpu_lib):
    """One batched call over scenes of different grids and cuboid counts (incl. an
    empty scene) writes exactly what the single-scene call writes."""
    rng = np.random.default_rng(21)
    grids = [I.Grid((-0.2, -0.3, 0.0), 0.03, (20, 17, 9)), I.Grid((0.0, 0.0, 0.0), 0.05, (8, 8, 8)),
             I.Grid((-0.64, -0.64, -0.14), 0.02, (64, 64, 64)), I.Grid((-0.1, 0.1, 0.2), 0.01, (33, 40, 25))]
    cubs = [I.scene_tiny(rng, n_boxes=3), np.zeros((0, 6), np.float32), I.scene_tiny(rng, n_boxes=40),
            I.scene_clutter(rng, n_boxes=120)]
    dc = [_cuda(c).reshape(-1, 6) for c in cubs]
    batch = B.scene_build_esdf_batch(dc, grids)
    for c, g, got in zip(dc, grids, batch):
        assert torch.equal(got, B.scene_build_esdf(c, g))
    for c, g, got in zip(cubs, grids, batch):
        assert np.abs(to_np(got) - oracle.esdf_build(c, g)).max() <= TOL_M


@pytest.mark.parametrize("name", ["batched", "stress"])
def test_esdf_full_size_windows(gpu_lib, name):
    """Full 128^3 / 256^3 grids on the GPU; the oracle recomputes random 12^3
    windows of them (a window is a grid whose origin sits on a voxel corner)."""
    spec = I.WORKLOADS[name]
    cub, grids = I.make_scenes(spec, n_scenes=1)
    g = grids[0]
    got = to_np(B.scene_build_esdf(_cuda(cub[0]), g))
    rng = np.random.default_rng(11)
    w = 12
    for _ in range(6):
        i0 = [int(rng.integers(0, g.n[a] - w)) for a in range(3)]
        sub = I.Grid(tuple(g.origin[a] + i0[a] * g.res for a in range(3)), g.res, (w, w, w))
        want = oracle.esdf_build(cub[0], sub)
        part = got[i0[2]:i0[2] + w, i0[1]:i0[1] + w, i0[0]:i0[0] + w]
        assert np.abs(part - want).max() <= TOL_M


# ------------------------------------------------------------------ FK

def test_fk_sphere_centres_and_pose(gpu_lib):
    robot = I.make_robot()
    rng = np.random.default_rng(1)
    q = I.sample_configs(rng, robot.limits, 500, shrink=-0.1)   # include configurations beyond the limits
    q = np.concatenate([np.zeros((1, 7), np.float32),
                        np.array([[0, -math.pi / 4, 0, -3 * math.pi / 4, 0, math.pi / 2, math.pi / 4]], np.float32), q])
    planner = api.Planner(robot)
    pose, sph = planner.fk(q, spheres=True)
    pose, sph = to_np(pose), to_np(sph)
    orc = oracle.Oracle(robot, I.CostParams(), [I.WORKLOADS["tiny"].grid], [np.zeros((0, 6), np.float32)], T=1)
    want_sph = orc.sphere_centres(q)
    want_pose = oracle.flange_pose(robot.dh, q)
    assert np.abs(sph - want_sph).max() <= TOL_M
    assert np.abs(pose[:, :3] - want_pose[:, :3]).max() <= TOL_M
    dq = np.minimum(np.abs(pose[:, 3:] - want_pose[:, 3:]).max(1), np.abs(pose[:, 3:] + want_pose[:, 3:]).max(1))
    assert dq.max() <= 1e-5


# ------------------------------------------------------------------ cost / adjoint

def _random_batch(T, S=24, seed=0, name="tiny"):
    wl, orc = oracle_workload(name, n_scenes=1, n_problems=2, S=S, T=T)
    rng = np.random.default_rng(seed)
    x = np.stack([I.random_trajectories(rng, wl.q_start[p], S, T, wl.robot.limits, spread=1.2)
                  for p in range(wl.P)])
    # a few entries beyond the joint limits exercise the limit term
    x[:, ::5, 0, 3] = wl.robot.limits[3, 1] + 0.05
    return wl, orc, x


def _oracle_cost(orc, wl, x, grad=True, terms=False):
    outs = [orc.cost(int(wl.scene_of_problem[p]), wl.q_start[p], wl.goal[p], x[p], grad=grad, terms=terms)
            for p in range(wl.P)]
    return [np.stack([o[i] for o in outs]) for i in range(len(outs[0]))]


@pytest.mark.parametrize("T", [1, 7, 32, 33, 64, 100, 128])
def test_cost_and_terms_match_oracle(gpu_lib, T):
    wl, orc, x = _random_batch(T, seed=T)
    planner, batch = gpu_side(wl)
    cost, terms = B.cost(planner.robot, batch.desc, batch.pr, _cuda(x), terms=True)
    want_c, want_t = _oracle_cost(orc, wl, x, grad=False, terms=True)
    rel = np.abs(to_np(cost) - want_c) / np.maximum(np.abs(want_c), 1e-6)
    assert rel.max() <= TOL_COST, rel.max()
    assert (want_t[..., 0] > 0).any(), "case should have active collision terms"
    sc = np.maximum(np.abs(want_c)[..., None], 1e-6)
    assert (np.abs(to_np(terms) - want_t) / sc).max() <= TOL_COST


@pytest.mark.parametrize("T", [7, 64])
def test_kinematic_terms_periodic_in_joint_angles(gpu_lib, T):
    """The world and goal terms depend on the joints only through the chain's
    sines and cosines: shifting every joint angle by up to three whole turns
    leaves them at the oracle's values for the unshifted trajectories."""
    wl, orc, x = _random_batch(T, seed=200 + T)
    rng = np.random.default_rng(T)
    turns = rng.integers(-3, 4, size=x.shape)
    xs = (x + 2.0 * math.pi * turns).astype(np.float32)
    planner, batch = gpu_side(wl)
    _, terms = B.cost(planner.robot, batch.desc, batch.pr, _cuda(xs), terms=True)
    want_c, want_t = _oracle_cost(orc, wl, x.astype(np.float64), grad=False, terms=True)
    sc = np.maximum(np.abs(want_c)[..., None], 1e-6)
    got = to_np(terms)
    for j in (0, 2):                            # world, goal
        assert (np.abs(got[..., j] - want_t[..., j]) / sc[..., 0]).max() <= TOL_COST, j
    assert (want_t[..., 0] > 0).any() and (want_t[..., 2] > 0).any()


@pytest.mark.parametrize("T", [1, 5, 32, 47, 64, 128])
def test_gradient_matches_oracle(gpu_lib, T):
    wl, orc, x = _random_batch(T, seed=100 + T)
    planner, batch = gpu_side(wl)
    c, g = B.cost_grad(planner.robot, batch.desc, batch.pr, _cuda(x))
    want_c, want_g = _oracle_cost(orc, wl, x)
    rel_c = np.abs(to_np(c) - want_c) / np.maximum(np.abs(want_c), 1e-6)
    assert rel_c.max() <= TOL_COST
    gg = to_np(g)
    errs = np.array([rel_l2(gg[p, s], want_g[p, s]) for p in range(wl.P) for s in range(wl.S)])
    assert errs.max() <= TOL_GRAD, (errs.max(), np.sort(errs)[-5:])


def test_goal_quaternion_sign_and_scale(gpu_lib):
    """Goal quaternions are normalised on entry and q and -q name one rotation:
    with the goal quaternions multiplied by -1, 2.5 or -0.3 the cost, its goal
    term and the gradient stay at the oracle's values for the unit goals."""
    wl, orc, x = _random_batch(32, S=8, seed=11)
    want_c, want_g = _oracle_cost(orc, wl, x)
    _, want_t = _oracle_cost(orc, wl, x, grad=False, terms=True)
    assert (want_t[..., 2] > 0).all()
    planner = api.Planner(wl.robot, wl.cost, wl.opt)
    planner.set_scenes(wl.cuboids, wl.grids)
    sc = np.maximum(np.abs(want_c), 1e-6)
    for f in (-1.0, 2.5, -0.3):
        goal = wl.goal.copy()
        goal[:, 3:] *= f
        batch = planner.batch(wl.q_start, goal, wl.scene_of_problem, wl.S, wl.T)
        _, terms = B.cost(planner.robot, batch.desc, batch.pr, _cuda(x), terms=True)
        assert (np.abs(to_np(terms)[..., 2] - want_t[..., 2]) / sc).max() <= TOL_COST, f
        c, g = B.cost_grad(planner.robot, batch.desc, batch.pr, _cuda(x))
        assert (np.abs(to_np(c) - want_c) / sc).max() <= TOL_COST, f
        gg = to_np(g)
        errs = [rel_l2(gg[p, s], want_g[p, s]) for p in range(wl.P) for s in range(wl.S)]
        assert max(errs) <= TOL_GRAD, (f, max(errs))


def test_gradient_scale_and_autograd(gpu_lib):
    wl, orc, x = _random_batch(32, S=8, seed=7)
    planner, batch = gpu_side(wl)
    xt = _cuda(x).requires_grad_(True)
    c = api.trajectory_cost(xt, planner.robot, batch)
    w = torch.linspace(0.5, 2.0, c.numel(), device="cuda").reshape(c.shape)
    (c * w).sum().backward()
    _, g = B.cost_grad(planner.robot, batch.desc, batch.pr, _cuda(x))
    torch.testing.assert_close(xt.grad, g * w[..., None, None], rtol=1e-6, atol=1e-6)
    _, want_g = _oracle_cost(orc, wl, x)
    assert rel_l2(to_np(xt.grad), want_g * to_np(w)[..., None, None]) <= TOL_GRAD


def test_evaluate_matches_oracle(gpu_lib):
    wl, orc, x = _random_batch(32, S=32, seed=3)
    # include trajectories that end exactly at the goal configuration
    x[:, :4] = np.linspace(wl.q_start, wl.q_goal, 32, axis=1)[:, None]
    planner, batch = gpu_side(wl)
    ok, met = B.evaluate(planner.robot, batch.desc, batch.pr, _cuda(x))
    ok, met = to_np(ok).astype(bool), to_np(met)
    for p in range(wl.P):
        w_ok, w_met = orc.evaluate(int(wl.scene_of_problem[p]), wl.q_start[p], wl.goal[p], x[p])
        assert np.abs(met[p, :, 0] - w_met[:, 0]).max() <= TOL_M            # clearance
        assert np.abs(met[p, :, 1] - w_met[:, 1]).max() <= TOL_M            # translation error
        assert np.abs(met[p, :, 2] - w_met[:, 2]).max() <= 1e-4             # rotation error (rad)
        assert (np.abs(met[p, :, 3] - w_met[:, 3]) / np.maximum(w_met[:, 3], 1)).max() <= TOL_COST
        assert np.abs(met[p, :, 4] - w_met[:, 4]).max() <= 1e-6
        assert (np.abs(met[p, :, 5] - w_met[:, 5]) / np.maximum(w_met[:, 5], 1e-6)).max() <= TOL_COST
        # success flags are decided in each side's precision: equal unless a metric is within rounding of its threshold
        near = (np.abs(w_met[:, 0]) < 1e-5) | (np.abs(w_met[:, 1] - I.DELTA_T) < 1e-5) | \
               (np.abs(w_met[:, 2] - I.DELTA_R) < 1e-4)
        assert (ok[p] == w_ok)[~near].all()
        # the straight lines end on the goal configuration: zero pose error on both sides
        assert met[p, :4, 1].max() < 1e-5 and w_met[:4, 1].max() < 1e-6
        assert met[p, :4, 2].max() < 2e-3 and w_met[:4, 2].max() < 1e-5


def test_out_of_range_scene_gives_nan_not_fault(gpu_lib):
    wl, orc, x = _random_batch(16, S=4, seed=9)
    planner, batch = gpu_side(wl)
    bad = planner.batch(wl.q_start, wl.goal, np.array([0, 7], np.int32), wl.S, wl.T)
    c = to_np(B.cost(planner.robot, bad.desc, bad.pr, _cuda(x)))
    assert np.isfinite(c[0]).all() and np.isnan(c[1]).all()
    ok, _ = B.evaluate(planner.robot, bad.desc, bad.pr, _cuda(x))
    assert to_np(ok)[1].sum() == 0


def test_nan_trajectory_stays_in_bounds(gpu_lib):
    wl, orc, x = _random_batch(32, S=4, seed=10)
    x = x.copy()
    x[0, 1, 5, 2] = np.nan
    x[0, 2, 7, 1] = np.inf
    planner, batch = gpu_side(wl)
    c, g = B.cost_grad(planner.robot, batch.desc, batch.pr, _cuda(x))
    torch.cuda.synchronize()
    c = to_np(c)
    assert np.isnan(c[0, 1]) and np.isfinite(c[0, 0])


def test_invalid_arguments_raise(gpu_lib):
    wl, orc, x = _random_batch(8, S=2, seed=12)
    planner, batch = gpu_side(wl)
    with pytest.raises(B.DseedError):
        B.cost(planner.robot, batch.desc, batch.pr, _cuda(x).double())
    d = B.plan_desc(wl.P, wl.S, wl.T, I.CostParams(dt=0.0))
    with pytest.raises(B.DseedError, match="dt"):
        B.cost(planner.robot, d, batch.pr, _cuda(x))


def test_lipschitz_early_out_is_exact(gpu_lib):
    """Skipping the interpolation of spheres whose nearest voxel proves the hinge
    inactive must not change a single bit of cost, gradient or plan."""
    wl, orc = oracle_workload("batched", n_scenes=4, n_problems=4, S=16, iters=30)
    planner, batch = gpu_side(wl)
    rng = np.random.default_rng(4)
    x = np.stack([I.random_trajectories(rng, wl.q_start[p], wl.S, wl.T, wl.robot.limits) for p in range(wl.P)])
    c1, g1 = B.cost_grad(planner.robot, batch.desc, batch.pr, _cuda(x))
    out1 = {k: v.clone() for k, v in planner.plan(batch, wl.seeds).items()}
    off = B.SceneTable(planner.esdfs, planner.grids, lipschitz=0.0)
    batch0 = api.Batch(wl.q_start, wl.goal, wl.scene_of_problem, off, wl.S, wl.T, wl.cost, wl.opt)
    c0, g0 = B.cost_grad(planner.robot, batch0.desc, batch0.pr, _cuda(x))
    out0 = B.plan_batch(planner.robot, batch0.desc, batch0.pr, _cuda(wl.seeds), planner.workspace(batch0))
    assert torch.equal(c0, c1) and torch.equal(g0, g1)
    for k in ("traj", "cost", "success", "best"):
        assert torch.equal(out0[k], out1[k]), k
