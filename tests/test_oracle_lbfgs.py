"""Pins of the oracle's L-BFGS: a convex quadratic must converge to the direct
solution of its linear system, and a trajectory optimisation must never accept
a point of higher cost."""
import numpy as np

import oracle
from paper_2410_16727_gb300 import inputs as I


def test_quadratic_converges_to_linear_solve():
    rng = np.random.default_rng(0)
    n = 60
    Q, _ = np.linalg.qr(rng.normal(size=(n, n)))
    A = Q @ np.diag(np.linspace(1.0, 50.0, n)) @ Q.T
    b = rng.normal(size=n)
    x_star = np.linalg.solve(A, b)
    opt = I.OptParams(iters=400, max_step=10.0)
    x, f, trace, acc = oracle.lbfgs_quadratic(A, b, np.zeros(n), opt)
    assert np.abs(x - x_star).max() < 1e-8
    assert abs(f - (-0.5 * b @ x_star)) < 1e-10
    assert np.all(np.diff(trace) <= 1e-12)


def test_quadratic_step_cap_and_history_one():
    # m = 1 and a tight step cap still converge, only more slowly
    rng = np.random.default_rng(1)
    n = 14
    M = rng.normal(size=(n, n))
    A = M @ M.T + n * np.eye(n)
    b = rng.normal(size=n) * 3
    opt = I.OptParams(iters=3000, m=1, max_step=0.05)
    x, f, trace, acc = oracle.lbfgs_quadratic(A, b, np.ones(n), opt)
    np.testing.assert_allclose(x, np.linalg.solve(A, b), atol=1e-8)


def test_plan_accepts_only_descent_and_reports_final_cost():
    spec = I.WORKLOADS["tiny"]
    cub, grids = I.make_scenes(spec)
    orc = oracle.Oracle(I.make_robot(), I.CostParams(), grids, cub, T=16)
    wl = I.build_workload(spec, cub, grids, orc.clearance, orc.flange_pose, S=4, T=16, iters=40)
    out = orc.plan(wl.scene_of_problem, wl.q_start, wl.goal, wl.seeds, wl.opt, trace=True)
    tr = out["trace"]
    assert np.all(np.diff(tr, axis=-1) <= 1e-12)
    f = orc.cost(0, wl.q_start[0], wl.goal[0], out["traj"][0], grad=False)
    np.testing.assert_allclose(f, out["cost"][0], rtol=1e-12)
    # the optimiser makes progress from the seeds
    f0 = orc.cost(0, wl.q_start[0], wl.goal[0], wl.seeds[0], grad=False)
    assert (out["cost"][0] < f0).all()
