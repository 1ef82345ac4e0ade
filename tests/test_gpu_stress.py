"""Stress workload at full size in the benchmark's launch configuration:
1024 problems x 128 seeds x 64 waypoints, 200 iterations, dense-clutter scenes
of 200 cuboids with 256^3 ESDFs at 5 mm, one plan call.  The FP64 oracle
re-plans a 1% sample of the seeds.  The problems share two scenes instead of
sixteen: the oracle's brute-force ESDF build of a 256^3, 200-cuboid scene takes
seconds, and two keep the test short without changing the per-seed work."""
import numpy as np
import pytest
import torch

from gpu_helpers import check_success_agreement, gpu_side, oracle_workload, rel_l2, to_np
from paper_2410_16727_gb300 import binding as B

pytestmark = pytest.mark.gpu

AGREE = 0.99


@pytest.fixture(scope="module")
def stress():
    return oracle_workload("stress", n_scenes=2)


def test_stress_plan_sampled_parity(gpu_lib, stress):
    wl, orc = stress
    assert (wl.P, wl.S, wl.T, wl.opt.iters) == (1024, 128, 64, 200)
    planner, batch = gpu_side(wl)
    out = planner.plan(batch, wl.seeds)
    torch.cuda.synchronize()
    ok = to_np(out["success"]).astype(bool)
    cost = to_np(out["cost"])
    rng = np.random.default_rng(5)
    flat = rng.choice(wl.P * wl.S, size=(wl.P * wl.S) // 100, replace=False)
    p_idx, s_idx = np.divmod(flat, wl.S)
    ref = orc.plan(wl.scene_of_problem[p_idx], wl.q_start[p_idx], wl.goal[p_idx],
                   wl.seeds[p_idx, s_idx][:, None], wl.opt)
    ref_ok = ref["success"][:, 0]
    check_success_agreement(ok[p_idx, s_idx], to_np(out["metrics"])[p_idx, s_idx], ref_ok, ref["metrics"][:, 0],
                            AGREE, to_np(out["traj"])[p_idx, s_idx], ref["traj"][:, 0])
    both = ok[p_idx, s_idx] & ref_ok
    rel = np.abs(cost[p_idx, s_idx][both] - ref["cost"][both, 0]) / ref["cost"][both, 0]
    assert np.median(rel) < 1e-2
    assert ok.mean() > 0.3            # the clutter is hard, but the optimiser solves a good share


def test_stress_cost_grad_sampled(gpu_lib, stress):
    """Cost and gradient of the seeds themselves (T = 64, two waypoints per
    lane) on a 0.1% sample, against the oracle within the parity tolerances."""
    wl, orc = stress
    planner, batch = gpu_side(wl)
    c, g = B.cost_grad(planner.robot, batch.desc, batch.pr,
                       torch.as_tensor(np.ascontiguousarray(wl.seeds)).cuda())
    c, g = to_np(c), to_np(g)
    rng = np.random.default_rng(8)
    for f in rng.choice(wl.P * wl.S, size=(wl.P * wl.S) // 1000, replace=False):
        p, s = divmod(int(f), wl.S)
        wc, wg = orc.cost(int(wl.scene_of_problem[p]), wl.q_start[p], wl.goal[p], wl.seeds[p, s:s + 1])
        assert abs(c[p, s] - wc[0]) <= 1e-4 * max(abs(wc[0]), 1e-6)
        assert rel_l2(g[p, s], wg[0]) <= 1e-3
