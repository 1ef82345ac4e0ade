"""The attempts loop on the GPU planner (api.planner_attempts, Sec. 5.2):
attempt 1 is the one-shot plan of its seeds, later attempts only re-plan the
unsolved problems with new seeds, and a returned trajectory passes the
success test."""
import numpy as np
import pytest
import torch

from gpu_helpers import gpu_side, oracle_workload, to_np
from paper_2410_16727_gb300 import api, binding as B, inputs as I

pytestmark = pytest.mark.gpu


def test_attempts_on_the_planner(gpu_lib):
    # a small budget (4 seeds, 8 iterations) leaves problems unsolved after one attempt
    wl, _ = oracle_workload("tiny", n_scenes=4, n_problems=24, S=4, T=32, iters=8)
    planner, batch = gpu_side(wl, opt=I.OptParams(iters=8))

    def seed_fn(attempt, problems):
        if attempt == 1:
            return wl.seeds[problems]
        # a new batch of the plain method's seeds
        return np.stack([I.make_seeds(np.random.default_rng(1000 * attempt + int(p)), wl.q_start[p], wl.q_goal[p],
                                      wl.S, wl.T, wl.robot.limits) for p in problems]).astype(np.float32)

    one = api.planner_attempts(planner, wl.q_start, wl.goal, wl.scene_of_problem, seed_fn, wl.S, wl.T, 1)
    ref = planner.plan(batch, torch.as_tensor(wl.seeds).cuda())
    best = to_np(ref["best"])
    np.testing.assert_array_equal(one["solved"], best >= 0)
    for p in np.nonzero(best >= 0)[0]:
        np.testing.assert_array_equal(one["traj"][p], to_np(ref["traj"])[p, best[p]])
    assert 0 < one["solved"].mean() < 1, "the case should leave problems for later attempts"

    many = api.planner_attempts(planner, wl.q_start, wl.goal, wl.scene_of_problem, seed_fn, wl.S, wl.T, 6)
    assert (many["solved"] >= one["solved"]).all() and many["solved"].sum() > one["solved"].sum()
    np.testing.assert_array_equal(many["attempts"][one["solved"]], 1)
    # every returned trajectory passes the success test on its own
    idx = np.nonzero(many["solved"])[0]
    b1 = planner.batch(wl.q_start[idx], wl.goal[idx], wl.scene_of_problem[idx], 1, wl.T)
    ok, _ = B.evaluate(planner.robot, b1.desc, b1.pr, torch.as_tensor(many["traj"][idx][:, None]).cuda())
    assert to_np(ok).all()
