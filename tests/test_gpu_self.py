"""GPU parity of the self-collision term (C_self) against the FP64 oracle:
the checked-pair set, a two-sphere closed form, cost and gradient on
trajectories with self contact (one and two waypoints per lane), the success
metrics, plans, and the serving loop with the term."""
import dataclasses

import numpy as np
import pytest
import torch

import oracle
from golden.read import read
from gpu_helpers import check_success_agreement, rel_l2, to_np
from paper_2410_16727_gb300 import api, binding as B, inputs as I

pytestmark = pytest.mark.gpu

COST = dataclasses.replace(I.CostParams(), w_self=100.0, eta_self=0.01)


def _cuda(a):
    return torch.as_tensor(np.ascontiguousarray(a, np.float32)).cuda()


def _tiny(n_problems):
    spec = I.WORKLOADS["tiny"]
    cub, grids = I.make_scenes(spec)
    orc = oracle.Oracle(I.make_robot(), COST, grids, cub, T=32)
    wl = I.build_workload(spec, cub, grids, orc.clearance, orc.flange_pose, n_problems=n_problems)
    return wl, orc


@pytest.fixture(scope="module")
def tiny():
    return _tiny(8)


@pytest.fixture(scope="module")
def tiny32():
    return _tiny(32)


def _gpu(wl, T=None, S=None):
    planner = api.Planner(wl.robot, COST, wl.opt)
    planner.set_scenes(wl.cuboids, wl.grids)
    batch = planner.batch(wl.q_start, wl.goal, wl.scene_of_problem, S or wl.S, T or wl.T)
    return planner, batch


def test_pair_set_matches_oracle(gpu_lib, tiny):
    wl, orc = tiny
    mask = B.Robot(wl.robot).self_pairs()
    assert np.array_equal(mask, orc.self_mask)


def test_two_sphere_closed_form(gpu_lib):
    gold = read("franka_fk.txt")
    r = 0.35
    robot = dataclasses.replace(I.make_robot(), sph_frame=np.array([1, 8], np.int32),
                                sph_o=np.zeros((2, 3), np.float32), sph_r=np.array([r, r], np.float32),
                                self_margin=-10.0)
    only = I.CostParams(w_c=0.0, w_v=0.0, w_a=0.0, w_j=0.0, w_p=0.0, w_R=0.0, w_l=0.0, w_self=100.0)
    planner = api.Planner(robot, only)
    spec = I.WORKLOADS["tiny"]
    planner.set_scenes([np.zeros((0, 6), np.float32)], [spec.grid])
    q0 = np.zeros((1, 7), np.float32)
    batch = planner.batch(q0, np.array([[0, 0, 0, 1, 0, 0, 0]], np.float32), np.zeros(1, np.int32), 1, 1)
    c, g = B.cost_grad(planner.robot, batch.desc, batch.pr, _cuda(q0.reshape(1, 1, 1, 7)))
    d = float(np.linalg.norm(gold["zero_flange_p"] - gold["zero_origin_1"]))
    want = only.w_self * (2 * float(np.float32(r)) + only.eta_self - d)
    assert abs(float(c[0, 0]) - want) <= 1e-4 * want
    assert abs(float(g[0, 0, 0, 0])) <= 1e-4


@pytest.mark.parametrize("T", [32, 48])
def test_cost_and_gradient_match_oracle(gpu_lib, tiny, T):
    wl, orc = tiny
    rng = np.random.default_rng(T)
    planner, batch = _gpu(wl, T=T, S=16)
    x = np.stack([I.random_trajectories(rng, wl.q_start[p], 16, T, wl.robot.limits, spread=1.5)
                  for p in range(wl.P)]).astype(np.float32)
    c, g = B.cost_grad(planner.robot, batch.desc, batch.pr, _cuda(x))
    c, g = to_np(c), to_np(g)
    n_self = 0
    for p in range(wl.P):
        wc, wg, terms = orc.cost(int(wl.scene_of_problem[p]), wl.q_start[p], wl.goal[p], x[p], grad=True,
                                 terms=True)
        # the oracle's collision term with the self term off, to count trajectories in self contact
        for s in range(16):
            assert abs(c[p, s] - wc[s]) <= 1e-4 * max(abs(wc[s]), 1e-6), (p, s, c[p, s], wc[s])
            assert rel_l2(g[p, s], wg[s]) <= 1e-3, (p, s)
        n_self += int((terms[:, 0] > 0).sum())
    assert n_self > 16


def test_evaluate_matches_oracle(gpu_lib, tiny):
    wl, orc = tiny
    rng = np.random.default_rng(5)
    planner, batch = _gpu(wl, S=8)
    x = np.stack([I.random_trajectories(rng, wl.q_start[p], 8, wl.T, wl.robot.limits, spread=1.5)
                  for p in range(wl.P)]).astype(np.float32)
    ok, met = B.evaluate(planner.robot, batch.desc, batch.pr, _cuda(x))
    met = to_np(met)
    for p in range(wl.P):
        wok, wmet = orc.evaluate(int(wl.scene_of_problem[p]), wl.q_start[p], wl.goal[p], x[p])
        assert np.abs(met[p, :, 0] - wmet[:, 0]).max() <= 1e-4          # min clearance incl. self pairs
        far = np.abs(wmet[:, 0]) > 1e-3
        assert np.array_equal(to_np(ok)[p][far].astype(bool), wok[far])


@pytest.mark.parametrize("iters", [1, 5, 10])
def test_plan_first_iterations_follow_oracle(gpu_lib, tiny, iters):
    wl, orc = tiny
    opt = dataclasses.replace(wl.opt, iters=iters)
    planner = api.Planner(wl.robot, COST, opt)
    planner.set_scenes(wl.cuboids, wl.grids)
    out = planner.plan(planner.batch(wl.q_start, wl.goal, wl.scene_of_problem, wl.S, wl.T), wl.seeds)
    ref = orc.plan(wl.scene_of_problem, wl.q_start, wl.goal, wl.seeds, opt)
    rel = np.abs(to_np(out["cost"]) - ref["cost"]) / np.maximum(ref["cost"], 1e-6)
    tol = 1e-4 if iters == 1 else 1e-3
    assert np.quantile(rel, 0.95) <= tol and rel.max() <= 10 * tol, (np.quantile(rel, 0.95), rel.max())


def test_plan_agrees_with_oracle(gpu_lib, tiny32):
    """100 iterations on 32 problems x 32 seeds (1024 seeds).  The FP32 and FP64
    runs follow each other to ~1e-6 relative cost for the first iterations
    (previous test) and part ways by millimetres later on some seeds.  Success
    flags agree on >= 99% of the seeds, every seed on which they differ ends
    near a success threshold on one side (clearance within 5 mm of zero with
    the self pairs included, or just beyond a soft joint limit), and every seed
    away from the thresholds agrees."""
    wl, orc = tiny32
    planner, batch = _gpu(wl)
    out = planner.plan(batch, wl.seeds)
    ok = to_np(out["success"]).astype(bool)
    met = to_np(out["metrics"])
    ref = orc.plan(wl.scene_of_problem, wl.q_start, wl.goal, wl.seeds, wl.opt)
    agree, near, _ = check_success_agreement(ok, met, ref["success"], ref["metrics"], 0.99, to_np(out["traj"]),
                                             ref["traj"])
    assert near < 0.6
    both = ok & ref["success"]
    if both.any():
        rel = np.abs(to_np(out["cost"])[both] - ref["cost"][both]) / ref["cost"][both]
        assert np.median(rel) < 2e-2
    # successful plans are free of self-collision (the clearance includes the checked pairs)
    assert (met[ok][:, 0] >= 0).all()
    # the GPU's success test is the oracle's: the FP64 evaluation of the GPU's own trajectories
    traj = to_np(out["traj"])
    for p in range(wl.P):
        want, wmet = orc.evaluate(int(wl.scene_of_problem[p]), wl.q_start[p], wl.goal[p], traj[p])
        far = np.abs(wmet[:, 0]) > 1e-5
        assert np.array_equal(ok[p][far], want[far])


def test_server_serves_self_term(gpu_lib, tiny):
    """Served requests with the self-collision term compute what the one-shot
    plan computes for them (one and two waypoints per lane, rounds of 7 of 30
    iterations), and the term is active on them."""
    wl, orc = tiny
    from paper_2410_16727_gb300 import serving as SV
    opt = I.OptParams(iters=30)
    planner = api.Planner(wl.robot, COST, opt)
    planner.set_scenes(wl.cuboids, wl.grids)
    sv = SV.Server(wl.robot, 256 << 20, max_requests=16, round_iters=7, cost=COST, opt=opt)
    for s, (c, g) in enumerate(zip(wl.cuboids, wl.grids)):
        sv.add_scene(s, c, g)
    rng = np.random.default_rng(11)
    cases, tickets = [], []
    for p, (S, T) in enumerate([(8, 32), (4, 48), (6, 64)]):
        x = I.random_trajectories(rng, wl.q_start[p], S, T, wl.robot.limits, spread=1.5).astype(np.float32)
        cases.append((p, x))
        tickets.append(sv.submit(int(wl.scene_of_problem[p]), wl.q_start[p], wl.goal[p], x))
    sv.drain(tickets)
    n_self = 0
    for t, (p, x) in zip(tickets, cases):
        assert sv.poll(t)[0] == 2
        got = sv.result(t)
        batch = planner.batch(wl.q_start[p:p + 1], wl.goal[p:p + 1], np.array([wl.scene_of_problem[p]], np.int32),
                              x.shape[0], x.shape[1])
        want = {k: to_np(v)[0] for k, v in planner.plan(batch, x[None]).items()}
        np.testing.assert_allclose(got["traj"].numpy(), want["traj"], rtol=1e-5, atol=1e-5)
        np.testing.assert_allclose(got["cost"].numpy(), want["cost"], rtol=1e-5, atol=1e-5)
        assert (got["success"].numpy() == want["success"]).all()
        assert int(got["best"][0]) == int(want["best"])
        # the seeds start with an active collision term (world and self)
        _, _, terms = orc.cost(int(wl.scene_of_problem[p]), wl.q_start[p], wl.goal[p], x, grad=True, terms=True)
        n_self += int((terms[:, 0] > 0).sum())
    assert n_self > 0
    sv.close()
