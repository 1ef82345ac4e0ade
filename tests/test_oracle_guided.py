"""Pins of the oracle's cost-guided DDIM sampler (the appendix's Eq. 5, read
for a deterministic sampler: after each denoising step that reaches a step
index below k, except the last, n capped descent steps on the plan cost).

Fixed by the mathematics, not by the oracle's own formulas: the squared-cosine
schedule's closed form where no step is capped; a zero noise prediction makes
every DDIM step a rescaling, so the sampler ends at clip(noise / sqrt(abar)) of
its first step; one descent step with a small alpha moves along minus the
gradient of x -> C(decoded x), checked by central differences of the C
oracle's cost; a huge alpha saturates every entry at the cap; the number of
descent phases follows from the step schedule (counted by hand below)."""
import math

import numpy as np
import pytest

import oracle
from oracle import denoiser_oracle as DO
from paper_2410_16727_gb300 import inputs as I, netspec as NS

ROBOT = I.make_robot()
RES = 4.0
T = 6


def _problem(N=3, seed=0, cuboids=np.zeros((0, 6), np.float32)):
    rng = np.random.default_rng(seed)
    qs = I.sample_configs(rng, ROBOT.limits, N).astype(np.float64)
    qg = I.sample_configs(rng, ROBOT.limits, N).astype(np.float64)
    goal = oracle.flange_pose(ROBOT.dh, qg)
    grid = I.WORKLOADS["tiny"].grid
    orc = oracle.Oracle(ROBOT, I.CostParams(), [grid], [cuboids], T=T)

    def cost_grad(q):
        return np.stack([orc.cost(0, qs[n], goal[n], q[n][None])[1][0] for n in range(q.shape[0])])

    def cost(q):
        return np.array([orc.cost(0, qs[n], goal[n], q[n][None], grad=False)[0] for n in range(q.shape[0])])

    lin = DO.straight_path(DO.normalise_joints(ROBOT.limits, qs), DO.normalise_joints(ROBOT.limits, qg), T)
    return qs, qg, goal, lin, cost, cost_grad


def test_cosine_schedule_closed_form():
    K, s = 100, 0.008
    abar = DO.cosine_abar(K, s)
    f = lambda t: math.cos(math.pi / 2 * (t / K + s) / (1 + s)) ** 2
    # where no beta reached its cap, abar_k = f(k + 1) / f(0)
    for k in range(K - 2):
        assert abs(abar[k] - f(k + 1) / f(0)) < 1e-12
    assert np.all(np.diff(abar) < 0) and 0 < abar[-1] < abar[0] < 1


@pytest.mark.parametrize("steps", [2, 5, 10])
def test_eps_free_ddim_is_a_rescaling(steps):
    spec = NS.NetSpec(T=T)
    abar = DO.cosine_abar(spec.K)
    qs, qg, goal, lin, cost, cost_grad = _problem()
    rng = np.random.default_rng(steps)
    for scale in (1.0, 1e-3 * math.sqrt(abar[-1])):       # clipped and unclipped
        noise = rng.normal(size=(3, T, 7)) * scale
        _, x = DO.guided_ddim(spec, None, noise, qs, qg, goal, None, ROBOT.limits, RES, abar, steps, 2.0,
                              60, 20, 0.0, 0.02, cost_grad, eps_fn=lambda x, k: np.zeros_like(x))
        np.testing.assert_allclose(x, np.clip(noise / math.sqrt(abar[spec.K - 1]), -2.0, 2.0), rtol=1e-12,
                                   atol=1e-15)


def test_descent_step_follows_the_decoded_cost_gradient():
    box = np.array([[0.3, 0.0, 0.5, 0.1, 0.2, 0.3]], np.float32)
    qs, qg, goal, lin, cost, cost_grad = _problem(N=2, seed=3, cuboids=box)
    rng = np.random.default_rng(4)
    x0 = rng.normal(size=(2, T, 7)) * 0.3
    alpha = 1e-9
    x1 = DO.guided_descent(x0, lin, ROBOT.limits, RES, 1, alpha, np.inf, cost_grad)
    g = (x1 - x0) / -alpha                       # the step's gradient in the diffused space
    h = 1e-6
    decoded_cost = lambda x: cost(DO.decode_joints(ROBOT.limits, lin, x, RES))
    for n in range(2):
        for idx in [(1, 2), (3, 0), (5, 6), (0, 4)]:
            xp, xm = x0.copy(), x0.copy()
            xp[(n,) + idx] += h
            xm[(n,) + idx] -= h
            fd = (decoded_cost(xp)[n] - decoded_cost(xm)[n]) / (2 * h)
            assert abs(g[(n,) + idx] - fd) <= 1e-5 * max(1.0, abs(fd)), (n, idx, g[(n,) + idx], fd)


def test_descent_step_is_capped_per_entry():
    qs, qg, goal, lin, cost, cost_grad = _problem(N=2, seed=5)
    x0 = np.random.default_rng(6).normal(size=(2, T, 7)) * 0.3
    g = cost_grad(DO.decode_joints(ROBOT.limits, lin, x0, RES))
    x1 = DO.guided_descent(x0, lin, ROBOT.limits, RES, 1, 1e9, 0.02, cost_grad)
    moved = g != 0
    np.testing.assert_allclose((x1 - x0)[moved], -0.02 * np.sign(g[moved]), rtol=0, atol=1e-15)
    # and with a small alpha the guided cost goes down
    x5 = DO.guided_descent(x0, lin, ROBOT.limits, RES, 5, 1e-4, 0.02, cost_grad)
    dec = lambda x: DO.decode_joints(ROBOT.limits, lin, x, RES)
    assert np.all(cost(dec(x5)) < cost(dec(x0)))


@pytest.mark.parametrize("steps, phases", [(5, 3), (10, 6), (2, 1)])
def test_descent_phases_follow_the_schedule(steps, phases):
    # steps = 5 over K = 100: indices 99, 74, 50, 25, 0; the steps reaching 50, 25 and 0
    # are below k = 60, and the step reaching 0 is not the last one (that one ends at abar = 1):
    # 3 phases.  steps = 10: 99, 88, ..., 11, 0 -> reaching 55, 44, 33, 22, 11, 0: 6 phases.
    # steps = 2: 99, 0 -> the first step reaches 0 and is not the last: 1 phase.
    spec = NS.NetSpec(T=T)
    qs, qg, goal, lin, cost, cost_grad = _problem()
    calls = []

    def counting(q):
        calls.append(1)
        return np.zeros_like(q)

    DO.guided_ddim(spec, None, np.zeros((3, T, 7)), qs, qg, goal, None, ROBOT.limits, RES,
                   DO.cosine_abar(spec.K), steps, 2.0, 60, 7, 1.0, 0.02, counting,
                   eps_fn=lambda x, k: np.zeros_like(x))
    assert len(calls) == 7 * phases


def test_schedule_matches_the_samplers():
    # the CUDA path's schedule (a table it computes for itself) equals the definition
    from paper_2410_16727_gb300 import denoiser as DN
    np.testing.assert_allclose(DN.cosine_abar(100), DO.cosine_abar(100), rtol=1e-13, atol=0)
