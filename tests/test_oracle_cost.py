"""Pins of the oracle's cost terms and gradient.

Each term is checked against a value fixed by the mathematics rather than by
retyping the oracle: finite differences of a cubic, a pose error of known size,
a sphere in the affine face region of a box, a joint a known distance beyond its
limit; the full gradient against central differences."""
import math

import numpy as np
import pytest

import oracle
from paper_2410_16727_gb300 import inputs as I

ROBOT = I.make_robot()
EMPTY = np.zeros((0, 6), np.float32)
GRID = I.WORKLOADS["tiny"].grid


def _orc(cost, cuboids=EMPTY, robot=ROBOT, grid=GRID, T=8):
    return oracle.Oracle(robot, cost, [grid], [cuboids], T=T)


def test_smoothness_exact_on_cubic():
    T, dt = 12, 0.05
    cp = I.CostParams(w_p=0.0, w_R=0.0, w_l=0.0)
    c = np.array([0.3, -0.2, 0.5, 0.1, -0.4, 0.25, 0.05])
    t = np.arange(1, T + 1)[:, None]
    x = c[None, :] * (t * dt) ** 3
    orc = _orc(cp, T=T)
    f, _, terms = orc.cost(0, np.zeros(7), [0, 0, 0, 1, 0, 0, 0], x[None], grad=True, terms=True)
    # closed forms of the backward differences of y_t = c (t dt)^3 with y_0 = y_-1 = y_-2 = 0
    tt = np.arange(1, T + 1, dtype=np.float64)[:, None]
    v = c * dt ** 2 * (3 * tt ** 2 - 3 * tt + 1)
    a = np.where(tt >= 2, c * dt * (6 * tt - 6), c * dt)
    j = np.where(tt >= 3, 6 * c, np.where(tt == 2, 5 * c, c))
    want = (cp.w_v * v ** 2 + cp.w_a * a ** 2 + cp.w_j * j ** 2).sum()
    assert abs(terms[0, 1] - want) < 1e-12 * max(1.0, want)
    assert terms[0, 0] == 0.0 and terms[0, 2] == 0.0 and terms[0, 3] == 0.0
    # the evaluation's max-jerk metric sees the interior value 6c
    _, met = orc.evaluate(0, np.zeros(7), [0, 0, 0, 1, 0, 0, 0], x[None])
    assert abs(met[0, 3] - 6 * np.abs(c).max()) < 1e-9


def test_linear_trajectory_has_no_interior_acceleration():
    T = 10
    cp = I.CostParams(w_v=0.0, w_j=0.0, w_p=0.0, w_R=0.0, w_l=0.0)
    qs = np.array([0.1, 0.2, -0.3, -1.0, 0.0, 1.0, 0.3])
    step = np.array([0.01, -0.02, 0.03, 0.0, 0.05, -0.01, 0.02])
    x = qs[None, :] + np.arange(1, T + 1)[:, None] * step[None, :]
    _, terms = _orc(cp, T=T).cost(0, qs, [0, 0, 0, 1, 0, 0, 0], x[None], grad=False, terms=True)
    # only a_1 = step / dt^2 is non-zero (the start is held at rest)
    want = cp.w_a * ((step / cp.dt ** 2) ** 2).sum()
    assert abs(terms[0, 1] - want) < 1e-12 * want


def _quat_mul(a, b):
    w1, v1 = a[0], np.asarray(a[1:])
    w2, v2 = b[0], np.asarray(b[1:])
    return np.concatenate([[w1 * w2 - v1 @ v2], w1 * v2 + w2 * v1 + np.cross(v1, v2)])


def test_goal_cost_zero_at_goal_and_closed_forms():
    rng = np.random.default_rng(0)
    T = 4
    cp = I.CostParams(w_c=0.0, w_v=0.0, w_a=0.0, w_j=0.0, w_l=0.0)
    orc = _orc(cp, T=T)
    for _ in range(5):
        qg = I.sample_configs(rng, ROBOT.limits, 1)[0]
        qs = I.sample_configs(rng, ROBOT.limits, 1)[0]
        x = np.tile(qg.astype(np.float64), (T, 1))
        pose = oracle.flange_pose(ROBOT.dh, qg)[0]
        f, g, terms = orc.cost(0, qs, pose, x[None], grad=True, terms=True)
        assert terms[0, 2] < 1e-20
        assert np.abs(g).max() < 1e-8
        # a goal displaced by d and rotated by theta about a unit axis
        d = rng.normal(size=3) * 0.05
        axis = rng.normal(size=3)
        axis /= np.linalg.norm(axis)
        theta = rng.uniform(0.05, 2.5)
        qrot = np.concatenate([[math.cos(theta / 2)], math.sin(theta / 2) * axis])
        goal = np.concatenate([pose[:3] + d, _quat_mul(pose[3:], qrot)])
        _, terms = orc.cost(0, qs, goal, x[None], grad=False, terms=True)
        want = cp.w_p * (d @ d) + cp.w_R * math.sin(theta / 2) ** 2
        assert abs(terms[0, 2] - want) < 1e-9 * max(1.0, want)
        # and the evaluation reports the displacement and the angle
        _, met = orc.evaluate(0, qs, goal, x[None])
        assert abs(met[0, 1] - np.linalg.norm(d)) < 1e-12
        assert abs(met[0, 2] - min(theta, 2 * math.pi - theta)) < 1e-7
        # goal quaternions are taken up to sign and scale (normalised on entry,
        # q and -q one rotation): the same closed forms hold for -2.5 q and 0.3 q
        for f in (-2.5, 0.3):
            goal_f = np.concatenate([goal[:3], f * goal[3:]])
            _, terms_f = orc.cost(0, qs, goal_f, x[None], grad=False, terms=True)
            assert abs(terms_f[0, 2] - want) < 1e-9 * max(1.0, want)
            _, met_f = orc.evaluate(0, qs, goal_f, x[None])
            assert abs(met_f[0, 2] - min(theta, 2 * math.pi - theta)) < 1e-7


def test_world_hinge_on_affine_face_region():
    # one sphere of radius 0.06 on the flange origin; at q = 0 the flange sits at
    # (0.088, 0, 0.926).  A large box whose -x face is 5 cm further along +x.
    r = I.make_robot()
    r.sph_frame = np.array([8], np.int32)
    r.sph_o = np.zeros((1, 3), np.float32)
    r.sph_r = np.array([0.06], np.float32)
    face = 0.138
    box = np.array([[face + 0.3, 0.0, 0.926, 0.3, 0.5, 0.5]], np.float32)
    grid = I.Grid((-0.2, -0.5, 0.5), 0.02, (40, 50, 40))
    cp = I.CostParams(w_v=0.0, w_a=0.0, w_j=0.0, w_p=0.0, w_R=0.0, w_l=0.0)
    T = 3
    orc = _orc(cp, box, robot=r, grid=grid, T=T)
    x = np.zeros((1, T, 7))
    f, g, terms = orc.cost(0, np.zeros(7), [0, 0, 0, 1, 0, 0, 0], x, grad=True, terms=True)
    hinge = 0.06 + cp.eta - (face - 0.088)
    assert abs(terms[0, 0] - T * cp.w_c * hinge) < 1e-5
    ok, met = orc.evaluate(0, np.zeros(7), [0.088, 0, 0.926, 0, 1, 0, 0], x)
    assert abs(met[0, 0] - ((face - 0.088) - 0.06)) < 1e-6
    assert met[0, 6] == 0.0 and not ok[0]   # the sphere reaches 1 cm into the box
    # dC/dc = -w_c grad(phi) = (+w_c, 0, 0): each joint contributes w_c times the
    # x component of its velocity at the flange, z_i x (p_flange - p_i)
    F = oracle.fk_frames(r.dh, np.zeros(7))
    for i in range(1, 8):
        z, p = F[i][:3, 2], F[i][:3, 3]
        J = np.cross(z, F[8][:3, 3] - p)
        want = cp.w_c * J[0]
        np.testing.assert_allclose(g[0, :, i - 1], want, atol=1e-6)


def test_joint_limit_penalty_closed_form():
    T = 5
    cp = I.CostParams(w_c=0.0, w_v=0.0, w_a=0.0, w_j=0.0, w_p=0.0, w_R=0.0)
    lim = ROBOT.limits.astype(np.float64)
    mid = lim.mean(axis=1)
    x = np.tile(mid, (T, 1))
    x[2, 3] = lim[3, 1] + 0.1
    x[4, 0] = lim[0, 0] - 0.2
    f, g, terms = _orc(cp, T=T).cost(0, mid, [0, 0, 0, 1, 0, 0, 0], x[None], grad=True, terms=True)
    assert abs(terms[0, 3] - cp.w_l * (0.1 ** 2 + 0.2 ** 2)) < 1e-9
    assert abs(g[0, 2, 3] - 2 * cp.w_l * 0.1) < 1e-6
    assert abs(g[0, 4, 0] + 2 * cp.w_l * 0.2) < 1e-6


def _fd_check(orc, qs, goal, x, h=1e-6, kink=0.05):
    f0, g, = orc.cost(0, qs, goal, x[None], grad=True)
    g = g[0].reshape(-1)
    flat = x.reshape(-1).astype(np.float64)
    fd = np.zeros_like(flat)
    smooth = np.ones(flat.size, bool)
    for i in range(flat.size):
        xp, xm = flat.copy(), flat.copy()
        xp[i] += h
        xm[i] -= h
        fp = orc.cost(0, qs, goal, xp.reshape(x.shape)[None], grad=False)[0]
        fm = orc.cost(0, qs, goal, xm.reshape(x.shape)[None], grad=False)[0]
        fd[i] = (fp - fm) / (2 * h)
        # a hinge kink or cell face between x-h and x+h shows as unequal one-sided slopes
        smooth[i] = abs((fp - f0[0]) / h - (f0[0] - fm) / h) < kink
    return g, fd, smooth


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_gradient_matches_central_differences(seed):
    rng = np.random.default_rng(100 + seed)
    T = 6
    cub = I.scene_tiny(np.random.default_rng(seed))
    orc = _orc(I.CostParams(), cub, T=T)
    qs = I.sample_configs(rng, ROBOT.limits, 1)[0]
    qg = I.sample_configs(rng, ROBOT.limits, 1)[0]
    goal = oracle.flange_pose(ROBOT.dh, qg)[0]
    x = I.random_trajectories(rng, qs, 1, T, ROBOT.limits, spread=1.5)[0].astype(np.float64)
    # push a few entries beyond the limits so the limit term is exercised
    x[1, 3] = float(ROBOT.limits[3, 1]) + 0.05
    g, fd, smooth = _fd_check(orc, qs, goal, x)
    assert smooth.mean() > 0.9
    err = np.abs(g - fd)[smooth]
    assert err.max() <= 1e-5 * max(1.0, np.abs(g).max()), err.max()
    _, terms = orc.cost(0, qs, goal, x[None], grad=False, terms=True)
    assert terms[0, 0] > 0.0, "case should have active collision terms"


def test_gradient_dense_clutter_collisions():
    rng = np.random.default_rng(77)
    T = 4
    cub = I.scene_clutter(np.random.default_rng(5), n_boxes=60, side=(0.05, 0.2))
    orc = _orc(I.CostParams(), cub, T=T)
    qs = I.sample_configs(rng, ROBOT.limits, 1)[0]
    x = I.random_trajectories(rng, qs, 1, T, ROBOT.limits)[0].astype(np.float64)
    goal = oracle.flange_pose(ROBOT.dh, x[-1])[0]
    goal[:3] += 0.03
    g, fd, smooth = _fd_check(orc, qs, goal, x)
    assert smooth.mean() > 0.85
    err = np.abs(g - fd)[smooth]
    assert err.max() <= 1e-5 * max(1.0, np.abs(g).max())
