"""Pins of the oracle's success decision and best-seed pick.

A plan succeeds (Sec. 5.1) when its final flange lies within delta_t = 5 mm of
the goal position and within delta_r = 2.86 degrees of the goal orientation, no
collision sphere reaches into an obstacle at any waypoint, and every waypoint
respects the joint limits; the plan a problem returns is its lowest-cost
successful seed, the lowest index among equal costs, none (-1) when no seed
succeeds.  The thresholds come from the cited fixture
``tests/golden/success_thresholds.txt``.  Each case sits just inside or just
outside one threshold, so a degrees/radians slip, swapped thresholds, ``<=`` for
``<``, a margin on the limits or clearance, or a wrong tie-break fails a named
test here."""
import math

import numpy as np
import pytest

import oracle
from paper_2410_16727_gb300 import inputs as I
from golden.read import read

ROBOT = I.make_robot()
EMPTY = np.zeros((0, 6), np.float32)
GRID = I.WORKLOADS["tiny"].grid
T = 4
GOLD = read("success_thresholds.txt")
DELTA_T = float(GOLD["delta_t_m"][0])
DELTA_R = math.radians(float(GOLD["delta_r_deg"][0]))


def _quat_mul(a, b):
    w1, v1 = a[0], np.asarray(a[1:])
    w2, v2 = b[0], np.asarray(b[1:])
    return np.concatenate([[w1 * w2 - v1 @ v2], w1 * v2 + w2 * v1 + np.cross(v1, v2)])


@pytest.fixture(scope="module")
def setup():
    orc = oracle.Oracle(ROBOT, I.CostParams(), [GRID], [EMPTY], T=T)
    rng = np.random.default_rng(2024)
    qg = I.sample_configs(rng, ROBOT.limits, 1)[0].astype(np.float64)
    pose = oracle.flange_pose(ROBOT.dh, qg)[0]
    x = np.tile(qg, (T, 1))[None]          # at rest on the goal configuration
    return orc, qg, pose, x, rng


def _goal(pose, d=0.0, theta=0.0, rng=None):
    """The flange pose displaced by |d| along a random direction and turned by
    theta about a random axis."""
    rng = rng or np.random.default_rng(0)
    u = rng.normal(size=3)
    u /= np.linalg.norm(u)
    ax = rng.normal(size=3)
    ax /= np.linalg.norm(ax)
    q = np.concatenate([[math.cos(theta / 2)], math.sin(theta / 2) * ax])
    return np.concatenate([pose[:3] + d * u, _quat_mul(pose[3:], q)])


def test_thresholds_fixture_and_defaults_agree():
    assert DELTA_T == 0.005 and abs(DELTA_R - 0.0499164) < 1e-6
    np.testing.assert_array_equal(oracle.success_thresholds(), [DELTA_T, DELTA_R])
    # the CUDA path's descriptors carry the same thresholds (rounded to float32)
    assert I.DELTA_T == DELTA_T and abs(I.DELTA_R - DELTA_R) < 1e-15


def test_at_goal_succeeds(setup):
    orc, qg, pose, x, _ = setup
    ok, met = orc.evaluate(0, qg, pose, x)
    assert bool(ok[0]) is True
    assert met[0, 1] < 1e-12 and met[0, 2] < 1e-6 and met[0, 6] == 1.0 and met[0, 4] == 0.0


@pytest.mark.parametrize("d_mm, want", [(4.9, True), (5.1, False), (0.0, True), (30.0, False)])
def test_translation_threshold(setup, d_mm, want):
    orc, qg, pose, x, _ = setup
    for k in range(4):                                  # several directions
        goal = _goal(pose, d=d_mm * 1e-3, rng=np.random.default_rng(k))
        ok, met = orc.evaluate(0, qg, goal, x)
        assert abs(met[0, 1] - d_mm * 1e-3) < 1e-12
        assert bool(ok[0]) is want, (d_mm, met[0])


@pytest.mark.parametrize("deg, want", [(2.80, True), (2.90, False), (1.0, True), (10.0, False)])
def test_rotation_threshold(setup, deg, want):
    orc, qg, pose, x, _ = setup
    for k in range(4):                                  # several axes
        goal = _goal(pose, theta=math.radians(deg), rng=np.random.default_rng(10 + k))
        ok, met = orc.evaluate(0, qg, goal, x)
        assert abs(met[0, 2] - math.radians(deg)) < 1e-7
        assert bool(ok[0]) is want, (deg, met[0])


def test_both_errors_just_inside_succeed_and_each_alone_just_outside_fails(setup):
    orc, qg, pose, x, _ = setup
    assert orc.evaluate(0, qg, _goal(pose, 4.9e-3, math.radians(2.8)), x)[0][0]
    assert not orc.evaluate(0, qg, _goal(pose, 5.1e-3, math.radians(2.8)), x)[0][0]
    assert not orc.evaluate(0, qg, _goal(pose, 4.9e-3, math.radians(2.9)), x)[0][0]


def test_thresholds_are_strict(setup):
    # an error equal to its threshold fails; the next larger double passes
    orc, qg, pose, x, _ = setup
    goal = _goal(pose, 3e-3, math.radians(2.0))
    _, met = orc.evaluate(0, qg, goal, x)
    pe, re = met[0, 1], met[0, 2]
    assert not orc.evaluate(0, qg, goal, x, thr=[pe, 1.0])[0][0]
    assert orc.evaluate(0, qg, goal, x, thr=[np.nextafter(pe, 1.0), 1.0])[0][0]
    assert not orc.evaluate(0, qg, goal, x, thr=[1.0, re])[0][0]
    assert orc.evaluate(0, qg, goal, x, thr=[1.0, np.nextafter(re, 4.0)])[0][0]


@pytest.mark.parametrize("joint, side, beyond, want", [
    (3, 1, 0.0, True), (3, 1, 1e-9, False), (0, 0, 0.0, True), (0, 0, 1e-9, False), (5, 1, 1e-9, False)])
def test_joint_limits_without_margin(setup, joint, side, beyond, want):
    # one interior waypoint exactly on a limit passes, a hair beyond fails
    orc, qg, pose, x, _ = setup
    xl = x.copy()
    lim = float(ROBOT.limits[joint, side])
    xl[0, 1, joint] = lim + (beyond if side == 1 else -beyond)
    ok, met = orc.evaluate(0, qg, pose, xl)
    assert met[0, 4] == pytest.approx(beyond, abs=1e-15)
    assert bool(ok[0]) is want


@pytest.mark.parametrize("clear_mm, want", [(1.0, True), (-1.0, False), (0.2, True), (-0.2, False)])
def test_collision_free_without_margin(clear_mm, want):
    # one 6 cm sphere on the flange facing the -x face of a large box: success needs
    # phi >= r at the sphere, not phi >= r + eta (the hinge's margin)
    r = I.make_robot()
    r.sph_frame = np.array([8], np.int32)
    r.sph_o = np.zeros((1, 3), np.float32)
    r.sph_r = np.array([0.06], np.float32)
    q = np.array([0.0, 0.0, 0.0, -0.17, 0.0, 0.1, 0.0])     # inside every limit
    pose = oracle.flange_pose(r.dh, q)[0]
    face = pose[0] + 0.06 + clear_mm * 1e-3
    box = np.array([[face + 0.3, pose[1], pose[2], 0.3, 0.5, 0.5]], np.float32)
    grid = I.Grid((-0.2, -0.5, 0.5), 0.02, (40, 50, 40))
    orc = oracle.Oracle(r, I.CostParams(), [grid], [box], T=3)
    x = np.tile(q, (1, 3, 1))
    ok, met = orc.evaluate(0, q, pose, x)
    assert abs(met[0, 0] - clear_mm * 1e-3) < 2e-6
    assert met[0, 4] == 0.0 and met[0, 1] < 1e-12
    assert bool(met[0, 6]) is want and bool(ok[0]) is want


# ---------------------------------------------------------------- best seed

def best_seed_case():
    """Problems whose seeds are kept as they are by a one-iteration plan (the
    first evaluation is always accepted), so success and cost are the seeds'
    own.  Returns (q_start, goal, seeds [P][S][T][7], expected best [P]).

    cheap_fail: at rest 0.03 rad of base rotation away from the goal
    configuration (the flange misses the goal by more than 5 mm), low cost;
    dear_ok: leaves the goal configuration and returns (large smoothness cost),
    ends on the goal; ok: at rest on the goal configuration (cost 0)."""
    rng = np.random.default_rng(7)
    qg = I.sample_configs(rng, ROBOT.limits, 1)[0].astype(np.float64)
    pose = oracle.flange_pose(ROBOT.dh, qg)[0]
    ok = np.tile(qg, (T, 1))
    cheap_fail = ok.copy()
    cheap_fail[:, 0] += 0.03
    dear_ok = ok.copy()
    dear_ok[1:T - 1, 2] += 0.4
    seeds = np.stack([
        np.stack([cheap_fail, dear_ok, cheap_fail]),          # only the dear seed succeeds -> 1
        np.stack([dear_ok, ok, ok]),                           # tie of two successes -> lower index 1
        np.stack([cheap_fail, cheap_fail, cheap_fail]),        # none succeeds -> -1
        np.stack([dear_ok, cheap_fail, ok]),                   # lowest cost among successes -> 2
    ])
    P = seeds.shape[0]
    return (np.tile(qg, (P, 1)), np.tile(pose, (P, 1)), seeds, np.array([1, 1, -1, 2]))


def test_best_seed_pick():
    qs, goal, seeds, want = best_seed_case()
    orc = oracle.Oracle(ROBOT, I.CostParams(), [GRID], [EMPTY], T=T)
    res = orc.plan(np.zeros(len(qs), np.int32), qs, goal, seeds, I.OptParams(iters=1))
    np.testing.assert_array_equal(res["traj"], seeds)      # one iteration keeps the seeds
    # the case is what it says: which seeds succeed, and their cost order
    np.testing.assert_array_equal(res["success"], [[0, 1, 0], [1, 1, 1], [0, 0, 0], [1, 0, 1]])
    c = res["cost"]
    assert c[0, 0] < c[0, 1] and c[3, 2] < c[3, 0]
    assert c[1, 1] == c[1, 2] and c[1, 1] < c[1, 0]
    np.testing.assert_array_equal(res["best"], want)
