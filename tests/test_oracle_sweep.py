"""Pins of the oracle's swept collision term: the world hinge at n_sweep
joint-space interpolants of every segment between consecutive waypoints
(y_0 = q_start), each interpolant's derivative split between the segment's two
waypoints.

* a stationary trajectory (every waypoint and the start equal to q): each
  interpolant is q, so the collision cost is T (1 + n) W(q) and the gradient is
  (1 + n) g(q) at waypoints 1..T-1 and (1 + n/2) g(q) at T, with W, g the
  hinge and its derivative at q alone (a one-waypoint problem without sweep);
* the sweep adds exactly the sum over segments and interpolants of W at the
  interpolant, each computed alone (u = 1/2 for n = 1; 1/3, 2/3 for n = 2);
* the full gradient against central differences with n = 2;
* the success test sees a collision between two free waypoints: clearance is
  the minimum over waypoints and interpolants, each computed alone.
"""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_2410_16727_gb300 import inputs as I

SPEC = I.WORKLOADS["tiny"]
ROBOT = I.make_robot()
WORLD = I.CostParams(w_v=0.0, w_a=0.0, w_j=0.0, w_p=0.0, w_R=0.0, w_l=0.0)


@pytest.fixture(scope="module")
def scene():
    cub, grids = I.make_scenes(SPEC, n_scenes=1)
    return cub, grids


def _orc(scene, cost, n):
    cub, grids = scene
    return oracle.Oracle(ROBOT, dataclasses.replace(cost, n_sweep=n), grids, cub, T=1)


def _single(orc0, q):
    """World hinge and its derivative at q alone (one waypoint, start = q)."""
    c, g, tr = orc0.cost(0, q, None, q[None, None], grad=True, terms=True)
    return tr[0, 0], g[0, 0]


def _contact_configs(orc0, n, seed, lo=1.0):
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < n:
        q = I.sample_configs(rng, ROBOT.limits, 1)[0].astype(np.float64)
        if _single(orc0, q)[0] > lo:
            out.append(q)
    return out


@pytest.mark.parametrize("n", [1, 2, 3])
def test_stationary_trajectory_closed_form(scene, n):
    orc0, orcn = _orc(scene, WORLD, 0), _orc(scene, WORLD, n)
    T = 5
    for q in _contact_configs(orc0, 3, 10 + n):
        W, g = _single(orc0, q)
        x = np.tile(q, (T, 1))[None]
        c, gr, tr = orcn.cost(0, q, None, x, grad=True, terms=True)
        assert abs(tr[0, 0] - T * (1 + n) * W) <= 1e-12 * T * (1 + n) * W
        want = np.tile((1 + n) * g, (T, 1))
        want[-1] = (1 + n / 2) * g
        assert np.abs(gr[0] - want).max() <= 1e-9 * max(1.0, np.abs(want).max())


@pytest.mark.parametrize("n", [1, 2])
def test_sweep_adds_interpolant_hinges(scene, n):
    orc0, orcn = _orc(scene, WORLD, 0), _orc(scene, WORLD, n)
    rng = np.random.default_rng(4)
    T = 6
    qs = I.sample_configs(rng, ROBOT.limits, 1)[0].astype(np.float64)
    for _ in range(4):
        x = I.random_trajectories(rng, qs, 1, T, ROBOT.limits, spread=1.5)[0].astype(np.float64)
        base = orc0.cost(0, qs, None, x[None], grad=False, terms=True)[1][0, 0]
        swept = orcn.cost(0, qs, None, x[None], grad=False, terms=True)[1][0, 0]
        y = np.vstack([qs[None], x])
        extra = 0.0
        for t in range(1, T + 1):
            for j in range(1, n + 1):
                u = j / (n + 1)
                extra += _single(orc0, (1 - u) * y[t] + u * y[t - 1])[0]
        assert abs(swept - base - extra) <= 1e-9 * max(1.0, extra)
    assert extra > 0


def test_sweep_gradient_central_differences(scene):
    orc2 = _orc(scene, I.CostParams(), 2)
    rng = np.random.default_rng(7)
    T, h = 4, 1e-6
    qs = I.sample_configs(rng, ROBOT.limits, 1)[0].astype(np.float64)
    checked = 0
    for _ in range(3):
        x = I.random_trajectories(rng, qs, 1, T, ROBOT.limits, spread=1.5)[0].astype(np.float64)
        f0, g = orc2.cost(0, qs, None, x[None], grad=True)
        for idx in np.ndindex(T, 7):
            xp, xm = x.copy(), x.copy()
            xp[idx] += h
            xm[idx] -= h
            fp = orc2.cost(0, qs, None, xp[None], grad=False)[0]
            fm = orc2.cost(0, qs, None, xm[None], grad=False)[0]
            if abs((fp - f0[0]) - (f0[0] - fm)) > 1e-3 * h * max(1.0, abs(g[0][idx])):   # a kink within h
                continue
            assert abs(g[0][idx] - (fp - fm) / (2 * h)) <= 1e-5 * max(1.0, np.abs(g).max())
            checked += 1
    assert checked > 50


def test_success_sees_collisions_between_waypoints(scene):
    orc0, orc3 = _orc(scene, I.CostParams(), 0), _orc(scene, I.CostParams(), 3)
    rng = np.random.default_rng(2)
    found = 0
    for _ in range(4000):
        qa, qb = I.sample_configs(rng, ROBOT.limits, 2).astype(np.float64)
        if orc0.clearance(0, qa)[0] < 0.01 or orc0.clearance(0, qb)[0] < 0.01:
            continue
        x = qb[None, None]
        _, m0 = orc0.evaluate(0, qa, None, x)
        _, m3 = orc3.evaluate(0, qa, None, x)
        between = min(orc0.clearance(0, (1 - u) * qb + u * qa)[0] for u in (0.25, 0.5, 0.75))
        assert m0[0, 0] == pytest.approx(orc0.clearance(0, qb)[0], abs=1e-12)
        assert m3[0, 0] == pytest.approx(min(m0[0, 0], between), abs=1e-12)
        if between < 0:
            assert m0[0, 6] == 1.0 and m3[0, 6] == 0.0     # free at the waypoints, not in between
            found += 1
            if found == 3:
                break
    assert found == 3
