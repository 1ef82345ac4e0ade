"""Pins of the oracle's self-collision term (C_self of the App. A.5 objective).

* two spheres, one on frame 1 and one on the flange, at q = 0: their centres are
  the published frame origins (golden file), so the hinge has a closed form;
* rotating the whole arm about the base axis (joint 1) moves every sphere rigidly:
  C_self is unchanged and its joint-1 derivative is zero;
* the checked-pair rule against a brute force from an independent FK (4x4 DH
  products in numpy) at the reference pose;
* the full gradient against central differences at self-contact configurations.
"""
import dataclasses
import math

import numpy as np
import pytest

import oracle
from golden.read import read
from paper_2410_16727_gb300 import inputs as I

GOLD = read("franka_fk.txt")
ROBOT = I.make_robot()
EMPTY = np.zeros((0, 6), np.float32)
GRID = I.WORKLOADS["tiny"].grid
SELF_ONLY = I.CostParams(w_c=0.0, w_v=0.0, w_a=0.0, w_j=0.0, w_p=0.0, w_R=0.0, w_l=0.0, w_self=100.0,
                         eta_self=0.01)


def _orc(cost, robot=ROBOT, T=1):
    return oracle.Oracle(robot, cost, [GRID], [EMPTY], T=T)


def _two_sphere_robot(r):
    return dataclasses.replace(ROBOT, sph_frame=np.array([1, 8], np.int32),
                               sph_o=np.zeros((2, 3), np.float32), sph_r=np.array([r, r], np.float32),
                               self_margin=-10.0)    # every pair on frames >= 2 apart is checked


def test_two_spheres_closed_form():
    r = 0.35
    orc = _orc(SELF_ONLY, _two_sphere_robot(r))
    assert orc.n_self_pairs == 1
    c1, c8 = GOLD["zero_origin_1"], GOLD["zero_flange_p"]
    d = float(np.linalg.norm(c8 - c1))
    r32 = float(np.float32(r))                      # the robot description is float32
    want = SELF_ONLY.w_self * (2 * r32 + SELF_ONLY.eta_self - d)
    q0 = np.zeros(7)
    f, g, terms = orc.cost(0, q0, None, q0[None, None], grad=True, terms=True)
    assert want > 0
    # the golden origins are exact decimals, the DH table float32: 1e-6 relative
    assert abs(terms[0, 0] - want) <= 1e-6 * want
    assert abs(g[0, 0, 0]) <= 1e-9                 # the base joint moves both spheres
    ok, met = orc.evaluate(0, q0, [0, 0, 0, 1, 0, 0, 0], q0[None, None])
    assert abs(met[0, 0] - (d - 2 * r32)) <= 1e-7   # clearance of the pair (the scene is empty)
    # the pair no longer collides when w_self = 0 turns the term off
    off = _orc(dataclasses.replace(SELF_ONLY, w_self=0.0), _two_sphere_robot(r))
    _, met_off = off.evaluate(0, q0, [0, 0, 0, 1, 0, 0, 0], q0[None, None])
    assert met_off[0, 0] > 1.0


def _independent_centres(robot, q):
    """Sphere centres from 4x4 modified-DH products (numpy, written here)."""
    def rx(a):
        c, s = math.cos(a), math.sin(a)
        return np.array([[1, 0, 0, 0], [0, c, -s, 0], [0, s, c, 0], [0, 0, 0, 1.0]])

    def rz(a):
        c, s = math.cos(a), math.sin(a)
        return np.array([[c, -s, 0, 0], [s, c, 0, 0], [0, 0, 1, 0], [0, 0, 0, 1.0]])

    def tr(x, z):
        M = np.eye(4)
        M[0, 3], M[2, 3] = x, z
        return M

    F = [np.eye(4)]
    dh = robot.dh.astype(np.float64)
    for i in range(8):
        a, d, al, off = dh[i]
        th = (q[i] if i < 7 else 0.0) + off
        F.append(F[-1] @ rx(al) @ tr(a, 0.0) @ rz(th) @ tr(0.0, d))
    o = robot.sph_o.astype(np.float64)
    return np.array([(F[f] @ np.append(o[k], 1.0))[:3] for k, f in enumerate(robot.sph_frame)])


def test_pair_rule_brute_force():
    orc = _orc(SELF_ONLY)
    c = _independent_centres(ROBOT, ROBOT.self_ref.astype(np.float64))
    r = ROBOT.sph_r.astype(np.float64)
    f = ROBOT.sph_frame
    ns = len(r)
    want = np.zeros((ns, ns), np.uint8)
    for i in range(ns):
        for j in range(ns):
            if i != j and abs(int(f[i]) - int(f[j])) >= 2 and \
                    np.linalg.norm(c[i] - c[j]) - r[i] - r[j] >= float(ROBOT.self_margin):
                want[i, j] = 1
    assert np.array_equal(orc.self_mask, want)
    assert orc.n_self_pairs == int(want.sum()) // 2 > 100
    # nothing is in contact at the reference pose (margin 2 cm > eta_self 1 cm)
    ref = ROBOT.self_ref.astype(np.float64)
    _, terms = orc.cost(0, ref, None, ref[None, None], grad=False, terms=True)
    assert terms[0, 0] == 0.0


def _contact_configs(orc, n, seed):
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < n:
        q = I.sample_configs(rng, ROBOT.limits, 1)[0].astype(np.float64)
        _, terms = orc.cost(0, q, None, q[None, None], grad=False, terms=True)
        if terms[0, 0] > 1.0:
            out.append(q)
    return out


def test_base_joint_invariance():
    orc = _orc(SELF_ONLY)
    for q in _contact_configs(orc, 5, 3):
        f, g = orc.cost(0, q, None, q[None, None], grad=True)
        q2 = q.copy()
        q2[0] += 0.7
        f2 = orc.cost(0, q2, None, q2[None, None], grad=False)
        assert abs(f2[0] - f[0]) <= 1e-9 * f[0]
        assert abs(g[0, 0, 0]) <= 1e-9 * max(1.0, np.abs(g).max())


@pytest.mark.parametrize("seed", [0, 1])
def test_self_gradient_central_differences(seed):
    orc = _orc(SELF_ONLY, T=1)
    h = 1e-6
    for q in _contact_configs(orc, 3, 10 + seed):
        f0, g = orc.cost(0, q, None, q[None, None], grad=True)
        for j in range(7):
            qp, qm = q.copy(), q.copy()
            qp[j] += h
            qm[j] -= h
            fp = orc.cost(0, q, None, qp[None, None], grad=False)[0]
            fm = orc.cost(0, q, None, qm[None, None], grad=False)[0]
            if abs((fp - f0[0]) - (f0[0] - fm)) > 0.05 * h:      # a pair switching on / off within h
                continue
            assert abs(g[0, 0, j] - (fp - fm) / (2 * h)) <= 1e-5 * max(1.0, np.abs(g).max())
