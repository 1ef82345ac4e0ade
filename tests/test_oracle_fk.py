"""Pins of the oracle's forward kinematics against the Franka closed forms.

The closed forms come from the manufacturer's DH table (tests/golden/franka_fk.txt),
not from the oracle; invariants check every frame of random configurations."""
import math

import numpy as np
import pytest

import oracle
from golden.read import read
from paper_2410_16727_gb300 import inputs as I

G = read("franka_fk.txt")
ROBOT = I.make_robot()


def test_zero_configuration_origins():
    F = oracle.fk_frames(ROBOT.dh, np.zeros(7))
    for i in range(1, 8):
        np.testing.assert_allclose(F[i][:3, 3], G[f"zero_origin_{i}"], atol=1e-6)
    np.testing.assert_allclose(F[8][:3, 3], G["zero_flange_p"], atol=1e-6)
    np.testing.assert_allclose(F[8][:3, :3], G["zero_flange_R"].reshape(3, 3), atol=1e-6)


def _same_quat(a, b, tol):
    a = np.asarray(a) / np.linalg.norm(a)
    b = np.asarray(b) / np.linalg.norm(b)
    return min(np.abs(a - b).max(), np.abs(a + b).max()) < tol


def test_zero_and_home_flange_pose():
    p0 = oracle.flange_pose(ROBOT.dh, np.zeros(7))[0]
    np.testing.assert_allclose(p0[:3], G["zero_flange_p"], atol=1e-6)
    assert _same_quat(p0[3:], G["zero_flange_quat"], 1e-6)
    ph = oracle.flange_pose(ROBOT.dh, G["home_q"])[0]
    np.testing.assert_allclose(ph[:3], G["home_flange_p"], atol=2e-6)
    assert _same_quat(ph[3:], G["home_flange_quat"], 2e-6)
    F = oracle.fk_frames(ROBOT.dh, G["home_q"])
    np.testing.assert_allclose(F[8][:3, :3], G["home_flange_R"].reshape(3, 3), atol=2e-6)


def test_frame_invariants_random():
    rng = np.random.default_rng(3)
    dh = ROBOT.dh.astype(np.float64)
    for _ in range(50):
        q = I.sample_configs(rng, ROBOT.limits, 1)[0]
        F = oracle.fk_frames(dh, q)
        for i in range(9):
            R = F[i][:3, :3]
            np.testing.assert_allclose(R.T @ R, np.eye(3), atol=1e-12)
            assert abs(np.linalg.det(R) - 1.0) < 1e-12
            np.testing.assert_allclose(F[i][3], [0, 0, 0, 1], atol=0)
        for i in range(1, 9):
            a, d = dh[i - 1, 0], dh[i - 1, 1]
            step = np.linalg.norm(F[i][:3, 3] - F[i - 1][:3, 3])
            assert abs(step - math.hypot(a, d)) < 1e-12
        # joint i turns about the z axis of frame i: rotating q_i moves the
        # frame-i origin not at all and keeps the z axis fixed
        for i in range(1, 8):
            q2 = q.astype(np.float64).copy()
            q2[i - 1] += 0.3
            F2 = oracle.fk_frames(dh, q2)
            np.testing.assert_allclose(F2[i][:3, 3], F[i][:3, 3], atol=1e-12)
            np.testing.assert_allclose(F2[i][:3, 2], F[i][:3, 2], atol=1e-12)


def test_sphere_centre_is_frame_transform_of_offset():
    rng = np.random.default_rng(5)
    r = I.make_robot(seed=1)
    # a zero-offset sphere sits on its frame origin
    r.sph_o[0] = 0.0
    orc = oracle.Oracle(r, I.CostParams(), [I.WORKLOADS["tiny"].grid], [np.zeros((0, 6), np.float32)], T=1)
    for _ in range(10):
        q = I.sample_configs(rng, r.limits, 1)[0]
        F = oracle.fk_frames(r.dh, q)
        c = orc.sphere_centres(q)[0]
        L = r.sph_frame[0]
        np.testing.assert_allclose(c[0], F[L][:3, 3], atol=1e-12)
        for k in range(r.n_spheres):
            Fk = F[r.sph_frame[k]]
            want = Fk[:3, :3] @ r.sph_o[k].astype(np.float64) + Fk[:3, 3]
            np.testing.assert_allclose(c[k], want, atol=1e-12)


def test_flange_quaternion_matches_rotation():
    """The pose quaternion rotates vectors like the flange rotation matrix."""
    rng = np.random.default_rng(9)
    for _ in range(20):
        q = I.sample_configs(rng, ROBOT.limits, 1)[0]
        R = oracle.fk_frames(ROBOT.dh, q)[8][:3, :3]
        w, x, y, z = oracle.flange_pose(ROBOT.dh, q)[0][3:]
        # rotation matrix of a unit quaternion (Rodrigues form)
        Rq = np.array([
            [1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
            [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
            [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])
        np.testing.assert_allclose(Rq, R, atol=1e-12)
        assert w >= 0.0


@pytest.mark.parametrize("name", ["tiny", "batched", "stress"])
def test_sphere_model_shape(name):
    r = I.make_robot()
    assert r.n_spheres == 50
    assert set(np.unique(r.sph_frame)) == set(range(1, 9))
    assert (r.sph_r >= 0.04).all() and (r.sph_r <= 0.08).all()
