"""Pins of the oracle's Eq. 2 loss measured on the robot (denoiser_oracle.fk_mse).

* sphere centres of its 4x4 modified-DH chain against the C oracle's chain, and
  the loss's surface points against the C oracle's chain for a robot whose
  spheres sit at those points;
* the six points of a sphere average to its centre and lie at its radius;
* pred = eps: zero loss and zero gradient;
* a prediction off only in the base joint turns every point about the world z
  axis by the same angle d: the loss is the mean of 4 rho^2 sin^2(d / 2) with rho
  each point's distance from that axis (points from the C oracle);
* per-sample weights combine single-sample losses linearly;
* the decoding reaches the joint limits at normalised -1 and +1;
* the gradient against central differences.
"""
import dataclasses
import math

import numpy as np
import pytest
import torch

import oracle
from oracle import denoiser_oracle as DO
from paper_2410_16727_gb300 import inputs as I

ROBOT = I.make_robot()
RES = 4.0


@pytest.fixture(scope="module")
def corc():
    spec = I.WORKLOADS["tiny"]
    return oracle.Oracle(ROBOT, I.CostParams(), [spec.grid], [np.zeros((0, 6), np.float32)], T=1)


@pytest.fixture(scope="module")
def sorc():
    """The C oracle of a robot whose (zero-radius) spheres are the loss's surface points."""
    offs, frs = DO.surface_offsets(ROBOT)
    pts = dataclasses.replace(ROBOT, sph_frame=frs.astype(np.int32), sph_o=offs, sph_r=np.zeros(len(frs)))
    spec = I.WORKLOADS["tiny"]
    return oracle.Oracle(pts, I.CostParams(), [spec.grid], [np.zeros((0, 6), np.float32)], T=1)


def _case(seed, N=2, T=5):
    rng = np.random.default_rng(seed)
    lin = rng.uniform(-0.8, 0.8, (N, T, 7))
    eps = rng.normal(size=(N, T, 7))
    return lin, eps


def test_points_match_the_c_chain(corc):
    rng = np.random.default_rng(0)
    q = I.sample_configs(rng, ROBOT.limits, 6).astype(np.float64)
    got = DO.robot_points(ROBOT, torch.as_tensor(q)).numpy()
    assert np.abs(got - corc.sphere_centres(q)).max() <= 1e-12


def test_surface_points_match_the_c_chain(sorc, corc):
    rng = np.random.default_rng(1)
    q = I.sample_configs(rng, ROBOT.limits, 6).astype(np.float64)
    offs, frs = DO.surface_offsets(ROBOT)
    got = DO.robot_points(ROBOT, torch.as_tensor(q), offs, frs).numpy()          # [6][300][3]
    assert np.abs(got - sorc.sphere_centres(q)).max() <= 1e-12
    # six per sphere, sphere-major: their mean is the centre, each at the radius from it
    pts = got.reshape(6, -1, 6, 3)
    c = corc.sphere_centres(q)
    assert np.abs(pts.mean(axis=2) - c).max() <= 1e-12
    dist = np.linalg.norm(pts - c[:, :, None, :], axis=-1)
    np.testing.assert_allclose(dist, np.broadcast_to(ROBOT.sph_r.astype(np.float64)[None, :, None], dist.shape),
                               atol=1e-12)


def test_zero_when_the_prediction_is_exact():
    lin, eps = _case(1)
    loss, g = DO.fk_mse(ROBOT, lin, eps, eps, RES)
    assert loss == 0.0 and np.abs(g).max() == 0.0


def test_base_joint_closed_form(sorc):
    lin, eps = _case(2, N=1, T=4)
    delta = 0.3
    pred = eps.copy()
    pred[..., 0] += delta
    lim = ROBOT.limits.astype(np.float64)
    half0 = (lim[0, 1] - lim[0, 0]) / 2.0
    d = half0 * delta / RES
    q = DO.decode(ROBOT, torch.as_tensor(lin), torch.as_tensor(eps), RES).numpy()[0]
    c = sorc.sphere_centres(q)                                   # [T][N_p][3]
    rho2 = c[..., 0] ** 2 + c[..., 1] ** 2
    want = (4.0 * rho2 * math.sin(d / 2) ** 2).sum() / (c.size)
    loss, _ = DO.fk_mse(ROBOT, lin, eps, pred, RES)
    assert abs(loss - want) <= 1e-12 * max(want, 1.0)
    assert want > 1e-3


def test_weights_combine_samples_linearly():
    lin, eps = _case(3)
    pred = eps + np.random.default_rng(4).normal(scale=0.2, size=eps.shape)
    l0, _ = DO.fk_mse(ROBOT, lin[:1], eps[:1], pred[:1], RES)
    l1, _ = DO.fk_mse(ROBOT, lin[1:], eps[1:], pred[1:], RES)
    w = np.array([5.0, 1.0])
    lw, _ = DO.fk_mse(ROBOT, lin, eps, pred, RES, weights=w)
    assert abs(lw - (w[0] * l0 + w[1] * l1) / 2) <= 1e-12 * lw


def test_decoding_spans_the_limits():
    lin = np.stack([-np.ones(7), np.ones(7)])[:, None]          # [2][1][7]
    q = DO.decode(ROBOT, torch.as_tensor(lin), torch.zeros(2, 1, 7, dtype=torch.float64), RES).numpy()
    np.testing.assert_allclose(q[0, 0], ROBOT.limits[:, 0], atol=1e-12)
    np.testing.assert_allclose(q[1, 0], ROBOT.limits[:, 1], atol=1e-12)


def test_gradient_central_differences():
    lin, eps = _case(5, N=2, T=3)
    pred = eps + np.random.default_rng(6).normal(scale=0.3, size=eps.shape)
    w = np.array([1.0, 5.0])
    _, g = DO.fk_mse(ROBOT, lin, eps, pred, RES, weights=w)
    h = 1e-6
    for idx in np.ndindex(*pred.shape):
        pp, pm = pred.copy(), pred.copy()
        pp[idx] += h
        pm[idx] -= h
        fd = (DO.fk_mse(ROBOT, lin, eps, pp, RES, weights=w)[0] - DO.fk_mse(ROBOT, lin, eps, pm, RES, weights=w)[0]) / (2 * h)
        assert abs(g[idx] - fd) <= 1e-6 * max(1e-3, np.abs(g).max())
