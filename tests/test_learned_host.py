"""Host-side interpolation weights of the learned path, without a GPU: the
straight start-goal path the denoiser's residual is measured from, and the
resampling of proposals from the network's horizon to a request's horizon
(linear interpolation in time, the start configuration at fraction 0)."""
import numpy as np
import pytest

from paper_2410_16727_gb300 import learned as L


@pytest.mark.parametrize("T0,T1", [(32, 64), (32, 48), (64, 32), (32, 33), (48, 32), (5, 3), (1, 4), (4, 1),
                                   (32, 32)])
def test_resample_weights_interpolate_linearly_in_time(T0, T1):
    rng = np.random.default_rng(100 * T0 + T1)
    N, D = 5, 7
    x = rng.normal(size=(N, T0, D))
    q0 = rng.normal(size=(N, D))
    Wx, Wq = L.resample_weights(T0, T1, D)
    assert Wx.shape == (T0 * D, T1 * D) and Wq.shape == (D, T1 * D)
    got = (x.reshape(N, T0 * D) @ Wx.astype(np.float64) + q0 @ Wq.astype(np.float64)).reshape(N, T1, D)
    knots = np.arange(T0 + 1) / T0                 # q0 at 0, input waypoint k at k / T0
    at = np.arange(1, T1 + 1) / T1
    for n in range(N):
        for d in range(D):
            want = np.interp(at, knots, np.concatenate([[q0[n, d]], x[n, :, d]]))
            np.testing.assert_allclose(got[n, :, d], want, rtol=0, atol=1e-6)
    # a partition of unity per output entry, and joints never mix
    np.testing.assert_allclose(Wx.sum(0) + Wq.sum(0), 1.0, atol=1e-6)
    rows = np.arange(T0 * D) % D
    cols = np.arange(T1 * D) % D
    assert (Wx[rows[:, None] != cols[None, :]] == 0).all()
    assert (Wq[np.arange(D)[:, None] != cols[None, :]] == 0).all()


def test_resample_to_half_the_horizon_takes_every_second_waypoint():
    Wx, Wq = L.resample_weights(64, 32, 7)
    x = np.random.default_rng(0).normal(size=(3, 64, 7)).astype(np.float32)
    got = (x.reshape(3, -1) @ Wx).reshape(3, 32, 7)
    assert np.array_equal(got, x[:, 1::2])
    assert not Wq.any()


@pytest.mark.parametrize("T", [1, 7, 32, 64])
def test_linear_path_weights(T):
    rng = np.random.default_rng(T)
    D = 7
    qs, qg = rng.uniform(-1, 1, size=(4, D)), rng.uniform(-1, 1, size=(4, D))
    W = L.linear_path_weights(T, D)
    got = (np.concatenate([qs, qg], 1) @ W.astype(np.float64)).reshape(4, T, D)
    t = np.arange(1, T + 1)[None, :, None] / T
    np.testing.assert_allclose(got, qs[:, None] + t * (qg - qs)[:, None], rtol=0, atol=1e-6)
    # the last waypoint is the goal configuration itself
    assert np.array_equal(W[D:, (T - 1) * D:], np.eye(D, dtype=np.float32))


def test_limit_normalisation_maps_limits_to_unit_interval():
    """App. A.4: joints scaled to [-1, 1] by their mechanical limits; the inverse
    undoes it.  Checked on the (scale, shift) rows the FiLM kernel applies."""
    import torch

    from paper_2410_16727_gb300 import inputs as I
    robot = I.make_robot()
    fwd = L._limits_affine(robot, torch.device("cpu"), False).numpy().astype(np.float64)[0]
    inv = L._limits_affine(robot, torch.device("cpu"), True).numpy().astype(np.float64)[0]
    lo, hi = robot.limits[:, 0].astype(np.float64), robot.limits[:, 1].astype(np.float64)
    f = lambda v, a: v * a[:7] + a[7:]
    np.testing.assert_allclose(f(lo, fwd), -1.0, atol=1e-6)
    np.testing.assert_allclose(f(hi, fwd), 1.0, atol=1e-6)
    np.testing.assert_allclose(f((lo + hi) / 2, fwd), 0.0, atol=1e-6)
    q = np.random.default_rng(0).uniform(lo, hi, size=(50, 7))
    np.testing.assert_allclose(f(f(q, fwd), inv), q, atol=1e-5)
