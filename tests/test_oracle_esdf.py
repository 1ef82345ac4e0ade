"""Pins of the oracle's ESDF build and trilinear lookup.

The box distances are checked against the closest-point construction (project p
onto the box; inside, distance to the nearest face), which is a different
formula from the oracle's; the interpolation against affine fields, which
trilinear interpolation reproduces exactly."""
import numpy as np
import pytest

import oracle
from paper_2410_16727_gb300 import inputs as I


def _closest_point_sdf(boxes, p):
    best = np.full(p.shape[0], 1000.0)
    for b in boxes.astype(np.float64):
        lo, hi = b[:3] - b[3:], b[:3] + b[3:]
        q = np.clip(p, lo, hi)
        outside = np.linalg.norm(p - q, axis=1)
        inside = np.all((p > lo) & (p < hi), axis=1)
        depth = np.minimum(p - lo, hi - p).min(axis=1)
        s = np.where(inside, -depth, outside)
        best = np.minimum(best, s)
    return best


def _centres(grid):
    nx, ny, nz = grid.n
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    o = np.asarray(grid.origin, np.float64)
    return np.stack([o[0] + (i + 0.5) * grid.res, o[1] + (j + 0.5) * grid.res,
                     o[2] + (k + 0.5) * grid.res], axis=-1).reshape(-1, 3)


@pytest.mark.parametrize("seed,n,nb", [(0, (8, 8, 8), 1), (1, (12, 10, 9), 2), (2, (16, 16, 16), 3),
                                       (3, (9, 13, 16), 3)])
def test_esdf_matches_closest_point_distance(seed, n, nb):
    rng = np.random.default_rng(seed)
    grid = I.Grid((-0.1, -0.05, 0.0), 0.037, n)
    ext = np.array(n) * grid.res
    boxes = []
    for _ in range(nb):
        h = rng.uniform(0.02, 0.12, size=3)
        c = np.asarray(grid.origin) + rng.uniform(0.2, 0.8, size=3) * ext
        boxes.append([*c, *h])
    boxes = np.asarray(boxes, np.float32)
    phi = oracle.esdf_build(boxes, grid)
    want = _closest_point_sdf(boxes, _centres(grid)).reshape(n[2], n[1], n[0])
    np.testing.assert_allclose(phi, want, atol=1e-12, rtol=0)
    assert (phi < 0).any() and (phi > 0).any()


def test_esdf_empty_scene_is_far():
    grid = I.Grid((0.0, 0.0, 0.0), 0.1, (4, 5, 6))
    phi = oracle.esdf_build(np.zeros((0, 6), np.float32), grid)
    assert phi.shape == (6, 5, 4) and (phi == 1000.0).all()


def test_esdf_zero_on_faces_and_unit_gradient():
    # one box whose +x face passes exactly through a plane of voxel centres
    grid = I.Grid((0.0, 0.0, 0.0), 0.125, (16, 16, 16))
    face_x = (8 + 0.5) * 0.125
    box = np.array([[face_x - 0.5, 1.0, 1.0, 0.5, 2.0, 2.0]], np.float32)
    phi = oracle.esdf_build(box, grid)
    np.testing.assert_allclose(phi[:, :, 8], 0.0, atol=1e-12)
    # in the face region the field is affine in x: the lookup gives distance
    # to the face exactly and a unit gradient along +x
    rng = np.random.default_rng(1)
    p = np.stack([rng.uniform(1.2, 1.8, 50), rng.uniform(0.4, 1.6, 50), rng.uniform(0.4, 1.6, 50)], 1)
    v, g = oracle.esdf_lookup(phi, grid, p)
    np.testing.assert_allclose(v, p[:, 0] - face_x, atol=1e-12)
    np.testing.assert_allclose(g, np.tile([1.0, 0.0, 0.0], (50, 1)), atol=1e-12)


def test_trilinear_exact_on_affine_field():
    rng = np.random.default_rng(2)
    grid = I.Grid((-0.3, 0.2, -0.1), 0.05, (11, 7, 9))
    gvec = rng.normal(size=3)
    b = 0.37
    c = _centres(grid)
    phi = (c @ gvec + b).reshape(9, 7, 11)
    lo = np.asarray(grid.origin) + 0.5 * grid.res
    hi = np.asarray(grid.origin) + (np.asarray(grid.n) - 0.5) * grid.res
    p = lo + rng.uniform(0, 1, size=(200, 3)) * (hi - lo)
    v, g = oracle.esdf_lookup(phi, grid, p)
    np.testing.assert_allclose(v, p @ gvec + b, atol=1e-12)
    np.testing.assert_allclose(g, np.tile(gvec, (200, 1)), atol=1e-11)


def test_trilinear_clamps_outside_grid():
    grid = I.Grid((0.0, 0.0, 0.0), 0.1, (5, 5, 5))
    gvec = np.array([1.0, 2.0, -3.0])
    phi = (_centres(grid) @ gvec).reshape(5, 5, 5)
    # beyond +x and below -z: value of the clamped point, zero gradient on those axes
    p = np.array([[0.9, 0.23, -0.4]])
    v, g = oracle.esdf_lookup(phi, grid, p)
    clamped = np.array([0.45, 0.23, 0.05])
    np.testing.assert_allclose(v, [clamped @ gvec], atol=1e-12)
    np.testing.assert_allclose(g[0], [0.0, 2.0, 0.0], atol=1e-12)
    # exactly on the last voxel centre: still inside, gradient kept
    v2, g2 = oracle.esdf_lookup(phi, grid, np.array([[0.45, 0.25, 0.25]]))
    np.testing.assert_allclose(g2[0], gvec, atol=1e-12)
