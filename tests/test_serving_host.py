"""Host-side parts of the serving workload, without a GPU: the request mix of
the serving configuration (seed counts {4, 16, 64, 256} and horizons
{32, 48, 64} drawn uniformly, a pool of scenes with 10-100 cuboids on grids of
64^3..192^3 voxels at 1-2 cm), the Poisson arrival times and the latency
summary."""
import math

import numpy as np

from paper_2410_16727_gb300 import serving as SV


def _fake_fns():
    # every candidate configuration is accepted; goal poses are not used here
    return (lambda s, q: np.full(np.asarray(q).reshape(-1, 7).shape[0], 1.0),
            lambda q: np.zeros((np.asarray(q).reshape(-1, 7).shape[0], 7)))


def test_scene_pool_follows_the_serving_recipe():
    cub, grids = SV.serving_scene_pool(24, seed=0)
    assert len(cub) == len(grids) == 24
    for c, g in zip(cub, grids):
        n = g.n[0]
        assert tuple(g.n) == (n, n, n) and n in SV.GRID_SIZES
        assert g.res in (0.01, 0.02)
        assert 10 <= len(c) <= 100 and c.shape[1] == 6
        # the grid is centred on the workspace point (0.1, 0, 0.5)
        centre = np.asarray(g.origin) + n * g.res / 2
        assert np.allclose(centre, (0.1, 0.0, 0.5))
    # the same seed gives the same scenes
    cub2, _ = SV.serving_scene_pool(24, seed=0)
    assert all(np.array_equal(a, b) for a, b in zip(cub, cub2))


def test_request_mix_is_uniform_and_seeds_are_shared():
    clear, pose = _fake_fns()
    n = 6000
    wl = SV.build_serving_workload(n, clear, pose, n_scenes=2, problems_per_scene=3, seed=0)
    assert len(wl.requests) == n and len(wl.problems) == 6
    S = np.array([s for _, s, _ in wl.requests])
    T = np.array([t for _, _, t in wl.requests])
    P = np.array([p for p, _, _ in wl.requests])
    # each value is drawn with probability 1/k: counts within 5 standard deviations
    for vals, allowed in ((S, SV.SEED_COUNTS), (T, SV.HORIZONS), (P, range(6))):
        allowed = list(allowed)
        assert set(vals.tolist()) == set(allowed)
        p = 1.0 / len(allowed)
        sd = math.sqrt(n * p * (1 - p))
        for a in allowed:
            assert abs((vals == a).sum() - n * p) < 5 * sd, (a, (vals == a).sum())
    lim = wl.robot.limits
    for p, s, t in wl.requests[:200]:
        x = wl.problems[p].seeds[(s, t)]
        assert x.shape == (s, t, 7) and x.dtype == np.float32
        assert (x >= lim[:, 0] - 1e-6).all() and (x <= lim[:, 1] + 1e-6).all()
    # the seeds of one (problem, S, T) are drawn once and reused by every request naming it
    keys = {(p, s, t) for p, s, t in wl.requests}
    assert sum(len(pr.seeds) for pr in wl.problems) == len(keys)
    # and do not depend on how many requests were drawn
    wl2 = SV.build_serving_workload(50, clear, pose, n_scenes=2, problems_per_scene=3, seed=0)
    for p, s, t in wl2.requests:
        assert np.array_equal(wl2.problems[p].seeds[(s, t)], wl.problems[p].seeds[(s, t)])
    assert wl2.requests == wl.requests[:50]


def test_seeds_interpolate_start_to_goal_configuration():
    clear, pose = _fake_fns()
    wl = SV.build_serving_workload(400, clear, pose, n_scenes=1, problems_per_scene=2, seed=3)
    for pr in wl.problems:
        for (s, t), x in pr.seeds.items():
            ts = np.arange(1, t + 1)[:, None] / t
            base = np.clip(pr.q_start + ts * (pr.q_goal - pr.q_start), wl.robot.limits[:, 0], wl.robot.limits[:, 1])
            # noise of standard deviation 0.1 around the straight path (clipped to the limits)
            dev = x.astype(np.float64) - base[None]
            assert abs(dev.mean()) < 0.05 and 0.05 < dev.std() < 0.12, (s, t, dev.std())


def test_poisson_arrivals():
    rate = 250.0
    a = SV.poisson_arrivals(20000, rate, seed=1)
    assert a.shape == (20000,) and (np.diff(a) > 0).all() and a[0] > 0
    gaps = np.diff(np.concatenate([[0.0], a]))
    # exponential gaps: mean 1/rate, standard deviation 1/rate
    assert abs(gaps.mean() * rate - 1.0) < 0.03
    assert abs(gaps.std() * rate - 1.0) < 0.05
    assert np.array_equal(a, SV.poisson_arrivals(20000, rate, seed=1))
    assert not np.array_equal(a, SV.poisson_arrivals(20000, rate, seed=2))


def test_summarize_percentiles_skip_unfinished_requests():
    lat = np.array([0.001 * k for k in range(1, 101)] + [np.nan] * 5)
    res = dict(latency_s=lat, plans_per_s=123.0, seed_success=0.5, problems_solved=0.75, rounds=7)
    s = SV.summarize(res)
    assert math.isclose(s["p50_ms"], 50.5) and math.isclose(s["p99_ms"], 99.01)
    assert math.isclose(s["mean_ms"], 50.5)
    assert s["plans_per_s"] == 123.0 and s["rounds"] == 7
    assert s["seed_success"] == 0.5 and s["problems_solved"] == 0.75
