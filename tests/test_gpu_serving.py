"""GPU tests of the serving loop (dseed_server_*): every served request computes
what dseed_plan_batch computes for it, alone or mixed with other requests of
other seed counts, horizons and scenes, under a tight HBM budget too."""
import numpy as np
import pytest
import torch

from gpu_helpers import gpu_side, oracle_workload, to_np
from paper_2410_16727_gb300 import binding as B, inputs as I, serving as SV

pytestmark = pytest.mark.gpu

ITERS = 30


def _plan_reference(planner, wl, p, seeds):
    batch = planner.batch(wl.q_start[p:p + 1], wl.goal[p:p + 1], np.array([wl.scene_of_problem[p]], np.int32),
                          seeds.shape[0], seeds.shape[1])
    out = planner.plan(batch, seeds[None])
    torch.cuda.synchronize()
    return {k: to_np(v)[0] for k, v in out.items()}


def _assert_same(got, want, tol=1e-5):
    np.testing.assert_allclose(got["traj"].numpy(), want["traj"], rtol=tol, atol=tol)
    np.testing.assert_allclose(got["cost"].numpy(), want["cost"], rtol=tol, atol=tol)
    assert (got["success"].numpy() == want["success"]).all()
    assert int(got["best"][0]) == int(want["best"])


@pytest.fixture(scope="module")
def setup():
    wl, orc = oracle_workload("tiny", n_scenes=3, n_problems=3, S=4, T=32, iters=ITERS)
    planner, _ = gpu_side(wl)
    rng = np.random.default_rng(5)
    cases = []
    for (S, T) in [(4, 32), (16, 48), (8, 64), (3, 17), (5, 100)]:
        p = int(rng.integers(0, wl.P))
        seeds = I.make_seeds(np.random.default_rng(S * 100 + T), wl.q_start[p], wl.q_goal[p], S, T, wl.robot.limits)
        cases.append((p, seeds))
    return wl, planner, cases


def _server(wl, arena_bytes=256 << 20, max_requests=64, round_iters=7):
    sv = SV.Server(wl.robot, arena_bytes, max_requests=max_requests, round_iters=round_iters, cost=wl.cost,
                   opt=I.OptParams(iters=ITERS))
    for s, (c, g) in enumerate(zip(wl.cuboids, wl.grids)):
        sv.add_scene(s, c, g)
    return sv


def test_served_requests_equal_plan_batch(gpu_lib, setup):
    wl, planner, cases = setup
    sv = _server(wl)
    tickets = [sv.submit(int(wl.scene_of_problem[p]), wl.q_start[p], wl.goal[p], seeds) for p, seeds in cases]
    sv.drain(tickets)
    for t, (p, seeds) in zip(tickets, cases):
        assert sv.poll(t)[0] == 2
        _assert_same(sv.result(t), _plan_reference(planner, wl, p, seeds))
    st = sv.stats()
    assert st.completed == len(cases) and st.failed == 0 and st.rounds >= (ITERS + 6) // 7
    sv.close()


def test_result_same_alone_and_in_the_mix(gpu_lib, setup):
    wl, planner, cases = setup
    p, seeds = cases[1]
    sv = _server(wl)
    t = sv.submit(int(wl.scene_of_problem[p]), wl.q_start[p], wl.goal[p], seeds)
    sv.drain([t])
    alone = {k: v.clone() for k, v in sv.result(t).items()}
    sv.close()
    # the same request arrives while 12 others are being planned and 12 more follow
    sv = _server(wl)
    rng = np.random.default_rng(7)
    others = []

    def random_request():
        q = int(rng.integers(0, wl.P))
        S, T = int(rng.choice([1, 4, 16, 40])), int(rng.choice([8, 32, 48, 64, 90]))
        s = I.make_seeds(rng, wl.q_start[q], wl.q_goal[q], S, T, wl.robot.limits)
        return sv.submit(int(wl.scene_of_problem[q]), wl.q_start[q], wl.goal[q], s)

    others += [random_request() for _ in range(12)]
    for _ in range(3):
        sv.step()
    t = sv.submit(int(wl.scene_of_problem[p]), wl.q_start[p], wl.goal[p], seeds)
    for _ in range(2):
        sv.step()
    others += [random_request() for _ in range(12)]
    sv.drain(others + [t])
    mixed = sv.result(t)
    _assert_same(mixed, {k: v.numpy() if k != "best" else int(v[0]) for k, v in alone.items()})
    assert all(torch.equal(mixed[k], alone[k]) for k in alone), "expected bit-identical results"
    assert sv.stats().completed == 25
    sv.close()


def test_tight_budget_queues_and_serves_in_order(gpu_lib, setup):
    wl, planner, cases = setup
    p, _ = cases[0]
    S, T = 16, 32
    req_bytes = SV_request_bytes(S, T)
    scene_bytes = sum(4 * g.voxels + 6 * 4 * len(c) + 512 for c, g in zip(wl.cuboids, wl.grids))
    table = 3 * 8 * 80 + 256
    arena = (scene_bytes + table + int(2.5 * req_bytes)) // 256 * 256 + 4096
    sv = _server(wl, arena_bytes=arena, max_requests=8, round_iters=10)
    seeds = [I.make_seeds(np.random.default_rng(k), wl.q_start[p], wl.q_goal[p], S, T, wl.robot.limits)
             for k in range(8)]
    tickets = [sv.submit(int(wl.scene_of_problem[p]), wl.q_start[p], wl.goal[p], s) for s in seeds]
    sv.step()
    st = sv.stats()
    assert st.active <= 2 and st.queued >= 6, (st.active, st.queued)
    sv.drain(tickets)
    st = sv.stats()
    assert st.completed == 8 and st.arena_peak <= arena
    done_at = [sv.poll(t)[2] for t in tickets]
    assert done_at == sorted(done_at)            # first come, first served
    for t, s in zip(tickets, seeds):
        _assert_same(sv.result(t), _plan_reference(planner, wl, p, s))
    sv.close()


def SV_request_bytes(S, T, m=5):
    n = 7 * T
    al = lambda v: (v + 63) // 64 * 64
    tot = 0
    for sz in (7, 7, S * n, S * n, S * n, S * n, m * S * n, m * S * n, 16 * S, S, (S + 3) // 4, 2):
        tot = al(tot + sz)
    return 4 * tot


def test_failures_are_reported_not_faulted(gpu_lib, setup):
    wl, planner, cases = setup
    p, seeds = cases[0]
    sv = _server(wl, arena_bytes=64 << 20)
    bad_scene = sv.submit(99, wl.q_start[p], wl.goal[p], seeds)
    huge = sv.submit(0, wl.q_start[p], wl.goal[p],
                     np.zeros((4000, 64, 7), np.float32))        # more state than the arena holds
    ok = sv.submit(int(wl.scene_of_problem[p]), wl.q_start[p], wl.goal[p], seeds)
    with pytest.raises(B.DseedError, match="used by"):
        sv.remove_scene(int(wl.scene_of_problem[p]))
    sv.drain([bad_scene, huge, ok])
    assert sv.poll(bad_scene)[0] == -1 and sv.poll(huge)[0] == -1 and sv.poll(ok)[0] == 2
    sv.remove_scene(int(wl.scene_of_problem[p]))           # no user left
    other = [s for s in range(len(wl.cuboids)) if s != int(wl.scene_of_problem[p])][0]
    with pytest.raises(B.DseedError, match="already resident"):
        sv.add_scene(other, wl.cuboids[other], wl.grids[other])
    sv.close()


def test_poisson_trace_small(gpu_lib, setup):
    """A short Poisson trace through the real-time driver: every request served,
    latencies positive, percentiles ordered."""
    wl, planner, cases = setup
    sw = SV.build_serving_workload(40, lambda s, q: np.full(len(q), 1.0), lambda q: planner.fk(q).cpu().numpy(),
                                   n_scenes=4, problems_per_scene=2, seed_counts=(4, 16), horizons=(32, 48))
    sv = SV.Server(sw.robot, 512 << 20, max_requests=64, round_iters=10, opt=I.OptParams(iters=20))
    for s, (c, g) in enumerate(zip(sw.cuboids, sw.grids)):
        sv.add_scene(s, c, g)
    res = SV.run_trace(sv, sw, SV.poisson_arrivals(40, rate=400.0), timeout_s=120)
    s = SV.summarize(res)
    assert np.isfinite(res["latency_s"]).all() and (res["latency_s"] > 0).all()
    assert 0 < s["p50_ms"] <= s["p99_ms"]
    sv.close()


def test_wait_limit_times_out_and_round_stays_in_flight(gpu_lib, setup):
    """A serving watchdog: with the wait limit at 0 a wait on a round still on
    the GPU returns DSEED_ETIMEOUT at once and retires nothing; with the limit
    restored the same request drains to exactly what it computes without the
    timeout.  The failure is made on the host (a zero limit), the GPU only runs
    an ordinary round."""
    wl, planner, cases = setup
    p = 0
    S, T = 1024, 128                       # a round long enough to be in flight when polled
    seeds = I.make_seeds(np.random.default_rng(11), wl.q_start[p], wl.q_goal[p], S, T, wl.robot.limits)

    def serve(limit_zero):
        sv = _server(wl, arena_bytes=1 << 30, round_iters=ITERS)
        torch.cuda.synchronize()
        t = sv.submit(int(wl.scene_of_problem[p]), wl.q_start[p], wl.goal[p], seeds)
        sv.step()                          # admits the request and launches its only round
        timed_out = False
        if limit_zero:
            sv.set_wait_limit(0.0)
            with pytest.raises(B.DseedTimeout, match="stays in flight"):
                sv.step(wait=True)
            timed_out = True
            assert sv.poll(t)[0] == 1      # still admitted: nothing retired
            st = sv.stats()
            assert st.completed == 0 and st.active == 1
            sv.set_wait_limit(60.0)
        sv.drain([t])
        assert sv.poll(t)[0] == 2
        res = {k: v.clone() for k, v in sv.result(t).items()}
        sv.close()
        return res, timed_out

    plain, _ = serve(False)
    after, timed_out = serve(True)
    assert timed_out
    for k in plain:
        assert torch.equal(plain[k], after[k]), k
    with pytest.raises(B.DseedError):
        sv = _server(wl)
        try:
            sv.set_wait_limit(-1.0)
        finally:
            sv.close()
