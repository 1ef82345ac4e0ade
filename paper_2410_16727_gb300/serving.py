"""Serving loop driver: Poisson arrivals fed in real time to the native server
(dseed_server_*), with plan latency percentiles and throughput.

The server (libdseed) does the scheduling: admission under the HBM budget,
continuous batching of every admitted request into rounds of the resumable
optimiser kernel, retirement and output copies.  This module only generates the
workload, submits requests when their arrival time passes, calls
dseed_server_step in a loop and reads the ticket states.
"""
from __future__ import annotations

import dataclasses
import time
from typing import Callable, Dict, List, Optional, Sequence

import numpy as np
import torch

from . import binding as B
from . import inputs as I


# ---------------------------------------------------------------------------- workload

SEED_COUNTS = (4, 16, 64, 256)
HORIZONS = (32, 48, 64)
GRID_SIZES = (64, 96, 128, 160, 192)


def serving_scene_pool(n_scenes: int = 64, seed: int = 0):
    """Scenes of 10-100 random cuboids with grids of 64^3..192^3 voxels at 1-2 cm,
    centred on the robot's workspace."""
    cub, grids = [], []
    for s in range(n_scenes):
        rng = I._rng(3000 + seed, s, 1)
        n = int(rng.choice(GRID_SIZES))
        res = float(rng.choice((0.01, 0.02)))
        ext = n * res
        origin = (0.1 - ext / 2, -ext / 2, 0.5 - ext / 2)
        grids.append(I.Grid(origin, res, (n, n, n)))
        cub.append(I.scene_tiny(rng, n_boxes=int(rng.integers(10, 101))))
    return cub, grids


@dataclasses.dataclass
class ServingProblem:
    scene: int
    q_start: np.ndarray
    goal: np.ndarray
    seeds: Dict[tuple, np.ndarray]      # (S, T) -> [S][T][7]
    q_goal: Optional[np.ndarray] = None  # the goal configuration the random seeds interpolate towards


@dataclasses.dataclass
class ServingWorkload:
    robot: I.Robot
    cuboids: list
    grids: list
    problems: List[ServingProblem]
    requests: List[tuple]               # (problem index, S, T)
    arrivals: Optional[np.ndarray] = None


def build_serving_workload(n_requests: int, clearance_fn, pose_fn, n_scenes: int = 64,
                           problems_per_scene: int = 2, seed: int = 0,
                           seed_counts: Sequence[int] = SEED_COUNTS,
                           horizons: Sequence[int] = HORIZONS) -> ServingWorkload:
    """Requests draw a scene problem, a seed count and a horizon uniformly; the
    seeds of each (problem, S, T) are drawn once and shared by the requests that
    use them (inputs only)."""
    robot = I.make_robot()
    cub, grids = serving_scene_pool(n_scenes, seed)
    spec = I.WorkloadSpec("serving", 3 + 100 * seed, n_scenes, n_scenes * problems_per_scene, 4, 32, 100, "tiny",
                          grids[0])
    wl = I.build_workload(spec, cub, grids, clearance_fn, pose_fn, n_problems=n_scenes * problems_per_scene,
                          S=1, T=32, robot=robot)
    problems = []
    for p in range(wl.P):
        problems.append(ServingProblem(int(wl.scene_of_problem[p]), wl.q_start[p], wl.goal[p], {}, wl.q_goal[p]))
    rng = I._rng(4000 + seed, 0, 0)
    reqs = []
    for _ in range(n_requests):
        p = int(rng.integers(0, len(problems)))
        S = int(rng.choice(seed_counts))
        T = int(rng.choice(horizons))
        key = (S, T)
        pr = problems[p]
        if key not in pr.seeds:
            pr.seeds[key] = I.make_seeds(I._rng(5000 + seed, p, S * 1000 + T), pr.q_start,
                                         wl.q_goal[p], S, T, robot.limits)
        reqs.append((p, S, T))
    return ServingWorkload(robot, cub, grids, problems, reqs)


# ---------------------------------------------------------------------------- server wrapper

class Server:
    """Owning wrapper: device arena (the HBM budget) + native server."""

    def __init__(self, robot: I.Robot, arena_bytes: int, max_requests: int = 4096, round_iters: int = 10,
                 cost: Optional[I.CostParams] = None, opt: Optional[I.OptParams] = None, device="cuda"):
        self.robot = B.Robot(robot)
        self.arena = torch.empty(int(arena_bytes), dtype=torch.uint8, device=device)
        self.cost = cost or I.CostParams()
        self.opt = opt or I.OptParams()
        desc = B.server_desc(arena_bytes, max_requests, round_iters, self.cost, self.opt)
        torch.cuda.synchronize()
        self.h = B.server_create(self.robot, desc, self.arena)
        self._keep: Dict[int, tuple] = {}

    def close(self):
        """Destroy the native server (it waits for its stream) and release the
        arena at once, so a new server can take the budget before this object
        is collected."""
        if getattr(self, "h", None) is not None:
            B.server_destroy(self.h)
            self.h = None
        self.arena = None

    def __del__(self):
        self.close()

    def add_scene(self, scene_id: int, cuboids, grid):
        B.server_add_scene(self.h, scene_id, cuboids, grid)

    def remove_scene(self, scene_id: int):
        B.server_remove_scene(self.h, scene_id)

    def submit(self, scene_id: int, q_start, goal, seeds: np.ndarray, out: Optional[dict] = None):
        """Queue a request; inputs are copied to pinned host buffers here, outputs
        land in `out` (pinned tensors traj, cost, success, best)."""
        S, T = int(seeds.shape[0]), int(seeds.shape[1])
        ins = dict(q=torch.as_tensor(np.asarray(q_start, np.float32)).pin_memory(),
                   g=torch.as_tensor(np.asarray(goal, np.float32)).pin_memory(),
                   s=torch.as_tensor(np.ascontiguousarray(seeds, np.float32)).pin_memory())
        if out is None:
            out = alloc_outputs(S, T)
        return self.submit_pinned(scene_id, ins, out)

    def submit_pinned(self, scene_id: int, ins: dict, out: dict) -> int:
        S, T = int(ins["s"].shape[0]), int(ins["s"].shape[1])
        r = B.Request()
        r.scene_id, r.S, r.T = int(scene_id), S, T
        r.q_start_host, r.goal_host, r.seeds_host = ins["q"].data_ptr(), ins["g"].data_ptr(), ins["s"].data_ptr()
        r.traj_host, r.cost_host = out["traj"].data_ptr(), out["cost"].data_ptr()
        r.success_host, r.best_host = out["success"].data_ptr(), out["best"].data_ptr()
        t = B.server_submit(self.h, r)
        self._keep[t] = (ins, out)
        return t

    def step(self, wait: bool = False) -> int:
        """One scheduling step; with wait, raises binding.DseedTimeout when the
        oldest round is not done within the wait limit (it stays in flight)."""
        return B.server_step(self.h, wait)

    def set_wait_limit(self, seconds: float):
        B.server_set_wait_limit(self.h, seconds)

    def poll(self, ticket: int):
        return B.server_poll(self.h, ticket)

    def result(self, ticket: int) -> dict:
        return self._keep[ticket][1]

    def release(self, ticket: int):
        self._keep.pop(ticket, None)

    def stats(self) -> B.ServerStats:
        return B.server_stats(self.h)

    def drain(self, tickets: Sequence[int], timeout_s: float = 600.0):
        t0 = time.monotonic()
        pending = set(tickets)
        while pending:
            self.step(wait=True)
            pending = {t for t in pending if self.poll(t)[0] not in (2, -1)}
            if time.monotonic() - t0 > timeout_s:
                raise TimeoutError(f"{len(pending)} requests still pending")


def alloc_outputs(S: int, T: int) -> dict:
    return dict(traj=torch.empty((S, T, 7), dtype=torch.float32).pin_memory(),
                cost=torch.empty((S,), dtype=torch.float32).pin_memory(),
                success=torch.empty((S,), dtype=torch.uint8).pin_memory(),
                best=torch.empty((1,), dtype=torch.int32).pin_memory())


def alloc_output_views(shapes: Sequence[tuple]) -> List[dict]:
    """Output buffers of requests of the given (S, T), as views of four pinned
    arrays (one allocation each instead of four per request)."""
    n_traj = sum(S * T * 7 for S, T in shapes)
    n_seed = sum(S for S, _ in shapes)
    traj = torch.empty(n_traj, dtype=torch.float32).pin_memory()
    cost = torch.empty(n_seed, dtype=torch.float32).pin_memory()
    succ = torch.empty(n_seed, dtype=torch.uint8).pin_memory()
    best = torch.empty(max(len(shapes), 1), dtype=torch.int32).pin_memory()
    outs, a, b = [], 0, 0
    for i, (S, T) in enumerate(shapes):
        outs.append(dict(traj=traj[a:a + S * T * 7].view(S, T, 7), cost=cost[b:b + S], success=succ[b:b + S],
                         best=best[i:i + 1]))
        a += S * T * 7
        b += S
    return outs


# ---------------------------------------------------------------------------- trace replay

def run_trace(server: Server, wl: ServingWorkload, arrivals: Optional[np.ndarray], timeout_s: float = 600.0) -> dict:
    """Replay the requests of `wl` at the given arrival times (seconds from the
    start; None = all at once).  Returns latencies (s) per request, throughput
    (plans/s over the span from the first arrival to the last completion), the
    success rate over all seeds and the server's stats."""
    n = len(wl.requests)
    pinned_in = {}
    for (p, S, T) in set(wl.requests):
        pr = wl.problems[p]
        pinned_in[(p, S, T)] = dict(q=torch.as_tensor(pr.q_start).pin_memory(),
                                    g=torch.as_tensor(pr.goal).pin_memory(),
                                    s=torch.as_tensor(pr.seeds[(S, T)]).pin_memory())
    # pinned output buffers for every request, views of four pinned arrays made
    # before the clock starts (pinned allocations are far slower than the copies)
    free_out: Dict[tuple, list] = {}
    for (S, T), out in zip([(S, T) for (_, S, T) in wl.requests], alloc_output_views(
            [(S, T) for (_, S, T) in wl.requests])):
        free_out.setdefault((S, T), []).append(out)

    def get_out(S, T):
        lst = free_out.setdefault((S, T), [])
        return lst.pop() if lst else alloc_outputs(S, T)

    arr = np.zeros(n) if arrivals is None else np.asarray(arrivals, np.float64)
    tickets = [None] * n
    lat = np.full(n, np.nan)
    succ_seeds = 0
    tot_seeds = 0
    solved = 0
    open_t = {}
    i = 0
    done = 0
    t0 = time.monotonic()
    t_first = None
    t_last = t0
    while done < n:
        now = time.monotonic() - t0
        while i < n and arr[i] <= now:
            p, S, T = wl.requests[i]
            out = get_out(S, T)
            tickets[i] = server.submit_pinned(wl.problems[p].scene, pinned_in[(p, S, T)], out)
            open_t[tickets[i]] = (i, S, T, out)
            if t_first is None:
                t_first = time.monotonic()
            i += 1
        nd = server.step(wait=False)
        if nd:
            for t in list(open_t.keys()):
                st, ts, td = server.poll(t)
                if st == 2 or st == -1:
                    k, S, T, out = open_t.pop(t)
                    lat[k] = td - min(ts, t0 + arr[k])        # from the request's arrival
                    if st == 2:
                        sc = out["success"].numpy()
                        succ_seeds += int(sc.sum())
                        tot_seeds += S
                        solved += int(out["best"][0] >= 0)
                    server.release(t)
                    free_out[(S, T)].append(out)
                    done += 1
                    t_last = time.monotonic()
        if time.monotonic() - t0 > timeout_s:
            raise TimeoutError(f"trace did not finish: {done} of {n} done")
        if nd == 0 and i < n and not open_t:
            # idle until the next arrival
            time.sleep(max(0.0, min(arr[i] - (time.monotonic() - t0), 0.001)))
    span = t_last - (t_first if t_first is not None else t0)
    st = server.stats()
    return dict(latency_s=lat, plans_per_s=n / span if span > 0 else float("inf"), span_s=span,
                seed_success=succ_seeds / max(tot_seeds, 1), problems_solved=solved / n,
                rounds=int(st.rounds), arena_peak=int(st.arena_peak))


def poisson_arrivals(n: int, rate: float, seed: int = 0) -> np.ndarray:
    rng = np.random.default_rng(9000 + seed)
    return np.cumsum(rng.exponential(1.0 / rate, size=n))


def summarize(res: dict) -> dict:
    lat = res["latency_s"]
    return dict(plans_per_s=res["plans_per_s"], p50_ms=float(np.nanpercentile(lat, 50) * 1e3),
                p99_ms=float(np.nanpercentile(lat, 99) * 1e3), mean_ms=float(np.nanmean(lat) * 1e3),
                seed_success=res["seed_success"], problems_solved=res["problems_solved"], rounds=res["rounds"])


def run_trace_seeded(server: Server, problems: Sequence[tuple], requests: Sequence[int], arrivals: Optional[np.ndarray],
                     propose: Callable[[List[int]], torch.Tensor], max_group: int = 64,
                     timeout_s: float = 600.0) -> dict:
    """Replay requests whose seeds are proposed on the GPU when they arrive
    (the learned seeding): problems[p] = (scene_id, q_start [7], goal [7]);
    requests[i] = problem index, or (problem index, horizon T) for a mix of
    horizons.  Arrived requests are grouped (up to max_group; with horizons,
    the arrived requests of the oldest one's horizon), propose(problem indices)
    -- propose(problem indices, T) with horizons -- enqueues their seeds
    [g][S][T][7] on the current stream (overlapping the server's own stream),
    the seeds are copied to pinned host memory, and each request is submitted
    once its copy has landed.  Latency runs from the arrival to the server's completion, so
    it includes the proposal.  Pinned buffers come from pools (allocating
    pinned memory can synchronise the device)."""
    n = len(requests)
    mixed = len(requests) > 0 and isinstance(requests[0], tuple)
    prob = (lambda k: requests[k][0]) if mixed else (lambda k: requests[k])
    arr = np.zeros(n) if arrivals is None else np.asarray(arrivals, np.float64)
    pin = {p: (torch.as_tensor(np.asarray(q, np.float32)).pin_memory(),
               torch.as_tensor(np.asarray(g, np.float32)).pin_memory()) for p, (_, q, g) in enumerate(problems)}
    lat = np.full(n, np.nan)
    waiting: List[int] = []
    props: List[tuple] = []
    open_t: Dict[int, tuple] = {}
    free_out: Dict[tuple, list] = {}
    free_blocks: Dict[tuple, list] = {}
    refs: Dict[int, list] = {}                    # id(block) -> [block, requests still using it]
    succ_seeds = tot_seeds = solved = 0
    i = done = 0
    t0 = time.monotonic()
    t_first, t_last = None, t0
    while done < n:
        now = time.monotonic() - t0
        while i < n and arr[i] <= now:
            waiting.append(i)
            if t_first is None:
                t_first = time.monotonic()
            i += 1
        if waiting and len(props) < 2:
            if mixed:
                Tg = requests[waiting[0]][1]
                grp = [k for k in waiting if requests[k][1] == Tg][:max_group]
                taken = set(grp)
                waiting = [k for k in waiting if k not in taken]
                seeds = propose([prob(k) for k in grp], Tg)
            else:
                grp, waiting = waiting[:max_group], waiting[max_group:]
                seeds = propose([prob(k) for k in grp])
            key = tuple(seeds.shape[1:])
            lst = free_blocks.setdefault(key, [])
            block = lst.pop() if lst else torch.empty((max_group,) + key, dtype=torch.float32).pin_memory()
            block[:len(grp)].copy_(seeds, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record()
            props.append((ev, grp, block))
        while props and props[0][0].query():
            _, grp, block = props.pop(0)
            refs[id(block)] = [block, len(grp)]
            S, T = int(block.shape[1]), int(block.shape[2])
            for j, k in enumerate(grp):
                p = prob(k)
                lo = free_out.setdefault((S, T), [])
                if not lo:                            # a group's worth of outputs in one allocation
                    lo.extend(alloc_output_views([(S, T)] * max_group))
                out = lo.pop()
                ins = dict(q=pin[p][0], g=pin[p][1], s=block[j])
                t = server.submit_pinned(problems[p][0], ins, out)
                open_t[t] = (k, S, T, out, block)
        nd = server.step(wait=False)
        if nd:
            for t in list(open_t.keys()):
                st, ts, td = server.poll(t)
                if st == 2 or st == -1:
                    k, S, T, out, block = open_t.pop(t)
                    lat[k] = td - (t0 + arr[k])
                    if st == 2:
                        succ_seeds += int(out["success"].numpy().sum())
                        tot_seeds += S
                        solved += int(out["best"][0] >= 0)
                    server.release(t)
                    free_out[(S, T)].append(out)
                    r = refs[id(block)]
                    r[1] -= 1
                    if r[1] == 0:
                        del refs[id(block)]
                        free_blocks[tuple(block.shape[1:])].append(block)
                    done += 1
                    t_last = time.monotonic()
        if time.monotonic() - t0 > timeout_s:
            raise TimeoutError(f"trace did not finish: {done} of {n} done")
        if nd == 0 and i < n and not open_t and not props and not waiting:
            time.sleep(max(0.0, min(arr[i] - (time.monotonic() - t0), 0.001)))
    span = t_last - (t_first if t_first is not None else t0)
    st = server.stats()
    return dict(latency_s=lat, plans_per_s=n / span if span > 0 else float("inf"), span_s=span,
                seed_success=succ_seeds / max(tot_seeds, 1), problems_solved=solved / n,
                rounds=int(st.rounds), arena_peak=int(st.arena_peak))
