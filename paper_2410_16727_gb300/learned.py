"""Learned seed proposal (the paper's DiffusionSeeder idea on top of the
plain optimiser): generate problems on shelf scenes, solve them with the plain
random-seed optimiser, train the conditional denoiser on the solutions
(Eq. 1, optionally weighted as in Eq. 2), then propose seeds by DDIM and
refine them with a few optimiser iterations.  The plain optimiser stays both
the fallback and the arbiter of success (tested by the same kernels).

Data handling (batch assembly, repetition of per-problem inputs) uses PyTorch
indexing on the device; every numeric step of the method -- the optimiser,
the ESDF and occupancy, normalisation, the network, DDIM -- runs in libdseed.
"""
from __future__ import annotations

import dataclasses
import math
import time
from typing import Optional

import numpy as np
import torch

from . import api
from . import binding as B
from . import denoiser as DN
from . import inputs as I
from . import netspec as NS

OCC_GRID = I.Grid((-0.30, -0.64, -0.14), 0.04, (32, 32, 32))    # same box as the shelf ESDF grid
# 32^3 occupancy boxes per scene family: the shelf box above; the clutter workspace's
# 1.28 m cube (same box as the clutter ESDF grid), which also holds the serving pool's scenes
OCC_GRIDS = {"shelf": OCC_GRID, "clutter": I.Grid((-0.64, -0.64, -0.14), 0.04, (32, 32, 32))}
RES_SCALE = 4.0    # diffused quantity: RES_SCALE * (normalised trajectory - straight joint path)


def _nn(name, *a):
    B.nn(name, *a)


@dataclasses.dataclass
class ProblemSet:
    """Problems on generated scenes (device tensors)."""
    cuboids: list
    grids: list
    scene_of_problem: torch.Tensor    # [P] int32
    q_start: torch.Tensor             # [P][7]
    q_goal: torch.Tensor              # [P][7]
    goal: torch.Tensor                # [P][7]
    occ: torch.Tensor                 # [n_scenes][32^3]
    table: B.SceneTable = None        # the scenes' ESDFs on the device
    T: int = 32                       # horizon the problems are planned at
    iters: int = 100                  # iterations of the plain method on them
    kind: str = "shelf"


def make_problems(planner: api.Planner, n_scenes: int, per_scene: int, seed: int, kind: str = "shelf",
                  T: Optional[int] = None) -> ProblemSet:
    """per_scene problems on each of n_scenes generated scenes.  shelf: the
    batched workload's shelf scenes (128^3 ESDF at 1 cm), T = 32, 100
    iterations; clutter: the stress workload's dense-clutter scenes (200
    cuboids, 256^3 ESDF at 5 mm), T = 64, 200 iterations.  Each family's
    random streams are keyed apart from the benchmark workloads' own."""
    if kind == "shelf":
        base, cid, T, iters = I.WORKLOADS["batched"], 40 + seed, T or 32, 100
    elif kind == "clutter":
        base, cid, T, iters = I.WORKLOADS["stress"], 60 + seed, T or 64, 200
    else:
        raise ValueError(kind)
    spec = I.WorkloadSpec("learned-" + kind, cid, n_scenes, n_scenes * per_scene, 1, T, iters, base.scene, base.grid)
    cub, grids = I.make_scenes(spec)
    planner.set_scenes(cub, grids)
    cf, pf = api.device_workload_fns(planner)
    wl = I.build_workload(spec, cub, grids, cf, pf, S=1)
    occ = occupancy(planner, cub, OCC_GRIDS[kind])
    dev = planner.device
    return ProblemSet(cub, grids, torch.as_tensor(wl.scene_of_problem).to(dev), torch.as_tensor(wl.q_start).to(dev),
                      torch.as_tensor(wl.q_goal).to(dev), torch.as_tensor(wl.goal).to(dev), occ, planner.table,
                      T=T, iters=iters, kind=kind)


def occupancy(planner: api.Planner, cuboids, grid: I.Grid = OCC_GRID) -> torch.Tensor:
    """32^3 occupancy of each scene over a workspace box (default: the shelf
    box): the ESDF at 4 cm voxels thresholded at 0 (1 inside a cuboid)."""
    dev = planner.device
    cts = [torch.as_tensor(c).to(dev).reshape(-1, 6) for c in cuboids]
    esdf = B.scene_build_esdf_batch(cts, [grid] * len(cts))
    phi = torch.stack(esdf).reshape(len(cts), -1).contiguous()
    occ = torch.empty_like(phi)
    _nn("clamp_affine", phi, -1e6, 0.0, 0.0, 1.0, occ, phi.numel())
    return occ


_AFFINE_CACHE: dict = {}


def _limits_affine(robot: I.Robot, dev, inverse: bool) -> torch.Tensor:
    """FiLM vector [1][14] (scale, shift) mapping joints to [-1, 1] by the
    mechanical limits (App. A.4), or back (cached per device: no host copy
    once built, so the proposal can be captured in a CUDA graph)."""
    key = (robot.limits.tobytes(), str(dev), inverse)
    t = _AFFINE_CACHE.get(key)
    if t is not None:
        return t
    lo = robot.limits[:, 0].astype(np.float64)
    hi = robot.limits[:, 1].astype(np.float64)
    if not inverse:
        sc, sh = 2.0 / (hi - lo), -2.0 * lo / (hi - lo) - 1.0
    else:
        sc, sh = (hi - lo) / 2.0, lo + (hi - lo) / 2.0
    t = torch.tensor(np.concatenate([sc, sh])[None], dtype=torch.float32, device=dev)
    _AFFINE_CACHE[key] = t
    return t


def normalise(robot, q: torch.Tensor, inverse: bool = False) -> torch.Tensor:
    rows = q.numel() // 7
    out = torch.empty_like(q)
    _nn("film", q.contiguous(), _limits_affine(robot, q.device, inverse), 1, rows, 7, out, None, None, None, 0)
    return out


def linear_path_weights(T: int, D: int) -> np.ndarray:
    """Interpolation matrix [2D][T*D] of the straight start-goal path:
    [q_s, q_g] @ W puts waypoint t (t = 1..T) at q_s + (t/T)(q_g - q_s)."""
    tau = np.arange(1, T + 1, dtype=np.float64) / T
    W = np.zeros((2 * D, T * D), np.float32)
    for t in range(T):
        for d in range(D):
            W[d, t * D + d] = 1.0 - tau[t]
            W[D + d, t * D + d] = tau[t]
    return W


def linear_path(qs_n: torch.Tensor, qg_n: torch.Tensor, T: int) -> torch.Tensor:
    """Straight start-goal joint path [N][T][7] (waypoint t at fraction t/T,
    t = 1..T, the start itself excluded like the optimiser's waypoints), from
    normalised start and goal configurations: one GEMM of [q_s, q_g] against
    the constant interpolation matrix [14][T*7]."""
    N, D = qs_n.shape
    key = ("lin", T, D, str(qs_n.device))
    W = _AFFINE_CACHE.get(key)
    if W is None:
        W = _AFFINE_CACHE[key] = torch.from_numpy(linear_path_weights(T, D)).to(qs_n.device)
    A = torch.cat([qs_n, qg_n], 1).contiguous()
    out = torch.empty((N, T, D), dtype=torch.float32, device=qs_n.device)
    _nn("gemm_f32", 0, 0, N, T * D, 2 * D, 1.0, A, 2 * D, W, T * D, 0.0, out, T * D, None)
    return out


def resample_weights(T0: int, T1: int, D: int):
    """Interpolation weights of `resample`: (Wx [T0*D][T1*D], Wq [D][T1*D]) so
    that x @ Wx + q0 @ Wq holds, at output waypoint j (fraction j / T1), the
    linear interpolation in time between the input waypoints around it (input
    waypoint k at fraction k / T0, the start q0 at fraction 0)."""
    Wx = np.zeros((T0 * D, T1 * D), np.float32)
    Wq = np.zeros((D, T1 * D), np.float32)
    for j in range(1, T1 + 1):
        u = j * T0 / T1                       # position in input waypoints (the start at 0)
        k0 = min(int(math.floor(u)), T0)
        f = u - k0
        for d in range(D):
            col = (j - 1) * D + d
            if k0 == 0:
                Wq[d, col] = 1.0 - f
            else:
                Wx[(k0 - 1) * D + d, col] += 1.0 - f
            if f > 0.0:
                Wx[k0 * D + d, col] += f
    return Wx, Wq


def resample(x: torch.Tensor, q0: torch.Tensor, T1: int) -> torch.Tensor:
    """Trajectories x [N][T0][7], whose waypoint k sits at fraction k / T0 of a
    path that starts at q0 [N][7] (fraction 0), resampled by linear
    interpolation in time to T1 waypoints at fractions j / T1, j = 1..T1:
    [N][T1][7].  Two GEMMs against constant interpolation weights (the
    waypoints' share, then the start's, accumulated)."""
    N, T0, D = x.shape
    if T1 == T0:
        return x
    key = ("resample", T0, T1, D, str(x.device))
    W = _AFFINE_CACHE.get(key)
    if W is None:
        Wx, Wq = resample_weights(T0, T1, D)
        W = _AFFINE_CACHE[key] = (torch.from_numpy(Wx).to(x.device), torch.from_numpy(Wq).to(x.device))
    out = torch.empty((N, T1, D), dtype=torch.float32, device=x.device)
    _nn("gemm_f32", 0, 0, N, T1 * D, T0 * D, 1.0, x.contiguous(), T0 * D, W[0], T1 * D, 0.0, out, T1 * D, None)
    _nn("gemm_f32", 0, 0, N, T1 * D, D, 1.0, q0.contiguous(), D, W[1], T1 * D, 1.0, out, T1 * D, None)
    return out


def to_residual(x_n: torch.Tensor, lin: torch.Tensor) -> torch.Tensor:
    out = torch.empty_like(x_n)
    _nn("axpby", RES_SCALE, x_n.contiguous(), -RES_SCALE, lin.contiguous(), out, x_n.numel())
    return out


def from_residual(r: torch.Tensor, lin: torch.Tensor) -> torch.Tensor:
    out = torch.empty_like(r)
    _nn("axpby", 1.0, lin.contiguous(), 1.0 / RES_SCALE, r.contiguous(), out, r.numel())
    return out


def random_seeds(ps: ProblemSet, robot: I.Robot, S: int, T: int, seed: int, p0: int = 0,
                 p1: Optional[int] = None) -> np.ndarray:
    """The plain method's seeds (linear start-goal interpolation plus noise,
    clipped to the limits) of problems p0..p1-1: [P][S][T][7]."""
    p1 = ps.q_start.shape[0] if p1 is None else p1
    qs, qg = ps.q_start[p0:p1].cpu().numpy(), ps.q_goal[p0:p1].cpu().numpy()
    return np.stack([I.make_seeds(I._rng(77 + seed, p0 + i, 3), qs[i], qg[i], S, T, robot.limits)
                     for i in range(p1 - p0)])


def solve(planner: api.Planner, ps: ProblemSet, seeds, iters: int, chunk: int = 256):
    """Plan every problem with the given seeds [P][S][T][7] for `iters`
    iterations; returns the output dict (device tensors, concatenated)."""
    P, S, T = seeds.shape[0], seeds.shape[1], seeds.shape[2]
    opt = I.OptParams(iters=iters)
    outs = []
    seeds_t = torch.as_tensor(seeds).to(planner.device) if not isinstance(seeds, torch.Tensor) else seeds
    for p0 in range(0, P, chunk):
        p1 = min(P, p0 + chunk)
        batch = api.Batch(ps.q_start[p0:p1], ps.goal[p0:p1], ps.scene_of_problem[p0:p1], ps.table, S, T,
                          planner.cost, opt, planner.device)
        outs.append({k: v.clone() for k, v in planner.plan(batch, seeds_t[p0:p1].contiguous()).items()})
    return {k: torch.cat([o[k] for o in outs]) for k in outs[0]}


@dataclasses.dataclass
class Dataset:
    x0: torch.Tensor       # [M][T][7] scaled residuals of the normalised solutions from the straight path
    qs: torch.Tensor       # [M][7] normalised starts
    qg: torch.Tensor       # [M][7] normalised goal configurations
    goal: torch.Tensor     # [M][7]
    scene: torch.Tensor    # [M] int64 index into occ
    occ: torch.Tensor      # [n_scenes][32^3]
    weight: torch.Tensor   # [M] 1 + alpha * 1(non-linear solution)


def build_dataset(planner: api.Planner, robot: I.Robot, ps: ProblemSet, S: int = 64, iters: Optional[int] = None,
                  alpha: float = 4.0, nonlinear_rad: float = 0.3, seed: int = 0, chunk: int = 256,
                  reverse: bool = True, T_net: int = 32) -> Dataset:
    """Solve every problem with S random seeds at the problems' horizon (ps.T,
    ps.iters iterations unless given); keep the best successful trajectory of
    each solved problem.  A solution that leaves the straight start-goal joint
    line by more than `nonlinear_rad` counts as non-linear and gets weight
    1 + alpha (the paper up-weights solutions a linear seed does not reach,
    Eq. 2).  With reverse, every solution is also added run backwards (App. A.4
    swaps start and goal): start = its last waypoint, goal = the original start
    configuration and its flange pose, waypoints y_{T-1}, ..., y_1, q_start.
    Solutions are resampled to the network's horizon T_net (for T = 64 and
    T_net = 32: every second waypoint)."""
    T = ps.T
    iters = ps.iters if iters is None else iters
    P = ps.q_start.shape[0]
    opt = I.OptParams(iters=iters)
    keeps, trajs = [], []
    for p0 in range(0, P, chunk):
        p1 = min(P, p0 + chunk)
        seeds = torch.as_tensor(random_seeds(ps, robot, S, T, seed, p0, p1)).to(planner.device)
        batch = api.Batch(ps.q_start[p0:p1], ps.goal[p0:p1], ps.scene_of_problem[p0:p1], ps.table, S, T,
                          planner.cost, opt, planner.device)
        out = planner.plan(batch, seeds)
        best = out["best"].long()
        keep = torch.nonzero(best >= 0).squeeze(1)
        keeps.append(keep + p0)
        trajs.append(out["traj"][keep, best[keep]].clone())
    keep = torch.cat(keeps)
    traj = torch.cat(trajs)                                        # [M][T][7]
    qs, qg = ps.q_start[keep], ps.q_goal[keep]
    goal = ps.goal[keep]
    scene = ps.scene_of_problem[keep]
    if reverse:
        rq_s = traj[:, -1].contiguous()
        rtraj = torch.cat([traj[:, :-1].flip(1), qs[:, None]], 1)
        rgoal = planner.fk(qs)
        traj = torch.cat([traj, rtraj])
        qs, qg = torch.cat([qs, rq_s]), torch.cat([qg, ps.q_start[keep]])
        goal = torch.cat([goal, rgoal])
        scene = torch.cat([scene, scene])
    tt = torch.arange(1, T + 1, device=planner.device, dtype=torch.float32)[None, :, None] / T
    lin = qs[:, None, :] + tt * (qg - qs)[:, None, :]
    dev = (traj - lin).abs().amax(dim=(1, 2))
    weight = 1.0 + alpha * (dev > nonlinear_rad).float()
    qs_n, qg_n = normalise(robot, qs.contiguous()), normalise(robot, qg.contiguous())
    traj = resample(traj.contiguous(), qs.contiguous(), T_net)
    x0 = to_residual(normalise(robot, traj.contiguous()), linear_path(qs_n, qg_n, T_net))
    return Dataset(x0, qs_n, qg_n, goal.contiguous(), scene.long(), ps.occ, weight.contiguous())


class GraphStep:
    """One training step's kernels (noising, forward, loss, backward) captured
    once in a CUDA graph over static input buffers, then replayed: the launch
    sequence of a fixed batch size never changes, so replaying it removes the
    host cost of issuing ~400 launches per step."""

    def __init__(self, net: DN.Denoiser, batch: int, weighted: bool, fk_robot: Optional[B.Robot] = None):
        s, dev = net.spec, net.dev
        self.net = net
        self.x0 = torch.zeros((batch, s.T, s.D), device=dev)
        self.qs = torch.zeros((batch, s.D), device=dev)
        self.qg = torch.zeros((batch, s.D), device=dev)
        self.goal = torch.zeros((batch, 7), device=dev)
        self.goal[:, 3] = 1.0
        self.occ = torch.zeros((batch, s.occ_n ** 3), device=dev)
        self.k = torch.zeros((batch,), dtype=torch.int32, device=dev)
        self.eps = torch.zeros((batch, s.T, s.D), device=dev)
        self.w = torch.ones((batch,), device=dev) if weighted else None
        args = (self.x0, self.qs, self.qg, self.goal, self.occ, self.k, self.eps, self.w)

        def step():
            # Eq. 2 on the robot needs the samples' straight paths (one GEMM, inside the graph)
            fk = None if fk_robot is None else (fk_robot, linear_path(self.qs, self.qg, s.T), RES_SCALE)
            return net.loss_and_grad(*args, fk=fk)

        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):                  # warm-up outside the capture
            step()
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        net.grads.zero_()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self.loss = step()
        torch.cuda.synchronize()
        net.grads.zero_()

    def run(self):
        self.graph.replay()
        return self.loss


def train(net: DN.Denoiser, data: Dataset, steps: int, batch: int = 256, lr: float = 3e-4, seed: int = 0,
          log_every: int = 0, weighted: bool = True, graph: bool = True, fk_robot: Optional[B.Robot] = None):
    """DDPM training (Eq. 1 / Eq. 2 weights) with Adam and a cosine learning
    rate; returns the loss curve [(step, loss)].  With fk_robot the error is
    measured on points on that robot's sphere surfaces (Eq. 2), else on the joints (Eq. 1)."""
    g = torch.Generator(device=data.x0.device)
    g.manual_seed(seed)
    M = data.x0.shape[0]
    losses = []
    gs = GraphStep(net, batch, weighted, fk_robot) if graph else None
    for it in range(steps):
        idx = torch.randint(0, M, (batch,), device=data.x0.device, generator=g)
        k = torch.randint(0, net.spec.K, (batch,), device=data.x0.device, generator=g, dtype=torch.int32)
        eps = torch.randn((batch, net.spec.T, net.spec.D), device=data.x0.device, generator=g)
        if gs is not None:
            gs.x0.copy_(data.x0[idx])
            gs.qs.copy_(data.qs[idx])
            gs.qg.copy_(data.qg[idx])
            gs.goal.copy_(data.goal[idx])
            gs.occ.copy_(data.occ[data.scene[idx]])
            gs.k.copy_(k)
            gs.eps.copy_(eps)
            if weighted:
                gs.w.copy_(data.weight[idx])
            loss = gs.run()
        else:
            qs_b, qg_b = data.qs[idx].contiguous(), data.qg[idx].contiguous()
            fk = None if fk_robot is None else (fk_robot, linear_path(qs_b, qg_b, net.spec.T), RES_SCALE)
            loss = net.loss_and_grad(data.x0[idx].contiguous(), qs_b, qg_b, data.goal[idx].contiguous(),
                                     data.occ[data.scene[idx]].contiguous(), k, eps,
                                     data.weight[idx].contiguous() if weighted else None, fk=fk)
        cos = 0.5 * (1 + math.cos(math.pi * it / max(steps, 1)))
        net.adam_step(lr=lr * (0.1 + 0.9 * cos))
        if log_every and (it % log_every == 0 or it == steps - 1):
            losses.append((it, float(loss)))
    return losses


def _propose_core(net: DN.Denoiser, robot: I.Robot, q_start, q_goal, goal, occ, noise, rows, steps: int,
                  bf16: bool, check: bool, guide_ctx=None, out_T: Optional[int] = None) -> torch.Tensor:
    qs = normalise(robot, q_start.contiguous())
    qg = normalise(robot, q_goal.contiguous())
    lin = linear_path(qs, qg, net.spec.T)[rows.long()].contiguous()
    guide = None
    if guide_ctx is not None:
        planner, table, scene_of_problem, gd = guide_ctx
        guide = _guide_fn(robot, planner, table, q_start, goal, scene_of_problem, lin,
                          noise.shape[0] // q_start.shape[0], net.spec.T, gd)
    r = net.ddim_sample(qs, qg, goal.contiguous(), occ.contiguous(), noise, steps=steps, bf16=bf16,
                        sample_problem=rows, check=check, guide=guide)
    x = from_residual(r, lin)
    _nn("clamp_affine", x, 1.0, 0.0, -1.0, 1.0, x, x.numel())
    P, S = q_start.shape[0], noise.shape[0] // q_start.shape[0]
    q = normalise(robot, x, inverse=True)
    if out_T is not None and out_T != net.spec.T:
        # the network's horizon resampled to the requested one (the start configuration at fraction 0)
        q = resample(q.view(P * S, net.spec.T, net.spec.D), q_start[rows.long()], out_T)
    return q.view(P, S, -1, net.spec.D)


def propose_for(net: DN.Denoiser, robot: I.Robot, q_start: torch.Tensor, q_goal: torch.Tensor, goal: torch.Tensor,
                occ: torch.Tensor, S: int, steps: int = 10, seed: int = 0, bf16: bool = True,
                out_T: Optional[int] = None) -> torch.Tensor:
    """DDIM proposals for P problems given as device tensors (q_start, q_goal,
    goal [P][7], occupancy rows [P][32^3]): S seed trajectories per problem,
    [P][S][T][7] in joint space.  DDIM generates the scaled residual from the
    straight start-goal path, which is added back; the result is clipped to
    the joint limits like the random seeds, then un-normalised, and resampled
    in time to out_T waypoints when that differs from the network's T."""
    P = q_start.shape[0]
    dev = q_start.device
    g = torch.Generator(device=dev)
    g.manual_seed(1000 + seed)
    noise = torch.randn((P * S, net.spec.T, net.spec.D), device=dev, generator=g)
    rows = torch.arange(P, device=dev, dtype=torch.int32).repeat_interleave(S)
    return _propose_core(net, robot, q_start, q_goal, goal, occ, noise, rows, steps, bf16, True, out_T=out_T)


@dataclasses.dataclass
class Guidance:
    """Cost-gradient guidance of the DDIM sampler (the paper's appendix, Eq. 5):
    after every denoising step that reaches a step index below k_guide, except
    the last one, the sampled trajectories take n_grad descent steps on the
    plan cost of their own problem (collision, smoothness, goal, limits; the
    cost kernel the optimiser uses): x <- x - clip(alpha dC/dx, +-cap), with
    dC/dx = dC/dq dq/dx through the residual and limit normalisation.  The
    paper prints the step as +alpha grad C with alpha = 1 on cuRobo's cost
    scale; read as a descent step, alpha here is on this cost's scale and each
    step is capped per entry (cap, in diffused units)."""
    k_guide: int = 60
    n_grad: int = 20
    alpha: float = 1e-3
    cap: float = 0.02


def _guide_fn(robot: I.Robot, planner: api.Planner, table: B.SceneTable, q_start, goal, scene_of_problem,
              lin: torch.Tensor, S: int, T: int, gd: Guidance):
    P = q_start.shape[0]
    dev = q_start.device
    batch = api.Batch(q_start, goal, scene_of_problem, table, S, T, planner.cost, None, dev)
    # dq/dx per joint: (hi - lo) / 2 (un-normalising) / RES_SCALE, as a FiLM row (scale, shift 0);
    # cached, so that no host copy happens inside a graph capture
    key = ("jac", robot.limits.tobytes(), str(dev))
    jac = _AFFINE_CACHE.get(key)
    if jac is None:
        lo = robot.limits[:, 0].astype(np.float64)
        hi = robot.limits[:, 1].astype(np.float64)
        jac = _AFFINE_CACHE[key] = torch.tensor(np.concatenate([(hi - lo) / 2.0 / RES_SCALE, np.zeros(7)])[None],
                                                dtype=torch.float32, device=dev)

    def guide(i, k_reached, x, last):
        if last or k_reached < 0 or k_reached >= gd.k_guide or gd.alpha == 0.0:
            return x
        for _ in range(gd.n_grad):
            xn = from_residual(x, lin)
            _nn("clamp_affine", xn, 1.0, 0.0, -1.0, 1.0, xn, xn.numel())
            q = normalise(robot, xn, inverse=True)
            _, gq = B.cost_grad(planner.robot, batch.desc, batch.pr, q.view(P, S, T, 7))
            gx = torch.empty_like(x)
            _nn("film", gq.view(-1, 7), jac, 1, P * S * T, 7, gx, None, None, None, 0)
            step = torch.empty_like(x)
            _nn("clamp_affine", gx, -gd.alpha, 0.0, -gd.cap, gd.cap, step, x.numel())
            out = torch.empty_like(x)
            _nn("axpby", 1.0, x, 1.0, step, out, x.numel())
            x = out
        return x

    guide.batch = batch            # keeps the descriptors' tensors alive
    return guide


def propose_guided(net: DN.Denoiser, robot: I.Robot, planner: api.Planner, ps: ProblemSet, S: int,
                   steps: int = 10, guidance: Optional[Guidance] = None, seed: int = 0) -> torch.Tensor:
    """Cost-gradient-guided DDIM proposals (Guidance) for every problem of a
    problem set: [P][S][T][7].  With alpha = 0 they equal propose()."""
    gd = guidance or Guidance()
    P = ps.q_start.shape[0]
    dev = ps.q_start.device
    T, D = net.spec.T, net.spec.D
    g = torch.Generator(device=dev)
    g.manual_seed(1000 + seed)
    noise = torch.randn((P * S, T, D), device=dev, generator=g)
    rows = torch.arange(P, device=dev, dtype=torch.int32).repeat_interleave(S)
    occ = ps.occ[ps.scene_of_problem.long()].contiguous()
    return _propose_core(net, robot, ps.q_start, ps.q_goal, ps.goal, occ, noise, rows, steps, True, True,
                         guide_ctx=(planner, ps.table, ps.scene_of_problem, gd))


class ProposalGraph:
    """DDIM proposals for up to G problems captured once as a CUDA graph over
    static buffers: the launch sequence of a fixed group size never changes,
    so a replay replaces the host cost of issuing every kernel of the U-Net at
    every step (a serving loop proposes for each group of arrivals).  Call with
    g <= G problems; rows past g compute on stale inputs and are not returned."""

    def __init__(self, net: DN.Denoiser, robot: I.Robot, G: int, S: int, steps: int, seed: int = 0,
                 guidance: Optional[Guidance] = None, planner: Optional[api.Planner] = None,
                 table: Optional[B.SceneTable] = None, out_T: Optional[int] = None):
        dev = net.dev
        s = net.spec
        self.G, self.S, self.net = G, S, net
        self.q_start = torch.zeros((G, 7), device=dev)
        self.q_goal = torch.zeros((G, 7), device=dev)
        self.goal = torch.zeros((G, 7), device=dev)
        self.goal[:, 3] = 1.0
        self.scene = torch.zeros((G,), dtype=torch.int32, device=dev)
        self.occ = torch.zeros((G, s.occ_n ** 3), device=dev)
        self.noise = torch.zeros((G * S, s.T, s.D), device=dev)
        self.rows = torch.arange(G, device=dev, dtype=torch.int32).repeat_interleave(S)
        self.gen = torch.Generator(device=dev)
        self.gen.manual_seed(2000 + seed)
        ctx = (planner, table, self.scene, guidance) if guidance is not None else None
        args = (net, robot, self.q_start, self.q_goal, self.goal, self.occ, self.noise, self.rows, steps, True, False,
                ctx, out_T)
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):                  # warm-up outside the capture (weight caches, constants)
            _propose_core(*args)
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        self.weights = net._tc_weights()              # the buffers the graph reads; kept alive here
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self.out = _propose_core(*args)
        torch.cuda.synchronize()

    def __call__(self, q_start, q_goal, goal, occ, scene: Optional[torch.Tensor] = None) -> torch.Tensor:
        """Seeds [g][S][T][7] for g <= G problems; scene (int32 [g], indices
        into the captured scene table) is needed with guidance."""
        g = q_start.shape[0]
        if self.net._tc_weights() is not self.weights:
            raise RuntimeError("the denoiser's parameters changed after capture: build a new ProposalGraph")
        if g > self.G:
            raise ValueError(f"group of {g} problems exceeds the captured size {self.G}")
        self.q_start[:g].copy_(q_start)
        self.q_goal[:g].copy_(q_goal)
        self.goal[:g].copy_(goal)
        if scene is not None:
            self.scene[:g].copy_(scene)
        self.occ[:g].copy_(occ)
        torch.randn(self.noise.shape, device=self.noise.device, generator=self.gen, out=self.noise)
        self.graph.replay()
        return self.out[:g]

    def check(self):
        self.net.check_tc()


class ProposalGraphs:
    """Several captured group sizes; a group of g problems replays the
    smallest graph with G >= g (less padded work for small groups)."""

    def __init__(self, net: DN.Denoiser, robot: I.Robot, sizes, S: int, steps: int, seed: int = 0, **kw):
        self.graphs = [ProposalGraph(net, robot, G, S, steps, seed + i, **kw) for i, G in enumerate(sorted(sizes))]

    def __call__(self, q_start, q_goal, goal, occ, scene: Optional[torch.Tensor] = None) -> torch.Tensor:
        g = q_start.shape[0]
        for pg in self.graphs:
            if g <= pg.G:
                return pg(q_start, q_goal, goal, occ, scene)
        raise ValueError(f"group of {g} problems exceeds the largest captured size {self.graphs[-1].G}")

    def check(self):
        self.graphs[0].check()


def propose(net: DN.Denoiser, robot: I.Robot, ps: ProblemSet, S: int, steps: int = 10, seed: int = 0,
            bf16: bool = True) -> torch.Tensor:
    """DDIM proposals for every problem of a problem set at its horizon: [P][S][ps.T][7]."""
    occ = ps.occ[ps.scene_of_problem.long()]
    return propose_for(net, robot, ps.q_start, ps.q_goal, ps.goal, occ, S, steps, seed, bf16, out_T=ps.T)


def diffusion_only(planner: api.Planner, ps: ProblemSet, seeds: torch.Tensor) -> dict:
    """Planning with the proposals alone (the paper's diffusion-only mode, App.
    Table 8): per problem the proposal with the smallest translation error is
    the plan; solved when that trajectory passes the success test (no
    optimiser iterations)."""
    P, S, T = seeds.shape[0], seeds.shape[1], seeds.shape[2]
    b = api.Batch(ps.q_start, ps.goal, ps.scene_of_problem, ps.table, S, T, planner.cost, None, planner.device)
    ok, met = B.evaluate(planner.robot, b.desc, b.pr, seeds.contiguous())
    pick = met[..., 1].argmin(dim=1)
    rows = torch.arange(P, device=seeds.device)
    return dict(problems_solved=float(ok[rows, pick].float().mean()),
                pos_err_median_mm=float(met[rows, pick, 1].median() * 1e3),
                seed_success=float(ok.float().mean()))


def evaluate(planner: api.Planner, ps: ProblemSet, seeds, iters: int) -> dict:
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out = solve(planner, ps, seeds, iters)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    return dict(problems_solved=float((out["best"] >= 0).float().mean()),
                seed_success=float(out["success"].float().mean()), plan_s=dt)


def main(argv=None):
    """Time DDIM proposals on generated shelf problems (untrained weights: the
    timing does not depend on them): python -m paper_2410_16727_gb300.learned
    --problems 512 --samples 64 --ddim-steps 10."""
    import argparse
    ap = argparse.ArgumentParser()
    ap.add_argument("--problems", type=int, default=512, help="problems (8 per scene)")
    ap.add_argument("--samples", type=int, default=64)
    ap.add_argument("--ddim-steps", type=int, default=10)
    ap.add_argument("--repeat", type=int, default=3)
    ap.add_argument("--graph", action="store_true", help="replay a captured CUDA graph")
    a = ap.parse_args(argv)
    robot = I.make_robot()
    planner = api.Planner(robot)
    ps = make_problems(planner, max(1, a.problems // 8), 8, seed=1)
    net = DN.Denoiser(NS.NetSpec(), seed=0)
    occ = ps.occ[ps.scene_of_problem.long()]
    if a.graph:
        pg = ProposalGraph(net, robot, ps.q_start.shape[0], a.samples, a.ddim_steps)
        run = lambda: pg(ps.q_start, ps.q_goal, ps.goal, occ)
    else:
        run = lambda: propose_for(net, robot, ps.q_start, ps.q_goal, ps.goal, occ, a.samples, a.ddim_steps)
    run()
    times = []
    for _ in range(a.repeat):
        torch.cuda.synchronize()
        t = time.perf_counter()
        run()
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t)
    net.check_tc()
    n = ps.q_start.shape[0] * a.samples
    print(f"DDIM proposal: {ps.q_start.shape[0]} problems x {a.samples} samples = {n} trajectories, "
          f"{a.ddim_steps} steps: {min(times) * 1e3:.2f} ms ({min(times) / a.ddim_steps * 1e3:.2f} ms per step)")


if __name__ == "__main__":
    main()
