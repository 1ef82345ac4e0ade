"""User-level API over the C ABI: scenes, problem batches, planning and an
autograd wrapper of the cost.  Argument marshalling only; the arithmetic runs
in libdseed's kernels."""
from __future__ import annotations

from typing import List, Optional, Sequence

import numpy as np
import torch

from . import binding as B
from . import inputs as I


class Batch:
    """Device copies of a batch of problems plus the C descriptors that point at them."""

    def __init__(self, q_start, goal, scene_of_problem, scenes: B.SceneTable, S: int, T: int,
                 cost: I.CostParams, opt: Optional[I.OptParams] = None, device="cuda",
                 delta_t: float = I.DELTA_T, delta_r: float = I.DELTA_R):
        dev = torch.device(device)
        self.q_start = _to(q_start, torch.float32, dev)
        self.goal = _to(goal, torch.float32, dev)
        self.scene_of_problem = _to(scene_of_problem, torch.int32, dev)
        self.scenes = scenes
        self.P = int(self.q_start.shape[0])
        self.S, self.T = int(S), int(T)
        self.desc = B.plan_desc(self.P, self.S, self.T, cost, opt, delta_t, delta_r)
        self.pr = B.make_problems(self.q_start, self.goal, self.scene_of_problem, scenes)
        self.device = dev


def _to(a, dtype, dev):
    if isinstance(a, torch.Tensor):
        return a.to(device=dev, dtype=dtype, non_blocking=True).contiguous()
    return torch.as_tensor(np.ascontiguousarray(a)).to(device=dev, dtype=dtype).contiguous()


class CostFn(torch.autograd.Function):
    """cost [P][S] of x [P][S][T][7]; backward runs the adjoint kernel with the
    incoming gradient as per-trajectory scale (forward state is recomputed)."""

    @staticmethod
    def forward(ctx, x, robot: B.Robot, batch: Batch):
        x = x.contiguous()
        ctx.save_for_backward(x)
        ctx.robot, ctx.batch = robot, batch
        return B.cost(robot, batch.desc, batch.pr, x)

    @staticmethod
    def backward(ctx, grad_out):
        (x,) = ctx.saved_tensors
        _, g = B.cost_grad(ctx.robot, ctx.batch.desc, ctx.batch.pr, x,
                           grad_scale=grad_out.contiguous().to(torch.float32))
        return g, None, None


def trajectory_cost(x: torch.Tensor, robot: B.Robot, batch: Batch) -> torch.Tensor:
    return CostFn.apply(x, robot, batch)


class Planner:
    """Robot + resident scenes; plans batches of problems with the fused optimiser."""

    def __init__(self, robot: I.Robot, cost: Optional[I.CostParams] = None,
                 opt: Optional[I.OptParams] = None, device="cuda"):
        self.device = torch.device(device)
        self.robot_desc = robot
        self.robot = B.Robot(robot)
        self.cost = cost or I.CostParams()
        self.opt = opt or I.OptParams()
        self.esdfs: List[torch.Tensor] = []
        self.grids: List = []
        self.table: Optional[B.SceneTable] = None
        self._ws: Optional[torch.Tensor] = None

    # -- scenes ---------------------------------------------------------------
    def set_scenes(self, cuboids: Sequence, grids: Sequence, out: Optional[List[torch.Tensor]] = None):
        """Build (or rebuild in place, when `out` is given) one ESDF per scene on the device.
        The scenes' cuboids are kept in one packed device buffer, so that
        rebuild_scenes() can refresh them from host memory with one copy."""
        rows = [np.asarray(c, np.float32).reshape(-1, 6) if not isinstance(c, torch.Tensor)
                else c.detach().reshape(-1, 6).to(torch.float32).cpu().numpy() for c in cuboids]
        counts = [r.shape[0] for r in rows]
        packed = np.concatenate(rows) if sum(counts) else np.zeros((0, 6), np.float32)
        self.cub_packed = torch.as_tensor(np.ascontiguousarray(packed)).to(self.device)
        offs = np.concatenate([[0], np.cumsum(counts)]).astype(int)
        cts = [self.cub_packed[offs[i]:offs[i + 1]] for i in range(len(rows))]
        if out is None:
            out = [torch.empty((g.n[2], g.n[1], g.n[0]), dtype=torch.float32, device=self.device) for g in grids]
        self.esdf_batch = B.EsdfBatch(cts, grids, out)
        self.esdf_batch.run()
        self.esdfs, self.grids = list(out), list(grids)
        self.table = B.SceneTable(self.esdfs, grids, self.device)
        return self.esdfs

    def rebuild_scenes(self, packed_host: Optional[torch.Tensor] = None):
        """Rebuild every ESDF of the current scene set; with packed_host (the
        scenes' cuboids concatenated in set_scenes order, [sum n][6], pinned
        for an asynchronous copy), first refresh the cuboids with one copy."""
        if packed_host is not None:
            self.cub_packed.copy_(packed_host.view(self.cub_packed.shape), non_blocking=True)
        self.esdf_batch.run()

    # -- kinematics -----------------------------------------------------------
    def fk(self, q, spheres: bool = False):
        return B.fk(self.robot, _to(q, torch.float32, self.device).reshape(-1, 7), spheres)

    def clearance(self, scene: int, q) -> torch.Tensor:
        """min over spheres of (phi - r) of single configurations q [N][7] in one scene."""
        q = _to(q, torch.float32, self.device).reshape(-1, 7)
        N = q.shape[0]
        batch = Batch(q, torch.tensor([[0, 0, 0, 1, 0, 0, 0]], dtype=torch.float32).expand(N, 7).contiguous(),
                      torch.full((N,), scene, dtype=torch.int32), self.table, 1, 1, self.cost, None, self.device)
        _, met = B.evaluate(self.robot, batch.desc, batch.pr, q.reshape(N, 1, 1, 7))
        return met[:, 0, 0]

    # -- planning -------------------------------------------------------------
    def batch(self, q_start, goal, scene_of_problem, S: int, T: int) -> Batch:
        return Batch(q_start, goal, scene_of_problem, self.table, S, T, self.cost, self.opt, self.device)

    def workspace(self, batch: Batch) -> torch.Tensor:
        need = B.plan_workspace_bytes(batch.desc)
        if self._ws is None or self._ws.numel() < need:
            self._ws = B.alloc_workspace(need, self.device)
        return self._ws

    def plan(self, batch: Batch, seeds, out: Optional[dict] = None) -> dict:
        seeds = _to(seeds, torch.float32, self.device)
        return B.plan_batch(self.robot, batch.desc, batch.pr, seeds, self.workspace(batch), out)


def device_workload_fns(planner: Planner):
    """clearance_fn / pose_fn for inputs.build_workload computed by the CUDA path."""

    def clearance(scene, q):
        return planner.clearance(scene, q).cpu().numpy()

    def pose(q):
        return planner.fk(q).cpu().numpy()

    return clearance, pose


def plan_attempts(plan_fn, seed_fn, P: int, n_attempts: int) -> dict:
    """The attempts loop (Sec. 5.2: up to N_atp attempts, each with a new batch of
    seeds, until a problem has a successful trajectory).  plan_fn(problems,
    seeds) plans the problems (a host int64 index array) from seeds
    [len(problems)][S][T][7] and returns the plan outputs of those problems
    ("traj", "cost", "success", "best", tensors of any device); seed_fn(attempt,
    problems) draws the attempt's seeds.  Attempt a plans only the problems no
    earlier attempt solved.  Returns per problem the best trajectory of the
    attempt that solved it ("traj" [P][T][7], NaN where none did), its cost,
    "attempts" (1-based attempt that solved it, 0: none) and "solved"."""
    if P < 0 or n_attempts < 1:
        raise ValueError("P must be >= 0 and n_attempts >= 1")
    todo = np.arange(P, dtype=np.int64)
    attempts = np.zeros(P, np.int32)
    traj, cost = None, np.full(P, np.nan, np.float32)
    for a in range(1, n_attempts + 1):
        if todo.size == 0:
            break
        out = plan_fn(todo, seed_fn(a, todo))
        best = out["best"].cpu().numpy().astype(np.int64)
        tr = out["traj"].cpu().numpy()
        cs = out["cost"].cpu().numpy()
        if traj is None:
            traj = np.full((P,) + tr.shape[2:], np.nan, np.float32)
        ok = best >= 0
        idx = todo[ok]
        traj[idx] = tr[np.nonzero(ok)[0], best[ok]]
        cost[idx] = cs[np.nonzero(ok)[0], best[ok]]
        attempts[idx] = a
        todo = todo[~ok]
    if traj is None:
        traj = np.zeros((0,), np.float32)
    return {"traj": traj, "cost": cost, "attempts": attempts, "solved": attempts > 0}


def planner_attempts(planner: "Planner", q_start, goal, scene_of_problem, seed_fn, S: int, T: int,
                     n_attempts: int) -> dict:
    """plan_attempts with a Planner: each attempt is one dseed_plan_batch of the
    problems still unsolved (q_start [P][7], goal [P][7], scene_of_problem [P]
    host arrays)."""
    q_start, goal = np.asarray(q_start), np.asarray(goal)
    sc = np.asarray(scene_of_problem, np.int32)

    def plan_fn(problems, seeds):
        batch = planner.batch(q_start[problems], goal[problems], sc[problems], S, T)
        return planner.plan(batch, seeds)

    return plan_attempts(plan_fn, seed_fn, int(q_start.shape[0]), n_attempts)
