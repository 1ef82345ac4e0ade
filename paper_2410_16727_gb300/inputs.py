"""Seeded synthetic inputs shared by the CUDA path, its tests and the FP64 oracle.

This module draws random numbers and lays out plain data only: the robot
description (Franka Panda DH rows, joint limits, a seed-generated collision
sphere table), cuboid scenes, voxel grids, start/goal joint configurations and
seed trajectories.  It holds none of the method's arithmetic: where a workload
needs a kinematic quantity (the goal pose of a sampled goal configuration, the
clearance of a candidate configuration) the caller passes in a function that
computes it with its own implementation.

Workloads follow the paper's setting (7-DoF Franka, T = 32 waypoints,
Sec. 4.1 "Dataset Generation"; cubby/dresser-like shelf scenes, Sec. 4.1 and
Appendix A.1) with synthetic cuboid scenes standing in for the MpiNets scenes,
which are not available here.  Every array is float32 (int32 for indices) and
C-contiguous.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, Dict, List, Optional

import numpy as np

# --------------------------------------------------------------------------
# Robot description (input data, not arithmetic)
# --------------------------------------------------------------------------

# Franka Panda, modified (Craig) Denavit-Hartenberg rows (a, d, alpha, theta_offset)
# for joints 1..7 and the fixed flange frame (row 8), from the manufacturer's
# published kinematic table.  Frame i moves with joint i (i = 1..7); the flange
# frame 8 is rigidly attached to frame 7.
FRANKA_DH = np.array([
    [0.0,     0.333,  0.0,           0.0],
    [0.0,     0.0,   -math.pi / 2,   0.0],
    [0.0,     0.316,  math.pi / 2,   0.0],
    [0.0825,  0.0,    math.pi / 2,   0.0],
    [-0.0825, 0.384, -math.pi / 2,   0.0],
    [0.0,     0.0,    math.pi / 2,   0.0],
    [0.088,   0.0,    math.pi / 2,   0.0],
    [0.0,     0.107,  0.0,           0.0],
], dtype=np.float64)

# Mechanical joint limits (rad), lower / upper, joints 1..7 (manufacturer values).
FRANKA_LIMITS = np.array([
    [-2.8973, 2.8973],
    [-1.7628, 1.7628],
    [-2.8973, 2.8973],
    [-3.0718, -0.0698],
    [-2.8973, 2.8973],
    [-0.0175, 3.7525],
    [-2.8973, 2.8973],
], dtype=np.float64)

# The arm's "ready" configuration (manufacturer's home pose), used as the reference
# pose of the self-collision pair rule.
FRANKA_READY = np.array([0.0, -math.pi / 4, 0.0, -3 * math.pi / 4, 0.0, math.pi / 2, math.pi / 4],
                        dtype=np.float64)

# Collision-sphere layout: for each frame 1..8, how many spheres, and the segment
# (start, end) in that frame's coordinates along which they are spread.  The
# segments follow the link bodies: each runs to the next joint origin as read off
# the DH rows above (written out here as constants), or along the link body where
# two joint origins coincide.  Frame 8 carries the gripper volume along +z.
SPHERES_PER_FRAME = (6, 6, 7, 7, 8, 6, 5, 5)          # 50 spheres in total
SPHERE_SEGMENTS = (
    ((0.0, 0.0, -0.19), (0.0, 0.0, 0.0)),            # link 1: column below joint 2
    ((0.0, 0.0, 0.0), (0.0, -0.316, 0.0)),           # link 2: towards joint 3/4 axis
    ((0.0, 0.0, -0.15), (0.0825, 0.0, 0.0)),         # link 3: elbow housing
    ((0.0, 0.0, 0.0), (-0.0825, 0.384, 0.0)),        # link 4: forearm start
    ((0.0, 0.0, -0.25), (0.0, 0.0, 0.0)),            # link 5: forearm
    ((0.0, 0.0, 0.0), (0.088, 0.0, 0.0)),            # link 6: wrist
    ((0.0, 0.0, 0.0), (0.0, 0.0, 0.107)),            # link 7: flange stub
    ((0.0, 0.0, 0.0), (0.0, 0.0, 0.10)),             # frame 8: gripper volume
)


@dataclasses.dataclass
class Robot:
    dh: np.ndarray          # [8][4] float32: a, d, alpha, theta_offset
    limits: np.ndarray      # [7][2] float32: lower, upper
    sph_frame: np.ndarray   # [Ns] int32: frame index 1..8 the sphere is fixed to
    sph_o: np.ndarray       # [Ns][3] float32: offset in that frame (m)
    sph_r: np.ndarray       # [Ns] float32: radius (m)
    # self-collision pair rule: spheres on frames at least two apart whose
    # surfaces are at least self_margin apart at the reference pose self_ref
    self_ref: np.ndarray = dataclasses.field(default_factory=lambda: FRANKA_READY.astype(np.float32))
    self_margin: float = 0.02

    @property
    def n_spheres(self) -> int:
        return int(self.sph_r.shape[0])


def make_robot(seed: int = 0, jitter: float = 0.01,
               r_range=(0.04, 0.08)) -> Robot:
    """Franka Panda with a seed-generated 50-sphere collision model.

    Sphere k on frame i sits at u * (segment end - start) + start with
    u ~ U[0, 1] plus N(0, jitter^2) per axis, radius ~ U[r_range]."""
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([7001, seed])))
    frames, offs, rads = [], [], []
    for fi, (cnt, (a, b)) in enumerate(zip(SPHERES_PER_FRAME, SPHERE_SEGMENTS)):
        a = np.asarray(a)
        b = np.asarray(b)
        for _ in range(cnt):
            u = rng.uniform(0.0, 1.0)
            o = a + u * (b - a) + rng.normal(0.0, jitter, size=3)
            frames.append(fi + 1)
            offs.append(o)
            rads.append(rng.uniform(*r_range))
    return Robot(
        dh=FRANKA_DH.astype(np.float32),
        limits=FRANKA_LIMITS.astype(np.float32),
        sph_frame=np.asarray(frames, dtype=np.int32),
        sph_o=np.asarray(offs, dtype=np.float32).reshape(-1, 3),
        sph_r=np.asarray(rads, dtype=np.float32),
    )


# --------------------------------------------------------------------------
# Cost / optimiser parameters (the values are workload inputs for both sides)
# --------------------------------------------------------------------------

@dataclasses.dataclass
class CostParams:
    w_c: float = 100.0      # collision hinge weight
    eta: float = 0.01       # collision margin (m)
    dt: float = 0.05        # waypoint spacing (s)
    w_v: float = 1e-2       # velocity weight
    w_a: float = 1e-4       # acceleration weight
    w_j: float = 1e-6       # jerk weight
    w_p: float = 1e4        # goal position weight
    w_R: float = 1e3        # goal orientation weight
    w_l: float = 1e3        # joint-limit weight
    w_self: float = 0.0     # self-collision hinge weight (0: the self term is off)
    eta_self: float = 0.01  # self-collision margin (m)
    n_sweep: int = 0        # joint-space interpolants checked per segment between waypoints (0: off)

    def as_array(self) -> np.ndarray:
        return np.array([self.w_c, self.eta, self.dt, self.w_v, self.w_a, self.w_j,
                         self.w_p, self.w_R, self.w_l, self.w_self, self.eta_self], dtype=np.float64)


@dataclasses.dataclass
class OptParams:
    iters: int = 100        # cost+gradient evaluations, each followed by one L-BFGS update
    m: int = 5              # L-BFGS history
    c1: float = 1e-4        # Armijo constant
    max_step: float = 0.1   # cap on max |step| (rad)
    gamma0: float = 1e-3    # H0 scale while the history is empty
    alpha_min: float = 1e-4  # step length below which the history is cleared

    def as_array(self) -> np.ndarray:
        return np.array([self.iters, self.m, self.c1, self.max_step, self.gamma0,
                         self.alpha_min], dtype=np.float64)


# Success thresholds: translation 5 mm, rotation 2.86 degrees (paper Sec. 5.1).
DELTA_T = 0.005
DELTA_R = 2.86 * math.pi / 180.0


# --------------------------------------------------------------------------
# Voxel grids and cuboid scenes
# --------------------------------------------------------------------------

@dataclasses.dataclass
class Grid:
    origin: tuple           # (x, y, z) of the grid corner (m)
    res: float              # voxel edge (m)
    n: tuple                # (nx, ny, nz)

    @property
    def voxels(self) -> int:
        return int(self.n[0]) * int(self.n[1]) * int(self.n[2])


def _boxes(rows) -> np.ndarray:
    return np.asarray(rows, dtype=np.float32).reshape(-1, 6)


def _outside_keepout(cx, cy, hx, hy, radius):
    # the box footprint must stay clear of a vertical cylinder at the base
    dx = max(abs(cx) - hx, 0.0)
    dy = max(abs(cy) - hy, 0.0)
    return dx * dx + dy * dy >= radius * radius


def scene_tiny(rng: np.random.Generator, n_boxes: int = 10,
               side=(0.05, 0.3), keepout: float = 0.2) -> np.ndarray:
    """Random axis-aligned cuboids inside the 1 m^3 workspace [-0.5,0.5]^2 x [0,1],
    kept out of a 0.2 m cylinder around the robot base.  Rows: cx,cy,cz,hx,hy,hz."""
    rows = []
    while len(rows) < n_boxes:
        h = rng.uniform(side[0], side[1], size=3) / 2
        c = np.array([rng.uniform(-0.5 + h[0], 0.5 - h[0]),
                      rng.uniform(-0.5 + h[1], 0.5 - h[1]),
                      rng.uniform(0.0 + h[2], 1.0 - h[2])])
        if _outside_keepout(c[0], c[1], h[0], h[1], keepout):
            rows.append([*c, *h])
    return _boxes(rows)


def scene_shelf(rng: np.random.Generator, n_total=(20, 60)) -> np.ndarray:
    """A cabinet in front of the robot (+x): thin back/side/top/bottom walls, 2-4
    shelves, and random boxes resting on the shelf surfaces; 20-60 cuboids."""
    rows = []
    xf = rng.uniform(0.40, 0.60)                 # front face
    depth = rng.uniform(0.25, 0.33)
    xb = xf + depth                              # back face
    width = rng.uniform(0.6, 1.0)
    yc = rng.uniform(-0.2, 0.2)
    zb = rng.uniform(0.0, 0.3)
    zt = zb + rng.uniform(0.5, 0.8)
    th = lambda: rng.uniform(0.01, 0.02)         # wall thickness
    xm = 0.5 * (xf + xb)
    t = th(); rows.append([xb + t / 2, yc, 0.5 * (zb + zt), t / 2, width / 2, (zt - zb) / 2])  # back
    for sgn in (-1, 1):                          # sides
        t = th(); rows.append([xm, yc + sgn * (width / 2 + t / 2), 0.5 * (zb + zt), depth / 2, t / 2, (zt - zb) / 2])
    t = th(); rows.append([xm, yc, zt + t / 2, depth / 2, width / 2, t / 2])   # top
    t = th(); rows.append([xm, yc, zb - t / 2, depth / 2, width / 2, t / 2])   # bottom
    n_shelves = int(rng.integers(2, 5))
    levels = np.sort(rng.uniform(0.0, 1.0, size=n_shelves))
    surfaces = [zb]
    for k, u in enumerate(levels):
        z = zb + (zt - zb) * (k + 0.5 + 0.5 * (u - 0.5)) / (n_shelves + 1)
        t = th(); rows.append([xm, yc, z, depth / 2, width / 2, t / 2])
        surfaces.append(z + t / 2)
    n_want = int(rng.integers(n_total[0], n_total[1] + 1))
    while len(rows) < n_want:
        h = rng.uniform(0.03, 0.2, size=3) / 2
        h[0] = min(h[0], depth / 2 - 0.005)
        zs = surfaces[int(rng.integers(0, len(surfaces)))]
        cx = rng.uniform(xf + h[0], xb - h[0])
        cy = rng.uniform(yc - width / 2 + h[1], yc + width / 2 - h[1])
        rows.append([cx, cy, zs + h[2], h[0], h[1], h[2]])
    return _boxes(rows)


def scene_clutter(rng: np.random.Generator, n_boxes: int = 200,
                  side=(0.02, 0.15), keepout: float = 0.25) -> np.ndarray:
    """Dense clutter: many small cuboids in the 1 m^3 workspace, clear of the base."""
    return scene_tiny(rng, n_boxes=n_boxes, side=side, keepout=keepout)


# --------------------------------------------------------------------------
# Problems and seeds
# --------------------------------------------------------------------------

# clearance_fn(scene_index, q[N][7] float32) -> min over spheres of (phi - r), [N]
ClearanceFn = Callable[[int, np.ndarray], np.ndarray]
# pose_fn(q[N][7] float32) -> flange pose [N][7] (x, y, z, qw, qx, qy, qz)
PoseFn = Callable[[np.ndarray], np.ndarray]


def _rng(*key) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence(list(key))))


def sample_configs(rng: np.random.Generator, limits: np.ndarray, n: int,
                   shrink: float = 0.05) -> np.ndarray:
    lo = limits[:, 0].astype(np.float64)
    hi = limits[:, 1].astype(np.float64)
    mid, half = 0.5 * (lo + hi), 0.5 * (hi - lo) * (1.0 - shrink)
    return (mid + half * rng.uniform(-1.0, 1.0, size=(n, 7))).astype(np.float32)


def make_seeds(rng: np.random.Generator, q_start: np.ndarray, q_goal: np.ndarray,
               S: int, T: int, limits: np.ndarray, sigma: float = 0.1) -> np.ndarray:
    """S seeds of T waypoints: linear start->goal joint interpolation at t/T,
    t = 1..T, plus N(0, sigma^2) noise per entry, clipped to the joint limits.
    Returns [S][T][7] float32."""
    t = (np.arange(1, T + 1, dtype=np.float64) / T)[:, None]
    lin = q_start.astype(np.float64)[None, :] + t * (q_goal - q_start).astype(np.float64)[None, :]
    x = lin[None, :, :] + rng.normal(0.0, sigma, size=(S, T, 7))
    x = np.clip(x, limits[:, 0].astype(np.float64), limits[:, 1].astype(np.float64))
    return x.astype(np.float32)


@dataclasses.dataclass
class Workload:
    name: str
    robot: Robot
    cost: CostParams
    opt: OptParams
    grids: List[Grid]              # one per scene
    cuboids: List[np.ndarray]      # one [n][6] array per scene
    scene_of_problem: np.ndarray   # [P] int32
    q_start: np.ndarray            # [P][7]
    q_goal: np.ndarray             # [P][7]
    goal: np.ndarray               # [P][7] flange pose of q_goal
    seeds: np.ndarray              # [P][S][T][7]

    @property
    def P(self) -> int:
        return int(self.q_start.shape[0])

    @property
    def S(self) -> int:
        return int(self.seeds.shape[1])

    @property
    def T(self) -> int:
        return int(self.seeds.shape[2])


@dataclasses.dataclass
class WorkloadSpec:
    name: str
    config_id: int
    n_scenes: int
    n_problems: int
    S: int
    T: int
    iters: int
    scene: str                     # "tiny" | "shelf" | "clutter"
    grid: Grid


WORKLOADS: Dict[str, WorkloadSpec] = {
    # 1 scene of 10 cuboids, 64^3 at 2 cm, 32 seeds x 32 waypoints, 100 iterations
    "tiny": WorkloadSpec("tiny", 1, 1, 1, 32, 32, 100, "tiny",
                         Grid((-0.64, -0.64, -0.14), 0.02, (64, 64, 64))),
    # 256 shelf scenes (one per problem), 128^3 at 1 cm, 64 seeds x 32, 100 iterations
    "batched": WorkloadSpec("batched", 2, 256, 256, 64, 32, 100, "shelf",
                            Grid((-0.30, -0.64, -0.14), 0.01, (128, 128, 128))),
    # 16 dense-clutter scenes of 200 cuboids, 256^3 at 5 mm, 1024 problems x 128 seeds x 64, 200 iterations
    "stress": WorkloadSpec("stress", 5, 16, 1024, 128, 64, 200, "clutter",
                           Grid((-0.64, -0.64, -0.14), 0.005, (256, 256, 256))),
}


def make_scene(kind: str, rng: np.random.Generator) -> np.ndarray:
    if kind == "tiny":
        return scene_tiny(rng)
    if kind == "shelf":
        return scene_shelf(rng)
    if kind == "clutter":
        return scene_clutter(rng)
    raise ValueError(kind)


def make_scenes(spec: WorkloadSpec, n_scenes: Optional[int] = None, seed_offset: int = 0):
    """Cuboid lists and grids of the workload's scenes (scene s keyed on (config, s))."""
    n = spec.n_scenes if n_scenes is None else n_scenes
    cuboids = [make_scene(spec.scene, _rng(1000 * spec.config_id + seed_offset, s, 1)) for s in range(n)]
    return cuboids, [spec.grid for _ in range(n)]


def build_workload(spec: WorkloadSpec, cuboids: List[np.ndarray], grids: List[Grid],
                   clearance_fn: ClearanceFn, pose_fn: PoseFn,
                   n_problems: Optional[int] = None, S: Optional[int] = None,
                   T: Optional[int] = None, iters: Optional[int] = None,
                   margin: float = 0.01, robot: Optional[Robot] = None,
                   seed_offset: int = 0) -> Workload:
    """Draw collision-free start/goal pairs and seeds for the scenes of a workload.

    Problem p uses scene p * n_scenes // P.  Its random stream is keyed on
    (config id, p): start and goal are the first two of batches of 16 candidate
    configurations whose clearance (from clearance_fn: min over spheres of
    phi - r, computed by the caller on its own ESDF of that scene) is at least
    `margin`.  goal = pose_fn(q_goal).  Seeds come from a separate stream keyed on
    (config id, p), so they do not depend on how many candidates were rejected."""
    robot = robot if robot is not None else make_robot()
    P = spec.n_problems if n_problems is None else n_problems
    S = spec.S if S is None else S
    T = spec.T if T is None else T
    n_scenes = len(cuboids)
    scene_of_problem = (np.arange(P) * n_scenes // max(P, 1)).astype(np.int32)
    q_start = np.zeros((P, 7), np.float32)
    q_goal = np.zeros((P, 7), np.float32)
    pending = list(range(P))
    rngs = {p: _rng(1000 * spec.config_id + seed_offset, p, 2) for p in range(P)}
    found: Dict[int, list] = {p: [] for p in range(P)}
    rounds = 0
    while pending:
        rounds += 1
        if rounds > 200:
            raise RuntimeError("could not find collision-free start/goal pairs")
        by_scene: Dict[int, list] = {}
        cands = {}
        for p in pending:
            cands[p] = sample_configs(rngs[p], robot.limits, 16)
            by_scene.setdefault(int(scene_of_problem[p]), []).append(p)
        for s, plist in by_scene.items():
            q = np.concatenate([cands[p] for p in plist], axis=0)
            clr = np.asarray(clearance_fn(s, q), dtype=np.float64).reshape(-1)
            for i, p in enumerate(plist):
                ok = clr[16 * i:16 * (i + 1)] >= margin
                for j in np.nonzero(ok)[0]:
                    if len(found[p]) < 2:
                        found[p].append(cands[p][j])
        pending = [p for p in pending if len(found[p]) < 2]
    for p in range(P):
        q_start[p], q_goal[p] = found[p][0], found[p][1]
    goal = np.asarray(pose_fn(q_goal), dtype=np.float32).reshape(P, 7)
    seeds = np.stack([make_seeds(_rng(1000 * spec.config_id + seed_offset, p, 3),
                                 q_start[p], q_goal[p], S, T, robot.limits)
                      for p in range(P)], axis=0)
    opt = OptParams(iters=spec.iters if iters is None else iters)
    return Workload(spec.name, robot, CostParams(), opt, list(grids), list(cuboids),
                    scene_of_problem, q_start, q_goal, goal, np.ascontiguousarray(seeds))


def random_trajectories(rng: np.random.Generator, q_start: np.ndarray, B: int, T: int,
                        limits: np.ndarray, spread: float = 0.6) -> np.ndarray:
    """Random smooth-ish trajectories around q_start (for cost/gradient parity cases
    that need many different states rather than optimiser seeds).  [B][T][7]."""
    q_end = sample_configs(rng, limits, B)
    t = (np.arange(1, T + 1, dtype=np.float64) / T)[None, :, None]
    base = q_start[None, None, :].astype(np.float64) + t * (q_end[:, None, :] - q_start[None, None, :])
    wig = spread * 0.2 * np.sin(np.pi * t * rng.uniform(0.5, 2.0, size=(B, 1, 7)) + rng.uniform(0, 6.28, size=(B, 1, 7)))
    x = base + wig + rng.normal(0.0, 0.02, size=(B, T, 7))
    return x.astype(np.float32)
