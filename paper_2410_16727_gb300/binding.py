"""Thin Python binding of libdseed (include/dseed.h).

Argument marshalling only: every function checks tensor devices, dtypes and
shapes, packs the C descriptors and calls the entry point of the same name on
the current CUDA stream.  All arithmetic runs in the library's kernels.  There
is no fallback: if libdseed.so is missing or a call fails, an exception says so.
"""
from __future__ import annotations

import ctypes as C
import math
import os
from typing import Optional, Sequence

import numpy as np
import torch

from . import build as _build

MAX_SPHERES = 64
MAX_T = 128
MAX_HISTORY = 8
N_METRICS = 7
ESDF_FAR = 1000.0

_lib = None


class RobotDesc(C.Structure):
    _fields_ = [("dh", (C.c_float * 4) * 8), ("limits", (C.c_float * 2) * 7), ("n_spheres", C.c_int),
                ("sphere_frame", C.c_int * MAX_SPHERES), ("sphere_offset", (C.c_float * 3) * MAX_SPHERES),
                ("sphere_radius", C.c_float * MAX_SPHERES), ("self_ref", C.c_float * 7),
                ("self_margin", C.c_float)]


class Grid(C.Structure):
    _fields_ = [("origin", C.c_float * 3), ("res", C.c_float), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int)]


class EsdfJob(C.Structure):
    _fields_ = [("cuboids_dev", C.c_void_p), ("n", C.c_int), ("grid", Grid), ("esdf_dev", C.c_void_p)]


class Scene(C.Structure):
    _fields_ = [("esdf_dev", C.c_void_p), ("grid", Grid), ("lipschitz", C.c_float)]


COST_FIELDS = ("w_c", "eta", "dt", "w_v", "w_a", "w_j", "w_p", "w_R", "w_l", "w_self", "eta_self")


class CostParams(C.Structure):
    _fields_ = [(k, C.c_float) for k in COST_FIELDS] + [("n_sweep", C.c_int)]


class OptParams(C.Structure):
    _fields_ = [("iters", C.c_int), ("m", C.c_int), ("c1", C.c_float), ("max_step", C.c_float),
                ("gamma0", C.c_float), ("alpha_min", C.c_float)]


class PlanDesc(C.Structure):
    _fields_ = [("P", C.c_int), ("S", C.c_int), ("T", C.c_int), ("cost", CostParams), ("opt", OptParams),
                ("delta_t", C.c_float), ("delta_r", C.c_float)]


class Problems(C.Structure):
    _fields_ = [("q_start_dev", C.c_void_p), ("goal_dev", C.c_void_p), ("scene_of_problem_dev", C.c_void_p),
                ("scenes_dev", C.c_void_p), ("n_scenes", C.c_int)]


class LbfgsLayout(C.Structure):
    _fields_ = [(k, C.c_size_t) for k in ("x", "g", "x_trial", "d", "s", "y", "rho", "yy", "f", "alpha", "gts",
                                          "meta", "total")]


class ServerDesc(C.Structure):
    _fields_ = [("arena_bytes", C.c_size_t), ("max_requests", C.c_int), ("round_iters", C.c_int),
                ("cost", CostParams), ("opt", OptParams), ("delta_t", C.c_float), ("delta_r", C.c_float)]


class Request(C.Structure):
    _fields_ = [("scene_id", C.c_int), ("S", C.c_int), ("T", C.c_int), ("q_start_host", C.c_void_p),
                ("goal_host", C.c_void_p), ("seeds_host", C.c_void_p), ("traj_host", C.c_void_p),
                ("cost_host", C.c_void_p), ("success_host", C.c_void_p), ("best_host", C.c_void_p)]


class ConvTc(C.Structure):
    _fields_ = [("a0_dev", C.c_void_p), ("c0", C.c_int), ("a1_dev", C.c_void_p), ("c1", C.c_int),
                ("n_samples", C.c_int), ("L", C.c_int), ("taps", C.c_int), ("pad", C.c_int),
                ("w_dev", C.c_void_p), ("cout", C.c_int), ("cout_pad", C.c_int), ("bias_dev", C.c_void_p),
                ("epilogue", C.c_int), ("rows_per_sample", C.c_int), ("gn_eps", C.c_float),
                ("gamma_dev", C.c_void_p), ("beta_dev", C.c_void_p), ("film_dev", C.c_void_p),
                ("film_ld", C.c_int), ("film_add_dev", C.c_void_p), ("sample_problem_dev", C.c_void_p), ("res_dev", C.c_void_p), ("out_dev", C.c_void_p),
                ("out_ld", C.c_int), ("err_dev", C.c_void_p)]


class ServerStats(C.Structure):
    _fields_ = [("submitted", C.c_longlong), ("admitted", C.c_longlong), ("completed", C.c_longlong),
                ("failed", C.c_longlong), ("rounds", C.c_longlong), ("queued", C.c_int), ("active", C.c_int),
                ("arena_used", C.c_size_t), ("arena_peak", C.c_size_t)]


class DeviceInfo(C.Structure):
    _fields_ = [(k, C.c_int) for k in ("sm_count", "sm_clock_khz", "l2_bytes", "cc_major", "cc_minor",
                                      "fp32_lanes_per_sm")]


class DseedError(RuntimeError):
    pass


class DseedTimeout(DseedError):
    """DSEED_ETIMEOUT: a serving wait on the GPU reached the server's wait limit
    (the work stays in flight)."""


ETIMEOUT = -4


_SIGS = {
    "dseed_abi_version": ([], C.c_int),
    "dseed_last_error": ([], C.c_char_p),
    "dseed_device_info": ([C.c_int, C.POINTER(DeviceInfo)], C.c_int),
    "dseed_robot_create": ([C.POINTER(RobotDesc), C.POINTER(C.c_void_p)], C.c_int),
    "dseed_robot_destroy": ([C.c_void_p], None),
    "dseed_scene_build_esdf": ([C.c_void_p, C.c_int, C.POINTER(Grid), C.c_void_p, C.c_void_p], C.c_int),
    "dseed_scene_build_esdf_batch": ([C.c_void_p, C.c_int, C.c_void_p], C.c_int),
    "dseed_fk": ([C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "dseed_cost": ([C.c_void_p, C.POINTER(PlanDesc), C.POINTER(Problems), C.c_void_p, C.c_void_p, C.c_void_p,
                    C.c_void_p], C.c_int),
    "dseed_cost_grad": ([C.c_void_p, C.POINTER(PlanDesc), C.POINTER(Problems), C.c_void_p, C.c_void_p, C.c_void_p,
                         C.c_void_p, C.c_void_p], C.c_int),
    "dseed_evaluate": ([C.c_void_p, C.POINTER(PlanDesc), C.POINTER(Problems), C.c_void_p, C.c_void_p, C.c_void_p,
                        C.c_void_p], C.c_int),
    "dseed_lbfgs_layout": ([C.POINTER(PlanDesc), C.POINTER(LbfgsLayout)], C.c_int),
    "dseed_lbfgs_init": ([C.POINTER(PlanDesc), C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "dseed_lbfgs_step": ([C.POINTER(PlanDesc), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "dseed_plan_workspace_bytes": ([C.POINTER(PlanDesc), C.POINTER(C.c_size_t)], C.c_int),
    "dseed_plan_batch": ([C.c_void_p, C.POINTER(PlanDesc), C.POINTER(Problems), C.c_void_p, C.c_void_p, C.c_size_t,
                          C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "dseed_arena_create": ([C.c_size_t, C.POINTER(C.c_void_p)], C.c_int),
    "dseed_arena_destroy": ([C.c_void_p], None),
    "dseed_arena_alloc": ([C.c_void_p, C.c_size_t, C.POINTER(C.c_size_t)], C.c_int),
    "dseed_arena_free": ([C.c_void_p, C.c_size_t], C.c_int),
    "dseed_arena_usage": ([C.c_void_p, C.POINTER(C.c_size_t), C.POINTER(C.c_size_t), C.POINTER(C.c_size_t)], C.c_int),
    "dseed_server_create": ([C.c_void_p, C.POINTER(ServerDesc), C.c_void_p, C.POINTER(C.c_void_p)], C.c_int),
    "dseed_server_destroy": ([C.c_void_p], None),
    "dseed_server_add_scene": ([C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.POINTER(Grid)], C.c_int),
    "dseed_server_remove_scene": ([C.c_void_p, C.c_int], C.c_int),
    "dseed_server_submit": ([C.c_void_p, C.POINTER(Request), C.POINTER(C.c_longlong)], C.c_int),
    "dseed_server_step": ([C.c_void_p, C.c_int, C.POINTER(C.c_int)], C.c_int),
    "dseed_server_set_wait_limit": ([C.c_void_p, C.c_double], C.c_int),
    "dseed_server_poll": ([C.c_void_p, C.c_longlong, C.POINTER(C.c_int), C.POINTER(C.c_double),
                           C.POINTER(C.c_double)], C.c_int),
    "dseed_server_stats": ([C.c_void_p, C.POINTER(ServerStats)], C.c_int),
    "dseed_nn_gemm_f32": ([C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_float, C.c_void_p, C.c_int, C.c_void_p,
                           C.c_int, C.c_float, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p], C.c_int),
    "dseed_nn_gemm_bf16": ([C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p],
                           C.c_int),
    "dseed_nn_im2col1d": ([C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                           C.c_void_p, C.c_int, C.c_void_p], C.c_int),
    "dseed_nn_col2im1d": ([C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                           C.c_void_p, C.c_void_p], C.c_int),
    "dseed_nn_colsum": ([C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_int, C.c_void_p], C.c_int),
    "dseed_nn_groupnorm_fwd": ([C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_float,
                                C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "dseed_nn_groupnorm_bwd": ([C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                                C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
    "dseed_nn_mish": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_longlong, C.c_int, C.c_void_p], C.c_int),
    "dseed_nn_film": ([C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                       C.c_void_p, C.c_int, C.c_void_p], C.c_int),
    "dseed_nn_axpby": ([C.c_float, C.c_void_p, C.c_float, C.c_void_p, C.c_void_p, C.c_longlong, C.c_void_p], C.c_int),
    "dseed_nn_copy_cols": ([C.c_void_p, C.c_longlong, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_int, C.c_int,
                            C.c_int, C.c_void_p], C.c_int),
    "dseed_nn_upsample2": ([C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_int, C.c_void_p], C.c_int),
    "dseed_nn_gather": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_longlong, C.c_longlong, C.c_int, C.c_void_p],
                        C.c_int),
    "dseed_nn_gather_rows": ([C.c_void_p, C.c_void_p, C.c_longlong, C.c_int, C.c_void_p, C.c_void_p], C.c_int),
    "dseed_nn_sinusoid": ([C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p], C.c_int),
    "dseed_nn_adam": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_longlong, C.c_float, C.c_float, C.c_float,
                       C.c_float, C.c_float, C.c_int, C.c_void_p], C.c_int),
    "dseed_nn_ddpm_noise": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_void_p,
                             C.c_void_p], C.c_int),
    "dseed_nn_mse": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_int,
                      C.c_void_p], C.c_int),
    "dseed_nn_fk_mse": ([C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_float,
                         C.c_void_p, C.c_void_p, C.c_int, C.c_void_p], C.c_int),
    "dseed_nn_ddim_step": ([C.c_void_p, C.c_void_p, C.c_float, C.c_float, C.c_longlong, C.c_float, C.c_void_p,
                           C.c_void_p], C.c_int),
    "dseed_nn_to_bf16": ([C.c_void_p, C.c_void_p, C.c_longlong, C.c_void_p], C.c_int),
    "dseed_nn_clamp_affine": ([C.c_void_p, C.c_float, C.c_float, C.c_float, C.c_float, C.c_void_p, C.c_longlong,
                               C.c_void_p], C.c_int),
    "dseed_nn_conv_tc": ([C.POINTER(ConvTc), C.c_void_p], C.c_int),
    "dseed_nn_im2col1d_bf16": ([C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                C.c_void_p, C.c_void_p], C.c_int),
    "dseed_nn_upsample2_bf16": ([C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p], C.c_int),
    "dseed_robot_self_pairs": ([C.c_void_p, C.POINTER(C.c_ulonglong), C.POINTER(C.c_int)], C.c_int),
    "dseed_plan_batch_static": ([C.c_void_p, C.POINTER(PlanDesc), C.POINTER(Problems), C.c_void_p, C.c_void_p,
                                 C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p], C.c_int),
}

STATIC_SCRATCH_BYTES = 32 << 20


def library_path() -> str:
    return _build.LIB


def load():
    """Load libdseed.so (built by paper_2410_16727_gb300.build / __graft_entry__.build)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise DseedError(f"libdseed.so is not built ({path}); run `python -m paper_2410_16727_gb300.build`")
    lib = C.CDLL(path)
    for name, (args, res) in _SIGS.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def _check(rc: int, what: str):
    if rc != 0:
        msg = load().dseed_last_error().decode(errors="replace")
        raise (DseedTimeout if rc == ETIMEOUT else DseedError)(f"{what} failed with status {rc}: {msg}")


def _stream() -> int:
    return torch.cuda.current_stream().cuda_stream


def _dev(t: Optional[torch.Tensor], dtype, name: str, shape=None):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise DseedError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise DseedError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise DseedError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise DseedError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return t.data_ptr()


# ---------------------------------------------------------------------------- descriptors

def abi_version() -> int:
    return int(load().dseed_abi_version())


def device_info(device: int = 0) -> dict:
    """SM count, peak SM clock (kHz), L2 bytes, compute capability, FP32 lanes per SM."""
    d = DeviceInfo()
    _check(load().dseed_device_info(int(device), C.byref(d)), "dseed_device_info")
    return {k: int(getattr(d, k)) for k, _ in DeviceInfo._fields_}


def last_error() -> str:
    return load().dseed_last_error().decode(errors="replace")


class Robot:
    """Owning wrapper of a DseedRobot handle built from an inputs.Robot-like object."""

    def __init__(self, robot):
        d = RobotDesc()
        dh = robot.dh.tolist()
        lim = robot.limits.tolist()
        for i in range(8):
            for c in range(4):
                d.dh[i][c] = float(dh[i][c])
        for j in range(7):
            d.limits[j][0], d.limits[j][1] = float(lim[j][0]), float(lim[j][1])
        ns = int(len(robot.sph_r))
        if ns > MAX_SPHERES:
            raise DseedError(f"{ns} spheres exceed the limit of {MAX_SPHERES}")
        d.n_spheres = ns
        for k in range(ns):
            d.sphere_frame[k] = int(robot.sph_frame[k])
            for c in range(3):
                d.sphere_offset[k][c] = float(robot.sph_o[k][c])
            d.sphere_radius[k] = float(robot.sph_r[k])
        ref = np.asarray(getattr(robot, "self_ref", np.zeros(7)), np.float64).reshape(7)
        for j in range(7):
            d.self_ref[j] = float(ref[j])
        d.self_margin = float(getattr(robot, "self_margin", 0.0))
        h = C.c_void_p()
        _check(load().dseed_robot_create(C.byref(d), C.byref(h)), "dseed_robot_create")
        self.handle = h
        self.n_spheres = ns

    def self_pairs(self) -> np.ndarray:
        """Checked self-collision pairs as a symmetric [ns][ns] uint8 matrix (caller's sphere order)."""
        mask = (C.c_ulonglong * MAX_SPHERES)()
        n = C.c_int()
        _check(load().dseed_robot_self_pairs(self.handle, mask, C.byref(n)), "dseed_robot_self_pairs")
        out = np.zeros((self.n_spheres, self.n_spheres), np.uint8)
        for i in range(self.n_spheres):
            for j in range(self.n_spheres):
                out[i, j] = (mask[i] >> j) & 1
        return out

    def __del__(self):
        if getattr(self, "handle", None) is not None and _lib is not None:
            _lib.dseed_robot_destroy(self.handle)
            self.handle = None


def make_grid(g) -> Grid:
    out = Grid()
    for a in range(3):
        out.origin[a] = float(g.origin[a])
    out.res = float(g.res)
    out.nx, out.ny, out.nz = (int(v) for v in g.n)
    return out


def plan_desc(P: int, S: int, T: int, cost, opt=None, delta_t: float = 0.005,
              delta_r: float = 2.86 * math.pi / 180.0) -> PlanDesc:
    d = PlanDesc()
    d.P, d.S, d.T = int(P), int(S), int(T)
    for k, v in zip(COST_FIELDS, cost.as_array()):
        setattr(d.cost, k, float(v))
    d.cost.n_sweep = int(cost.n_sweep)
    if opt is not None:
        d.opt.iters, d.opt.m = int(opt.iters), int(opt.m)
        d.opt.c1, d.opt.max_step = float(opt.c1), float(opt.max_step)
        d.opt.gamma0, d.opt.alpha_min = float(opt.gamma0), float(opt.alpha_min)
    d.delta_t, d.delta_r = float(delta_t), float(delta_r)
    return d


class SceneTable:
    """Device table of DseedScene entries (ESDF pointer + grid) for a list of
    ESDF tensors; keeps the tensors alive."""

    def __init__(self, esdfs: Sequence[torch.Tensor], grids: Sequence, device=None, lipschitz: float = 1.0):
        if len(esdfs) != len(grids) or not esdfs:
            raise DseedError("need one grid per ESDF and at least one scene")
        arr = (Scene * len(esdfs))()
        for i, (e, g) in enumerate(zip(esdfs, grids)):
            gg = make_grid(g)
            _dev(e, torch.float32, f"esdf[{i}]", (gg.nz, gg.ny, gg.nx))
            arr[i].esdf_dev = e.data_ptr()
            arr[i].grid = gg
            arr[i].lipschitz = float(lipschitz)
        raw = torch.frombuffer(bytearray(bytes(arr)), dtype=torch.uint8)
        self.table = raw.to(device or esdfs[0].device)
        self.esdfs = list(esdfs)
        self.grids = list(grids)
        self.n = len(esdfs)


def make_problems(q_start: torch.Tensor, goal: torch.Tensor, scene_of_problem: torch.Tensor,
                  scenes: SceneTable) -> Problems:
    P = q_start.shape[0]
    pr = Problems()
    pr.q_start_dev = _dev(q_start, torch.float32, "q_start", (P, 7))
    pr.goal_dev = _dev(goal, torch.float32, "goal", (P, 7))
    pr.scene_of_problem_dev = _dev(scene_of_problem, torch.int32, "scene_of_problem", (P,))
    pr.scenes_dev = scenes.table.data_ptr()
    pr.n_scenes = scenes.n
    return pr


# ---------------------------------------------------------------------------- entry points

def scene_build_esdf(cuboids: torch.Tensor, grid, out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """ESDF [nz][ny][nx] of cuboids [n][6] (device tensors)."""
    g = make_grid(grid)
    n = int(cuboids.shape[0])
    if out is None:
        out = torch.empty((g.nz, g.ny, g.nx), dtype=torch.float32, device=cuboids.device)
    cp = _dev(cuboids, torch.float32, "cuboids", (n, 6)) if n > 0 else None
    _check(load().dseed_scene_build_esdf(cp, n, C.byref(g), _dev(out, torch.float32, "esdf"), _stream()),
           "dseed_scene_build_esdf")
    return out


def scene_build_esdf_batch(cuboids: Sequence[torch.Tensor], grids: Sequence,
                           outs: Optional[Sequence[torch.Tensor]] = None) -> list:
    """ESDFs of several scenes in one call (device cuboid tensors [n_i][6])."""
    jobs = (EsdfJob * len(cuboids))()
    res = []
    for q, (c, g) in enumerate(zip(cuboids, grids)):
        gg = make_grid(g)
        out = outs[q] if outs is not None else torch.empty((gg.nz, gg.ny, gg.nx), dtype=torch.float32,
                                                             device=c.device)
        n = int(c.shape[0])
        jobs[q].cuboids_dev = _dev(c, torch.float32, f"cuboids[{q}]", (n, 6)) if n > 0 else None
        jobs[q].n = n
        jobs[q].grid = gg
        jobs[q].esdf_dev = _dev(out, torch.float32, f"esdf[{q}]", (gg.nz, gg.ny, gg.nx))
        res.append(out)
    _check(load().dseed_scene_build_esdf_batch(C.cast(jobs, C.c_void_p), len(cuboids), _stream()),
           "dseed_scene_build_esdf_batch")
    return res


class EsdfBatch:
    """A prepared dseed_scene_build_esdf_batch call: the job records for fixed
    cuboid and ESDF tensors are built once, so a rebuild (new cuboid values in
    the same tensors) costs one C call."""

    def __init__(self, cuboids: Sequence[torch.Tensor], grids: Sequence, outs: Sequence[torch.Tensor]):
        self.jobs = (EsdfJob * len(cuboids))()
        self.keep = (list(cuboids), list(outs))
        for q, (c, g, out) in enumerate(zip(cuboids, grids, outs)):
            gg = make_grid(g)
            n = int(c.shape[0])
            self.jobs[q].cuboids_dev = _dev(c, torch.float32, f"cuboids[{q}]", (n, 6)) if n > 0 else None
            self.jobs[q].n = n
            self.jobs[q].grid = gg
            self.jobs[q].esdf_dev = _dev(out, torch.float32, f"esdf[{q}]", (gg.nz, gg.ny, gg.nx))
        self.n = len(cuboids)

    def run(self):
        _check(load().dseed_scene_build_esdf_batch(C.cast(self.jobs, C.c_void_p), self.n, _stream()),
               "dseed_scene_build_esdf_batch")


def fk(robot: Robot, q: torch.Tensor, spheres: bool = False):
    """Flange poses [N][7] (and sphere centres [N][Ns][3]) of q [N][7]."""
    N = int(q.shape[0])
    pose = torch.empty((N, 7), dtype=torch.float32, device=q.device)
    sph = torch.empty((N, robot.n_spheres, 3), dtype=torch.float32, device=q.device) if spheres else None
    _check(load().dseed_fk(robot.handle, _dev(q, torch.float32, "q", (N, 7)), N, pose.data_ptr(),
                           sph.data_ptr() if sph is not None else None, _stream()), "dseed_fk")
    return (pose, sph) if spheres else pose


def cost(robot: Robot, desc: PlanDesc, pr: Problems, x: torch.Tensor, terms: bool = False):
    P, S, T = desc.P, desc.S, desc.T
    out = torch.empty((P, S), dtype=torch.float32, device=x.device)
    tr = torch.empty((P, S, 4), dtype=torch.float32, device=x.device) if terms else None
    _check(load().dseed_cost(robot.handle, C.byref(desc), C.byref(pr), _dev(x, torch.float32, "x", (P, S, T, 7)),
                             out.data_ptr(), tr.data_ptr() if tr is not None else None, _stream()), "dseed_cost")
    return (out, tr) if terms else out


def cost_grad(robot: Robot, desc: PlanDesc, pr: Problems, x: torch.Tensor,
              grad_scale: Optional[torch.Tensor] = None):
    P, S, T = desc.P, desc.S, desc.T
    c = torch.empty((P, S), dtype=torch.float32, device=x.device)
    g = torch.empty((P, S, T, 7), dtype=torch.float32, device=x.device)
    _check(load().dseed_cost_grad(robot.handle, C.byref(desc), C.byref(pr),
                                  _dev(x, torch.float32, "x", (P, S, T, 7)),
                                  _dev(grad_scale, torch.float32, "grad_scale", (P, S)), c.data_ptr(), g.data_ptr(),
                                  _stream()), "dseed_cost_grad")
    return c, g


def evaluate(robot: Robot, desc: PlanDesc, pr: Problems, x: torch.Tensor):
    P, S, T = desc.P, desc.S, desc.T
    ok = torch.empty((P, S), dtype=torch.uint8, device=x.device)
    met = torch.empty((P, S, N_METRICS), dtype=torch.float32, device=x.device)
    _check(load().dseed_evaluate(robot.handle, C.byref(desc), C.byref(pr),
                                 _dev(x, torch.float32, "x", (P, S, T, 7)), ok.data_ptr(), met.data_ptr(), _stream()),
           "dseed_evaluate")
    return ok, met


def lbfgs_layout(desc: PlanDesc) -> LbfgsLayout:
    lay = LbfgsLayout()
    _check(load().dseed_lbfgs_layout(C.byref(desc), C.byref(lay)), "dseed_lbfgs_layout")
    return lay


def lbfgs_init(desc: PlanDesc, x0: torch.Tensor, state: torch.Tensor):
    _check(load().dseed_lbfgs_init(C.byref(desc), _dev(x0, torch.float32, "x0"), _dev(state, torch.uint8, "state"),
                                   _stream()), "dseed_lbfgs_init")


def lbfgs_step(desc: PlanDesc, f_trial: torch.Tensor, g_trial: torch.Tensor, state: torch.Tensor):
    _check(load().dseed_lbfgs_step(C.byref(desc), _dev(f_trial, torch.float32, "f_trial"),
                                   _dev(g_trial, torch.float32, "g_trial"), _dev(state, torch.uint8, "state"),
                                   _stream()), "dseed_lbfgs_step")


def lbfgs_view(state: torch.Tensor, lay: LbfgsLayout, desc: PlanDesc, name: str) -> torch.Tensor:
    """A typed view of one array of the L-BFGS state buffer."""
    B, n, m = desc.P * desc.S, 7 * desc.T, desc.opt.m
    shapes = {"x": (B, n), "g": (B, n), "x_trial": (B, n), "d": (B, n), "s": (B, m, n), "y": (B, m, n),
              "rho": (B, 8), "yy": (B,), "f": (B,), "alpha": (B,), "gts": (B,), "meta": (B, 4)}
    shape = shapes[name]
    count = 1
    for s in shape:
        count *= s
    off = getattr(lay, name)
    dtype = torch.int32 if name == "meta" else torch.float32
    return state[off:off + 4 * count].view(dtype).view(shape)


def plan_workspace_bytes(desc: PlanDesc) -> int:
    b = C.c_size_t()
    _check(load().dseed_plan_workspace_bytes(C.byref(desc), C.byref(b)), "dseed_plan_workspace_bytes")
    return int(b.value)


def alloc_workspace(nbytes: int, device) -> torch.Tensor:
    # torch's caching allocator returns 512-byte aligned blocks
    return torch.empty(max(nbytes, 1), dtype=torch.uint8, device=device)


def plan_batch(robot: Robot, desc: PlanDesc, pr: Problems, seeds: torch.Tensor, workspace: torch.Tensor,
               out: Optional[dict] = None) -> dict:
    """Run the fused optimiser; returns dict(traj, cost, success, metrics, best)."""
    P, S, T = desc.P, desc.S, desc.T
    dev = seeds.device
    if out is None:
        out = dict(traj=torch.empty((P, S, T, 7), dtype=torch.float32, device=dev),
                   cost=torch.empty((P, S), dtype=torch.float32, device=dev),
                   success=torch.empty((P, S), dtype=torch.uint8, device=dev),
                   metrics=torch.empty((P, S, N_METRICS), dtype=torch.float32, device=dev),
                   best=torch.empty((P,), dtype=torch.int32, device=dev))
    met = out.get("metrics")
    _check(load().dseed_plan_batch(robot.handle, C.byref(desc), C.byref(pr),
                                   _dev(seeds, torch.float32, "seeds", (P, S, T, 7)),
                                   _dev(workspace, torch.uint8, "workspace"), workspace.numel(),
                                   _dev(out["traj"], torch.float32, "traj", (P, S, T, 7)),
                                   _dev(out["cost"], torch.float32, "cost", (P, S)),
                                   _dev(out["success"], torch.uint8, "success", (P, S)),
                                   met.data_ptr() if met is not None else None,
                                   _dev(out["best"], torch.int32, "best", (P,)), _stream()), "dseed_plan_batch")
    return out


def plan_batch_static(robot: Robot, desc: PlanDesc, pr: Problems, seeds: torch.Tensor,
                      out: Optional[dict] = None) -> dict:
    """dseed_plan_batch_static: the fused optimiser with the library's own static
    scratch instead of a caller workspace, for callers that may not allocate
    device memory (the outputs must then be preallocated and passed in `out`)."""
    P, S, T = desc.P, desc.S, desc.T
    dev = seeds.device
    if out is None:
        out = dict(traj=torch.empty((P, S, T, 7), dtype=torch.float32, device=dev),
                   cost=torch.empty((P, S), dtype=torch.float32, device=dev),
                   success=torch.empty((P, S), dtype=torch.uint8, device=dev),
                   metrics=torch.empty((P, S, N_METRICS), dtype=torch.float32, device=dev),
                   best=torch.empty((P,), dtype=torch.int32, device=dev))
    met = out.get("metrics")
    _check(load().dseed_plan_batch_static(robot.handle, C.byref(desc), C.byref(pr),
                                          _dev(seeds, torch.float32, "seeds", (P, S, T, 7)),
                                          _dev(out["traj"], torch.float32, "traj", (P, S, T, 7)),
                                          _dev(out["cost"], torch.float32, "cost", (P, S)),
                                          _dev(out["success"], torch.uint8, "success", (P, S)),
                                          met.data_ptr() if met is not None else None,
                                          _dev(out["best"], torch.int32, "best", (P,)), _stream()),
           "dseed_plan_batch_static")
    return out


# ---------------------------------------------------------------------------- arena / server

class Arena:
    """Host-side arena manager (dseed_arena_*): offsets only, no device memory."""

    def __init__(self, nbytes: int):
        h = C.c_void_p()
        _check(load().dseed_arena_create(nbytes, C.byref(h)), "dseed_arena_create")
        self.handle = h

    def alloc(self, nbytes: int) -> Optional[int]:
        off = C.c_size_t()
        rc = load().dseed_arena_alloc(self.handle, nbytes, C.byref(off))
        if rc == -2:
            return None
        _check(rc, "dseed_arena_alloc")
        return int(off.value)

    def free(self, offset: int):
        _check(load().dseed_arena_free(self.handle, offset), "dseed_arena_free")

    def usage(self):
        u, p, l = C.c_size_t(), C.c_size_t(), C.c_size_t()
        _check(load().dseed_arena_usage(self.handle, C.byref(u), C.byref(p), C.byref(l)), "dseed_arena_usage")
        return int(u.value), int(p.value), int(l.value)

    def __del__(self):
        if getattr(self, "handle", None) is not None and _lib is not None:
            _lib.dseed_arena_destroy(self.handle)
            self.handle = None


def server_desc(arena_bytes: int, max_requests: int, round_iters: int, cost, opt,
                delta_t: float = 0.005, delta_r: float = 2.86 * math.pi / 180.0) -> ServerDesc:
    d = ServerDesc()
    d.arena_bytes, d.max_requests, d.round_iters = int(arena_bytes), int(max_requests), int(round_iters)
    pd = plan_desc(0, 1, 1, cost, opt, delta_t, delta_r)
    d.cost, d.opt = pd.cost, pd.opt
    d.delta_t, d.delta_r = pd.delta_t, pd.delta_r
    return d


def server_create(robot: Robot, desc: ServerDesc, arena: torch.Tensor) -> C.c_void_p:
    h = C.c_void_p()
    _check(load().dseed_server_create(robot.handle, C.byref(desc), _dev(arena, torch.uint8, "arena"), C.byref(h)),
           "dseed_server_create")
    return h


def server_destroy(h):
    load().dseed_server_destroy(h)


def server_add_scene(h, scene_id: int, cuboids, grid):
    import numpy as np
    c = np.ascontiguousarray(np.asarray(cuboids, dtype=np.float32).reshape(-1, 6))
    g = make_grid(grid)
    _check(load().dseed_server_add_scene(h, int(scene_id), c.ctypes.data if c.size else None, int(c.shape[0]),
                                         C.byref(g)), "dseed_server_add_scene")


def server_remove_scene(h, scene_id: int):
    _check(load().dseed_server_remove_scene(h, int(scene_id)), "dseed_server_remove_scene")


def server_submit(h, req: Request) -> int:
    t = C.c_longlong()
    _check(load().dseed_server_submit(h, C.byref(req), C.byref(t)), "dseed_server_submit")
    return int(t.value)


def server_step(h, wait: bool = False) -> int:
    n = C.c_int()
    _check(load().dseed_server_step(h, 1 if wait else 0, C.byref(n)), "dseed_server_step")
    return int(n.value)


def server_set_wait_limit(h, seconds: float):
    _check(load().dseed_server_set_wait_limit(h, float(seconds)), "dseed_server_set_wait_limit")


def server_poll(h, ticket: int):
    st, t0, t1 = C.c_int(), C.c_double(), C.c_double()
    _check(load().dseed_server_poll(h, int(ticket), C.byref(st), C.byref(t0), C.byref(t1)), "dseed_server_poll")
    return int(st.value), float(t0.value), float(t1.value)


def server_stats(h) -> ServerStats:
    s = ServerStats()
    _check(load().dseed_server_stats(h, C.byref(s)), "dseed_server_stats")
    return s


# ---------------------------------------------------------------------------- denoiser layers

def nn(name: str, *args):
    """Call dseed_nn_<name>(*args, stream) and raise on failure.  Tensors are
    passed by data pointer (None -> NULL)."""
    conv = []
    for a in args:
        if isinstance(a, torch.Tensor):
            if not a.is_cuda or not a.is_contiguous():
                raise DseedError(f"nn_{name}: tensors must be contiguous CUDA tensors")
            conv.append(a.data_ptr())
        else:
            conv.append(a)
    fn = getattr(load(), "dseed_nn_" + name)
    _check(fn(*conv, _stream()), "dseed_nn_" + name)


EPI_F32, EPI_BF16, EPI_GN = 0, 1, 2


def conv_tc(a0: torch.Tensor, w: torch.Tensor, out: torch.Tensor, *, n_samples: int, L: int, taps: int = 1,
            pad: int = 0, cout: int, a1: Optional[torch.Tensor] = None, bias: Optional[torch.Tensor] = None,
            epilogue: int = EPI_BF16, rows_per_sample: int = 1, gn_eps: float = 1e-5,
            gamma: Optional[torch.Tensor] = None, beta: Optional[torch.Tensor] = None,
            film: Optional[torch.Tensor] = None, sample_problem: Optional[torch.Tensor] = None,
            res: Optional[torch.Tensor] = None, out_ld: Optional[int] = None, err: Optional[torch.Tensor] = None,
            film_ld: int = 0, film_add: Optional[torch.Tensor] = None):
    """dseed_nn_conv_tc: tensor-core convolution with a fused layer tail.
    a0 / a1 BF16 [n_samples][L][c] (channels-last, contiguous); w BF16
    [cout_pad][taps][c0 + c1]; out [n_samples * L][out_ld] (FP32 for EPI_F32)."""
    def ptr(t, name, dtype=None):
        if t is None:
            return None
        if not t.is_cuda or not t.is_contiguous():
            raise DseedError(f"conv_tc: {name} must be a contiguous CUDA tensor")
        if dtype is not None and t.dtype != dtype:
            raise DseedError(f"conv_tc: {name} must be {dtype}")
        return t.data_ptr()
    d = ConvTc()
    d.a0_dev = ptr(a0, "a0", torch.bfloat16)
    d.c0 = int(a0.shape[-1])
    d.a1_dev = ptr(a1, "a1", torch.bfloat16)
    d.c1 = int(a1.shape[-1]) if a1 is not None else 0
    d.n_samples, d.L, d.taps, d.pad = int(n_samples), int(L), int(taps), int(pad)
    d.w_dev = ptr(w, "w", torch.bfloat16)
    d.cout, d.cout_pad = int(cout), int(w.shape[0])
    d.bias_dev = ptr(bias, "bias", torch.float32)
    d.epilogue, d.rows_per_sample, d.gn_eps = int(epilogue), int(rows_per_sample), float(gn_eps)
    d.gamma_dev, d.beta_dev = ptr(gamma, "gamma", torch.float32), ptr(beta, "beta", torch.float32)
    if film is not None and film_ld:
        if not film.is_cuda or film.dtype != torch.float32 or film.stride(-1) != 1:
            raise DseedError("conv_tc: film must be FP32 CUDA rows")
        d.film_dev = film.data_ptr()                 # a column slice of a wider row-major buffer
    else:
        d.film_dev = ptr(film, "film", torch.float32)
    d.film_ld = int(film_ld)
    if film_add is not None:
        if not film_add.is_cuda or film_add.dtype != torch.float32 or film_add.stride(-1) != 1:
            raise DseedError("conv_tc: film_add must be FP32 CUDA values")
        d.film_add_dev = film_add.data_ptr()       # may be a column slice of a wider row
    d.sample_problem_dev = ptr(sample_problem, "sample_problem", torch.int32)
    d.res_dev = ptr(res, "res", torch.bfloat16)
    d.out_dev = ptr(out, "out", torch.float32 if epilogue == EPI_F32 else torch.bfloat16)
    d.out_ld = int(out_ld if out_ld is not None else cout)
    d.err_dev = ptr(err, "err", torch.int32)
    _check(load().dseed_nn_conv_tc(C.byref(d), _stream()), "dseed_nn_conv_tc")
    return out
