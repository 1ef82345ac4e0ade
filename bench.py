"""Benchmark of the seed-parallel trajectory optimiser on one GB300 (or N, as
independent replicas under torchrun).

One step = the whole hot path over one batch: the brute-force ESDF build of
every scene, then the fused optimiser (FK -> spheres -> ESDF trilinear + hinge,
smoothness, goal, limits, hand-written adjoint, L-BFGS update; `iters` times)
and the success test / best-seed selection.  Default workload (the largest that
fits one GPU, "stress"): 1024 problems over 16 dense-clutter scenes of 200
cuboids (256^3 ESDF at 5 mm), 128 seeds x 64 waypoints, 200 iterations; the
"batched" workload (256 problems, one shelf scene each, 128^3 at 1 cm, 64 seeds
x 32 waypoints, 100 iterations) is measured alongside.  Metric: seed-timestep
cost+grad evaluations per second = P * S * T * iters / step time.

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle on
a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)

from paper_2410_16727_gb300 import dist as D  # noqa: E402
from paper_2410_16727_gb300 import inputs as I  # noqa: E402

METRIC = "seed-timestep cost+grad evals/s"
UNIT = "ST-evals/s"
# Algorithmic FP32 work per seed-timestep evaluation of the fused kernel: about
# 4 kflop for kinematics, sphere placement, 50 trilinear lookups with their
# gradient, the Jacobian-transpose adjoint and the smoothness/goal/limit terms,
# plus about 0.3 kflop for the L-BFGS update's share.
FLOP_PER_ST = 4300.0
# Algorithmic HBM bytes per seed-timestep evaluation when nothing is reused from
# L2: the ESDF corners of 50 spheres (8 x 4 B each) plus the trajectory in and
# gradient out (56 B).
HBM_BYTES_PER_ST_NO_REUSE = 50 * 8 * 4 + 56

# ncu counters of one k_plan launch (dram__bytes_read.sum + dram__bytes_write.sum,
# lts__t_sector_hit_rate.pct), per seed-timestep evaluation, valid only for the
# kernel source they were taken with (KERNEL_SOURCES hashed below); the command
# and the raw figures are in profiles/k_plan_<workload>.md.
KERNEL_SOURCES = ("paper_2410_16727_gb300/csrc/device.cuh", "paper_2410_16727_gb300/csrc/kernels_plan.cu",
                  "paper_2410_16727_gb300/csrc/internal.h")
NCU_COUNTERS = {
    # k_plan<2,0,0>, 128 of the 1024 stress problems (all 16 scenes), 200 iterations:
    # 2479.99 MB read + 2392.27 MB written over 128*128*64*200 evaluations; L2 hit 97.57%
    "stress": {"dram_bytes_per_st": (2479.985e6 + 2392.271e6) / (128 * 128 * 64 * 200), "l2_hit_pct": 97.57,
               "kernel_hash": "7c0dbba8147b5a19",
               "capture": "ncu dram__bytes_read/write.sum, lts__t_sector_hit_rate.pct of one k_plan launch, "
                          "128 stress problems, scaled by evaluations (profiles/k_plan_stress.md)"},
    # k_plan<1,0,0>, the full 256-problem batched launch: 368.66 MB read + 69.44 MB written;
    # L2 hit rate 98.36% from the 64-problem launch
    "batched": {"dram_bytes_per_st": (368.663e6 + 69.440e6) / (256 * 64 * 32 * 100), "l2_hit_pct": 98.36,
                "kernel_hash": "7c0dbba8147b5a19",
                "capture": "ncu dram__bytes_read/write.sum of the full batched k_plan launch, "
                           "lts__t_sector_hit_rate.pct of a 64-problem launch (profiles/k_plan_batched.md)"},
}


def kernel_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(HERE, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_peaks() -> dict:
    try:
        with open(os.path.join(HERE, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="dseed", choices=["dseed", "reference"])
    ap.add_argument("--workload", default="stress", choices=list(I.WORKLOADS))
    ap.add_argument("--also", default="batched",
                    help="comma-separated workloads measured alongside the headline ('' for none)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=10000)
    ap.add_argument("--serve-round-iters", type=int, default=10, help="L-BFGS iterations per serving round")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-proposal comparison")
    ap.add_argument("--sweep", type=int, default=2,
                    help="interpolants per segment of the swept-check comparison (0: skip it)")
    ap.add_argument("--learned-scenes", type=int, default=512, help="training scenes (x 196 problems each)")
    ap.add_argument("--learned-steps", type=int, default=24000,
                    help="shelf denoiser training steps (batch 256; 6000 leave it under-trained, most visibly with "
                         "Eq. 2's loss measured on the robot)")
    ap.add_argument("--clutter-steps", type=int, default=24000, help="dense-clutter denoiser training steps (batch 256)")
    ap.add_argument("--learned-requests", type=int, default=2000, help="requests of the seeded serving runs")
    ap.add_argument("--no-learned-stress", action="store_true",
                    help="skip the learned proposal on the stress workload and the serving mix")
    ap.add_argument("--clutter-scenes", type=int, default=256,
                    help="dense-clutter training scenes (x 128 problems each) of the stress-workload denoiser")
    ap.add_argument("--learned-fk", action="store_true",
                    help="also train a denoiser with Eq. 2's loss measured on the robot and compare it")
    ap.add_argument("--problems", type=int, default=None,
                    help="smaller case for profiling: this many problems (and scenes) of the workload")
    return ap.parse_args()


# ---------------------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.path = tempfile.mktemp(suffix=".csv")
        self.proc = None
        self.gpu = gpu_index

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------- GPU arm

def workload_spec(args, name: str) -> I.WorkloadSpec:
    spec = I.WORKLOADS[name]
    if args.problems:
        # smaller case of the same workload (profiling): this many problems, at most as many scenes
        spec = I.WorkloadSpec(spec.name, spec.config_id, min(spec.n_scenes, args.problems), args.problems,
                              spec.S, spec.T, spec.iters, spec.scene, spec.grid)
    return spec


def workload_config(spec: I.WorkloadSpec, world: int) -> dict:
    """The `config` object of both arms (the same dict for the same workload)."""
    return {"workload": f"{spec.name}: {spec.n_problems} problems x {spec.S} seeds x {spec.T} waypoints, "
                        f"{spec.iters} L-BFGS iterations, {spec.n_scenes} {spec.scene} scenes, "
                        f"ESDF {spec.grid.n[0]}^3 at {spec.grid.res * 1000:g} mm",
            "problems": spec.n_problems, "seeds": spec.S, "waypoints": spec.T, "iters": spec.iters,
            "scenes": spec.n_scenes, "l2": "flushed between steps (512 MiB write); inputs larger than L2",
            "parallelism": f"replicas x{world}"}


def fp32_peak(device: int):
    """Peak FP32 rate of the device (TFLOP/s) from its attributes: SMs x FP32
    lanes x 2 (FMA) x peak SM clock."""
    from paper_2410_16727_gb300 import binding as B
    d = B.device_info(device)
    peak = d["sm_count"] * d["fp32_lanes_per_sm"] * 2 * d["sm_clock_khz"] * 1e3 / 1e12
    return peak, (f"derived from cudaDeviceGetAttribute: {d['sm_count']} SMs x {d['fp32_lanes_per_sm']} FP32 "
                  f"lanes x 2 x {d['sm_clock_khz'] / 1e3:g} MHz"), d


def measure_plain(args, spec: I.WorkloadSpec, rank: int, world: int, with_e2e: bool):
    """Time steps (ESDF build of every scene + fused plan + best seed) of one
    workload with its inputs resident; with_e2e also times the same step end to
    end from pinned host buffers through the public API."""
    import torch
    from paper_2410_16727_gb300 import api, binding as B

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    robot = I.make_robot()
    # each rank plans its own problems (replicas of the workload with different seeds)
    cub, grids = I.make_scenes(spec, seed_offset=rank)
    planner = api.Planner(robot, I.CostParams(), I.OptParams(iters=spec.iters), dev)
    planner.set_scenes(cub, grids)
    clear_fn, pose_fn = api.device_workload_fns(planner)
    wl = I.build_workload(spec, cub, grids, clear_fn, pose_fn, seed_offset=rank)
    P, S, T, iters = wl.P, wl.S, wl.T, wl.opt.iters
    st_evals = P * S * T * iters

    # resident device inputs and outputs
    batch = planner.batch(wl.q_start, wl.goal, wl.scene_of_problem, S, T)
    seeds = torch.as_tensor(wl.seeds).to(dev)
    ws = planner.workspace(batch)
    out = dict(traj=torch.empty((P, S, T, 7), device=dev), cost=torch.empty((P, S), device=dev),
               success=torch.empty((P, S), dtype=torch.uint8, device=dev),
               metrics=torch.empty((P, S, B.N_METRICS), device=dev),
               best=torch.empty((P,), dtype=torch.int32, device=dev))
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    def step(ev=None):
        if ev:
            ev[0].record(stream)
        planner.rebuild_scenes()
        if ev:
            ev[1].record(stream)
        B.plan_batch(planner.robot, batch.desc, batch.pr, seeds, ws, out)
        if ev:
            ev[2].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    sampler = ClockSampler(local)
    barrier()
    with sampler:
        t0 = time.perf_counter()
        for k in range(args.steps):
            flush.zero_()      # L2 flush between steps (outside the events)
            step(evs[k])
        barrier()
        wall = time.perf_counter() - t0
    torch.cuda.synchronize()
    esdf_ms = [e[0].elapsed_time(e[1]) for e in evs]
    plan_ms = [e[1].elapsed_time(e[2]) for e in evs]
    step_ms = [a + b for a, b in zip(esdf_ms, plan_ms)]
    ms = D.max_over_ranks(sum(step_ms) / len(step_ms), dev)
    success_rate = float(out["success"].float().mean())
    solved = float((out["best"] >= 0).float().mean())

    e2e = None
    if with_e2e:
        # end to end through the public API with host buffers: H2D of the step's
        # inputs (cuboids, starts, goals, scene ids, seeds) from pinned memory, the
        # step, D2H of trajectories, costs, success flags and best seeds
        h_cub = planner.cub_packed.cpu().pin_memory()      # every scene's cuboids, packed
        h_q = torch.as_tensor(wl.q_start).pin_memory()
        h_goal = torch.as_tensor(wl.goal).pin_memory()
        h_sc = torch.as_tensor(wl.scene_of_problem).pin_memory()
        h_seeds = torch.as_tensor(wl.seeds).pin_memory()
        h_out = {k: torch.empty(v.shape, dtype=v.dtype).pin_memory() for k, v in out.items() if k != "metrics"}
        d_q, d_goal, d_sc = batch.q_start, batch.goal, batch.scene_of_problem
        h2d = sum(t.numel() * t.element_size() for t in (h_cub, h_q, h_goal, h_sc, h_seeds))
        d2h = sum(t.numel() * t.element_size() for t in h_out.values())

        def e2e_step():
            d_q.copy_(h_q, non_blocking=True)
            d_goal.copy_(h_goal, non_blocking=True)
            d_sc.copy_(h_sc, non_blocking=True)
            seeds.copy_(h_seeds, non_blocking=True)
            planner.rebuild_scenes(h_cub)                    # one copy of all cuboids, then the ESDF build
            B.plan_batch(planner.robot, batch.desc, batch.pr, seeds, ws, out)
            for k, v in h_out.items():
                v.copy_(out[k], non_blocking=True)

        for _ in range(2):
            e2e_step()
        torch.cuda.synchronize()
        e_ms = []
        e_sampler = ClockSampler(local)
        with e_sampler:
            for _ in range(max(2, args.steps)):
                flush.zero_()
                torch.cuda.synchronize()
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                e2e_step()
                b.record(stream)
                b.synchronize()
                e_ms.append(a.elapsed_time(b))
        e2e_ms = D.max_over_ranks(sum(e_ms) / len(e_ms), dev)
        e2e = {"value": D.job_throughput(st_evals, e2e_ms, world), "unit": UNIT, "ms_per_step": e2e_ms,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "ms_per_step_min": D.max_over_ranks(min(e_ms), dev), "clocks": e_sampler.summary()}

    plan_avg = sum(plan_ms) / len(plan_ms)
    esdf_avg = sum(esdf_ms) / len(esdf_ms)
    peak, peak_src, dinfo = fp32_peak(local)
    achieved = FLOP_PER_ST * st_evals / (plan_avg * 1e-3) / 1e12
    roof = {"bound": "alu", "kernel": "k_plan (fused cost+adjoint+L-BFGS)", "achieved": achieved, "peak": peak,
            "unit": "TFLOP/s", "frac": achieved / peak, "peak_source": peak_src,
            "flop_per_unit": FLOP_PER_ST, "unit_of_work": "seed-timestep evaluation",
            "units_per_launch": st_evals, "ms_per_launch": plan_avg, "traffic": None,
            "traffic_source": None}
    # HBM side of the same launch (the cost+adjoint gathers): ncu DRAM bytes and
    # L2 hit rate of the kernel as built now, scaled to this launch's evaluations
    hbm = {"peak_gbs": measured_peaks().get("hbm_gbs"), "peak_source": "MEASURED_PEAKS.json hbm_gbs",
           "algorithmic_bytes_per_unit_no_l2_reuse": HBM_BYTES_PER_ST_NO_REUSE,
           "no_reuse_gbs_at_this_rate": HBM_BYTES_PER_ST_NO_REUSE * st_evals / (plan_avg * 1e-3) / 1e9}
    ctr = NCU_COUNTERS.get(spec.name)
    if ctr and ctr["kernel_hash"] == kernel_hash():
        traffic = ctr["dram_bytes_per_st"] * st_evals
        roof["traffic"] = traffic
        roof["traffic_source"] = ctr["capture"]
        hbm.update(dram_bytes_per_launch=traffic, achieved_gbs=traffic / (plan_avg * 1e-3) / 1e9,
                   l2_hit_pct=ctr["l2_hit_pct"], counters_from=ctr["capture"])
        if hbm["peak_gbs"]:
            hbm["frac"] = hbm["achieved_gbs"] / hbm["peak_gbs"]
    else:
        hbm["note"] = "no ncu capture of the kernel as built now"
    roof["hbm"] = hbm
    res = dict(
        config=workload_config(spec, world), ms_per_step=ms, value=D.job_throughput(st_evals, ms, world),
        plans_per_s=P * world / (ms * 1e-3), breakdown_ms={"esdf_build": esdf_avg, "plan": plan_avg},
        seed_success=success_rate, problems_solved=solved, wall_s_timed=wall,
        # our kernels in the timed region: per step the ESDF build (one launch per 256
        # scenes), the fused plan and the best-seed pick
        gpu_launches=args.steps * ((len(cub) + 255) // 256 + 2),
        gpu_launches_per_step=(len(cub) + 255) // 256 + 2,
        roofline=roof, clocks=sampler.summary(), device=dinfo)
    if e2e is not None:
        res["e2e"] = e2e
    del flush, ws, out, seeds
    torch.cuda.empty_cache()
    return res, wl


def run_gpu(args, rank: int, world: int):
    spec = workload_spec(args, args.workload)
    part, wl = measure_plain(args, spec, rank, world, with_e2e=not args.no_e2e)
    res = dict(metric=METRIC, value=part.pop("value"), unit=UNIT, n_gpus=world, steps=args.steps,
               warmup=args.warmup, ms_per_step=part.pop("ms_per_step"), higher_is_better=True, scaling="weak",
               vs_baseline=None, dtype="f32", data="synthetic", config=part.pop("config"))
    res.update(part)
    if "e2e" not in res:
        res["e2e"] = {"value": None, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    also = {}
    for name in [n for n in args.also.split(",") if n and n != args.workload]:
        a, _ = measure_plain(args, workload_spec(args, name), rank, world, with_e2e=False)
        a.pop("clocks", None)
        a.pop("device", None)
        also[name] = a
    if also:
        res["also"] = also
    return res, wl


# ---------------------------------------------------------------------------- swept check

def run_sweep(args, wl) -> dict:
    """Waypoint-only plans against plans with the swept check (args.sweep
    joint-space interpolants per segment) on the benchmark's own problems: plan
    time (ESDFs built, inputs resident, 2 GB of ESDF so L2 holds no whole
    input), success, and every result re-checked at 8 interpolants per segment
    (the continuous-collision test the waypoint-only success does not make)."""
    import dataclasses
    import torch
    from paper_2410_16727_gb300 import api, binding as B

    def planner_for(n):
        pl = api.Planner(wl.robot, dataclasses.replace(wl.cost, n_sweep=n), wl.opt)
        pl.set_scenes(wl.cuboids, wl.grids)
        return pl, pl.batch(wl.q_start, wl.goal, wl.scene_of_problem, wl.S, wl.T)

    checker, cbatch = planner_for(8)
    seeds = torch.as_tensor(np.ascontiguousarray(wl.seeds)).cuda()
    rows = []
    for n in (0, args.sweep):
        pl, batch = planner_for(n)
        for _ in range(2):
            out = pl.plan(batch, seeds)
        torch.cuda.synchronize()
        ts = []
        for _ in range(5):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            out = pl.plan(batch, seeds)
            b.record()
            b.synchronize()
            ts.append(a.elapsed_time(b))
        ok = out["success"].bool()
        ok8 = B.evaluate(checker.robot, cbatch.desc, cbatch.pr, out["traj"])[0].bool() & ok
        best = out["best"].long()
        has = best >= 0
        best_ok8 = torch.zeros_like(has)
        best_ok8[has] = ok8[has.nonzero()[:, 0], best[has]]
        ms = statistics.median(ts)
        P, S, T, it = wl.P, wl.S, wl.T, wl.opt.iters
        rows.append({"n_sweep": n, "plan_ms": ms,
                     "config_evals_per_s": P * S * T * (1 + n) * (it + 1) / (ms * 1e-3),
                     "seed_success": float(ok.float().mean()), "problems_solved": float(ok.any(1).float().mean()),
                     "seed_success_checked_8": float(ok8.float().mean()),
                     "problems_solved_checked_8": float(ok8.any(1).float().mean()),
                     "best_seed_passes_8": float(best_ok8[has].float().mean()) if bool(has.any()) else None})
        del pl, batch, out
    return {"workload": f"the benchmark's {wl.P} problems x {wl.S} seeds x {wl.T} waypoints, "
                        f"{wl.opt.iters} iterations; success re-checked at 8 interpolants per segment",
            "runs": rows}


# ---------------------------------------------------------------------------- serving

def run_serving(args, rank: int) -> dict:
    """Serving workload: Poisson arrivals of planning requests with seed counts
    in {4, 16, 64, 256} and horizons in {32, 48, 64} over a pool of 64 scenes
    (64^3..192^3 ESDFs at 1-2 cm, 10-100 cuboids), 100 iterations each, under a
    120 GB HBM budget.  First the saturation throughput (all requests at once),
    then p50/p99 latency at 0.25, 0.5 and 0.8 of it."""
    import torch
    from paper_2410_16727_gb300 import api, serving as SV

    n = args.serve_requests
    robot = I.make_robot()
    cub, grids = SV.serving_scene_pool(64, seed=rank)
    planner = api.Planner(robot)
    planner.set_scenes(cub, grids)
    cf, pf = api.device_workload_fns(planner)
    sw = SV.build_serving_workload(n, cf, pf, n_scenes=64, seed=rank)
    budget = 120 * 10 ** 9
    out = {"workload": f"{n} requests, S in {{4,16,64,256}}, T in {{32,48,64}}, 64 scenes 64^3-192^3 at 1-2 cm, "
                       f"100 iterations, 120 GB budget, rounds of {args.serve_round_iters} iterations"}

    def fresh():
        sv = SV.Server(sw.robot, budget, max_requests=4096, round_iters=args.serve_round_iters)
        for s, (c, g) in enumerate(zip(sw.cuboids, sw.grids)):
            sv.add_scene(s, c, g)
        torch.cuda.synchronize()
        return sv

    sv = fresh()
    warm = SV.ServingWorkload(sw.robot, sw.cuboids, sw.grids, sw.problems, sw.requests[:64])
    SV.run_trace(sv, warm, None)
    sat = SV.summarize(SV.run_trace(sv, sw, None))
    out["saturation"] = sat
    st_per_req = float(np.mean([S * T for (_, S, T) in sw.requests])) * 100
    out["saturation_st_evals_per_s"] = sat["plans_per_s"] * st_per_req
    sv.close()
    for frac in (0.25, 0.5, 0.8):
        sv = fresh()
        rate = frac * sat["plans_per_s"]
        res = SV.summarize(SV.run_trace(sv, sw, SV.poisson_arrivals(n, rate, seed=int(frac * 100))))
        res["offered_plans_per_s"] = rate
        out[f"load_{frac}"] = res
        sv.close()
    return out


# ---------------------------------------------------------------------------- tensor-core roofline

def conv_tc_roofline() -> dict:
    """The denoiser's widest layer as the DDIM sampler runs it for 32768
    trajectories: a 256 -> 256-channel, 5-tap convolution over 262144 rows (8
    waypoints each) with the fused group norm / Mish / FiLM epilogue, timed alone
    with CUDA events (inputs larger than L2); achieved = 2 M N K / time against
    the measured BF16 dense peak (burst figure: a kernel timed alone)."""
    import torch
    from paper_2410_16727_gb300 import binding as B

    N, L, C, k = 32768, 8, 256, 5
    g = torch.Generator(device="cuda")
    g.manual_seed(0)
    x = torch.randn((N, L, C), device="cuda", generator=g).to(torch.bfloat16)
    w = (torch.randn((C, k, C), device="cuda", generator=g) / (k * C) ** 0.5).to(torch.bfloat16)
    bias, beta = torch.zeros(C, device="cuda"), torch.zeros(C, device="cuda")
    gamma = torch.ones(C, device="cuda")
    film = torch.randn((512, 2 * C), device="cuda", generator=g)
    rows = torch.arange(512, device="cuda", dtype=torch.int32).repeat_interleave(64)
    res = torch.randn((N * L, C), device="cuda", generator=g).to(torch.bfloat16)
    out = torch.empty((N * L, C), dtype=torch.bfloat16, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")

    def run():
        B.conv_tc(x, w, out, n_samples=N, L=L, taps=k, pad=k // 2, cout=C, bias=bias, epilogue=B.EPI_GN,
                  rows_per_sample=L, gamma=gamma, beta=beta, film=film, sample_problem=rows, res=res, err=err)

    for _ in range(3):
        run()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(20)]
    for a, b in evs:
        a.record()
        run()
        b.record()
    torch.cuda.synchronize()
    if int(err.item()) != 0:
        raise RuntimeError("conv_tc reported a pipeline wait that gave up")
    ms = statistics.mean(a.elapsed_time(b) for a, b in evs)
    flop = 2.0 * N * L * C * (k * C)
    achieved = flop / (ms * 1e-3) / 1e12
    peak, src = None, "MEASURED_PEAKS.json bf16_tflops (burst)"
    try:
        with open(os.path.join(HERE, "MEASURED_PEAKS.json")) as f:
            peak = float(json.load(f)["bf16_tflops"])
    except (OSError, KeyError, ValueError):
        peak, src = 1900.0, "fallback 1.9 PFLOP/s bf16 burst"
    return {"bound": "tensor", "kernel": "k_conv_tc<256, GN> (5-tap 256->256, 262144 rows, fused epilogue)",
            "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak, "ms": ms,
            "peak_source": src, "traffic": None}


def conv_tc_shapes() -> list:
    """The denoiser's tensor-core convolution classes at the sampling size
    (32768 trajectories), each timed alone with CUDA events: the group-norm
    epilogue (no FiLM or residual) against the plain BF16 epilogue of the same
    product, so the epilogue's share of each class is visible.  A profiling aid,
    not part of the benchmark line."""
    import torch
    from paper_2410_16727_gb300 import binding as B

    cases = [("256 -> 256, 5 taps, L = 8, group norm", 8, 256, 0, 256, 5, B.EPI_GN),
             ("256 -> 256, 5 taps, L = 8, plain", 8, 256, 0, 256, 5, B.EPI_BF16),
             ("128 -> 128, 5 taps, L = 16, group norm", 16, 128, 0, 128, 5, B.EPI_GN),
             ("128 -> 128, 5 taps, L = 16, plain", 16, 128, 0, 128, 5, B.EPI_BF16),
             ("256 + 256 -> 128, 5 taps, L = 8, group norm (two-tile units)", 8, 256, 256, 128, 5, B.EPI_GN),
             ("64 -> 64, 5 taps, L = 32, group norm (resident weights)", 32, 64, 0, 64, 5, B.EPI_GN),
             ("64 -> 64, 5 taps, L = 32, plain (resident weights)", 32, 64, 0, 64, 5, B.EPI_BF16)]
    N = 32768
    g = torch.Generator(device="cuda")
    g.manual_seed(0)
    rows = []
    for name, L, C0, C1, cout, k, epi in cases:
        x0 = torch.randn((N, L, C0), device="cuda", generator=g).to(torch.bfloat16)
        x1 = torch.randn((N, L, C1), device="cuda", generator=g).to(torch.bfloat16) if C1 else None
        w = (torch.randn((cout, k, C0 + C1), device="cuda", generator=g) / (k * (C0 + C1)) ** 0.5).to(torch.bfloat16)
        zeros, ones = torch.zeros(cout, device="cuda"), torch.ones(cout, device="cuda")
        out = torch.empty((N * L, cout), dtype=torch.bfloat16, device="cuda")
        err = torch.zeros(1, dtype=torch.int32, device="cuda")
        kw = dict(a1=x1, n_samples=N, L=L, taps=k, pad=k // 2, cout=cout, bias=zeros, epilogue=epi, err=err)
        if epi == B.EPI_GN:
            kw.update(rows_per_sample=L, gamma=ones, beta=zeros)
        for _ in range(3):
            B.conv_tc(x0, w, out, **kw)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(20):
            B.conv_tc(x0, w, out, **kw)
        b.record()
        b.synchronize()
        if int(err.item()) != 0:
            raise RuntimeError("conv_tc reported a pipeline wait that gave up")
        us = a.elapsed_time(b) / 20 * 1e3
        rows.append({"layer": name, "us": us, "tflops": 2.0 * N * L * cout * k * (C0 + C1) / us / 1e6})
    return rows


# ---------------------------------------------------------------------------- learned proposal

def run_learned(args) -> dict:
    """Learned seeding against the plain method on held-out problems.

    Training: problems on generated shelf scenes (196 per scene), solved by the
    plain optimiser (64 random seeds x 100 iterations); the best successful
    trajectory of each solved problem trains the denoiser (Adam, batch 256).
    Evaluation: 512 problems on 64 unseen shelf scenes.  Offline: problems
    solved and wall time of the plain method at several iteration budgets and of
    DDIM proposals + 20 refinement iterations, and the plain method's result at
    the learned pipeline's wall time.  Serving: the same problems as Poisson
    arrivals at one offered load, plain (64 seeds x 100 iterations) vs seeded
    (proposals on arrival + 20 iterations), p50/p99 latency and plans/s."""
    import torch
    from paper_2410_16727_gb300 import api, binding as B, denoiser as DN, learned as L, netspec as NS, serving as SV

    robot = I.make_robot()
    planner = api.Planner(robot)
    out = {}
    t0 = time.perf_counter()
    tr = L.make_problems(planner, args.learned_scenes, 196, seed=0)
    data = L.build_dataset(planner, robot, tr)
    torch.cuda.synchronize()
    out["train_data"] = {"problems": int(tr.q_start.shape[0]), "trajectories": int(data.x0.shape[0]),
                         "seconds": round(time.perf_counter() - t0, 1)}
    net = DN.Denoiser(NS.NetSpec(), seed=0)
    t0 = time.perf_counter()
    losses = L.train(net, data, args.learned_steps, batch=256, lr=3e-4, log_every=max(1, args.learned_steps // 4))
    torch.cuda.synchronize()
    out["training"] = {"steps": args.learned_steps, "batch": 256, "params": int(net.n_params),
                       "seconds": round(time.perf_counter() - t0, 1), "loss": [round(l, 4) for _, l in losses]}
    net_fk = None
    if args.learned_fk:
        # the same data and schedule, the error measured on points on the robot's sphere surfaces (Eq. 2)
        net_fk = DN.Denoiser(NS.NetSpec(), seed=0)
        t0 = time.perf_counter()
        losses = L.train(net_fk, data, args.learned_steps, batch=256, lr=3e-4,
                         log_every=max(1, args.learned_steps // 4), fk_robot=B.Robot(robot))
        torch.cuda.synchronize()
        out["training_fk_loss"] = {"steps": args.learned_steps, "seconds": round(time.perf_counter() - t0, 1),
                                   "loss_m2": [float(f"{l:.4g}") for _, l in losses]}
    del data, tr
    te = L.make_problems(planner, 64, 8, seed=1)
    P = int(te.q_start.shape[0])

    def timed(fn):
        torch.cuda.synchronize()
        t = time.perf_counter()
        r = fn()
        torch.cuda.synchronize()
        return r, time.perf_counter() - t

    def score(o):
        return float((o["best"] >= 0).float().mean()), float(o["success"].float().mean())

    rnd = torch.as_tensor(L.random_seeds(te, robot, 64, 32, seed=5)).cuda()
    L.solve(planner, te, rnd, 100, chunk=P)                                   # warm-up
    plain = {}
    for it in (100, 50, 30, 20, 10, 5):
        o, dt = timed(lambda: L.solve(planner, te, rnd, it, chunk=P))
        sv, ss = score(o)
        plain[it] = {"iters": it, "solved": round(sv, 4), "seed_success": round(ss, 4), "ms": round(dt * 1e3, 2)}
    out["heldout"] = {"problems": P, "scenes": 64, "plain_seeds": 64, "plain": list(plain.values())}
    def evaluate_net(model):
        learned, diff_only = [], []
        for S, d, it in ((64, 10, 20), (12, 5, 20), (12, 5, 10)):
            L.propose(model, robot, te, S, steps=d)                            # warm-up
            seeds, t_d = timed(lambda: L.propose(model, robot, te, S, steps=d))
            if it == 20:
                diff_only.append({"samples": S, "ddim_steps": d, **L.diffusion_only(planner, te, seeds)})
            o, t_p = timed(lambda: L.solve(planner, te, seeds, it, chunk=P))
            sv, ss = score(o)
            total = (t_d + t_p) * 1e3
            # the plain method at the same wall time: its largest measured budget that fits
            fit = [v for v in plain.values() if v["ms"] <= total]
            eq = max(fit, key=lambda v: v["iters"]) if fit else None
            learned.append({"samples": S, "ddim_steps": d, "iters": it, "solved": round(sv, 4),
                            "seed_success": round(ss, 4), "ddim_ms": round(t_d * 1e3, 2),
                            "plan_ms": round(t_p * 1e3, 2), "total_ms": round(total, 2),
                            "plain_at_equal_time": ({"iters": eq["iters"], "solved": eq["solved"], "ms": eq["ms"]}
                                                    if eq else None)})
        return learned, diff_only

    out["heldout"]["learned"], out["heldout"]["diffusion_only"] = evaluate_net(net)
    if net_fk is not None:
        lf, df = evaluate_net(net_fk)
        out["heldout"]["fk_loss"] = {"learned": lf, "diffusion_only": df}
        del net_fk
    # the (12, 5) proposal for all 512 problems as one CUDA-graph replay, without and
    # with cost-gradient guidance (Eq. 5, k = 60, n = 20)
    occ_all = te.occ[te.scene_of_problem.long()]
    graphed = []
    for guided in (False, True):
        kw = dict(guidance=L.Guidance(), planner=planner, table=te.table) if guided else {}
        gall = L.ProposalGraph(net, robot, P, 12, 5, seed=1, **kw)
        gall(te.q_start, te.q_goal, te.goal, occ_all, te.scene_of_problem)
        seeds, t_d = timed(lambda: gall(te.q_start, te.q_goal, te.goal, occ_all, te.scene_of_problem))
        seeds = seeds.contiguous().clone()
        gall.check()
        for it in (10, 20):
            o, t_p = timed(lambda: L.solve(planner, te, seeds, it, chunk=P))
            sv_, ss_ = score(o)
            total = (t_d + t_p) * 1e3
            fit = [v for v in plain.values() if v["ms"] <= total]
            eq = max(fit, key=lambda v: v["iters"]) if fit else None
            graphed.append({"samples": 12, "ddim_steps": 5, "guided": guided, "iters": it, "solved": round(sv_, 4),
                            "seed_success": round(ss_, 4), "ddim_ms": round(t_d * 1e3, 2),
                            "plan_ms": round(t_p * 1e3, 2), "total_ms": round(total, 2),
                            "plain_at_equal_time": ({"iters": eq["iters"], "solved": eq["solved"], "ms": eq["ms"]}
                                                    if eq else None)})
        del gall
    out["heldout"]["learned_graph"] = graphed

    out["roofline_tc"] = conv_tc_roofline()

    # serving: the held-out problems as Poisson arrivals
    budget = 16 * 10 ** 9
    problems = [(int(te.scene_of_problem[p]), te.q_start[p].cpu().numpy(), te.goal[p].cpu().numpy())
                for p in range(P)]
    rng = np.random.default_rng(77)
    n = args.learned_requests
    reqs = [int(x) for x in rng.integers(0, P, n)]
    rnd_host = rnd.cpu().numpy()

    def server(iters):
        # rounds of 10 iterations let new requests join a 100-iteration batch; a
        # 20-iteration seeded request runs in one round
        sv = SV.Server(robot, budget, max_requests=4096, round_iters=min(iters, 20), opt=I.OptParams(iters=iters))
        for s, (c, g) in enumerate(zip(te.cuboids, te.grids)):
            sv.add_scene(s, c, g)
        torch.cuda.synchronize()
        return sv

    sw = SV.ServingWorkload(robot, te.cuboids, te.grids,
                            [SV.ServingProblem(pr[0], pr[1], pr[2], {(64, 32): rnd_host[p]}) for p, pr in
                             enumerate(problems)], [(p, 64, 32) for p in reqs])
    sv = server(100)
    SV.run_trace(sv, SV.ServingWorkload(robot, te.cuboids, te.grids, sw.problems, sw.requests[:64]), None)
    sat = SV.summarize(SV.run_trace(sv, sw, None))
    sv.close()
    occ = te.occ[te.scene_of_problem.long()]
    rate = 0.5 * sat["plans_per_s"]
    arr = SV.poisson_arrivals(n, rate, seed=5)
    sv = server(100)
    res_p = SV.summarize(SV.run_trace(sv, sw, arr))
    sv.close()
    out["serving"] = {"workload": f"{n} requests over the {P} held-out problems, T = 32, 16 GB budget, rounds of "
                                  f"up to 20 iterations; offered load = half the plain method's saturation",
                      "plain": {"seeds": 64, "iters": 100, "saturation": sat, "at_load": res_p},
                      "offered_plans_per_s": rate}
    S_l, d_l = 12, 5
    for key, it_l, kw in (("seeded", 20, {}),
                          ("seeded_guided", 10, dict(guidance=L.Guidance(), planner=planner, table=te.table))):
        graph = L.ProposalGraphs(net, robot, (2, 8, 64), S_l, d_l, **kw)     # a group of arrivals = one replay

        def propose(idx):
            ix = torch.as_tensor(idx, dtype=torch.long, device=occ.device)
            return graph(te.q_start[ix], te.q_goal[ix], te.goal[ix], occ[ix], te.scene_of_problem[ix])

        svl = server(it_l)
        SV.run_trace_seeded(svl, problems, reqs[:64], None, propose)
        sat_l = SV.summarize(SV.run_trace_seeded(svl, problems, reqs, None, propose))
        svl.close()
        svl = server(it_l)
        res_l = SV.summarize(SV.run_trace_seeded(svl, problems, reqs, arr, propose))
        svl.close()
        graph.check()
        out["serving"][key] = {"samples": S_l, "ddim_steps": d_l, "guided": bool(kw), "iters": it_l,
                               "saturation": sat_l, "at_load": res_l}
        del graph
    return out


# ---------------------------------------------------------------------------- learned proposal on the stress and serving workloads

def run_learned_stress(args, wl) -> dict:
    """Learned seeding on the stress workload and in the serving mix.

    Training: problems on generated dense-clutter scenes (the stress family,
    other seeds), solved by the plain optimiser at the stress horizon (64
    seeds x 200 iterations, T = 64); the best successful solution of each
    solved problem (and its reversal) trains the denoiser at 32 waypoints
    (every second waypoint).  Stress: the benchmark's own 1024 problems, plain
    (its 128 random seeds at several iteration budgets) against DDIM
    proposals (32 waypoints resampled in time to 64) refined by the plain
    optimiser; plans/s at matched success.  Serving mix: the serving
    workload's requests (horizons 32, 48, 64) seeded on arrival (the proposals
    resampled to each request's horizon) against the plain requests."""
    import torch
    from paper_2410_16727_gb300 import api, denoiser as DN, learned as L, netspec as NS, serving as SV

    robot = I.make_robot()
    out = {}
    planner = api.Planner(robot)
    t0 = time.perf_counter()
    tr = L.make_problems(planner, args.clutter_scenes, 128, seed=0, kind="clutter")
    data = L.build_dataset(planner, robot, tr)
    torch.cuda.synchronize()
    out["train_data"] = {"scenes": args.clutter_scenes, "problems": int(tr.q_start.shape[0]),
                         "trajectories": int(data.x0.shape[0]), "seconds": round(time.perf_counter() - t0, 1),
                         "solved_at": "T = 64, 64 random seeds x 200 iterations; trained at 32 waypoints"}
    net = DN.Denoiser(NS.NetSpec(), seed=0)
    t0 = time.perf_counter()
    losses = L.train(net, data, args.clutter_steps, batch=256, lr=3e-4, log_every=max(1, args.clutter_steps // 4))
    torch.cuda.synchronize()
    out["training"] = {"steps": args.clutter_steps, "batch": 256, "seconds": round(time.perf_counter() - t0, 1),
                       "loss": [round(l, 4) for _, l in losses]}
    del data, tr
    planner.set_scenes(wl.cuboids, wl.grids)
    dev = planner.device
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a)).to(dev)
    occ = L.occupancy(planner, wl.cuboids, L.OCC_GRIDS["clutter"])
    ps = L.ProblemSet(wl.cuboids, wl.grids, t(wl.scene_of_problem), t(wl.q_start), t(wl.q_goal), t(wl.goal), occ,
                      planner.table, T=wl.T, iters=wl.opt.iters, kind="clutter")
    P = wl.P

    def timed(fn):
        torch.cuda.synchronize()
        t_ = time.perf_counter()
        r = fn()
        torch.cuda.synchronize()
        return r, time.perf_counter() - t_

    def score(o):
        return float((o["best"] >= 0).float().mean()), float(o["success"].float().mean())

    rnd = t(wl.seeds)
    plain = []
    L.solve(planner, ps, rnd, 10, chunk=P)                                     # warm-up
    for S_p, it in ((128, 200), (128, 100), (128, 50), (64, 200), (32, 200)):
        o, dt = timed(lambda: L.solve(planner, ps, rnd[:, :S_p].contiguous(), it, chunk=P))
        sv_, ss_ = score(o)
        plain.append({"seeds": S_p, "iters": it, "solved": round(sv_, 4), "seed_success": round(ss_, 4),
                      "ms": round(dt * 1e3, 2), "plans_per_s": round(P / dt, 1)})
    # the attempts loop (Sec. 5.2, the paper's baseline with N_atp attempts): attempt 1 is the
    # plain 128 x 200 plan of the benchmark's seeds, each later attempt re-plans the problems still
    # unsolved with a new batch of the plain method's seeds (drawn on the host, outside the timing)
    spent = []

    def plan_fn(problems, seeds):
        idx = torch.as_tensor(problems, device=dev)
        b = api.Batch(ps.q_start[idx], ps.goal[idx], ps.scene_of_problem[idx], ps.table, seeds.shape[1], wl.T,
                      planner.cost, I.OptParams(iters=200), dev)
        o, dt_ = timed(lambda: {k: v.clone() for k, v in
                                planner.plan(b, torch.as_tensor(seeds).to(dev).contiguous()).items()})
        spent.append(dt_)
        return o

    def seed_fn(attempt, problems):
        if attempt == 1:
            return rnd[torch.as_tensor(problems, device=dev)]
        return np.stack([I.make_seeds(I._rng(9100 + attempt, int(q), 1), wl.q_start[q], wl.q_goal[q], 128, wl.T,
                                      robot.limits) for q in problems]).astype(np.float32)

    n_atp = 10
    att = api.plan_attempts(plan_fn, seed_fn, P, n_atp)
    cum = np.cumsum(spent)
    attempts_rows = []
    for k in (1, 2, 5, 10):
        used = min(k, len(spent))
        solved_k = float(((att["attempts"] > 0) & (att["attempts"] <= k)).mean())
        attempts_rows.append({"seeds": 128, "iters": 200, "max_attempts": k, "solved": round(solved_k, 4),
                              "ms": round(float(cum[used - 1]) * 1e3, 2),
                              "plans_per_s": round(P / float(cum[used - 1]), 1)})
    learned = []
    occ_rows = occ[ps.scene_of_problem.long()].contiguous()
    for S_l in (16, 32):
        graph = L.ProposalGraph(net, robot, P, S_l, 5, seed=3, out_T=wl.T)
        graph(ps.q_start, ps.q_goal, ps.goal, occ_rows)                      # warm-up
        seeds, t_d = timed(lambda: graph(ps.q_start, ps.q_goal, ps.goal, occ_rows).contiguous().clone())
        graph.check()
        for it in (25, 50, 100, 200):
            o, t_p = timed(lambda: L.solve(planner, ps, seeds, it, chunk=P))
            sv_, ss_ = score(o)
            total = t_d + t_p
            learned.append({"samples": S_l, "ddim_steps": 5, "iters": it, "solved": round(sv_, 4),
                            "seed_success": round(ss_, 4), "ddim_ms": round(t_d * 1e3, 2),
                            "plan_ms": round(t_p * 1e3, 2), "ms": round(total * 1e3, 2),
                            "plans_per_s": round(P / total, 1)})
        del graph, seeds
    ref = plain[0]
    match = [r for r in learned if r["solved"] >= ref["solved"]]
    best = max(match, key=lambda r: r["plans_per_s"]) if match else None
    out["stress"] = {"problems": P, "plain": plain, "plain_attempts": attempts_rows, "learned": learned,
                     "matched_success": ({"plain": ref, "learned": best,
                                          "plans_per_s_ratio": round(best["plans_per_s"] / ref["plans_per_s"], 2)}
                                         if best else None)}
    # serving mix: the serving workload's requests, plain vs seeded on arrival
    n = args.learned_requests
    cub, grids = SV.serving_scene_pool(64, seed=0)
    planner.set_scenes(cub, grids)
    cf, pf = api.device_workload_fns(planner)
    sw = SV.build_serving_workload(n, cf, pf, n_scenes=64, seed=0)
    occ_s = L.occupancy(planner, sw.cuboids, L.OCC_GRIDS["clutter"])
    problems = [(pr.scene, pr.q_start, pr.goal) for pr in sw.problems]
    budget = 120 * 10 ** 9

    def server(iters, round_iters):
        sv = SV.Server(sw.robot, budget, max_requests=4096, round_iters=round_iters, opt=I.OptParams(iters=iters))
        for s_, (c, g) in enumerate(zip(sw.cuboids, sw.grids)):
            sv.add_scene(s_, c, g)
        torch.cuda.synchronize()
        return sv

    sv = server(100, args.serve_round_iters)
    SV.run_trace(sv, SV.ServingWorkload(sw.robot, sw.cuboids, sw.grids, sw.problems, sw.requests[:64]), None)
    sat = SV.summarize(SV.run_trace(sv, sw, None))
    sv.close()
    rate = 0.5 * sat["plans_per_s"]
    arr = SV.poisson_arrivals(n, rate, seed=11)
    sv = server(100, args.serve_round_iters)
    at_p = SV.summarize(SV.run_trace(sv, sw, arr))
    sv.close()
    res_s = {"workload": f"{n} serving requests (S in {{4,16,64,256}}, T in {{32,48,64}}, 64 scenes), plain "
                         f"100 iterations vs seeded on arrival; offered load = half the plain saturation",
             "plain": {"saturation": sat, "at_load": at_p}, "offered_plans_per_s": rate}
    S_l = 16
    q_s = torch.as_tensor(np.stack([pr.q_start for pr in sw.problems])).to(dev)
    q_g = torch.as_tensor(np.stack([pr.q_goal for pr in sw.problems])).to(dev)
    g_s = torch.as_tensor(np.stack([pr.goal for pr in sw.problems])).to(dev)
    sc_s = torch.as_tensor(np.array([pr.scene for pr in sw.problems])).to(dev).long()
    graphs = {T_: L.ProposalGraphs(net, robot, (2, 8, 64), S_l, 5, seed=5 + T_, out_T=T_) for T_ in (32, 48, 64)}

    def propose(idx, T_):
        ix = torch.as_tensor(idx, dtype=torch.long, device=dev)
        return graphs[T_](q_s[ix], q_g[ix], g_s[ix], occ_s[sc_s[ix]])

    reqs = [(p_, T_) for (p_, _, T_) in sw.requests]
    res_s["seeded"] = []
    for it_l in (20, 50):
        svl = server(it_l, it_l)
        SV.run_trace_seeded(svl, problems, reqs[:64], None, propose)
        sat_l = SV.summarize(SV.run_trace_seeded(svl, problems, reqs, None, propose))
        svl.close()
        svl = server(it_l, it_l)
        at_l = SV.summarize(SV.run_trace_seeded(svl, problems, reqs, arr, propose))
        svl.close()
        res_s["seeded"].append({"samples": S_l, "ddim_steps": 5, "iters": it_l, "saturation": sat_l,
                                "at_load": at_l})
    for g_ in graphs.values():
        g_.check()
    out["serving_mix"] = res_s
    return out


# ---------------------------------------------------------------------------- CPU oracle

def host_cpu_model() -> str:
    """The host CPU's model name (x86 /proc/cpuinfo, else lscpu, which names Arm
    cores), with the machine architecture."""
    import platform
    name = ""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    name = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    if not name:
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for line in out.splitlines():
                if line.strip().lower().startswith("model name"):
                    name = line.split(":", 1)[1].strip()
                    break
        except (OSError, subprocess.SubprocessError):
            pass
    return f"{name or 'unknown'} ({platform.machine()})"


def _oracle_problems(spec, n: int, seed_offset: int = 0):
    """The first n problems of the workload exactly as the GPU arm draws them,
    with the oracle's own ESDFs of the scenes they use (inputs drawn with the
    oracle's callbacks).  Returns (oracle, workload, ESDF build seconds)."""
    import oracle
    robot = I.make_robot()
    cub_all, grids_all = I.make_scenes(spec, seed_offset=seed_offset)
    scenes = sorted({p * spec.n_scenes // spec.n_problems for p in range(n)})
    t0 = time.perf_counter()
    orc = oracle.Oracle(robot, I.CostParams(), [grids_all[s] for s in scenes], [cub_all[s] for s in scenes],
                        T=spec.T)
    t_esdf = time.perf_counter() - t0
    wl = I.build_workload(spec, [cub_all[s] for s in scenes], [grids_all[s] for s in scenes],
                          orc.clearance, orc.flange_pose, n_problems=n, seed_offset=seed_offset)
    return orc, wl, t_esdf, len(scenes)


def oracle_sample(spec, seed_offset: int = 0):
    """The FP64 oracle on a 1% sample of the workload (its first ceil(P / 100)
    problems): the ESDF build of the scenes they use plus every seed's plan and
    success test, timed on all host cores.  Returns (ST evals/s, description, cores)."""
    import oracle
    n = max(1, -(-spec.n_problems // 100))
    orc, wl, t_esdf, n_sc = _oracle_problems(spec, n, seed_offset)
    t0 = time.perf_counter()
    orc.plan(wl.scene_of_problem, wl.q_start, wl.goal, wl.seeds, wl.opt)
    t_plan = time.perf_counter() - t0
    evals = n * spec.S * spec.T * spec.iters
    desc = (f"{n} of {spec.n_problems} problems ({n * spec.S} seeds x {spec.T} waypoints x {spec.iters} "
            f"iterations) + the ESDF build of the {n_sc} scene(s) they use: {t_plan:.1f} s plan + "
            f"{t_esdf:.1f} s ESDF")
    return evals / (t_plan + t_esdf), desc, oracle.num_threads()


def run_reference(args, rank: int, world: int):
    """The FP64 oracle on the host cores, one problem of the workload per step:
    the plans of its seeds, timed, plus its share of its scene's ESDF build
    (the build time, measured once, divided by the problems that share the scene)."""
    import oracle
    if world > 1:
        # the launcher gives every rank one OpenMP thread; rank 0 runs alone here
        # (the other ranks exit without work), so it takes the host's cores
        oracle.set_num_threads(len(os.sched_getaffinity(0)))
    spec = workload_spec(args, args.workload)
    n_needed = args.warmup + args.steps
    per_scene = max(1, spec.n_problems // spec.n_scenes)
    # problems 0..n-1, wrapping over the first few if more steps than problems are asked for
    n = min(n_needed, spec.n_problems)
    orc, wl, t_esdf, n_sc = _oracle_problems(spec, n)
    esdf_share = t_esdf / n_sc / per_scene
    step_s = []
    for k in range(n_needed):
        p = k % n
        t0 = time.perf_counter()
        orc.plan(wl.scene_of_problem[p:p + 1], wl.q_start[p:p + 1], wl.goal[p:p + 1], wl.seeds[p:p + 1], wl.opt)
        dt = time.perf_counter() - t0 + esdf_share
        if k >= args.warmup:
            step_s.append(dt)
    evals = spec.S * spec.T * spec.iters
    ms = statistics.mean(step_s) * 1e3
    v = evals / (ms * 1e-3)
    full_ms = spec.n_problems * ms
    sample = (f"one problem per step ({spec.S} seeds x {spec.T} waypoints x {spec.iters} iterations, plans timed) "
              f"+ 1/{per_scene} of its scene's measured ESDF build ({t_esdf / n_sc:.2f} s); "
              f"{args.steps} steps over problems 0..{n - 1}")
    return dict(impl="reference", metric=METRIC, value=v, unit=UNIT, n_gpus=world, steps=args.steps,
                warmup=args.warmup, ms_per_step=ms, higher_is_better=True, scaling="weak",
                vs_baseline=None, dtype="f64", data="synthetic", config=workload_config(spec, world),
                extrapolated_ms_per_full_workload=full_ms,
                cpu_baseline={"value": v, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                              "cpu_model": host_cpu_model(), "sample": sample},
                e2e={"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0})


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args, rank, world)), flush=True)
        return
    import torch
    if world > 1:
        torch.distributed.init_process_group("nccl")
    res, wl = run_gpu(args, rank, world)
    # the swept check, serving, the learned comparisons and the CPU baseline are
    # single-GPU measurements: with several ranks only the headline (and the
    # workloads alongside it) run, so the GPUs are held for the timed work alone
    single = world == 1
    if not single:
        res["sections"] = ("headline and alongside workloads only; the swept check, serving, learned "
                           "comparisons and CPU baseline are measured at n_gpus = 1")
    if rank == 0 and single and args.sweep > 0:
        res["sweep"] = run_sweep(args, wl)
    if single and not args.no_serving:
        res["serving"] = run_serving(args, rank)
    if rank == 0 and single and not args.no_learned:
        res["learned"] = run_learned(args)
        if args.workload == "stress" and not args.no_learned_stress:
            res["learned_stress"] = run_learned_stress(args, wl)
    if rank == 0 and single and not args.no_cpu_baseline:
        v, desc, cores = oracle_sample(workload_spec(args, args.workload))
        res["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                               "cpu_model": host_cpu_model(), "sample": desc}
    if rank == 0:
        print(json.dumps(res), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
