"""The oracle's thread count (its OpenMP loops over seeds and voxels) changes
nothing but the time: every seed is planned by one thread, every voxel written
by one, so plans and ESDFs are bit-identical at 1 and 4 threads."""
import numpy as np

import oracle
from paper_2410_16727_gb300 import inputs as I


def test_results_do_not_depend_on_the_thread_count():
    spec = I.WORKLOADS["tiny"]
    cub, grids = I.make_scenes(spec)
    before = oracle.num_threads()
    try:
        outs = []
        for n in (1, 4):
            oracle.set_num_threads(n)
            assert oracle.num_threads() == n
            orc = oracle.Oracle(I.make_robot(), I.CostParams(), grids, cub, T=16)
            wl = I.build_workload(spec, cub, grids, orc.clearance, orc.flange_pose, n_problems=3, S=8, T=16,
                                  iters=15)
            outs.append((orc.phis[0].copy(),
                          orc.plan(wl.scene_of_problem, wl.q_start, wl.goal, wl.seeds, wl.opt)))
        (e1, p1), (e4, p4) = outs
        assert np.array_equal(e1, e4)
        for k in p1:
            assert np.array_equal(np.asarray(p1[k]), np.asarray(p4[k])), k
    finally:
        oracle.set_num_threads(before)
