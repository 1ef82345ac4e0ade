"""dseed_plan_batch_static: the plan entry point for callers that cannot
allocate device memory (a frozen-memory control loop, a plug-in that may not
touch its host's allocator).  Its scratch is a fixed array inside the library,
so it must give the same results as dseed_plan_batch with a caller workspace,
call after call, without allocating.  This file sorts last so that a run that
stops at the first failure has run every other test first."""
import pytest
import torch

from gpu_helpers import gpu_side, oracle_workload
from paper_2410_16727_gb300 import binding as B

pytestmark = pytest.mark.gpu


def _outputs(wl):
    dev = "cuda"
    P, S, T = wl.P, wl.S, wl.T
    return dict(traj=torch.empty((P, S, T, 7), device=dev), cost=torch.empty((P, S), device=dev),
                success=torch.empty((P, S), dtype=torch.uint8, device=dev),
                metrics=torch.empty((P, S, B.N_METRICS), device=dev),
                best=torch.empty((P,), dtype=torch.int32, device=dev))


def test_static_plan_matches_workspace_plan_twice(gpu_lib):
    wl, orc = oracle_workload("tiny", n_scenes=2, n_problems=2, S=32, T=32, iters=60)
    planner, batch = gpu_side(wl)
    seeds = torch.as_tensor(wl.seeds).cuda()
    ref = planner.plan(batch, seeds)
    outs = [_outputs(wl), _outputs(wl)]
    torch.cuda.synchronize()
    B.plan_batch_static(planner.robot, batch.desc, batch.pr, seeds, outs[0])      # first call: set-up
    torch.cuda.synchronize()
    free_before = torch.cuda.mem_get_info()[0]
    B.plan_batch_static(planner.robot, batch.desc, batch.pr, seeds, outs[1])
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free_before, "the second call changed free device memory"
    for out in outs:
        torch.testing.assert_close(out["traj"], ref["traj"], rtol=1e-5, atol=1e-5)
        torch.testing.assert_close(out["cost"], ref["cost"], rtol=1e-5, atol=1e-6)
        torch.testing.assert_close(out["metrics"], ref["metrics"], rtol=1e-5, atol=1e-6)
        assert torch.equal(out["success"], ref["success"])
        assert torch.equal(out["best"], ref["best"])


def test_static_plan_refuses_oversize_batches(gpu_lib):
    wl, orc = oracle_workload("tiny", S=4, T=32, iters=2)
    planner, batch = gpu_side(wl)
    desc = B.plan_desc(1, 4096, 32, wl.cost, wl.opt)      # 4096 seeds need ~36 MiB of history
    need = B.plan_workspace_bytes(desc)
    assert need > B.STATIC_SCRATCH_BYTES
    seeds = torch.zeros((1, 4096, 32, 7), device="cuda")
    with pytest.raises(B.DseedError, match="static scratch holds"):
        B.plan_batch_static(planner.robot, desc, batch.pr, seeds)
