"""GPU parity of dseed_nn_fk_mse (Eq. 2's loss measured on the robot) against
the FP64 oracle: loss and gradient with and without per-sample weights, a
ragged sample count, a grid-stride case (fewer threads than waypoints) and an
empty batch; and a training step with it reduces the loss on a fixed batch."""
import numpy as np
import pytest
import torch

from gpu_helpers import rel_l2, to_np
from oracle import denoiser_oracle as DO
from paper_2410_16727_gb300 import binding as B, inputs as I

pytestmark = pytest.mark.gpu

ROBOT = I.make_robot()
RES = 4.0


def _run(h, lin, eps, pred, w, blocks):
    N, T = lin.shape[0], lin.shape[1]
    c = lambda a: torch.as_tensor(np.ascontiguousarray(a, np.float32)).cuda()
    dpred = torch.empty((N, T, 7), device="cuda")
    part = torch.empty(blocks, device="cuda")
    B.nn("fk_mse", h.handle, c(lin), c(eps), c(pred), None if w is None else c(w), N, T, RES, dpred, part, blocks)
    return float(part.sum()), to_np(dpred)


@pytest.mark.parametrize("N,T,blocks,weighted", [(37, 32, 64, True), (300, 32, 4, True), (5, 17, 64, False)])
def test_fk_mse_matches_oracle(gpu_lib, N, T, blocks, weighted):
    h = B.Robot(ROBOT)
    rng = np.random.default_rng(N + T)
    lin = rng.uniform(-0.8, 0.8, (N, T, 7)).astype(np.float32)
    eps = rng.normal(size=(N, T, 7)).astype(np.float32)
    pred = (eps + rng.normal(scale=0.3, size=eps.shape)).astype(np.float32)
    w = (1.0 + 4.0 * (rng.random(N) < 0.3)).astype(np.float32) if weighted else None
    loss, g = _run(h, lin, eps, pred, w, blocks)
    want, wg = DO.fk_mse(ROBOT, lin, eps, pred, RES, weights=w)
    assert abs(loss - want) <= 1e-4 * want, (loss, want)
    assert rel_l2(g, wg) <= 1e-3
    for n in range(0, N, max(1, N // 8)):
        assert rel_l2(g[n], wg[n]) <= 1e-3, n
    # joint by joint: the wrist columns are far smaller than the base's and must hold too
    for j in range(7):
        assert rel_l2(g[..., j], wg[..., j]) <= 1e-3, j


def test_fk_mse_empty_batch(gpu_lib):
    h = B.Robot(ROBOT)
    z = torch.empty((0, 32, 7), device="cuda")
    part = torch.full((8,), 7.0, device="cuda")
    B.nn("fk_mse", h.handle, z, z, z, None, 0, 32, RES, z, part, 8)
    assert float(part.abs().sum()) == 0.0


def test_fk_loss_training_reduces_the_loss(gpu_lib):
    from paper_2410_16727_gb300 import denoiser as DN, learned as LR, netspec as NS
    torch.manual_seed(0)
    spec = NS.NetSpec()
    net = DN.Denoiser(spec, seed=0)
    h = B.Robot(ROBOT)
    N = 32
    g = torch.Generator(device="cuda").manual_seed(1)
    x0 = torch.randn((N, spec.T, spec.D), device="cuda", generator=g) * 0.3
    qs = torch.rand((N, spec.D), device="cuda", generator=g) * 1.6 - 0.8
    qg = torch.rand((N, spec.D), device="cuda", generator=g) * 1.6 - 0.8
    goal = torch.zeros((N, 7), device="cuda")
    goal[:, 3] = 1.0
    occ = (torch.rand((N, spec.occ_n ** 3), device="cuda", generator=g) < 0.1).float()
    k = torch.randint(0, spec.K, (N,), device="cuda", generator=g, dtype=torch.int32)
    eps = torch.randn((N, spec.T, spec.D), device="cuda", generator=g)
    lin = LR.linear_path(qs, qg, spec.T)
    first = None
    for _ in range(60):
        loss = float(net.loss_and_grad(x0, qs, qg, goal, occ, k, eps, fk=(h, lin, LR.RES_SCALE)))
        first = loss if first is None else first
        net.adam_step(lr=1e-3)
    assert loss < 0.5 * first, (first, loss)
