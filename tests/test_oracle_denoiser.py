"""Pins of the FP64 denoiser oracle: finite-difference gradients of the whole
network, the patch structure of the occupancy encoder, the time-step embedding
and the DDPM / DDIM identities."""
import math

import numpy as np
import torch

from oracle import denoiser_oracle as DO
from paper_2410_16727_gb300 import netspec as NS

TINY = NS.NetSpec(T=8, D=3, chans=(4, 4, 8), kernel=3, groups=2, t_sin=4, t_dim=4, p_dim=4, occ_n=8, occ_p1=2,
                  occ_c1=2, occ_p2=2, occ_c2=2, o_dim=4, K=10)


def _inputs(spec, N, seed=0):
    rng = np.random.default_rng(seed)
    return dict(x0=rng.uniform(-1, 1, (N, spec.T, spec.D)), qs=rng.uniform(-1, 1, (N, spec.D)),
                qg=rng.uniform(-1, 1, (N, spec.D)),
                goal=rng.normal(size=(N, 7)), occ=(rng.random((N, spec.occ_n ** 3)) < 0.2).astype(np.float64),
                k=rng.integers(0, spec.K, N), eps=rng.normal(size=(N, spec.T, spec.D)))


def test_gradcheck_whole_network():
    N = 2
    inp = _inputs(TINY, N)
    rng = np.random.default_rng(1)
    flat = torch.tensor(rng.normal(scale=0.3, size=NS.param_count(TINY)), dtype=torch.float64, requires_grad=True)
    abar = np.linspace(0.99, 0.1, TINY.K)
    t = lambda a: torch.as_tensor(a, dtype=torch.float64)
    k = torch.as_tensor(inp["k"], dtype=torch.long)

    def loss(f):
        P = DO.unpack(TINY, f)
        xk = DO.ddpm_noise(t(inp["x0"]), t(inp["eps"]), k, abar)
        pred = DO.forward(TINY, P, xk, k, t(inp["qs"]), t(inp["qg"]), t(inp["goal"]), t(inp["occ"]))
        return ((pred - t(inp["eps"])) ** 2).mean()

    assert torch.autograd.gradcheck(loss, (flat,), eps=1e-6, atol=1e-7, rtol=1e-5, fast_mode=True)
    # loss_and_grads returns the same gradient
    l, g = DO.loss_and_grads(TINY, flat.detach().numpy(), inp["x0"], inp["qs"], inp["qg"], inp["goal"], inp["occ"],
                             inp["k"], inp["eps"], abar)
    flat.grad = None
    ref = loss(flat)
    ref.backward()
    assert abs(l - float(ref.detach())) < 1e-12
    np.testing.assert_allclose(g, flat.grad.numpy(), rtol=1e-10, atol=1e-14)


def test_occupancy_encoder_is_a_patch_linear_map():
    """Strided 3-D convolutions with kernel = stride act on disjoint patches: the
    first layer's output at patch (z, y, x) depends only on voxels of that patch,
    with weight entry (dz, dy, dx) -- checked voxel by voxel."""
    spec = TINY
    rng = np.random.default_rng(2)
    P = DO.unpack(spec, torch.tensor(rng.normal(size=NS.param_count(spec))))
    n, p1 = spec.occ_n, spec.occ_p1
    for _ in range(5):
        z, y, x = rng.integers(0, n, 3)
        occ = torch.zeros(1, 1, n, n, n, dtype=torch.float64)
        occ[0, 0, z, y, x] = 1.0
        w1 = P["o.c1.w"].view(spec.occ_c1, p1, p1, p1, 1).permute(0, 4, 1, 2, 3)
        out = torch.nn.functional.conv3d(occ, w1, P["o.c1.b"], stride=p1)
        expect = P["o.c1.b"].view(-1, 1, 1, 1).expand_as(out[0]).clone()
        dz, dy, dx = z % p1, y % p1, x % p1
        expect[:, z // p1, y // p1, x // p1] += P["o.c1.w"][:, (dz * p1 + dy) * p1 + dx]
        assert torch.allclose(out[0], expect, atol=1e-12)


def test_sinusoid_closed_form():
    k = torch.tensor([0, 1, 7])
    e = DO.sinusoid(k, 8)
    assert torch.all(e[0, 0::2] == 0) and torch.all(e[0, 1::2] == 1)
    for j, kk in enumerate([0, 1, 7]):
        for i in range(4):
            w = 10000 ** (-i / 4)
            assert abs(float(e[j, 2 * i]) - math.sin(kk * w)) < 1e-12
            assert abs(float(e[j, 2 * i + 1]) - math.cos(kk * w)) < 1e-12


def test_ddpm_and_ddim_identities():
    rng = np.random.default_rng(3)
    x0 = rng.uniform(-0.9, 0.9, (4, 8, 3))
    eps = rng.normal(size=x0.shape)
    abar = np.array([0.98, 0.7, 0.3, 0.05])
    k = np.array([0, 1, 2, 3])
    xk = DO.ddpm_noise(torch.tensor(x0), torch.tensor(eps), torch.tensor(k), abar).numpy()
    # noising is the affine map of the definition
    np.testing.assert_allclose(xk, np.sqrt(abar[k])[:, None, None] * x0 + np.sqrt(1 - abar[k])[:, None, None] * eps)
    # with the true noise, one DDIM step to abar = 1 returns the clean trajectory
    for n in range(4):
        back = DO.ddim_step(xk[n], eps[n], abar[k[n]], 1.0, clip=10.0)
        np.testing.assert_allclose(back, x0[n], atol=1e-12)
    # and a step to an intermediate level lands on that level's noising of x0
    mid = DO.ddim_step(xk[3], eps[3], abar[3], abar[1], clip=10.0)
    np.testing.assert_allclose(mid, np.sqrt(abar[1]) * x0[3] + np.sqrt(1 - abar[1]) * eps[3], atol=1e-12)


def test_group_norm_moments_and_mish():
    rng = np.random.default_rng(4)
    P = DO.unpack(TINY, torch.tensor(rng.normal(size=NS.param_count(TINY))))
    x = torch.tensor(rng.normal(size=(3, 4, 8)) * 5 + 2)
    P["d1b.g1.w"][:] = 1.0
    P["d1b.g1.b"][:] = 0.0
    y = DO._gn(x, P, "d1b.g1", TINY)
    g = y.view(3, 2, -1)
    assert torch.allclose(g.mean(-1), torch.zeros(3, 2, dtype=torch.float64), atol=1e-10)
    assert torch.allclose(g.var(-1, unbiased=False), torch.ones(3, 2, dtype=torch.float64), atol=1e-4)
    v = torch.tensor([0.0, 1.0, -2.0, 30.0], dtype=torch.float64)
    m = torch.nn.functional.mish(v)
    want = [0.0, math.tanh(math.log1p(math.e)), -2.0 * math.tanh(math.log1p(math.exp(-2.0))), 30.0]
    np.testing.assert_allclose(m.numpy(), want, rtol=1e-12, atol=1e-12)
