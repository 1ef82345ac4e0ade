"""GPU parity of the seed-proposal denoiser's own kernels against the FP64
oracle: forward pass, loss and every parameter gradient (FP32 training path),
BF16 tensor-core inference against the FP32 forward, DDIM and DDPM kernels,
and the GEMMs on their own."""
import numpy as np
import pytest
import torch

from oracle import denoiser_oracle as DO
from paper_2410_16727_gb300 import binding as B, denoiser as DN, netspec as NS

pytestmark = pytest.mark.gpu


def _inputs(spec, N, seed=0):
    rng = np.random.default_rng(seed)
    return dict(x0=rng.uniform(-1, 1, (N, spec.T, spec.D)).astype(np.float32),
                qs=rng.uniform(-1, 1, (N, spec.D)).astype(np.float32),
                qg=rng.uniform(-1, 1, (N, spec.D)).astype(np.float32),
                goal=rng.normal(size=(N, 7)).astype(np.float32),
                occ=(rng.random((N, spec.occ_n ** 3)) < 0.15).astype(np.float32),
                k=rng.integers(0, spec.K, N).astype(np.int32),
                eps=rng.normal(size=(N, spec.T, spec.D)).astype(np.float32))


def _cuda(a):
    return torch.as_tensor(a).cuda()


def _rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


@pytest.fixture(scope="module")
def net():
    d = DN.Denoiser(NS.NetSpec(), seed=3)
    # perturb the zero-initialised output layer so every parameter gets a gradient
    host = d.params.cpu().numpy()
    rng = np.random.default_rng(9)
    for name in ("fin.o.w", "fin.o.b"):
        off, shape = d.offsets[name]
        n = int(np.prod(shape))
        host[off:off + n] = rng.uniform(-0.1, 0.1, n)
    d.params.copy_(torch.from_numpy(host))
    return d


def test_forward_matches_oracle(gpu_lib, net):
    inp = _inputs(net.spec, 3)
    xk = inp["x0"]
    got = net.forward(_cuda(xk), _cuda(inp["k"]), _cuda(inp["qs"]), _cuda(inp["qg"]), _cuda(inp["goal"]),
                      _cuda(inp["occ"]))
    want = DO.predict(net.spec, net.params.cpu().numpy(), xk, inp["k"], inp["qs"], inp["qg"], inp["goal"], inp["occ"])
    assert _rel(got.cpu().numpy(), want) <= 1e-4


def test_loss_and_gradients_match_oracle(gpu_lib, net):
    inp = _inputs(net.spec, 4, seed=1)
    w = np.array([1.0, 5.0, 1.0, 5.0], np.float32)        # Eq. 2 style per-sample weights
    net.grads.zero_()
    loss = net.loss_and_grad(_cuda(inp["x0"]), _cuda(inp["qs"]), _cuda(inp["qg"]), _cuda(inp["goal"]),
                             _cuda(inp["occ"]), _cuda(inp["k"]), _cuda(inp["eps"]), _cuda(w))
    ref_loss, ref_g = DO.loss_and_grads(net.spec, net.params.cpu().numpy(), inp["x0"], inp["qs"], inp["qg"],
                                        inp["goal"], inp["occ"], inp["k"], inp["eps"], net.abar.cpu().double().numpy(), w)
    assert abs(float(loss) - ref_loss) <= 1e-4 * abs(ref_loss)
    g = net.grads.cpu().numpy()
    assert _rel(g, ref_g) <= 1e-3
    worst = []
    for name, (off, shape) in net.offsets.items():
        n = int(np.prod(shape))
        r = _rel(g[off:off + n], ref_g[off:off + n])
        worst.append((r, name))
        assert r <= 5e-3 or np.linalg.norm(ref_g[off:off + n]) < 1e-9, (name, r)
    net.grads.zero_()


def test_bf16_inference_close_to_fp32(gpu_lib, net):
    inp = _inputs(net.spec, 64, seed=2)
    args = [_cuda(inp[k]) for k in ("x0", "k", "qs", "qg", "goal", "occ")]
    f32 = net.forward(*args).cpu().numpy()
    b16 = net.infer(*args).cpu().numpy()
    assert _rel(b16, f32) <= 3e-2


def test_tensor_core_unet_matches_oracle(gpu_lib, net):
    """The sampling path (BF16 activations, tcgen05 convolutions with fused
    group norm / Mish / FiLM / residual) against the FP64 oracle forward."""
    inp = _inputs(net.spec, 40, seed=12)
    args = [_cuda(inp[k]) for k in ("x0", "k", "qs", "qg", "goal", "occ")]
    got = net.infer_tc(*args).cpu().numpy()
    want = DO.predict(net.spec, net.params.cpu().numpy(), inp["x0"], inp["k"], inp["qs"], inp["qg"], inp["goal"],
                      inp["occ"])
    assert _rel(got, want) <= 3e-2
    # per sample too: no sample (tile position, ragged last tile) is off
    for n in range(40):
        assert _rel(got[n], want[n]) <= 6e-2, n


def test_tensor_core_unet_full_size_sampled(gpu_lib, net):
    """The launch size of the sampler (512 problems x 64 samples = 32768
    trajectories: 8192 tiles at the first level, many per persistent CTA):
    sampled trajectories against the FP64 oracle, and the result of one
    trajectory does not depend on the batch it runs in."""
    N = 32768
    inp = _inputs(net.spec, 64, seed=21)
    rng = np.random.default_rng(22)
    pick = rng.integers(0, 64, N)                       # every sample is one of 64 reference inputs
    big = {k: v[pick] for k, v in inp.items()}
    args = [_cuda(big[k]) for k in ("x0", "k", "qs", "qg", "goal", "occ")]
    got = net.infer_tc(*args).cpu().numpy()
    small = net.infer_tc(*[_cuda(inp[k]) for k in ("x0", "k", "qs", "qg", "goal", "occ")]).cpu().numpy()
    for n in rng.choice(N, 64, replace=False):
        np.testing.assert_array_equal(got[n], small[pick[n]])
    ref_ids = np.unique(pick[rng.choice(N, 8, replace=False)])
    want = DO.predict(net.spec, net.params.cpu().numpy(), inp["x0"][ref_ids], inp["k"][ref_ids], inp["qs"][ref_ids],
                      inp["qg"][ref_ids], inp["goal"][ref_ids], inp["occ"][ref_ids])
    for i, r in enumerate(ref_ids):
        assert _rel(small[r], want[i]) <= 6e-2


def test_ddim_sampling_paths_agree(gpu_lib, net):
    """DDIM with shared per-problem conditions: the tensor-core path and the
    FP32 path give the same trajectories up to BF16 rounding."""
    rng = np.random.default_rng(13)
    P, S = 3, 5
    qs = _cuda(rng.uniform(-1, 1, (P, 7)).astype(np.float32))
    qg = _cuda(rng.uniform(-1, 1, (P, 7)).astype(np.float32))
    goal = _cuda(rng.normal(size=(P, 7)).astype(np.float32))
    occ = _cuda((rng.random((P, net.spec.occ_n ** 3)) < 0.1).astype(np.float32))
    noise = _cuda(rng.normal(size=(P * S, 32, 7)).astype(np.float32))
    rows = torch.arange(P, dtype=torch.int32, device="cuda").repeat_interleave(S)
    a = net.ddim_sample(qs, qg, goal, occ, noise, steps=4, bf16=True, sample_problem=rows).cpu().numpy()
    b = net.ddim_sample(qs, qg, goal, occ, noise, steps=4, bf16=False, sample_problem=rows).cpu().numpy()
    # Four chained steps of an untrained network amplify the BF16 rounding of each
    # evaluation (about 1% relative): over 16 input seeds the trajectories differ by
    # 0.2% to 7.2% (norm-relative).
    assert _rel(a, b) <= 1e-1


def test_gemm_kernels_against_float64():
    rng = np.random.default_rng(4)
    # the last three have few 64 x 64 output tiles and a long K: the 32 x 32 tiling
    for (M, N, K, ta, tb) in [(37, 65, 29, 0, 0), (130, 3, 71, 1, 0), (5, 200, 16, 0, 1), (64, 64, 64, 1, 1),
                              (512, 128, 2048, 0, 1), (100, 70, 300, 1, 0), (257, 33, 1031, 1, 1)]:
        A = rng.normal(size=(K, M) if ta else (M, K)).astype(np.float32)
        Bm = rng.normal(size=(N, K) if tb else (K, N)).astype(np.float32)
        C0 = rng.normal(size=(M, N)).astype(np.float32)
        bias = rng.normal(size=N).astype(np.float32)
        C = _cuda(C0.copy())
        B.nn("gemm_f32", ta, tb, M, N, K, 1.5, _cuda(A), A.shape[1], _cuda(Bm), Bm.shape[1], 0.5, C, N, _cuda(bias))
        want = 1.5 * ((A.T if ta else A).astype(np.float64) @ (Bm.T if tb else Bm)) + 0.5 * C0 + bias
        assert _rel(C.cpu().numpy(), want) <= 1e-5
    # accumulate into C with no bias and a long K: the split-K kernel
    for (M, N, K, ta, tb) in [(64, 96, 4096, 1, 0), (33, 70, 2999, 0, 0), (128, 128, 1024, 1, 0)]:
        A = rng.normal(size=(K, M) if ta else (M, K)).astype(np.float32)
        Bm = rng.normal(size=(N, K) if tb else (K, N)).astype(np.float32)
        C0 = rng.normal(size=(M, N)).astype(np.float32)
        C = _cuda(C0.copy())
        B.nn("gemm_f32", ta, tb, M, N, K, 0.75, _cuda(A), A.shape[1], _cuda(Bm), Bm.shape[1], 1.0, C, N, None)
        want = 0.75 * ((A.T if ta else A).astype(np.float64) @ (Bm.T if tb else Bm)) + C0
        assert _rel(C.cpu().numpy(), want) <= 1e-5
    for (R, Cn) in [(1, 5), (1000, 70), (4099, 256)]:
        y = rng.normal(size=(R, Cn)).astype(np.float32)
        base = rng.normal(size=Cn).astype(np.float32)
        out = _cuda(base.copy())
        B.nn("colsum", _cuda(y), R, Cn, out, 0)
        assert _rel(out.cpu().numpy(), y.astype(np.float64).sum(0)) <= 1e-5
        out = _cuda(base.copy())
        B.nn("colsum", _cuda(y), R, Cn, out, 1)
        assert _rel(out.cpu().numpy(), y.astype(np.float64).sum(0) + base) <= 1e-5
    # more row tiles than a grid's y dimension holds (65535): rows run along x
    M, N, K = 65535 * 64 + 1000, 8, 16
    A = rng.normal(size=(M, K)).astype(np.float32)
    Bm = rng.normal(size=(N, K)).astype(np.float32)
    C = torch.empty((M, N), device="cuda")
    B.nn("gemm_f32", 0, 1, M, N, K, 1.0, _cuda(A), K, _cuda(Bm), K, 0.0, C, N, None)
    rows = rng.choice(M, 256, replace=False)
    rows[0] = M - 1
    assert _rel(C[rows].cpu().numpy(), A[rows].astype(np.float64) @ Bm.T.astype(np.float64)) <= 1e-5
    y = rng.normal(size=(65535 * 256 + 77, 2)).astype(np.float32)
    out = torch.empty(2, device="cuda")
    B.nn("colsum", _cuda(y), y.shape[0], 2, out, 0)
    assert _rel(out.cpu().numpy(), y.astype(np.float64).sum(0)) <= 1e-4
    for (M, N, K) in [(300, 70, 48), (17, 129, 16), (1024, 256, 1280)]:
        A = rng.normal(size=(M, K)).astype(np.float32)
        W = rng.normal(size=(N, K)).astype(np.float32)
        Ab, Wb = _cuda(A).to(torch.bfloat16), _cuda(W).to(torch.bfloat16)
        C = torch.empty((M, N), device="cuda")
        B.nn("gemm_bf16", M, N, K, Ab, Wb, C, None)
        want = Ab.double().cpu().numpy() @ Wb.double().cpu().numpy().T     # exact products of the BF16 inputs
        assert _rel(C.cpu().numpy(), want) <= 1e-5


def test_ddpm_ddim_kernels():
    rng = np.random.default_rng(5)
    x0 = rng.uniform(-1, 1, (6, 32, 7)).astype(np.float32)
    eps = rng.normal(size=x0.shape).astype(np.float32)
    abar = DN.cosine_abar(100).astype(np.float32)
    k = rng.integers(0, 100, 6).astype(np.int32)
    xk = torch.empty_like(_cuda(x0))
    B.nn("ddpm_noise", _cuda(x0), _cuda(eps), _cuda(k), _cuda(abar), 6, 32 * 7, xk)
    want = DO.ddpm_noise(torch.tensor(x0, dtype=torch.float64), torch.tensor(eps, dtype=torch.float64),
                         torch.tensor(k), abar.astype(np.float64)).numpy()
    assert np.abs(xk.cpu().numpy() - want).max() <= 1e-5
    out = torch.empty_like(xk)
    B.nn("ddim_step", xk[2].contiguous(), _cuda(eps[2]), float(abar[k[2]]), float(abar[3]), 32 * 7, 1.0, out[2])
    want = DO.ddim_step(xk[2].cpu().double().numpy(), eps[2].astype(np.float64), float(abar[k[2]]),
                        float(abar[3]), 1.0)
    assert np.abs(out[2].cpu().numpy() - want).max() <= 1e-4


def test_training_reduces_the_loss(gpu_lib):
    """A few hundred Adam steps on a fixed batch: the kernels' gradients descend."""
    d = DN.Denoiser(NS.NetSpec(), seed=0)
    inp = _inputs(d.spec, 32, seed=6)
    args = [_cuda(inp[k]) for k in ("x0", "qs", "qg", "goal", "occ", "k", "eps")]
    losses = []
    for it in range(150):
        losses.append(float(d.loss_and_grad(*args)))
        d.adam_step(lr=1e-3)
    assert losses[-1] < 0.5 * losses[0], (losses[0], losses[-1])
