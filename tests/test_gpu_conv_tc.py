"""The tensor-core convolution (tcgen05 + TMA, fused layer tail) against
float64 references computed from the same BF16-rounded operands: plain GEMMs,
multi-tap convolutions with zero padding, two-source (concatenated) inputs,
ragged last tiles, and the group norm -> Mish -> FiLM -> residual epilogue."""
import numpy as np
import pytest
import torch

from paper_2410_16727_gb300 import binding as B

pytestmark = pytest.mark.gpu


def _bf(a):
    return torch.as_tensor(np.ascontiguousarray(a, np.float32)).cuda().to(torch.bfloat16)


def _f64(t):
    return t.float().cpu().double().numpy()


def _conv_ref(x, w, pad):
    """x [N][L][C] float64, w [O][k][C] -> [N][L][O] (stride 1, zero padding)."""
    N, L, C = x.shape
    O, k, _ = w.shape
    xp = np.zeros((N, L + k, C))
    xp[:, pad:pad + L] = x
    out = np.zeros((N, L, O))
    for j in range(k):
        out += xp[:, j:j + L] @ w[:, j, :].T
    return out


def _mish(v):
    return v * np.tanh(np.log1p(np.exp(np.minimum(v, 20.0))) + np.maximum(v - 20.0, 0.0))


@pytest.mark.parametrize("M,K,cout,cout_pad", [(300, 64, 7, 16), (128, 192, 64, 64), (1000, 128, 128, 128),
                                               (77, 512, 256, 256), (4096, 64, 64, 64),
                                               # two-tile units (128 outputs, K >= 1280; ragged last unit)
                                               (120001, 1280, 128, 128), (117000, 192, 256, 256)])
def test_plain_gemm(gpu_lib, M, K, cout, cout_pad):
    rng = np.random.default_rng(M + K)
    a = _bf(rng.normal(size=(M, K)))
    w = torch.zeros((cout_pad, K), dtype=torch.bfloat16, device="cuda")
    w[:cout] = _bf(rng.normal(size=(cout, K)) / np.sqrt(K))
    bias = torch.as_tensor(rng.normal(size=cout_pad).astype(np.float32)).cuda()
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    out32 = torch.full((M, cout), np.nan, dtype=torch.float32, device="cuda")
    B.conv_tc(a, w, out32, n_samples=M, L=1, cout=cout, bias=bias, epilogue=B.EPI_F32, err=err)
    ref = _f64(a) @ _f64(w)[:cout].T + bias.cpu().double().numpy()[:cout]
    got = out32.cpu().double().numpy()
    assert int(err.item()) == 0
    assert np.abs(got - ref).max() <= 1e-4 * max(1.0, np.abs(ref).max())
    ld = (cout + 7) // 8 * 8
    out16 = torch.zeros((M, ld), dtype=torch.bfloat16, device="cuda")
    B.conv_tc(a, w, out16, n_samples=M, L=1, cout=cout, bias=bias, epilogue=B.EPI_BF16, out_ld=ld, err=err)
    got16 = _f64(out16)[:, :cout]
    assert np.abs(got16 - ref).max() <= 8e-3 * max(1.0, np.abs(ref).max())
    assert np.all(_f64(out16)[:, cout:] == 0)            # columns past cout untouched


@pytest.mark.parametrize("N,L,C0,C1,k,cout,pad", [
    (9, 32, 64, 0, 5, 64, 2), (20, 16, 128, 0, 5, 128, 2), (33, 8, 256, 256, 5, 256, 2),
    (5, 16, 128, 128, 3, 128, 1), (7, 32, 64, 0, 1, 256, 0),
    # wide outputs run in CTA pairs: several units per CTA, odd tile count
    (4001, 8, 64, 0, 3, 256, 1), (4001, 16, 128, 0, 3, 128, 1),
    # two taps over row pairs (the stride-2 convolution), one-sided padding
    (301, 16, 128, 0, 2, 64, 1), (77, 8, 256, 0, 2, 128, 1), (50, 32, 64, 0, 3, 64, 0), (50, 16, 64, 0, 3, 64, 2),
    # two-tile units (128 outputs over at least 20 K blocks, at least 912 tiles; the last unit ragged)
    (7403, 16, 256, 256, 3, 128, 1), (14799, 8, 256, 0, 5, 128, 2), (3701, 32, 128, 128, 5, 128, 2),
    (14799, 8, 128, 128, 5, 256, 2),
    # 64 outputs with resident weights (<= 8 K blocks) over many tiles per CTA; and with streamed weights
    (4001, 32, 64, 0, 5, 64, 2), (1001, 32, 64, 64, 5, 64, 2)])
def test_conv_taps_and_concat(gpu_lib, N, L, C0, C1, k, cout, pad):
    rng = np.random.default_rng(N * L + C0 + k)
    x0 = _bf(rng.normal(size=(N, L, C0)))
    x1 = _bf(rng.normal(size=(N, L, C1))) if C1 else None
    cin = C0 + C1
    w = _bf(rng.normal(size=(cout, k, cin)) / np.sqrt(k * cin))
    bias = torch.as_tensor(rng.normal(size=cout).astype(np.float32)).cuda()
    out = torch.full((N * L, cout), np.nan, dtype=torch.float32, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    B.conv_tc(x0, w, out, a1=x1, n_samples=N, L=L, taps=k, pad=pad, cout=cout, bias=bias, epilogue=B.EPI_F32,
              err=err)
    x = _f64(x0) if x1 is None else np.concatenate([_f64(x0), _f64(x1)], 2)
    ref = _conv_ref(x, _f64(w), pad).reshape(N * L, cout) + bias.cpu().double().numpy()
    assert int(err.item()) == 0
    assert np.abs(out.cpu().double().numpy() - ref).max() <= 1e-4 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("N,L,C,cout,film,res", [(13, 32, 64, 64, True, False), (10, 16, 128, 128, False, True),
                                                 (21, 8, 256, 256, True, True), (6, 32, 64, 64, False, False),
                                                 # 256 outputs at 925 tiles; 128 outputs in two-tile units
                                                 (14799, 8, 256, 256, True, True), (14799, 8, 256, 128, True, True)])
def test_group_norm_epilogue(gpu_lib, N, L, C, cout, film, res):
    rng = np.random.default_rng(7 * N + L)
    k, pad, G = 5, 2, 8
    x = _bf(rng.normal(size=(N, L, C)))
    w = _bf(rng.normal(size=(cout, k, C)) / np.sqrt(k * C))
    bias = torch.as_tensor(rng.normal(size=cout).astype(np.float32)).cuda()
    gamma = torch.as_tensor(rng.uniform(0.5, 1.5, cout).astype(np.float32)).cuda()
    beta = torch.as_tensor(rng.normal(size=cout).astype(np.float32) * 0.2).cuda()
    P = 3
    sp = torch.as_tensor(rng.integers(0, P, N).astype(np.int32)).cuda()
    F = torch.as_tensor(rng.normal(size=(P, 2 * cout)).astype(np.float32)).cuda() if film else None
    R = _bf(rng.normal(size=(N * L, cout))) if res else None
    out = torch.zeros((N * L, cout), dtype=torch.bfloat16, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    B.conv_tc(x, w, out, n_samples=N, L=L, taps=k, pad=pad, cout=cout, bias=bias, epilogue=B.EPI_GN,
              rows_per_sample=L, gn_eps=1e-5, gamma=gamma, beta=beta, film=F, sample_problem=sp if film else None,
              res=R, err=err)
    y = _conv_ref(_f64(x), _f64(w), pad) + bias.cpu().double().numpy()          # [N][L][cout]
    yg = y.reshape(N, L, G, cout // G)
    mu = yg.mean(axis=(1, 3), keepdims=True)
    var = yg.var(axis=(1, 3), keepdims=True)
    y = ((yg - mu) / np.sqrt(var + 1e-5)).reshape(N, L, cout) * gamma.cpu().double().numpy() \
        + beta.cpu().double().numpy()
    y = _mish(y)
    if film:
        f = F.cpu().double().numpy()[sp.cpu().numpy()]
        y = y * f[:, None, :cout] + f[:, None, cout:]
    if res:
        y = y + _f64(R).reshape(N, L, cout)
    got = _f64(out).reshape(N, L, cout)
    assert int(err.item()) == 0
    assert np.all(np.abs(got - y) <= 8e-3 * np.abs(y) + 2e-3 * max(1.0, np.abs(y).max())), np.abs(got - y).max()


def test_group_norm_over_plain_rows(gpu_lib):
    """The first layer's form: a plain GEMM over im2col rows whose group norm
    spans 32 consecutive rows (one trajectory)."""
    rng = np.random.default_rng(3)
    N, T, K, cout = 11, 32, 64, 64
    a = _bf(rng.normal(size=(N * T, K)))
    w = _bf(rng.normal(size=(cout, K)) / 8.0)
    bias = torch.zeros(cout, device="cuda")
    gamma = torch.ones(cout, device="cuda")
    beta = torch.zeros(cout, device="cuda")
    out = torch.zeros((N * T, cout), dtype=torch.bfloat16, device="cuda")
    B.conv_tc(a, w, out, n_samples=N * T, L=1, cout=cout, bias=bias, epilogue=B.EPI_GN, rows_per_sample=T,
              gamma=gamma, beta=beta)
    y = (_f64(a) @ _f64(w).T).reshape(N, T, 8, 8)
    y = (y - y.mean(axis=(1, 3), keepdims=True)) / np.sqrt(y.var(axis=(1, 3), keepdims=True) + 1e-5)
    y = _mish(y.reshape(N * T, cout))
    assert np.all(np.abs(_f64(out) - y) <= 8e-3 * np.abs(y) + 4e-3)


def test_rejects_bad_descriptors(gpu_lib):
    a = torch.zeros((64, 48), dtype=torch.bfloat16, device="cuda")         # channels not a multiple of 64
    w = torch.zeros((64, 48), dtype=torch.bfloat16, device="cuda")
    out = torch.zeros((64, 64), dtype=torch.float32, device="cuda")
    with pytest.raises(B.DseedError):
        B.conv_tc(a, w, out, n_samples=64, L=1, cout=64, epilogue=B.EPI_F32)
    a = torch.zeros((64, 64), dtype=torch.bfloat16, device="cuda")
    w = torch.zeros((32, 64), dtype=torch.bfloat16, device="cuda")           # cout_pad 32 unsupported
    with pytest.raises(B.DseedError):
        B.conv_tc(a, w, out, n_samples=64, L=1, cout=32, epilogue=B.EPI_F32)


def test_persistent_tiles(gpu_lib):
    """More tiles than SMs several times over: every CTA walks many tiles,
    alternating its two accumulator buffers and wrapping the stage ring."""
    rng = np.random.default_rng(11)
    M, K, cout = 128 * 997 + 45, 128, 64
    a = _bf(rng.normal(size=(M, K)))
    w = _bf(rng.normal(size=(cout, K)) / np.sqrt(K))
    bias = torch.as_tensor(rng.normal(size=cout).astype(np.float32)).cuda()
    out = torch.full((M, cout), np.nan, dtype=torch.float32, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    B.conv_tc(a, w, out, n_samples=M, L=1, cout=cout, bias=bias, epilogue=B.EPI_F32, err=err)
    ref = _f64(a) @ _f64(w).T + bias.cpu().double().numpy()
    assert int(err.item()) == 0
    assert np.abs(out.cpu().double().numpy() - ref).max() <= 1e-4 * max(1.0, np.abs(ref).max())
    # group-norm epilogue over many tiles (2500 trajectories of 32 rows = 625 tiles)
    N, L, C = 2500, 32, 64
    x = _bf(rng.normal(size=(N, L, C)))
    w5 = _bf(rng.normal(size=(C, 5, C)) / np.sqrt(5 * C))
    ones, zeros = torch.ones(C, device="cuda"), torch.zeros(C, device="cuda")
    y = torch.zeros((N * L, C), dtype=torch.bfloat16, device="cuda")
    B.conv_tc(x, w5, y, n_samples=N, L=L, taps=5, pad=2, cout=C, bias=zeros, epilogue=B.EPI_GN, rows_per_sample=L,
              gamma=ones, beta=zeros, err=err)
    r = _conv_ref(_f64(x), _f64(w5), 2).reshape(N, L, 8, 8)
    r = (r - r.mean(axis=(1, 3), keepdims=True)) / np.sqrt(r.var(axis=(1, 3), keepdims=True) + 1e-5)
    r = _mish(r.reshape(N * L, C))
    assert int(err.item()) == 0
    assert np.all(np.abs(_f64(y) - r) <= 8e-3 * np.abs(r) + 4e-3)
