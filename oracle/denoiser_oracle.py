"""FP64 CPU oracle of the seed-proposal denoiser (test infrastructure only).

Plain PyTorch CPU operations in float64 -- conv1d, conv3d, group_norm, mish,
linear -- written from the architecture description (the paper's Sec. 4.2:
a 1-D temporal-convolution U-Net of conditional residual blocks, FiLM-conditioned
on a time-step MLP, a problem encoding of start and goal, and an observation
encoding; here a 3-D convolutional encoder of a 32^3 occupancy grid).
Gradients come from autograd.  It reads only the shared parameter layout
(netspec) and shares no code with the CUDA layers: the occupancy encoder uses
real strided 3-D convolutions where the CUDA path gathers patches, the 1-D
convolutions run channels-first where the CUDA path uses im2col + GEMM.

Pins (tests/test_oracle_denoiser.py): finite-difference gradcheck of the whole
network on a small configuration, group-norm moments, Mish closed forms, the
sinusoidal embedding's closed form, DDPM noising and the DDIM step identities.
"""
from __future__ import annotations

import math

import numpy as np
import torch
import torch.nn.functional as F

from paper_2410_16727_gb300 import netspec as NS

DT = torch.float64


def unpack(spec: NS.NetSpec, flat) -> dict:
    flat = torch.as_tensor(np.asarray(flat), dtype=DT) if not isinstance(flat, torch.Tensor) else flat
    out = {}
    for name, (off, shape) in NS.param_offsets(spec).items():
        n = int(np.prod(shape))
        out[name] = flat[off:off + n].view(shape)
    return out


def sinusoid(k: torch.Tensor, dim: int) -> torch.Tensor:
    """[N] integer steps -> [N][dim], pairs (sin, cos)(k / 10000^(i / (dim/2)))."""
    h = dim // 2
    i = torch.arange(h, dtype=DT)
    w = torch.exp(-math.log(10000.0) * i / h)
    a = k.to(DT)[:, None] * w[None, :]
    out = torch.empty(k.shape[0], dim, dtype=DT)
    out[:, 0::2] = torch.sin(a)
    out[:, 1::2] = torch.cos(a)
    return out


def _lin(x, P, name):
    return F.linear(x, P[name + ".w"], P[name + ".b"])


def _conv(x_ncl, P, name, stride=1):
    w = P[name + ".w"]                      # [out][k][in] -> [out][in][k]
    k = w.shape[1]
    return F.conv1d(x_ncl, w.permute(0, 2, 1), P[name + ".b"], stride=stride, padding=k // 2 if stride == 1 else 1)


def _gn(x_ncl, P, name, spec):
    return F.group_norm(x_ncl, spec.groups, P[name + ".w"], P[name + ".b"], eps=spec.gn_eps)


def _res_block(x, P, name, cin, cout, mc, spec):
    h = F.mish(_gn(_conv(x, P, name + ".c1"), P, name + ".g1", spec))
    film = _lin(mc, P, name + ".f")                        # [N][2 cout]
    h = h * film[:, :cout, None] + film[:, cout:, None]
    h = F.mish(_gn(_conv(h, P, name + ".c2"), P, name + ".g2", spec))
    r = _conv(x, P, name + ".r") if cin != cout else x
    return h + r


def condition(spec, P, k, qs, qg, goal, occ):
    t = _lin(F.mish(_lin(sinusoid(k, spec.t_sin), P, "t.l1")), P, "t.l2")
    p = _lin(F.mish(_lin(torch.cat([qs, qg, goal], 1), P, "p.l1")), P, "p.l2")
    N = qs.shape[0]
    n, p1, p2 = spec.occ_n, spec.occ_p1, spec.occ_p2
    vol = occ.view(N, 1, n, n, n)                          # (z, y, x)
    w1 = P["o.c1.w"].view(spec.occ_c1, p1, p1, p1, 1).permute(0, 4, 1, 2, 3)
    o = F.mish(F.conv3d(vol, w1, P["o.c1.b"], stride=p1))
    w2 = P["o.c2.w"].view(spec.occ_c2, p2, p2, p2, spec.occ_c1).permute(0, 4, 1, 2, 3)
    o = F.mish(F.conv3d(o, w2, P["o.c2.b"], stride=p2))     # [N][c2][g2][g2][g2]
    o = o.permute(0, 2, 3, 4, 1).reshape(N, -1)            # (patch, channel) order
    o = _lin(o, P, "o.l")
    return F.mish(torch.cat([t, p, o], 1))


def forward(spec: NS.NetSpec, P: dict, xk, k, qs, qg, goal, occ):
    """xk [N][T][D] (channels-last like the CUDA path) -> predicted noise [N][T][D]."""
    mc = condition(spec, P, k, qs, qg, goal, occ)
    c1, c2, c3 = spec.chans
    x = xk.permute(0, 2, 1)                                # [N][D][T]
    h = _res_block(x, P, "d1a", spec.D, c1, mc, spec)
    h = _res_block(h, P, "d1b", c1, c1, mc, spec)
    h = _conv(h, P, "down1", stride=2)
    h = _res_block(h, P, "d2a", c1, c2, mc, spec)
    s2 = _res_block(h, P, "d2b", c2, c2, mc, spec)
    h = _conv(s2, P, "down2", stride=2)
    h = _res_block(h, P, "d3a", c2, c3, mc, spec)
    s3 = _res_block(h, P, "d3b", c3, c3, mc, spec)
    h = _res_block(s3, P, "mid", c3, c3, mc, spec)
    h = torch.cat([h, s3], 1)
    h = _res_block(h, P, "u2a", 2 * c3, c2, mc, spec)
    h = _res_block(h, P, "u2b", c2, c2, mc, spec)
    h = _conv(torch.repeat_interleave(h, 2, dim=2), P, "up2")
    h = torch.cat([h, s2], 1)
    h = _res_block(h, P, "u1a", 2 * c2, c1, mc, spec)
    h = _res_block(h, P, "u1b", c1, c1, mc, spec)
    h = _conv(torch.repeat_interleave(h, 2, dim=2), P, "up1")
    h = F.mish(_gn(_conv(h, P, "fin.c"), P, "fin.g", spec))
    out = _conv(h, P, "fin.o")
    return out.permute(0, 2, 1)


def ddpm_noise(x0, eps, k, abar):
    ab = torch.as_tensor(abar, dtype=DT)[k.long()].view(-1, *([1] * (x0.dim() - 1)))
    return torch.sqrt(ab) * x0 + torch.sqrt(1 - ab) * eps


def loss_and_grads(spec, flat_params, x0, qs, qg, goal, occ, k, eps, abar, weights=None):
    """Eq. 1 (weighted per sample as in Eq. 2): mean over all entries of
    w_n (Theta(x_k, k, cond) - eps)^2.  Returns (loss, dL/dparams flat)."""
    flat = torch.as_tensor(np.asarray(flat_params), dtype=DT).clone().requires_grad_(True)
    P = unpack(spec, flat)
    t = lambda a: torch.as_tensor(np.asarray(a), dtype=DT)
    x0, qs, qg, goal, occ, eps = t(x0), t(qs), t(qg), t(goal), t(occ), t(eps)
    k = torch.as_tensor(np.asarray(k), dtype=torch.long)
    xk = ddpm_noise(x0, eps, k, abar)
    pred = forward(spec, P, xk, k, qs, qg, goal, occ)
    w = torch.ones(x0.shape[0], dtype=DT) if weights is None else t(weights)
    loss = (w.view(-1, 1, 1) * (pred - eps) ** 2).sum() / pred.numel()
    loss.backward()
    return float(loss.detach()), flat.grad.detach().numpy()


def predict(spec, flat_params, xk, k, qs, qg, goal, occ):
    P = unpack(spec, torch.as_tensor(np.asarray(flat_params), dtype=DT))
    t = lambda a: torch.as_tensor(np.asarray(a), dtype=DT)
    with torch.no_grad():
        return forward(spec, P, t(xk), torch.as_tensor(np.asarray(k), dtype=torch.long), t(qs), t(qg), t(goal),
                       t(occ)).numpy()


def ddim_step(xk, eps, ab_k, ab_prev, clip):
    """Deterministic DDIM update from step k to an earlier step (eta = 0)."""
    x0 = np.clip((xk - np.sqrt(1 - ab_k) * eps) / np.sqrt(ab_k), -clip, clip)
    return np.sqrt(ab_prev) * x0 + np.sqrt(1 - ab_prev) * eps
