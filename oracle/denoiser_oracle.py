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

Cost-guided sampling (guided_ddim, the appendix's Eq. 5 read for a
deterministic DDIM sampler; pins in tests/test_oracle_guided.py: the closed form
of eps-free DDIM, the descent direction against central differences of the cost
in the diffused space, the per-entry cap, and the guided-step count of the
schedule).

Also Eq. 2's loss measured on the robot (fk_mse, Sec. 4.3: the error taken on
points spread over the surface of every link): the drawn and the predicted noise are
decoded to the joint configurations they stand for, and the points on the
collision spheres' surfaces at the six axis directions of each sphere's frame
are placed by a forward-kinematics chain of 4x4 modified-DH products written
here (pins in tests/test_oracle_fk_loss.py: zero at pred = eps, a base-joint
rotation's closed form, per-sample weights, the points against the C oracle's
chain, central differences).
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


# ------------------------------------------------------------------ Eq. 2 on the robot

# The six axis directions of a sphere's frame, in this order for every sphere.
SURFACE_DIRS = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]], np.float64)


def surface_offsets(robot):
    """Frame offsets [6 N_s][3] and frames [6 N_s] of the points of Eq. 2: for
    sphere k (offset o_k, radius r_k in frame sph_frame[k]) the points
    o_k + r_k u for the six axis directions u, sphere-major."""
    o = np.asarray(robot.sph_o, np.float64)
    r = np.asarray(robot.sph_r, np.float64)
    pts = (o[:, None, :] + r[:, None, None] * SURFACE_DIRS[None]).reshape(-1, 3)
    return pts, np.repeat(np.asarray(robot.sph_frame, np.int64), len(SURFACE_DIRS))


def robot_points(robot, q: torch.Tensor, offsets=None, frames=None) -> torch.Tensor:
    """Points [..., N_p, 3] of joint configurations q [..., 7]: frame i = frame
    i-1 RotX(alpha_i) TransX(a_i) RotZ(q_i + offset_i) TransZ(d_i) (modified DH,
    rows (a, d, alpha, offset) of robot.dh; the eighth row, the flange, has no
    joint), point k at offsets[k] in frame frames[k] (default: the collision
    spheres' centres)."""
    dh = torch.as_tensor(np.asarray(robot.dh, np.float64))
    lead = q.shape[:-1]
    one = torch.ones(lead, dtype=DT)
    zero = torch.zeros(lead, dtype=DT)

    def mat(rows):
        return torch.stack([torch.stack(r, -1) for r in rows], -2)

    chain = [torch.eye(4, dtype=DT).expand(*lead, 4, 4)]
    for i in range(8):
        a, d, al, off = (float(v) for v in dh[i])
        th = (q[..., i] if i < 7 else zero) + off
        ca, sa = math.cos(al), math.sin(al)
        rx = mat([[one, zero, zero, zero], [zero, ca * one, -sa * one, zero], [zero, sa * one, ca * one, zero],
                  [zero, zero, zero, one]])
        tx = mat([[one, zero, zero, a * one], [zero, one, zero, zero], [zero, zero, one, zero], [zero, zero, zero, one]])
        rz = mat([[torch.cos(th), -torch.sin(th), zero, zero], [torch.sin(th), torch.cos(th), zero, zero],
                  [zero, zero, one, zero], [zero, zero, zero, one]])
        tz = mat([[one, zero, zero, zero], [zero, one, zero, zero], [zero, zero, one, d * one], [zero, zero, zero, one]])
        chain.append(chain[-1] @ rx @ tx @ rz @ tz)
    F = torch.stack(chain, -3)                                            # [..., 9, 4, 4]
    o = torch.as_tensor(np.asarray(robot.sph_o if offsets is None else offsets, np.float64))
    oh = torch.cat([o, torch.ones(o.shape[0], 1, dtype=DT)], 1)           # [N_p, 4]
    fr = torch.as_tensor(np.asarray(robot.sph_frame if frames is None else frames, np.int64))
    Fk = F[..., fr, :, :]                                                 # [..., N_p, 4, 4]
    return (Fk @ oh[..., None])[..., :3, 0]


def decode(robot, lin, v, res_scale: float) -> torch.Tensor:
    """Joint configuration a diffused-space vector v stands for: the residual
    v / res_scale added to the normalised straight path lin, un-normalised by
    the limits (mid + half * n)."""
    lim = torch.as_tensor(np.asarray(robot.limits, np.float64))
    mid, half = (lim[:, 0] + lim[:, 1]) / 2, (lim[:, 1] - lim[:, 0]) / 2
    return mid + half * (lin + v / res_scale)


def fk_mse(robot, lin, eps, pred, res_scale: float, weights=None):
    """Eq. 2 measured on the robot: with c_k(q) the points of surface_offsets,
    loss = sum_n w_n sum_{t,k} |c_k(q(pred_nt)) - c_k(q(eps_nt))|^2 / (N T N_p 3).
    lin, eps, pred [N][T][7]; returns (loss, dloss/dpred [N][T][7])."""
    t = lambda a: torch.as_tensor(np.asarray(a), dtype=DT)
    lin, eps = t(lin), t(eps)
    pr = t(pred).clone().requires_grad_(True)
    N = lin.shape[0]
    w = torch.ones(N, dtype=DT) if weights is None else t(weights)
    offs, frs = surface_offsets(robot)
    cl = robot_points(robot, decode(robot, lin, eps, res_scale), offs, frs)
    cp = robot_points(robot, decode(robot, lin, pr, res_scale), offs, frs)
    loss = (w.view(-1, 1, 1, 1) * (cp - cl) ** 2).sum() / cp.numel()
    loss.backward()
    return float(loss.detach()), pr.grad.detach().numpy()


# ------------------------------------------------------------------ cost-guided sampling (Eq. 5)

def normalise_joints(limits, q):
    """Joints to [-1, 1] by the mechanical limits (App. A.4): 2 (q - lo) / (hi - lo) - 1."""
    lim = np.asarray(limits, np.float64)
    lo, hi = lim[:, 0], lim[:, 1]
    return 2.0 * (np.asarray(q, np.float64) - lo) / (hi - lo) - 1.0


def straight_path(qs_n, qg_n, T: int):
    """The straight start-goal path in normalised joints at waypoints t = 1..T
    (fraction t / T): [N][T][7]."""
    tau = (np.arange(1, T + 1, dtype=np.float64) / T)[None, :, None]
    return (1.0 - tau) * np.asarray(qs_n, np.float64)[:, None, :] + tau * np.asarray(qg_n, np.float64)[:, None, :]


def decode_joints(limits, lin, r, res_scale: float):
    """Joint trajectories a diffused residual r stands for: the normalised
    straight path plus r / res_scale, clipped to [-1, 1] (inside the limits),
    un-normalised as mid + half * n."""
    lim = np.asarray(limits, np.float64)
    mid, half = (lim[:, 0] + lim[:, 1]) / 2.0, (lim[:, 1] - lim[:, 0]) / 2.0
    return mid + half * np.clip(lin + r / res_scale, -1.0, 1.0)


def ddim_schedule(K: int, steps: int):
    """Evenly spaced step indices of the K-step schedule, from K - 1 down to 0."""
    return np.linspace(K - 1, 0, steps).round().astype(int)


def guided_ddim(spec, flat_params, noise, q_start, q_goal, goal, occ, limits, res_scale, abar, steps, clip,
                k_guide, n_grad, alpha, cap, cost_grad, eps_fn=None):
    """DDIM sampling with the cost guidance of the paper's appendix (Eq. 5),
    as read for a deterministic sampler: after each denoising step that reaches
    a step index below k_guide, except the last step, the samples take n_grad
    descent steps on the plan cost C of their problem,
        x <- x + clip(-alpha dC/dx, -cap, cap),   dC/dx = dC/dq * half / res_scale,
    where q = decode_joints(x) and half = (hi - lo) / 2 per joint (the limit clip
    of the decoding passes the gradient through).  All per sample: noise, the
    starts, goal configurations, goal poses and occupancy rows [N][...].
    cost_grad(q [N][T][7]) -> dC/dq [N][T][7]; eps_fn(x, k) replaces the
    network's noise prediction when given.  Returns (joint-space proposals
    [N][T][7], final residuals [N][T][7])."""
    noise = np.asarray(noise, np.float64)
    N, T = noise.shape[0], noise.shape[1]
    lim = np.asarray(limits, np.float64)
    qs_n, qg_n = normalise_joints(lim, q_start), normalise_joints(lim, q_goal)
    lin = straight_path(qs_n, qg_n, T)
    ks = ddim_schedule(spec.K, steps)
    x = noise.copy()
    for i, k in enumerate(ks):
        if eps_fn is not None:
            eps = eps_fn(x, int(k))
        else:
            eps = predict(spec, flat_params, x, np.full(N, int(k)), qs_n, qg_n, goal, occ)
        last = i + 1 == len(ks)
        x = ddim_step(x, eps, float(abar[k]), 1.0 if last else float(abar[ks[i + 1]]), clip)
        if not last and int(ks[i + 1]) < k_guide and alpha != 0.0:
            x = guided_descent(x, lin, lim, res_scale, n_grad, alpha, cap, cost_grad)
    return decode_joints(lim, lin, x, res_scale), x


def guided_descent(x, lin, limits, res_scale, n_grad, alpha, cap, cost_grad):
    """n_grad capped descent steps on C(decode_joints(x)) in the diffused space:
    x <- x + clip(-alpha (dC/dq) (half / res_scale), -cap, cap)."""
    lim = np.asarray(limits, np.float64)
    half = (lim[:, 1] - lim[:, 0]) / 2.0
    x = np.asarray(x, np.float64)
    for _ in range(n_grad):
        g = cost_grad(decode_joints(lim, lin, x, res_scale))
        x = x + np.clip(-alpha * g * half / res_scale, -cap, cap)
    return x


def cosine_abar(K: int, s: float = 0.008) -> np.ndarray:
    """The squared-cosine noise schedule: with f(t) = cos^2(pi/2 (t/K + s)/(1 + s)),
    beta_k = 1 - f(k + 1) / f(k) capped at 0.999, and abar_k = prod_{j <= k} (1 - beta_j),
    k = 0..K-1."""
    f = [math.cos(math.pi / 2 * (t / K + s) / (1 + s)) ** 2 for t in range(K + 1)]
    out = np.empty(K)
    acc = 1.0
    for k in range(K):
        acc *= 1.0 - min(1.0 - f[k + 1] / f[k], 0.999)
        out[k] = acc
    return out
