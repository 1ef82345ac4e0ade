"""Conditional denoiser that proposes seed trajectories (the learned part of the
method, paper Sec. 4.2-4.3), built from libdseed's layer kernels.

Orchestration only: each layer call below is one C-ABI kernel launch
(binding.nn); this module decides their order, keeps the activations the
backward pass needs (a tape of closures, replayed in reverse), and owns the
parameter, gradient and Adam buffers (device tensors).  Training runs in FP32.
Sampling runs the U-Net through `unet_tc`: BF16 activations, every
convolution one tcgen05 tensor-core kernel with its group norm, Mish, FiLM and
residual fused in (dseed_nn_conv_tc).  `infer` (BF16 operands on the legacy
mma.sync path, FP32 activations) is kept as the second BF16 reference.

Inputs of one sample: the noisy trajectory x_k [T][D], the diffusion step k,
the normalised start and goal configurations [D], the goal pose [7] and the
scene's 32^3 occupancy grid.  Output: the predicted noise [T][D] (Eq. 1).
Joint values are normalised to [-1, 1] by the mechanical limits (App. A.4);
the diffused quantity is the deviation of the normalised trajectory from the
straight start-goal joint path (see learned.py).
"""
from __future__ import annotations

import math
from typing import Callable, Dict, List, Optional

import numpy as np
import torch

from . import binding as B
from . import netspec as NS


def _nn(name, *a):
    B.nn(name, *a)


class Tape:
    def __init__(self):
        self.ops: List[Callable] = []
        self.grads: Dict[int, torch.Tensor] = {}
        self.keep: List[torch.Tensor] = []

    def record(self, fn):
        self.ops.append(fn)

    def grad(self, t: torch.Tensor) -> Optional[torch.Tensor]:
        return self.grads.get(id(t))

    def add_grad(self, t: torch.Tensor, g: torch.Tensor):
        cur = self.grads.get(id(t))
        if cur is None:
            self.grads[id(t)] = g
            self.keep.append(t)
        else:
            _nn("axpby", 1.0, cur, 1.0, g, cur, cur.numel())


def cosine_abar(K: int, s: float = 0.008) -> np.ndarray:
    """Cumulative noise schedule abar_k, k = 0..K-1 (squared-cosine schedule)."""
    f = lambda t: math.cos((t / K + s) / (1 + s) * math.pi / 2) ** 2
    betas = np.array([min(1 - f(k + 1) / f(k), 0.999) for k in range(K)])
    return np.cumprod(1.0 - betas)


class Denoiser:
    def __init__(self, spec: NS.NetSpec = NS.NetSpec(), device="cuda", seed: int = 0):
        self.spec = spec
        self.dev = torch.device(device)
        self.offsets = NS.param_offsets(spec)
        self.n_params = NS.param_count(spec)
        self.params = torch.zeros(self.n_params, dtype=torch.float32, device=self.dev)
        self.grads = torch.zeros_like(self.params)
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.step_count = 0
        m1, m2 = NS.occ_patch_maps(spec)
        self.map1 = torch.tensor(m1, dtype=torch.int32, device=self.dev)
        self.map2 = torch.tensor(m2, dtype=torch.int32, device=self.dev)
        self.abar = torch.tensor(cosine_abar(spec.K), dtype=torch.float32, device=self.dev)
        self.abar_host = cosine_abar(spec.K)
        self._bf16: Dict[str, torch.Tensor] = {}
        self._tc_err = torch.zeros(1, dtype=torch.int32, device=self.dev)
        self._ks_cache: Dict[int, torch.Tensor] = {}
        self.init_params(seed)

    # ------------------------------------------------------------------ parameters
    def P(self, name: str) -> torch.Tensor:
        off, shape = self.offsets[name]
        n = int(np.prod(shape))
        return self.params[off:off + n]

    def G(self, name: str) -> torch.Tensor:
        off, shape = self.offsets[name]
        n = int(np.prod(shape))
        return self.grads[off:off + n]

    def init_params(self, seed: int):
        """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights and biases; group-norm
        gains 1, offsets 0; the output convolution starts at zero."""
        rng = np.random.default_rng(seed)
        host = np.zeros(self.n_params, np.float32)
        for name, (off, shape) in self.offsets.items():
            n = int(np.prod(shape))
            if ".g" in name and name.endswith(".w") and len(shape) == 1:
                host[off:off + n] = 1.0
                continue
            if ".g" in name and name.endswith(".b") and len(shape) == 1:
                continue
            wname = name[:-2] + ".w"
            wshape = self.offsets[wname][1]
            fan_in = int(np.prod(wshape[1:]))
            bound = 1.0 / math.sqrt(fan_in)
            host[off:off + n] = rng.uniform(-bound, bound, size=n)
        for name in ("fin.o.w", "fin.o.b"):
            off, shape = self.offsets[name]
            host[off:off + int(np.prod(shape))] = 0.0
        self.params.copy_(torch.from_numpy(host))
        self.m.zero_()
        self.v.zero_()
        self.step_count = 0
        self._bf16.clear()

    # ------------------------------------------------------------------ layers (FP32, with tape)
    def linear(self, x, name, tape, R=None):
        """x [R][in] -> [R][out] with weight name.w [out][in], bias name.b."""
        W, b = self.P(name + ".w"), self.P(name + ".b")
        out_f, in_f = self.offsets[name + ".w"][1][0], int(np.prod(self.offsets[name + ".w"][1][1:]))
        R = x.numel() // in_f if R is None else R
        y = torch.empty((R, out_f), dtype=torch.float32, device=self.dev)
        if self.bf16_mode:
            xb = torch.empty((R, _pad16(in_f)), dtype=torch.bfloat16, device=self.dev)
            _nn("im2col1d", x, R, 1, in_f, 1, 1, 0, 1, _pad16(in_f), xb, 1)
            _nn("gemm_bf16", R, out_f, _pad16(in_f), xb, self.w_bf16(name + ".w", out_f, in_f), y, b)
            return y
        _nn("gemm_f32", 0, 1, R, out_f, in_f, 1.0, x, in_f, W, in_f, 0.0, y, out_f, b)
        if tape is not None:
            def bwd():
                dy = tape.grad(y)
                if dy is None:
                    return
                _nn("gemm_f32", 1, 0, out_f, in_f, R, 1.0, dy, out_f, x, in_f, 1.0, self.G(name + ".w"), in_f, None)
                _nn("colsum", dy, R, out_f, self.G(name + ".b"), 1)
                dx = torch.empty_like(x)
                _nn("gemm_f32", 0, 0, R, in_f, out_f, 1.0, dy, out_f, W, in_f, 0.0, dx, in_f, None)
                tape.add_grad(x, dx)
            tape.record(bwd)
        return y

    def conv(self, x, N, L, name, k, s, p, tape):
        """x [N][L][Cin] -> [N][Lo][Cout], weight [Cout][k][Cin]."""
        W, b = self.P(name + ".w"), self.P(name + ".b")
        cout, kk, cin = self.offsets[name + ".w"][1]
        assert kk == k
        Lo = (L + 2 * p - k) // s + 1
        kc = k * cin
        y = torch.empty((N, Lo, cout), dtype=torch.float32, device=self.dev)
        if self.bf16_mode:
            cols = torch.empty((N * Lo, _pad16(kc)), dtype=torch.bfloat16, device=self.dev)
            _nn("im2col1d", x, N, L, cin, k, s, p, Lo, _pad16(kc), cols, 1)
            _nn("gemm_bf16", N * Lo, cout, _pad16(kc), cols, self.w_bf16(name + ".w", cout, kc), y, b)
            return y, Lo
        cols = torch.empty((N * Lo, kc), dtype=torch.float32, device=self.dev)
        _nn("im2col1d", x, N, L, cin, k, s, p, Lo, kc, cols, 0)
        _nn("gemm_f32", 0, 1, N * Lo, cout, kc, 1.0, cols, kc, W, kc, 0.0, y, cout, b)
        if tape is not None:
            def bwd():
                dy = tape.grad(y)
                if dy is None:
                    return
                _nn("gemm_f32", 1, 0, cout, kc, N * Lo, 1.0, dy, cout, cols, kc, 1.0, self.G(name + ".w"), kc, None)
                _nn("colsum", dy, N * Lo, cout, self.G(name + ".b"), 1)
                dcols = torch.empty_like(cols)
                _nn("gemm_f32", 0, 0, N * Lo, kc, cout, 1.0, dy, cout, W, kc, 0.0, dcols, kc, None)
                dx = torch.zeros_like(x)
                _nn("col2im1d", dcols, N, L, cin, k, s, p, Lo, kc, dx)
                tape.add_grad(x, dx)
            tape.record(bwd)
        return y, Lo

    def groupnorm(self, x, N, L, C, name, tape):
        gamma, beta = self.P(name + ".w"), self.P(name + ".b")
        G = self.spec.groups
        y = torch.empty_like(x)
        mean = torch.empty((N, G), dtype=torch.float32, device=self.dev)
        rstd = torch.empty_like(mean)
        _nn("groupnorm_fwd", x, N, L, C, G, gamma, beta, self.spec.gn_eps, y, mean, rstd)
        if tape is not None:
            def bwd():
                dy = tape.grad(y)
                if dy is None:
                    return
                dx = torch.empty_like(x)
                dg = torch.empty((N, C), dtype=torch.float32, device=self.dev)
                db = torch.empty_like(dg)
                _nn("groupnorm_bwd", dy, x, N, L, C, G, gamma, mean, rstd, dx, dg, db)
                _nn("colsum", dg, N, C, self.G(name + ".w"), 1)
                _nn("colsum", db, N, C, self.G(name + ".b"), 1)
                tape.add_grad(x, dx)
            tape.record(bwd)
        return y

    def mish(self, x, tape):
        y = torch.empty_like(x)
        _nn("mish", x, None, y, x.numel(), 0)
        if tape is not None:
            def bwd():
                dy = tape.grad(y)
                if dy is None:
                    return
                dx = torch.empty_like(x)
                _nn("mish", x, dy, dx, x.numel(), 1)
                tape.add_grad(x, dx)
            tape.record(bwd)
        return y

    def film(self, h, f, N, L, C, tape):
        y = torch.empty_like(h)
        _nn("film", h, f, N, L, C, y, None, None, None, 0)
        if tape is not None:
            def bwd():
                dy = tape.grad(y)
                if dy is None:
                    return
                dh = torch.empty_like(h)
                df = torch.empty_like(f)
                _nn("film", h, f, N, L, C, None, dy, dh, df, 1)
                tape.add_grad(h, dh)
                tape.add_grad(f, df)
            tape.record(bwd)
        return y

    def add(self, a, b, tape):
        y = torch.empty_like(a)
        _nn("axpby", 1.0, a, 1.0, b, y, a.numel())
        if tape is not None:
            def bwd():
                dy = tape.grad(y)
                if dy is None:
                    return
                tape.add_grad(a, dy)
                tape.add_grad(b, dy.clone())
            tape.record(bwd)
        return y

    def concat(self, tensors, R, tape, shape=None):
        widths = [t.numel() // R for t in tensors]
        Ct = sum(widths)
        y = torch.empty(shape if shape is not None else (R, Ct), dtype=torch.float32, device=self.dev)
        off = 0
        for t, w in zip(tensors, widths):
            _nn("copy_cols", t, R, w, w, 0, y, Ct, off, 0)
            off += w
        if tape is not None:
            def bwd():
                dy = tape.grad(y)
                if dy is None:
                    return
                o = 0
                for t, w in zip(tensors, widths):
                    g = torch.empty((R, w), dtype=torch.float32, device=self.dev)
                    _nn("copy_cols", dy, R, w, Ct, o, g, w, 0, 0)
                    tape.add_grad(t, g.view(t.shape))
                    o += w
            tape.record(bwd)
        return y

    def upsample(self, x, N, L, C, tape):
        y = torch.empty((N, 2 * L, C), dtype=torch.float32, device=self.dev)
        _nn("upsample2", x, N, L, C, y, 0)
        if tape is not None:
            def bwd():
                dy = tape.grad(y)
                if dy is None:
                    return
                dx = torch.empty_like(x)
                _nn("upsample2", dy, N, L, C, dx, 1)
                tape.add_grad(x, dx)
            tape.record(bwd)
        return y

    def gather(self, x, idx, N, per, tape):
        y = torch.empty((N, per), dtype=torch.float32, device=self.dev)
        _nn("gather", x, idx, y, N, per, 0)
        if tape is not None:
            def bwd():
                dy = tape.grad(y)
                if dy is None:
                    return
                dx = torch.zeros((N, per), dtype=torch.float32, device=self.dev)
                _nn("gather", dy, idx, dx, N, per, 1)
                tape.add_grad(x, dx.view(x.shape))
            tape.record(bwd)
        return y

    # ------------------------------------------------------------------ BF16 weights
    bf16_mode = False

    def w_bf16(self, name, out_f, kc):
        w = self._bf16.get(name)
        if w is None:
            # [out][kc] FP32 -> [out][pad16(kc)] BF16 (zero tail) via im2col with L = 1
            w = torch.empty((out_f, _pad16(kc)), dtype=torch.bfloat16, device=self.dev)
            _nn("im2col1d", self.P(name), out_f, 1, kc, 1, 1, 0, 1, _pad16(kc), w, 1)
            self._bf16[name] = w
        return w

    # ------------------------------------------------------------------ network
    def res_block(self, x, N, L, name, cin, cout, mc, tape):
        k = self.spec.kernel
        a, _ = self.conv(x, N, L, name + ".c1", k, 1, k // 2, tape)
        b = self.groupnorm(a, N, L, cout, name + ".g1", tape)
        c = self.mish(b, tape)
        f = self.linear(mc, name + ".f", tape)
        d = self.film(c, f, N, L, cout, tape)
        e, _ = self.conv(d, N, L, name + ".c2", k, 1, k // 2, tape)
        g = self.groupnorm(e, N, L, cout, name + ".g2", tape)
        h = self.mish(g, tape)
        if cin != cout:
            r, _ = self.conv(x, N, L, name + ".r", 1, 1, 0, tape)
        else:
            r = x
        return self.add(h, r, tape)

    def time_embed(self, k, tape):
        """Time-step MLP of sinusoidal features of k [R] (int32) -> [R][t_dim]."""
        s = self.spec
        R = k.shape[0]
        te = torch.empty((R, s.t_sin), dtype=torch.float32, device=self.dev)
        _nn("sinusoid", k, R, s.t_sin, te)
        t1 = self.mish(self.linear(te, "t.l1", tape), tape)
        return self.linear(t1, "t.l2", tape)

    def problem_embed(self, qs, qg, goal, occ, tape, last_linear=None):
        """Problem MLP (q_start, q_goal, goal pose) and occupancy encoder -> [P][p_dim], [P][o_dim].
        last_linear(x, R) (inference only) replaces the encoder's flattened last linear."""
        s = self.spec
        N = qs.shape[0]
        pin = self.concat([qs, qg, goal], N, tape)
        p1 = self.mish(self.linear(pin, "p.l1", tape), tape)
        p2 = self.linear(p1, "p.l2", tape)
        o0 = self.gather(occ, self.map1, N, s.occ_n ** 3, tape)                      # [N][8^3][4^3]
        o1 = self.mish(self.linear(o0, "o.c1", tape, R=N * s.occ_g1 ** 3), tape)     # [N*8^3][c1]
        o2 = self.gather(o1, self.map2, N, s.occ_g1 ** 3 * s.occ_c1, tape)           # [N][4^3][2^3 c1]
        o3 = self.mish(self.linear(o2, "o.c2", tape, R=N * s.occ_g2 ** 3), tape)     # [N*4^3][c2]
        if last_linear is not None:
            o4 = last_linear(o3, N)
        else:
            o4 = self.linear(o3, "o.l", tape, R=N)                                   # flattened per sample
        return p2, o4

    def condition(self, k, qs, qg, goal, occ, tape):
        """cond = [time MLP (sinusoid(k)), problem MLP (q_start, q_goal, goal pose),
        occupancy encoder]; returns Mish(cond) [N][cond_dim], the input of every
        FiLM layer."""
        N = qs.shape[0]
        t2 = self.time_embed(k, tape)
        p2, o4 = self.problem_embed(qs, qg, goal, occ, tape)
        cond = self.concat([t2, p2, o4], N, tape)
        return self.mish(cond, tape)

    def unet(self, x, N, mc, tape):
        s = self.spec
        c1, c2, c3 = s.chans
        T = s.T
        h = self.res_block(x, N, T, "d1a", s.D, c1, mc, tape)
        h = self.res_block(h, N, T, "d1b", c1, c1, mc, tape)
        h, L2 = self.conv(h, N, T, "down1", 3, 2, 1, tape)
        h = self.res_block(h, N, L2, "d2a", c1, c2, mc, tape)
        s2 = self.res_block(h, N, L2, "d2b", c2, c2, mc, tape)
        h, L3 = self.conv(s2, N, L2, "down2", 3, 2, 1, tape)
        h = self.res_block(h, N, L3, "d3a", c2, c3, mc, tape)
        s3 = self.res_block(h, N, L3, "d3b", c3, c3, mc, tape)
        h = self.res_block(s3, N, L3, "mid", c3, c3, mc, tape)
        h = self.concat([h, s3], N * L3, tape, shape=(N, L3, 2 * c3))
        h = self.res_block(h, N, L3, "u2a", 2 * c3, c2, mc, tape)
        h = self.res_block(h, N, L3, "u2b", c2, c2, mc, tape)
        h = self.upsample(h, N, L3, c2, tape)
        h, _ = self.conv(h, N, L2, "up2", 3, 1, 1, tape)
        h = self.concat([h, s2], N * L2, tape, shape=(N, L2, 2 * c2))
        h = self.res_block(h, N, L2, "u1a", 2 * c2, c1, mc, tape)
        h = self.res_block(h, N, L2, "u1b", c1, c1, mc, tape)
        h = self.upsample(h, N, L2, c1, tape)
        h, _ = self.conv(h, N, T, "up1", 3, 1, 1, tape)
        h, _ = self.conv(h, N, T, "fin.c", s.kernel, 1, s.kernel // 2, tape)
        h = self.mish(self.groupnorm(h, N, T, c1, "fin.g", tape), tape)
        out, _ = self.conv(h, N, T, "fin.o", 1, 1, 0, tape)
        return out

    def forward(self, xk, k, qs, qg, goal, occ, tape: Optional[Tape] = None):
        """Predicted noise [N][T][D] (FP32)."""
        N = xk.shape[0]
        mc = self.condition(k, qs, qg, goal, occ, tape)
        return self.unet(xk, N, mc, tape)

    @staticmethod
    def backward(tape: Tape, out: torch.Tensor, dout: torch.Tensor):
        tape.grads[id(out)] = dout
        for fn in reversed(tape.ops):
            fn()

    # ------------------------------------------------------------------ training
    def loss_and_grad(self, x0, qs, qg, goal, occ, k, eps, weights=None, fk=None):
        """Eq. 1 (optionally weighted per sample as in Eq. 2): noise the clean
        normalised trajectories x0 to step k with eps, predict the noise,
        accumulate parameter gradients of the mean squared error into self.grads.
        With fk = (robot, lin, res_scale) the error is measured on the robot as
        in Eq. 2 (dseed_nn_fk_mse): eps and the prediction are decoded to joint
        configurations around the samples' normalised straight paths lin
        [N][T][7] and compared through the robot's sphere centres.
        Returns the loss (device scalar)."""
        N = x0.shape[0]
        per = x0.numel() // N
        xk = torch.empty_like(x0)
        _nn("ddpm_noise", x0, eps, k, self.abar, N, per, xk)
        tape = Tape()
        pred = self.forward(xk, k, qs, qg, goal, occ, tape)
        dpred = torch.empty_like(pred)
        blocks = 64
        part = torch.empty(blocks, dtype=torch.float32, device=self.dev)
        if fk is None:
            _nn("mse", pred, eps, weights, N, per, dpred, part, blocks)
        else:
            robot, lin, res_scale = fk
            _nn("fk_mse", robot.handle, lin, eps, pred, weights, N, x0.shape[1], float(res_scale), dpred, part,
                blocks)
        self.backward(tape, pred, dpred)
        return part.sum()

    def adam_step(self, lr=3e-4, b1=0.9, b2=0.999, eps=1e-8, wd=0.0):
        self.step_count += 1
        _nn("adam", self.params, self.grads, self.m, self.v, self.n_params, lr, b1, b2, eps, wd, self.step_count)
        self.grads.zero_()
        self._bf16.clear()

    # ------------------------------------------------------------------ inference
    def infer(self, xk, k, qs, qg, goal, occ):
        """Predicted noise with every GEMM on the BF16 tensor cores."""
        self.bf16_mode = True
        try:
            return self.forward(xk, k, qs, qg, goal, occ, None)
        finally:
            self.bf16_mode = False

    def ddim_sample(self, qs, qg, goal, occ, noise, steps: int = 10, bf16: bool = True, clip: float = 2.0,
                    sample_problem: Optional[torch.Tensor] = None, check: bool = True,
                    guide: Optional[Callable] = None):
        """DDIM (deterministic) from x_K = noise over `steps` evenly spaced steps
        of the K-step schedule; returns normalised trajectories [N][T][D].
        qs, qg, goal, occ are per problem; sample_problem [N] (int32) maps each
        sample to its problem (default: sample n -> problem n).  The condition
        and the FiLM rows are computed once per problem and step; with bf16 the
        U-Net runs on the tensor cores (unet_tc), else in FP32.  check=False
        skips reading the kernels' error flag (a host sync), for graph capture.
        guide(i, k_reached, x, last) -> x, when given, is applied after every
        step (cost-gradient guidance)."""
        K = self.spec.K
        ks = np.linspace(K - 1, 0, steps).round().astype(int)
        x = noise.clone()
        N = x.shape[0]
        P = qs.shape[0]
        rows = sample_problem if sample_problem is not None else torch.arange(N, dtype=torch.int32, device=self.dev)
        if bf16:
            Fs = self.film_static(qs, qg, goal, occ)
            kdev = self._ks_cache.get(steps)
            if kdev is None:                 # made once, outside any graph capture (no host copy inside one)
                kdev = self._ks_cache[steps] = torch.tensor(ks, dtype=torch.int32).to(self.dev)
            Ft = self.film_time_rows(kdev)
        for i, kk in enumerate(ks):
            if bf16:
                eps = self.unet_tc(x, N, Fs, rows, film_add=Ft[i])
            else:
                kp = torch.full((P,), int(kk), dtype=torch.int32, device=self.dev)
                mc_p = self.condition(kp, qs, qg, goal, occ, None)
                mc = torch.empty((N, mc_p.shape[1]), dtype=torch.float32, device=self.dev)
                _nn("gather_rows", mc_p, rows, N, mc_p.shape[1], mc)
                eps = self.unet(x, N, mc, None)
            ab_k = float(self.abar_host[kk])
            ab_prev = float(self.abar_host[ks[i + 1]]) if i + 1 < len(ks) else 1.0
            out = torch.empty_like(x)
            _nn("ddim_step", x, eps, ab_k, ab_prev, x.numel(), clip, out)
            x = out
            if guide is not None:
                k_reached = int(ks[i + 1]) if i + 1 < len(ks) else -1
                x = guide(i, k_reached, x, i + 1 == len(ks))
        if bf16 and check:
            self.check_tc()
        return x

    # ------------------------------------------------------------------ tensor-core inference
    def _tc_weights(self) -> dict:
        """BF16 weights in the layouts dseed_nn_conv_tc reads, and 16-byte
        aligned FP32 copies of biases and group-norm affines; rebuilt after any
        parameter update (the cache is cleared with the BF16 one)."""
        pk = self._bf16.get("__tc__")
        if pk is not None:
            return pk
        s = self.spec
        pk = {}

        def f32(name):
            t = torch.empty(self.offsets[name][1], dtype=torch.float32, device=self.dev)
            t.copy_(self.P(name).view(t.shape))
            return t

        def packed(name, rows_pad=None, cols_pad=None):
            co, k, ci = self.offsets[name + ".w"][1]
            kc = k * ci
            cp = cols_pad or kc
            w = torch.zeros((rows_pad or co, cp), dtype=torch.bfloat16, device=self.dev)
            _nn("im2col1d", self.P(name + ".w"), co, 1, kc, 1, 1, 0, 1, cp, w, 1)   # [co][kc] -> [co][cp]
            return w

        for name, cin, cout in NS.res_blocks(s):
            first = cin == s.D
            pk[name + ".c1"] = packed(name + ".c1", cols_pad=64 if first else None)
            pk[name + ".c2"] = packed(name + ".c2")
            if cin != cout:
                if first:
                    # the first block's 1x1 residual reads the 5-tap im2col rows of the
                    # input: its weights sit at the centre tap's columns, zeros elsewhere
                    co, _, ci = self.offsets[name + ".r.w"][1]
                    wr = torch.zeros((co, 64), dtype=torch.float32, device=self.dev)
                    c0 = (s.kernel // 2) * ci
                    wr[:, c0:c0 + ci] = self.P(name + ".r.w").view(co, ci)
                    pk[name + ".r"] = wr.to(torch.bfloat16).contiguous()
                else:
                    pk[name + ".r"] = packed(name + ".r")
                pk[name + ".r.b"] = f32(name + ".r.b")
            for t in ("c1.b", "c2.b", "g1.w", "g1.b", "g2.w", "g2.b"):
                pk[name + "." + t] = f32(name + "." + t)
        for name in ("fin.c",):
            pk[name] = packed(name)
            pk[name + ".b"] = f32(name + ".b")
        # the occupancy encoder's flattened linear [out][in] (in a multiple of 64)
        o_out, o_in = self.offsets["o.l.w"][1]
        pk["o.l"] = self.P("o.l.w").view(o_out, o_in).to(torch.bfloat16).contiguous()
        pk["o.l.b"] = f32("o.l.b")
        for name in ("down1", "down2"):
            # stride-2, 3-tap convolution as a 2-tap one over row pairs [x(2o), x(2o+1)]:
            # tap 0 (the pair o - 1) carries w0 on its second row, tap 1 (pair o) w1, w2
            co, _, ci = self.offsets[name + ".w"][1]
            w = self.P(name + ".w").view(co, 3, ci)
            w2 = torch.zeros((co, 2, 2 * ci), dtype=torch.float32, device=self.dev)
            w2[:, 0, ci:] = w[:, 0]
            w2[:, 1, :ci] = w[:, 1]
            w2[:, 1, ci:] = w[:, 2]
            pk[name + ".s2"] = w2.to(torch.bfloat16).reshape(co, 4 * ci).contiguous()
            pk[name + ".b"] = f32(name + ".b")
        for name in ("up2", "up1"):
            # nearest x2 upsampling then a 3-tap convolution, as one 3-tap convolution of
            # the input with 2 C outputs: channels [0, C) are output row 2m (taps w0,
            # w1 + w2, 0), channels [C, 2C) output row 2m + 1 (taps 0, w0 + w1, w2)
            co, _, ci = self.offsets[name + ".w"][1]
            w = self.P(name + ".w").view(co, 3, ci)
            wu = torch.zeros((2 * co, 3, ci), dtype=torch.float32, device=self.dev)
            wu[:co, 0] = w[:, 0]
            wu[:co, 1] = w[:, 1] + w[:, 2]
            wu[co:, 1] = w[:, 0] + w[:, 1]
            wu[co:, 2] = w[:, 2]
            pk[name + ".u2"] = wu.to(torch.bfloat16).reshape(2 * co, 3 * ci).contiguous()
            b = f32(name + ".b")
            pk[name + ".u2.b"] = torch.cat([b, b]).contiguous()
        # every block's FiLM linear stacked: rows [sum 2 cout], columns split into the
        # time-embedding part and the problem/occupancy part of the condition
        ft_rows = sum(2 * co for _, _, co in NS.res_blocks(s))
        Wt = torch.empty((ft_rows, s.t_dim), dtype=torch.float32, device=self.dev)
        Wpo = torch.empty((ft_rows, s.cond_dim - s.t_dim), dtype=torch.float32, device=self.dev)
        bf = torch.empty((ft_rows,), dtype=torch.float32, device=self.dev)
        off = 0
        pk["film_off"] = {}
        for name, _, co in NS.res_blocks(s):
            Wf = self.P(name + ".f.w")
            _nn("copy_cols", Wf, 2 * co, s.t_dim, s.cond_dim, 0, Wt[off:], s.t_dim, 0, 0)
            _nn("copy_cols", Wf, 2 * co, s.cond_dim - s.t_dim, s.cond_dim, s.t_dim, Wpo[off:],
                s.cond_dim - s.t_dim, 0, 0)
            bf[off:off + 2 * co].copy_(self.P(name + ".f.b"))
            pk["film_off"][name] = off
            off += 2 * co
        pk["film_Wt"], pk["film_Wpo"], pk["film_b"], pk["film_rows"] = Wt, Wpo, bf, ft_rows
        pk["fin.o"] = packed("fin.o", rows_pad=16)
        pk["fin.o.b"] = f32("fin.o.b")
        for t in ("fin.g.w", "fin.g.b"):
            pk[t] = f32(t)
        self._bf16["__tc__"] = pk
        return pk

    def _tc_block(self, W, srcs, N, L, name, cin, cout, film, rows, plain_in=None, film_ld=0, film_add=None):
        """Conditional residual block: conv-GN-Mish-FiLM, conv-GN-Mish + residual,
        as two (three with a 1x1 residual projection) fused kernels."""
        s = self.spec
        a0, a1 = srcs[0], (srcs[1] if len(srcs) > 1 else None)
        gn = dict(epilogue=B.EPI_GN, rows_per_sample=L, gn_eps=s.gn_eps, cout=cout, err=self._tc_err)
        fm = dict(film=film, film_ld=film_ld, sample_problem=rows, film_add=film_add)
        h = torch.empty((N, L, cout), dtype=torch.bfloat16, device=self.dev)
        if plain_in is not None:                      # first layer: im2col rows of the 7-channel input
            B.conv_tc(plain_in[0], W[name + ".c1"], h, n_samples=N * L, L=1, bias=W[name + ".c1.b"],
                      gamma=W[name + ".g1.w"], beta=W[name + ".g1.b"], **fm, **gn)
        else:
            B.conv_tc(a0, W[name + ".c1"].view(cout, s.kernel, cin), h, a1=a1, n_samples=N, L=L, taps=s.kernel,
                      pad=s.kernel // 2, bias=W[name + ".c1.b"], gamma=W[name + ".g1.w"], beta=W[name + ".g1.b"],
                      **fm, **gn)
        if cin != cout:
            r = torch.empty((N, L, cout), dtype=torch.bfloat16, device=self.dev)
            if plain_in is not None:
                B.conv_tc(plain_in[1], W[name + ".r"], r, n_samples=N * L, L=1, cout=cout, bias=W[name + ".r.b"],
                          epilogue=B.EPI_BF16, err=self._tc_err)
            else:
                B.conv_tc(a0, W[name + ".r"].view(cout, 1, cin), r, a1=a1, n_samples=N, L=L, cout=cout,
                          bias=W[name + ".r.b"], epilogue=B.EPI_BF16, err=self._tc_err)
        else:
            r = a0
        out = torch.empty((N, L, cout), dtype=torch.bfloat16, device=self.dev)
        B.conv_tc(h, W[name + ".c2"].view(cout, s.kernel, cout), out, n_samples=N, L=L, taps=s.kernel,
                  pad=s.kernel // 2, bias=W[name + ".c2.b"], gamma=W[name + ".g2.w"], beta=W[name + ".g2.b"],
                  res=r, **gn)
        return out

    def _tc_linear(self, W, x, R, name):
        """x FP32 [R][in] -> FP32 [R][out] on the tensor cores (BF16 operands, FP32
        accumulation): the occupancy encoder's flattened 2048 -> 128 linear, a
        few hundred rows with a long K."""
        out_f, in_f = W[name].shape
        xb = torch.empty((R, in_f), dtype=torch.bfloat16, device=self.dev)
        _nn("to_bf16", x, xb, R * in_f)
        y = torch.empty((R, out_f), dtype=torch.float32, device=self.dev)
        B.conv_tc(xb, W[name], y, n_samples=R, L=1, cout=out_f, bias=W[name + ".b"], epilogue=B.EPI_F32,
                  err=self._tc_err)
        return y

    def _tc_down(self, W, x, N, L, name, cout):
        """Stride-2 convolution (k = 3, pad 1) as a 2-tap convolution of the
        input's row pairs (the input viewed as [N][L/2][2 C]): no im2col buffer."""
        cin = x.shape[-1]
        Lo = L // 2
        y = torch.empty((N, Lo, cout), dtype=torch.bfloat16, device=self.dev)
        B.conv_tc(x.view(N, Lo, 2 * cin), W[name + ".s2"], y, n_samples=N, L=Lo, taps=2, pad=1, cout=cout,
                  bias=W[name + ".b"], epilogue=B.EPI_BF16, err=self._tc_err)
        return y, Lo

    def _tc_upconv(self, W, x, N, L, name, cout):
        """Nearest x2 upsampling followed by a 3-tap convolution, as one 3-tap
        convolution of x with 2 cout outputs whose halves are the even and odd
        output rows ([N][L][2 cout] is the memory of [N][2 L][cout])."""
        y = torch.empty((N, 2 * L, cout), dtype=torch.bfloat16, device=self.dev)
        B.conv_tc(x, W[name + ".u2"], y.view(N, L, 2 * cout), n_samples=N, L=L, taps=3, pad=1, cout=2 * cout,
                  bias=W[name + ".u2.b"], epilogue=B.EPI_BF16, err=self._tc_err)
        return y

    def unet_tc(self, x, N, film: torch.Tensor, rows: torch.Tensor,
                film_add: Optional[torch.Tensor] = None) -> torch.Tensor:
        """Predicted noise [N][T][D] (FP32) of x [N][T][D] (FP32) on the tensor
        cores.  film [P][sum 2 cout] = every block's FiLM rows per problem (from
        film_static / film_add_time); film_add [sum 2 cout] (optional) is added
        to every row (the time part shared by all problems at one DDIM step);
        rows [N] int32 = the problem of each sample."""
        s = self.spec
        c1, c2, c3 = s.chans
        T, D = s.T, s.D
        W = self._tc_weights()
        cols = torch.empty((N * T, 64), dtype=torch.bfloat16, device=self.dev)
        _nn("im2col1d", x, N, T, D, s.kernel, 1, s.kernel // 2, T, 64, cols, 1)
        FT, offs = W["film_rows"], W["film_off"]
        fa = (lambda name: film_add[offs[name]:]) if film_add is not None else (lambda name: None)
        blk = lambda srcs, L, name, ci, co, plain=None: self._tc_block(W, srcs, N, L, name, ci, co,
                                                                        film[:, offs[name]:], rows, plain, FT,
                                                                        fa(name))
        h = blk([None], T, "d1a", D, c1, (cols, cols))
        h = blk([h], T, "d1b", c1, c1)
        h, L2 = self._tc_down(W, h, N, T, "down1", c1)
        h = blk([h], L2, "d2a", c1, c2)
        s2 = blk([h], L2, "d2b", c2, c2)
        h, L3 = self._tc_down(W, s2, N, L2, "down2", c2)
        h = blk([h], L3, "d3a", c2, c3)
        s3 = blk([h], L3, "d3b", c3, c3)
        h = blk([s3], L3, "mid", c3, c3)
        h = blk([h, s3], L3, "u2a", 2 * c3, c2)
        h = blk([h], L3, "u2b", c2, c2)
        h = self._tc_upconv(W, h, N, L3, "up2", c2)
        h = blk([h, s2], L2, "u1a", 2 * c2, c1)
        h = blk([h], L2, "u1b", c1, c1)
        h = self._tc_upconv(W, h, N, L2, "up1", c1)
        g = torch.empty((N, T, c1), dtype=torch.bfloat16, device=self.dev)
        B.conv_tc(h, W["fin.c"].view(c1, s.kernel, c1), g, n_samples=N, L=T, taps=s.kernel, pad=s.kernel // 2,
                  cout=c1, bias=W["fin.c.b"], epilogue=B.EPI_GN, rows_per_sample=T, gn_eps=s.gn_eps,
                  gamma=W["fin.g.w"], beta=W["fin.g.b"], err=self._tc_err)
        out = torch.empty((N, T, D), dtype=torch.float32, device=self.dev)
        B.conv_tc(g, W["fin.o"], out, n_samples=N * T, L=1, cout=D, bias=W["fin.o.b"], epilogue=B.EPI_F32,
                  out_ld=D, err=self._tc_err)
        return out

    def film_static(self, qs, qg, goal, occ) -> torch.Tensor:
        """The per-problem part of every block's FiLM rows, [P][sum 2 cout]:
        W_f[:, problem/occupancy columns] Mish([p, o]) + b_f (the condition is
        Mish of a concatenation, so the FiLM linear splits into a time part and
        this part, which stays fixed over the DDIM steps)."""
        s = self.spec
        W = self._tc_weights()
        P = qs.shape[0]
        p2, o4 = self.problem_embed(qs, qg, goal, occ, None, last_linear=lambda x, R: self._tc_linear(W, x, R, "o.l"))
        po = self.mish(self.concat([p2, o4], P, None), None)
        F = torch.empty((P, W["film_rows"]), dtype=torch.float32, device=self.dev)
        K = s.cond_dim - s.t_dim
        _nn("gemm_f32", 0, 1, P, W["film_rows"], K, 1.0, po, K, W["film_Wpo"], K, 0.0, F, W["film_rows"],
            W["film_b"])
        return F

    def film_time_rows(self, k: torch.Tensor) -> torch.Tensor:
        """The time part of every block's FiLM rows, W_f[:, time columns]
        Mish(t(k)), for a vector of steps k [R]: [R][sum 2 cout]."""
        s = self.spec
        W = self._tc_weights()
        FT = W["film_rows"]
        mt = self.mish(self.time_embed(k, None), None)
        R = k.shape[0]
        Ft = torch.empty((R, FT), dtype=torch.float32, device=self.dev)
        _nn("gemm_f32", 0, 1, R, FT, s.t_dim, 1.0, mt, s.t_dim, W["film_Wt"], s.t_dim, 0.0, Ft, FT, None)
        return Ft

    def film_add_time(self, Fs: torch.Tensor, k: torch.Tensor) -> torch.Tensor:
        """FiLM rows = Fs + W_f[:, time columns] Mish(t(k)); k [1] (one step for
        every problem, a rank-1 update) or [P] (a step per row)."""
        s = self.spec
        W = self._tc_weights()
        FT = W["film_rows"]
        mt = self.mish(self.time_embed(k, None), None)                  # [R][t_dim]
        R = k.shape[0]
        Ft = torch.empty((R, FT), dtype=torch.float32, device=self.dev)
        _nn("gemm_f32", 0, 1, R, FT, s.t_dim, 1.0, mt, s.t_dim, W["film_Wt"], s.t_dim, 0.0, Ft, FT, None)
        F = Fs.clone()
        P = Fs.shape[0]
        if R == 1:
            ones = torch.ones((P, 1), dtype=torch.float32, device=self.dev)
            _nn("gemm_f32", 0, 0, P, FT, 1, 1.0, ones, 1, Ft, FT, 1.0, F, FT, None)
        else:
            _nn("axpby", 1.0, Fs, 1.0, Ft, F, F.numel())
        return F

    def check_tc(self):
        """Raise if a tensor-core kernel reported a pipeline wait that gave up."""
        code = int(self._tc_err.item())
        if code != 0:
            self._tc_err.zero_()
            raise B.DseedError(f"conv_tc: a pipeline wait gave up (code {code})")

    def infer_tc(self, xk, k, qs, qg, goal, occ):
        """Predicted noise with the tensor-core U-Net (condition per sample)."""
        N = xk.shape[0]
        film = self.film_add_time(self.film_static(qs, qg, goal, occ), k)
        rows = torch.arange(N, dtype=torch.int32, device=self.dev)
        out = self.unet_tc(xk.contiguous(), N, film, rows)
        self.check_tc()
        return out

    # ------------------------------------------------------------------ checkpoints
    def state(self) -> dict:
        return {"spec": self.spec.__dict__, "params": self.params.detach().cpu().numpy()}

    def load_state(self, st: dict):
        self.params.copy_(torch.from_numpy(np.asarray(st["params"], np.float32)))
        self._bf16.clear()


def _pad16(n: int) -> int:
    return (n + 15) // 16 * 16
