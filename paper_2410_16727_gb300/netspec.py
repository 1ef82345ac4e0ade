"""Architecture of the seed-proposal denoiser: hyperparameters and the ordered
list of parameter tensors (names and shapes) that lay out the flat FP32
parameter vector.  Data only -- shared by the CUDA path and its FP64 oracle the
way the robot description is; neither side's arithmetic lives here.

The network follows the paper's Sec. 4.2 ("Model Architecture"): a 3-level 1-D
temporal-convolution U-Net of conditional residual blocks (conv - group norm -
Mish, FiLM from the condition, conv - group norm - Mish, residual), a time-step
MLP, a problem encoding of the start and goal configurations and the goal
pose, and an observation encoding -- here a small 3-D convolutional encoder of
a 32^3 occupancy grid of the scene (in place of the paper's ViT on depth
images).
Channel widths (64, 128, 256) instead of the paper's (256, 512, 1024) give
about 4M parameters.

Shapes: Linear weights [out][in]; Conv1d weights [out][k][in] (matching the
im2col column order (tap, channel)); patch-3D-conv weights [out][P^3 * in]
with patch entries ordered (dz, dy, dx, channel).
"""
from __future__ import annotations

import dataclasses
from collections import OrderedDict
from typing import Dict, List, Tuple


@dataclasses.dataclass(frozen=True)
class NetSpec:
    T: int = 32                 # waypoints
    D: int = 7                  # joints
    chans: Tuple[int, int, int] = (64, 128, 256)
    kernel: int = 5
    groups: int = 8
    t_sin: int = 32             # sinusoidal time features
    t_dim: int = 128
    p_dim: int = 64
    occ_n: int = 32             # occupancy grid side
    occ_p1: int = 4             # first patch size  (32^3 -> 8^3)
    occ_c1: int = 16
    occ_p2: int = 2             # second patch size (8^3 -> 4^3)
    occ_c2: int = 32
    o_dim: int = 128
    K: int = 100                # diffusion steps (Sec. 4.3: K = 100)
    gn_eps: float = 1e-5

    @property
    def cond_dim(self) -> int:
        return self.t_dim + self.p_dim + self.o_dim

    @property
    def occ_g1(self) -> int:
        return self.occ_n // self.occ_p1

    @property
    def occ_g2(self) -> int:
        return self.occ_g1 // self.occ_p2


def res_blocks(spec: NetSpec) -> List[Tuple[str, int, int]]:
    c1, c2, c3 = spec.chans
    return [("d1a", spec.D, c1), ("d1b", c1, c1), ("d2a", c1, c2), ("d2b", c2, c2), ("d3a", c2, c3),
            ("d3b", c3, c3), ("mid", c3, c3), ("u2a", 2 * c3, c2), ("u2b", c2, c2), ("u1a", 2 * c2, c1),
            ("u1b", c1, c1)]


def param_shapes(spec: NetSpec) -> "OrderedDict[str, tuple]":
    s = OrderedDict()
    s["t.l1.w"] = (spec.t_dim, spec.t_sin)
    s["t.l1.b"] = (spec.t_dim,)
    s["t.l2.w"] = (spec.t_dim, spec.t_dim)
    s["t.l2.b"] = (spec.t_dim,)
    s["p.l1.w"] = (spec.p_dim, 2 * spec.D + 7)  # start and goal configurations + goal pose
    s["p.l1.b"] = (spec.p_dim,)
    s["p.l2.w"] = (spec.p_dim, spec.p_dim)
    s["p.l2.b"] = (spec.p_dim,)
    s["o.c1.w"] = (spec.occ_c1, spec.occ_p1 ** 3)
    s["o.c1.b"] = (spec.occ_c1,)
    s["o.c2.w"] = (spec.occ_c2, spec.occ_p2 ** 3 * spec.occ_c1)
    s["o.c2.b"] = (spec.occ_c2,)
    s["o.l.w"] = (spec.o_dim, spec.occ_g2 ** 3 * spec.occ_c2)
    s["o.l.b"] = (spec.o_dim,)
    k = spec.kernel
    for name, ci, co in res_blocks(spec):
        s[f"{name}.c1.w"] = (co, k, ci)
        s[f"{name}.c1.b"] = (co,)
        s[f"{name}.g1.w"] = (co,)
        s[f"{name}.g1.b"] = (co,)
        s[f"{name}.f.w"] = (2 * co, spec.cond_dim)
        s[f"{name}.f.b"] = (2 * co,)
        s[f"{name}.c2.w"] = (co, k, co)
        s[f"{name}.c2.b"] = (co,)
        s[f"{name}.g2.w"] = (co,)
        s[f"{name}.g2.b"] = (co,)
        if ci != co:
            s[f"{name}.r.w"] = (co, 1, ci)
            s[f"{name}.r.b"] = (co,)
    c1, c2, _ = spec.chans
    s["down1.w"] = (c1, 3, c1)
    s["down1.b"] = (c1,)
    s["down2.w"] = (c2, 3, c2)
    s["down2.b"] = (c2,)
    s["up2.w"] = (c2, 3, c2)
    s["up2.b"] = (c2,)
    s["up1.w"] = (c1, 3, c1)
    s["up1.b"] = (c1,)
    s["fin.c.w"] = (c1, k, c1)
    s["fin.c.b"] = (c1,)
    s["fin.g.w"] = (c1,)
    s["fin.g.b"] = (c1,)
    s["fin.o.w"] = (spec.D, 1, c1)
    s["fin.o.b"] = (spec.D,)
    return s


def param_offsets(spec: NetSpec) -> Dict[str, Tuple[int, tuple]]:
    out, off = {}, 0
    for name, shape in param_shapes(spec).items():
        n = 1
        for d in shape:
            n *= d
        out[name] = (off, shape)
        off += n
    return out


def param_count(spec: NetSpec) -> int:
    total = 0
    for shape in param_shapes(spec).values():
        n = 1
        for d in shape:
            n *= d
        total += n
    return total


def occ_patch_maps(spec: NetSpec):
    """Index maps of the two patch gathers (permutations of one sample's data):
    map1[e1] for the 32^3 grid -> [8^3 patches][4^3 entries]; map2[e2] for the
    [8^3][c1] features -> [4^3 patches][2^3 * c1 entries]."""
    n, p1, g1 = spec.occ_n, spec.occ_p1, spec.occ_g1
    map1 = []
    for pz in range(g1):
        for py in range(g1):
            for px in range(g1):
                for dz in range(p1):
                    for dy in range(p1):
                        for dx in range(p1):
                            map1.append(((pz * p1 + dz) * n + (py * p1 + dy)) * n + (px * p1 + dx))
    p2, g2, c1 = spec.occ_p2, spec.occ_g2, spec.occ_c1
    map2 = []
    for qz in range(g2):
        for qy in range(g2):
            for qx in range(g2):
                for dz in range(p2):
                    for dy in range(p2):
                        for dx in range(p2):
                            l1 = ((qz * p2 + dz) * g1 + (qy * p2 + dy)) * g1 + (qx * p2 + dx)
                            for c in range(c1):
                                map2.append(l1 * c1 + c)
    return map1, map2
