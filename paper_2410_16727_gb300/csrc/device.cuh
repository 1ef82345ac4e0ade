// device.cuh -- device functions of the seed-trajectory optimiser.
//
// Mapping: one warp owns one seed trajectory.  During an evaluation lane l
// owns waypoints l, l + 32, ... (TPL = waypoints per lane); the trajectory,
// the accepted point and the gradients live in the warp's slice of shared
// memory, so the L-BFGS update can use a flat mapping (lane l owns vector
// entries l, l + 32, ...) with conflict-free, coalesced accesses.
#pragma once

#include <cuda_runtime.h>
#include <math_constants.h>

#include "internal.h"

namespace dseed {

// ----------------------------------------------------------------- warp reductions
// Butterfly (xor) reductions: every lane ends with the same bits, since each
// stage adds the same two operands in both partner lanes.
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ float warp_min(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// ----------------------------------------------------------------- scene / ESDF
struct SceneView {
    const float *__restrict__ phi;
    float ox, oy, oz, inv_res, res;
    float skip_pad;           // L sqrt(3) res + 1e-5, or +inf when the early-out is off
    float lip;                // Lipschitz bound L of phi (0: early-outs off)
    int nx, ny, nz;
    bool ok;                  // descriptor usable: non-null ESDF, every dimension >= 2, res > 0
};

// Scene idx of the table (the caller checks 0 <= idx < n_scenes).
__device__ __forceinline__ SceneView load_scene(const DseedScene *scenes, int idx) {
    const DseedScene &s = scenes[idx];
    SceneView v;
    v.ok = s.esdf_dev != nullptr && s.grid.nx >= 2 && s.grid.ny >= 2 && s.grid.nz >= 2 && s.grid.res > 0.0f;
    v.phi = s.esdf_dev;
    v.ox = s.grid.origin[0];
    v.oy = s.grid.origin[1];
    v.oz = s.grid.origin[2];
    v.inv_res = 1.0f / s.grid.res;
    v.res = s.grid.res;
    v.skip_pad = s.lipschitz > 0.0f ? s.lipschitz * 1.7320508f * s.grid.res + 1e-5f : CUDART_INF_F;
    v.lip = s.lipschitz > 0.0f ? s.lipschitz : 0.0f;
    v.nx = s.grid.nx;
    v.ny = s.grid.ny;
    v.nz = s.grid.nz;
    return v;
}

// Cell of a continuous voxel coordinate u = (p - origin) / res - 1/2 along one
// axis: u is clamped into [0, n - 1], the cell is i0 = min(floor(u), n - 2)
// and f = u - i0.  Returns true when the point lay outside the grid (the
// gradient is zero along that axis).  NaN and infinities land on a valid cell
// (fmaxf/fminf drop NaN), so no access can leave the grid.
__device__ __forceinline__ bool cell_axis(float u, int n, int &i0, float &f) {
    const float hi = (float)(n - 1);
    const bool clamped = !(u >= 0.0f && u <= hi);
    u = fminf(fmaxf(u, 0.0f), hi);
    const int c = min(__float2int_rd(u), n - 2);
    i0 = c;
    f = u - (float)c;
    return clamped;
}

// Cell index only (the corner (i0, j0, k0) of the cell that holds u): the same
// cell as cell_axis, from floor(u) clamped to [0, n - 2] (NaN converts to 0,
// out-of-range values saturate).
__device__ __forceinline__ int cell_index(float u, int n) {
    return min(max(__float2int_rd(u), 0), n - 2);
}

// ESDF value at that corner; grids are limited to 2^31 voxels so the index is 32-bit.
__device__ __forceinline__ float corner_value(const SceneView &sv, float ux, float uy, float uz) {
    const int idx = (cell_index(uz, sv.nz) * sv.ny + cell_index(uy, sv.ny)) * sv.nx + cell_index(ux, sv.nx);
    return __ldg(sv.phi + idx);
}

__device__ __forceinline__ const float *cell_ptr(const SceneView &sv, int ix, int iy, int iz) {
    return sv.phi + ((size_t)iz * (size_t)sv.ny + (size_t)iy) * (size_t)sv.nx + ix;
}

// Trilinear interpolation of the ESDF at voxel coordinates (ux, uy, uz) from
// the 8 corners of its cell (point loads through the read-only path), with the
// analytic gradient in world units (d phi / d u divided by res).
template <bool GRAD>
__device__ __forceinline__ float esdf_interp(const SceneView &sv, float ux, float uy, float uz,
                                             float &gx, float &gy, float &gz) {
    int ix, iy, iz;
    float fx, fy, fz;
    const bool cx = cell_axis(ux, sv.nx, ix, fx);
    const bool cy = cell_axis(uy, sv.ny, iy, fy);
    const bool cz = cell_axis(uz, sv.nz, iz, fz);
    const size_t sy = (size_t)sv.nx, sz = (size_t)sv.nx * (size_t)sv.ny;
    const float *b = cell_ptr(sv, ix, iy, iz);
    const float v000 = __ldg(b), v100 = __ldg(b + 1);
    const float v010 = __ldg(b + sy), v110 = __ldg(b + sy + 1);
    const float v001 = __ldg(b + sz), v101 = __ldg(b + sz + 1);
    const float v011 = __ldg(b + sz + sy), v111 = __ldg(b + sz + sy + 1);
    const float c00 = fmaf(fx, v100 - v000, v000);
    const float c10 = fmaf(fx, v110 - v010, v010);
    const float c01 = fmaf(fx, v101 - v001, v001);
    const float c11 = fmaf(fx, v111 - v011, v011);
    const float c0 = fmaf(fy, c10 - c00, c00);
    const float c1 = fmaf(fy, c11 - c01, c01);
    if (GRAD) {
        const float d00 = v100 - v000, d10 = v110 - v010, d01 = v101 - v001, d11 = v111 - v011;
        const float dx0 = fmaf(fy, d10 - d00, d00), dx1 = fmaf(fy, d11 - d01, d01);
        const float ey0 = c10 - c00, ey1 = c11 - c01;
        gx = cx ? 0.0f : fmaf(fz, dx1 - dx0, dx0) * sv.inv_res;
        gy = cy ? 0.0f : fmaf(fz, ey1 - ey0, ey0) * sv.inv_res;
        gz = cz ? 0.0f : (c1 - c0) * sv.inv_res;
    }
    return fmaf(fz, c1 - c0, c0);
}

// ----------------------------------------------------------------- kinematics
// One step of the modified-DH chain: R <- R RotX(alpha) RotZ(theta),
// p <- p + a x_prev + d z_new (R row-major, columns x, y, z).
__device__ __forceinline__ void dh_step(float (&R)[9], float (&p)[3], float a, float d, float ca,
                                        float sa, float ct, float st) {
    p[0] = fmaf(a, R[0], p[0]);
    p[1] = fmaf(a, R[3], p[1]);
    p[2] = fmaf(a, R[6], p[2]);
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        float xr = R[3 * r], yr = R[3 * r + 1], zr = R[3 * r + 2];
        float y1 = fmaf(ca, yr, sa * zr);
        float z1 = fmaf(ca, zr, -sa * yr);
        R[3 * r] = fmaf(ct, xr, st * y1);
        R[3 * r + 1] = fmaf(ct, y1, -st * xr);
        R[3 * r + 2] = z1;
    }
    p[0] = fmaf(d, R[2], p[0]);
    p[1] = fmaf(d, R[5], p[1]);
    p[2] = fmaf(d, R[8], p[2]);
}

// Goal: position and rotation matrix of the (normalised) goal quaternion.
struct Goal {
    float p[3];
    float R[9];
};

__device__ __forceinline__ Goal make_goal(const float *g) {
    Goal G;
    G.p[0] = g[0];
    G.p[1] = g[1];
    G.p[2] = g[2];
    float w = g[3], x = g[4], y = g[5], z = g[6];
    float inv = rsqrtf(w * w + x * x + y * y + z * z);
    w *= inv; x *= inv; y *= inv; z *= inv;
    G.R[0] = 1.0f - 2.0f * (y * y + z * z); G.R[1] = 2.0f * (x * y - w * z); G.R[2] = 2.0f * (x * z + w * y);
    G.R[3] = 2.0f * (x * y + w * z); G.R[4] = 1.0f - 2.0f * (x * x + z * z); G.R[5] = 2.0f * (y * z - w * x);
    G.R[6] = 2.0f * (x * z - w * y); G.R[7] = 2.0f * (y * z + w * x); G.R[8] = 1.0f - 2.0f * (x * x + y * y);
    return G;
}

enum { MODE_COST = 0, MODE_GRAD = 1, MODE_EVAL = 2 };

struct WaypointAcc {
    float c_world, c_goal;
    float min_clear;          // MODE_EVAL
    float pos_err, rot_err;   // MODE_EVAL, last waypoint only
};

// World and goal terms of one waypoint q (and, in MODE_GRAD, their gradient
// added into gq).  Adjoint by Jacobian-transpose accumulation: each active
// sphere applies the force g_k = dC/dc_k = -w_c grad(phi) at c_k; joint i
// receives z_i . sum over spheres beyond joint i of (c_k - p_i) x g_k.  With
// running sums F = sum g_k and M = sum c_k x g_k over the spheres met so far,
// that is z_i . (M_all - M_<i) - (z_i x p_i) . (F_all - F_<i): the prefix
// part b_i is recorded when frame i is reached, the rest once all spheres and
// the goal wrench are in.  The 8-frame loop stays rolled: one copy of the
// sphere loop keeps the fused kernel small enough for the instruction cache
// (unrolled, the plans were 32% slower with the same results).

// Self-collision scratch of one lane, in its warp's shared slice (element e of
// lane l at sbuf[e * 32 + l]): the transforms (R row-major, p) of frames 1..6
// for the later frames' pair tests, then per-frame deposits (force, moment) of
// the pair reactions, applied to the joints that move that frame.
constexpr int kSelfFrames = 6;
constexpr int kSelfFloats = kSelfFrames * 12 + kSelfFrames * 6;   // per lane

__device__ __forceinline__ unsigned long long frame_bits(const KRobot &rb, int a) {
    const int b = rb.frame_begin[a - 1], e = rb.frame_begin[a];
    const unsigned long long hi = e >= 64 ? ~0ull : ((1ull << e) - 1ull);
    const unsigned long long lo = b >= 64 ? ~0ull : ((1ull << b) - 1ull);
    return hi & ~lo;
}

// Per-lane scratch of the frame loop (element e of lane l at fsc[e * 32], fsc
// already offset by l): the joint axes z_i [0, 21), the moments z_i x p_i of
// the axes about the origin [21, 42) and the adjoint prefixes b_i [42, 49),
// written as the chain is walked and read by the adjoint's second pass.  The
// loop runs rolled, so these are indexed by the frame number; in shared memory
// they stay out of the L1 cache that the ESDF gathers use.
constexpr int kFrameScratch = 49;

// The configuration is q = qt (interp false) or the swept-check interpolant
// q = qt + u (qp - qt) of the segment from qp = y_{t-1} to qt = y_t (interp
// true: world term only, no goal or self term).
template <int MODE, bool SELF = false>
__device__ __forceinline__ void waypoint_terms(const KRobot &rb, const KCost &kc, const SceneView &sv,
                                               const float *qt, const float *qp, float u, bool interp, bool last,
                                               const Goal &G, WaypointAcc &acc, float (&gq)[7], float *fsc,
                                               float *sbuf = nullptr) {
    const bool self_on = SELF && !interp;
    float R[9] = {1.f, 0.f, 0.f, 0.f, 1.f, 0.f, 0.f, 0.f, 1.f};
    float p[3] = {0.f, 0.f, 0.f};
    float *const zs = fsc, *const ws_ = fsc + 21 * 32, *const bj = fsc + 42 * 32;
    float Fx = 0.f, Fy = 0.f, Fz = 0.f, Mx = 0.f, My = 0.f, Mz = 0.f;
#pragma unroll 1
    for (int L = 1; L <= 8; ++L) {
        float st, ct;
        if (L <= 7) {
            const float qL = interp ? fmaf(u, qp[L - 1] - qt[L - 1], qt[L - 1]) : qt[L - 1];
            sincosf(qL + rb.off[L - 1], &st, &ct);
        } else {
            st = rb.sf8;
            ct = rb.cf8;
        }
        dh_step(R, p, rb.a[L - 1], rb.d[L - 1], rb.ca[L - 1], rb.sa[L - 1], ct, st);
        if (MODE == MODE_GRAD && L <= 7) {
            const int i = L <= 7 ? L - 1 : 0;
            float z0 = R[2], z1 = R[5], z2 = R[8];
            float w0 = z1 * p[2] - z2 * p[1];
            float w1 = z2 * p[0] - z0 * p[2];
            float w2 = z0 * p[1] - z1 * p[0];
            bj[i * 32] = (z0 * Mx + z1 * My + z2 * Mz) - (w0 * Fx + w1 * Fy + w2 * Fz);
            zs[(3 * i) * 32] = z0; zs[(3 * i + 1) * 32] = z1; zs[(3 * i + 2) * 32] = z2;
            ws_[(3 * i) * 32] = w0; ws_[(3 * i + 1) * 32] = w1; ws_[(3 * i + 2) * 32] = w2;
        }
        if (self_on) {
            // C_self against frames a <= L - 2: for a checked pair (k on frame L, j on
            // frame a) the hinge w_s max(0, r_k + r_j + eta_s - |c_k - c_j|) pushes
            // sphere k with g = dC/dc_k = -w_s (c_k - c_j) / |c_k - c_j| (entered now,
            // as for the world spheres of frame L) and sphere j with -g; the joints
            // that move both see no net effect, so -g is deposited at c_k on frame a
            // and cancels g for the joints that move frame a (added in the second pass)
            const int lane = threadIdx.x & 31;
            if (L == 1)
                for (int e = 0; e < kSelfFrames * 6; ++e) sbuf[(kSelfFrames * 12 + e) * 32 + lane] = 0.f;
            const unsigned fm = rb.self_frames[L - 1];
            if (fm) {
                const float4 fbL = rb.fbound[L - 1];
                const float bx = fmaf(R[0], fbL.x, fmaf(R[1], fbL.y, fmaf(R[2], fbL.z, p[0])));
                const float by = fmaf(R[3], fbL.x, fmaf(R[4], fbL.y, fmaf(R[5], fbL.z, p[1])));
                const float bz = fmaf(R[6], fbL.x, fmaf(R[7], fbL.y, fmaf(R[8], fbL.z, p[2])));
                for (int a = 1; a <= L - 2; ++a) {
                    if (!((fm >> (a - 1)) & 1u)) continue;
                    float Ra[12];
#pragma unroll
                    for (int e = 0; e < 12; ++e) Ra[e] = sbuf[((a - 1) * 12 + e) * 32 + lane];
                    if (MODE != MODE_EVAL) {
                        // frame-level bound: every sphere lies within fbound.w (radius included) of
                        // its frame's bounding centre, so |c_k - c_j| - r_k - r_j >= dd - wL - wa
                        const float4 fba = rb.fbound[a - 1];
                        const float ax = fmaf(Ra[0], fba.x, fmaf(Ra[1], fba.y, fmaf(Ra[2], fba.z, Ra[9])));
                        const float ay = fmaf(Ra[3], fba.x, fmaf(Ra[4], fba.y, fmaf(Ra[5], fba.z, Ra[10])));
                        const float az = fmaf(Ra[6], fba.x, fmaf(Ra[7], fba.y, fmaf(Ra[8], fba.z, Ra[11])));
                        const float dd = sqrtf((bx - ax) * (bx - ax) + (by - ay) * (by - ay) + (bz - az) * (bz - az));
                        if (dd - fbL.w - fba.w >= kc.eta_s + 1e-4f) continue;
                    }
                    const unsigned long long abits = frame_bits(rb, a);
                    for (int k = rb.frame_begin[L - 1]; k < rb.frame_begin[L]; ++k) {
                        unsigned long long sel = rb.self_mask[k] & abits;
                        if (!sel) continue;
                        const float4 sk = rb.sph[k];
                        const float ckx = fmaf(R[0], sk.x, fmaf(R[1], sk.y, fmaf(R[2], sk.z, p[0])));
                        const float cky = fmaf(R[3], sk.x, fmaf(R[4], sk.y, fmaf(R[5], sk.z, p[1])));
                        const float ckz = fmaf(R[6], sk.x, fmaf(R[7], sk.y, fmaf(R[8], sk.z, p[2])));
                        while (sel) {
                            const int j = __ffsll((long long)sel) - 1;
                            sel &= sel - 1ull;
                            const float4 sj = rb.sph[j];
                            const float cjx = fmaf(Ra[0], sj.x, fmaf(Ra[1], sj.y, fmaf(Ra[2], sj.z, Ra[9])));
                            const float cjy = fmaf(Ra[3], sj.x, fmaf(Ra[4], sj.y, fmaf(Ra[5], sj.z, Ra[10])));
                            const float cjz = fmaf(Ra[6], sj.x, fmaf(Ra[7], sj.y, fmaf(Ra[8], sj.z, Ra[11])));
                            const float dx = ckx - cjx, dy = cky - cjy, dz = ckz - cjz;
                            const float dist = sqrtf(dx * dx + dy * dy + dz * dz);
                            if (MODE == MODE_EVAL) acc.min_clear = fminf(acc.min_clear, dist - sk.w - sj.w);
                            const float h = sk.w + sj.w + kc.eta_s - dist;
                            if (h > 0.0f) {
                                acc.c_world = fmaf(kc.w_s, h, acc.c_world);
                                if (MODE == MODE_GRAD && dist > 0.0f) {
                                    const float inv = kc.w_s / dist;
                                    const float gx = -dx * inv, gy = -dy * inv, gz = -dz * inv;
                                    const float mx = cky * gz - ckz * gy, my = ckz * gx - ckx * gz,
                                                mz = ckx * gy - cky * gx;
                                    Fx += gx; Fy += gy; Fz += gz;
                                    Mx += mx; My += my; Mz += mz;
                                    float *dep = sbuf + (kSelfFrames * 12 + (a - 1) * 6) * 32 + lane;
                                    dep[0] -= gx; dep[32] -= gy; dep[64] -= gz;
                                    dep[96] -= mx; dep[128] -= my; dep[160] -= mz;
                                }
                            }
                        }
                    }
                }
            }
            if (L <= kSelfFrames) {
#pragma unroll
                for (int e = 0; e < 9; ++e) sbuf[((L - 1) * 12 + e) * 32 + lane] = R[e];
#pragma unroll
                for (int e = 0; e < 3; ++e) sbuf[((L - 1) * 12 + 9 + e) * 32 + lane] = p[e];
            }
        }
        // frame L in voxel coordinates: u = Rv o + pv for an offset o
        float Rv[9], pv[3];
#pragma unroll
        for (int r = 0; r < 9; ++r) Rv[r] = R[r] * sv.inv_res;
        pv[0] = fmaf(p[0] - sv.ox, sv.inv_res, -0.5f);
        pv[1] = fmaf(p[1] - sv.oy, sv.inv_res, -0.5f);
        pv[2] = fmaf(p[2] - sv.oz, sv.inv_res, -0.5f);
        const int k1 = rb.frame_begin[L];
        if (MODE != MODE_EVAL && sv.lip > 0.0f && k1 > rb.frame_begin[L - 1]) {
            // all spheres of the frame lie inside its bounding sphere (centre b,
            // radius R): for sphere k, phi(c_k) >= v_b - L (2 sqrt(3) res + R - r_k)
            // (corner of b's cell to corner of c_k's cell, through the clamped
            // points), so one read clears the whole frame when it exceeds
            // r_k + eta for every k
            const float4 fb = rb.fbound[L - 1];
            const float ux = fmaf(Rv[0], fb.x, fmaf(Rv[1], fb.y, fmaf(Rv[2], fb.z, pv[0])));
            const float uy = fmaf(Rv[3], fb.x, fmaf(Rv[4], fb.y, fmaf(Rv[5], fb.z, pv[1])));
            const float uz = fmaf(Rv[6], fb.x, fmaf(Rv[7], fb.y, fmaf(Rv[8], fb.z, pv[2])));
            const float one_m_l = 1.0f - sv.lip;
            const float thr = kc.eta + sv.lip * (2.0f * 1.7320508f * sv.res + fb.w) +
                              fmaxf(one_m_l * rb.frmin[L - 1], one_m_l * rb.frmax[L - 1]) + 1e-5f;
            if (corner_value(sv, ux, uy, uz) >= thr) continue;
        }
        for (int k = rb.frame_begin[L - 1]; k < k1; ++k) {
            // one corner of the sphere's cell first: every corner lies within sqrt(3) res
            // of the others, so for an L-Lipschitz field phi(c) >= v0 - L sqrt(3) res, and
            // v0 >= r + eta + skip_pad means the hinge is inactive (the other 7 loads skipped)
            float v0 = -CUDART_INF_F;
            if (MODE != MODE_EVAL) {
                const float4 s = rb.sph[k];
                const float ux = fmaf(Rv[0], s.x, fmaf(Rv[1], s.y, fmaf(Rv[2], s.z, pv[0])));
                const float uy = fmaf(Rv[3], s.x, fmaf(Rv[4], s.y, fmaf(Rv[5], s.z, pv[1])));
                const float uz = fmaf(Rv[6], s.x, fmaf(Rv[7], s.y, fmaf(Rv[8], s.z, pv[2])));
                v0 = corner_value(sv, ux, uy, uz);
            }
            // then the full interpolation of a sphere the bound cannot clear
            {
                const float4 s = rb.sph[k];
                const float hinge_at = s.w + kc.eta;
                if (MODE != MODE_EVAL && v0 >= hinge_at + sv.skip_pad) continue;
                const float ux = fmaf(Rv[0], s.x, fmaf(Rv[1], s.y, fmaf(Rv[2], s.z, pv[0])));
                const float uy = fmaf(Rv[3], s.x, fmaf(Rv[4], s.y, fmaf(Rv[5], s.z, pv[1])));
                const float uz = fmaf(Rv[6], s.x, fmaf(Rv[7], s.y, fmaf(Rv[8], s.z, pv[2])));
                float gx, gy, gz;
                const float phi = esdf_interp<MODE == MODE_GRAD>(sv, ux, uy, uz, gx, gy, gz);
                if (MODE == MODE_EVAL) acc.min_clear = fminf(acc.min_clear, phi - s.w);
                const float h = hinge_at - phi;
                if (h > 0.0f) {
                    acc.c_world = fmaf(kc.w_c, h, acc.c_world);
                    if (MODE == MODE_GRAD) {
                        // moment about the world origin needs the centre in world units
                        const float cx = fmaf(R[0], s.x, fmaf(R[1], s.y, fmaf(R[2], s.z, p[0])));
                        const float cy = fmaf(R[3], s.x, fmaf(R[4], s.y, fmaf(R[5], s.z, p[1])));
                        const float cz = fmaf(R[6], s.x, fmaf(R[7], s.y, fmaf(R[8], s.z, p[2])));
                        const float fx = -kc.w_c * gx, fy = -kc.w_c * gy, fz = -kc.w_c * gz;
                        Fx += fx; Fy += fy; Fz += fz;
                        Mx += cy * fz - cz * fy;
                        My += cz * fx - cx * fz;
                        Mz += cx * fy - cy * fx;
                    }
                }
            }
        }
    }
    if (last) {
        // C_goal = w_p |p - p*|^2 + w_R (1 - <q, q*>^2), with
        // 1 - <q, q*>^2 = (3 - tr(R*^T R)) / 4 for unit quaternions.
        float e0 = p[0] - G.p[0], e1 = p[1] - G.p[1], e2 = p[2] - G.p[2];
        // A = R R*^T
        float A[9];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j)
                A[3 * i + j] = R[3 * i] * G.R[3 * j] + R[3 * i + 1] * G.R[3 * j + 1] + R[3 * i + 2] * G.R[3 * j + 2];
        float tr = A[0] + A[4] + A[8];
        acc.c_goal = kc.w_p * (e0 * e0 + e1 * e1 + e2 * e2) + kc.w_R * 0.25f * (3.0f - tr);
        float v0 = A[5] - A[7], v1 = A[6] - A[2], v2 = A[1] - A[3];
        if (MODE == MODE_EVAL) {
            acc.pos_err = sqrtf(e0 * e0 + e1 * e1 + e2 * e2);
            acc.rot_err = atan2f(0.5f * sqrtf(v0 * v0 + v1 * v1 + v2 * v2), 0.5f * (tr - 1.0f));
        }
        if (MODE == MODE_GRAD) {
            // position: force 2 w_p e at the flange origin; orientation: torque
            // -(w_R / 4) (A12 - A21, A20 - A02, A01 - A10) (d tr(A) = dw . v)
            float fx = 2.0f * kc.w_p * e0, fy = 2.0f * kc.w_p * e1, fz = 2.0f * kc.w_p * e2;
            Fx += fx; Fy += fy; Fz += fz;
            Mx += p[1] * fz - p[2] * fy;
            My += p[2] * fx - p[0] * fz;
            Mz += p[0] * fy - p[1] * fx;
            float tq = -0.25f * kc.w_R;
            Mx = fmaf(tq, v0, Mx);
            My = fmaf(tq, v1, My);
            Mz = fmaf(tq, v2, Mz);
        }
    }
    if (MODE == MODE_GRAD) {
        {
            // second pass: the joint axes z_i and moments z_i x p_i recorded by the
            // first pass (kept in the frame scratch rather than live across the
            // sphere loop) against the total wrench
            // self-collision reactions deposited on frames 1..6: joint i moves frames
            // >= i + 1, so it takes the deposits of frames a >= i + 1 (a suffix sum)
            float SD[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            if (self_on) {
                const int lane = threadIdx.x & 31;
                for (int a = 0; a < kSelfFrames; ++a)
#pragma unroll
                    for (int e = 0; e < 6; ++e) SD[e] += sbuf[(kSelfFrames * 12 + a * 6 + e) * 32 + lane];
            }
#pragma unroll
            for (int i = 0; i < 7; ++i) {
                const float z0 = zs[(3 * i) * 32], z1 = zs[(3 * i + 1) * 32], z2 = zs[(3 * i + 2) * 32];
                const float w0 = ws_[(3 * i) * 32], w1 = ws_[(3 * i + 1) * 32], w2 = ws_[(3 * i + 2) * 32];
                gq[i] += (z0 * Mx + z1 * My + z2 * Mz) - (w0 * Fx + w1 * Fy + w2 * Fz) - bj[i * 32];
                if (self_on) {
                    gq[i] += (z0 * SD[3] + z1 * SD[4] + z2 * SD[5]) - (w0 * SD[0] + w1 * SD[1] + w2 * SD[2]);
                    if (i < kSelfFrames) {
                        const int lane = threadIdx.x & 31;
#pragma unroll
                        for (int e = 0; e < 6; ++e) SD[e] -= sbuf[(kSelfFrames * 12 + i * 6 + e) * 32 + lane];
                    }
                }
            }
        }
    }
}

// ----------------------------------------------------------------- one trajectory
// Shared-memory slice of one warp (floats):
//   xs [(T + 3) * 7]   y_-2, y_-1, y_0 (= q_start) then the trial waypoints 1..T
//   es [3 * (T + 3) * 7] velocity / acceleration / jerk adjoint weights, rows >= T zero;
//                      before they are written, the lanes' frame-loop scratch (at least
//                      21 * 32 floats)
//   gs [T * 7]         gradient of the trial point
//   xa, ga, dd [T * 7] accepted point, its gradient, current search direction (optimiser;
//                      the direction may live in global memory instead, see carve)
//   v [32]             L-BFGS scalars: rho per slot [0, 8), y^T y of the newest pair [8],
//                      alpha_i of the two-loop [16, 24)
__host__ __device__ constexpr int es_floats(int T) {
    return 3 * (T + kPad) * 7 > kFrameScratch * 32 ? 3 * (T + kPad) * 7 : kFrameScratch * 32;
}
__host__ __device__ constexpr int warp_smem_floats(int T) { return (T + kPad) * 7 + es_floats(T) + 4 * 7 * T + 32; }

struct WarpSmem {
    float *xs, *es, *gs, *xa, *ga, *dd, *v;
    float *self;      // [kSelfFloats][32] self-collision scratch (SELF kernels only)
};

// Per-warp shared floats, with the self-collision scratch when SELF.
__host__ __device__ constexpr int warp_smem_floats(int T, bool self) {
    return warp_smem_floats(T) + (self ? kSelfFloats * 32 : 0);
}

// Per-warp shared floats of a slice whose search direction lives elsewhere
// (global memory), with the self-collision scratch when SELF.
__host__ __device__ constexpr int warp_smem_floats_nodd(int T, bool self) { return warp_smem_floats(T, self) - 7 * T; }

// Slice of one warp.  dd_global: the search direction is kept in global
// memory at that address instead of the slice (the slice then omits it).
__device__ __forceinline__ WarpSmem carve(float *base, int T, float *dd_global = nullptr) {
    WarpSmem w;
    w.xs = base;
    w.es = w.xs + (T + kPad) * 7;
    w.gs = w.es + es_floats(T);
    w.xa = w.gs + T * 7;
    w.ga = w.xa + T * 7;
    if (dd_global) {
        w.dd = dd_global;
        w.v = w.ga + T * 7;
    } else {
        w.dd = w.ga + T * 7;
        w.v = w.dd + T * 7;
    }
    w.self = w.v + 32;
    return w;
}

struct EvalOut {
    float cost;
    float terms[4];                       // world, smooth, goal, limit
    float min_clear, pos_err, rot_err, max_jerk, lim_viol;
};

// Cost (MODE_COST), cost and gradient into ws.gs (MODE_GRAD), or cost and
// success metrics (MODE_EVAL) of the trajectory held in ws.xs.  Warp-uniform
// result.  ws.es rows T..T+2 must be zero (MODE_GRAD).
template <int TPL, int MODE, bool SELF = false, bool SWEEP = false>
__device__ __forceinline__ EvalOut warp_eval(const KRobot &rb, const KCost &kc, const SceneView &sv,
                                             int T, const Goal &G, const WarpSmem &ws, bool want_terms) {
    const int lane = threadIdx.x & 31;
    float c_world = 0.f, c_smooth = 0.f, c_goal = 0.f, c_limit = 0.f;
    float min_clear = CUDART_INF_F, pos_err = 0.f, rot_err = 0.f, max_jerk = 0.f, lim_viol = 0.f;
    // With several waypoints per lane (and no swept check) the waypoint loop stays
    // rolled, so the kinematics / sphere / adjoint body is in the instruction
    // stream once: each waypoint's gradient row is kept in ws.gs (the lane's own
    // rows only) instead of a register array indexed by the waypoint.
    constexpr bool kRoll = TPL >= 2 && !SWEEP;
    float gq[kRoll ? 1 : TPL][7];
    const float inv_dt = kc.inv_dt;
    const int R3 = (T + kPad) * 7;
    if (MODE == MODE_GRAD && SWEEP) {
        // gs row t - 1 collects the interpolants' share of waypoint t - 1 from the lane of waypoint t
        for (int e = lane; e < T * 7; e += 32) ws.gs[e] = 0.f;
        __syncwarp();
    }
    if (kRoll) {
#pragma unroll 1
        for (int u = 0; u < TPL; ++u) {
            const int t0 = lane + 32 * u;   // waypoint t = t0 + 1
            if (t0 < T) {
                float gw[7];
#pragma unroll
                for (int j = 0; j < 7; ++j) gw[j] = 0.f;
                WaypointAcc acc{0.f, 0.f, CUDART_INF_F, 0.f, 0.f};
                const float *y = ws.xs + (t0 + kPad) * 7;
                waypoint_terms<MODE, SELF>(rb, kc, sv, y, y, 0.0f, false, t0 == T - 1, G, acc, gw, ws.es + lane,
                                           ws.self);
                c_world += acc.c_world;
                c_goal += acc.c_goal;
                if (MODE == MODE_EVAL) {
                    min_clear = fminf(min_clear, acc.min_clear);
                    if (t0 == T - 1) { pos_err = acc.pos_err; rot_err = acc.rot_err; }
                }
                if (MODE == MODE_GRAD) {
#pragma unroll
                    for (int j = 0; j < 7; ++j) ws.gs[t0 * 7 + j] = gw[j];
                }
            }
        }
    }
#pragma unroll
    for (int u = 0; u < (kRoll ? 0 : TPL); ++u) {
        const int t0 = lane + 32 * u;   // waypoint t = t0 + 1
#pragma unroll
        for (int j = 0; j < 7; ++j) gq[u][j] = 0.f;
        if (t0 < T && !SWEEP) {
            WaypointAcc acc{0.f, 0.f, CUDART_INF_F, 0.f, 0.f};
            const float *y = ws.xs + (t0 + kPad) * 7;
            waypoint_terms<MODE, SELF>(rb, kc, sv, y, y, 0.0f, false, t0 == T - 1, G, acc, gq[u], ws.es + lane,
                                       ws.self);
            c_world += acc.c_world;
            c_goal += acc.c_goal;
            if (MODE == MODE_EVAL) {
                min_clear = fminf(min_clear, acc.min_clear);
                if (t0 == T - 1) { pos_err = acc.pos_err; rot_err = acc.rot_err; }
            }
        }
        if (t0 < T && SWEEP) {
            const float *y = ws.xs + (t0 + kPad) * 7;   // y_t; y - 7 = y_{t-1} (y_0 = q_start)
            // s = 0: the waypoint; s = 1..n_sweep: the interpolants of segment (y_{t-1}, y_t)
            for (int s = 0; s <= kc.n_sweep; ++s) {
                const float us = (float)s * kc.sweep_u;   // weight of y_{t-1}
                float gw[7];
#pragma unroll
                for (int j = 0; j < 7; ++j) gw[j] = 0.f;
                WaypointAcc acc{0.f, 0.f, CUDART_INF_F, 0.f, 0.f};
                waypoint_terms<MODE, SELF>(rb, kc, sv, y, y - 7, us, s > 0, s == 0 && t0 == T - 1, G, acc, gw,
                                           ws.es + lane, ws.self);
                c_world += acc.c_world;
                c_goal += acc.c_goal;
                if (MODE == MODE_EVAL) {
                    min_clear = fminf(min_clear, acc.min_clear);
                    if (s == 0 && t0 == T - 1) { pos_err = acc.pos_err; rot_err = acc.rot_err; }
                }
                if (MODE == MODE_GRAD) {
#pragma unroll
                    for (int j = 0; j < 7; ++j) gq[u][j] = fmaf(1.0f - us, gw[j], gq[u][j]);
                    if (s > 0 && t0 > 0) {
                        float *gp = ws.gs + (t0 - 1) * 7;
#pragma unroll
                        for (int j = 0; j < 7; ++j) gp[j] = fmaf(us, gw[j], gp[j]);
                    }
                }
            }
        }
    }
    if (MODE == MODE_GRAD) {
        // every lane is done with its frame scratch: restore the zero rows of es
        __syncwarp();
        for (int e = lane; e < kPad * 7 * 3; e += 32) ws.es[(e / (kPad * 7)) * R3 + T * 7 + e % (kPad * 7)] = 0.f;
    }
#pragma unroll(kRoll ? 1 : TPL)
    for (int u = 0; u < TPL; ++u) {
        const int t0 = lane + 32 * u;
        if (t0 < T) {
            const float *y = ws.xs + (t0 + kPad) * 7;   // y_t; y - 7 = y_{t-1}, ...
            float *gr = kRoll ? ws.gs + t0 * 7 : gq[kRoll ? 0 : u];
#pragma unroll
            for (int j = 0; j < 7; ++j) {
                const float y0 = y[j], y1 = y[j - 7], y2 = y[j - 14], y3 = y[j - 21];
                const float v = (y0 - y1) * inv_dt;
                const float a = (y0 - 2.0f * y1 + y2) * (inv_dt * inv_dt);
                const float jk = (y0 - 3.0f * y1 + 3.0f * y2 - y3) * (inv_dt * inv_dt * inv_dt);
                c_smooth += kc.w_v * v * v + kc.w_a * a * a + kc.w_j * jk * jk;
                const float hi = rb.hi[j], lo = rb.lo[j];
                float viol = 0.f;
                if (y0 > hi) {
                    viol = y0 - hi;
                    c_limit += kc.w_l * viol * viol;
                    if (MODE == MODE_GRAD) gr[j] += 2.0f * kc.w_l * viol;
                } else if (y0 < lo) {
                    viol = lo - y0;
                    c_limit += kc.w_l * viol * viol;
                    if (MODE == MODE_GRAD) gr[j] -= 2.0f * kc.w_l * viol;
                }
                if (MODE == MODE_EVAL) {
                    max_jerk = fmaxf(max_jerk, fabsf(jk));
                    lim_viol = fmaxf(lim_viol, viol);
                }
                if (MODE == MODE_GRAD) {
                    ws.es[t0 * 7 + j] = 2.0f * kc.w_v * v * inv_dt;
                    ws.es[R3 + t0 * 7 + j] = 2.0f * kc.w_a * a * (inv_dt * inv_dt);
                    ws.es[2 * R3 + t0 * 7 + j] = 2.0f * kc.w_j * jk * (inv_dt * inv_dt * inv_dt);
                }
            }
        }
    }
    if (MODE == MODE_GRAD) {
        __syncwarp();
        // transposed stencils: waypoint s receives e_v(s) - e_v(s+1),
        // e_a(s) - 2 e_a(s+1) + e_a(s+2), e_j(s) - 3 e_j(s+1) + 3 e_j(s+2) - e_j(s+3)
#pragma unroll(kRoll ? 1 : TPL)
        for (int u = 0; u < TPL; ++u) {
            const int t0 = lane + 32 * u;
            if (t0 < T) {
                const float *ev = ws.es + t0 * 7, *ea = ev + R3, *ej = ev + 2 * R3;
                const float *gr = kRoll ? ws.gs + t0 * 7 : gq[kRoll ? 0 : u];
#pragma unroll
                for (int j = 0; j < 7; ++j) {
                    float g = gr[j];
                    g += ev[j] - ev[j + 7];
                    g += ea[j] - 2.0f * ea[j + 7] + ea[j + 14];
                    g += ej[j] - 3.0f * ej[j + 7] + 3.0f * ej[j + 14] - ej[j + 21];
                    if (SWEEP) g += ws.gs[t0 * 7 + j];      // from the interpolants after waypoint t
                    ws.gs[t0 * 7 + j] = g;
                }
            }
        }
    }
    EvalOut o;
    o.cost = warp_sum(c_world + c_smooth + c_goal + c_limit);
    if (want_terms) {
        o.terms[0] = warp_sum(c_world);
        o.terms[1] = warp_sum(c_smooth);
        o.terms[2] = warp_sum(c_goal);
        o.terms[3] = warp_sum(c_limit);
    }
    if (MODE == MODE_EVAL) {
        o.min_clear = warp_min(min_clear);
        o.max_jerk = warp_max(max_jerk);
        o.lim_viol = warp_max(lim_viol);
        const int src = (T - 1) & 31;
        o.pos_err = __shfl_sync(0xffffffffu, pos_err, src);
        o.rot_err = __shfl_sync(0xffffffffu, rot_err, src);
    }
    return o;
}

// ----------------------------------------------------------------- L-BFGS
// Warp-uniform scalars of one seed's optimiser state.
struct LbUni {
    float f, alpha, gts;
    int hist, newest, first, accepts;
};

__device__ __forceinline__ int ring_prev(int k, int m) { return k == 0 ? m - 1 : k - 1; }
__device__ __forceinline__ int ring_next(int k, int m) { return k + 1 == m ? 0 : k + 1; }

// One L-BFGS update in the flat mapping (lane owns entries lane + 32 i of the
// n = 7T vector; NPL >= ceil(n / 32)), matching DseedOptParams: Armijo
// accept/reject of the trial point (xt, gt, ft), history push, the direction
// d = -H g by the two-loop recursion, and the next trial point into xt_next
// (may alias xt).  S, Y: this seed's history [m][n] in global memory, by ring
// slot; rho = 1 / s^T y per slot in ws.v[0..m), y^T y of the newest pair in
// ws.v[8]; the alphas of the first loop go to ws.v[16 + c].  The history is
// read from L2 in both loops, one round of loads per pair (s and y together),
// which leaves the registers to more resident warps.  After a rejected trial g
// and the history are unchanged, so the stored direction ws.dd is reused (the
// recursion would give the same numbers).
template <int NPL>
__device__ __forceinline__ void lbfgs_update(const KOpt &ko, int n, LbUni &st, const float *xt,
                                             const float *gt, float ft, const WarpSmem &ws,
                                             float *__restrict__ S, float *__restrict__ Y, float *xt_next) {
    const int lane = threadIdx.x & 31;
    const int m = ko.m;
    bool new_dir = false, accepted = false;
    if (st.first) {
        st.first = 0;
        accepted = true;
    } else if (ft <= st.f + ko.c1 * st.gts) {
        float sy = 0.f, ss = 0.f, yy = 0.f;
        float sv[NPL], yv[NPL];
#pragma unroll
        for (int i = 0; i < NPL; ++i) {
            const int e = lane + 32 * i;
            sv[i] = 0.f; yv[i] = 0.f;
            if (e < n) { sv[i] = xt[e] - ws.xa[e]; yv[i] = gt[e] - ws.ga[e]; }
            sy = fmaf(sv[i], yv[i], sy);
            ss = fmaf(sv[i], sv[i], ss);
            yy = fmaf(yv[i], yv[i], yy);
        }
        sy = warp_sum(sy);
        ss = warp_sum(ss);
        yy = warp_sum(yy);
        if (sy > 1e-10f * sqrtf(ss) * sqrtf(yy)) {
            const int k = st.newest < 0 ? 0 : ring_next(st.newest, m);
#pragma unroll
            for (int i = 0; i < NPL; ++i) {
                const int e = lane + 32 * i;
                if (e < n) { S[(size_t)k * n + e] = sv[i]; Y[(size_t)k * n + e] = yv[i]; }
            }
            if (lane == 0) { ws.v[k] = 1.0f / sy; ws.v[8] = yy; }
            st.newest = k;
            st.hist = min(st.hist + 1, m);
        }
        accepted = true;
        st.alpha = fminf(1.0f, 2.0f * st.alpha);
    } else {
        st.alpha *= 0.5f;
        if (st.alpha < ko.alpha_min) {
            st.hist = 0;
            st.newest = -1;
            st.alpha = 1.0f;
            new_dir = true;
        }
    }
    float gv[NPL];
#pragma unroll
    for (int i = 0; i < NPL; ++i) {
        const int e = lane + 32 * i;
        gv[i] = 0.f;
        if (e < n) {
            if (accepted) { ws.xa[e] = xt[e]; ws.ga[e] = gt[e]; gv[i] = gt[e]; }
            else gv[i] = ws.ga[e];
        }
    }
    if (accepted) {
        st.f = ft;
        st.accepts += 1;
        new_dir = true;
    }
    __syncwarp();
    if (new_dir) {
        // two-loop recursion: newest to oldest, then oldest to newest
        const int h = st.hist;
        float qv[NPL];
#pragma unroll
        for (int i = 0; i < NPL; ++i) qv[i] = gv[i];
        {
            int k = st.newest;
            for (int c = 0; c < h; ++c) {
                // both vectors of the pair in one round of loads (y is not needed
                // until the reduction of s^T q is in, but its latency overlaps it)
                const float *Sk = S + (size_t)k * n, *Yk = Y + (size_t)k * n;
                constexpr bool kPair = NPL <= 14;          // registers to spare for y
                float yk[kPair ? NPL : 1];
                float dot = 0.f;
#pragma unroll
                for (int i = 0; i < NPL; ++i) {
                    const int e = lane + 32 * i;
                    if (kPair) yk[kPair ? i : 0] = 0.f;
                    if (e < n) {
                        dot = fmaf(Sk[e], qv[i], dot);
                        if (kPair) yk[kPair ? i : 0] = Yk[e];
                    }
                }
                const float a = ws.v[k] * warp_sum(dot);
                if (lane == 0) ws.v[16 + c] = a;
#pragma unroll
                for (int i = 0; i < NPL; ++i) {
                    const int e = lane + 32 * i;
                    if (kPair) qv[i] = fmaf(-a, yk[kPair ? i : 0], qv[i]);
                    else if (e < n) qv[i] = fmaf(-a, Yk[e], qv[i]);
                }
                k = ring_prev(k, m);
            }
            __syncwarp();
            const float gamma = h > 0 ? (1.0f / ws.v[st.newest]) / ws.v[8] : ko.gamma0;
#pragma unroll
            for (int i = 0; i < NPL; ++i) qv[i] *= gamma;
            // k is now the slot before the oldest; walk forward again
            for (int c = h - 1; c >= 0; --c) {
                k = ring_next(k, m);
                const float *Sk = S + (size_t)k * n, *Yk = Y + (size_t)k * n;
                constexpr bool kPair = NPL <= 14;
                float sk[kPair ? NPL : 1];
                float dot = 0.f;
#pragma unroll
                for (int i = 0; i < NPL; ++i) {
                    const int e = lane + 32 * i;
                    if (kPair) sk[kPair ? i : 0] = 0.f;
                    if (e < n) {
                        dot = fmaf(Yk[e], qv[i], dot);
                        if (kPair) sk[kPair ? i : 0] = Sk[e];
                    }
                }
                const float cf = ws.v[16 + c] - ws.v[k] * warp_sum(dot);
#pragma unroll
                for (int i = 0; i < NPL; ++i) {
                    const int e = lane + 32 * i;
                    if (kPair) qv[i] = fmaf(cf, sk[kPair ? i : 0], qv[i]);
                    else if (e < n) qv[i] = fmaf(cf, Sk[e], qv[i]);
                }
            }
        }
        float gd = 0.f;
#pragma unroll
        for (int i = 0; i < NPL; ++i) gd = fmaf(gv[i], -qv[i], gd);
        gd = warp_sum(gd);
        const bool descent = gd < 0.0f;
#pragma unroll
        for (int i = 0; i < NPL; ++i) {
            const int e = lane + 32 * i;
            if (e < n) ws.dd[e] = descent ? -qv[i] : -gv[i];
        }
        __syncwarp();
    }
    // step = alpha d, scaled so that max |step| <= max_step; next trial point
    float dv[NPL], mx = 0.f;
#pragma unroll
    for (int i = 0; i < NPL; ++i) {
        const int e = lane + 32 * i;
        dv[i] = e < n ? ws.dd[e] : 0.f;
        mx = fmaxf(mx, fabsf(st.alpha * dv[i]));
    }
    mx = warp_max(mx);
    const float scale = mx > ko.max_step ? ko.max_step / mx : 1.0f;
    float gts = 0.f;
#pragma unroll
    for (int i = 0; i < NPL; ++i) {
        const int e = lane + 32 * i;
        const float step = st.alpha * dv[i] * scale;
        if (e < n) xt_next[e] = ws.xa[e] + step;
        gts = fmaf(gv[i], step, gts);
    }
    st.gts = warp_sum(gts);
    __syncwarp();
}

}  // namespace dseed
