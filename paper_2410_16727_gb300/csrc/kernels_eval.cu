// kernels_eval.cu -- forward kinematics, cost, cost+adjoint and evaluation kernels.
#include <cuda_runtime.h>

#include <type_traits>

#include "device.cuh"

namespace dseed {

constexpr int kWarpsPerBlock = 4;

// ---------------------------------------------------------------- FK
// One thread per configuration: flange pose (position from the matrix chain,
// orientation from the chained half-angle quaternions qx(alpha) qz(theta)) and
// optionally every sphere centre in the caller's sphere order.
__global__ void __launch_bounds__(128) k_fk(const __grid_constant__ KRobot rb, const float *__restrict__ q,
                                            int N, float *__restrict__ pose, float *__restrict__ spheres) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    float R[9] = {1.f, 0.f, 0.f, 0.f, 1.f, 0.f, 0.f, 0.f, 1.f};
    float p[3] = {0.f, 0.f, 0.f};
    float qw = 1.f, qx = 0.f, qy = 0.f, qz = 0.f;
    for (int L = 1; L <= 8; ++L) {
        float th = rb.off[L - 1] + (L <= 7 ? q[(size_t)i * 7 + L - 1] : 0.0f);
        float st, ct, sh, ch;
        sincosf(th, &st, &ct);
        sincosf(0.5f * th, &sh, &ch);
        dh_step(R, p, rb.a[L - 1], rb.d[L - 1], rb.ca[L - 1], rb.sa[L - 1], ct, st);
        // q <- q (x) (ca2, sa2, 0, 0)
        const float c2 = rb.ca2[L - 1], s2 = rb.sa2[L - 1];
        float w1 = qw * c2 - qx * s2, x1 = qw * s2 + qx * c2, y1 = qy * c2 + qz * s2, z1 = qz * c2 - qy * s2;
        // q <- q (x) (ch, 0, 0, sh)
        qw = w1 * ch - z1 * sh;
        qx = x1 * ch + y1 * sh;
        qy = y1 * ch - x1 * sh;
        qz = z1 * ch + w1 * sh;
        if (spheres) {
            for (int k = rb.frame_begin[L - 1]; k < rb.frame_begin[L]; ++k) {
                const float4 s = rb.sph[k];
                float *c = spheres + ((size_t)i * rb.n_spheres + rb.sph_orig[k]) * 3;
                c[0] = fmaf(R[0], s.x, fmaf(R[1], s.y, fmaf(R[2], s.z, p[0])));
                c[1] = fmaf(R[3], s.x, fmaf(R[4], s.y, fmaf(R[5], s.z, p[1])));
                c[2] = fmaf(R[6], s.x, fmaf(R[7], s.y, fmaf(R[8], s.z, p[2])));
            }
        }
    }
    const float inv = rsqrtf(qw * qw + qx * qx + qy * qy + qz * qz) * (qw < 0.f ? -1.f : 1.f);
    float *o = pose + (size_t)i * 7;
    o[0] = p[0]; o[1] = p[1]; o[2] = p[2];
    o[3] = qw * inv; o[4] = qx * inv; o[5] = qy * inv; o[6] = qz * inv;
}

// ---------------------------------------------------------------- cost / grad / evaluate
// One warp per trajectory.  A problem whose scene index is out of range, or
// whose scene descriptor is unusable, gets a NaN cost, NaN gradient and no
// success (and no memory outside the inputs is touched).
template <int TPL, int MODE, bool SELF, bool SWEEP>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
    k_eval(const __grid_constant__ KRobot rb, const __grid_constant__ KCost kc, const __grid_constant__ KBatch kb,
           const float *__restrict__ x, const float *__restrict__ grad_scale, float *__restrict__ cost,
           float *__restrict__ terms, float *__restrict__ grad, uint8_t *__restrict__ success,
           float *__restrict__ metrics) {
    extern __shared__ float smem[];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long B = (long long)kb.P * kb.S;
    const long long b = (long long)blockIdx.x * kWarpsPerBlock + wid;
    if (b >= B) return;
    const int T = kb.T, n = 7 * T;
    const int p = (int)(b / kb.S);
    WarpSmem ws = carve(smem + wid * warp_smem_floats(T, SELF), T);
    const int si = kb.scene_of_problem[p];
    const bool in_table = si >= 0 && si < kb.n_scenes;
    if (!in_table || !load_scene(kb.scenes, si).ok) {
        if (lane == 0) {
            if (cost) cost[b] = CUDART_NAN_F;
            if (success) success[b] = 0;
        }
        if (MODE == MODE_GRAD)
            for (int e = lane; e < n; e += 32) grad[b * n + e] = CUDART_NAN_F;
        return;
    }
    for (int e = lane; e < kPad * 7; e += 32) ws.xs[e] = kb.q_start[(size_t)p * 7 + e % 7];
    const float *xb = x + b * n;
    for (int e = lane; e < n; e += 32) ws.xs[kPad * 7 + e] = __ldg(xb + e);
    if (MODE == MODE_GRAD) {
        const int R3 = (T + kPad) * 7;
        for (int e = lane; e < kPad * 7; e += 32) {
            ws.es[T * 7 + e] = 0.f;
            ws.es[R3 + T * 7 + e] = 0.f;
            ws.es[2 * R3 + T * 7 + e] = 0.f;
        }
    }
    const Goal G = make_goal(kb.goal + (size_t)p * 7);
    const SceneView sv = load_scene(kb.scenes, si);
    __syncwarp();
    const EvalOut o = warp_eval<TPL, MODE, SELF, SWEEP>(rb, kc, sv, T, G, ws, terms != nullptr);
    __syncwarp();
    if (lane == 0) {
        if (cost) cost[b] = o.cost;
        if (terms)
            for (int i = 0; i < 4; ++i) terms[b * 4 + i] = o.terms[i];
    }
    if (MODE == MODE_GRAD) {
        const float sc = grad_scale ? grad_scale[b] : 1.0f;
        for (int e = lane; e < n; e += 32) grad[b * n + e] = ws.gs[e] * sc;
    }
    if (MODE == MODE_EVAL && lane == 0) {
        const bool free = o.min_clear >= 0.0f;
        const bool ok = free && o.pos_err < kb.delta_t && o.rot_err < kb.delta_r && o.lim_viol == 0.0f;
        success[b] = ok ? 1 : 0;
        if (metrics) {
            float *m = metrics + b * DSEED_N_METRICS;
            m[0] = o.min_clear; m[1] = o.pos_err; m[2] = o.rot_err; m[3] = o.max_jerk;
            m[4] = o.lim_viol; m[5] = o.cost; m[6] = free ? 1.0f : 0.0f;
        }
    }
}

static size_t eval_smem_bytes(int T, bool self) {
    return (size_t)kWarpsPerBlock * warp_smem_floats(T, self) * sizeof(float);
}

template <int MODE>
static int launch_eval_mode(const KRobot &rb, const KCost &kc, const KBatch &kb, const float *x,
                            const float *grad_scale, float *cost, float *terms, float *grad, uint8_t *success,
                            float *metrics, cudaStream_t st) {
    const long long B = (long long)kb.P * kb.S;
    if (B == 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((B + kWarpsPerBlock - 1) / kWarpsPerBlock);
    const bool self = kc.w_s > 0.f;
    const size_t smem = eval_smem_bytes(kb.T, self);
    auto go = [&](auto kern) {
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return (int)e;
        }
        kern<<<blocks, kWarpsPerBlock * 32, smem, st>>>(rb, kc, kb, x, grad_scale, cost, terms, grad, success, metrics);
        return (int)cudaGetLastError();
    };
    // variants: waypoints per lane x self-collision term x swept check
    auto by_t = [&](auto self_c, auto sweep_c) {
        constexpr bool kSelf = decltype(self_c)::value, kSweep = decltype(sweep_c)::value;
        if (kb.T <= 32) return go(k_eval<1, MODE, kSelf, kSweep>);
        if (kb.T <= 64) return go(k_eval<2, MODE, kSelf, kSweep>);
        return go(k_eval<4, MODE, kSelf, kSweep>);
    };
    using T_ = std::true_type;
    using F_ = std::false_type;
    const bool sweep = kc.n_sweep > 0;
    return self ? (sweep ? by_t(T_{}, T_{}) : by_t(T_{}, F_{})) : (sweep ? by_t(F_{}, T_{}) : by_t(F_{}, F_{}));
}

int launch_cost(const KRobot &rb, const KCost &kc, const KBatch &kb, const float *x, float *cost, float *terms,
                cudaStream_t st) {
    return launch_eval_mode<MODE_COST>(rb, kc, kb, x, nullptr, cost, terms, nullptr, nullptr, nullptr, st);
}

int launch_cost_grad(const KRobot &rb, const KCost &kc, const KBatch &kb, const float *x, const float *grad_scale,
                     float *cost, float *grad, cudaStream_t st) {
    return launch_eval_mode<MODE_GRAD>(rb, kc, kb, x, grad_scale, cost, nullptr, grad, nullptr, nullptr, st);
}

int launch_evaluate(const KRobot &rb, const KCost &kc, const KBatch &kb, const float *x, uint8_t *success,
                    float *metrics, cudaStream_t st) {
    return launch_eval_mode<MODE_EVAL>(rb, kc, kb, x, nullptr, nullptr, nullptr, nullptr, success, metrics, st);
}

int launch_fk(const KRobot &rb, const float *q, int N, float *pose, float *spheres, cudaStream_t st) {
    if (N == 0) return cudaSuccess;
    k_fk<<<(N + 127) / 128, 128, 0, st>>>(rb, q, N, pose, spheres);
    return (int)cudaGetLastError();
}

// ---------------------------------------------------------------- Eq. 2 in the workspace
// One thread per (trajectory, waypoint).  The drawn noise eps and the predicted
// noise pred stand for the joint configurations q(v) = mid + half (lin + v / res)
// (lin: the normalised straight start-goal path; mid, half: centre and
// half-width of each joint's limits); both are placed by the kinematic chain
// and the squared distances between the predicted and the drawn points on the
// robot (on each collision sphere's surface, at the six axis directions of its
// frame: c_k + r_k u in frame coordinates) are summed, weighted per trajectory.
// The derivative with respect to pred runs back through the predicted chain by
// Jacobian-transpose accumulation: each point pushes with g = dloss/dc at its
// predicted position, joint i receives z_i . (M - M_<i) - (z_i x p_i) . (F -
// F_<i) with F, M the sum of the pushes and of their moments about the origin
// (the _<i parts are the points met before frame i), times half / res.
__global__ void __launch_bounds__(256) k_fk_mse(const __grid_constant__ KRobot rb, const float *__restrict__ lin,
                                                const float *__restrict__ eps, const float *__restrict__ pred,
                                                const float *__restrict__ w, int N, int T, float inv_res,
                                                float inv_norm, float *__restrict__ dpred,
                                                float *__restrict__ loss_partial) {
    __shared__ float red[256];
    float acc = 0.f;
    const long long total = (long long)N * T;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const float wn = w ? w[i / T] : 1.f;
        const float *li = lin + i * 7, *ei = eps + i * 7, *pi = pred + i * 7;
        float Rl[9] = {1.f, 0.f, 0.f, 0.f, 1.f, 0.f, 0.f, 0.f, 1.f}, pl[3] = {0.f, 0.f, 0.f};
        float Rp[9] = {1.f, 0.f, 0.f, 0.f, 1.f, 0.f, 0.f, 0.f, 1.f}, pp[3] = {0.f, 0.f, 0.f};
        float zj[7][3], wj[7][3], bj[7];
        float Fx = 0.f, Fy = 0.f, Fz = 0.f, Mx = 0.f, My = 0.f, Mz = 0.f, dsum = 0.f;
        const float gs = 2.f * wn * inv_norm;
#pragma unroll
        for (int L = 1; L <= 8; ++L) {
            float stl, ctl, stp, ctp;
            if (L <= 7) {
                const int j = L - 1;
                const float mid = 0.5f * (rb.hi[j] + rb.lo[j]), half = 0.5f * (rb.hi[j] - rb.lo[j]);
                sincosf(fmaf(half, fmaf(ei[j], inv_res, li[j]), mid) + rb.off[j], &stl, &ctl);
                sincosf(fmaf(half, fmaf(pi[j], inv_res, li[j]), mid) + rb.off[j], &stp, &ctp);
            } else {
                stl = stp = rb.sf8;
                ctl = ctp = rb.cf8;
            }
            dh_step(Rl, pl, rb.a[L - 1], rb.d[L - 1], rb.ca[L - 1], rb.sa[L - 1], ctl, stl);
            dh_step(Rp, pp, rb.a[L - 1], rb.d[L - 1], rb.ca[L - 1], rb.sa[L - 1], ctp, stp);
            if (L <= 7) {
                const int j = L - 1;
                zj[j][0] = Rp[2]; zj[j][1] = Rp[5]; zj[j][2] = Rp[8];
                wj[j][0] = Rp[5] * pp[2] - Rp[8] * pp[1];
                wj[j][1] = Rp[8] * pp[0] - Rp[2] * pp[2];
                wj[j][2] = Rp[2] * pp[1] - Rp[5] * pp[0];
                bj[j] = (zj[j][0] * Mx + zj[j][1] * My + zj[j][2] * Mz) - (wj[j][0] * Fx + wj[j][1] * Fy + wj[j][2] * Fz);
            }
            for (int k = rb.frame_begin[L - 1]; k < rb.frame_begin[L]; ++k)
#pragma unroll 1
                for (int u = 0; u < 6; ++u) {
                    // the point on sphere k's surface along axis u / 2 of its frame, sign by u % 2
                    const float4 sk = rb.sph[k];
                    const float sgn = (u & 1) ? -sk.w : sk.w;
                    const float ox = sk.x + (u >> 1 == 0 ? sgn : 0.f);
                    const float oy = sk.y + (u >> 1 == 1 ? sgn : 0.f);
                    const float oz = sk.z + (u >> 1 == 2 ? sgn : 0.f);
                    const float cx = fmaf(Rp[0], ox, fmaf(Rp[1], oy, fmaf(Rp[2], oz, pp[0])));
                    const float cy = fmaf(Rp[3], ox, fmaf(Rp[4], oy, fmaf(Rp[5], oz, pp[1])));
                    const float cz = fmaf(Rp[6], ox, fmaf(Rp[7], oy, fmaf(Rp[8], oz, pp[2])));
                    const float dx = cx - fmaf(Rl[0], ox, fmaf(Rl[1], oy, fmaf(Rl[2], oz, pl[0])));
                    const float dy = cy - fmaf(Rl[3], ox, fmaf(Rl[4], oy, fmaf(Rl[5], oz, pl[1])));
                    const float dz = cz - fmaf(Rl[6], ox, fmaf(Rl[7], oy, fmaf(Rl[8], oz, pl[2])));
                    dsum += dx * dx + dy * dy + dz * dz;
                    const float gx = gs * dx, gy = gs * dy, gz = gs * dz;
                    Fx += gx; Fy += gy; Fz += gz;
                    Mx += cy * gz - cz * gy;
                    My += cz * gx - cx * gz;
                    Mz += cx * gy - cy * gx;
                }
        }
        acc = fmaf(wn, dsum, acc);
#pragma unroll
        for (int j = 0; j < 7; ++j) {
            const float half = 0.5f * (rb.hi[j] - rb.lo[j]);
            const float gq = (zj[j][0] * Mx + zj[j][1] * My + zj[j][2] * Mz) -
                             (wj[j][0] * Fx + wj[j][1] * Fy + wj[j][2] * Fz) - bj[j];
            dpred[i * 7 + j] = gq * half * inv_res;
        }
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) loss_partial[blockIdx.x] = red[0] * inv_norm;
}

int launch_fk_mse(const KRobot &rb, const float *lin, const float *eps, const float *pred, const float *w, int N,
                  int T, float res_scale, float *dpred, float *loss_partial, int blocks, cudaStream_t st) {
    const double norm = (double)N * T * rb.n_spheres * 6.0 * 3.0;     // six surface points per sphere
    const float inv_norm = norm > 0.0 ? (float)(1.0 / norm) : 0.f;
    k_fk_mse<<<blocks, 256, 0, st>>>(rb, lin, eps, pred, w, N, T, (float)(1.0 / (double)res_scale), inv_norm, dpred,
                                     loss_partial);
    return (int)cudaGetLastError();
}

}  // namespace dseed
