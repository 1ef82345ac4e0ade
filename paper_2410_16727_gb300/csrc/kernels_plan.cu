// kernels_plan.cu -- batched L-BFGS (standalone step) and the fused optimiser.
//
// The fused optimiser runs every iteration of one seed inside one warp: the
// trial point, its gradient, the accepted point and the smoothness adjoint
// stay in the warp's shared memory, the (s, y) history in the workspace (hot
// in L2: only resident warps touch theirs), and the only HBM traffic per
// iteration is whatever the ESDF gathers miss in L1/L2.  Seeds are
// independent, so no warp ever waits on another.
#include <cuda_runtime.h>

#include <type_traits>

#include "device.cuh"

namespace dseed {

#ifndef DSEED_PLAN_WARPS
#define DSEED_PLAN_WARPS 4
#endif
#ifndef DSEED_PLAN_MINBLOCKS
#define DSEED_PLAN_MINBLOCKS 5
#endif
constexpr int kPlanWarps = DSEED_PLAN_WARPS;    // warps per block of the standalone L-BFGS step
// Block shape of the fused plan.  A T <= 32 plan fits 96 registers without
// spills, so five blocks of four warps stay resident (shared memory would allow
// six, but the 80-register build is slower).  Longer horizons and the
// self-collision scratch are limited by shared memory per warp: two-warp blocks
// pack it more finely (T = 64: 14 resident warps instead of 12), and the
// minimum-block counts below leave each variant at least the registers it uses.
__host__ __device__ constexpr int plan_warps(int tpl, bool self) { return tpl == 1 && !self ? kPlanWarps : 2; }
// With several waypoints per lane (and no self term) the search direction lives
// in the workspace instead of shared memory: it is read once per iteration, and
// the 7 T floats it frees let more warps stay resident (T = 64: 16 instead of 14).
__host__ __device__ constexpr bool plan_dd_global(int tpl, bool self) { return tpl >= 2 && !self; }
__host__ __device__ constexpr int plan_min_blocks(int tpl, bool self) {
    return tpl == 1 && !self ? DSEED_PLAN_MINBLOCKS : self ? (tpl == 1 ? 5 : tpl == 2 ? 3 : 2) : (tpl == 2 ? 8 : 4);
}
__host__ __device__ constexpr int plan_warp_floats(int T, int tpl, bool self) {
    return plan_dd_global(tpl, self) ? warp_smem_floats_nodd(T, self) : warp_smem_floats(T, self);
}

// ---------------------------------------------------------------- standalone L-BFGS
__global__ void k_lbfgs_init(long long B, int n, int m, const float *__restrict__ x0, KLbfgsPtrs p) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < B * n) p.x_trial[i] = x0[i];
    if (i < B) {
        p.f[i] = CUDART_INF_F;
        p.alpha[i] = 1.0f;
        p.gts[i] = 0.0f;
        p.meta[i * 4 + 0] = 0;    // history count
        p.meta[i * 4 + 1] = -1;   // newest slot
        p.meta[i * 4 + 2] = 1;    // first evaluation pending
        p.meta[i * 4 + 3] = 0;    // accepts
    }
}

template <int NPL>
__global__ void __launch_bounds__(kPlanWarps * 32)
    k_lbfgs_step(const __grid_constant__ KOpt ko, long long B, int T, const float *__restrict__ f_trial,
                 const float *__restrict__ g_trial, KLbfgsPtrs p) {
    extern __shared__ float smem[];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long b = (long long)blockIdx.x * kPlanWarps + wid;
    if (b >= B) return;
    const int n = 7 * T, m = ko.m;
    WarpSmem ws = carve(smem + wid * warp_smem_floats(T), T);
    float *xt = ws.xs + kPad * 7;
    for (int e = lane; e < n; e += 32) {
        xt[e] = p.x_trial[b * n + e];
        ws.gs[e] = g_trial[b * n + e];
        ws.xa[e] = p.x[b * n + e];
        ws.ga[e] = p.g[b * n + e];
        ws.dd[e] = p.d[b * n + e];
    }
    if (lane < 8) ws.v[lane] = p.rho[b * 8 + lane];
    if (lane == 8) ws.v[8] = p.yy[b];
    LbUni st;
    st.f = p.f[b];
    st.alpha = p.alpha[b];
    st.gts = p.gts[b];
    st.hist = p.meta[b * 4 + 0];
    st.newest = p.meta[b * 4 + 1];
    st.first = p.meta[b * 4 + 2];
    st.accepts = p.meta[b * 4 + 3];
    __syncwarp();
    lbfgs_update<NPL>(ko, n, st, xt, ws.gs, f_trial[b], ws, p.s + (size_t)b * m * n, p.y + (size_t)b * m * n, xt);
    for (int e = lane; e < n; e += 32) {
        p.x_trial[b * n + e] = xt[e];
        p.x[b * n + e] = ws.xa[e];
        p.g[b * n + e] = ws.ga[e];
        p.d[b * n + e] = ws.dd[e];
    }
    if (lane < 8) p.rho[b * 8 + lane] = ws.v[lane];
    if (lane == 8) p.yy[b] = ws.v[8];
    if (lane == 0) {
        p.f[b] = st.f;
        p.alpha[b] = st.alpha;
        p.gts[b] = st.gts;
        p.meta[b * 4 + 0] = st.hist;
        p.meta[b * 4 + 1] = st.newest;
        p.meta[b * 4 + 2] = st.first;
        p.meta[b * 4 + 3] = st.accepts;
    }
}

// ---------------------------------------------------------------- fused optimiser
// Drop a seed's dead L-BFGS history from L2 without writing it back to HBM:
// once the seed's last update is done nothing reads the pairs again, and a
// write-back would only cost DRAM traffic.  Only the 128-byte lines lying
// wholly inside [base, base + nfloats) are dropped; a line shared with a
// neighbouring seed's region may still be live and is left alone.
__device__ __forceinline__ void discard_dead_lines(const float *base, size_t nfloats) {
    const int lane = threadIdx.x & 31;
    const uintptr_t a = reinterpret_cast<uintptr_t>(base), e = a + nfloats * sizeof(float);
    const uintptr_t first = (a + 127) & ~static_cast<uintptr_t>(127), last = e & ~static_cast<uintptr_t>(127);
    for (uintptr_t l = first + (uintptr_t)lane * 128; l < last; l += 32 * 128)
        asm volatile("discard.global.L2 [%0], 128;" ::"l"(__cvta_generic_to_global(reinterpret_cast<const void *>(l)))
                     : "memory");
}

// Per warp: load seed -> iters x (cost+adjoint of the trial point, L-BFGS
// update) -> success test of the accepted point -> outputs.  best_key[p] holds
// (cost bits << 32 | seed) of the best successful seed (costs are >= 0, so
// their bit patterns order like the values); it must start at ~0.
template <int TPL, bool SELF, bool SWEEP>
__global__ void __launch_bounds__(plan_warps(TPL, SELF) * 32, plan_min_blocks(TPL, SELF))
    k_plan(const __grid_constant__ KRobot rb, const __grid_constant__ KCost kc, const __grid_constant__ KOpt ko,
           const __grid_constant__ KBatch kb, const float *seeds, float *__restrict__ hist_s,
           float *__restrict__ hist_y, float *__restrict__ dirs, unsigned long long *__restrict__ best_key,
           float *traj, float *__restrict__ cost, uint8_t *__restrict__ success, float *__restrict__ metrics) {
    constexpr int NPL = 7 * TPL;
    extern __shared__ float smem[];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long B = (long long)kb.P * kb.S;
    const long long b = (long long)blockIdx.x * plan_warps(TPL, SELF) + wid;
    if (b >= B) return;
    const int T = kb.T, n = 7 * T, m = ko.m;
    const int p = (int)(b / kb.S);
    constexpr bool kDdGlobal = plan_dd_global(TPL, SELF);
    WarpSmem ws = carve(smem + wid * plan_warp_floats(T, TPL, SELF), T, kDdGlobal ? dirs + (size_t)b * n : nullptr);
    float *xt = ws.xs + kPad * 7;
    const int si = kb.scene_of_problem[p];
    const bool in_table = si >= 0 && si < kb.n_scenes;
    if (!in_table || !load_scene(kb.scenes, si).ok) {
        for (int e = lane; e < n; e += 32) traj[b * n + e] = seeds[b * n + e];
        if (lane == 0) {
            cost[b] = CUDART_NAN_F;
            success[b] = 0;
            if (metrics)
                for (int i = 0; i < DSEED_N_METRICS; ++i) metrics[b * DSEED_N_METRICS + i] = CUDART_NAN_F;
        }
        return;
    }
    const int R3 = (T + kPad) * 7;
    for (int e = lane; e < kPad * 7; e += 32) {
        ws.xs[e] = kb.q_start[(size_t)p * 7 + e % 7];
        ws.es[T * 7 + e] = 0.f;
        ws.es[R3 + T * 7 + e] = 0.f;
        ws.es[2 * R3 + T * 7 + e] = 0.f;
    }
    // plain loads: traj may alias seeds (each warp reads its own seed before writing it)
    for (int e = lane; e < n; e += 32) xt[e] = seeds[b * n + e];
    const Goal G = make_goal(kb.goal + (size_t)p * 7);
    const SceneView sv = load_scene(kb.scenes, si);
    float *S = hist_s + (size_t)b * m * n, *Y = hist_y + (size_t)b * m * n;
    LbUni st{CUDART_INF_F, 1.0f, 0.0f, 0, -1, 1, 0};
    __syncwarp();
    for (int it = 0; it < ko.iters; ++it) {
        const EvalOut o = warp_eval<TPL, MODE_GRAD, SELF, SWEEP>(rb, kc, sv, T, G, ws, false);
        __syncwarp();
        lbfgs_update<NPL>(ko, n, st, xt, ws.gs, o.cost, ws, S, Y, xt);
    }
    // every lane's history stores are done before its lines are dropped
    __syncwarp();
    discard_dead_lines(S, (size_t)m * n);
    discard_dead_lines(Y, (size_t)m * n);
    // success test of the accepted point
    for (int e = lane; e < n; e += 32) xt[e] = ws.xa[e];
    __syncwarp();
    const EvalOut o = warp_eval<TPL, MODE_EVAL, SELF, SWEEP>(rb, kc, sv, T, G, ws, false);
    for (int e = lane; e < n; e += 32) traj[b * n + e] = ws.xa[e];
    const bool free = o.min_clear >= 0.0f;
    const bool ok = free && o.pos_err < kb.delta_t && o.rot_err < kb.delta_r && o.lim_viol == 0.0f;
    if (lane == 0) {
        cost[b] = st.f;
        success[b] = ok ? 1 : 0;
        if (metrics) {
            float *mt = metrics + b * DSEED_N_METRICS;
            mt[0] = o.min_clear; mt[1] = o.pos_err; mt[2] = o.rot_err; mt[3] = o.max_jerk;
            mt[4] = o.lim_viol; mt[5] = o.cost; mt[6] = free ? 1.0f : 0.0f;
        }
        if (ok && st.f >= 0.0f) {
            const unsigned long long key =
                ((unsigned long long)__float_as_uint(st.f) << 32) | (unsigned long long)(unsigned)(b - (long long)p * kb.S);
            atomicMin(best_key + p, key);
        }
    }
}

__global__ void k_best(int P, const unsigned long long *__restrict__ key, int *__restrict__ best) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < P) best[p] = key[p] == ~0ull ? -1 : (int)(key[p] & 0xffffffffull);
}

static size_t plan_smem_bytes(int T, bool self = false, int warps = kPlanWarps) {
    return (size_t)warps * warp_smem_floats(T, self) * sizeof(float);
}
static size_t fused_plan_smem_bytes(int T, int tpl, bool self, int warps) {
    return (size_t)warps * plan_warp_floats(T, tpl, self) * sizeof(float);
}

template <typename K>
static int set_smem(K kern, size_t smem) {
    if (smem > 48 * 1024)
        return (int)cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return cudaSuccess;
}

int launch_lbfgs_init(int B, int n, const float *x0, const KLbfgsPtrs &p, int m, cudaStream_t st) {
    const long long total = (long long)B * n;
    if (total == 0) return cudaSuccess;
    k_lbfgs_init<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(B, n, m, x0, p);
    return (int)cudaGetLastError();
}

int launch_lbfgs_step(const KOpt &ko, int B, int T, const float *f_trial, const float *g_trial,
                      const KLbfgsPtrs &p, cudaStream_t st) {
    if (B == 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((B + kPlanWarps - 1) / kPlanWarps);
    const size_t smem = plan_smem_bytes(T);
    auto go = [&](auto kern) {
        int e = set_smem(kern, smem);
        if (e) return e;
        kern<<<blocks, kPlanWarps * 32, smem, st>>>(ko, (long long)B, T, f_trial, g_trial, p);
        return (int)cudaGetLastError();
    };
    if (T <= 32) return go(k_lbfgs_step<7>);
    if (T <= 64) return go(k_lbfgs_step<14>);
    return go(k_lbfgs_step<28>);
}

int launch_plan(const KRobot &rb, const KCost &kc, const KOpt &ko, const KBatch &kb, const float *seeds,
                float *hist_s, float *hist_y, float *dirs, unsigned long long *best_key, float *traj, float *cost,
                uint8_t *success, float *metrics, int *best, cudaStream_t st) {
    if (kb.P == 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(best_key, 0xff, sizeof(unsigned long long) * kb.P, st);
    if (e != cudaSuccess) return (int)e;
    const long long B = (long long)kb.P * kb.S;
    const bool self = kc.w_s > 0.f;
    const int tpl = kb.T <= 32 ? 1 : kb.T <= 64 ? 2 : 4;
    const int warps = self ? plan_warps(tpl, true) : plan_warps(tpl, false);
    const unsigned blocks = (unsigned)((B + warps - 1) / warps);
    const size_t smem = fused_plan_smem_bytes(kb.T, tpl, self, warps);
    auto go = [&](auto kern) {
        int r = set_smem(kern, smem);
        if (r) return r;
        kern<<<blocks, warps * 32, smem, st>>>(rb, kc, ko, kb, seeds, hist_s, hist_y, dirs, best_key, traj, cost,
                                               success, metrics);
        return (int)cudaGetLastError();
    };
    // variants: waypoints per lane x self-collision term x swept check
    auto by_t = [&](auto self_c, auto sweep_c) {
        constexpr bool kSelf = decltype(self_c)::value, kSweep = decltype(sweep_c)::value;
        if (kb.T <= 32) return go(k_plan<1, kSelf, kSweep>);
        if (kb.T <= 64) return go(k_plan<2, kSelf, kSweep>);
        return go(k_plan<4, kSelf, kSweep>);
    };
    using T_ = std::true_type;
    using F_ = std::false_type;
    const bool sweep = kc.n_sweep > 0;
    const int r = self ? (sweep ? by_t(T_{}, T_{}) : by_t(T_{}, F_{})) : (sweep ? by_t(F_{}, T_{}) : by_t(F_{}, F_{}));
    if (r) return r;
    k_best<<<(kb.P + 127) / 128, 128, 0, st>>>(kb.P, best_key, best);
    return (int)cudaGetLastError();
}

}  // namespace dseed
