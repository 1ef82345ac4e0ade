// kernels_serve.cu -- resumable fused optimiser for the serving loop.
//
// A serving round runs every active request for up to K iterations in one
// launch per waypoint class (T <= 32, <= 64, <= 128).  Warp w finds its
// request by binary search over the round's table and its seed as the offset
// inside it.  The optimiser state of each seed (trial point, accepted point,
// gradient, direction, scalars, history) lives in the request's region of the
// serving arena between rounds, so a seed computes exactly what the one-shot
// plan computes for it, whichever requests share its rounds.
#include <cuda_runtime.h>

#include <type_traits>

#include "device.cuh"

namespace dseed {

#ifndef DSEED_SERVE_MINBLOCKS
#define DSEED_SERVE_MINBLOCKS 4
#endif
#ifndef DSEED_SERVE_MINBLOCKS_T32
#define DSEED_SERVE_MINBLOCKS_T32 5
#endif
constexpr int kServeWarps = 4;

// Resident blocks the registers are sized for: five (96 registers) for T <= 32
// without the swept check, whose round fits them with a few spilled bytes;
// four (128) otherwise, where the round's bookkeeping would spill more; with the
// self-collision term (its pair loops and the per-lane frame transforms in shared
// memory) shared memory limits the blocks, so the registers are left free.
// With several waypoints per lane (and no self term) the search direction stays
// in the request's arena region instead of shared memory, as in the one-shot
// plan: two-warp blocks, sixteen resident warps at T <= 64 instead of twelve.
constexpr bool serve_dd_global(int tpl, bool self) { return tpl >= 2 && !self; }
constexpr int serve_warps(int tpl, bool self) { return serve_dd_global(tpl, self) ? 2 : kServeWarps; }
constexpr int serve_min_blocks(int tpl, bool self, bool sweep) {
    return self ? 1 : serve_dd_global(tpl, self) ? (tpl == 2 ? 8 : 4)
                    : (tpl == 1 && !sweep) ? DSEED_SERVE_MINBLOCKS_T32 : DSEED_SERVE_MINBLOCKS;
}
constexpr int serve_warp_floats(int tpl, bool self) {
    return serve_dd_global(tpl, self) ? warp_smem_floats_nodd(32 * tpl, self) : warp_smem_floats(32 * tpl, self);
}

template <int TPL, bool SELF, bool SWEEP>
__global__ void __launch_bounds__(serve_warps(TPL, SELF) * 32, serve_min_blocks(TPL, SELF, SWEEP))
    k_serve(const __grid_constant__ KRobot rb, const __grid_constant__ KCost kc, const __grid_constant__ KOpt ko,
            float delta_t, float delta_r, const ServeEntry *__restrict__ table, int n_entries, long long total_warps) {
    constexpr int NPL = 7 * TPL;
    extern __shared__ float smem[];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr bool kDdGlobal = serve_dd_global(TPL, SELF);
    const long long w = (long long)blockIdx.x * serve_warps(TPL, SELF) + wid;
    if (w >= total_warps) return;
    int lo = 0, hi = n_entries - 1;                 // last entry with warp_begin <= w
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (table[mid].warp_begin <= w) lo = mid; else hi = mid - 1;
    }
    const ServeEntry &E = table[lo];
    const int s = (int)(w - E.warp_begin);
    const int T = E.T, n = 7 * T, m = ko.m;
    if (s < 0 || s >= E.S || T > 32 * TPL) return;
    const ServeLayout L = serve_layout(E.S, T, m);
    float *R = E.region;
    float *g_xt = R + L.xt + (size_t)s * n, *g_xa = R + L.xa + (size_t)s * n;
    float *g_ga = R + L.ga + (size_t)s * n, *g_dd = R + L.dd + (size_t)s * n;
    float *S_ = R + L.hs + (size_t)s * m * n, *Y_ = R + L.hy + (size_t)s * m * n;
    float *sc = R + L.sc + (size_t)s * 16;
    WarpSmem ws = carve(smem + wid * serve_warp_floats(TPL, SELF), T, kDdGlobal ? g_dd : nullptr);
    float *xt = ws.xs + kPad * 7;
    SceneView sv;
    {
        DseedScene one = E.scene;
        sv = load_scene(&one, 0);
    }
    if (!sv.ok) {
        if (E.final_round && lane == 0) {
            R[L.cost + s] = CUDART_NAN_F;
            reinterpret_cast<uint8_t *>(R + L.succ)[s] = 0;
        }
        return;
    }
    const int R3 = (T + kPad) * 7;
    for (int e = lane; e < kPad * 7; e += 32) {
        ws.xs[e] = R[L.qs + e % 7];
        ws.es[T * 7 + e] = 0.f;
        ws.es[R3 + T * 7 + e] = 0.f;
        ws.es[2 * R3 + T * 7 + e] = 0.f;
    }
    LbUni st{CUDART_INF_F, 1.0f, 0.0f, 0, -1, 1, 0};
    for (int e = lane; e < n; e += 32) xt[e] = g_xt[e];
    if (E.iters_done > 0) {
        for (int e = lane; e < n; e += 32) {
            ws.xa[e] = g_xa[e];
            ws.ga[e] = g_ga[e];
            if (!kDdGlobal) ws.dd[e] = g_dd[e];
        }
        if (lane < 9) ws.v[lane] = sc[3 + lane];     // rho[0..8) at v[0..8), y^T y at v[8]
        st.f = sc[0];
        st.alpha = sc[1];
        st.gts = sc[2];
        st.hist = __float_as_int(sc[12]);
        st.newest = __float_as_int(sc[13]);
        st.first = __float_as_int(sc[14]);
        st.accepts = __float_as_int(sc[15]);
    }
    const Goal G = make_goal(R + L.goal);
    __syncwarp();
    for (int it = 0; it < E.iters_round; ++it) {
        const EvalOut o = warp_eval<TPL, MODE_GRAD, SELF, SWEEP>(rb, kc, sv, T, G, ws, false);
        __syncwarp();
        lbfgs_update<NPL>(ko, n, st, xt, ws.gs, o.cost, ws, S_, Y_, xt);
    }
    if (!E.final_round) {
        for (int e = lane; e < n; e += 32) {
            g_xt[e] = xt[e];
            g_xa[e] = ws.xa[e];
            g_ga[e] = ws.ga[e];
            if (!kDdGlobal) g_dd[e] = ws.dd[e];
        }
        if (lane < 9) sc[3 + lane] = ws.v[lane];
        if (lane == 0) {
            sc[0] = st.f;
            sc[1] = st.alpha;
            sc[2] = st.gts;
            sc[12] = __int_as_float(st.hist);
            sc[13] = __int_as_float(st.newest);
            sc[14] = __int_as_float(st.first);
            sc[15] = __int_as_float(st.accepts);
        }
        return;
    }
    // last round: success test of the accepted point, outputs
    for (int e = lane; e < n; e += 32) xt[e] = ws.xa[e];
    __syncwarp();
    const EvalOut o = warp_eval<TPL, MODE_EVAL, SELF, SWEEP>(rb, kc, sv, T, G, ws, false);
    for (int e = lane; e < n; e += 32) g_xa[e] = ws.xa[e];
    const bool ok = o.min_clear >= 0.0f && o.pos_err < delta_t && o.rot_err < delta_r && o.lim_viol == 0.0f;
    if (lane == 0) {
        R[L.cost + s] = st.f;
        reinterpret_cast<uint8_t *>(R + L.succ)[s] = ok ? 1 : 0;
        if (ok && st.f >= 0.0f) {
            const unsigned long long key = ((unsigned long long)__float_as_uint(st.f) << 32) | (unsigned)s;
            atomicMin(reinterpret_cast<unsigned long long *>(R + L.key), key);
        }
    }
}

// Request traffic of a serving round (the seeds and problem of each admitted
// request in, the outputs of each finishing request out) as one launch instead
// of four small copies per request: block b copies entry b, 16 bytes a thread
// per step when source, destination and size allow, else 4 or 1.
__global__ void __launch_bounds__(256) k_io_copies(const IoCopy *__restrict__ table, int n) {
    const int b = blockIdx.x;
    if (b >= n) return;
    const IoCopy c = table[b];
    const uintptr_t s = reinterpret_cast<uintptr_t>(c.src), d = reinterpret_cast<uintptr_t>(c.dst);
    const unsigned long long bytes = c.bytes;
    if (((s | d | bytes) & 15) == 0) {
        const uint4 *src = reinterpret_cast<const uint4 *>(c.src);
        uint4 *dst = reinterpret_cast<uint4 *>(c.dst);
        for (unsigned long long i = threadIdx.x; i < bytes / 16; i += blockDim.x) dst[i] = src[i];
    } else if (((s | d | bytes) & 3) == 0) {
        const unsigned *src = reinterpret_cast<const unsigned *>(c.src);
        unsigned *dst = reinterpret_cast<unsigned *>(c.dst);
        for (unsigned long long i = threadIdx.x; i < bytes / 4; i += blockDim.x) dst[i] = src[i];
    } else {
        const unsigned char *src = reinterpret_cast<const unsigned char *>(c.src);
        unsigned char *dst = reinterpret_cast<unsigned char *>(c.dst);
        for (unsigned long long i = threadIdx.x; i < bytes; i += blockDim.x) dst[i] = src[i];
    }
}

int launch_io_copies(const IoCopy *table_dev, int n, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_io_copies<<<(unsigned)n, 256, 0, st>>>(table_dev, n);
    return (int)cudaGetLastError();
}

int launch_serve(const KRobot &rb, const KCost &kc, const KOpt &ko, float delta_t, float delta_r, int tpl,
                 const ServeEntry *table, int n_entries, long long total_warps, cudaStream_t st) {
    if (n_entries == 0 || total_warps == 0) return cudaSuccess;
    const bool self = kc.w_s > 0.f;
    const int warps = serve_warps(tpl, self);
    const unsigned blocks = (unsigned)((total_warps + warps - 1) / warps);
    const size_t smem = (size_t)warps * serve_warp_floats(tpl, self) * sizeof(float);
    auto go = [&](auto kern) {
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return (int)e;
        }
        kern<<<blocks, warps * 32, smem, st>>>(rb, kc, ko, delta_t, delta_r, table, n_entries, total_warps);
        return (int)cudaGetLastError();
    };
    // variants: waypoints per lane x self-collision term x swept check
    auto by_t = [&](auto self_c, auto sweep_c) {
        constexpr bool kSelf = decltype(self_c)::value, kSweep = decltype(sweep_c)::value;
        if (tpl == 1) return go(k_serve<1, kSelf, kSweep>);
        if (tpl == 2) return go(k_serve<2, kSelf, kSweep>);
        return go(k_serve<4, kSelf, kSweep>);
    };
    using T_ = std::true_type;
    using F_ = std::false_type;
    const bool sweep = kc.n_sweep > 0;
    return self ? (sweep ? by_t(T_{}, T_{}) : by_t(T_{}, F_{})) : (sweep ? by_t(F_{}, T_{}) : by_t(F_{}, F_{}));
}

}  // namespace dseed
