// internal.h -- structures shared by the host ABI layer and the kernels of libdseed.
#pragma once

#include <cstddef>
#include <cstdint>

#include "dseed.h"

namespace dseed {

constexpr int kWarp = 32;
constexpr int kPad = 3;          // rows y_-2, y_-1, y_0 ahead of the trajectory in shared memory

// Robot as the kernels read it: passed by value as a __grid_constant__ kernel
// parameter, so every lane reads it through the constant cache (all lanes of a
// warp read the same entry at the same time).  Spheres are sorted by frame.
struct KRobot {
    float a[8], d[8], ca[8], sa[8], off[8];  // DH rows: a, d, cos(alpha), sin(alpha), theta offset
    float ca2[8], sa2[8];                    // cos/sin(alpha / 2) for the quaternion chain
    float lo[7], hi[7];                      // joint limits
    int n_spheres;
    int frame_begin[9];                      // spheres of frame L (1..8): [frame_begin[L-1], frame_begin[L])
    float4 fbound[8];                        // per frame: bounding-sphere centre (frame coordinates), radius
    float frmin[8], frmax[8];                // per frame: smallest / largest sphere radius
    float cf8, sf8;                          // cos / sin of the flange frame's fixed theta offset
    float4 sph[DSEED_MAX_SPHERES];           // offset xyz, radius (sorted by frame)
    int sph_orig[DSEED_MAX_SPHERES];         // index in the caller's description
    // self-collision: bit j of self_mask[k] = the (sorted) pair (k, j) is checked;
    // bit a - 1 of self_frames[L - 1] = frame a <= L - 2 has a checked pair with frame L
    unsigned long long self_mask[DSEED_MAX_SPHERES];
    unsigned self_frames[8];
};

struct KCost {
    float w_c, eta, inv_dt, w_v, w_a, w_j, w_p, w_R, w_l;
    float w_s, eta_s;                        // self-collision hinge (w_s = 0: off)
    int n_sweep;                             // interpolants per segment (0: waypoints only)
    float sweep_u;                           // 1 / (n_sweep + 1): interpolant j sits at u = j sweep_u
};

struct KOpt {
    int iters, m;
    float c1, max_step, gamma0, alpha_min;
};

struct KBatch {
    int P, S, T;
    const float *q_start;                    // [P][7]
    const float *goal;                       // [P][7]
    const int *scene_of_problem;             // [P]
    const DseedScene *scenes;                // [n_scenes]
    int n_scenes;
    float delta_t, delta_r;
};

// Byte offsets of the L-BFGS state arrays (mirrors DseedLbfgsLayout).
struct KLbfgsPtrs {
    float *x, *g, *x_trial, *d, *s, *y, *rho, *yy, *f, *alpha, *gts;
    int *meta;
};

// Launchers (return a cudaError_t as int); defined in the kernels_*.cu files.
constexpr int kMaxEsdfJobs = 256;                // ESDF jobs per launch (carried in the kernel parameters)
int launch_esdf_build(const DseedEsdfJob *jobs, int n_jobs, cudaStream_t st);
int launch_fk(const KRobot &rb, const float *q, int N, float *pose, float *spheres, cudaStream_t st);
int launch_fk_mse(const KRobot &rb, const float *lin, const float *eps, const float *pred, const float *w, int N,
                  int T, float res_scale, float *dpred, float *loss_partial, int blocks, cudaStream_t st);
int launch_cost(const KRobot &rb, const KCost &kc, const KBatch &kb, const float *x, float *cost,
                float *terms, cudaStream_t st);
int launch_cost_grad(const KRobot &rb, const KCost &kc, const KBatch &kb, const float *x,
                     const float *grad_scale, float *cost, float *grad, cudaStream_t st);
int launch_evaluate(const KRobot &rb, const KCost &kc, const KBatch &kb, const float *x,
                    uint8_t *success, float *metrics, cudaStream_t st);
int launch_lbfgs_init(int B, int n, const float *x0, const KLbfgsPtrs &p, int m, cudaStream_t st);
int launch_lbfgs_step(const KOpt &ko, int B, int T, const float *f_trial, const float *g_trial,
                      const KLbfgsPtrs &p, cudaStream_t st);
int launch_plan(const KRobot &rb, const KCost &kc, const KOpt &ko, const KBatch &kb,
                const float *seeds, float *hist_s, float *hist_y, float *dirs, unsigned long long *best_key,
                float *traj, float *cost, uint8_t *success, float *metrics, int *best, cudaStream_t st);

}  // namespace dseed

namespace dseed {

// ---------------------------------------------------------------- serving
// Device memory of one served request (offsets in floats from its region base;
// every array 64-float (256-byte) aligned).  S seeds of n = 7T unknowns,
// history m.  The trial point starts as the request's seeds.
struct ServeLayout {
    size_t qs, goal, xt, xa, ga, dd, hs, hy, sc, cost, succ, key, total;
};

__host__ __device__ inline size_t serve_align(size_t v) { return (v + 63) & ~(size_t)63; }

__host__ __device__ inline ServeLayout serve_layout(int S, int T, int m) {
    const size_t n = 7 * (size_t)T, Sn = (size_t)S * n;
    ServeLayout l;
    size_t off = 0;
    l.qs = off;   off = serve_align(off + 7);
    l.goal = off; off = serve_align(off + 7);
    l.xt = off;   off = serve_align(off + Sn);
    l.xa = off;   off = serve_align(off + Sn);
    l.ga = off;   off = serve_align(off + Sn);
    l.dd = off;   off = serve_align(off + Sn);
    l.hs = off;   off = serve_align(off + (size_t)m * Sn);
    l.hy = off;   off = serve_align(off + (size_t)m * Sn);
    l.sc = off;   off = serve_align(off + 16 * (size_t)S);   // per seed: f, alpha, gts, yy, rho[8], hist, newest, first, accepts
    l.cost = off; off = serve_align(off + (size_t)S);
    l.succ = off; off = serve_align(off + ((size_t)S + 3) / 4);   // uint8 per seed
    l.key = off;  off = serve_align(off + 2);                     // one uint64
    l.total = off;
    return l;
}

// One request in a serving round (built on the host, read by every warp of it).
struct ServeEntry {
    long long warp_begin;     // first warp of this request in the launch
    float *region;            // request region base
    DseedScene scene;
    int S, T;
    int iters_done;           // iterations done before this round (0: start from the seeds)
    int iters_round;          // iterations to run in this round
    int final_round;          // 1: test success and write the outputs after this round
    int pad;
};

int launch_serve(const KRobot &rb, const KCost &kc, const KOpt &ko, float delta_t, float delta_r, int tpl,
                 const ServeEntry *table, int n_entries, long long total_warps, cudaStream_t st);

// One copy of the serving loop's request traffic: `bytes` from src to dst, both
// addresses the device can dereference (device memory, or pinned host memory
// through its mapped device address).
struct IoCopy {
    const void *src;
    void *dst;
    unsigned long long bytes;
};

// All copies of table_dev [n] in one launch (a block per copy).
int launch_io_copies(const IoCopy *table_dev, int n, cudaStream_t st);

}  // namespace dseed
