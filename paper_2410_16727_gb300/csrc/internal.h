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
};

struct KCost {
    float w_c, eta, inv_dt, w_v, w_a, w_j, w_p, w_R, w_l;
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
                const float *seeds, float *hist_s, float *hist_y, unsigned long long *best_key,
                float *traj, float *cost, uint8_t *success, float *metrics, int *best, cudaStream_t st);

}  // namespace dseed
