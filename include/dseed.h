/*
 * dseed.h -- C ABI of libdseed: seed-parallel trajectory optimisation for a
 * 7-DoF arm on one NVIDIA GB300 (sm_103a).
 *
 * The library optimises many seed trajectories per planning problem in
 * parallel, as the motion optimiser of the paper does (Sec. 4.4
 * "Optimization", Appendix A.5 "Optimization Problem"):
 *
 *     min over x_1..x_T   C_goal(X_d, FK(x_T)) + C_smooth + C_world + C_limit
 *
 * with y_0 = q_start held fixed.  Per waypoint t and collision sphere k the
 * world cost is w_c * max(0, r_k + eta - phi(c_k)), phi the trilinear
 * interpolation of a voxel ESDF (Euclidean signed distance field) at the
 * sphere centre c_k placed by forward kinematics; C_smooth is the weighted sum
 * of squared backward-difference velocities, accelerations and jerks at
 * spacing dt (start at rest: y_-1 = y_-2 = y_0); C_goal = w_p |p - p*|^2 +
 * w_R (1 - <q, q*>^2) on the flange pose at waypoint T; C_limit is a quadratic
 * penalty outside the joint limits.  Each iteration evaluates cost and
 * gradient (hand-written adjoint) of every seed and takes one L-BFGS step
 * with Armijo accept/reject.  Success (Sec. 5.1): collision free, translation
 * error below delta_t, rotation error below delta_r, within the limits.
 *
 * Conventions for every entry point:
 *   - Pointers named *_dev are device pointers, *_host host pointers; all
 *     other pointers are host pointers to small descriptors, read during the
 *     call and not retained.
 *   - The caller owns every buffer.  Only dseed_robot_create allocates (a
 *     small host object).  No call allocates device memory.
 *   - Calls taking a stream are asynchronous and stream ordered: they enqueue
 *     kernels on `stream` and return; outputs are valid once the stream has
 *     reached that point.  Inputs must stay valid until then.
 *   - Return 0 (DSEED_OK) on success or a negative status; the thread-local
 *     message of the last failure is returned by dseed_last_error().  Errors of
 *     kernels that have already been enqueued surface as DSEED_ECUDA on a
 *     later call or on the caller's stream synchronisation.
 *   - Arrays are dense, row-major, float32 unless stated, last index fastest.
 *     Trajectories are [P][S][T][7]: problem, seed, waypoint (t = 1..T), joint.
 *     Poses are [x, y, z, qw, qx, qy, qz] (metres, unit quaternion; the
 *     library normalises goal quaternions and treats q and -q alike).
 */
#ifndef DSEED_H
#define DSEED_H

#include <stddef.h>
#include <stdint.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DSEED_ABI_VERSION 4

#define DSEED_MAX_SPHERES 64    /* collision spheres per robot */
#define DSEED_MAX_T 128         /* waypoints per trajectory */
#define DSEED_MAX_HISTORY 8     /* L-BFGS history length m */
#define DSEED_MAX_SWEEP 8       /* interpolants per segment of the swept collision check */
#define DSEED_ESDF_FAR 1000.0f  /* ESDF value of a scene with no cuboid (m) */

/* status codes */
#define DSEED_OK 0
#define DSEED_EINVAL (-1)       /* bad argument: null pointer, size out of range, NaN parameter */
#define DSEED_ENOMEM (-2)       /* host allocation failed, or a caller buffer is too small */
#define DSEED_ECUDA (-3)        /* a CUDA call or kernel launch failed (message has the CUDA error) */
#define DSEED_ETIMEOUT (-4)     /* serving only: a wait on the GPU reached the server's wait limit */

/* Robot: a serial 7-joint arm in modified Denavit-Hartenberg form plus a
 * fixed flange frame, and its collision spheres.  Frame i (i = 1..7) turns
 * with joint i; frame 8 is the flange:
 *   T_i = T_{i-1} RotX(alpha_i) TransX(a_i) RotZ(q_i + theta_offset_i) TransZ(d_i)
 * (the forward kinematics FK of Eq. 2 and of C_goal in Appendix A.5). */
typedef struct {
    float dh[8][4];                          /* rows i = 1..8: a, d, alpha, theta_offset */
    float limits[7][2];                      /* lower, upper (rad) */
    int   n_spheres;                         /* 1..DSEED_MAX_SPHERES */
    int   sphere_frame[DSEED_MAX_SPHERES];   /* frame 1..8 the sphere is fixed to */
    float sphere_offset[DSEED_MAX_SPHERES][3]; /* centre in that frame (m) */
    float sphere_radius[DSEED_MAX_SPHERES];  /* radius (m), > 0 */
    /* Self-collision pairs (C_self of the App. A.5 objective): spheres on frames
     * at least two apart whose surfaces are at least self_margin apart at the
     * reference configuration self_ref (closer pairs overlap by construction of
     * the sphere model and are never checked). */
    float self_ref[7];                       /* rad */
    float self_margin;                       /* m */
} DseedRobotDesc;

typedef struct DseedRobot DseedRobot;        /* opaque, host memory */

/* Voxel grid: voxel (i, j, k) has its centre at origin + (i, j, k) * res +
 * res / 2 and is stored at index ((k * ny) + j) * nx + i.  nx, ny, nz >= 2. */
typedef struct {
    float origin[3];
    float res;
    int   nx, ny, nz;
} DseedGrid;

/* One scene as the optimiser reads it: its ESDF on the device, the grid, and
 * a Lipschitz bound L of the field (|phi(a) - phi(b)| <= L |a - b| between voxel
 * centres).  A true distance field, such as dseed_scene_build_esdf writes, has
 * L = 1.  With L > 0 the cost and adjoint kernels read only the voxel nearest to
 * a sphere centre when that value already proves the hinge inactive (value >=
 * r + eta + L sqrt(3) res + 1e-5), and skip the trilinear interpolation: the
 * results are the same as with the full interpolation.  L = 0 turns this off
 * (for fields that are not distance fields).  The success test always
 * interpolates. */
typedef struct {
    const float *esdf_dev;                   /* [nz][ny][nx] */
    DseedGrid    grid;
    float        lipschitz;                  /* L >= 0 */
} DseedScene;

/* Cost weights (Appendix A.5 objective; values are the caller's choice). */
typedef struct {
    float w_c;    /* collision hinge weight */
    float eta;    /* collision margin (m) */
    float dt;     /* waypoint spacing (s) */
    float w_v, w_a, w_j;   /* squared velocity / acceleration / jerk weights */
    float w_p;    /* goal position weight */
    float w_R;    /* goal orientation weight */
    float w_l;    /* joint-limit weight */
    float w_self;   /* self-collision hinge weight w_s (0: no self term); C_self = w_s sum over the
                     * robot's checked sphere pairs and waypoints of max(0, r_i + r_j + eta_self - |c_i - c_j|),
                     * added to the collision term; with w_self > 0 a trajectory is collision free
                     * only if it is also free of self-collision */
    float eta_self; /* self-collision margin (m) */
    int   n_sweep;  /* swept collision, 0..DSEED_MAX_SWEEP (0: waypoints only).  The robot executes a
                     * trajectory by linear interpolation in joint space, so each segment (y_{t-1}, y_t),
                     * t = 1..T with y_0 = q_start, is also checked at the n_sweep configurations
                     * q = (1 - u) y_t + u y_{t-1}, u = j / (n_sweep + 1), j = 1..n_sweep: the collision
                     * hinge (world term only) is added there, its derivative reaches y_t with weight 1 - u
                     * and y_{t-1} with weight u, and the success test's clearance includes them */
} DseedCostParams;

/* L-BFGS settings.  One iteration = one cost+gradient evaluation of the trial
 * point followed by one update: accept the trial when f_trial <= f + c1 *
 * g^T (x_trial - x) (always on the first evaluation), pushing (s, y) into the
 * history when s^T y > 1e-10 |s| |y|, and doubling alpha up to 1; otherwise
 * halve alpha (below alpha_min: clear the history, alpha = 1).  Then
 * d = -H g by the two-loop recursion (H0 = gamma I with gamma = s^T y / y^T y
 * of the newest pair, gamma0 when the history is empty; d = -g when not a
 * descent direction), step = alpha d scaled so that max |step| <= max_step,
 * next trial = x + step.  The result is the last accepted point. */
typedef struct {
    int   iters;      /* evaluations, >= 1 */
    int   m;          /* history length, 1..DSEED_MAX_HISTORY */
    float c1;
    float max_step;   /* rad */
    float gamma0;
    float alpha_min;
} DseedOptParams;

/* Shape and settings of one batch: P problems of S seeds of T waypoints. */
typedef struct {
    int P;            /* >= 0 */
    int S;            /* >= 1 */
    int T;            /* 1..DSEED_MAX_T */
    DseedCostParams cost;
    DseedOptParams  opt;
    float delta_t;    /* success: translation error below (m), Sec. 5.1 uses 0.005 */
    float delta_r;    /* success: rotation error below (rad), Sec. 5.1 uses 2.86 deg */
} DseedPlanDesc;

/* The problems of a batch, all in device memory. */
typedef struct {
    const float      *q_start_dev;            /* [P][7] y_0 */
    const float      *goal_dev;               /* [P][7] goal flange pose X_d */
    const int        *scene_of_problem_dev;   /* [P] index into scenes_dev */
    const DseedScene *scenes_dev;             /* [n_scenes] */
    int               n_scenes;
} DseedProblems;

/* Per-trajectory metrics written by dseed_evaluate (and by the plan):
 * min over waypoints and spheres of phi(c_k) - r_k, translation error |p - p*|,
 * rotation error (rad), max |jerk| over waypoints and joints (Appendix A.6),
 * worst joint-limit violation (rad), total cost, 1 if collision free else 0. */
#define DSEED_N_METRICS 7

/* ---------------------------------------------------------------- basics */

/* DSEED_ABI_VERSION of the library: a binding written against this header
 * checks it before use.  Never fails. */
int dseed_abi_version(void);
/* Message of the calling thread's last failed call ("" before any failure);
 * owned by the library, valid until that thread's next failing call. */
const char *dseed_last_error(void);

/* What the roofline of the optimiser's FP32 kernels is computed from (no
 * counterpart in the paper): streaming multiprocessors, their peak clock (kHz),
 * L2 bytes, compute capability and FP32 lanes per SM, from the CUDA runtime's
 * device attributes of `device`.  ECUDA when the device cannot be queried. */
typedef struct {
    int sm_count, sm_clock_khz, l2_bytes, cc_major, cc_minor, fp32_lanes_per_sm;
} DseedDeviceInfo;
int dseed_device_info(int device, DseedDeviceInfo *out);

/* Copy and check a robot description.  *out receives a handle owned by the
 * caller until dseed_robot_destroy.  EINVAL on a null pointer, a sphere count
 * outside 1..DSEED_MAX_SPHERES, a frame outside 1..8, a non-positive radius,
 * lower > upper or a non-finite entry. */
int  dseed_robot_create(const DseedRobotDesc *desc, DseedRobot **out);
void dseed_robot_destroy(DseedRobot *robot);
/* The self-collision pairs the robot checks (rule in DseedRobotDesc), in the
 * caller's sphere order: bit j of mask_host[i] set for a checked pair (i, j),
 * symmetric; *n_pairs (optional) receives the number of pairs.  mask_host
 * holds n_spheres entries.  Host-only; EINVAL on a null robot or mask. */
int  dseed_robot_self_pairs(const DseedRobot *robot, unsigned long long *mask_host, int *n_pairs);

/* ------------------------------------------------------------------ ESDF */

/* Per-voxel brute-force ESDF of a union of axis-aligned cuboids (the
 * optimiser's collision field, Sec. 4.4).  For every voxel centre p:
 *   phi(p) = min(DSEED_ESDF_FAR, min_k sdf_k(p)),
 *   sdf_k(p) = |max(|p - c_k| - h_k, 0)| + min(max_i(|p - c_k|_i - h_k,i), 0),
 * positive outside all cuboids, minus the deepest penetration inside one.
 * cuboids_dev: [n][6] = cx, cy, cz, hx, hy, hz (centre, half extents, m);
 * may be NULL when n == 0.  esdf_dev: [nz][ny][nx], written in full.
 * EINVAL on n < 0, a grid dimension < 2, res <= 0 or a null output. */
int dseed_scene_build_esdf(const float *cuboids_dev, int n, const DseedGrid *grid,
                           float *esdf_dev, cudaStream_t stream);

/* One ESDF to build: cuboids_dev [n][6] (may be NULL when n == 0), its grid,
 * and the output esdf_dev [nz][ny][nx]. */
typedef struct {
    const float *cuboids_dev;
    int          n;
    DseedGrid    grid;
    float       *esdf_dev;
} DseedEsdfJob;

/* The same per-voxel ESDF as dseed_scene_build_esdf for n_jobs scenes at once
 * (grids may differ), in as few launches as possible.  jobs_host is a host
 * array, read during the call.  EINVAL as for the single-scene call, for the
 * first offending job. */
int dseed_scene_build_esdf_batch(const DseedEsdfJob *jobs_host, int n_jobs, cudaStream_t stream);

/* ------------------------------------------------------------ kinematics */

/* Forward kinematics of N configurations q_dev [N][7] (FK of the goal term
 * C_goal(X_d, FK(q_T)), App. A.5; the sphere placement c = R_L o + p_L of the
 * collision model, Sec. 4.4): flange poses pose_dev [N][7] (qw >= 0) and, when
 * spheres_dev is not NULL, the sphere centres [N][n_spheres][3] in the order
 * of the robot description.  EINVAL on a null robot, N < 0, or (N > 0) a null
 * q_dev or pose_dev; N = 0 enqueues nothing. */
int dseed_fk(const DseedRobot *robot, const float *q_dev, int N, float *pose_dev,
             float *spheres_dev, cudaStream_t stream);

/* ---------------------------------------------------------- cost, adjoint */

/* Cost of trajectories x_dev [P][S][T][7] of the problems in `pr` (the
 * objective of App. A.5, see the top of this file): cost_dev [P][S]; terms_dev
 * (optional) [P][S][4] = C_world (+ C_self), C_smooth, C_goal, C_limit.
 * desc->opt is not read.  EINVAL on a null robot, a bad descriptor (sizes, a
 * non-finite or out-of-range parameter), a null problem array or (P > 0) a
 * null x_dev or cost_dev.  A problem whose scene index is out of range gets a
 * NaN cost rather than an out-of-bounds read. */
int dseed_cost(const DseedRobot *robot, const DseedPlanDesc *desc, const DseedProblems *pr,
               const float *x_dev, float *cost_dev, float *terms_dev, cudaStream_t stream);

/* Cost and its gradient dC/dx by the hand-written adjoint (reverse pass
 * through the hinge, the trilinear lookup, the sphere placement and the
 * kinematic chain, plus the transposed finite-difference stencils): the
 * gradient the optimiser of Sec. 4.4 / App. A.5 descends.  cost_dev [P][S],
 * grad_dev [P][S][T][7].  grad_scale_dev (optional) [P][S] multiplies each
 * trajectory's gradient (the incoming adjoint of a reverse-mode caller).
 * Errors as dseed_cost, and EINVAL for a null grad_dev when P > 0. */
int dseed_cost_grad(const DseedRobot *robot, const DseedPlanDesc *desc, const DseedProblems *pr,
                    const float *x_dev, const float *grad_scale_dev, float *cost_dev,
                    float *grad_dev, cudaStream_t stream);

/* Success flags success_dev [P][S] (1 = success, the test of Sec. 5.1: no
 * sphere inside an obstacle at any waypoint, translation error < delta_t,
 * rotation error < delta_r, every waypoint within the limits) and metrics_dev
 * (optional) [P][S][DSEED_N_METRICS] (the layout listed at DSEED_N_METRICS) of
 * trajectories x_dev [P][S][T][7].
 * Errors as dseed_cost, with success_dev in place of cost_dev. */
int dseed_evaluate(const DseedRobot *robot, const DseedPlanDesc *desc, const DseedProblems *pr,
                   const float *x_dev, uint8_t *success_dev, float *metrics_dev,
                   cudaStream_t stream);

/* ---------------------------------------------------------------- L-BFGS */

/* L-BFGS state of B = P * S seeds of n = 7 T unknowns in one caller buffer.
 * Byte offsets of the arrays inside it (all 256-byte aligned): */
typedef struct {
    size_t x;         /* float [B][n] accepted point */
    size_t g;         /* float [B][n] gradient at x */
    size_t x_trial;   /* float [B][n] next trial point (read by the caller's evaluation) */
    size_t d;         /* float [B][n] current search direction */
    size_t s;         /* float [B][m][n] history s_i, by ring slot */
    size_t y;         /* float [B][m][n] history y_i, by ring slot */
    size_t rho;       /* float [B][8] 1 / s_i^T y_i, by ring slot */
    size_t yy;        /* float [B] y^T y of the newest pair */
    size_t f;         /* float [B] cost at x (+inf before the first evaluation) */
    size_t alpha;     /* float [B] step length */
    size_t gts;       /* float [B] g^T (x_trial - x) */
    size_t meta;      /* int [B][4] history count, newest slot, first-evaluation flag, accepts */
    size_t total;     /* bytes of the whole state */
} DseedLbfgsLayout;

/* Offsets of that state for desc (P, S, T, opt.m).  Host-only; EINVAL on a bad
 * descriptor (opt included) or a null out. */
int dseed_lbfgs_layout(const DseedPlanDesc *desc, DseedLbfgsLayout *out);

/* Start every seed at x0_dev [B][n]: x_trial = x0, f = +inf, alpha = 1, empty
 * history.  state_dev: caller buffer of at least layout.total bytes.  EINVAL on
 * a bad descriptor or (B > 0) a null x0_dev or state_dev. */
int dseed_lbfgs_init(const DseedPlanDesc *desc, const float *x0_dev, void *state_dev,
                     cudaStream_t stream);

/* One L-BFGS update (K4) of every seed, given the cost f_trial_dev [B] and
 * gradient g_trial_dev [B][n] of the current trial point: accept/reject, history
 * update, two-loop direction, next trial point (see DseedOptParams; the
 * optimiser of Sec. 4.4 takes one such step per cost evaluation, N_iters of them,
 * Table 1).  EINVAL on a bad descriptor or (B > 0) a null pointer. */
int dseed_lbfgs_step(const DseedPlanDesc *desc, const float *f_trial_dev,
                     const float *g_trial_dev, void *state_dev, cudaStream_t stream);

/* ------------------------------------------------------------------ plan */

/* Bytes of device workspace dseed_plan_batch needs for `desc`.  Host-only;
 * EINVAL on a bad descriptor (sizes, non-finite or out-of-range parameters) or
 * a null bytes. */
int dseed_plan_workspace_bytes(const DseedPlanDesc *desc, size_t *bytes);

/* Optimise every seed of every problem for desc->opt.iters iterations, on
 * the device in one pass, then test success (the seed-parallel optimisation of
 * Sec. 4.4 with N_iters = desc->opt.iters, Table 1; success and the pick of the
 * returned trajectory as in Sec. 5.1).
 * seeds_dev [P][S][T][7] initial trajectories; workspace_dev at least
 * dseed_plan_workspace_bytes (256-byte aligned; contents need not be set).
 * Outputs: traj_dev [P][S][T][7] last accepted point of each seed, cost_dev
 * [P][S] its cost, success_dev [P][S] (1 = success), metrics_dev (optional)
 * [P][S][DSEED_N_METRICS], best_dev [P] index of the lowest-cost successful
 * seed (ties -> lowest index), -1 when no seed succeeds.  traj_dev may alias
 * seeds_dev.  EINVAL on a null robot, a bad descriptor, a null problem array
 * or (P > 0) a null plan buffer, or a workspace not 256-byte aligned; ENOMEM
 * when workspace_bytes is below the size needed; P = 0 enqueues nothing. */
int dseed_plan_batch(const DseedRobot *robot, const DseedPlanDesc *desc, const DseedProblems *pr,
                     const float *seeds_dev, void *workspace_dev, size_t workspace_bytes,
                     float *traj_dev, float *cost_dev, uint8_t *success_dev, float *metrics_dev,
                     int *best_dev, cudaStream_t stream);

/* --------------------------------------------------------------- serving */

/* Device-memory arena manager (host bookkeeping only): first-fit over
 * [0, bytes) in 256-byte units, neighbouring free blocks merged on free.  The
 * server below uses it to place scenes and request state inside the caller's
 * arena; it is exposed so that its policy can be used and tested on its own. */
typedef struct DseedArena DseedArena;
int  dseed_arena_create(size_t bytes, DseedArena **out);
void dseed_arena_destroy(DseedArena *arena);
/* Reserve `bytes` (rounded up to 256): *offset receives the start, or the call
 * returns DSEED_ENOMEM (nothing reserved) when no free block is large enough. */
int  dseed_arena_alloc(DseedArena *arena, size_t bytes, size_t *offset);
/* Release a block returned by dseed_arena_alloc; EINVAL for an unknown offset. */
int  dseed_arena_free(DseedArena *arena, size_t offset);
/* Bytes reserved now, the most ever reserved, and the largest free block. */
int  dseed_arena_usage(const DseedArena *arena, size_t *used, size_t *peak, size_t *largest_free);

/* Serving loop with continuous batching (the paper measures plan time per
 * problem, Sec. 5.1, Table 1; requests of uneven seed counts, horizons and
 * grids arrive while others are being planned).
 *
 * The server owns no device memory of its own: the caller hands it one device
 * arena of arena_bytes, which is the HBM budget for resident scenes (ESDF +
 * cuboids) and for the optimiser state of admitted requests.  Requests queue on
 * the host in arrival order; dseed_server_step admits queued requests while
 * their state fits in the arena (first come, first served: the head of the
 * queue waits for memory rather than being overtaken), then runs one round:
 * up to round_iters L-BFGS iterations of every admitted request, all requests
 * together, in one launch per waypoint class (T <= 32, <= 64, <= 128).  A
 * request finishes after desc->opt.iters iterations; its outputs are copied to
 * its host buffers and its memory returns to the arena.  Each seed computes
 * exactly what dseed_plan_batch computes for it, whatever shares its rounds.
 * At most two rounds are in flight on the server's stream, so a new request
 * starts within about two rounds. */
typedef struct DseedServer DseedServer;

typedef struct {
    size_t arena_bytes;      /* size of arena_dev (the HBM budget) */
    int    max_requests;     /* requests admitted at the same time, >= 1 */
    int    round_iters;      /* iterations per round, >= 1 */
    DseedCostParams cost;
    DseedOptParams  opt;     /* opt.iters: iterations of every request */
    float  delta_t, delta_r; /* success thresholds */
} DseedServerDesc;

/* One planning request.  Host buffers (pinned memory recommended; they must
 * stay valid until the request is done): q_start [7], goal [7], seeds
 * [S][T][7]; outputs traj [S][T][7], cost [S], success [S], best (index of the
 * lowest-cost successful seed or -1).  When all six array buffers are pinned
 * (page-locked, so the device can address them), the request's inputs and
 * outputs move with the other requests' in one batched copy kernel per round
 * instead of separate copies; any other buffer is copied with cudaMemcpyAsync. */
typedef struct {
    int scene_id;
    int S, T;                /* S >= 1, 1 <= T <= DSEED_MAX_T */
    const float *q_start_host, *goal_host, *seeds_host;
    float *traj_host, *cost_host;
    uint8_t *success_host;
    int *best_host;
} DseedRequest;

typedef struct {
    long long submitted, admitted, completed, failed, rounds;
    int queued, active;                  /* now */
    size_t arena_used, arena_peak;       /* bytes */
} DseedServerStats;

/* Create a server on the current device.  arena_dev: caller's device buffer of
 * desc->arena_bytes (256-byte aligned), used by the server until destroy.
 * The server creates its own CUDA stream and events and a small pinned host
 * staging area; it allocates no device memory. */
int  dseed_server_create(const DseedRobot *robot, const DseedServerDesc *desc, void *arena_dev,
                         DseedServer **out);
/* Waits for the server's stream, then frees its host resources. */
void dseed_server_destroy(DseedServer *server);
/* Make a scene resident: copy cuboids_host [n][6] into the arena and build its
 * ESDF there (Lipschitz bound 1).  ENOMEM when it does not fit; EINVAL for a
 * used id or a bad grid.  Asynchronous on the server's stream. */
int  dseed_server_add_scene(DseedServer *server, int scene_id, const float *cuboids_host, int n,
                            const DseedGrid *grid);
/* Release a scene once the work already enqueued on the server's stream is done
 * (a bounded wait, DSEED_ETIMEOUT at the wait limit); EINVAL while queued or
 * admitted requests use it. */
int  dseed_server_remove_scene(DseedServer *server, int scene_id);
/* Queue a request (host-side only, returns at once); *ticket identifies it. */
int  dseed_server_submit(DseedServer *server, const DseedRequest *req, long long *ticket);
/* One scheduling step: retire finished rounds (outputs are in the host buffers
 * of requests reported done), admit queued requests, and launch one round if
 * any request is admitted and fewer than two rounds are in flight.  Never
 * blocks on the GPU unless `wait` is non-zero, in which case it first waits for
 * the oldest round in flight.  *n_done (optional) receives the number of
 * requests that finished in this call.
 * Every wait of the server on the GPU (this one, the reuse of a staging buffer
 * before a round's table upload, and dseed_server_remove_scene's wait for work
 * that reads the scene) polls an event against the wait limit; when the limit
 * is reached the call returns DSEED_ETIMEOUT (the failure-detection status of
 * a serving watchdog) with the round still in flight and nothing retired, so a
 * later call can wait again or the caller can give up on the device. */
int  dseed_server_step(DseedServer *server, int wait, int *n_done);
/* Limit, in seconds (>= 0; 0 = do not wait at all), of every wait of the
 * server on the GPU; 60 s when the server is created.  EINVAL for a negative
 * or NaN limit. */
int  dseed_server_set_wait_limit(DseedServer *server, double seconds);
/* State of a ticket: 0 queued, 1 admitted, 2 done, -1 failed (scene missing
 * or request larger than the whole arena).  t_submit/t_done (optional)
 * receive the host steady-clock times in seconds of submission and of the step
 * that saw it finish. */
int  dseed_server_poll(DseedServer *server, long long ticket, int *state, double *t_submit, double *t_done);
int  dseed_server_stats(const DseedServer *server, DseedServerStats *out);

/* ------------------------------------------------- learned seed proposal */

/* Layers of the conditional denoiser that proposes seed trajectories (Sec.
 * 4.2 "Model Architecture": a 1-D temporal-convolution U-Net of conditional
 * residual blocks conditioned on a time-step embedding and an observation +
 * problem encoding; Sec. 4.3 "Model Training and Inference": the noise
 * prediction objective of Eq. 1 and DDIM sampling, App. A.3 / A.5).  The
 * caller strings the layers together; every arithmetic step runs here.
 *
 * Tensors are FP32, channels-last [N][L][C] (C fastest) unless stated; all
 * pointers are device pointers; calls are asynchronous on `stream`; no call
 * allocates.  EINVAL on negative sizes or NULL required pointers. */

/* C[M][N] = alpha op(A) op(B) + beta C (+ bias[N] if bias_dev != NULL), FP32.
 * op(A) = A ([M][K], lda) or, with trans_a, A^T (A stored [K][M]); likewise B. */
int dseed_nn_gemm_f32(int trans_a, int trans_b, int M, int N, int K, float alpha, const float *A_dev, int lda,
                      const float *B_dev, int ldb, float beta, float *C_dev, int ldc, const float *bias_dev,
                      cudaStream_t stream);
/* C[M][N] (FP32) = A[M][K] W[N][K]^T (+ bias[N]) on the tensor cores: A and W
 * BF16 row-major, K a multiple of 16, FP32 accumulation. */
int dseed_nn_gemm_bf16(int M, int N, int K, const void *A_dev, const void *W_dev, float *C_dev,
                       const float *bias_dev, cudaStream_t stream);
/* im2col for a 1-D convolution of x [N][L][C] with kernel k, stride s, padding
 * p: cols[N * Lo][kc_pad], entry (j, c) of row (n, lo) = x[n][lo s - p + j][c]
 * (0 outside [0, L) and for columns >= k C).  cols is BF16 when bf16 != 0. */
int dseed_nn_im2col1d(const float *x_dev, int N, int L, int C, int k, int s, int p, int Lo, int kc_pad,
                      void *cols_dev, int bf16, cudaStream_t stream);
/* Adjoint of im2col: dx[N][L][C] += the column entries that came from it. */
int dseed_nn_col2im1d(const float *cols_dev, int N, int L, int C, int k, int s, int p, int Lo, int kc_pad,
                      float *dx_dev, cudaStream_t stream);
/* out[c] = (out[c] if accumulate) + sum_r y[r][c] over y [R][C]. */
int dseed_nn_colsum(const float *y_dev, int R, int C, float *out_dev, int accumulate, cudaStream_t stream);
/* Group normalisation over (L, C / G) per sample and group, affine gamma/beta
 * [C]; mean / rstd [N][G] are saved for the backward pass. */
int dseed_nn_groupnorm_fwd(const float *x_dev, int N, int L, int C, int G, const float *gamma_dev,
                           const float *beta_dev, float eps, float *y_dev, float *mean_dev, float *rstd_dev,
                           cudaStream_t stream);
/* Backward of the above: dx [N][L][C]; per-sample partials dgamma_n, dbeta_n
 * [N][C] (sum them over N with dseed_nn_colsum). */
int dseed_nn_groupnorm_bwd(const float *dy_dev, const float *x_dev, int N, int L, int C, int G,
                           const float *gamma_dev, const float *mean_dev, const float *rstd_dev, float *dx_dev,
                           float *dgamma_n_dev, float *dbeta_n_dev, cudaStream_t stream);
/* Mish(x) = x tanh(softplus(x)) elementwise (backward: out = dy * Mish'(x)). */
int dseed_nn_mish(const float *x_dev, const float *dy_dev, float *out_dev, long long n, int backward,
                  cudaStream_t stream);
/* FiLM conditioning of a residual block: y = h * film[:, :C] + film[:, C:]
 * with film [N][2C] broadcast over L; backward gives dh and dfilm [N][2C]. */
int dseed_nn_film(const float *h_dev, const float *film_dev, int N, int L, int C, float *y_dev,
                  const float *dy_dev, float *dh_dev, float *dfilm_dev, int backward, cudaStream_t stream);
/* out = a x + b y elementwise (y may be NULL). */
int dseed_nn_axpby(float a, const float *x_dev, float b, const float *y_dev, float *out_dev, long long n,
                   cudaStream_t stream);
/* Channel-slice copy for concatenation and its adjoint: for R rows,
 * out[r][out_off + c] (+)= in[r][in_off + c], c < C_in. */
int dseed_nn_copy_cols(const float *in_dev, long long R, int C_in, int in_stride, int in_off, float *out_dev,
                       int out_stride, int out_off, int accumulate, cudaStream_t stream);
/* Nearest-neighbour upsampling by 2 along L ([N][L][C] -> [N][2L][C]); the
 * backward (backward != 0) maps [N][2L][C] gradients to [N][L][C]. */
int dseed_nn_upsample2(const float *x_dev, int N, int L, int C, float *y_dev, int backward, cudaStream_t stream);
/* Per-row gather out[r][e] = in[r][idx[e]] over n rows of `per` entries, or the
 * adjoint scatter-add (scatter != 0): out[r][idx[e]] += in[r][e]. */
int dseed_nn_gather(const float *in_dev, const int *idx_dev, float *out_dev, long long n, long long per,
                    int scatter, cudaStream_t stream);
/* Row gather: out[r] = in[rows[r]] for rows [R_out] (int32), rows of C floats
 * (one condition vector per problem broadcast to its samples). */
int dseed_nn_gather_rows(const float *in_dev, const int *rows_dev, long long R_out, int C, float *out_dev,
                         cudaStream_t stream);
/* Sinusoidal embedding of integer diffusion steps k [N] into [N][dim]. */
int dseed_nn_sinusoid(const int *k_dev, int N, int dim, float *out_dev, cudaStream_t stream);
/* One Adam step with decoupled weight decay on n parameters (step >= 1). */
int dseed_nn_adam(float *p_dev, const float *g_dev, float *m_dev, float *v_dev, long long n, float lr, float beta1,
                  float beta2, float eps, float weight_decay, int step, cudaStream_t stream);
/* Forward noising of Eq. 1: x_k = sqrt(abar[k_n]) x0 + sqrt(1 - abar[k_n]) eps
 * for N samples of `per` values; abar_dev [K] the cumulative noise schedule. */
int dseed_nn_ddpm_noise(const float *x0_dev, const float *eps_dev, const int *k_dev, const float *abar_dev, int N,
                        int per, float *xk_dev, cudaStream_t stream);
/* The loss of Eq. 1 with optional per-sample weights w [N] (Eq. 2's
 * (1 + alpha 1(tau)) factor): loss = sum w_n (pred - target)^2 / (N per),
 * written as `blocks` partial sums into loss_partial_dev; dpred = dloss/dpred. */
int dseed_nn_mse(const float *pred_dev, const float *target_dev, const float *w_dev, int N, int per,
                 float *dpred_dev, float *loss_partial_dev, int blocks, cudaStream_t stream);
/* The loss of Eq. 2 measured on the robot (Sec. 4.3: the noise and the
 * predicted noise both go through forward kinematics to points on the robot).
 * eps_dev, pred_dev [N][T][7] live in the diffused space, the scaled residual
 * from the straight path: vector v stands for the joint configuration
 * q(v) = mid + half (lin + v / res_scale) per waypoint and joint, lin_dev
 * [N][T][7] the normalised straight start-goal path, mid and half the centre
 * and half-width of the robot's joint limits.  With c_k(q) the points on the
 * robot's surface -- for every collision sphere the six points of its
 * surface along the axes of its frame, N_p = 6 N_s -- and w_dev [N] optional
 * weights (Eq. 2's 1 + alpha 1(tau); NULL = 1):
 *   loss = sum_n w_n sum_{t,k} |c_k(q(pred_nt)) - c_k(q(eps_nt))|^2 / (N T N_p 3),
 * written as `blocks` (1..1024) partial sums into loss_partial_dev; dpred_dev
 * [N][T][7] = dloss/dpred.  Device arrays are the caller's; asynchronous on
 * stream.  EINVAL: NULL robot or array, T outside 1..DSEED_MAX_T, res_scale
 * not > 0. */
int dseed_nn_fk_mse(const DseedRobot *robot, const float *lin_dev, const float *eps_dev, const float *pred_dev,
                    const float *w_dev, int N, int T, float res_scale, float *dpred_dev, float *loss_partial_dev,
                    int blocks, cudaStream_t stream);
/* One deterministic DDIM step (App. A.5) from step k to an earlier step:
 * x0 = clamp((x_k - sqrt(1 - ab_k) eps) / sqrt(ab_k), -clip, clip),
 * out = sqrt(ab_prev) x0 + sqrt(1 - ab_prev) eps. */
int dseed_nn_ddim_step(const float *xk_dev, const float *eps_dev, float ab_k, float ab_prev, long long n, float clip,
                       float *out_dev, cudaStream_t stream);
/* out = min(max(a x + b, lo), hi) elementwise (e.g. occupancy from an ESDF:
 * a = -1e6, b = 0, lo = 0, hi = 1). */
int dseed_nn_clamp_affine(const float *x_dev, float a, float b, float lo, float hi, float *out_dev, long long n,
                          cudaStream_t stream);
/* FP32 -> BF16 (round to nearest even). */
int dseed_nn_to_bf16(const float *x_dev, void *y_dev, long long n, cudaStream_t stream);

/* Inference convolution on the tensor cores (tcgen05 MMA with BF16 operands
 * staged by TMA and FP32 accumulation in tensor memory), with the rest of the
 * layer fused into its epilogue (Sec. 4.2: conditional residual blocks of
 * conv - group norm - Mish, FiLM from the condition, residual add).
 *
 * out[n][lo][o] = bias[o] + sum_{j < taps} sum_c W[o][j][c] A[n][lo - pad + j][c]
 * with A = the channel concatenation of a0 [n_samples][L][c0] and a1
 * [n_samples][L][c1] (BF16, channels-last; rows outside [0, L) read as zero),
 * W BF16 [cout_pad][taps][c0 + c1] (rows >= cout zero).  A plain GEMM
 * out[m] = W a[m] is L = 1, taps = 1, pad = 0.
 *
 * epilogue 0: out FP32 [n_samples * L][out_ld], columns < cout.
 * epilogue 1: out BF16 [..][out_ld], columns < cout.
 * epilogue 2: y = Mish(GroupNorm(out)) over groups of cout / 8 channels and
 *   rows_per_sample consecutive rows (affine gamma, beta; biased variance, eps
 *   gn_eps); then y = y * film[s][o] + film[s][cout + o] when film_dev is given
 *   (rows film_ld floats apart, plus film_add[o] / film_add[cout + o] when
 *   film_add_dev is given; s = sample_problem[row / rows_per_sample], or
 *   row / rows_per_sample when sample_problem_dev is NULL); then y += res[row][o] (BF16 [..][cout]) when
 *   res_dev is given; out BF16 [..][out_ld].  Needs cout = cout_pad.
 *
 * Limits (EINVAL otherwise): c0, c1 multiples of 64 (c1 may be 0); L a power of
 * two <= 128; 1 <= taps <= 8, 0 <= pad < taps; cout_pad in {16, 64, 128, 256}
 * (16 only for epilogues 0/1), 1 <= cout <= cout_pad; rows_per_sample a power
 * of two <= 32 dividing n_samples * L (epilogue 2); out_ld >= cout (a multiple
 * of 8 for BF16 output); every pointer 16-byte aligned.  err_dev (optional, int)
 * is set non-zero if a pipeline wait inside the kernel gave up (2 s); the
 * output is then undefined.  Requires a GPU of compute capability 10.x. */
typedef struct {
    const void *a0_dev;
    int c0;
    const void *a1_dev;
    int c1;
    int n_samples, L, taps, pad;
    const void *w_dev;
    int cout, cout_pad;
    const float *bias_dev;
    int epilogue;
    int rows_per_sample;
    float gn_eps;
    const float *gamma_dev, *beta_dev;
    const float *film_dev;
    int film_ld;             /* floats between FiLM rows (0: 2 cout) */
    const float *film_add_dev;   /* optional [2 cout], added to every FiLM row */
    const int *sample_problem_dev;
    const void *res_dev;
    void *out_dev;
    int out_ld;
    int *err_dev;
} DseedConvTc;
int dseed_nn_conv_tc(const DseedConvTc *desc, cudaStream_t stream);
/* im2col of a BF16 activation (as dseed_nn_im2col1d, BF16 in and out). */
int dseed_nn_im2col1d_bf16(const void *x_dev, int N, int L, int C, int k, int s, int p, int Lo, int kc_pad,
                           void *cols_dev, cudaStream_t stream);
/* Nearest-neighbour x2 upsampling along L of a BF16 activation [N][L][C] -> [N][2L][C]. */
int dseed_nn_upsample2_bf16(const void *x_dev, int N, int L, int C, void *y_dev, cudaStream_t stream);

/* ------------------------------------------------ plan without allocation */

/* The paper has no counterpart to this call; it exists for callers that
 * cannot allocate device memory.  Examples: a control loop that has frozen
 * its memory after start-up, a plug-in running inside a host process whose
 * allocator it may not touch, or code that must not trigger the implicit
 * synchronisation a cudaMalloc/cudaFree can cause.  Such a caller cannot
 * provide the workspace dseed_plan_batch asks for.
 *
 * dseed_plan_batch_static does the same work as dseed_plan_batch (same
 * kernels, same results) but keeps its scratch (the L-BFGS history, for
 * T > 32 the search directions, and the per-problem best-seed keys) in one
 * array of DSEED_STATIC_SCRATCH_BYTES
 * bytes that lives in the library itself, as a file-scope device variable.
 * The caller still passes every input and output buffer.  The call never
 * allocates: no cudaMalloc, no cudaFree, no allocating library routine.
 *
 * Limits and rules:
 *   - The scratch needed is what dseed_plan_workspace_bytes reports for
 *     `desc`; a batch needing more than DSEED_STATIC_SCRATCH_BYTES is refused
 *     with DSEED_ENOMEM and a message giving both sizes (for T = 32 and m = 5
 *     that is about 3700 seeds per call).
 *   - Every GPU on which the library's device code is loaded holds the array
 *     until the process exits.
 *   - The first call on a device looks up the array's device address (with
 *     that device current) and caches it with the id of the current context;
 *     make that first call before any stream capture begins.  After a device
 *     reset the next call sees a new context and looks the address up again
 *     (also before any capture).
 *   - All calls share the one array, and it keeps what the last call left in
 *     it.  The call resets the parts that must start at zero itself, but two
 *     calls whose work overlaps on the GPU (different streams without
 *     ordering, or different host threads) race on the array: order them. */
#define DSEED_STATIC_SCRATCH_BYTES (32u << 20)

int dseed_plan_batch_static(const DseedRobot *robot, const DseedPlanDesc *desc, const DseedProblems *pr,
                            const float *seeds_dev, float *traj_dev, float *cost_dev,
                            uint8_t *success_dev, float *metrics_dev, int *best_dev,
                            cudaStream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* DSEED_H */
