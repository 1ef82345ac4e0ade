// abi.cu -- host side of the C ABI declared in include/dseed.h: argument
// checks, robot handles, workspace layouts and kernel launches.
#include <cuda.h>            // driver-API types only; entry points come through the runtime
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>

#include "internal.h"

struct DseedRobot {
    dseed::KRobot k;
    unsigned long long self_mask[DSEED_MAX_SPHERES];   // checked pairs in the caller's sphere order
    int n_self_pairs;
};

namespace {

thread_local std::string g_last_error;

int fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

int cuda_status(int err, const char *what) {
    if (err == cudaSuccess) return DSEED_OK;
    return fail(DSEED_ECUDA, "%s: %s", what, cudaGetErrorString((cudaError_t)err));
}

bool finite(float v) { return std::isfinite(v); }

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

int check_desc(const DseedPlanDesc *d, bool need_opt) {
    if (!d) return fail(DSEED_EINVAL, "desc is NULL");
    if (d->P < 0) return fail(DSEED_EINVAL, "P = %d < 0", d->P);
    if (d->S < 1) return fail(DSEED_EINVAL, "S = %d < 1", d->S);
    if (d->T < 1 || d->T > DSEED_MAX_T) return fail(DSEED_EINVAL, "T = %d outside 1..%d", d->T, DSEED_MAX_T);
    if ((long long)d->P * d->S > (1LL << 31) - 1) return fail(DSEED_EINVAL, "P * S too large");
    const DseedCostParams &c = d->cost;
    const float cv[] = {c.w_c, c.eta, c.dt, c.w_v, c.w_a, c.w_j, c.w_p, c.w_R, c.w_l, c.w_self, c.eta_self,
                        d->delta_t, d->delta_r};
    for (float v : cv)
        if (!finite(v)) return fail(DSEED_EINVAL, "non-finite cost or success parameter");
    if (!(c.dt > 0.f)) return fail(DSEED_EINVAL, "dt must be > 0");
    if (c.w_self < 0.f || c.eta_self < 0.f) return fail(DSEED_EINVAL, "w_self and eta_self must be >= 0");
    if (c.n_sweep < 0 || c.n_sweep > DSEED_MAX_SWEEP)
        return fail(DSEED_EINVAL, "n_sweep = %d outside 0..%d", c.n_sweep, DSEED_MAX_SWEEP);
    if (need_opt) {
        const DseedOptParams &o = d->opt;
        if (o.iters < 1) return fail(DSEED_EINVAL, "iters = %d < 1", o.iters);
        if (o.m < 1 || o.m > DSEED_MAX_HISTORY) return fail(DSEED_EINVAL, "m = %d outside 1..%d", o.m, DSEED_MAX_HISTORY);
        const float ov[] = {o.c1, o.max_step, o.gamma0, o.alpha_min};
        for (float v : ov)
            if (!finite(v)) return fail(DSEED_EINVAL, "non-finite optimiser parameter");
        if (!(o.max_step > 0.f) || !(o.gamma0 > 0.f) || !(o.alpha_min > 0.f))
            return fail(DSEED_EINVAL, "max_step, gamma0 and alpha_min must be > 0");
    }
    return DSEED_OK;
}

int check_problems(const DseedPlanDesc *d, const DseedProblems *pr) {
    if (!pr) return fail(DSEED_EINVAL, "problems is NULL");
    if (d->P == 0) return DSEED_OK;
    if (!pr->q_start_dev || !pr->goal_dev || !pr->scene_of_problem_dev || !pr->scenes_dev)
        return fail(DSEED_EINVAL, "a problem array is NULL");
    if (pr->n_scenes < 1) return fail(DSEED_EINVAL, "n_scenes = %d < 1", pr->n_scenes);
    return DSEED_OK;
}

dseed::KCost make_cost(const DseedCostParams &c) {
    dseed::KCost k;
    k.w_c = c.w_c;
    k.eta = c.eta;
    k.inv_dt = (float)(1.0 / (double)c.dt);
    k.w_v = c.w_v;
    k.w_a = c.w_a;
    k.w_j = c.w_j;
    k.w_p = c.w_p;
    k.w_R = c.w_R;
    k.w_l = c.w_l;
    k.w_s = c.w_self;
    k.eta_s = c.eta_self;
    k.n_sweep = c.n_sweep;
    k.sweep_u = (float)(1.0 / (double)(c.n_sweep + 1));
    return k;
}

dseed::KOpt make_opt(const DseedOptParams &o) {
    dseed::KOpt k;
    k.iters = o.iters;
    k.m = o.m;
    k.c1 = o.c1;
    k.max_step = o.max_step;
    k.gamma0 = o.gamma0;
    k.alpha_min = o.alpha_min;
    return k;
}

dseed::KBatch make_batch(const DseedPlanDesc *d, const DseedProblems *pr) {
    dseed::KBatch k;
    k.P = d->P;
    k.S = d->S;
    k.T = d->T;
    k.q_start = pr->q_start_dev;
    k.goal = pr->goal_dev;
    k.scene_of_problem = pr->scene_of_problem_dev;
    k.scenes = pr->scenes_dev;
    k.n_scenes = pr->n_scenes;
    k.delta_t = d->delta_t;
    k.delta_r = d->delta_r;
    return k;
}

DseedLbfgsLayout lbfgs_layout(long long B, int n, int m) {
    DseedLbfgsLayout l;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align256(off + bytes);
        return o;
    };
    l.x = take(sizeof(float) * B * n);
    l.g = take(sizeof(float) * B * n);
    l.x_trial = take(sizeof(float) * B * n);
    l.d = take(sizeof(float) * B * n);
    l.s = take(sizeof(float) * B * m * n);
    l.y = take(sizeof(float) * B * m * n);
    l.rho = take(sizeof(float) * B * 8);
    l.yy = take(sizeof(float) * B);
    l.f = take(sizeof(float) * B);
    l.alpha = take(sizeof(float) * B);
    l.gts = take(sizeof(float) * B);
    l.meta = take(sizeof(int) * B * 4);
    l.total = off;
    return l;
}

dseed::KLbfgsPtrs lbfgs_ptrs(void *base, const DseedLbfgsLayout &l) {
    char *c = static_cast<char *>(base);
    dseed::KLbfgsPtrs p;
    p.x = reinterpret_cast<float *>(c + l.x);
    p.g = reinterpret_cast<float *>(c + l.g);
    p.x_trial = reinterpret_cast<float *>(c + l.x_trial);
    p.d = reinterpret_cast<float *>(c + l.d);
    p.s = reinterpret_cast<float *>(c + l.s);
    p.y = reinterpret_cast<float *>(c + l.y);
    p.rho = reinterpret_cast<float *>(c + l.rho);
    p.yy = reinterpret_cast<float *>(c + l.yy);
    p.f = reinterpret_cast<float *>(c + l.f);
    p.alpha = reinterpret_cast<float *>(c + l.alpha);
    p.gts = reinterpret_cast<float *>(c + l.gts);
    p.meta = reinterpret_cast<int *>(c + l.meta);
    return p;
}

// Plan workspace: history s [B][m][n], history y [B][m][n], best keys [P].
struct PlanLayout {
    size_t s, y, d, key, total;
};

PlanLayout plan_layout(const DseedPlanDesc *d) {
    const long long B = (long long)d->P * d->S;
    const size_t n = 7 * (size_t)d->T, m = (size_t)d->opt.m;
    PlanLayout l;
    l.s = 0;
    l.y = align256(sizeof(float) * B * m * n);
    l.d = l.y + align256(sizeof(float) * B * m * n);                 // search directions (T > 32)
    l.key = l.d + (d->T > 32 ? align256(sizeof(float) * B * n) : 0);
    l.total = l.key + align256(sizeof(unsigned long long) * std::max(d->P, 1));
    return l;
}

// Frames 1..8 of the modified-DH chain at q (double precision, host): R row-major, p.
void host_fk(const DseedRobotDesc *d, const float *q, double R[9][9], double P[9][3]) {
    double Rc[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1}, pc[3] = {0, 0, 0};
    for (int i = 0; i < 8; ++i) {
        const double a = d->dh[i][0], dd = d->dh[i][1], al = d->dh[i][2];
        const double th = (i < 7 ? (double)q[i] : 0.0) + d->dh[i][3];
        const double ca = std::cos(al), sa = std::sin(al), ct = std::cos(th), st = std::sin(th);
        // p += a x_prev; R = R RotX(alpha) RotZ(theta); p += d z_new
        for (int r = 0; r < 3; ++r) pc[r] += a * Rc[3 * r];
        for (int r = 0; r < 3; ++r) {
            const double x = Rc[3 * r], y = Rc[3 * r + 1], z = Rc[3 * r + 2];
            const double y1 = ca * y + sa * z, z1 = -sa * y + ca * z;
            Rc[3 * r] = ct * x + st * y1;
            Rc[3 * r + 1] = -st * x + ct * y1;
            Rc[3 * r + 2] = z1;
        }
        for (int r = 0; r < 3; ++r) pc[r] += dd * Rc[3 * r + 2];
        for (int e = 0; e < 9; ++e) R[i + 1][e] = Rc[e];
        for (int e = 0; e < 3; ++e) P[i + 1][e] = pc[e];
    }
}

// The robot's self-collision pairs (rule in dseed.h): spheres on frames at least
// two apart whose surfaces are at least self_margin apart at self_ref.
void self_pairs(const DseedRobotDesc *d, DseedRobot *r) {
    double R[9][9], P[9][3];
    host_fk(d, d->self_ref, R, P);
    const int ns = d->n_spheres;
    double c[DSEED_MAX_SPHERES][3];
    for (int k = 0; k < ns; ++k) {
        const int L = d->sphere_frame[k];
        for (int row = 0; row < 3; ++row)
            c[k][row] = R[L][3 * row] * d->sphere_offset[k][0] + R[L][3 * row + 1] * d->sphere_offset[k][1] +
                        R[L][3 * row + 2] * d->sphere_offset[k][2] + P[L][row];
    }
    std::memset(r->self_mask, 0, sizeof(r->self_mask));
    r->n_self_pairs = 0;
    for (int i = 0; i < ns; ++i)
        for (int j = i + 1; j < ns; ++j) {
            const int df = d->sphere_frame[i] - d->sphere_frame[j];
            if (df > -2 && df < 2) continue;
            const double dx = c[i][0] - c[j][0], dy = c[i][1] - c[j][1], dz = c[i][2] - c[j][2];
            if (std::sqrt(dx * dx + dy * dy + dz * dz) - d->sphere_radius[i] - d->sphere_radius[j] >=
                (double)d->self_margin) {
                r->self_mask[i] |= 1ull << j;
                r->self_mask[j] |= 1ull << i;
                ++r->n_self_pairs;
            }
        }
    // the kernels' form: sorted sphere indices, and per frame the earlier frames with pairs
    dseed::KRobot &k = r->k;
    int sorted_of[DSEED_MAX_SPHERES];
    for (int q = 0; q < ns; ++q) sorted_of[k.sph_orig[q]] = q;
    for (int q = 0; q < ns; ++q) {
        const unsigned long long m = r->self_mask[k.sph_orig[q]];
        unsigned long long sm = 0;
        for (int j = 0; j < ns; ++j)
            if ((m >> j) & 1ull) sm |= 1ull << sorted_of[j];
        k.self_mask[q] = sm;
    }
    for (int L = 1; L <= 8; ++L) {
        unsigned fm = 0;
        for (int a = 1; a <= L - 2; ++a)
            for (int q = k.frame_begin[L - 1]; q < k.frame_begin[L]; ++q)
                for (int j = k.frame_begin[a - 1]; j < k.frame_begin[a]; ++j)
                    if ((k.self_mask[q] >> j) & 1ull) fm |= 1u << (a - 1);
        k.self_frames[L - 1] = fm;
    }
}

}  // namespace

namespace dseed {
// Shared with the serving runtime (server.cu).
int set_error(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}
KRobot robot_params(const DseedRobot *robot) { return robot->k; }
KCost cost_params(const DseedCostParams &c) { return make_cost(c); }
KOpt opt_params(const DseedOptParams &o) { return make_opt(o); }
int check_cost_opt(const DseedCostParams &c, const DseedOptParams &o, float delta_t, float delta_r) {
    DseedPlanDesc d;
    std::memset(&d, 0, sizeof(d));
    d.P = 0;
    d.S = 1;
    d.T = 1;
    d.cost = c;
    d.opt = o;
    d.delta_t = delta_t;
    d.delta_r = delta_r;
    return check_desc(&d, true);
}
}  // namespace dseed

extern "C" {

int dseed_abi_version(void) { return DSEED_ABI_VERSION; }

int dseed_device_info(int device, DseedDeviceInfo *out) {
    if (!out) return fail(DSEED_EINVAL, "out is NULL");
    int v[5] = {0, 0, 0, 0, 0};
    const cudaDeviceAttr attrs[5] = {cudaDevAttrMultiProcessorCount, cudaDevAttrClockRate, cudaDevAttrL2CacheSize,
                                     cudaDevAttrComputeCapabilityMajor, cudaDevAttrComputeCapabilityMinor};
    for (int i = 0; i < 5; ++i) {
        const cudaError_t e = cudaDeviceGetAttribute(&v[i], attrs[i], device);
        if (e != cudaSuccess) return fail(DSEED_ECUDA, "cudaDeviceGetAttribute: %s", cudaGetErrorString(e));
    }
    out->sm_count = v[0];
    out->sm_clock_khz = v[1];
    out->l2_bytes = v[2];
    out->cc_major = v[3];
    out->cc_minor = v[4];
    // FP32 lanes per SM: 128 on every compute capability 8.6+ part, 10.x included
    out->fp32_lanes_per_sm = (v[3] > 8 || (v[3] == 8 && v[4] >= 6)) ? 128 : 64;
    return DSEED_OK;
}

const char *dseed_last_error(void) { return g_last_error.c_str(); }

int dseed_robot_create(const DseedRobotDesc *desc, DseedRobot **out) {
    if (!desc || !out) return fail(DSEED_EINVAL, "desc or out is NULL");
    *out = nullptr;
    const int ns = desc->n_spheres;
    if (ns < 1 || ns > DSEED_MAX_SPHERES) return fail(DSEED_EINVAL, "n_spheres = %d outside 1..%d", ns, DSEED_MAX_SPHERES);
    for (int i = 0; i < 8; ++i)
        for (int c = 0; c < 4; ++c)
            if (!finite(desc->dh[i][c])) return fail(DSEED_EINVAL, "non-finite DH entry (%d, %d)", i, c);
    for (int j = 0; j < 7; ++j) {
        if (!finite(desc->limits[j][0]) || !finite(desc->limits[j][1]) || desc->limits[j][0] > desc->limits[j][1])
            return fail(DSEED_EINVAL, "bad limits of joint %d", j + 1);
    }
    for (int k = 0; k < ns; ++k) {
        if (desc->sphere_frame[k] < 1 || desc->sphere_frame[k] > 8)
            return fail(DSEED_EINVAL, "sphere %d: frame %d outside 1..8", k, desc->sphere_frame[k]);
        if (!(desc->sphere_radius[k] > 0.f) || !finite(desc->sphere_radius[k]))
            return fail(DSEED_EINVAL, "sphere %d: radius must be finite and > 0", k);
        for (int c = 0; c < 3; ++c)
            if (!finite(desc->sphere_offset[k][c])) return fail(DSEED_EINVAL, "sphere %d: non-finite offset", k);
    }
    for (int j = 0; j < 7; ++j)
        if (!finite(desc->self_ref[j])) return fail(DSEED_EINVAL, "non-finite self_ref entry %d", j);
    if (!finite(desc->self_margin)) return fail(DSEED_EINVAL, "non-finite self_margin");
    DseedRobot *r = new (std::nothrow) DseedRobot;
    if (!r) return fail(DSEED_ENOMEM, "host allocation of the robot failed");
    std::memset(&r->k, 0, sizeof(r->k));
    dseed::KRobot &k = r->k;
    for (int i = 0; i < 8; ++i) {
        const double al = desc->dh[i][2];
        k.a[i] = desc->dh[i][0];
        k.d[i] = desc->dh[i][1];
        k.ca[i] = (float)std::cos(al);
        k.sa[i] = (float)std::sin(al);
        k.ca2[i] = (float)std::cos(0.5 * al);
        k.sa2[i] = (float)std::sin(0.5 * al);
        k.off[i] = desc->dh[i][3];
    }
    for (int j = 0; j < 7; ++j) {
        k.lo[j] = desc->limits[j][0];
        k.hi[j] = desc->limits[j][1];
    }
    k.n_spheres = ns;
    int idx = 0;
    for (int L = 1; L <= 8; ++L) {
        k.frame_begin[L - 1] = idx;
        for (int s = 0; s < ns; ++s)
            if (desc->sphere_frame[s] == L) {
                k.sph[idx] = make_float4(desc->sphere_offset[s][0], desc->sphere_offset[s][1],
                                         desc->sphere_offset[s][2], desc->sphere_radius[s]);
                k.sph_orig[idx] = s;
                ++idx;
            }
    }
    k.frame_begin[8] = idx;
    // per-frame bounding sphere of the collision spheres: centre = midpoint of
    // their bounding box, radius = max over spheres of |o - centre| + r
    for (int L = 0; L < 8; ++L) {
        const int b = k.frame_begin[L], e = k.frame_begin[L + 1];
        float lo[3] = {0.f, 0.f, 0.f}, hi[3] = {0.f, 0.f, 0.f}, rmin = 0.f, rmax = 0.f;
        for (int q = b; q < e; ++q) {
            const float o[3] = {k.sph[q].x, k.sph[q].y, k.sph[q].z};
            for (int c = 0; c < 3; ++c) {
                lo[c] = q == b ? o[c] : std::min(lo[c], o[c]);
                hi[c] = q == b ? o[c] : std::max(hi[c], o[c]);
            }
            rmin = q == b ? k.sph[q].w : std::min(rmin, k.sph[q].w);
            rmax = q == b ? k.sph[q].w : std::max(rmax, k.sph[q].w);
        }
        double cen[3], rad = 0.0;
        for (int c = 0; c < 3; ++c) cen[c] = 0.5 * ((double)lo[c] + (double)hi[c]);
        for (int q = b; q < e; ++q) {
            const double dx = k.sph[q].x - cen[0], dy = k.sph[q].y - cen[1], dz = k.sph[q].z - cen[2];
            rad = std::max(rad, std::sqrt(dx * dx + dy * dy + dz * dz) + (double)k.sph[q].w);
        }
        // round the radius up so the float value still bounds every sphere
        k.fbound[L] = make_float4((float)cen[0], (float)cen[1], (float)cen[2], (float)(rad * (1.0 + 1e-6) + 1e-6));
        k.frmin[L] = rmin;
        k.frmax[L] = rmax;
    }
    k.cf8 = (float)std::cos((double)desc->dh[7][3]);
    k.sf8 = (float)std::sin((double)desc->dh[7][3]);
    self_pairs(desc, r);
    *out = r;
    return DSEED_OK;
}

int dseed_robot_self_pairs(const DseedRobot *robot, unsigned long long *mask_host, int *n_pairs) {
    if (!robot || !mask_host) return fail(DSEED_EINVAL, "robot or mask is NULL");
    for (int i = 0; i < robot->k.n_spheres; ++i) mask_host[i] = robot->self_mask[i];
    if (n_pairs) *n_pairs = robot->n_self_pairs;
    return DSEED_OK;
}

void dseed_robot_destroy(DseedRobot *robot) { delete robot; }

static int check_esdf_job(const float *cuboids_dev, int n, const DseedGrid *grid, const float *esdf_dev) {
    if (!grid || !esdf_dev) return fail(DSEED_EINVAL, "grid or esdf is NULL");
    if (n < 0 || (n > 0 && !cuboids_dev)) return fail(DSEED_EINVAL, "bad cuboid count or NULL cuboids");
    if (grid->nx < 2 || grid->ny < 2 || grid->nz < 2) return fail(DSEED_EINVAL, "grid dimensions must be >= 2");
    if ((long long)grid->nx * grid->ny * grid->nz > (1LL << 31) - 1)
        return fail(DSEED_EINVAL, "grid of more than 2^31 voxels");
    if (!(grid->res > 0.f) || !finite(grid->res) || !finite(grid->origin[0]) || !finite(grid->origin[1]) ||
        !finite(grid->origin[2]))
        return fail(DSEED_EINVAL, "bad grid origin or resolution");
    return DSEED_OK;
}

int dseed_scene_build_esdf(const float *cuboids_dev, int n, const DseedGrid *grid, float *esdf_dev,
                           cudaStream_t stream) {
    int r = check_esdf_job(cuboids_dev, n, grid, esdf_dev);
    if (r) return r;
    DseedEsdfJob job;
    job.cuboids_dev = cuboids_dev;
    job.n = n;
    job.grid = *grid;
    job.esdf_dev = esdf_dev;
    return cuda_status(dseed::launch_esdf_build(&job, 1, stream), "esdf build");
}

int dseed_scene_build_esdf_batch(const DseedEsdfJob *jobs_host, int n_jobs, cudaStream_t stream) {
    if (n_jobs < 0 || (n_jobs > 0 && !jobs_host)) return fail(DSEED_EINVAL, "bad job count or NULL jobs");
    for (int q = 0; q < n_jobs; ++q) {
        int r = check_esdf_job(jobs_host[q].cuboids_dev, jobs_host[q].n, &jobs_host[q].grid, jobs_host[q].esdf_dev);
        if (r) return fail(r, "job %d: %s", q, g_last_error.c_str());
    }
    return cuda_status(dseed::launch_esdf_build(jobs_host, n_jobs, stream), "esdf build (batch)");
}

int dseed_fk(const DseedRobot *robot, const float *q_dev, int N, float *pose_dev, float *spheres_dev,
             cudaStream_t stream) {
    if (!robot) return fail(DSEED_EINVAL, "robot is NULL");
    if (N < 0) return fail(DSEED_EINVAL, "N < 0");
    if (N > 0 && (!q_dev || !pose_dev)) return fail(DSEED_EINVAL, "q or pose is NULL");
    return cuda_status(dseed::launch_fk(robot->k, q_dev, N, pose_dev, spheres_dev, stream), "fk");
}

int dseed_nn_fk_mse(const DseedRobot *robot, const float *lin_dev, const float *eps_dev, const float *pred_dev,
                    const float *w_dev, int N, int T, float res_scale, float *dpred_dev, float *loss_partial_dev,
                    int blocks, cudaStream_t stream) {
    if (!robot) return fail(DSEED_EINVAL, "robot is NULL");
    if (N < 0 || T < 1 || T > DSEED_MAX_T) return fail(DSEED_EINVAL, "fk_mse: N = %d, T = %d", N, T);
    if (!finite(res_scale) || !(res_scale > 0.f)) return fail(DSEED_EINVAL, "fk_mse: res_scale must be > 0");
    if (blocks < 1 || blocks > 1024) return fail(DSEED_EINVAL, "fk_mse: blocks = %d outside 1..1024", blocks);
    if (!loss_partial_dev || (N > 0 && (!lin_dev || !eps_dev || !pred_dev || !dpred_dev)))
        return fail(DSEED_EINVAL, "fk_mse: a required array is NULL");
    return cuda_status(dseed::launch_fk_mse(robot->k, lin_dev, eps_dev, pred_dev, w_dev, N, T, res_scale, dpred_dev,
                                            loss_partial_dev, blocks, stream),
                       "fk_mse");
}

int dseed_cost(const DseedRobot *robot, const DseedPlanDesc *desc, const DseedProblems *pr, const float *x_dev,
               float *cost_dev, float *terms_dev, cudaStream_t stream) {
    if (!robot) return fail(DSEED_EINVAL, "robot is NULL");
    int r = check_desc(desc, false);
    if (r) return r;
    if ((r = check_problems(desc, pr))) return r;
    if (desc->P > 0 && (!x_dev || !cost_dev)) return fail(DSEED_EINVAL, "x or cost is NULL");
    return cuda_status(dseed::launch_cost(robot->k, make_cost(desc->cost), make_batch(desc, pr), x_dev, cost_dev,
                                          terms_dev, stream),
                       "cost");
}

int dseed_cost_grad(const DseedRobot *robot, const DseedPlanDesc *desc, const DseedProblems *pr, const float *x_dev,
                    const float *grad_scale_dev, float *cost_dev, float *grad_dev, cudaStream_t stream) {
    if (!robot) return fail(DSEED_EINVAL, "robot is NULL");
    int r = check_desc(desc, false);
    if (r) return r;
    if ((r = check_problems(desc, pr))) return r;
    if (desc->P > 0 && (!x_dev || !cost_dev || !grad_dev)) return fail(DSEED_EINVAL, "x, cost or grad is NULL");
    return cuda_status(dseed::launch_cost_grad(robot->k, make_cost(desc->cost), make_batch(desc, pr), x_dev,
                                               grad_scale_dev, cost_dev, grad_dev, stream),
                       "cost_grad");
}

int dseed_evaluate(const DseedRobot *robot, const DseedPlanDesc *desc, const DseedProblems *pr, const float *x_dev,
                   uint8_t *success_dev, float *metrics_dev, cudaStream_t stream) {
    if (!robot) return fail(DSEED_EINVAL, "robot is NULL");
    int r = check_desc(desc, false);
    if (r) return r;
    if ((r = check_problems(desc, pr))) return r;
    if (desc->P > 0 && (!x_dev || !success_dev)) return fail(DSEED_EINVAL, "x or success is NULL");
    return cuda_status(dseed::launch_evaluate(robot->k, make_cost(desc->cost), make_batch(desc, pr), x_dev,
                                              success_dev, metrics_dev, stream),
                       "evaluate");
}

int dseed_lbfgs_layout(const DseedPlanDesc *desc, DseedLbfgsLayout *out) {
    int r = check_desc(desc, true);
    if (r) return r;
    if (!out) return fail(DSEED_EINVAL, "out is NULL");
    *out = lbfgs_layout((long long)desc->P * desc->S, 7 * desc->T, desc->opt.m);
    return DSEED_OK;
}

int dseed_lbfgs_init(const DseedPlanDesc *desc, const float *x0_dev, void *state_dev, cudaStream_t stream) {
    int r = check_desc(desc, true);
    if (r) return r;
    const long long B = (long long)desc->P * desc->S;
    if (B > 0 && (!x0_dev || !state_dev)) return fail(DSEED_EINVAL, "x0 or state is NULL");
    const DseedLbfgsLayout l = lbfgs_layout(B, 7 * desc->T, desc->opt.m);
    return cuda_status(dseed::launch_lbfgs_init((int)B, 7 * desc->T, x0_dev, lbfgs_ptrs(state_dev, l), desc->opt.m,
                                                stream),
                       "lbfgs init");
}

int dseed_lbfgs_step(const DseedPlanDesc *desc, const float *f_trial_dev, const float *g_trial_dev, void *state_dev,
                     cudaStream_t stream) {
    int r = check_desc(desc, true);
    if (r) return r;
    const long long B = (long long)desc->P * desc->S;
    if (B > 0 && (!f_trial_dev || !g_trial_dev || !state_dev)) return fail(DSEED_EINVAL, "f, g or state is NULL");
    const DseedLbfgsLayout l = lbfgs_layout(B, 7 * desc->T, desc->opt.m);
    return cuda_status(dseed::launch_lbfgs_step(make_opt(desc->opt), (int)B, desc->T, f_trial_dev, g_trial_dev,
                                                lbfgs_ptrs(state_dev, l), stream),
                       "lbfgs step");
}

int dseed_plan_workspace_bytes(const DseedPlanDesc *desc, size_t *bytes) {
    int r = check_desc(desc, true);
    if (r) return r;
    if (!bytes) return fail(DSEED_EINVAL, "bytes is NULL");
    *bytes = plan_layout(desc).total;
    return DSEED_OK;
}

int dseed_plan_batch(const DseedRobot *robot, const DseedPlanDesc *desc, const DseedProblems *pr,
                     const float *seeds_dev, void *workspace_dev, size_t workspace_bytes, float *traj_dev,
                     float *cost_dev, uint8_t *success_dev, float *metrics_dev, int *best_dev, cudaStream_t stream) {
    if (!robot) return fail(DSEED_EINVAL, "robot is NULL");
    int r = check_desc(desc, true);
    if (r) return r;
    if ((r = check_problems(desc, pr))) return r;
    if (desc->P == 0) return DSEED_OK;
    if (!seeds_dev || !workspace_dev || !traj_dev || !cost_dev || !success_dev || !best_dev)
        return fail(DSEED_EINVAL, "a plan buffer is NULL");
    if (reinterpret_cast<uintptr_t>(workspace_dev) % 256 != 0) return fail(DSEED_EINVAL, "workspace not 256-byte aligned");
    const PlanLayout l = plan_layout(desc);
    if (workspace_bytes < l.total)
        return fail(DSEED_ENOMEM, "workspace of %zu bytes, %zu needed", workspace_bytes, l.total);
    char *w = static_cast<char *>(workspace_dev);
    return cuda_status(dseed::launch_plan(robot->k, make_cost(desc->cost), make_opt(desc->opt), make_batch(desc, pr),
                                          seeds_dev, reinterpret_cast<float *>(w + l.s),
                                          reinterpret_cast<float *>(w + l.y), reinterpret_cast<float *>(w + l.d),
                                          reinterpret_cast<unsigned long long *>(w + l.key), traj_dev, cost_dev,
                                          success_dev, metrics_dev, best_dev, stream),
                       "plan");
}

}  // extern "C"

// ---------------------------------------------------------------- plan without allocation
// Scratch of dseed_plan_batch_static: one file-scope device array.  Host code
// may not use the symbol as an address (on the host it names a stand-in);
// its device address is looked up once per device with that device current.
static __device__ __align__(256) unsigned char g_plan_scratch[DSEED_STATIC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_scratch_mutex;
// per device: the array's address and the id of the context it was looked up in
struct ScratchSlot {
    void *ptr = nullptr;
    unsigned long long ctx_id = 0;
    bool valid = false;
};
ScratchSlot g_scratch[kMaxDevices];

// Unique id (for the process lifetime) of the current context, 0 when none is
// current.  A device reset destroys the context that an address was looked up
// in, and the next context may load the module elsewhere, so the cached address
// is only reused while the context id matches.
unsigned long long current_ctx_id() {
    static PFN_cuCtxGetCurrent_v4000 get_current = nullptr;
    static PFN_cuCtxGetId_v12000 get_id = nullptr;
    static bool resolved = false;
    if (!resolved) {
        cudaDriverEntryPointQueryResult q1, q2;
        void *f1 = nullptr, *f2 = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
            q1 == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(f1);
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
            q2 == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<PFN_cuCtxGetId_v12000>(f2);
        resolved = true;
    }
    if (!get_current || !get_id) return 0;
    CUcontext ctx = nullptr;
    if (get_current(&ctx) != CUDA_SUCCESS || !ctx) return 0;
    unsigned long long id = 0;
    return get_id(ctx, &id) == CUDA_SUCCESS ? id : 0;
}

int static_scratch(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(DSEED_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return fail(DSEED_EINVAL, "device %d beyond the %d supported", dev, kMaxDevices);
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    ScratchSlot &slot = g_scratch[dev];
    const unsigned long long id = current_ctx_id();
    if (!slot.valid || id == 0 || slot.ctx_id != id) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_plan_scratch);     // makes the device's primary context current if needed
        if (e != cudaSuccess)
            return fail(DSEED_ECUDA, "cudaGetSymbolAddress of the static scratch: %s", cudaGetErrorString(e));
        slot.ptr = p;
        slot.ctx_id = current_ctx_id();
        slot.valid = true;
    }
    *out = slot.ptr;
    return DSEED_OK;
}
}  // namespace

extern "C" int dseed_plan_batch_static(const DseedRobot *robot, const DseedPlanDesc *desc, const DseedProblems *pr,
                                       const float *seeds_dev, float *traj_dev, float *cost_dev,
                                       uint8_t *success_dev, float *metrics_dev, int *best_dev, cudaStream_t stream) {
    if (!robot) return fail(DSEED_EINVAL, "robot is NULL");
    int r = check_desc(desc, true);
    if (r) return r;
    if ((r = check_problems(desc, pr))) return r;
    if (desc->P == 0) return DSEED_OK;
    if (!seeds_dev || !traj_dev || !cost_dev || !success_dev || !best_dev)
        return fail(DSEED_EINVAL, "a plan buffer is NULL");
    const PlanLayout l = plan_layout(desc);
    if (l.total > (size_t)DSEED_STATIC_SCRATCH_BYTES)
        return fail(DSEED_ENOMEM, "batch needs %zu bytes of scratch, the static scratch holds %zu", l.total,
                    (size_t)DSEED_STATIC_SCRATCH_BYTES);
    void *base = nullptr;
    if ((r = static_scratch(&base))) return r;
    char *w = static_cast<char *>(base);
    // launch_plan resets the best-seed keys; the history is written before it is read
    return cuda_status(dseed::launch_plan(robot->k, make_cost(desc->cost), make_opt(desc->opt), make_batch(desc, pr),
                                          seeds_dev, reinterpret_cast<float *>(w + l.s),
                                          reinterpret_cast<float *>(w + l.y), reinterpret_cast<float *>(w + l.d),
                                          reinterpret_cast<unsigned long long *>(w + l.key), traj_dev, cost_dev,
                                          success_dev, metrics_dev, best_dev, stream),
                       "plan (static scratch)");
}
