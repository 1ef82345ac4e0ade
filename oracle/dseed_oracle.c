/*
 * dseed_oracle.c -- FP64 CPU oracle for seed-parallel trajectory optimisation.
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the test suite, the smoke check
 * and the benchmark's CPU-baseline leg load this library.  It shares no code,
 * header, table or constant with the CUDA path: every quantity below is written
 * out from its definition, in double precision, in the plainest form that can
 * be checked against the text by eye.  Loops run in index order; the only
 * parallelism is OpenMP over independent seeds in orc_plan().
 *
 * What it computes (the optimisation problem of the paper's Appendix A.5
 * "Optimization Problem": minimise C_goal(X_d, FK(q_T)) + C_smooth + C_world
 * subject to joint limits, over many seed trajectories, each refined by
 * L-BFGS).  The paper leaves the cost forms, weights, kinematic model and
 * optimiser details to its motion optimiser; the readings used here are:
 *   - kinematics: modified DH chain of a 7-DoF Franka Panda + fixed flange,
 *   - world cost: linear hinge w_c * max(0, r + eta - phi(c)) per sphere and
 *     waypoint, phi = trilinear interpolation of a voxel ESDF,
 *   - smoothness: squared backward finite differences (vel/acc/jerk) with the
 *     start held at rest,
 *   - goal: w_p |p - p*|^2 + w_R (1 - <q, q*>^2) at the last waypoint,
 *   - joint limits: quadratic penalty outside [lower, upper],
 *   - self collision (C_self, optional): linear hinge w_s * max(0, r_i + r_j +
 *     eta_s - |c_i - c_j|) over the sphere pairs the robot marks as checked,
 *   - swept collision (optional): the world hinge also at n_sweep joint-space
 *     interpolants of every segment between consecutive waypoints (the robot
 *     executes the trajectory by linear interpolation between waypoints),
 *   - success (Sec. 5.1 and Appendix A.6): collision free, translation error
 *     below delta_t, rotation error below delta_r, within limits,
 *   - optimiser: L-BFGS (history m) with Armijo accept/reject and step halving.
 *
 * Parity pins (tests/test_oracle_*.py): FK closed forms at q = 0 and at the
 * home pose; analytic point-to-box distances; exact trilinear interpolation of
 * affine fields; exact finite differences of polynomials; central-difference
 * gradients; L-BFGS on a convex quadratic against a direct solve.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Types shared with the ctypes wrapper (oracle/oracle.py)                  */
/* ------------------------------------------------------------------------ */

typedef struct {
    const double *dh;        /* [8][4]: a, d, alpha, theta_offset (modified DH) */
    const double *lim;       /* [7][2]: lower, upper (rad) */
    int ns;                  /* number of collision spheres */
    const int *sph_frame;    /* [ns]: frame 1..8 the sphere is fixed to */
    const double *sph_o;     /* [ns][3]: offset in that frame */
    const double *sph_r;     /* [ns]: radius */
    const unsigned char *self_pair;  /* [ns][ns]: 1 = pair checked for self-collision (or NULL) */
} orc_robot;

typedef struct {
    double w_c, eta, dt, w_v, w_a, w_j, w_p, w_R, w_l;
    double w_s, eta_s;       /* self-collision hinge weight and margin (w_s = 0: off) */
    int n_sweep;             /* interpolants checked per segment (0: waypoints only) */
} orc_cost_params;

typedef struct {
    const double *phi;       /* [nz][ny][nx], x fastest */
    double origin[3];        /* corner of the grid (m) */
    double res;              /* voxel edge (m) */
    int n[3];                /* nx, ny, nz */
} orc_grid;

typedef struct {
    const orc_robot *robot;
    const orc_cost_params *cp;
    const orc_grid *grid;
    const double *q_start;   /* [7]: y_0, held fixed */
    const double *goal;      /* [7]: x, y, z, qw, qx, qy, qz */
    int T;                   /* waypoints optimised: y_1 .. y_T */
} orc_problem;

typedef struct {
    int iters;               /* cost+gradient evaluations */
    int m;                   /* history length */
    double c1;               /* Armijo constant */
    double max_step;         /* cap on max |step| */
    double gamma0;           /* H0 scale with an empty history */
    double alpha_min;        /* clear the history when the step falls below this */
} orc_opt;

#define ORC_FAR 1000.0       /* ESDF value with no obstacle */

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads of the calling thread's later parallel loops over seeds (n >= 1);
 * every seed is planned by one thread, so the results do not depend on it. */
void orc_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n >= 1) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ------------------------------------------------------------------------ */
/* Small linear algebra on 4x4 homogeneous transforms (row-major)           */
/* ------------------------------------------------------------------------ */

static void mat4_identity(double M[16])
{
    memset(M, 0, 16 * sizeof(double));
    M[0] = M[5] = M[10] = M[15] = 1.0;
}

static void mat4_mul(const double A[16], const double B[16], double C[16])
{
    double tmp[16];
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) {
            double s = 0.0;
            for (int k = 0; k < 4; ++k) s += A[4 * r + k] * B[4 * k + c];
            tmp[4 * r + c] = s;
        }
    memcpy(C, tmp, sizeof(tmp));
}

static void rot_x(double a, double M[16])
{
    mat4_identity(M);
    M[5] = cos(a); M[6] = -sin(a);
    M[9] = sin(a); M[10] = cos(a);
}

static void rot_z(double a, double M[16])
{
    mat4_identity(M);
    M[0] = cos(a); M[1] = -sin(a);
    M[4] = sin(a); M[5] = cos(a);
}

static void trans_x(double a, double M[16]) { mat4_identity(M); M[3] = a; }
static void trans_z(double d, double M[16]) { mat4_identity(M); M[11] = d; }

static void cross3(const double a[3], const double b[3], double c[3])
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

static double dot3(const double a[3], const double b[3])
{
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

/* ------------------------------------------------------------------------ */
/* Forward kinematics (FK in Eq. 2 and in C_goal(X_d, FK(q_T)), App. A.5)    */
/* ------------------------------------------------------------------------ */

/* Frames 0..8 of the chain as 4x4 transforms: frame 0 is the base, frame i
 * (i = 1..7) moves with joint i, frame 8 is the flange.  Modified DH:
 *   T_i = T_{i-1} * RotX(alpha_i) * TransX(a_i) * RotZ(theta_i) * TransZ(d_i),
 * theta_i = q_i + offset_i for the seven joints and offset_8 for the flange. */
void orc_fk(const double *dh, const double *q, double *frames /* [9][16] */)
{
    double A[16], B[16];
    mat4_identity(frames);
    for (int i = 1; i <= 8; ++i) {
        const double *row = dh + 4 * (i - 1);
        double a = row[0], d = row[1], alpha = row[2], off = row[3];
        double theta = (i <= 7 ? q[i - 1] : 0.0) + off;
        memcpy(A, frames + 16 * (i - 1), sizeof(A));
        rot_x(alpha, B);   mat4_mul(A, B, A);
        trans_x(a, B);     mat4_mul(A, B, A);
        rot_z(theta, B);   mat4_mul(A, B, A);
        trans_z(d, B);     mat4_mul(A, B, A);
        memcpy(frames + 16 * i, A, sizeof(A));
    }
}

static void frame_origin(const double *F, double p[3]) { p[0] = F[3]; p[1] = F[7]; p[2] = F[11]; }
static void frame_zaxis(const double *F, double z[3]) { z[0] = F[2]; z[1] = F[6]; z[2] = F[10]; }

/* Sphere centre: c = R_L o + p_L for the frame L the sphere is fixed to. */
static void sphere_centre(const double *frames, int L, const double o[3], double c[3])
{
    const double *F = frames + 16 * L;
    for (int r = 0; r < 3; ++r)
        c[r] = F[4 * r + 0] * o[0] + F[4 * r + 1] * o[1] + F[4 * r + 2] * o[2] + F[4 * r + 3];
}

void orc_sphere_centres(const orc_robot *rb, const double *q, double *c /* [ns][3] */)
{
    double frames[9 * 16];
    orc_fk(rb->dh, q, frames);
    for (int k = 0; k < rb->ns; ++k)
        sphere_centre(frames, rb->sph_frame[k], rb->sph_o + 3 * k, c + 3 * k);
}

/* Sphere pairs checked for self-collision: spheres fixed to frames at least two
 * apart (a frame and its neighbours in the chain are never tested against each
 * other) whose surfaces are at least `margin` apart at the reference
 * configuration q_ref (pairs that are close there overlap by construction of
 * the sphere model).  mask[i * ns + j] = mask[j * ns + i] = 1 for such pairs. */
int orc_self_pairs(const orc_robot *rb, const double *q_ref, double margin, unsigned char *mask)
{
    int ns = rb->ns, count = 0;
    double *c = (double *)malloc(sizeof(double) * 3 * ns);
    orc_sphere_centres(rb, q_ref, c);
    memset(mask, 0, (size_t)ns * ns);
    for (int i = 0; i < ns; ++i)
        for (int j = i + 1; j < ns; ++j) {
            int df = rb->sph_frame[i] - rb->sph_frame[j];
            if (df < 2 && df > -2) continue;
            double d[3] = { c[3 * i] - c[3 * j], c[3 * i + 1] - c[3 * j + 1], c[3 * i + 2] - c[3 * j + 2] };
            double gap = sqrt(dot3(d, d)) - rb->sph_r[i] - rb->sph_r[j];
            if (gap >= margin) {
                mask[i * ns + j] = mask[j * ns + i] = 1;
                ++count;
            }
        }
    free(c);
    return count;
}

/* Unit quaternion (w, x, y, z) of a rotation matrix, taking the square root of
 * the largest of 1 + trace and 1 + 2 R_ii - trace for stability; w >= 0. */
static void mat_to_quat(const double *F, double qout[4])
{
    double R00 = F[0], R01 = F[1], R02 = F[2];
    double R10 = F[4], R11 = F[5], R12 = F[6];
    double R20 = F[8], R21 = F[9], R22 = F[10];
    double tr = R00 + R11 + R22, w, x, y, z;
    if (tr >= R00 && tr >= R11 && tr >= R22) {
        w = 0.5 * sqrt(1.0 + tr);
        x = (R21 - R12) / (4.0 * w); y = (R02 - R20) / (4.0 * w); z = (R10 - R01) / (4.0 * w);
    } else if (R00 >= R11 && R00 >= R22) {
        x = 0.5 * sqrt(1.0 + R00 - R11 - R22);
        w = (R21 - R12) / (4.0 * x); y = (R01 + R10) / (4.0 * x); z = (R02 + R20) / (4.0 * x);
    } else if (R11 >= R22) {
        y = 0.5 * sqrt(1.0 - R00 + R11 - R22);
        w = (R02 - R20) / (4.0 * y); x = (R01 + R10) / (4.0 * y); z = (R12 + R21) / (4.0 * y);
    } else {
        z = 0.5 * sqrt(1.0 - R00 - R11 + R22);
        w = (R10 - R01) / (4.0 * z); x = (R02 + R20) / (4.0 * z); y = (R12 + R21) / (4.0 * z);
    }
    double nrm = sqrt(w * w + x * x + y * y + z * z);
    double s = (w < 0.0 ? -1.0 : 1.0) / nrm;
    qout[0] = w * s; qout[1] = x * s; qout[2] = y * s; qout[3] = z * s;
}

/* End-effector pose (problem statement, Sec. 3: translation + quaternion):
 * flange origin and orientation, [x, y, z, qw, qx, qy, qz]. */
void orc_flange_pose(const double *dh, const double *q, double *pose)
{
    double frames[9 * 16];
    orc_fk(dh, q, frames);
    frame_origin(frames + 16 * 8, pose);
    mat_to_quat(frames + 16 * 8, pose + 3);
}

/* ------------------------------------------------------------------------ */
/* ESDF from cuboids and its trilinear lookup                                */
/* ------------------------------------------------------------------------ */

/* Signed distance to one axis-aligned box (centre c, half extents h): the
 * Euclidean distance to the box outside it, minus the depth of penetration
 * inside it.  box = [cx, cy, cz, hx, hy, hz]. */
static double box_sdf(const double *box, const double p[3])
{
    double d[3], out = 0.0, in = -INFINITY;
    for (int i = 0; i < 3; ++i) {
        d[i] = fabs(p[i] - box[i]) - box[3 + i];
        double e = d[i] > 0.0 ? d[i] : 0.0;
        out += e * e;
        if (d[i] > in) in = d[i];
    }
    return sqrt(out) + (in < 0.0 ? in : 0.0);
}

/* Euclidean signed distance field of a union of boxes on a voxel grid: at the
 * centre of voxel (i, j, k), origin + (i + 1/2, j + 1/2, k + 1/2) * res, the
 * minimum over boxes of the box SDF (ORC_FAR when there is no box).  Storage
 * index ((k * ny) + j) * nx + i. */
void orc_esdf_build(const double *boxes, int nbox, const orc_grid *g, double *phi)
{
    int nx = g->n[0], ny = g->n[1], nz = g->n[2];
    #pragma omp parallel for schedule(static)
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                double p[3] = { g->origin[0] + (i + 0.5) * g->res,
                                g->origin[1] + (j + 0.5) * g->res,
                                g->origin[2] + (k + 0.5) * g->res };
                double best = ORC_FAR;
                for (int b = 0; b < nbox; ++b) {
                    double s = box_sdf(boxes + 6 * b, p);
                    if (s < best) best = s;
                }
                phi[((size_t)k * ny + j) * nx + i] = best;
            }
}

/* Trilinear interpolation of phi at p, and its gradient.  Continuous voxel
 * coordinate u = (p - origin) / res - 1/2 per axis, clamped to [0, n - 1]; the
 * cell is i0 = min(floor(u), n - 2) with fraction f = u - i0.  The value is the
 * sum over the 8 cell corners of phi times the product of the 1-D hat weights
 * (1 - f or f); the gradient differentiates those weights and divides by res,
 * and is zero along an axis where p lies outside the grid (u was clamped). */
double orc_esdf_lookup(const orc_grid *g, const double p[3], double *grad)
{
    int i0[3], clamped[3];
    double f[3];
    for (int a = 0; a < 3; ++a) {
        double u = (p[a] - g->origin[a]) / g->res - 0.5;
        double hi = (double)(g->n[a] - 1);
        clamped[a] = (u < 0.0 || u > hi);
        if (u < 0.0) u = 0.0;
        if (u > hi) u = hi;
        int c = (int)floor(u);
        if (c > g->n[a] - 2) c = g->n[a] - 2;
        i0[a] = c;
        f[a] = u - c;
    }
    double val = 0.0, dv[3] = { 0.0, 0.0, 0.0 };
    for (int dz = 0; dz < 2; ++dz)
        for (int dy = 0; dy < 2; ++dy)
            for (int dx = 0; dx < 2; ++dx) {
                int idx[3] = { dx, dy, dz };
                double w[3], dw[3];
                for (int a = 0; a < 3; ++a) {
                    w[a] = idx[a] ? f[a] : 1.0 - f[a];
                    dw[a] = idx[a] ? 1.0 : -1.0;
                }
                double v = g->phi[((size_t)(i0[2] + dz) * g->n[1] + (i0[1] + dy)) * g->n[0] + (i0[0] + dx)];
                val += v * w[0] * w[1] * w[2];
                dv[0] += v * dw[0] * w[1] * w[2];
                dv[1] += v * w[0] * dw[1] * w[2];
                dv[2] += v * w[0] * w[1] * dw[2];
            }
    if (grad)
        for (int a = 0; a < 3; ++a) grad[a] = clamped[a] ? 0.0 : dv[a] / g->res;
    return val;
}

/* ------------------------------------------------------------------------ */
/* Cost and gradient of one seed trajectory (App. A.5 objective)             */
/* ------------------------------------------------------------------------ */

/* Waypoint t of the padded trajectory: y_t = x_t for t >= 1; the start y_0 and
 * the two earlier pads y_{-1}, y_{-2} all equal q_start (start at rest). */
static double traj_y(const orc_problem *pb, const double *x, int t, int j)
{
    return t >= 1 ? x[7 * (t - 1) + j] : pb->q_start[j];
}

static void quat_normalise(const double *in, double out[4])
{
    double n = sqrt(in[0] * in[0] + in[1] * in[1] + in[2] * in[2] + in[3] * in[3]);
    for (int i = 0; i < 4; ++i) out[i] = in[i] / n;
}

/* World hinge at one configuration q[7]: sum over spheres of
 * w_c * max(0, r + eta - phi(c)).  gq (optional) receives its derivative with
 * respect to q; min_clear (optional) is lowered to min over spheres of phi - r. */
static double world_hinge(const orc_problem *pb, const double *q, double *gq, double *min_clear)
{
    const orc_robot *rb = pb->robot;
    const orc_cost_params *cp = pb->cp;
    double frames[9 * 16], zax[8][3], org[8][3], c_world = 0.0;
    orc_fk(rb->dh, q, frames);
    for (int i = 1; i <= 7; ++i) {
        frame_zaxis(frames + 16 * i, zax[i]);
        frame_origin(frames + 16 * i, org[i]);
    }
    if (gq) memset(gq, 0, sizeof(double) * 7);
    for (int k = 0; k < rb->ns; ++k) {
        int L = rb->sph_frame[k];
        double c[3], gphi[3];
        sphere_centre(frames, L, rb->sph_o + 3 * k, c);
        double phi = orc_esdf_lookup(pb->grid, c, gphi);
        if (min_clear && phi - rb->sph_r[k] < *min_clear) *min_clear = phi - rb->sph_r[k];
        double h = rb->sph_r[k] + cp->eta - phi;
        if (h <= 0.0) continue;
        c_world += cp->w_c * h;
        if (!gq) continue;
        double dc[3] = { -cp->w_c * gphi[0], -cp->w_c * gphi[1], -cp->w_c * gphi[2] };
        int top = L < 7 ? L : 7;
        for (int i = 1; i <= top; ++i) {
            double r[3] = { c[0] - org[i][0], c[1] - org[i][1], c[2] - org[i][2] }, J[3];
            cross3(zax[i], r, J);
            gq[i - 1] += dot3(dc, J);
        }
    }
    return c_world;
}

/* Interpolant j (1..n_sweep) of segment t (1..T): q = (1 - u) y_t + u y_{t-1},
 * u = j / (n_sweep + 1); returns u. */
static double sweep_config(const orc_problem *pb, const double *x, int t, int j, double q[7])
{
    double u = (double)j / (double)(pb->cp->n_sweep + 1);
    for (int i = 0; i < 7; ++i) q[i] = (1.0 - u) * traj_y(pb, x, t, i) + u * traj_y(pb, x, t - 1, i);
    return u;
}

/* Total cost of x = [T][7] (waypoints 1..T).  grad (optional) receives dC/dx,
 * terms (optional) receives [C_world (+ C_self), C_smooth, C_goal, C_limit]. */
double orc_cost(const orc_problem *pb, const double *x, double *grad, double *terms)
{
    const orc_robot *rb = pb->robot;
    const orc_cost_params *cp = pb->cp;
    int T = pb->T;
    double c_world = 0.0, c_smooth = 0.0, c_goal = 0.0, c_limit = 0.0;
    if (grad) memset(grad, 0, sizeof(double) * 7 * T);

    /* C_smooth: for t = 1..T, squared velocity, acceleration and jerk by
     * backward differences at spacing dt. */
    static const double sv[2] = { 1.0, -1.0 };
    static const double sa[3] = { 1.0, -2.0, 1.0 };
    static const double sj[4] = { 1.0, -3.0, 3.0, -1.0 };
    double dt = cp->dt;
    for (int t = 1; t <= T; ++t)
        for (int j = 0; j < 7; ++j) {
            double v = 0.0, a = 0.0, jk = 0.0;
            for (int s = 0; s < 2; ++s) v += sv[s] * traj_y(pb, x, t - s, j);
            for (int s = 0; s < 3; ++s) a += sa[s] * traj_y(pb, x, t - s, j);
            for (int s = 0; s < 4; ++s) jk += sj[s] * traj_y(pb, x, t - s, j);
            v /= dt; a /= dt * dt; jk /= dt * dt * dt;
            c_smooth += cp->w_v * v * v + cp->w_a * a * a + cp->w_j * jk * jk;
            if (grad) {
                for (int s = 0; s < 2; ++s) if (t - s >= 1) grad[7 * (t - s - 1) + j] += 2.0 * cp->w_v * v * sv[s] / dt;
                for (int s = 0; s < 3; ++s) if (t - s >= 1) grad[7 * (t - s - 1) + j] += 2.0 * cp->w_a * a * sa[s] / (dt * dt);
                for (int s = 0; s < 4; ++s) if (t - s >= 1) grad[7 * (t - s - 1) + j] += 2.0 * cp->w_j * jk * sj[s] / (dt * dt * dt);
            }
        }

    /* joint limits: quadratic penalty outside [lower, upper] */
    for (int t = 1; t <= T; ++t)
        for (int j = 0; j < 7; ++j) {
            double q = x[7 * (t - 1) + j], lo = rb->lim[2 * j], hi = rb->lim[2 * j + 1];
            if (q > hi) {
                c_limit += cp->w_l * (q - hi) * (q - hi);
                if (grad) grad[7 * (t - 1) + j] += 2.0 * cp->w_l * (q - hi);
            } else if (q < lo) {
                c_limit += cp->w_l * (lo - q) * (lo - q);
                if (grad) grad[7 * (t - 1) + j] -= 2.0 * cp->w_l * (lo - q);
            }
        }

    /* C_world (and C_self) at every waypoint, and C_goal at the last one */
    double frames[9 * 16];
    const int use_self = cp->w_s > 0.0 && rb->self_pair != NULL;
    double *cent = use_self ? (double *)malloc(sizeof(double) * 3 * rb->ns) : NULL;
    for (int t = 1; t <= T; ++t) {
        const double *q = x + 7 * (t - 1);
        orc_fk(rb->dh, q, frames);
        double zax[8][3], org[8][3];
        for (int i = 1; i <= 7; ++i) {
            frame_zaxis(frames + 16 * i, zax[i]);
            frame_origin(frames + 16 * i, org[i]);
        }
        if (use_self) {
            /* C_self: for each checked pair, w_s * max(0, r_i + r_j + eta_s - |c_i - c_j|);
             * dC/dc_i = -w_s (c_i - c_j) / |c_i - c_j| = -dC/dc_j, through the joints
             * that move each sphere (velocity z_m x (c - p_m) per unit angle) */
            for (int k = 0; k < rb->ns; ++k)
                sphere_centre(frames, rb->sph_frame[k], rb->sph_o + 3 * k, cent + 3 * k);
            for (int i = 0; i < rb->ns; ++i)
                for (int j = i + 1; j < rb->ns; ++j) {
                    if (!rb->self_pair[i * rb->ns + j]) continue;
                    double d[3] = { cent[3 * i] - cent[3 * j], cent[3 * i + 1] - cent[3 * j + 1],
                                    cent[3 * i + 2] - cent[3 * j + 2] };
                    double dist = sqrt(dot3(d, d));
                    double h = rb->sph_r[i] + rb->sph_r[j] + cp->eta_s - dist;
                    if (h <= 0.0) continue;
                    c_world += cp->w_s * h;
                    if (!grad) continue;
                    for (int side = 0; side < 2; ++side) {
                        int k = side == 0 ? i : j;
                        double sgn = side == 0 ? -1.0 : 1.0;
                        double dc[3] = { sgn * cp->w_s * d[0] / dist, sgn * cp->w_s * d[1] / dist,
                                         sgn * cp->w_s * d[2] / dist };
                        int L = rb->sph_frame[k], top = L < 7 ? L : 7;
                        for (int m = 1; m <= top; ++m) {
                            double r[3] = { cent[3 * k] - org[m][0], cent[3 * k + 1] - org[m][1],
                                            cent[3 * k + 2] - org[m][2] }, J[3];
                            cross3(zax[m], r, J);
                            grad[7 * (t - 1) + (m - 1)] += dot3(dc, J);
                        }
                    }
                }
        }
        for (int k = 0; k < rb->ns; ++k) {
            int L = rb->sph_frame[k];
            double c[3], gphi[3];
            sphere_centre(frames, L, rb->sph_o + 3 * k, c);
            double phi = orc_esdf_lookup(pb->grid, c, gphi);
            double h = rb->sph_r[k] + cp->eta - phi;
            if (h > 0.0) {
                c_world += cp->w_c * h;
                if (grad) {
                    /* dC/dc = -w_c grad(phi); joint i (<= L) moves c with
                     * velocity z_i x (c - p_i) per unit angle */
                    double dc[3] = { -cp->w_c * gphi[0], -cp->w_c * gphi[1], -cp->w_c * gphi[2] };
                    int top = L < 7 ? L : 7;
                    for (int i = 1; i <= top; ++i) {
                        double r[3] = { c[0] - org[i][0], c[1] - org[i][1], c[2] - org[i][2] }, J[3];
                        cross3(zax[i], r, J);
                        grad[7 * (t - 1) + (i - 1)] += dot3(dc, J);
                    }
                }
            }
        }
        if (t == T) {
            double p[3], qe[4], qd[4];
            frame_origin(frames + 16 * 8, p);
            mat_to_quat(frames + 16 * 8, qe);
            quat_normalise(pb->goal + 3, qd);
            double e[3] = { p[0] - pb->goal[0], p[1] - pb->goal[1], p[2] - pb->goal[2] };
            double dq = qe[0] * qd[0] + qe[1] * qd[1] + qe[2] * qd[2] + qe[3] * qd[3];
            c_goal = cp->w_p * dot3(e, e) + cp->w_R * (1.0 - dq * dq);
            if (grad)
                for (int i = 1; i <= 7; ++i) {
                    double r[3] = { p[0] - org[i][0], p[1] - org[i][1], p[2] - org[i][2] }, J[3];
                    cross3(zax[i], r, J);
                    /* rotating about the world axis z_i: dq/dtheta = 1/2 (0, z_i) (x) q */
                    const double *z = zax[i];
                    double dqe[4] = {
                        0.5 * (-(z[0] * qe[1] + z[1] * qe[2] + z[2] * qe[3])),
                        0.5 * (z[0] * qe[0] + (z[1] * qe[3] - z[2] * qe[2])),
                        0.5 * (z[1] * qe[0] + (z[2] * qe[1] - z[0] * qe[3])),
                        0.5 * (z[2] * qe[0] + (z[0] * qe[2] - z[1] * qe[1])),
                    };
                    double ddq = dqe[0] * qd[0] + dqe[1] * qd[1] + dqe[2] * qd[2] + dqe[3] * qd[3];
                    grad[7 * (T - 1) + (i - 1)] += 2.0 * cp->w_p * dot3(e, J) - 2.0 * cp->w_R * dq * ddq;
                }
        }
    }
    free(cent);

    /* swept collision: the world hinge at the interpolants of every segment
     * (y_{t-1}, y_t), t = 1..T; the derivative g at q reaches y_t with weight
     * 1 - u and y_{t-1} (when it is optimised, t >= 2) with weight u */
    for (int t = 1; t <= T; ++t)
        for (int j = 1; j <= cp->n_sweep; ++j) {
            double q[7], gq[7];
            double u = sweep_config(pb, x, t, j, q);
            c_world += world_hinge(pb, q, grad ? gq : NULL, NULL);
            if (!grad) continue;
            for (int i = 0; i < 7; ++i) {
                grad[7 * (t - 1) + i] += (1.0 - u) * gq[i];
                if (t >= 2) grad[7 * (t - 2) + i] += u * gq[i];
            }
        }
    if (terms) { terms[0] = c_world; terms[1] = c_smooth; terms[2] = c_goal; terms[3] = c_limit; }
    return c_world + c_smooth + c_goal + c_limit;
}

/* ------------------------------------------------------------------------ */
/* Success test and trajectory metrics (Sec. 5.1, Appendix A.6)              */
/* ------------------------------------------------------------------------ */

/* metrics[7] = min over waypoints/spheres of (phi - r) (and, with the self cost
 * on, of the checked pairs' |c_i - c_j| - r_i - r_j; with n_sweep > 0, also over
 * the segments' interpolants and spheres), translation error |p - p*|,
 * rotation error 2 acos(|<q, q*>|), max |jerk| over waypoints and joints,
 * worst joint-limit violation, total cost, 1/0 collision free.
 * thr = [delta_t, delta_r].  Returns 1 on success. */
int orc_evaluate(const orc_problem *pb, const double *x, const double *thr, double *metrics)
{
    const orc_robot *rb = pb->robot;
    int T = pb->T;
    double frames[9 * 16], min_clear = INFINITY, max_jerk = 0.0, lim_viol = 0.0;
    for (int t = 1; t <= T; ++t) {
        orc_fk(rb->dh, x + 7 * (t - 1), frames);
        for (int k = 0; k < rb->ns; ++k) {
            double c[3];
            sphere_centre(frames, rb->sph_frame[k], rb->sph_o + 3 * k, c);
            double clr = orc_esdf_lookup(pb->grid, c, NULL) - rb->sph_r[k];
            if (clr < min_clear) min_clear = clr;
        }
        if (pb->cp->w_s > 0.0 && rb->self_pair != NULL)
            for (int i = 0; i < rb->ns; ++i)
                for (int j = i + 1; j < rb->ns; ++j) {
                    if (!rb->self_pair[i * rb->ns + j]) continue;
                    double ci[3], cj[3];
                    sphere_centre(frames, rb->sph_frame[i], rb->sph_o + 3 * i, ci);
                    sphere_centre(frames, rb->sph_frame[j], rb->sph_o + 3 * j, cj);
                    double d[3] = { ci[0] - cj[0], ci[1] - cj[1], ci[2] - cj[2] };
                    double clr = sqrt(dot3(d, d)) - rb->sph_r[i] - rb->sph_r[j];
                    if (clr < min_clear) min_clear = clr;
                }
        for (int j = 1; j <= pb->cp->n_sweep; ++j) {
            double q[7];
            sweep_config(pb, x, t, j, q);
            world_hinge(pb, q, NULL, &min_clear);
        }
        for (int j = 0; j < 7; ++j) {
            double jk = (traj_y(pb, x, t, j) - 3.0 * traj_y(pb, x, t - 1, j)
                         + 3.0 * traj_y(pb, x, t - 2, j) - traj_y(pb, x, t - 3, j))
                        / (pb->cp->dt * pb->cp->dt * pb->cp->dt);
            if (fabs(jk) > max_jerk) max_jerk = fabs(jk);
            double q = x[7 * (t - 1) + j];
            double v = q > rb->lim[2 * j + 1] ? q - rb->lim[2 * j + 1] : (q < rb->lim[2 * j] ? rb->lim[2 * j] - q : 0.0);
            if (v > lim_viol) lim_viol = v;
        }
    }
    double pose[7], qd[4];
    orc_flange_pose(rb->dh, x + 7 * (T - 1), pose);
    quat_normalise(pb->goal + 3, qd);
    double e[3] = { pose[0] - pb->goal[0], pose[1] - pb->goal[1], pose[2] - pb->goal[2] };
    double pos_err = sqrt(dot3(e, e));
    double dq = fabs(pose[3] * qd[0] + pose[4] * qd[1] + pose[5] * qd[2] + pose[6] * qd[3]);
    double rot_err = 2.0 * acos(dq < 1.0 ? dq : 1.0);
    int collision_free = min_clear >= 0.0;
    int ok = collision_free && pos_err < thr[0] && rot_err < thr[1] && lim_viol == 0.0;
    if (metrics) {
        metrics[0] = min_clear; metrics[1] = pos_err; metrics[2] = rot_err; metrics[3] = max_jerk;
        metrics[4] = lim_viol; metrics[5] = orc_cost(pb, x, NULL, NULL); metrics[6] = collision_free;
    }
    return ok;
}

/* ------------------------------------------------------------------------ */
/* L-BFGS with Armijo accept/reject (one objective evaluation per iteration) */
/* ------------------------------------------------------------------------ */

typedef double (*orc_objective)(void *ctx, const double *x, double *g);

/* Each iteration evaluates f and g at the trial point, then:
 *   accept when f_trial <= f + c1 * g^T (x_trial - x) (always on the first
 *   evaluation): push (s, y) = (x_trial - x, g_trial - g) into the history when
 *   s^T y > 1e-10 |s| |y|, move to the trial point, alpha = min(1, 2 alpha);
 *   otherwise halve alpha, clearing the history and resetting alpha = 1 once
 *   alpha < alpha_min.
 * Then d = -H g by the two-loop recursion (H0 = gamma I, gamma = s^T y / y^T y
 * of the newest pair, gamma0 with an empty history), d = -g if it is not a
 * descent direction, step = alpha d scaled so that max |step| <= max_step, and
 * the next trial point is x + step.  The result is the last accepted point.
 * trace (optional, [iters]) receives the accepted f after each iteration. */
int orc_lbfgs(orc_objective obj, void *ctx, int n, const orc_opt *op,
              const double *x0, double *x_out, double *f_out, double *trace)
{
    int m = op->m;
    double *x = calloc((size_t)n, sizeof(double)), *g = calloc((size_t)n, sizeof(double));
    double *xt = calloc((size_t)n, sizeof(double)), *gt = calloc((size_t)n, sizeof(double));
    double *d = calloc((size_t)n, sizeof(double)), *qv = calloc((size_t)n, sizeof(double));
    double *S = calloc((size_t)m * n, sizeof(double)), *Y = calloc((size_t)m * n, sizeof(double));
    double *rho = calloc((size_t)m, sizeof(double)), *al = calloc((size_t)m, sizeof(double));
    int hist = 0, newest = -1, accepts = 0, first = 1;
    double f = INFINITY, alpha = 1.0, gts = 0.0;
    memcpy(xt, x0, sizeof(double) * n);
    for (int it = 0; it < op->iters; ++it) {
        double ft = obj(ctx, xt, gt);
        if (first) {
            memcpy(x, xt, sizeof(double) * n); memcpy(g, gt, sizeof(double) * n);
            f = ft; first = 0; ++accepts;
        } else if (ft <= f + op->c1 * gts) {
            double sy = 0.0, ss = 0.0, yy = 0.0;
            for (int i = 0; i < n; ++i) {
                double si = xt[i] - x[i], yi = gt[i] - g[i];
                sy += si * yi; ss += si * si; yy += yi * yi;
            }
            if (sy > 1e-10 * sqrt(ss) * sqrt(yy)) {
                newest = (newest + 1) % m;
                for (int i = 0; i < n; ++i) {
                    S[(size_t)newest * n + i] = xt[i] - x[i];
                    Y[(size_t)newest * n + i] = gt[i] - g[i];
                }
                rho[newest] = 1.0 / sy;
                if (hist < m) ++hist;
            }
            memcpy(x, xt, sizeof(double) * n); memcpy(g, gt, sizeof(double) * n);
            f = ft; ++accepts;
            alpha = alpha * 2.0 < 1.0 ? alpha * 2.0 : 1.0;
        } else {
            alpha *= 0.5;
            if (alpha < op->alpha_min) { hist = 0; newest = -1; alpha = 1.0; }
        }
        if (trace) trace[it] = f;

        /* two-loop recursion: newest to oldest, then oldest to newest */
        memcpy(qv, g, sizeof(double) * n);
        for (int h = 0; h < hist; ++h) {
            int k = ((newest - h) % m + m) % m;
            double a = 0.0;
            for (int i = 0; i < n; ++i) a += S[(size_t)k * n + i] * qv[i];
            al[k] = rho[k] * a;
            for (int i = 0; i < n; ++i) qv[i] -= al[k] * Y[(size_t)k * n + i];
        }
        double gamma = op->gamma0;
        if (hist > 0) {
            double yy = 0.0;
            for (int i = 0; i < n; ++i) yy += Y[(size_t)newest * n + i] * Y[(size_t)newest * n + i];
            gamma = (1.0 / rho[newest]) / yy;
        }
        for (int i = 0; i < n; ++i) qv[i] *= gamma;
        for (int h = hist - 1; h >= 0; --h) {
            int k = ((newest - h) % m + m) % m;
            double b = 0.0;
            for (int i = 0; i < n; ++i) b += Y[(size_t)k * n + i] * qv[i];
            b *= rho[k];
            for (int i = 0; i < n; ++i) qv[i] += (al[k] - b) * S[(size_t)k * n + i];
        }
        double gd = 0.0;
        for (int i = 0; i < n; ++i) { d[i] = -qv[i]; gd += g[i] * d[i]; }
        if (!(gd < 0.0))
            for (int i = 0; i < n; ++i) d[i] = -g[i];
        double mx = 0.0;
        for (int i = 0; i < n; ++i) if (fabs(alpha * d[i]) > mx) mx = fabs(alpha * d[i]);
        double scale = mx > op->max_step ? op->max_step / mx : 1.0;
        gts = 0.0;
        for (int i = 0; i < n; ++i) {
            double st = alpha * d[i] * scale;
            xt[i] = x[i] + st;
            gts += g[i] * st;
        }
    }
    memcpy(x_out, x, sizeof(double) * n);
    if (f_out) *f_out = f;
    free(x); free(g); free(xt); free(gt); free(d); free(qv); free(S); free(Y); free(rho); free(al);
    return accepts;
}

static double traj_objective(void *ctx, const double *x, double *g)
{
    return orc_cost((const orc_problem *)ctx, x, g, NULL);
}

/* Optimise S seeds for each of P problems (seeds [P][S][T][7]).  Outputs:
 * x_out [P][S][T][7], f_out [P][S], success [P][S], metrics [P][S][7]
 * (see orc_evaluate), trace [P][S][iters] (optional), best [P] = index of the
 * lowest-cost successful seed (ties -> lowest index), -1 when none succeeds. */
void orc_plan(const orc_problem *probs, int P, int S, const double *seeds, const orc_opt *op,
              const double *thr, double *x_out, double *f_out, int *success,
              double *metrics, double *trace, int *best)
{
    int T = probs[0].T, n = 7 * T;
    #pragma omp parallel for schedule(dynamic, 1)
    for (int ps = 0; ps < P * S; ++ps) {
        int p = ps / S;
        size_t off = (size_t)ps * n;
        orc_lbfgs(traj_objective, (void *)&probs[p], n, op, seeds + off, x_out + off,
                  f_out + ps, trace ? trace + (size_t)ps * op->iters : NULL);
        success[ps] = orc_evaluate(&probs[p], x_out + off, thr, metrics ? metrics + 7 * (size_t)ps : NULL);
    }
    for (int p = 0; p < P; ++p) {
        best[p] = -1;
        for (int s = 0; s < S; ++s)
            if (success[p * S + s] && (best[p] < 0 || f_out[p * S + s] < f_out[p * S + best[p]]))
                best[p] = s;
    }
}

/* Batched cost/gradient of B trajectories that all belong to problem pb. */
void orc_cost_batch(const orc_problem *pb, int B, const double *x, double *cost, double *grad)
{
    int n = 7 * pb->T;
    #pragma omp parallel for schedule(dynamic, 1)
    for (int b = 0; b < B; ++b)
        cost[b] = orc_cost(pb, x + (size_t)b * n, grad ? grad + (size_t)b * n : NULL, NULL);
}

/* Convex quadratic f(x) = 1/2 x^T A x - b^T x, used to pin the L-BFGS above
 * against a direct linear solve. */
typedef struct { const double *A; const double *b; int n; } quad_ctx;

static double quad_objective(void *ctx, const double *x, double *g)
{
    const quad_ctx *qc = (const quad_ctx *)ctx;
    double f = 0.0;
    for (int i = 0; i < qc->n; ++i) {
        double Ax = 0.0;
        for (int j = 0; j < qc->n; ++j) Ax += qc->A[(size_t)i * qc->n + j] * x[j];
        g[i] = Ax - qc->b[i];
        f += 0.5 * x[i] * Ax - qc->b[i] * x[i];
    }
    return f;
}

int orc_lbfgs_quadratic(const double *A, const double *b, int n, const orc_opt *op,
                        const double *x0, double *x_out, double *f_out, double *trace)
{
    quad_ctx qc = { A, b, n };
    return orc_lbfgs(quad_objective, &qc, n, op, x0, x_out, f_out, trace);
}
