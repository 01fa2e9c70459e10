/*
 * FP64 CPU oracle for batched edge validation -- TEST INFRASTRUCTURE ONLY
 * (see vp_oracle.h).  Plain definitions, written for a reader to check
 * against the paper by eye: 4x4 homogeneous matrices, linear loops, no
 * hierarchy, no reordering.  Build: gcc -O2 -ffp-contract=off (no fast-math).
 */
#include "vp_oracle.h"

#include <math.h>
#include <stddef.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* 4x4 homogeneous transforms, row-major                                    */

static void mat_identity(double m[16])
{
    memset(m, 0, 16 * sizeof(double));
    m[0] = m[5] = m[10] = m[15] = 1.0;
}

static void mat_mul(const double a[16], const double b[16], double out[16])
{
    double t[16];
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            double s = 0.0;
            for (int k = 0; k < 4; ++k) s += a[4 * i + k] * b[4 * k + j];
            t[4 * i + j] = s;
        }
    memcpy(out, t, sizeof(t));
}

/* The fixed [R|t] of a joint as a 4x4. */
static void mat_from_3x4(const double *rt, double m[16])
{
    mat_identity(m);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 4; ++j) m[4 * i + j] = rt[4 * i + j];
}

/* Rotation by angle q about unit axis a (Rodrigues' formula):
 * R = I + sin(q) [a]x + (1 - cos(q)) [a]x^2. */
static void mat_rotation(const double a[3], double q, double m[16])
{
    double K[9] = {0.0, -a[2], a[1], a[2], 0.0, -a[0], -a[1], a[0], 0.0};
    double K2[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += K[3 * i + k] * K[3 * k + j];
            K2[3 * i + j] = s;
        }
    double s = sin(q), c = cos(q);
    mat_identity(m);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            m[4 * i + j] = (i == j ? 1.0 : 0.0) + s * K[3 * i + j] + (1.0 - c) * K2[3 * i + j];
}

/* Translation by d along unit axis a. */
static void mat_translation(const double a[3], double d, double m[16])
{
    mat_identity(m);
    m[3] = a[0] * d;
    m[7] = a[1] * d;
    m[11] = a[2] * d;
}

static void mat_apply(const double m[16], const double x[3], double out[3])
{
    for (int i = 0; i < 3; ++i)
        out[i] = m[4 * i + 0] * x[0] + m[4 * i + 1] * x[1] + m[4 * i + 2] * x[2] + m[4 * i + 3];
}

/* ------------------------------------------------------------------------ */
/* Forward kinematics                                                       */

/* All link frames as 4x4: T[0] = I, T[j+1] = T[parent(j)+1] * F_j * M_j(q_j). */
static void link_frames4(const vpo_robot *r, const double *q, double *T /* [D+1][16] */)
{
    mat_identity(T);
    for (int j = 0; j < r->n_joints; ++j) {
        const double *parent = T + 16 * (r->parent[j] + 1);
        double F[16], M[16], PF[16];
        mat_from_3x4(r->origin + 12 * j, F);
        if (r->type[j] == VPO_REVOLUTE)
            mat_rotation(r->axis + 3 * j, q[j], M);
        else
            mat_translation(r->axis + 3 * j, q[j], M);
        mat_mul(parent, F, PF);
        mat_mul(PF, M, T + 16 * (j + 1));
    }
}

void vpo_link_frames(const vpo_robot *r, const double *q, double *frames)
{
    double T[16 * (VPO_MAX_JOINTS + 1)];
    int L = r->n_joints + 1;
    if (r->n_joints > VPO_MAX_JOINTS) return;
    link_frames4(r, q, T);
    for (int l = 0; l < L; ++l)
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 4; ++j) frames[12 * l + 4 * i + j] = T[16 * l + 4 * i + j];
}

void vpo_fk(const vpo_robot *r, const double *q, double *centres)
{
    double T[16 * (VPO_MAX_JOINTS + 1)];
    if (r->n_joints > VPO_MAX_JOINTS) return;
    link_frames4(r, q, T);
    for (int s = 0; s < r->n_spheres; ++s)
        mat_apply(T + 16 * r->sphere_link[s], r->sphere_centre + 3 * s, centres + 3 * s);
}

void vpo_fk_batch(const vpo_robot *r, const double *q, int64_t n, double *centres)
{
    for (int64_t i = 0; i < n; ++i)
        vpo_fk(r, q + i * r->n_joints, centres + i * 3 * r->n_spheres);
}

/* ------------------------------------------------------------------------ */
/* Signed distances, point to primitive                                     */

static double norm3(const double v[3]) { return sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]); }

double vpo_dist_sphere(const double *x, const double *sph)
{
    double v[3] = {x[0] - sph[0], x[1] - sph[1], x[2] - sph[2]};
    return norm3(v) - sph[3];
}

/* Capsule = points within radius of segment p0-p1.  Closest segment point at
 * t = clamp((x - p0).u / u.u, 0, 1), u = p1 - p0 (t = 0 for a point segment). */
double vpo_dist_capsule(const double *x, const double *cap)
{
    const double *p0 = cap, *p1 = cap + 3;
    double u[3] = {p1[0] - p0[0], p1[1] - p0[1], p1[2] - p0[2]};
    double w[3] = {x[0] - p0[0], x[1] - p0[1], x[2] - p0[2]};
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    double t = 0.0;
    if (uu > 0.0) {
        t = (w[0] * u[0] + w[1] * u[1] + w[2] * u[2]) / uu;
        if (t < 0.0) t = 0.0;
        if (t > 1.0) t = 1.0;
    }
    double v[3] = {w[0] - t * u[0], w[1] - t * u[1], w[2] - t * u[2]};
    return norm3(v) - cap[6];
}

/* Oriented cuboid: y = R^T (x - c) in box coordinates, e = |y| - h;
 * d = |max(e, 0)| + min(max_i e_i, 0). */
double vpo_dist_cuboid(const double *x, const double *box)
{
    const double *c = box, *R = box + 3, *h = box + 12;
    double d[3] = {x[0] - c[0], x[1] - c[1], x[2] - c[2]};
    double e[3], out2 = 0.0, emax = -INFINITY;
    for (int i = 0; i < 3; ++i) {
        /* column i of R is box axis i in the world */
        double yi = R[0 * 3 + i] * d[0] + R[1 * 3 + i] * d[1] + R[2 * 3 + i] * d[2];
        e[i] = fabs(yi) - h[i];
        if (e[i] > 0.0) out2 += e[i] * e[i];
        if (e[i] > emax) emax = e[i];
    }
    return sqrt(out2) + (emax < 0.0 ? emax : 0.0);
}

/* ------------------------------------------------------------------------ */
/* State validity                                                           */

static int all_finite(const double *q, int n)
{
    for (int i = 0; i < n; ++i)
        if (!isfinite(q[i])) return 0;
    return 1;
}

double vpo_state_clearance(const vpo_robot *r, const vpo_env *e, const double *q)
{
    if (!all_finite(q, r->n_joints)) return -INFINITY;
    double c[3 * VPO_MAX_SPHERES];
    if (r->n_spheres > VPO_MAX_SPHERES || r->n_joints > VPO_MAX_JOINTS) return NAN;
    vpo_fk(r, q, c);
    double K = INFINITY;
    for (int s = 0; s < r->n_spheres; ++s) {
        const double *x = c + 3 * s;
        double rs = r->sphere_radius[s];
        for (int o = 0; o < e->n_spheres; ++o) {
            double k = vpo_dist_sphere(x, e->spheres + 4 * o) - rs;
            if (k < K) K = k;
        }
        for (int o = 0; o < e->n_capsules; ++o) {
            double k = vpo_dist_capsule(x, e->capsules + 7 * o) - rs;
            if (k < K) K = k;
        }
        for (int o = 0; o < e->n_cuboids; ++o) {
            double k = vpo_dist_cuboid(x, e->cuboids + 15 * o) - rs;
            if (k < K) K = k;
        }
    }
    for (int p = 0; p < r->n_pairs; ++p) {
        int a = r->pairs[2 * p], b = r->pairs[2 * p + 1];
        double v[3] = {c[3 * a] - c[3 * b], c[3 * a + 1] - c[3 * b + 1], c[3 * a + 2] - c[3 * b + 2]};
        double k = norm3(v) - r->sphere_radius[a] - r->sphere_radius[b];
        if (k < K) K = k;
    }
    return K;
}

void vpo_clearance_batch(const vpo_robot *r, const vpo_env *e, const double *q, int64_t n, double *K)
{
    for (int64_t i = 0; i < n; ++i) K[i] = vpo_state_clearance(r, e, q + i * r->n_joints);
}

int vpo_state_valid(const vpo_robot *r, const vpo_env *e, const double *q)
{
    return vpo_state_clearance(r, e, q) >= 0.0;
}

/* ------------------------------------------------------------------------ */
/* Edges                                                                    */

int32_t vpo_edge_count(const float *q0, const float *q1, int32_t D, float res)
{
    float dmax = 0.0f;
    for (int d = 0; d < D; ++d) {
        if (!isfinite(q0[d]) || !isfinite(q1[d])) return -1;
        float dd = fabsf(q1[d] - q0[d]);
        if (dd > dmax) dmax = dd;
    }
    float steps = ceilf(dmax / res);
    if (!(steps <= (float)VPO_MAX_STEPS)) return -1;
    int32_t k = (int32_t)steps + 1;
    return k < 2 ? 2 : k;
}

void vpo_edge_state(const float *q0, const float *q1, int32_t D, int32_t k, int32_t i, double *q)
{
    double t = (double)i / (double)(k - 1);
    for (int d = 0; d < D; ++d) q[d] = (double)q0[d] + t * ((double)q1[d] - (double)q0[d]);
}

static int endpoints_finite(const float *q0, const float *q1, int32_t D)
{
    for (int d = 0; d < D; ++d)
        if (!isfinite(q0[d]) || !isfinite(q1[d])) return 0;
    return 1;
}

int vpo_edge_valid(const vpo_robot *r, const vpo_env *e, const float *q0, const float *q1, int32_t k)
{
    int D = r->n_joints;
    if (k < 2 || k > VPO_MAX_STEPS + 1 || !endpoints_finite(q0, q1, D)) return 0;
    double q[VPO_MAX_JOINTS];
    for (int32_t i = 0; i < k; ++i) {
        vpo_edge_state(q0, q1, D, k, i, q);
        if (!vpo_state_valid(r, e, q)) return 0;
    }
    return 1;
}

int64_t vpo_validate_edges(const vpo_robot *r, const vpo_env *e, const float *q0, const float *q1,
                           const int32_t *counts, float res, int64_t E, uint8_t *valid)
{
    int D = r->n_joints;
    int64_t bad = 0;
    for (int64_t i = 0; i < E; ++i) {
        const float *a = q0 + i * D, *b = q1 + i * D;
        int32_t k = counts ? counts[i] : vpo_edge_count(a, b, D, res);
        if (k < 2 || k > VPO_MAX_STEPS + 1) ++bad;
        valid[i] = (uint8_t)vpo_edge_valid(r, e, a, b, k);
    }
    return bad;
}

int vpo_edge_classify(const vpo_robot *r, const vpo_env *e, const float *q0, const float *q1,
                      int32_t k, double band, int32_t *n_band, int32_t *n_eval)
{
    int D = r->n_joints;
    int32_t nb = 0, ne = 0;
    int cls = 0;
    if (k < 2 || k > VPO_MAX_STEPS + 1 || !endpoints_finite(q0, q1, D)) {
        cls = 1;
    } else {
        double q[VPO_MAX_JOINTS];
        for (int32_t i = 0; i < k; ++i) {
            vpo_edge_state(q0, q1, D, k, i, q);
            double K = vpo_state_clearance(r, e, q);
            ++ne;
            if (K < -band) { cls = 1; break; }
            if (K <= band) { ++nb; cls = 2; }
        }
    }
    if (n_band) *n_band = nb;
    if (n_eval) *n_eval = ne;
    return cls;
}

void vpo_classify_edges(const vpo_robot *r, const vpo_env *e, const float *q0, const float *q1,
                        const int32_t *counts, float res, int64_t E, double band,
                        int8_t *cls, int32_t *n_band)
{
    int D = r->n_joints;
    for (int64_t i = 0; i < E; ++i) {
        const float *a = q0 + i * D, *b = q1 + i * D;
        int32_t k = counts ? counts[i] : vpo_edge_count(a, b, D, res);
        cls[i] = (int8_t)vpo_edge_classify(r, e, a, b, k, band, n_band ? n_band + i : NULL, NULL);
    }
}

/* ------------------------------------------------------------------------ */
/* Penetration cost and its gradient (an addition beside the paper)         */

/* Gradient of the signed distance at x (unit vector; zero at a point where
 * it is undefined: a sphere centre, a point on a capsule's axis). */
static void grad_sphere(const double *x, const double *sph, double g[3])
{
    double v[3] = {x[0] - sph[0], x[1] - sph[1], x[2] - sph[2]};
    double n = norm3(v);
    for (int i = 0; i < 3; ++i) g[i] = n > 0.0 ? v[i] / n : 0.0;
}

static void grad_capsule(const double *x, const double *cap, double g[3])
{
    const double *p0 = cap, *p1 = cap + 3;
    double u[3] = {p1[0] - p0[0], p1[1] - p0[1], p1[2] - p0[2]};
    double w[3] = {x[0] - p0[0], x[1] - p0[1], x[2] - p0[2]};
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    double t = 0.0;
    if (uu > 0.0) {
        t = (w[0] * u[0] + w[1] * u[1] + w[2] * u[2]) / uu;
        if (t < 0.0) t = 0.0;
        if (t > 1.0) t = 1.0;
    }
    double v[3] = {w[0] - t * u[0], w[1] - t * u[1], w[2] - t * u[2]};
    double n = norm3(v);
    for (int i = 0; i < 3; ++i) g[i] = n > 0.0 ? v[i] / n : 0.0;
}

static void grad_cuboid(const double *x, const double *box, double g[3])
{
    const double *c = box, *R = box + 3, *h = box + 12;
    double d[3] = {x[0] - c[0], x[1] - c[1], x[2] - c[2]};
    double y[3], e[3], gb[3] = {0.0, 0.0, 0.0};
    double out2 = 0.0;
    int imax = 0;
    for (int i = 0; i < 3; ++i) {
        y[i] = R[0 * 3 + i] * d[0] + R[1 * 3 + i] * d[1] + R[2 * 3 + i] * d[2];
        e[i] = fabs(y[i]) - h[i];
        if (e[i] > 0.0) out2 += e[i] * e[i];
        if (e[i] > e[imax]) imax = i;
    }
    if (out2 > 0.0) {
        double n = sqrt(out2);
        for (int i = 0; i < 3; ++i)
            gb[i] = e[i] > 0.0 ? (y[i] < 0.0 ? -1.0 : 1.0) * e[i] / n : 0.0;
    } else {
        gb[imax] = y[imax] < 0.0 ? -1.0 : 1.0;
    }
    for (int i = 0; i < 3; ++i) g[i] = R[3 * i + 0] * gb[0] + R[3 * i + 1] * gb[1] + R[3 * i + 2] * gb[2];
}

/* 1 iff joint j moves link l (l = j+1 or a descendant of it). */
static int joint_moves_link(const vpo_robot *r, int j, int l)
{
    for (int a = l - 1; a >= 0; a = r->parent[a])
        if (a == j) return 1;
    return 0;
}

double vpo_cost(const vpo_robot *r, const vpo_env *e, const double *q, double margin, double *grad)
{
    int D = r->n_joints, S = r->n_spheres;
    double T[16 * (VPO_MAX_JOINTS + 1)], c[3 * VPO_MAX_SPHERES], gs[3 * VPO_MAX_SPHERES];
    if (D > VPO_MAX_JOINTS || S > VPO_MAX_SPHERES) return NAN;
    link_frames4(r, q, T);
    for (int s = 0; s < S; ++s) mat_apply(T + 16 * r->sphere_link[s], r->sphere_centre + 3 * s, c + 3 * s);

    double cost = 0.0;
    for (int s = 0; s < S; ++s) {
        const double *x = c + 3 * s;
        double rs = r->sphere_radius[s] + margin;
        double *g = gs + 3 * s;
        g[0] = g[1] = g[2] = 0.0;
        for (int kind = 0; kind < 3; ++kind) {
            int n = kind == 0 ? e->n_spheres : kind == 1 ? e->n_capsules : e->n_cuboids;
            for (int o = 0; o < n; ++o) {
                double d, gd[3];
                if (kind == 0) { d = vpo_dist_sphere(x, e->spheres + 4 * o); grad_sphere(x, e->spheres + 4 * o, gd); }
                else if (kind == 1) { d = vpo_dist_capsule(x, e->capsules + 7 * o); grad_capsule(x, e->capsules + 7 * o, gd); }
                else { d = vpo_dist_cuboid(x, e->cuboids + 15 * o); grad_cuboid(x, e->cuboids + 15 * o, gd); }
                double pen = rs - d;
                if (pen > 0.0) {
                    cost += pen * pen;
                    /* d/dx of pen^2 = -2 pen grad d */
                    for (int i = 0; i < 3; ++i) g[i] += -2.0 * pen * gd[i];
                }
            }
        }
    }
    if (grad) {
        /* dc/dq_j = sum over spheres moved by joint j of g_s . dc_s/dq_j, with
         * dc_s/dq_j = a_j x (c_s - p_j) (revolute) or a_j (prismatic), a_j and
         * p_j the joint's world axis and origin. */
        for (int j = 0; j < D; ++j) {
            double JF[16], F[16];
            mat_from_3x4(r->origin + 12 * j, F);
            mat_mul(T + 16 * (r->parent[j] + 1), F, JF);
            const double *ax = r->axis + 3 * j;
            double a[3], p[3] = {JF[3], JF[7], JF[11]};
            for (int i = 0; i < 3; ++i) a[i] = JF[4 * i] * ax[0] + JF[4 * i + 1] * ax[1] + JF[4 * i + 2] * ax[2];
            double sum = 0.0;
            for (int s = 0; s < S; ++s) {
                if (!joint_moves_link(r, j, r->sphere_link[s])) continue;
                const double *g = gs + 3 * s;
                double dc[3];
                if (r->type[j] == VPO_REVOLUTE) {
                    double v[3] = {c[3 * s] - p[0], c[3 * s + 1] - p[1], c[3 * s + 2] - p[2]};
                    dc[0] = a[1] * v[2] - a[2] * v[1];
                    dc[1] = a[2] * v[0] - a[0] * v[2];
                    dc[2] = a[0] * v[1] - a[1] * v[0];
                } else {
                    dc[0] = a[0]; dc[1] = a[1]; dc[2] = a[2];
                }
                sum += g[0] * dc[0] + g[1] * dc[1] + g[2] * dc[2];
            }
            grad[j] = sum;
        }
    }
    return cost;
}

void vpo_cost_batch(const vpo_robot *r, const vpo_env *e, const double *q, int64_t n, double margin,
                    double *cost, double *grad)
{
    int D = r->n_joints;
    for (int64_t i = 0; i < n; ++i)
        cost[i] = vpo_cost(r, e, q + i * D, margin, grad ? grad + i * D : NULL);
}
