/*
 * FP64 CPU oracle for batched edge validation.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may include, link or
 * call this code: only the tests, the package's smoke check and the CPU
 * baseline leg of the benchmark use it.  It shares no code with the CUDA
 * library and computes the plain definitions of the paper's method
 * (Thomason, Kingston, Kavraki, "Motions in Microseconds via Vectorized
 * Sampling-Based Planning", arXiv 2309.14545), in double precision, in linear
 * order, with no sphere hierarchy, no rake and no early exit inside a state.
 *
 *   FK (Sec. "Vectorized Forward Kinematics"): link frames T_0 = I,
 *     T_{j+1} = T_{parent(j)+1} * F_j * M_j(q_j); sphere centres
 *     c_s = T_{link(s)} * local_s (only sphere positions are needed).
 *   Collision checking (Sec. "Vectorized Collision Checking"): robot spheres
 *     against environment spheres, capsules and oriented cuboids, and robot
 *     sphere pairs against each other.
 *   Motion validation (Sec. "Vectorized Motion Validation"): an edge is valid
 *     iff every state of its discretisation is valid; the rake and the sphere
 *     hierarchy only reorder or skip work and leave that verdict unchanged.
 *   Linear interpolation in a Euclidean C-space (Sec. "Bringing it Together").
 *
 * Readings where the paper is silent (kept identical in the CUDA library's
 * documentation): states i = 0..k-1 at t = i/(k-1), both endpoints included;
 * k = max(2, ceil(max_d |q1_d - q0_d| / res) + 1) computed in float32 (the
 * precision the method runs in, so both sides take this integer decision the
 * same way); a state is valid iff its clearance K(q) >= 0; a state or edge
 * with a non-finite coordinate is invalid.
 *
 * Parity pins: every function here is checked in tests/ against closed forms,
 * library routines, brute force or invariants (see the tests' docstrings);
 * the collision cost and its gradient are an addition beside the paper.
 */
#ifndef VP_ORACLE_H
#define VP_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define VPO_REVOLUTE 0
#define VPO_PRISMATIC 1
/* Longest edge, in resolution steps, the method accepts. */
#define VPO_MAX_STEPS 16777216
/* Size limits of this implementation (stack arrays). */
#define VPO_MAX_JOINTS 64
#define VPO_MAX_SPHERES 1024

typedef struct {
    int32_t n_joints;
    const int32_t *parent;   /* [D], -1 = base, else an earlier joint      */
    const int32_t *type;     /* [D], VPO_REVOLUTE / VPO_PRISMATIC          */
    const double *axis;      /* [D][3] unit axis in the joint frame        */
    const double *origin;    /* [D][3][4] fixed [R|t], parent frame -> joint */
    int32_t n_spheres;
    const int32_t *sphere_link;   /* [S] 0 = base, j+1 = after joint j     */
    const double *sphere_centre;  /* [S][3] in the link frame              */
    const double *sphere_radius;  /* [S]                                   */
    int32_t n_pairs;
    const int32_t *pairs;         /* [P][2] sphere indices                 */
} vpo_robot;

typedef struct {
    int32_t n_spheres;  const double *spheres;   /* [n][4]  c, r            */
    int32_t n_capsules; const double *capsules;  /* [n][7]  p0, p1, r       */
    int32_t n_cuboids;  const double *cuboids;   /* [n][15] c, R(3x3), h    */
} vpo_env;

/* Link frames [D+1][3][4]; frame 0 is the base (identity). */
void vpo_link_frames(const vpo_robot *r, const double *q, double *frames);
/* World sphere centres [S][3]. */
void vpo_fk(const vpo_robot *r, const double *q, double *centres);
void vpo_fk_batch(const vpo_robot *r, const double *q, int64_t n, double *centres);

/* Signed distances from a point to an environment primitive (negative inside). */
double vpo_dist_sphere(const double *x, const double *sphere);
double vpo_dist_capsule(const double *x, const double *capsule);
double vpo_dist_cuboid(const double *x, const double *cuboid);

/* Clearance K(q): min over (sphere, primitive) of d - r_s and over self pairs
 * of |c_a - c_b| - r_a - r_b; -inf for a non-finite q; +inf if nothing to test. */
double vpo_state_clearance(const vpo_robot *r, const vpo_env *e, const double *q);
void vpo_clearance_batch(const vpo_robot *r, const vpo_env *e, const double *q, int64_t n, double *K);
int vpo_state_valid(const vpo_robot *r, const vpo_env *e, const double *q);

/* State count of an edge (float32 arithmetic); -1 when the edge has a
 * non-finite coordinate or is longer than VPO_MAX_STEPS steps. */
int32_t vpo_edge_count(const float *q0, const float *q1, int32_t D, float res);
/* State i of a k-state edge, in double. */
void vpo_edge_state(const float *q0, const float *q1, int32_t D, int32_t k, int32_t i, double *q);
/* Edge verdict (1 = every state valid), linear order.  A count below 2 or
 * above VPO_MAX_STEPS + 1 (longer than any edge a resolution may give) makes
 * the edge invalid without checking a state. */
int vpo_edge_valid(const vpo_robot *r, const vpo_env *e, const float *q0, const float *q1, int32_t k);
/* Verdicts for E edges; counts may be NULL (then k follows from res).
 * Returns the number of edges whose count was invalid (below 2, above
 * VPO_MAX_STEPS + 1, or none; they are reported invalid). */
int64_t vpo_validate_edges(const vpo_robot *r, const vpo_env *e, const float *q0, const float *q1,
                           const int32_t *counts, float res, int64_t E, uint8_t *valid);

/* Edge class against a clearance band b: 0 = pinned free (every state K > b),
 * 1 = pinned collide (some state K < -b), 2 = band.  Stops at the first state
 * with K < -b.  *n_band receives the number of band states seen, *n_eval the
 * number of states evaluated. */
int vpo_edge_classify(const vpo_robot *r, const vpo_env *e, const float *q0, const float *q1,
                      int32_t k, double band, int32_t *n_band, int32_t *n_eval);
void vpo_classify_edges(const vpo_robot *r, const vpo_env *e, const float *q0, const float *q1,
                        const int32_t *counts, float res, int64_t E, double band,
                        int8_t *cls, int32_t *n_band);

/* Penetration cost c(q) = sum_s sum_o max(0, r_s + margin - d(c_s, o))^2 over
 * environment primitives; if grad != NULL, dc/dq [D] from the geometric
 * Jacobian.  The paper has no such cost: it is an addition beside it. */
double vpo_cost(const vpo_robot *r, const vpo_env *e, const double *q, double margin, double *grad);
void vpo_cost_batch(const vpo_robot *r, const vpo_env *e, const double *q, int64_t n, double margin,
                    double *cost, double *grad);

#ifdef __cplusplus
}
#endif
#endif
