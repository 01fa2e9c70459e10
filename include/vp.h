/*
 * vp.h -- C ABI of libvp: batched motion (edge) validation on one GPU.
 *
 * Method: Thomason, Kingston, Kavraki, "Motions in Microseconds via Vectorized
 * Sampling-Based Planning" (arXiv 2309.14545), Sec. III ("Method"):
 *   - a state validity function and an edge validity function over a robot
 *     in an environment (Sec. III, first paragraph);
 *   - forward kinematics that poses many configurations at once and computes
 *     only collision-sphere positions (Sec. III-B, III-C);
 *   - collision checks of robot spheres against sphere / capsule / cuboid
 *     primitives and robot self pairs (Sec. III-C);
 *   - the "raked" edge validator: spatially spread states checked together,
 *     a per-link bounding-sphere "mid-phase", checks interleaved with FK, and
 *     termination at the first collision (Sec. III-D, Fig. 2);
 *   - linear interpolation between configurations in a Euclidean C-space
 *     (Sec. III-E).
 *
 * Conventions for every call
 *   - Every function returns a vp_status and never aborts the process.
 *   - Argument errors are detected on the host before anything is launched
 *     (VP_ERR_ARG / VP_ERR_CAPACITY / VP_ERR_NOT_LOADED); the message is in
 *     vp_last_error(ctx).
 *   - Problems only visible on the device (an explicit state count < 2, an
 *     edge longer than VP_MAX_STEPS steps, a watchdog timeout) set bits in a
 *     device status word; vp_sync_status() synchronises, reads and clears it.
 *     Such an edge is reported invalid.
 *   - Pointers named "device" are CUDA device pointers (e.g. a torch tensor's
 *     data_ptr()) on the context's device; the caller owns them and keeps
 *     them alive until the work on `stream` completes.  `stream` is a
 *     cudaStream_t (NULL = the legacy default stream); compute calls are
 *     asynchronous with respect to the host.
 *   - Host descriptors passed to the loaders are copied; the caller keeps
 *     ownership.
 *   - Configurations are float32, row-major [n, D] with D = the robot's joint
 *     count.  Lengths in metres, angles in radians.
 *   - A configuration with a non-finite coordinate is invalid; an edge with a
 *     non-finite endpoint coordinate is invalid.  Joint limits are a property
 *     of the workload, not a check: out-of-limit configurations are validated
 *     as given.
 *   - A vp_ctx is not thread-safe; distinct contexts are independent.
 */
#ifndef VP_H
#define VP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct vp_ctx vp_ctx;

typedef enum {
    VP_OK = 0,
    VP_ERR_ARG = 1,        /* invalid argument; nothing was launched            */
    VP_ERR_CUDA = 2,       /* a CUDA runtime call failed                         */
    VP_ERR_CAPACITY = 3,   /* robot or environment beyond a compiled limit       */
    VP_ERR_NOT_LOADED = 4, /* robot or environment not loaded                    */
    VP_ERR_TIMEOUT = 5,    /* a device watchdog gave up (work left unfinished)   */
    VP_ERR_DEVICE = 6      /* bad input found on the device (see vp_sync_status) */
} vp_status;

enum { VP_JOINT_REVOLUTE = 0, VP_JOINT_PRISMATIC = 1 };

/* vp_validate_edges modes. */
enum {
    VP_MODE_PLAIN = 0,    /* one launch, one warp per edge, fixed tiling          */
    VP_MODE_BATCHED = 1,  /* persistent length-bucketed work queue, tuned tiling  */
    VP_MODE_PER_EDGE = 2  /* one plain launch per edge (the literal baseline)     */
};

/* Compiled limits. */
#define VP_MAX_JOINTS 16
#define VP_MAX_SPHERES 256
#define VP_MAX_PAIRS 1024
#define VP_MAX_ENV_BYTES (160 * 1024) /* packed environment held in shared memory */
#define VP_MAX_STEPS 16777216         /* longest edge, in resolution steps; an
                                       * explicit count may be at most
                                       * VP_MAX_STEPS + 1 states              */

/* Device status bits (OR-ed into the status word). */
#define VP_DEVERR_COUNT 0x1u   /* an explicit count < 2                    */
#define VP_DEVERR_LENGTH 0x2u  /* an edge longer than VP_MAX_STEPS steps, or
                                * an explicit count > VP_MAX_STEPS + 1     */
#define VP_DEVERR_TIMEOUT 0x4u /* the persistent kernel's watchdog fired   */

/*
 * Robot: a forest of joint chains on a fixed base (host memory, copied).
 *   joint_parent[j]  -1 (the base) or an earlier joint index.
 *   joint_type[j]    VP_JOINT_REVOLUTE / VP_JOINT_PRISMATIC.
 *   joint_axis       [D][3] unit axis in the joint's frame.
 *   joint_origin     [D][3][4] fixed [R | t] from the parent's frame to the
 *                    joint's frame, row-major.
 *   Link 0 is the base; link j+1 is the frame after joint j moved by q_j:
 *   T_{j+1} = T_{parent(j)+1} * origin_j * (Rot(axis_j, q_j) or Trans(axis_j q_j)).
 *   sphere_link[s], sphere_centre [S][3] (in the link's frame), sphere_radius[s].
 *   link_spheres     [D+1][4] conservative bounding sphere per link (centre in
 *                    the link frame, radius; radius <= 0 for a link with no
 *                    spheres), or NULL.  Given spheres must contain every
 *                    sphere of their link (else VP_ERR_ARG).  The library
 *                    also bounds each link's spheres itself and uses the
 *                    smaller of the two (vp_link_bounds reports the choice);
 *                    verdicts do not depend on it.  The paper's "mid-phase"
 *                    (Sec. III-D).
 *   self_pairs       [P][2] sphere indices checked against each other.
 */
typedef struct {
    int32_t n_joints;
    const int32_t *joint_parent;
    const int32_t *joint_type;
    const double *joint_axis;
    const double *joint_origin;
    int32_t n_spheres;
    const int32_t *sphere_link;
    const double *sphere_centre;
    const double *sphere_radius;
    const double *link_spheres;
    int32_t n_pairs;
    const int32_t *self_pairs;
} vp_robot_desc;

/*
 * Environment primitives (host memory, copied), Sec. III-C:
 *   spheres  [n][4]  centre, radius
 *   capsules [n][7]  segment end p0, end p1, radius
 *   cuboids  [n][15] centre, R (3x3 row-major; column i = box axis i in the
 *                    world frame), half-extents
 * Packed for the device (with each primitive's world box): 48 bytes per
 * sphere, 64 per capsule, 96 per cuboid.
 */
typedef struct {
    int32_t n_spheres;
    const double *spheres;
    int32_t n_capsules;
    const double *capsules;
    int32_t n_cuboids;
    const double *cuboids;
} vp_env_desc;

/* Create a context on CUDA device `device`.  Allocates a small device status
 * word.  The caller's current device is left unchanged. */
vp_status vp_create(vp_ctx **out, int device);
/* Free everything the context owns.  NULL is accepted. */
vp_status vp_destroy(vp_ctx *ctx);
/* Message of the last failed call on ctx (valid until the next call). */
const char *vp_last_error(const vp_ctx *ctx);

/* Load (replace) the robot.  Synchronous.  Errors: VP_ERR_ARG for malformed
 * tables, VP_ERR_CAPACITY beyond the VP_MAX_* limits. */
vp_status vp_load_robot(vp_ctx *ctx, const vp_robot_desc *robot);
/* Load (replace) the environment into a device buffer the context owns.
 * Synchronous.  VP_ERR_CAPACITY if it packs to more than VP_MAX_ENV_BYTES. */
vp_status vp_load_env(vp_ctx *ctx, const vp_env_desc *env);

/* FK (Sec. III-B): world sphere centres of n configurations.  q: device
 * float [n][D]; centres: device float [n][S][3], spheres in the robot's
 * original order.  By default the first call after a robot load generates
 * and compiles that robot's FK kernel (vp_fk_codegen; tens of ms, on the
 * host) and uses it from then on; where that fails (no NVRTC) the
 * table-driven kernel serves instead.  vp_fk_codegen pins either. */
vp_status vp_fk_spheres(vp_ctx *ctx, const float *q, int64_t n, float *centres, void *stream);

/* State validity (Sec. III-C): valid[i] = 1 iff configuration i collides with
 * nothing (clearance >= 0 up to float32 rounding).  q: device float [n][D];
 * valid: device uint8 [n]. */
vp_status vp_validate_states(vp_ctx *ctx, const float *q, int64_t n, uint8_t *valid, void *stream);

/* State counts of edges (test hook for the discretisation, Sec. III-D):
 * counts[e] = max(2, ceil(max_d |q1_d - q0_d| / resolution) + 1), computed in
 * float32 with IEEE division; -1 for an edge with a non-finite coordinate or
 * more than VP_MAX_STEPS steps.  q0, q1: device float [E][D]; counts: device
 * int32 [E]. */
vp_status vp_edge_counts(vp_ctx *ctx, const float *q0, const float *q1, float resolution,
                         int64_t n_edges, int32_t *counts, void *stream);

/* Edge validity (Sec. III-D): valid[e] = 1 iff every state
 * q(t) = q0 + t (q1 - q0), t = i/(k-1), i = 0..k-1, is valid, where k is
 * counts[e] (device int32 [E], 2 <= k <= VP_MAX_STEPS + 1) or, with
 * counts == NULL, the count from `resolution` as in vp_edge_counts.  An
 * explicit count below 2 sets VP_DEVERR_COUNT, one above VP_MAX_STEPS + 1
 * sets VP_DEVERR_LENGTH; either edge is reported invalid.  States are
 * visited in raked order (a spread set of states per round).  Each state is
 * posed and checked in the order vp_set_check_order selects -- every link
 * posed first, or each link checked as soon as it is posed -- against self
 * pairs (link-pair bounding spheres, then sphere pairs) and primitives (link
 * bounding spheres -- the mid-phase -- then fine spheres); the edge stops at
 * the first collision.  mode: VP_MODE_*.
 * q0, q1: device float [E][D]; valid: device uint8 [E]. */
vp_status vp_validate_edges(vp_ctx *ctx, const float *q0, const float *q1, const int32_t *counts,
                            float resolution, int64_t n_edges, uint8_t *valid, int mode, void *stream);

/* Edge validity from host memory: vp_validate_edges (mode VP_MODE_PLAIN or
 * VP_MODE_BATCHED) on host arrays, the copies overlapped with the work.
 * q0, q1: host float [E][D]; counts: host int32 [E] or NULL; valid: host
 * uint8 [E] (written).  The batch is cut into chunks -- in VP_MODE_PLAIN up
 * to eight of about 2^19 edges, in VP_MODE_BATCHED (where each launch has a
 * fixed cost) a quarter and the rest once E >= 2^20 -- and each chunk's
 * inputs go to the device on a copy stream while the previous chunk is
 * validated on `stream`; each chunk's verdicts come back on a second copy
 * stream as soon as they are known.  The call
 * returns once the work is enqueued; `stream` completes only when every
 * verdict is in `valid`, so synchronise it before reading them and keep the
 * host arrays alive until then.  Page-locked host memory lets the copies run
 * asynchronously; pageable memory works but serialises them.  The context
 * keeps device copies of the arrays (grown on demand, which synchronises the
 * device).  Verdicts equal vp_validate_edges' on the same arrays; the
 * kernel-time hook does not time this call. */
vp_status vp_validate_edges_host(vp_ctx *ctx, const float *q0, const float *q1, const int32_t *counts,
                                 float resolution, int64_t n_edges, uint8_t *valid, int mode, void *stream);

/* Work counters for the FLOP model: edge validation in `mode` (VP_MODE_PLAIN
 * or VP_MODE_BATCHED, the latter launched directly rather than from its
 * graph) with counters of the work done (VP_WORK_* indices) added into `work`
 * (device uint64 [VP_WORK_N]; the caller zeroes it).  Only lanes holding a
 * state of a live edge are counted (a lane parked on a repeated state, in a
 * finished lane group or in a group that already has a collision on the
 * current state, is not), except by the VP_WORK_LANE_* slot counters. */
enum {
    VP_WORK_STATES = 0,     /* states posed (FK run)                          */
    VP_WORK_LINK_CENTRES,   /* link bounding-sphere centres computed          */
    VP_WORK_COARSE_SPHERE,  /* coarse tests, by primitive type                */
    VP_WORK_COARSE_CAPSULE,
    VP_WORK_COARSE_CUBOID,
    VP_WORK_FINE_SPHERE,    /* fine tests (incl. the sphere centre), by type  */
    VP_WORK_FINE_CAPSULE,
    VP_WORK_FINE_CUBOID,
    VP_WORK_PAIR_COARSE,    /* link-pair bounding-sphere tests                */
    VP_WORK_PAIR_FINE,      /* sphere-pair tests                              */
    VP_WORK_EDGES_DONE,     /* edges finished                                 */
    /* lane slots: the same work counted over every lane of a running warp,
     * live or idle (lockstep cost; live / slots = SIMT lane efficiency)    */
    VP_WORK_LANE_STATES,    /* poses run                                      */
    VP_WORK_LANE_COARSE,    /* coarse primitive tests, all types              */
    VP_WORK_LANE_FINE,      /* fine primitive tests, all types                */
    VP_WORK_LANE_PAIR_FINE, /* sphere-pair tests                              */
    VP_WORK_BOX_TESTS,      /* (link, primitive) world-box overlap tests that
                             * cull coarse tests (one per pair per warp)      */
    VP_WORK_FINE_OWN,       /* fine primitive tests on lanes whose own coarse
                             * test hit the link (the rest run in lockstep)   */
    VP_WORK_PAIR_FINE_OWN,  /* sphere-pair tests on lanes whose own link-pair
                             * test hit                                       */
    VP_WORK_N = 32
};
vp_status vp_validate_edges_work(vp_ctx *ctx, const float *q0, const float *q1, const int32_t *counts,
                                 float resolution, int64_t n_edges, uint8_t *valid, int mode, uint64_t *work,
                                 void *stream);

/* Penetration cost (an addition beside the paper, which defines none):
 * cost[i] = sum_s sum_o max(0, r_s + margin - d(c_s, o))^2 over environment
 * primitives o (d = signed distance, negative inside).  If grad != NULL, the
 * reverse-mode FK adjoint writes dcost/dq into grad (device float [n][D]).
 * q: device float [n][D]; cost: device float [n]. */
vp_status vp_collision_cost(vp_ctx *ctx, const float *q, int64_t n, float margin, float *cost,
                            float *grad, void *stream);

/* Tune the batched mode on a sample of edges (runs kernels and synchronises
 * the device).  First it counts, on the batch's first (up to) 65,536 start
 * configurations, how often each self-pair link pair and each primitive
 * collides with the robot, and orders both most often first: the link pairs
 * for the frequent-first orders (4 and 5), the primitives (within each kind,
 * and the kinds by their totals) for every check order -- a state that
 * collides then meets its collision sooner.  Then it chooses the tiling, and
 * the check order together with the screening rounds, by timing whole
 * launches.  The choice is cached in the context per robot, environment and
 * edge-length profile.  The verdicts do not depend on any of it, except as
 * vp_set_check_order describes for states within rounding of contact. */
vp_status vp_autotune(vp_ctx *ctx, const float *q0, const float *q1, const int32_t *counts,
                      float resolution, int64_t n_edges, void *stream);

/* Kernel timing for profiling: enable != 0 makes later vp_validate_edges
 * calls record CUDA events around their main validation kernel (inside the
 * replayed graph in VP_MODE_BATCHED); enable == 0 stops it.  If last_ms is
 * not NULL it receives the duration of that kernel in the most recent timed
 * call (waits for it to finish), or -1 if there is none. */
vp_status vp_kernel_time(vp_ctx *ctx, int enable, float *last_ms);

/* Time budget of the batched mode's persistent kernel per launch (seconds,
 * default 60).  Past it the kernel stops taking work, sets VP_DEVERR_TIMEOUT
 * and returns; edges it did not reach keep their previous output.  0 makes
 * the kernel give up at once (a way to exercise the path).  Negative or
 * non-finite values: VP_ERR_ARG. */
vp_status vp_set_watchdog(vp_ctx *ctx, double seconds);

/* The batched mode's current tiling: lanes per edge (the lane-group size,
 * 4, 8, 16 or 32) of each edge-length bucket, as vp_autotune left it (or the
 * defaults).  Bucket b holds edges of 2^(b+1)+1 .. 2^(b+2) states (bucket 0
 * also 2; the last, 8, everything above 512).  Writes min(n, 9) entries into
 * the host array lanes (n >= 0; lanes may be NULL when n == 0) and the
 * bucket count (9) into *n_buckets when it is not NULL. */
vp_status vp_tiling(vp_ctx *ctx, int32_t *lanes, int n, int *n_buckets);

/* Set the batched mode's tiling by hand (replaces the autotuner's choice
 * until the next vp_autotune or vp_load_robot / vp_load_env): lanes[b] for
 * buckets b < n (n <= 9; the rest keep their value), each 4, 8, 16 or 32;
 * VP_ERR_ARG otherwise, with nothing changed. */
vp_status vp_set_tiling(vp_ctx *ctx, const int32_t *lanes, int n);

/* Screening rounds of the batched mode.  Its first launch gives each edge
 * to a lane group for at most `rounds` raked rounds (lanes-per-edge states
 * each); edges still undecided then go to a second launch that spreads each
 * of them over whole warps, so a long collision-free edge does not keep one
 * lane group busy while the rest of the GPU idles.  0 = no limit (edges are
 * finished in the first launch).  vp_autotune chooses it along with the
 * tiling; vp_set_screen_rounds pins it (rounds >= 0, else VP_ERR_ARG) until
 * the next vp_autotune or load.  The verdicts do not depend on it. */
vp_status vp_set_screen_rounds(vp_ctx *ctx, int rounds);
vp_status vp_screen_rounds(vp_ctx *ctx, int *rounds);

/* Check order of the validation kernels (edges and states, every mode):
 * VP_ORDER_FREQUENT, or a combination of two bits:
 *   VP_ORDER_PRIMS_FIRST: primitives (link bounding spheres, then fine
 *     spheres) before self pairs; without it, self pairs first;
 *   VP_ORDER_INTERLEAVE: checks interleaved with posing, the paper's order
 *     (Sec. III-D): links are posed in order and each is checked as soon as
 *     it is posed (its self pairs with earlier links, and its spheres against
 *     the primitives), so that links after a collision are never posed;
 *     without it, every link is posed first and the checks run after.
 * VP_ORDER_FREQUENT (4): the link pairs that collide most often first (as
 *   vp_autotune counted them; before that, their packed order) -- those
 *   that hold three quarters of the counted collisions -- with each link
 *   posed only when a check first needs it; then primitives; then the
 *   remaining link pairs.
 * VP_ORDER_FREQUENT_TWO_PASS (5): the frequent-first order over a whole
 *   batch in two passes (VP_MODE_BATCHED; elsewhere as 4).  The first pass
 *   checks only the leading link pairs on each edge's first-round states;
 *   a second pass takes the edges left undecided and checks the rest on
 *   those states, so that the rest runs in full warps instead of in the
 *   few lanes of a warp whose other edges have already collided.
 * 0 (the default) is "pose all, self pairs first".  Which order finds a
 * colliding configuration with the least work depends on the robot and the
 * scene; vp_autotune times all six.  vp_set_check_order pins one
 * (VP_ERR_ARG outside 0..5) until the next vp_autotune or load.  The
 * verdicts do not depend on it, except for states within rounding of
 * contact: the orders rebuild link frames along different float paths. */
#define VP_ORDER_PRIMS_FIRST 0x1
#define VP_ORDER_INTERLEAVE 0x2
#define VP_ORDER_FREQUENT 0x4
#define VP_ORDER_FREQUENT_TWO_PASS 5
vp_status vp_set_check_order(vp_ctx *ctx, int order);
vp_status vp_check_order(vp_ctx *ctx, int *order);

/* The link-level spheres the validation kernels test first (Sec. III-D: one
 * sphere per link over-approximating it), as vp_load_robot packed them, in
 * each link's frame (host memory; synchronous; no device work).  n_links
 * must be the robot's joint count + 1.  Outputs, each of which may be NULL:
 *   link_sphere  [n_links][4] centre, radius: the given sphere or the
 *                library's bound of the link's spheres, whichever is smaller
 *                (radius < 0: the link has no spheres);
 *   half_sphere  [n_links][2][4] for a link of 4 or more spheres, the bounds
 *                of its two halves, tested before its spheres (radius < 0:
 *                the link is not split);
 *   sphere_half  [n_spheres] 0 or 1, the half holding each of the caller's
 *                spheres (-1: its link is not split).
 * Radii include the 1e-5 m float margin.  VP_ERR_NOT_LOADED without a robot,
 * VP_ERR_ARG for a wrong n_links. */
vp_status vp_link_bounds(vp_ctx *ctx, int n_links, float *link_sphere, float *half_sphere, int32_t *sphere_half);

/* Batched randomized shortcutting (Sec. III-E, "Bringing it Together": the
 * planners simplify paths by randomized shortcutting).  paths: device float
 * [P][W][D] (D = the robot's joints), in/out; lengths: device int32 [P]
 * (waypoints in use, 2..W), in/out.  For each of T steps, path p takes the
 * random numbers (u0, u1) = draws[t][p][0..1] (device float [T][P][2], in
 * [0, 1)): i = floor(u0 n), j = floor(u1 n) with the products rounded to
 * float32, clamped to n - 1 and ordered; if n >= 3 and j - i >= 2, the edge
 * waypoint i -> waypoint j is validated as vp_validate_edges does at
 * `resolution` (one batched call for all paths per step) and, when valid,
 * the waypoints strictly between are removed (later ones move up; entries
 * past the new length are left as they were).  A length outside [3, W]
 * leaves the path unchanged.  Asynchronous on `stream`; uses a scratch the
 * context keeps (grown on demand).  Needs a robot and an environment. */
vp_status vp_shortcut_paths(vp_ctx *ctx, float *paths, int32_t *lengths, int64_t P, int32_t W, const float *draws,
                            int32_t T, float resolution, void *stream);

/* Per-robot forward kinematics by code generation (Sec. III-B: the paper's
 * tracing compiler turns the robot's kinematics into straight-line code with
 * its constants folded in).  enable == 1: generate a CUDA kernel for the
 * loaded robot (every joint and sphere unrolled, fixed transforms and sphere
 * offsets as literals, zero terms dropped), compile it with NVRTC for the
 * current device (the first time), and make vp_fk_spheres use it; it
 * computes what the table-driven kernel computes, in the same order of
 * operations.  enable == 0: the table-driven kernel.  enable == -1: the
 * default after every robot load -- the generated kernel, built on the
 * first vp_fk_spheres call, or the table-driven one where building fails.
 * Loading a robot drops the generated kernel.  *compile_ms (may be NULL)
 * gets the generation and compile time (0 if none was built).  VP_ERR_CUDA
 * (and the previous choice stays in use) when enable == 1 and NVRTC is
 * missing or compilation fails; VP_ERR_ARG for another value of enable. */
vp_status vp_fk_codegen(vp_ctx *ctx, int enable, double *compile_ms);

/* Batched RRT-Connect (Sec. III-E, "Bringing it Together": RRT-Connect is one
 * of the planners built on the vectorized primitives), device-resident: B
 * independent problems (start[b] -> goal[b], device float [B][D]), each
 * grown from its own random configurations samples[b][0..T) (device float
 * [B][T][D], the caller's draws):
 *   trees A (from the start) and B (from the goal); per sample, EXTEND(A):
 *   the l2-nearest node steps toward the sample by at most `range` (radians;
 *   the sample itself when within range) and is added if that edge is valid
 *   (as vp_validate_edges checks it at `resolution`); if not trapped,
 *   CONNECT(B) extends B toward the new node until it is reached (solved)
 *   or B is trapped; then A and B swap roles.
 * Nearest-node distances and steps are FP32 with each operation rounded
 * separately (no fused multiply-add); ties go to the lowest node index.  A
 * tree holds at most `cap` nodes (cap >= 2); a full tree is trapped.
 * Outputs (device int32 unless noted): status[b] = 1 solved, 0 not within T
 * samples, -1 start or goal invalid; iters[b] = samples used; path: device
 * float [B][2 cap][D], the solved path start ... goal (path_len[b] rows;
 * 0 when unsolved); tree_sizes [B][2].  Uses a scratch the context keeps
 * (grown on demand: B * 2 * cap * (D + 1) * 4 bytes).  The watchdog of
 * vp_set_watchdog bounds the launch.  Asynchronous on `stream`. */
vp_status vp_rrt_connect(vp_ctx *ctx, const float *start, const float *goal, int64_t B, const float *samples,
                         int32_t T, float range, float resolution, int32_t cap, int32_t *status, int32_t *iters,
                         float *path, int32_t *path_len, int32_t *tree_sizes, void *stream);

/* Nearest neighbours in a Euclidean configuration space (Sec. III-E,
 * "Bringing it Together": the planners' NN structure uses the l2 distance,
 * a sum of squared coordinate differences).  For each query q_n, the index
 * of the point p_m with the least d = sum_d (q_n,d - p_m,d)^2, computed in
 * FP32 in coordinate order (one FMA per coordinate), the lowest index among
 * equal distances; dist2[n] gets that d.  Brute force over all points.
 * points: device float [M][D] (1 <= M < 2^32 - 1); queries: device float
 * [N][D]; 1 <= D <= 16.  index: device int64 [N], 8-byte aligned (also the
 * call's scratch); dist2: device float [N] or NULL.  A query whose
 * distances are all non-finite gets index -1.  Needs no robot or
 * environment; asynchronous on `stream`.  VP_ERR_ARG / VP_ERR_CAPACITY on
 * bad sizes. */
vp_status vp_nearest(vp_ctx *ctx, const float *points, int64_t M, const float *queries, int64_t N, int D,
                     int64_t *index, float *dist2, void *stream);

/* Measured FP32 FMA throughput of CUDA device `device` in TFLOP/s (an FMA is
 * two flops): independent FMA chains on every SM at full occupancy, one
 * launch grown to about seconds / 4, best of three (0 < seconds <= 60; the
 * call takes about that long).  A measurement hook: the denominator the
 * validation kernels' FLOP rate is reported against beside the one derived
 * from lane counts and the clock.  Synchronous; the current device is left
 * unchanged. */
vp_status vp_measure_fp32_peak(int device, double seconds, double *tflops);

/* Synchronise `stream`, read and clear the device status word: VP_OK,
 * VP_ERR_DEVICE (count / length bits) or VP_ERR_TIMEOUT.  The bits are
 * returned in *bits when bits != NULL. */
vp_status vp_sync_status(vp_ctx *ctx, void *stream, uint32_t *bits);

/*
 * Edge validation that allocates no device memory.
 *
 * The paper has no counterpart to this call.  It serves callers that must
 * not allocate device memory while they run -- e.g. a planner re-validating
 * edges inside a robot's real-time control loop, where cudaMalloc can block,
 * synchronise the device and take unbounded time, or a process whose device
 * memory is fixed at start-up.  Such callers cannot create a vp_ctx
 * (vp_create and vp_load_env allocate), so this call takes the robot and
 * environment descriptors directly and produces the same verdicts as
 * vp_validate_edges in VP_MODE_PLAIN.
 *
 * Scratch: the packed environment and the device status word live in one
 * file-scope static __device__ array of 256 + VP_NOALLOC_MAX_ENV_BYTES
 * bytes, which every GPU that loads the library holds until the process
 * exits.  An environment that packs to more than VP_NOALLOC_MAX_ENV_BYTES
 * (48 B per sphere, 64 B per capsule, 96 B per cuboid: each primitive with
 * its world box, as for vp_env_desc) is rejected with VP_ERR_CAPACITY
 * before anything runs.  The call calls no cudaMalloc,
 * cudaFree or other device-allocating routine; host side it packs the robot
 * with small temporaries and stages the environment in a per-thread static
 * buffer.
 *
 * Runs on the calling thread's current device.  The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress) and the
 * device's launch limits.  Every call copies the environment from pageable
 * host memory and synchronises `stream`.  Every call shares the array and it
 * keeps the previous call's contents:
 * each call restages the environment and clears the status word on
 * `stream` first.  Calls that overlap on the GPU (other host threads, other
 * streams) race on the array and must be serialised by the caller.
 *
 * Arguments are those of vp_validate_edges (q0, q1, counts, valid: device
 * pointers on the current device; `stream`: a cudaStream_t or NULL).  The
 * call returns after the work on `stream` has finished; device-side input
 * errors come back as VP_ERR_DEVICE (the affected edges are reported
 * invalid).  If errbuf != NULL, a message of at most errbuf_len bytes
 * (NUL-terminated) describes a failure.
 */
#define VP_NOALLOC_MAX_ENV_BYTES (64 * 1024)
vp_status vp_validate_edges_noalloc(const vp_robot_desc *robot, const vp_env_desc *env, const float *q0,
                                    const float *q1, const int32_t *counts, float resolution, int64_t n_edges,
                                    uint8_t *valid, void *stream, char *errbuf, int32_t errbuf_len);

#ifdef __cplusplus
}
#endif
#endif /* VP_H */
