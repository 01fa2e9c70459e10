// Device building blocks: frames, primitive tests, shared-memory staging of
// the environment, and the fused "pose one link, check it, move on" loop.
//
// Sec. III-B/C/D of arXiv 2309.14545: FK poses many configurations in
// lockstep (here: one configuration per lane), only sphere positions are
// computed, each link is checked right after it is posed (coarse bounding
// sphere first, fine spheres only for obstacles the coarse sphere touches,
// then self pairs), and the whole group of lanes stops at the first
// collision.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

#include "vp_types.h"

// Launch bounds of the validation kernels: 128 threads per block; with up
// to 9 links the register budget is capped so that `blocks` blocks stay
// resident per SM (measured best: 6 batched, 5 plain); the 17-link
// instances keep 4 (128 registers: a tighter cap makes them spill).
#define VP_VALIDATION_BOUNDS(LMAX, blocks) __launch_bounds__(128, (LMAX) <= 9 ? (blocks) : 4)
// (the 8- and 9-link instances share the first budget, 15 and 17 the second)

namespace vp {

constexpr unsigned kFull = 0xffffffffu;

// ---------------------------------------------------------------------------
// rigid frames: R row-major (columns are the frame's axes in the world), p

struct Fr {
    float r0, r1, r2, r3, r4, r5, r6, r7, r8;
    float px, py, pz;
};

__device__ __forceinline__ void fr_identity(Fr &f) {
    f.r0 = 1.f; f.r1 = 0.f; f.r2 = 0.f;
    f.r3 = 0.f; f.r4 = 1.f; f.r5 = 0.f;
    f.r6 = 0.f; f.r7 = 0.f; f.r8 = 1.f;
    f.px = 0.f; f.py = 0.f; f.pz = 0.f;
}

// world point of local point (x, y, z): R x + p (9 FMA)
__device__ __forceinline__ float3 fr_apply(const Fr &f, float x, float y, float z) {
    return make_float3(fmaf(f.r0, x, fmaf(f.r1, y, fmaf(f.r2, z, f.px))),
                       fmaf(f.r3, x, fmaf(f.r4, y, fmaf(f.r5, z, f.py))),
                       fmaf(f.r6, x, fmaf(f.r7, y, fmaf(f.r8, z, f.pz))));
}
// R^T v: a world direction in the frame's coordinates.
__device__ __forceinline__ float3 fr_unrotate(const Fr &f, float x, float y, float z) {
    return make_float3(fmaf(f.r0, x, fmaf(f.r3, y, f.r6 * z)), fmaf(f.r1, x, fmaf(f.r4, y, f.r7 * z)),
                       fmaf(f.r2, x, fmaf(f.r5, y, f.r8 * z)));
}

// The joint's motion parameters: (sin q, cos q) for a revolute joint, (q, 0)
// for a prismatic one.
__device__ __forceinline__ void joint_motion(const JointC &J, float q, float &s, float &c) {
    if (J.meta & kMetaPrismatic) {
        s = q;
        c = 0.f;
    } else {
        sincosf(q, &s, &c);
    }
}

// (sin q, cos q) for the collision checks: the SFU approximations
// (__sincosf) after reducing q to [-pi, pi] by Cody and Waite's method (2 pi
// split into a head of 8 significant bits, whose products with the small
// integer k are exact, and the tail 2 pi - head).  On [-pi, pi] the
// approximations' absolute error is at most 2^-21.41 (3.6e-7), so a chain of
// n revolute joints displaces a point at distance d from them by at most
// about n * 3.6e-7 * d: under 4e-6 m for seven joints within 1.5 m, far
// inside the boundary band of the verdicts.  FK, the cost and its gradient
// keep the accurate sincosf.
__device__ __forceinline__ void sincos_reduced(float q, float &s, float &c) {
    constexpr float kInv2Pi = 0.159154943f, kHead = 6.28125f, kTail = 1.93530717958e-3f;
    const float k = rintf(q * kInv2Pi);
    __sincosf(fmaf(-k, kTail, fmaf(-k, kHead, q)), &s, &c);
}

// joint_motion for the collision checks (sincos_reduced)
__device__ __forceinline__ void joint_motion_check(const JointC &J, float q, float &s, float &c) {
    if (J.meta & kMetaPrismatic) {
        s = q;
        c = 0.f;
    } else {
        sincos_reduced(q, s, c);
    }
}

// f <- f * origin_j * M_j: one joint of the chain, from its motion
// parameters (s, c) as given by joint_motion.  SIMPLE: the robot has only
// canonical axes (x, y, z) and identity origin rotations, so the code for
// general ones is left out.
template <bool SIMPLE = false>
__device__ __forceinline__ void apply_joint_sc(const JointC &J, float s, float c, Fr &f) {
    const int meta = J.meta;
    // translation of the fixed origin, in the parent frame
    const float tx = J.o[3], ty = J.o[7], tz = J.o[11];
    f.px = fmaf(f.r0, tx, fmaf(f.r1, ty, fmaf(f.r2, tz, f.px)));
    f.py = fmaf(f.r3, tx, fmaf(f.r4, ty, fmaf(f.r5, tz, f.py)));
    f.pz = fmaf(f.r6, tx, fmaf(f.r7, ty, fmaf(f.r8, tz, f.pz)));
    if (!SIMPLE && !(meta & kMetaOriginRotIdentity)) {
        const float *o = J.o;
        Fr g = f;
        f.r0 = fmaf(g.r0, o[0], fmaf(g.r1, o[4], g.r2 * o[8]));
        f.r1 = fmaf(g.r0, o[1], fmaf(g.r1, o[5], g.r2 * o[9]));
        f.r2 = fmaf(g.r0, o[2], fmaf(g.r1, o[6], g.r2 * o[10]));
        f.r3 = fmaf(g.r3, o[0], fmaf(g.r4, o[4], g.r5 * o[8]));
        f.r4 = fmaf(g.r3, o[1], fmaf(g.r4, o[5], g.r5 * o[9]));
        f.r5 = fmaf(g.r3, o[2], fmaf(g.r4, o[6], g.r5 * o[10]));
        f.r6 = fmaf(g.r6, o[0], fmaf(g.r7, o[4], g.r8 * o[8]));
        f.r7 = fmaf(g.r6, o[1], fmaf(g.r7, o[5], g.r8 * o[9]));
        f.r8 = fmaf(g.r6, o[2], fmaf(g.r7, o[6], g.r8 * o[10]));
    }
    if (meta & kMetaPrismatic) {
        const float q = s;
        const float ax = J.ax[0] * q, ay = J.ax[1] * q, az = J.ax[2] * q;
        f.px = fmaf(f.r0, ax, fmaf(f.r1, ay, fmaf(f.r2, az, f.px)));
        f.py = fmaf(f.r3, ax, fmaf(f.r4, ay, fmaf(f.r5, az, f.py)));
        f.pz = fmaf(f.r6, ax, fmaf(f.r7, ay, fmaf(f.r8, az, f.pz)));
        return;
    }
    const int axis = (meta >> kMetaAxisShift) & 3;
    if (axis == kAxisZ) {
        // columns 0, 1 rotate: c0' = c c0 + s c1, c1' = c c1 - s c0
        float a0 = f.r0, a1 = f.r3, a2 = f.r6;
        f.r0 = fmaf(c, a0, s * f.r1); f.r1 = fmaf(c, f.r1, -s * a0);
        f.r3 = fmaf(c, a1, s * f.r4); f.r4 = fmaf(c, f.r4, -s * a1);
        f.r6 = fmaf(c, a2, s * f.r7); f.r7 = fmaf(c, f.r7, -s * a2);
    } else if (axis == kAxisY) {
        // c0' = c c0 - s c2, c2' = s c0 + c c2
        float a0 = f.r0, a1 = f.r3, a2 = f.r6;
        f.r0 = fmaf(c, a0, -s * f.r2); f.r2 = fmaf(c, f.r2, s * a0);
        f.r3 = fmaf(c, a1, -s * f.r5); f.r5 = fmaf(c, f.r5, s * a1);
        f.r6 = fmaf(c, a2, -s * f.r8); f.r8 = fmaf(c, f.r8, s * a2);
    } else if (axis == kAxisX) {
        // c1' = c c1 + s c2, c2' = c c2 - s c1
        float a0 = f.r1, a1 = f.r4, a2 = f.r7;
        f.r1 = fmaf(c, a0, s * f.r2); f.r2 = fmaf(c, f.r2, -s * a0);
        f.r4 = fmaf(c, a1, s * f.r5); f.r5 = fmaf(c, f.r5, -s * a1);
        f.r7 = fmaf(c, a2, s * f.r8); f.r8 = fmaf(c, f.r8, -s * a2);
    } else if (!SIMPLE) {
        // Rodrigues: M = c I + (1 - c) a a^T + s [a]x, then R <- R M
        const float x = J.ax[0], y = J.ax[1], z = J.ax[2], v = 1.f - c;
        const float m00 = fmaf(v * x, x, c), m01 = fmaf(v * x, y, -s * z), m02 = fmaf(v * x, z, s * y);
        const float m10 = fmaf(v * y, x, s * z), m11 = fmaf(v * y, y, c), m12 = fmaf(v * y, z, -s * x);
        const float m20 = fmaf(v * z, x, -s * y), m21 = fmaf(v * z, y, s * x), m22 = fmaf(v * z, z, c);
        Fr g = f;
        f.r0 = fmaf(g.r0, m00, fmaf(g.r1, m10, g.r2 * m20));
        f.r1 = fmaf(g.r0, m01, fmaf(g.r1, m11, g.r2 * m21));
        f.r2 = fmaf(g.r0, m02, fmaf(g.r1, m12, g.r2 * m22));
        f.r3 = fmaf(g.r3, m00, fmaf(g.r4, m10, g.r5 * m20));
        f.r4 = fmaf(g.r3, m01, fmaf(g.r4, m11, g.r5 * m21));
        f.r5 = fmaf(g.r3, m02, fmaf(g.r4, m12, g.r5 * m22));
        f.r6 = fmaf(g.r6, m00, fmaf(g.r7, m10, g.r8 * m20));
        f.r7 = fmaf(g.r6, m01, fmaf(g.r7, m11, g.r8 * m21));
        f.r8 = fmaf(g.r6, m02, fmaf(g.r7, m12, g.r8 * m22));
    }
}

// f <- f * origin_j * M_j(q).
__device__ __forceinline__ void apply_joint(const JointC &J, float q, Fr &f) {
    float s, c;
    joint_motion(J, q, s, c);
    apply_joint_sc(J, s, c, f);
}

// ---------------------------------------------------------------------------
// primitive tests, squared forms: "does a ball (c, r) touch the primitive?"

__device__ __forceinline__ bool hit_sphere(float3 c, float r, float4 o) {
    const float dx = c.x - o.x, dy = c.y - o.y, dz = c.z - o.z;
    const float rr = r + o.w;
    return fmaf(dx, dx, fmaf(dy, dy, dz * dz)) < rr * rr;
}

// capsule: a = (p0, radius), b = (u = p1 - p0, 1/|u|^2)
__device__ __forceinline__ bool hit_capsule(float3 c, float r, float4 a, float4 b) {
    const float wx = c.x - a.x, wy = c.y - a.y, wz = c.z - a.z;
    const float t = __saturatef(fmaf(wx, b.x, fmaf(wy, b.y, wz * b.z)) * b.w);
    const float ex = fmaf(-t, b.x, wx), ey = fmaf(-t, b.y, wy), ez = fmaf(-t, b.z, wz);
    const float rr = r + a.w;
    return fmaf(ex, ex, fmaf(ey, ey, ez * ez)) < rr * rr;
}

// cuboid: a_i = (box axis i, -axis_i . centre), h = half-extents
__device__ __forceinline__ bool hit_cuboid(float3 c, float r, float4 a0, float4 a1, float4 a2, float4 h) {
    const float y0 = fmaf(a0.x, c.x, fmaf(a0.y, c.y, fmaf(a0.z, c.z, a0.w)));
    const float y1 = fmaf(a1.x, c.x, fmaf(a1.y, c.y, fmaf(a1.z, c.z, a1.w)));
    const float y2 = fmaf(a2.x, c.x, fmaf(a2.y, c.y, fmaf(a2.z, c.z, a2.w)));
    const float e0 = fmaxf(fabsf(y0) - h.x, 0.f);
    const float e1 = fmaxf(fabsf(y1) - h.y, 0.f);
    const float e2 = fmaxf(fabsf(y2) - h.z, 0.f);
    return fmaf(e0, e0, fmaf(e1, e1, e2 * e2)) < r * r;
}

// ---------------------------------------------------------------------------
// environment staging: one 1-D TMA bulk copy global -> shared per block

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Stage n_float4 float4s from global `src` into shared `dst` with
// cp.async.bulk completing on an mbarrier.  Every thread of the block calls
// this.  The wait is bounded (about one second); on expiry the status word
// gets VP_DEVERR_TIMEOUT and false is returned (the block must not use dst).
// n_float4: how much of the buffer to copy (default all of it).
__device__ __forceinline__ bool stage_env(float4 *dst, const EnvView &env, uint64_t *bar, unsigned *status,
                                          int n_float4 = -1) {
    if (n_float4 < 0) n_float4 = env.n_float4;
    if (!env.staged || n_float4 == 0) return true;  // read in place
    const float4 *src = env.data;
    const uint32_t bytes = static_cast<uint32_t>(n_float4) * 16u;
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                     : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                smem_addr(dst)),
            "l"(src), "r"(bytes), "r"(smem_addr(bar))
            : "memory");
    }
    uint32_t done = 0;
    const uint64_t t0 = global_ns();
    while (true) {
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(smem_addr(bar))
            : "memory");
        if (done) break;
        if (global_ns() - t0 > 1000000000ull) break;
    }
    const int ok = __syncthreads_and(done != 0);
    if (!ok && threadIdx.x == 0) atomicOr(status, VP_DEVERR_TIMEOUT);
    return ok != 0;
}

// ---------------------------------------------------------------------------
// per-lane stash in shared memory, slot-major and lane-interleaved (conflict
// free): full frames of branch-point links (used by the FK and cost kernels)
// and the world centres of the links' bounding spheres (validation).

struct Stash {
    float *frames;   // [n_frame_slots][12][stride]
    float *centres;  // [n_links][3][stride]
    float *motion;   // [n_joints][2][stride]: (sin q, cos q) or (q, 0) of each joint
    int stride;      // blockDim.x
    __device__ __forceinline__ float &mo(int j, int k) const {
        return motion[(j * 2 + k) * stride + threadIdx.x];
    }
    __device__ __forceinline__ float &fr(int slot, int k) const {
        return frames[(slot * 12 + k) * stride + threadIdx.x];
    }
    __device__ __forceinline__ float &ce(int slot, int k) const {
        return centres[(slot * 3 + k) * stride + threadIdx.x];
    }
    __device__ __forceinline__ void store_frame(int slot, const Fr &f) const {
        fr(slot, 0) = f.r0; fr(slot, 1) = f.r1; fr(slot, 2) = f.r2;
        fr(slot, 3) = f.r3; fr(slot, 4) = f.r4; fr(slot, 5) = f.r5;
        fr(slot, 6) = f.r6; fr(slot, 7) = f.r7; fr(slot, 8) = f.r8;
        fr(slot, 9) = f.px; fr(slot, 10) = f.py; fr(slot, 11) = f.pz;
    }
    __device__ __forceinline__ void load_frame(int slot, Fr &f) const {
        f.r0 = fr(slot, 0); f.r1 = fr(slot, 1); f.r2 = fr(slot, 2);
        f.r3 = fr(slot, 3); f.r4 = fr(slot, 4); f.r5 = fr(slot, 5);
        f.r6 = fr(slot, 6); f.r7 = fr(slot, 7); f.r8 = fr(slot, 8);
        f.px = fr(slot, 9); f.py = fr(slot, 10); f.pz = fr(slot, 11);
    }
    __device__ __forceinline__ void store_centre(int slot, float3 c) const {
        ce(slot, 0) = c.x; ce(slot, 1) = c.y; ce(slot, 2) = c.z;
    }
    __device__ __forceinline__ float3 centre(int slot) const {
        return make_float3(ce(slot, 0), ce(slot, 1), ce(slot, 2));
    }
};

// Frame of link l recomputed from the base along its joint path (ascending
// joint indices = root-to-leaf order).  Used when a self pair needs the
// frame of an earlier link: recomputing it is cheaper than holding every
// partner's frame in shared memory, which would cap the resident warps.
template <class QF>
__device__ __forceinline__ void recompute_frame(const RobotParams &P, int l, const QF &qf, Fr &g) {
    fr_identity(g);
    unsigned m = P.links[l].path;
#pragma unroll 1
    while (m) {
        const int j = __ffs(m) - 1;
        m &= m - 1;
        apply_joint(P.joints[j], qf(j), g);
    }
}

// The same from the motion parameters the posing pass kept (FMAs only).
template <bool SIMPLE>
__device__ __forceinline__ void recompute_frame_cached(const RobotParams &P, int l, const Stash &st, Fr &g) {
    fr_identity(g);
    unsigned m = P.links[l].path;
#pragma unroll 1
    while (m) {
        const int j = __ffs(m) - 1;
        m &= m - 1;
        apply_joint_sc<SIMPLE>(P.joints[j], st.mo(j, 0), st.mo(j, 1), g);
    }
}

// The validation stash for n_links links and `stride` threads laid out at p
// (stash_floats(n_links) * stride floats); no frame slots.
__device__ __forceinline__ Stash stash_at(unsigned char *p, int n_links, int stride) {
    Stash st;
    st.frames = nullptr;
    st.centres = reinterpret_cast<float *>(p);
    st.motion = st.centres + static_cast<size_t>(n_links) * kCentreFloats * stride;
    st.stride = stride;
    return st;
}

// A link frame kept between requests: the frame of the last link asked for,
// and the joints on its path.  A request for a descendant link (whose path
// contains the kept one) only applies the joints past it -- joints are
// numbered parents first, so those come after every kept joint -- and any
// other request starts again from the base.  Fine tests and self-pair groups
// visit links in ascending order, so most requests extend the kept frame.
struct FrameCursor {
    Fr f;
    unsigned done = ~0u;  // path mask of f (~0: nothing kept)
};

template <bool SIMPLE>
__device__ __forceinline__ const Fr &frame_at(const RobotParams &P, int l, const Stash &st, FrameCursor &c) {
    const unsigned path = P.links[l].path;
    unsigned m = path & ~c.done;
    if ((path & c.done) != c.done) {
        fr_identity(c.f);
        m = path;
    }
#pragma unroll 1
    while (m) {
        const int j = __ffs(m) - 1;
        m &= m - 1;
        apply_joint_sc<SIMPLE>(P.joints[j], st.mo(j, 0), st.mo(j, 1), c.f);
    }
    c.done = path;
    return c.f;
}

// ---------------------------------------------------------------------------
// work counters (only in the counting variant)

struct Work {
    uint32_t v[VP_WORK_N];
};

template <bool STATS>
struct WorkRef {
    Work *w;
    bool real;  // this lane holds a state of the edge (not a parked duplicate)
    __device__ __forceinline__ void add(int i, uint32_t n) const {
        if (STATS && real) w->v[i] += n;
    }
    // lane-slot counters: every lane of the running warp, live or not
    __device__ __forceinline__ void slot(int i, uint32_t n) const {
        if (STATS) w->v[i] += n;
    }
};

// ---------------------------------------------------------------------------
// environment view in shared memory

struct EnvSm {
    const float4 *sph;  // [ns]
    const float4 *cap;  // [2 nc]
    const float4 *box;  // [4 nb]
    const float4 *bb_sph, *bb_cap, *bb_box;  // world boxes [2 n] of each kind
    int ns, nc, nb;
    int kind_order;     // kinds in visiting order, 4 bits each
    int order;          // check order (kOrder* bits)
};

// Views of the environment: the block's shared copy (STAGED), or the device
// buffer itself.  A compile-time choice keeps the loads' address space known.
template <bool STAGED>
__device__ __forceinline__ EnvSm env_views(const float4 *sm, const EnvView &env) {
    EnvSm e;
    const float4 *base = STAGED ? sm : env.data;
    e.sph = base;
    e.cap = base + env.ns;
    e.box = base + env.ns + 2 * env.nc;
    e.bb_sph = e.box + 4 * env.nb;
    e.bb_cap = e.bb_sph + 2 * env.ns;
    e.bb_box = e.bb_cap + 2 * env.nc;
    e.ns = env.ns;
    e.nc = env.nc;
    e.nb = env.nb;
    e.kind_order = env.kind_order;
    e.order = env.order;
    return e;
}

// The same, placement chosen at run time (generic loads).
__device__ __forceinline__ EnvSm env_views_rt(const float4 *sm, const EnvView &env) {
    return env.staged ? env_views<true>(sm, env) : env_views<false>(sm, env);
}

// Early-exit rules.  Every vote spans the full warp; a warp may hold one
// edge (kStopAny: stop as soon as any lane collides), independent states
// (kStopAll: stop once every lane has collided) or several edges in lane
// groups (kStopGroups: stop once every group has a colliding lane or is idle,
// i.e. already finished with its edge).
enum : int { kStopAny = 0, kStopAll = 1, kStopGroups = 2 };

struct Ctl {
    unsigned gmask;  // lanes of this lane's group (kStopGroups)
    bool idle;       // this lane must not drive the warp: its group is finished
                     // with its edge, or (set while checking) already has a
                     // collision on the current state
};

// The warp's stop vote after a fine test; marks a lane whose group (or, for
// kStopAll, the lane itself) has collided as idle for the rest of the state.
template <int MODE>
__device__ __forceinline__ bool group_stop(Ctl &c, bool col) {
    if (MODE == kStopAny) return __any_sync(kFull, col);
    if (MODE == kStopAll) {
        c.idle = c.idle || col;
        return __all_sync(kFull, col);
    }
    const bool gcol = (__ballot_sync(kFull, col) & c.gmask) != 0u;
    c.idle = c.idle || gcol;
    return __all_sync(kFull, c.idle);
}

// A lane's vote for extra (fine) work: idle lanes never ask for it.
__device__ __forceinline__ bool wants(const Ctl &c, bool v) { return v && !c.idle; }

// ---------------------------------------------------------------------------
// the check of one configuration

// Primitive kinds: float4 words per primitive, the ball test, the work counters.
template <int KIND>
struct Kind;
template <>
struct Kind<0> {
    static constexpr int kWords = 1, kCoarse = VP_WORK_COARSE_SPHERE, kFine = VP_WORK_FINE_SPHERE;
    __device__ static __forceinline__ bool hit(float3 c, float r, const float4 *o) { return hit_sphere(c, r, o[0]); }
    // the primitive in the coordinates of frame f (x_local = R^T (x - p))
    __device__ static __forceinline__ void to_frame(const Fr &f, const float4 *o, float4 *ol) {
        const float3 c = fr_unrotate(f, o[0].x - f.px, o[0].y - f.py, o[0].z - f.pz);
        ol[0] = make_float4(c.x, c.y, c.z, o[0].w);
    }
};
template <>
struct Kind<1> {
    static constexpr int kWords = 2, kCoarse = VP_WORK_COARSE_CAPSULE, kFine = VP_WORK_FINE_CAPSULE;
    __device__ static __forceinline__ bool hit(float3 c, float r, const float4 *o) {
        return hit_capsule(c, r, o[0], o[1]);
    }
    __device__ static __forceinline__ void to_frame(const Fr &f, const float4 *o, float4 *ol) {
        const float3 a = fr_unrotate(f, o[0].x - f.px, o[0].y - f.py, o[0].z - f.pz);
        const float3 u = fr_unrotate(f, o[1].x, o[1].y, o[1].z);
        ol[0] = make_float4(a.x, a.y, a.z, o[0].w);
        ol[1] = make_float4(u.x, u.y, u.z, o[1].w);
    }
};
template <>
struct Kind<2> {
    static constexpr int kWords = 4, kCoarse = VP_WORK_COARSE_CUBOID, kFine = VP_WORK_FINE_CUBOID;
    __device__ static __forceinline__ bool hit(float3 c, float r, const float4 *o) {
        return hit_cuboid(c, r, o[0], o[1], o[2], o[3]);
    }
    // axis a_i -> R^T a_i; offset -a_i . c -> a_i . p - a_i . c (the same planes)
    __device__ static __forceinline__ void to_frame(const Fr &f, const float4 *o, float4 *ol) {
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const float3 a = fr_unrotate(f, o[i].x, o[i].y, o[i].z);
            ol[i] = make_float4(a.x, a.y, a.z, fmaf(o[i].x, f.px, fmaf(o[i].y, f.py, fmaf(o[i].z, f.pz, o[i].w))));
        }
        ol[3] = o[3];
    }
};

// Warp-wide boxes of the links: for each link, the axis-aligned box of its
// bounding sphere over the warp's live lanes (empty when none is live).  Lane
// t keeps the box of link t mod LMAX, the link it tests in box_cull below.
struct LinkBox {
    float lx, ly, lz, hx, hy, hz;
};

__device__ __forceinline__ float warp_min(float v) {
    float r;
    asm volatile("redux.sync.min.f32 %0, %1, 0xffffffff;" : "=f"(r) : "f"(v));
    return r;
}
__device__ __forceinline__ float warp_max(float v) {
    float r;
    asm volatile("redux.sync.max.f32 %0, %1, 0xffffffff;" : "=f"(r) : "f"(v));
    return r;
}

// A primitive's world box [lo, hi] against a warp-wide box.
__device__ __forceinline__ bool box_hits(const float4 &lo, const float4 &hi, const LinkBox &b) {
    return (lo.x <= b.hx) & (hi.x >= b.lx) & (lo.y <= b.hy) & (hi.y >= b.ly) & (lo.z <= b.hz) & (hi.z >= b.lz);
}

// The two levels of the primitive cull: this lane's link box (link t mod
// LMAX), and the box of every live link at once (their union, the same in
// every lane).
struct WarpBoxes {
    LinkBox link, all;
};

template <int LMAX>
__device__ __forceinline__ WarpBoxes warp_link_boxes(const RobotParams &P, const Stash &stash, bool live) {
    const float inf = __int_as_float(0x7f800000);
    const int my_l = (threadIdx.x & 31) % LMAX;
    LinkBox b{inf, inf, inf, -inf, -inf, -inf};
#pragma unroll
    for (int l = 0; l < LMAX; ++l) {
        if (!((P.link_mask >> l) & 1u)) continue;  // warp-uniform
        const float r = P.links[l].bs.w;
        const float3 c = stash.centre(l);
        const float lx = warp_min(live ? c.x - r : inf), ly = warp_min(live ? c.y - r : inf),
                    lz = warp_min(live ? c.z - r : inf);
        const float hx = warp_max(live ? c.x + r : -inf), hy = warp_max(live ? c.y + r : -inf),
                    hz = warp_max(live ? c.z + r : -inf);
        if (my_l == l) b = LinkBox{lx, ly, lz, hx, hy, hz};
    }
    // lanes of links outside the mask hold the empty box, which leaves the
    // union unchanged
    const LinkBox u{warp_min(b.lx), warp_min(b.ly), warp_min(b.lz), warp_max(b.hx), warp_max(b.hy), warp_max(b.hz)};
    return WarpBoxes{b, u};
}

// A team of warps checking the same states together (the RRT-Connect
// kernel's second phase): warp `part` of `nparts` takes every nparts-th
// self-pair group and primitive batch, and a warp that finds a collision
// raises `flag` (shared memory) so that the others stop at their next group
// or batch.  The default (nparts == 1) is a warp checking everything.
struct Team {
    int part = 0, nparts = 1;
    volatile int *flag = nullptr;
};

// Every primitive of one kind (largest first) against every link's bounding
// sphere, then the fine spheres of each link some lane's coarse test hit.
// The cull has two levels.  Primitives go in batches of 32, lane t comparing
// the world box of primitive t of the batch with the union of the live
// links' warp-wide boxes; the survivors then go 32 / LMAX at a time, lane t
// comparing survivor t / LMAX with link t mod LMAX's warp-wide box, and a
// ballot leaves the (link, primitive) pairs whose boxes overlap; only those
// take the exact ball test.  Both levels are conservative (the primitive
// boxes carry a rounding margin, and the union holds every link box), so the
// verdicts are those of testing every pair.  Returns the warp's stop
// decision.
template <int KIND, int MODE, bool STATS, int LMAX, bool SIMPLE, bool TEAM = false>
__device__ __forceinline__ bool prim_pass(const RobotParams &P, const float4 *prims, const float4 *boxes, int n,
                                          const WarpBoxes &wb, const Stash &stash, FrameCursor &fc, Ctl &ctl,
                                          bool &col, const WorkRef<STATS> &w, const Team &team = Team{}) {
    using K = Kind<KIND>;
    constexpr int PB = 32 / LMAX > 0 ? 32 / LMAX : 1;  // primitives per batch
    constexpr unsigned kLinks = (1u << LMAX) - 1u;
    const int lane = threadIdx.x & 31;
    const int my_l = lane % LMAX, my_p = lane / LMAX;
    const bool my_on = my_p < PB && ((P.link_mask >> my_l) & 1u);
    // a team splits the second level: every warp of it checks the same
    // states, so it sees the same survivors, and takes every nparts-th
    // group of them (the first level is one ballot per 32 primitives)
    int chunk = 0;
#pragma unroll 1
    for (int k0 = 0; k0 < n; k0 += 32) {
        if (TEAM && *team.flag) return true;  // another warp of the team found a collision
        bool ou = false;
        if (k0 + lane < n) {
            ou = box_hits(boxes[2 * (k0 + lane)], boxes[2 * (k0 + lane) + 1], wb.all);
            w.slot(VP_WORK_BOX_TESTS, 1);
        }
#pragma unroll 1
        for (unsigned mu = __ballot_sync(kFull, ou); mu;) {  // warp-uniform: the batch's survivors
            int sel = -1;  // survivor my_p of the next PB, as an index into the batch
#pragma unroll
            for (int i = 0; i < PB; ++i) {
                if (i == my_p && mu) sel = __ffs(mu) - 1;
                mu &= mu - 1;
            }
            const bool mine = !TEAM || chunk % team.nparts == team.part;
            ++chunk;
            bool ov = false;
            if (mine && my_on && sel >= 0) {
                ov = box_hits(boxes[2 * (k0 + sel)], boxes[2 * (k0 + sel) + 1], wb.link);
                w.slot(VP_WORK_BOX_TESTS, 1);
            }
            unsigned m = __ballot_sync(kFull, ov);
            while (m) {  // warp-uniform: survivors with an overlapping link
                const int p = (__ffs(m) - 1) / LMAX;
                const unsigned lm = (m >> (p * LMAX)) & kLinks;
                m &= ~(kLinks << (p * LMAX));
                const int k = k0 + __shfl_sync(kFull, sel, p * LMAX);
                float4 o[K::kWords];
#pragma unroll
                for (int i = 0; i < K::kWords; ++i) o[i] = prims[k * K::kWords + i];
                unsigned bits = 0;
#pragma unroll 1
                for (unsigned t = lm; t; t &= t - 1) {  // the links that survived the cull
                    const int l = __ffs(t) - 1;
                    bits |= static_cast<unsigned>(K::hit(stash.centre(l), P.links[l].bs.w, o)) << l;
                }
                w.slot(VP_WORK_LANE_COARSE, __popc(lm));
                if (!ctl.idle) w.add(K::kCoarse, __popc(lm));
                if (ctl.idle) bits = 0;
                unsigned any = __reduce_or_sync(kFull, bits);
                while (any) {
                    const int l = __ffs(any) - 1;
                    any &= any - 1;
                    const LinkC &L = P.links[l];
                    const Fr &f = frame_at<SIMPLE>(P, l, stash, fc);
                    const bool h = (bits >> l) & 1u;
                    float4 ol[K::kWords];  // the primitive in the link's frame: spheres tested in local coordinates
                    K::to_frame(f, o, ol);
                    // a link split in halves: each half's bounding sphere first; a
                    // half no lane touches is skipped by the whole warp
                    int a0 = L.s0, a1 = L.s1;
                    bool hA = h, hB = h;
                    if (L.sm < L.s1) {
                        const float4 g0 = P.halves[l][0], g1 = P.halves[l][1];
                        hA = h && K::hit(make_float3(g0.x, g0.y, g0.z), g0.w, ol);
                        hB = h && K::hit(make_float3(g1.x, g1.y, g1.z), g1.w, ol);
                        w.slot(VP_WORK_LANE_COARSE, 2);
                        if (!ctl.idle) w.add(K::kCoarse, 2);
                        if (!__any_sync(kFull, hA)) a0 = L.sm;
                        if (!__any_sync(kFull, hB)) a1 = L.sm;
                    }
                    w.slot(VP_WORK_LANE_FINE, a1 - a0);
                    if (!ctl.idle) w.add(K::kFine, a1 - a0);
                    if (STATS) w.add(VP_WORK_FINE_OWN, (hA ? max(0, L.sm - a0) : 0) + (hB ? max(0, a1 - L.sm) : 0));
#pragma unroll 1
                    for (int s = a0; s < a1; ++s) {
                        const float4 sp = P.spheres[s];
                        col |= (s < L.sm ? hA : hB) && K::hit(make_float3(sp.x, sp.y, sp.z), sp.w, ol);
                    }
                    if (group_stop<MODE>(ctl, col)) {
                        if (TEAM && (threadIdx.x & 31) == 0) *team.flag = 1;
                        return true;
                    }
                }
            }
        }
    }
    return false;
}

// Checks interleaved with posing: one link's primitives of one kind.  Every
// lane's link bounding sphere (centre cl, the link's radius) is tested
// against each primitive whose world box overlaps the link's warp-wide box
// `lb` (lane t compares primitive k0 + t of each batch of 32), then the
// link's fine spheres -- in the link frame f, which the posing pass holds in
// registers -- wherever some lane's coarse test hit.  Returns the warp's
// stop decision.
template <int KIND, int MODE, bool STATS>
__device__ __forceinline__ bool link_prim_pass(const RobotParams &P, int l, const Fr &f, float3 cl,
                                               const float4 *prims, const float4 *boxes, int n, const LinkBox &lb,
                                               Ctl &ctl, bool &col, const WorkRef<STATS> &w) {
    using K = Kind<KIND>;
    const int lane = threadIdx.x & 31;
    const LinkC &L = P.links[l];
    const float rl = L.bs.w;
#pragma unroll 1
    for (int k0 = 0; k0 < n; k0 += 32) {
        const int kb = k0 + lane;
        bool ov = false;
        if (kb < n) {
            ov = box_hits(boxes[2 * kb], boxes[2 * kb + 1], lb);
            w.slot(VP_WORK_BOX_TESTS, 1);
        }
        unsigned m = __ballot_sync(kFull, ov);
        while (m) {  // warp-uniform: primitives whose box overlaps the link's
            const int k = k0 + __ffs(m) - 1;
            m &= m - 1;
            float4 o[K::kWords];
#pragma unroll
            for (int i = 0; i < K::kWords; ++i) o[i] = prims[k * K::kWords + i];
            const bool h = !ctl.idle && K::hit(cl, rl, o);
            w.slot(VP_WORK_LANE_COARSE, 1);
            if (!ctl.idle) w.add(K::kCoarse, 1);
            if (!__any_sync(kFull, h)) continue;
            float4 ol[K::kWords];
            K::to_frame(f, o, ol);
            int a0 = L.s0, a1 = L.s1;
            bool hA = h, hB = h;
            if (L.sm < L.s1) {
                const float4 g0 = P.halves[l][0], g1 = P.halves[l][1];
                hA = h && K::hit(make_float3(g0.x, g0.y, g0.z), g0.w, ol);
                hB = h && K::hit(make_float3(g1.x, g1.y, g1.z), g1.w, ol);
                w.slot(VP_WORK_LANE_COARSE, 2);
                if (!ctl.idle) w.add(K::kCoarse, 2);
                if (!__any_sync(kFull, hA)) a0 = L.sm;
                if (!__any_sync(kFull, hB)) a1 = L.sm;
            }
            w.slot(VP_WORK_LANE_FINE, a1 - a0);
            if (!ctl.idle) w.add(K::kFine, a1 - a0);
            if (STATS) w.add(VP_WORK_FINE_OWN, (hA ? max(0, L.sm - a0) : 0) + (hB ? max(0, a1 - L.sm) : 0));
#pragma unroll 1
            for (int s = a0; s < a1; ++s) {
                const float4 sp = P.spheres[s];
                col |= (s < L.sm ? hA : hB) && K::hit(make_float3(sp.x, sp.y, sp.z), sp.w, ol);
            }
            if (group_stop<MODE>(ctl, col)) return true;
        }
    }
    return false;
}

// The paper's order (Sec. III-D, checks interleaved with FK): links are
// posed in order and each is checked as soon as it is posed -- its self
// pairs with the links posed before it, and its bounding sphere and fine
// spheres against the primitives -- so that once the state has collided
// (under MODE's stop rule) no later link is posed.  Which of the link's two
// checks comes first follows kOrderPrimsFirst.  Verdicts equal those of
// pose_and_check's pose-all order.
template <int MODE, bool STATS, int LMAX, bool SIMPLE, class QF>
__device__ __forceinline__ bool pose_and_check_interleaved(const RobotParams &P, const QF &qf, const EnvSm &env,
                                                           const Stash &stash, const Ctl &ctl_in,
                                                           const WorkRef<STATS> &w) {
    bool col = false;
    Ctl ctl = ctl_in;
    const int D = P.n_joints;
    const bool prims_first = (env.order & kOrderPrimsFirst) != 0;
    const float inf = __int_as_float(0x7f800000);
    w.add(VP_WORK_STATES, 1);
    w.slot(VP_WORK_LANE_STATES, 1);
    Fr f;
    fr_identity(f);
    FrameCursor cur_a;
#pragma unroll 1
    for (int l = 0; l <= D; ++l) {
        if (l > 0) {
            const JointC &J = P.joints[l - 1];
            const int pm = (J.meta >> kMetaParentShift) & 0xFF;
            if (pm == kParentBase)
                fr_identity(f);
            else if (pm != kParentPrev)
                recompute_frame_cached<SIMPLE>(P, (J.meta >> kMetaParentLinkShift) & 0xFF, stash, f);
            float ms, mc;
            joint_motion_check(J, qf(l - 1), ms, mc);
            stash.mo(l - 1, 0) = ms;
            stash.mo(l - 1, 1) = mc;
            apply_joint_sc<SIMPLE>(J, ms, mc, f);
        }
        const LinkC &L = P.links[l];
        if (L.s0 >= L.s1) continue;  // no spheres: nothing to check on this link
        const float3 cl = fr_apply(f, L.bs.x, L.bs.y, L.bs.z);
        stash.store_centre(l, cl);
        w.add(VP_WORK_LINK_CENTRES, 1);
#pragma unroll 1
        for (int phase = 0; phase < 2; ++phase) {
            if ((phase == 0) != prims_first) {  // self pairs whose later link is l
#pragma unroll 1
                for (int g = L.g0; g < L.g1; ++g) {
                    const GroupC G = P.groups[g];
                    const float3 ca = stash.centre(G.la);
                    const float dx = ca.x - cl.x, dy = ca.y - cl.y, dz = ca.z - cl.z;
                    const float rr = P.links[G.la].bs.w + L.bs.w;
                    const bool h = fmaf(dx, dx, fmaf(dy, dy, dz * dz)) < rr * rr;
                    if (!ctl.idle) w.add(VP_WORK_PAIR_COARSE, 1);
                    if (!__any_sync(kFull, wants(ctl, h))) continue;
                    const Fr &fa = frame_at<SIMPLE>(P, G.la, stash, cur_a);
                    w.slot(VP_WORK_LANE_PAIR_FINE, G.p1 - G.p0);
                    if (!ctl.idle) w.add(VP_WORK_PAIR_FINE, G.p1 - G.p0);
                    if (!ctl.idle && h) w.add(VP_WORK_PAIR_FINE_OWN, G.p1 - G.p0);
#pragma unroll 1
                    for (int p = G.p0; p < G.p1; ++p) {
                        const PairC pr = P.pairs[p];
                        const float4 sa = P.spheres[pr.a], sb = P.spheres[pr.b];
                        const float3 a = fr_apply(fa, sa.x, sa.y, sa.z);
                        const float3 b = fr_apply(f, sb.x, sb.y, sb.z);
                        const float ex = a.x - b.x, ey = a.y - b.y, ez = a.z - b.z;
                        const float r2 = sa.w + sb.w;
                        col |= h && (fmaf(ex, ex, fmaf(ey, ey, ez * ez)) < r2 * r2);
                    }
                    if (group_stop<MODE>(ctl, col)) return col;
                }
            } else {  // primitives against link l
                const bool live = !ctl.idle;
                const float r = L.bs.w;
                const LinkBox lb{warp_min(live ? cl.x - r : inf), warp_min(live ? cl.y - r : inf),
                                 warp_min(live ? cl.z - r : inf), warp_max(live ? cl.x + r : -inf),
                                 warp_max(live ? cl.y + r : -inf), warp_max(live ? cl.z + r : -inf)};
#pragma unroll 1
                for (int ki = 0; ki < 3; ++ki) {
                    const int kind = (env.kind_order >> (4 * ki)) & 15;
                    bool stop;
                    if (kind == 0)
                        stop = link_prim_pass<0, MODE, STATS>(P, l, f, cl, env.sph, env.bb_sph, env.ns, lb, ctl, col, w);
                    else if (kind == 1)
                        stop = link_prim_pass<1, MODE, STATS>(P, l, f, cl, env.cap, env.bb_cap, env.nc, lb, ctl, col, w);
                    else
                        stop = link_prim_pass<2, MODE, STATS>(P, l, f, cl, env.box, env.bb_box, env.nb, lb, ctl, col, w);
                    if (stop) return col;
                }
            }
        }
    }
    return col;
}

// On-demand posing for the frequent-first order: the joints whose motion
// parameters are stashed (posed) and the links whose bounding-sphere centres
// are stashed (centred), warp-uniform bit masks.  ensure() poses the joints
// on the path to link l that are not posed yet -- walking the path from the
// base (joints are numbered parents first) -- and stashes the centre of
// every sphere-carrying link it passes.
struct LazyPose {
    unsigned posed = 0, centred = 0;
};

template <bool SIMPLE, bool STATS, class QF>
__device__ __forceinline__ void ensure_link(const RobotParams &P, int l, const QF &qf, const Stash &stash,
                                            LazyPose &lp, const WorkRef<STATS> &w) {
    if ((lp.centred >> l) & 1u) return;
    Fr f;
    fr_identity(f);
    const LinkC &L0 = P.links[0];
    if (!(lp.centred & 1u) && L0.s0 < L0.s1) {  // the base link: identity frame
        stash.store_centre(0, make_float3(L0.bs.x, L0.bs.y, L0.bs.z));
        w.add(VP_WORK_LINK_CENTRES, 1);
    }
    lp.centred |= 1u;
    unsigned m = P.links[l].path;
#pragma unroll 1
    while (m) {
        const int j = __ffs(m) - 1;
        m &= m - 1;
        const JointC &J = P.joints[j];
        float ms, mc;
        if ((lp.posed >> j) & 1u) {
            ms = stash.mo(j, 0);
            mc = stash.mo(j, 1);
        } else {
            joint_motion_check(J, qf(j), ms, mc);
            stash.mo(j, 0) = ms;
            stash.mo(j, 1) = mc;
            lp.posed |= 1u << j;
        }
        apply_joint_sc<SIMPLE>(J, ms, mc, f);
        const int lj = j + 1;
        if (!((lp.centred >> lj) & 1u)) {
            const LinkC &L = P.links[lj];
            if (L.s0 < L.s1) {
                stash.store_centre(lj, fr_apply(f, L.bs.x, L.bs.y, L.bs.z));
                w.add(VP_WORK_LINK_CENTRES, 1);
            }
            lp.centred |= 1u << lj;
        }
    }
}

// Self-pair groups gorder[gi0 .. gi1) for the frequent-first order, each
// link posed when a group first needs it (pose_only: the posing alone,
// uncounted).  Returns the warp's stop decision.
template <int MODE, bool STATS, bool SIMPLE, class QF>
__device__ __forceinline__ bool frequent_groups(const RobotParams &P, int gi0, int gi1, const QF &qf,
                                                const Stash &stash, LazyPose &lp, FrameCursor &cur_a,
                                                FrameCursor &cur_b, Ctl &ctl, bool &col, const WorkRef<STATS> &w,
                                                bool pose_only = false) {
    const WorkRef<STATS> wp{w.w, w.real && !pose_only};
#pragma unroll 1
    for (int gi = gi0; gi < gi1; ++gi) {
        const GroupC G = P.groups[P.gorder[gi]];
#pragma unroll 1
        for (int side = 0; side < 2; ++side) ensure_link<SIMPLE>(P, side ? G.lb : G.la, qf, stash, lp, wp);
        if (pose_only) continue;
        const float3 ca = stash.centre(G.la), cb = stash.centre(G.lb);
        const float dx = ca.x - cb.x, dy = ca.y - cb.y, dz = ca.z - cb.z;
        const float rr = P.links[G.la].bs.w + P.links[G.lb].bs.w;
        const bool h = fmaf(dx, dx, fmaf(dy, dy, dz * dz)) < rr * rr;
        if (!ctl.idle) w.add(VP_WORK_PAIR_COARSE, 1);
        if (!__any_sync(kFull, wants(ctl, h))) continue;
        const Fr &fb = frame_at<SIMPLE>(P, G.lb, stash, cur_b);
        const Fr &fa = frame_at<SIMPLE>(P, G.la, stash, cur_a);
        w.slot(VP_WORK_LANE_PAIR_FINE, G.p1 - G.p0);
        if (!ctl.idle) w.add(VP_WORK_PAIR_FINE, G.p1 - G.p0);
        if (!ctl.idle && h) w.add(VP_WORK_PAIR_FINE_OWN, G.p1 - G.p0);
#pragma unroll 1
        for (int p = G.p0; p < G.p1; ++p) {
            const PairC pr = P.pairs[p];
            const float4 sa = P.spheres[pr.a], sb = P.spheres[pr.b];
            const float3 a = fr_apply(fa, sa.x, sa.y, sa.z);
            const float3 b = fr_apply(fb, sb.x, sb.y, sb.z);
            const float ex = a.x - b.x, ey = a.y - b.y, ez = a.z - b.z;
            const float r2 = sa.w + sb.w;
            col |= h && (fmaf(ex, ex, fmaf(ey, ey, ez * ez)) < r2 * r2);
        }
        if (group_stop<MODE>(ctl, col)) return true;
    }
    return false;
}

// The frequent-first order: the link pairs that collide most often
// (RobotParams::gorder, counted on a sample; the first n_gfront of them),
// each link posed only when a pair first needs it, so that a state that
// collides there poses only those links' paths; then, if the state is still
// free, every remaining link is posed and the primitives are checked as in
// pose_and_check_all; then the remaining link pairs.  Verdicts equal those
// of the other orders.  Only phases first_phase .. last_phase run (a state
// checked in two parts is counted once, in the part with phase 0).
template <int MODE, bool STATS, int LMAX, bool SIMPLE, class QF>
__device__ __forceinline__ bool pose_and_check_frequent(const RobotParams &P, const QF &qf, const EnvSm &env,
                                                        const Stash &stash, const Ctl &ctl_in,
                                                        const WorkRef<STATS> &w, int first_phase = 0,
                                                        int last_phase = 2) {
    bool col = false;
    Ctl ctl = ctl_in;
    if (first_phase == 0) {
        w.add(VP_WORK_STATES, 1);
        w.slot(VP_WORK_LANE_STATES, 1);
    }
    LazyPose lp;
    FrameCursor cur_a, cur_b;
    // phase 0: the leading link pairs; 1: primitives; 2: the other link
    // pairs (one loop, so that the group code is laid out once).  A state's
    // second part (first_phase > 0) still walks phase 0, posing only: the
    // same posing calls in the same order give it the values of one check
    // (phase 0 ran to its end there, since the state had not collided).
#pragma unroll 1
    for (int phase = 0; phase <= last_phase; ++phase) {
        if (phase != 1) {
            const int g0 = phase == 0 ? 0 : P.n_gfront, g1 = phase == 0 ? P.n_gfront : P.n_groups;
            if (frequent_groups<MODE, STATS, SIMPLE>(P, g0, g1, qf, stash, lp, cur_a, cur_b, ctl, col, w,
                                                     phase < first_phase))
                return col;
            continue;
        }
        // primitives: every sphere-carrying link posed, then as pose_and_check_all
#pragma unroll 1
        for (int l = 0; l < P.n_links; ++l)
            if (((P.link_mask >> l) & 1u) && !((lp.centred >> l) & 1u)) ensure_link<SIMPLE>(P, l, qf, stash, lp, w);
        const WarpBoxes wb = warp_link_boxes<LMAX>(P, stash, !ctl.idle);
        FrameCursor fc;
#pragma unroll 1
        for (int ki = 0; ki < 3; ++ki) {
            const int kind = (env.kind_order >> (4 * ki)) & 15;
            bool stop;
            if (kind == 0)
                stop = prim_pass<0, MODE, STATS, LMAX, SIMPLE>(P, env.sph, env.bb_sph, env.ns, wb, stash, fc, ctl, col,
                                                            w);
            else if (kind == 1)
                stop = prim_pass<1, MODE, STATS, LMAX, SIMPLE>(P, env.cap, env.bb_cap, env.nc, wb, stash, fc, ctl, col,
                                                            w);
            else
                stop = prim_pass<2, MODE, STATS, LMAX, SIMPLE>(P, env.box, env.bb_box, env.nb, wb, stash, fc, ctl, col,
                                                            w);
            if (stop) return col;
        }
    }
    return col;
}

// Pose one configuration and check it (Sec. III-B/C/D):
//   1. pose every link (FK is cheap next to the checks), keeping each
//      joint's (sin, cos) and the world centre of each link's bounding
//      sphere in the per-lane stash;
//   2. self pairs: link-pair bounding-sphere test, then the sphere pairs of
//      the link pairs some lane's coarse test hit;
//   3. primitives, kind by kind, each against every link's bounding sphere
//      (pairs first culled by warp-wide boxes, see prim_pass), then fine
//      spheres where a coarse test hit.
// Steps 2 and 3 swap when the environment view says so (kOrderPrimsFirst).
// Frames needed by fine tests are recomputed from the kept (sin, cos).  The
// order of checks is chosen for early exit: a colliding configuration is
// most often found by a self pair or a large primitive; it does not change
// the verdict.  LMAX bounds the link count (a compile-time bound for the
// per-link loops and the cull's lane layout).
// Returns this lane's collision flag; the warp stops early per MODE.
template <int MODE, bool STATS, int LMAX, bool SIMPLE, class QF, bool TEAM = false>
__device__ __forceinline__ bool pose_and_check_all(const RobotParams &P, const QF &qf, const EnvSm &env,
                                                   const Stash &stash, const Ctl &ctl_in, const WorkRef<STATS> &w,
                                                   const Team &team = Team{}) {
    bool col = false;
    Ctl ctl = ctl_in;
    const int D = P.n_joints;
    w.add(VP_WORK_STATES, 1);
    w.slot(VP_WORK_LANE_STATES, 1);
    // 1. pose
    {
        Fr f;
        fr_identity(f);
        for (int l = 0; l <= D; ++l) {
            if (l > 0) {
                const JointC &J = P.joints[l - 1];
                const int pm = (J.meta >> kMetaParentShift) & 0xFF;
                if (pm == kParentBase)
                    fr_identity(f);
                else if (pm != kParentPrev)
                    recompute_frame_cached<SIMPLE>(P, (J.meta >> kMetaParentLinkShift) & 0xFF, stash, f);
                float ms, mc;
                joint_motion_check(J, qf(l - 1), ms, mc);
                stash.mo(l - 1, 0) = ms;
                stash.mo(l - 1, 1) = mc;
                apply_joint_sc<SIMPLE>(J, ms, mc, f);
            }
            const LinkC &L = P.links[l];
            if (L.s0 < L.s1) {
                stash.store_centre(l, fr_apply(f, L.bs.x, L.bs.y, L.bs.z));
                w.add(VP_WORK_LINK_CENTRES, 1);
            }
        }
    }
    // 2./3. self pairs, and primitives against every link, in the order the
    //    environment view gives (which finds a colliding state sooner
    //    depends on the scene: self contact for two arms in free space,
    //    obstacles for one arm in clutter).  Self-pair groups are sorted by
    //    later link, then earlier link, so each side's frame cursor mostly
    //    extends the frame it holds; primitive pairs are culled by warp-wide
    //    link boxes.
#pragma unroll 1
    for (int phase = 0; phase < 2; ++phase) {
        if ((phase == 0) != ((env.order & kOrderPrimsFirst) != 0)) {  // self pairs
            FrameCursor cur_a, cur_b;
            for (int g = TEAM ? team.part : 0; g < P.n_groups; g += TEAM ? team.nparts : 1) {
                if (TEAM && *team.flag) return col;  // another warp of the team found a collision
                const GroupC G = P.groups[g];
                const float3 ca = stash.centre(G.la), cb = stash.centre(G.lb);
                const float dx = ca.x - cb.x, dy = ca.y - cb.y, dz = ca.z - cb.z;
                const float rr = P.links[G.la].bs.w + P.links[G.lb].bs.w;
                const bool h = fmaf(dx, dx, fmaf(dy, dy, dz * dz)) < rr * rr;
                if (!ctl.idle) w.add(VP_WORK_PAIR_COARSE, 1);
                if (__any_sync(kFull, wants(ctl, h))) {
                    const Fr &fb = frame_at<SIMPLE>(P, G.lb, stash, cur_b);
                    const Fr &fa = frame_at<SIMPLE>(P, G.la, stash, cur_a);
                    w.slot(VP_WORK_LANE_PAIR_FINE, G.p1 - G.p0);
                    if (!ctl.idle) w.add(VP_WORK_PAIR_FINE, G.p1 - G.p0);
                    if (!ctl.idle && h) w.add(VP_WORK_PAIR_FINE_OWN, G.p1 - G.p0);
#pragma unroll 1
                    for (int p = G.p0; p < G.p1; ++p) {
                        const PairC pr = P.pairs[p];
                        const float4 sa = P.spheres[pr.a], sb = P.spheres[pr.b];
                        const float3 a = fr_apply(fa, sa.x, sa.y, sa.z);
                        const float3 b = fr_apply(fb, sb.x, sb.y, sb.z);
                        const float ex = a.x - b.x, ey = a.y - b.y, ez = a.z - b.z;
                        const float r2 = sa.w + sb.w;
                        col |= h && (fmaf(ex, ex, fmaf(ey, ey, ez * ez)) < r2 * r2);
                    }
                    if (group_stop<MODE>(ctl, col)) {
                        if (TEAM && (threadIdx.x & 31) == 0) *team.flag = 1;
                        return col;
                    }
                }
            }
        } else {  // primitives
            const WarpBoxes wb = warp_link_boxes<LMAX>(P, stash, !ctl.idle);
            FrameCursor fc;
            for (int ki = 0; ki < 3; ++ki) {
                const int kind = (env.kind_order >> (4 * ki)) & 15;
                bool stop;
                if (kind == 0)
                    stop = prim_pass<0, MODE, STATS, LMAX, SIMPLE, TEAM>(P, env.sph, env.bb_sph, env.ns, wb, stash, fc,
                                                                      ctl, col, w, team);
                else if (kind == 1)
                    stop = prim_pass<1, MODE, STATS, LMAX, SIMPLE, TEAM>(P, env.cap, env.bb_cap, env.nc, wb, stash, fc,
                                                                      ctl, col, w, team);
                else
                    stop = prim_pass<2, MODE, STATS, LMAX, SIMPLE, TEAM>(P, env.box, env.bb_box, env.nb, wb, stash, fc,
                                                                      ctl, col, w, team);
                if (stop) return col;
            }
        }
    }
    return col;
}

// Kernel families: each edge kernel is instantiated once per family of
// check orders, so that each holds the code (and the registers) of one
// order only.
enum : int { kFamPoseAll = 0, kFamInterleave = 1, kFamFrequent = 2, kFamCount = 3 };

__host__ __device__ __forceinline__ int family_of(int order) {
    return (order & kOrderFrequent) ? kFamFrequent : ((order & kOrderInterleave) ? kFamInterleave : kFamPoseAll);
}

// One state checked in the order of family FAM (the prims-first bit of
// env.order still applies within it).
// The frequent-first family runs its phases first_phase .. last_phase only
// (the two-pass order's passes); the others ignore them.
template <int FAM, int MODE, bool STATS, int LMAX, bool SIMPLE, class QF>
__device__ __forceinline__ bool check_state(const RobotParams &P, const QF &qf, const EnvSm &env, const Stash &stash,
                                            const Ctl &ctl, const WorkRef<STATS> &w, int first_phase = 0,
                                            int last_phase = 2) {
    if constexpr (FAM == kFamFrequent)
        return pose_and_check_frequent<MODE, STATS, LMAX, SIMPLE>(P, qf, env, stash, ctl, w, first_phase,
                                                                  last_phase);
    else if constexpr (FAM == kFamInterleave)
        return pose_and_check_interleaved<MODE, STATS, LMAX, SIMPLE>(P, qf, env, stash, ctl, w);
    else
        return pose_and_check_all<MODE, STATS, LMAX, SIMPLE>(P, qf, env, stash, ctl, w);
}

// The same with the family chosen at run time from env.order (one kernel
// holding every order: state validation).
template <int MODE, bool STATS, int LMAX, bool SIMPLE, class QF>
__device__ __forceinline__ bool pose_and_check(const RobotParams &P, const QF &qf, const EnvSm &env,
                                               const Stash &stash, const Ctl &ctl, const WorkRef<STATS> &w) {
    const int fam = family_of(env.order);
    if (fam == kFamFrequent) return check_state<kFamFrequent, MODE, STATS, LMAX, SIMPLE>(P, qf, env, stash, ctl, w);
    if (fam == kFamInterleave) return check_state<kFamInterleave, MODE, STATS, LMAX, SIMPLE>(P, qf, env, stash, ctl, w);
    return check_state<kFamPoseAll, MODE, STATS, LMAX, SIMPLE>(P, qf, env, stash, ctl, w);
}

}  // namespace vp
