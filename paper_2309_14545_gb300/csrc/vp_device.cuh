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

// f <- f * origin_j * M_j(q): one joint of the chain.
__device__ __forceinline__ void apply_joint(const JointC &J, float q, Fr &f) {
    const int meta = J.meta;
    // translation of the fixed origin, in the parent frame
    const float tx = J.o[3], ty = J.o[7], tz = J.o[11];
    f.px = fmaf(f.r0, tx, fmaf(f.r1, ty, fmaf(f.r2, tz, f.px)));
    f.py = fmaf(f.r3, tx, fmaf(f.r4, ty, fmaf(f.r5, tz, f.py)));
    f.pz = fmaf(f.r6, tx, fmaf(f.r7, ty, fmaf(f.r8, tz, f.pz)));
    if (!(meta & kMetaOriginRotIdentity)) {
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
        const float ax = J.ax[0] * q, ay = J.ax[1] * q, az = J.ax[2] * q;
        f.px = fmaf(f.r0, ax, fmaf(f.r1, ay, fmaf(f.r2, az, f.px)));
        f.py = fmaf(f.r3, ax, fmaf(f.r4, ay, fmaf(f.r5, az, f.py)));
        f.pz = fmaf(f.r6, ax, fmaf(f.r7, ay, fmaf(f.r8, az, f.pz)));
        return;
    }
    float s, c;
    sincosf(q, &s, &c);
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
    } else {
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
__device__ __forceinline__ bool stage_env(float4 *dst, const float4 *src, int n_float4, uint64_t *bar,
                                          unsigned *status) {
    if (n_float4 == 0) return true;
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
// free): full frames of branch-point links (a joint whose parent is not the
// previous joint reads its parent's frame here) and world centres of the
// bounding spheres of links that are the earlier member of a self pair.

struct Stash {
    float *frames;   // [n_frame_slots][12][stride]
    float *centres;  // [n_centre_slots][3][stride]
    int stride;      // blockDim.x
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
    while (m) {
        const int j = __ffs(m) - 1;
        m &= m - 1;
        apply_joint(P.joints[j], qf(j), g);
    }
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
};

// ---------------------------------------------------------------------------
// environment view in shared memory

struct EnvSm {
    const float4 *sph;  // [ns]
    const float4 *cap;  // [2 nc]
    const float4 *box;  // [4 nb]
    int ns, nc, nb;
};

// Early-exit rules.  Every vote spans the full warp; a warp may hold one
// edge (kStopAny: stop as soon as any lane collides), independent states
// (kStopAll: stop once every lane has collided) or several edges in lane
// groups (kStopGroups: stop once every group has a colliding lane or is idle,
// i.e. already finished with its edge).
enum : int { kStopAny = 0, kStopAll = 1, kStopGroups = 2 };

struct Ctl {
    unsigned gmask;  // lanes of this lane's group (kStopGroups)
    bool idle;       // this lane's group is finished and must not drive the warp
};

template <int MODE>
__device__ __forceinline__ bool group_stop(const Ctl &c, bool col) {
    if (MODE == kStopAny) return __any_sync(kFull, col);
    if (MODE == kStopAll) return __all_sync(kFull, col);
    const bool gcol = (__ballot_sync(kFull, col) & c.gmask) != 0u;
    return __all_sync(kFull, gcol || c.idle);
}

// A lane's vote for extra (fine) work: idle groups never ask for it.
template <int MODE>
__device__ __forceinline__ bool wants(const Ctl &c, bool v) {
    return MODE == kStopGroups ? (v && !c.idle) : v;
}

// Coarse tests issued per warp vote, per primitive kind (independent
// dependency chains for the schedulers to interleave).
#ifndef VP_UNROLL_SPHERE
#define VP_UNROLL_SPHERE 8
#endif
#ifndef VP_UNROLL_CAPSULE
#define VP_UNROLL_CAPSULE 8
#endif
#ifndef VP_UNROLL_CUBOID
#define VP_UNROLL_CUBOID 8
#endif

// Primitive kinds: float4 words per primitive and the ball test.
struct SphereKind {
    static constexpr int kWords = 1;
    __device__ static __forceinline__ bool hit(float3 c, float r, const float4 *o) { return hit_sphere(c, r, o[0]); }
};
struct CapsuleKind {
    static constexpr int kWords = 2;
    __device__ static __forceinline__ bool hit(float3 c, float r, const float4 *o) {
        return hit_capsule(c, r, o[0], o[1]);
    }
};
struct CuboidKind {
    static constexpr int kWords = 4;
    __device__ static __forceinline__ bool hit(float3 c, float r, const float4 *o) {
        return hit_cuboid(c, r, o[0], o[1], o[2], o[3]);
    }
};

// One primitive kind against link l: coarse tests of the link's bounding
// sphere on U primitives at a time (independent chains, one warp vote per
// chunk), then fine tests of the link's spheres on each primitive some lane's
// coarse sphere touched.  Returns the group's stop decision.
template <class K, int U, int MODE, bool STATS>
__device__ __forceinline__ bool env_pass(const RobotParams &P, const LinkC &L, const Fr &f, float3 cl, float Rl,
                                         const float4 *prims, int n, const Ctl &ctl, bool &col,
                                         const WorkRef<STATS> &w, int fine_counter) {
    for (int o0 = 0; o0 < n; o0 += U) {
        unsigned bits = 0;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (o0 + u < n) {
                float4 ob[K::kWords];
#pragma unroll
                for (int k = 0; k < K::kWords; ++k) ob[k] = prims[(o0 + u) * K::kWords + k];
                bits |= static_cast<unsigned>(K::hit(cl, Rl, ob)) << u;
            }
        }
        if (MODE == kStopGroups && ctl.idle) bits = 0;
        unsigned any = 0;
        if (__any_sync(kFull, bits != 0)) {
#pragma unroll
            for (int u = 0; u < U; ++u) any |= static_cast<unsigned>(__any_sync(kFull, (bits >> u) & 1u)) << u;
        }
        while (any) {
            const int u = __ffs(any) - 1;
            any &= any - 1;
            const bool h = (bits >> u) & 1u;
            float4 ob[K::kWords];
#pragma unroll
            for (int k = 0; k < K::kWords; ++k) ob[k] = prims[(o0 + u) * K::kWords + k];
            w.add(fine_counter, L.s1 - L.s0);
            for (int s = L.s0; s < L.s1; ++s) {
                const float4 sp = P.spheres[s];
                col |= h && K::hit(fr_apply(f, sp.x, sp.y, sp.z), sp.w, ob);
            }
            if (group_stop<MODE>(ctl, col)) return true;
        }
    }
    return false;
}

// Check link l (posed as f) against the environment, coarse then fine, then
// its self-collision groups.  `col` accumulates this lane's collision; the
// return value is the group's stop decision.
template <int MODE, bool STATS, class QF>
__device__ __forceinline__ bool check_link(const RobotParams &P, int l, const Fr &f, float3 &cl, const QF &qf,
                                           const EnvSm &env, const Stash &stash, const Ctl &ctl, bool &col,
                                           const WorkRef<STATS> &w) {
    const LinkC &L = P.links[l];
    const bool has_spheres = L.s0 < L.s1;
    if (has_spheres) {
        cl = fr_apply(f, L.bs.x, L.bs.y, L.bs.z);
        const float Rl = L.bs.w;
        w.add(VP_WORK_LINK_CENTRES, 1);
        w.add(VP_WORK_COARSE_SPHERE, env.ns);
        w.add(VP_WORK_COARSE_CAPSULE, env.nc);
        w.add(VP_WORK_COARSE_CUBOID, env.nb);
        if (env_pass<SphereKind, VP_UNROLL_SPHERE, MODE, STATS>(P, L, f, cl, Rl, env.sph, env.ns, ctl, col, w, VP_WORK_FINE_SPHERE))
            return true;
        if (env_pass<CapsuleKind, VP_UNROLL_CAPSULE, MODE, STATS>(P, L, f, cl, Rl, env.cap, env.nc, ctl, col, w,
                                                  VP_WORK_FINE_CAPSULE))
            return true;
        if (env_pass<CuboidKind, VP_UNROLL_CUBOID, MODE, STATS>(P, L, f, cl, Rl, env.box, env.nb, ctl, col, w,
                                                 VP_WORK_FINE_CUBOID))
            return true;
    }
    // self pairs whose later link is l
    for (int g = L.g0; g < L.g1; ++g) {
        const GroupC G = P.groups[g];
        const LinkC &La = P.links[G.la];
        float3 ca;
        if (G.slot_a >= 0)
            ca = stash.centre(G.slot_a);
        else if (G.slot_a == kSlotBase)
            ca = make_float3(La.bs.x, La.bs.y, La.bs.z);
        else
            ca = cl;
        const float dx = ca.x - cl.x, dy = ca.y - cl.y, dz = ca.z - cl.z;
        const float rr = La.bs.w + L.bs.w;
        const bool h = fmaf(dx, dx, fmaf(dy, dy, dz * dz)) < rr * rr;
        w.add(VP_WORK_PAIR_COARSE, 1);
        if (__any_sync(kFull, wants<MODE>(ctl, h))) {
            Fr fa;
            if (G.slot_a >= 0)
                recompute_frame(P, G.la, qf, fa);
            else if (G.slot_a == kSlotBase)
                fr_identity(fa);
            else
                fa = f;
            w.add(VP_WORK_PAIR_FINE, G.p1 - G.p0);
            for (int p = G.p0; p < G.p1; ++p) {
                const PairC pr = P.pairs[p];
                const float4 sa = P.spheres[pr.a], sb = P.spheres[pr.b];
                const float3 a = fr_apply(fa, sa.x, sa.y, sa.z);
                const float3 b = fr_apply(f, sb.x, sb.y, sb.z);
                const float ex = a.x - b.x, ey = a.y - b.y, ez = a.z - b.z;
                const float r2 = sa.w + sb.w;
                col |= h && (fmaf(ex, ex, fmaf(ey, ey, ez * ez)) < r2 * r2);
            }
            if (group_stop<MODE>(ctl, col)) return true;
        }
    }
    return false;
}

// Pose a configuration link by link and check each link as soon as it is
// posed (Sec. III-D: checks interleaved into FK; links after a collision are
// never posed).  qf(j) returns joint j's coordinate for this lane.
// Returns this lane's collision flag (the warp stops early per MODE).
template <int MODE, bool STATS, class QF>
__device__ __forceinline__ bool pose_and_check(const RobotParams &P, const QF &qf, const EnvSm &env,
                                               const Stash &stash, const Ctl &ctl, const WorkRef<STATS> &w) {
    bool col = false;
    Fr f;
    fr_identity(f);
    float3 cl = make_float3(0.f, 0.f, 0.f);
    w.add(VP_WORK_STATES, 1);
    const int D = P.n_joints;
    // link 0 is the base (identity frame); link l > 0 follows joint l - 1.
    // One call site for check_link keeps the kernel's code compact.
    for (int l = 0; l <= D; ++l) {
        if (l > 0) {
            const JointC &J = P.joints[l - 1];
            const int pm = (J.meta >> kMetaParentShift) & 0xFF;
            if (pm == kParentBase)
                fr_identity(f);
            else if (pm != kParentPrev)
                stash.load_frame(pm, f);
            apply_joint(J, qf(l - 1), f);
        }
        if (check_link<MODE, STATS>(P, l, f, cl, qf, env, stash, ctl, col, w)) return col;
        const LinkC &Lk = P.links[l];
        if (Lk.slot >= 0) stash.store_frame(Lk.slot, f);
        if (Lk.cslot >= 0) stash.store_centre(Lk.cslot, cl);
    }
    return col;
}

}  // namespace vp
