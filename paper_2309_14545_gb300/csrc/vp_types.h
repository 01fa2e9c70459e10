// Packed robot and environment tables shared by the host packer and the
// kernels.  The robot travels as a __grid_constant__ kernel parameter (it
// lives in the constant bank, read with warp-uniform indices); the
// environment is a float4 buffer that every block stages into shared memory.
#pragma once

#include <cstdint>

#include "../../include/vp.h"

#ifndef __CUDACC__
struct alignas(16) float4 { float x, y, z, w; };
#endif

namespace vp {

constexpr int kMaxJoints = VP_MAX_JOINTS;
constexpr int kMaxLinks = VP_MAX_JOINTS + 1;
constexpr int kMaxSpheres = VP_MAX_SPHERES;
constexpr int kMaxPairs = VP_MAX_PAIRS;
constexpr int kMaxGroups = 160;  // link pairs holding self pairs (<= 17*18/2)

// JointC::meta bit fields
constexpr int kMetaPrismatic = 1 << 0;
constexpr int kMetaOriginRotIdentity = 1 << 1;
constexpr int kMetaAxisShift = 2;  // 2 bits: 0 x, 1 y, 2 z, 3 general
constexpr int kAxisX = 0, kAxisY = 1, kAxisZ = 2, kAxisGeneral = 3;
constexpr int kMetaParentShift = 8;  // 8 bits: parent frame source
constexpr int kParentPrev = 0xFF;    // the previous joint's link (kept in registers)
constexpr int kParentBase = 0xFE;    // the base (identity)
// any other value: the frame-stash slot holding the parent link's frame
constexpr int kMetaParentLinkShift = 16;  // 8 bits: the parent link's index

// Shared-memory floats per lane for each kind of stash slot.
constexpr int kFrameFloats = 12;   // frame [R row-major | p] of a branch-point link
constexpr int kCentreFloats = 3;   // world centre of a link's bounding sphere

// Per-lane floats of the validation stash for n links: each link's centre,
// then each joint's motion parameters (sin q, cos q).
__host__ __device__ constexpr int stash_floats(int n_links) { return n_links * kCentreFloats + (n_links - 1) * 2; }

// Conservative inflation of every link bounding sphere (m): covers float32
// rounding in the coarse test so a coarse miss never hides a fine hit.
constexpr float kCoarseEps = 1e-5f;

struct JointC {  // 64 bytes
    float o[12];  // fixed origin [R | t], row-major
    float ax[3];  // unit axis in the joint frame
    int meta;
};

struct LinkC {  // 32 bytes
    float4 bs;       // bounding sphere: centre (link frame), radius (+eps); radius < 0: no spheres
    int16_t s0, s1;  // fine spheres [s0, s1) in sorted order
    int16_t g0, g1;  // self groups [g0, g1) checked once this link is posed
    int16_t slot;    // frame-stash slot (branch point; FK and cost kernels), -1 if none
    uint16_t path;   // joints from the base to this link (bit j = joint j)
    int16_t sm;      // the spheres split in halves [s0, sm), [sm, s1) (sm == s1: not split);
                     // RobotParams::halves holds their bounding spheres
    int16_t pad;
};

struct GroupC {      // one link pair (la <= lb) and its sphere pairs
    int16_t la;      // earlier link
    int16_t lb;      // later link
    int16_t p0, p1;  // pairs [p0, p1)
};

struct PairC {
    uint16_t a, b;  // sorted sphere indices: a on the group's la, b on lb
};

struct RobotParams {
    int n_joints, n_links, n_spheres, n_pairs, n_groups;
    int n_slots;    // frame-stash slots (branch points)
    unsigned link_mask;  // bit l: link l has spheres
    int simple;          // 1: canonical axes and identity origin rotations only
    int n_gfront;        // frequent-first order: groups gorder[0, n_gfront) go before the primitives
    JointC joints[kMaxJoints];
    LinkC links[kMaxLinks];
    float4 halves[kMaxLinks][2];  // bounding spheres of a split link's halves (link frame, radius + eps)
    float4 spheres[kMaxSpheres];  // local centre, radius (sorted by link)
    GroupC groups[kMaxGroups];
    PairC pairs[kMaxPairs];
    uint16_t perm[kMaxSpheres];   // sorted index -> caller's sphere index
    uint8_t gorder[kMaxGroups];   // the groups in the frequent-first order (kOrderFrequent):
                                  // most often colliding first, as counted on a sample
};

// Environment layout (float4 units): spheres [ns] (c, r); capsules [2 nc]
// ((p0, r), (u = p1 - p0, 1/|u|^2)); cuboids [4 nb] ((a_i, -a_i . c) for the
// three box axes a_i, then (h, 0)); then the world axis-aligned box of every
// primitive [2 (ns + nc + nb)] ((lo, 0), (hi, 0)), kinds in the same order
// (spheres, capsules, cuboids), each box grown outward by a margin that
// covers the float rounding of the exact tests (kBoxMargin*).  Each kind is
// stored largest bounding radius first; kind_order lists the kinds (0
// sphere, 1 capsule, 2 cuboid; 4 bits each) in order of their largest member.
struct EnvView {
    const float4 *data;
    int ns, nc, nb;
    int n_float4;    // total float4 count
    int kind_order;  // visiting order of the kinds
    int staged;      // 1: each block copies it into shared memory; 0: read in place (through L1)
    int order;       // check order (kOrder* bits, set per launch)
};

// Check orders (EnvView::order): 0-3 combine two bits, primitives before
// self pairs and checks interleaved with posing (each link checked as soon
// as it is posed, later links left unposed once the state has collided)
// instead of every link posed first; 4 is the frequent-first order.
constexpr int kOrderPrimsFirst = VP_ORDER_PRIMS_FIRST;
constexpr int kOrderInterleave = VP_ORDER_INTERLEAVE;
// Self-pair groups most often colliding first (RobotParams::gorder), each
// link posed when a check first needs it, then primitives; 5 is the same in
// two passes over a batch (the leading groups of every edge first).
constexpr int kOrderFrequent = VP_ORDER_FREQUENT;
constexpr int kOrderTwoPass = VP_ORDER_FREQUENT_TWO_PASS;
constexpr int kOrderCount = 6;

// Dynamic shared memory the environment takes in a block.
__host__ __device__ inline size_t env_smem_bytes(const EnvView &env) {
    return env.staged ? static_cast<size_t>(env.n_float4) * 16 : 0;
}

// float4s of the primitive data alone (the boxes that follow are for culling).
__host__ __device__ inline int env_prim_float4(const EnvView &env) { return env.ns + 2 * env.nc + 4 * env.nb; }

// Primitive box margin: kBoxMarginAbs + kBoxMarginRel * (1 + max |coordinate|)
// metres.  An fp32 ball test that reports contact implies a true distance
// below the radius plus a few ulp of the coordinates (about 1e-6 m per metre
// of coordinate); the margin is ten times that and more.
constexpr double kBoxMarginAbs = 1e-4;
constexpr double kBoxMarginRel = 1e-5;

}  // namespace vp
