// C ABI of libvp (see include/vp.h): context, robot / environment packing
// with argument checks, and dispatch to the kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "vp_batched.h"
#include "vp_cost.h"
#include "vp_internal.h"

using namespace vp;

struct vp_ctx {
    int device = 0;
    int num_sms = 0;
    size_t smem_optin = 0;
    RobotParams robot{};
    bool robot_loaded = false;
    std::vector<uint16_t> sorted_of;  // caller's sphere index -> sorted index
    float4 *env_buf = nullptr;
    std::vector<float4> env_host;  // the packed environment as on the device (visiting order)
    EnvView env{};
    uint64_t env_hash = 0;       // contents of the packed environment (tuning-cache key)
    bool env_loaded = false;
    unsigned *status = nullptr;  // device status word
    BatchedState batched;        // scratch and tuned tiling of the batched mode
    bool timing = false;         // record events around the validation kernel
    bool timed = false;          // a timed call has been issued
    cudaEvent_t ev_start = nullptr, ev_stop = nullptr;
    // shortcutting scratch: candidate edges, their waypoint pairs and verdicts
    float *sc_q0 = nullptr, *sc_q1 = nullptr;
    int2 *sc_ij = nullptr;
    uint8_t *sc_ok = nullptr;
    int64_t sc_cap = 0;
    int sc_dof = 0;
    // planner scratch: tree nodes and parents, and the problem counter
    float *rrt_nodes = nullptr;
    int *rrt_parent = nullptr, *rrt_queue = nullptr;  // rrt_queue: 3 counters
    int *rrt_pending = nullptr;                        // [B] ints, then [B] int4 (saved states)
    // vp_validate_edges_host: device copies of the caller's host arrays, the
    // copy streams and the events that chain the chunks
    float *hx_q0 = nullptr, *hx_q1 = nullptr;
    int32_t *hx_counts = nullptr;
    uint8_t *hx_valid = nullptr;
    size_t hx_cap_q = 0, hx_cap_e = 0;
    cudaStream_t hx_in = nullptr, hx_out = nullptr;
    // batched chunks alternate between two compute streams, each with its
    // own bucketing scratch, so that one chunk's persistent launch fills the
    // SMs the previous one's tail leaves idle
    cudaStream_t hx_cs[2] = {};
    BatchedState hx_slot[2];
    cudaEvent_t hx_ev[2 * 8 + 2] = {};
    size_t rrt_node_cap = 0, rrt_parent_cap = 0, rrt_pending_cap = 0;
    FkCodegen fk_gen;            // per-robot FK compiled at run time (vp_fk_codegen)
    int fk_mode = -1;            // 1 generated, 0 table-driven, -1 automatic (generated once it builds)
    bool fk_gen_failed = false;  // automatic mode: the generator failed for this robot (use the table)
    std::string err;
};

namespace {

class DeviceGuard {
   public:
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev_) != cudaSuccess) prev_ = -1;
        if (prev_ != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        if (prev_ >= 0) {
            int cur = -1;
            cudaGetDevice(&cur);
            if (cur != prev_) cudaSetDevice(prev_);
        }
    }

   private:
    int prev_ = -1;
};

vp_status fail(vp_ctx *ctx, vp_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (ctx) ctx->err = buf;
    return s;
}

vp_status cuda_fail(vp_ctx *ctx, cudaError_t e, const char *what) {
    return fail(ctx, VP_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

bool finite_all(const double *p, size_t n) {
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(p[i])) return false;
    return true;
}

double norm3(const double *v) { return std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]); }

vp_status check_loaded(vp_ctx *ctx) {
    if (!ctx) return VP_ERR_ARG;
    if (!ctx->robot_loaded) return fail(ctx, VP_ERR_NOT_LOADED, "robot not loaded");
    if (!ctx->env_loaded) return fail(ctx, VP_ERR_NOT_LOADED, "environment not loaded");
    return VP_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// lifetime

extern "C" vp_status vp_create(vp_ctx **out, int device) {
    if (!out) return VP_ERR_ARG;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return VP_ERR_ARG;
    vp_ctx *ctx = new vp_ctx();
    ctx->device = device;
    DeviceGuard g(device);
    cudaDeviceProp prop;
    cudaError_t e = cudaGetDeviceProperties(&prop, device);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->status, 256);
    if (e == cudaSuccess) e = cudaMemset(ctx->status, 0, 256);
    if (e != cudaSuccess) {
        if (ctx->status) cudaFree(ctx->status);
        delete ctx;
        return VP_ERR_CUDA;
    }
    ctx->num_sms = prop.multiProcessorCount;
    ctx->smem_optin = prop.sharedMemPerBlockOptin;
    *out = ctx;
    return VP_OK;
}

extern "C" vp_status vp_destroy(vp_ctx *ctx) {
    if (!ctx) return VP_OK;
    {
        DeviceGuard g(ctx->device);
        if (ctx->env_buf) cudaFree(ctx->env_buf);
        if (ctx->status) cudaFree(ctx->status);
        batched_release(ctx->batched);
        for (BatchedState &bs : ctx->hx_slot) batched_release(bs);
        for (cudaStream_t cs : ctx->hx_cs)
            if (cs) cudaStreamDestroy(cs);
        if (ctx->ev_start) cudaEventDestroy(ctx->ev_start);
        if (ctx->ev_stop) cudaEventDestroy(ctx->ev_stop);
        if (ctx->sc_q0) cudaFree(ctx->sc_q0);
        if (ctx->sc_q1) cudaFree(ctx->sc_q1);
        if (ctx->sc_ij) cudaFree(ctx->sc_ij);
        if (ctx->sc_ok) cudaFree(ctx->sc_ok);
        if (ctx->rrt_nodes) cudaFree(ctx->rrt_nodes);
        if (ctx->rrt_parent) cudaFree(ctx->rrt_parent);
        if (ctx->rrt_queue) cudaFree(ctx->rrt_queue);
        if (ctx->rrt_pending) cudaFree(ctx->rrt_pending);
        cudaFree(ctx->hx_q0);
        cudaFree(ctx->hx_q1);
        cudaFree(ctx->hx_counts);
        cudaFree(ctx->hx_valid);
        if (ctx->hx_in) cudaStreamDestroy(ctx->hx_in);
        if (ctx->hx_out) cudaStreamDestroy(ctx->hx_out);
        for (cudaEvent_t ev : ctx->hx_ev)
            if (ev) cudaEventDestroy(ev);
        fk_codegen_release(&ctx->fk_gen);
    }
    delete ctx;
    return VP_OK;
}

extern "C" const char *vp_last_error(const vp_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

// ---------------------------------------------------------------------------
// robot

extern "C" vp_status vp_load_robot(vp_ctx *ctx, const vp_robot_desc *r) {
    if (!ctx) return VP_ERR_ARG;
    if (!r) return fail(ctx, VP_ERR_ARG, "robot descriptor is NULL");
    const int D = r->n_joints, S = r->n_spheres, P = r->n_pairs;
    if (D < 1) return fail(ctx, VP_ERR_ARG, "n_joints must be >= 1");
    if (D > kMaxJoints) return fail(ctx, VP_ERR_CAPACITY, "n_joints %d > %d", D, kMaxJoints);
    if (S < 0 || P < 0) return fail(ctx, VP_ERR_ARG, "negative sphere or pair count");
    if (S > kMaxSpheres) return fail(ctx, VP_ERR_CAPACITY, "n_spheres %d > %d", S, kMaxSpheres);
    if (P > kMaxPairs) return fail(ctx, VP_ERR_CAPACITY, "n_pairs %d > %d", P, kMaxPairs);
    if (!r->joint_parent || !r->joint_type || !r->joint_axis || !r->joint_origin)
        return fail(ctx, VP_ERR_ARG, "joint table pointer is NULL");
    if (S > 0 && (!r->sphere_link || !r->sphere_centre || !r->sphere_radius))
        return fail(ctx, VP_ERR_ARG, "sphere table pointer is NULL");
    if (P > 0 && !r->self_pairs) return fail(ctx, VP_ERR_ARG, "self_pairs is NULL");
    const int L = D + 1;

    RobotParams rp;
    std::memset(&rp, 0, sizeof(rp));
    rp.n_joints = D;
    rp.n_links = L;
    rp.n_spheres = S;
    rp.n_pairs = P;

    // joints
    std::vector<int> parent_link(D);
    for (int j = 0; j < D; ++j) {
        const int p = r->joint_parent[j];
        if (p < -1 || p >= j) return fail(ctx, VP_ERR_ARG, "joint %d: parent %d must be -1 or an earlier joint", j, p);
        parent_link[j] = p + 1;
        const int t = r->joint_type[j];
        if (t != VP_JOINT_REVOLUTE && t != VP_JOINT_PRISMATIC) return fail(ctx, VP_ERR_ARG, "joint %d: bad type %d", j, t);
        const double *ax = r->joint_axis + 3 * j;
        const double *o = r->joint_origin + 12 * j;
        if (!finite_all(ax, 3) || !finite_all(o, 12)) return fail(ctx, VP_ERR_ARG, "joint %d: non-finite axis or origin", j);
        const double n = norm3(ax);
        if (std::fabs(n - 1.0) > 1e-6) return fail(ctx, VP_ERR_ARG, "joint %d: axis is not a unit vector", j);
        JointC &J = rp.joints[j];
        for (int i = 0; i < 12; ++i) J.o[i] = static_cast<float>(o[i]);
        for (int i = 0; i < 3; ++i) J.ax[i] = static_cast<float>(ax[i] / n);
        int meta = (t == VP_JOINT_PRISMATIC) ? kMetaPrismatic : 0;
        bool rot_id = true;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) rot_id &= o[4 * a + b] == (a == b ? 1.0 : 0.0);
        if (rot_id) meta |= kMetaOriginRotIdentity;
        int axis = kAxisGeneral;
        if (ax[0] == 1.0 && ax[1] == 0.0 && ax[2] == 0.0) axis = kAxisX;
        if (ax[0] == 0.0 && ax[1] == 1.0 && ax[2] == 0.0) axis = kAxisY;
        if (ax[0] == 0.0 && ax[1] == 0.0 && ax[2] == 1.0) axis = kAxisZ;
        meta |= axis << kMetaAxisShift;
        J.meta = meta;  // parent source filled in below
    }

    // spheres, sorted by link (stable)
    std::vector<int> order(S);
    for (int s = 0; s < S; ++s) {
        const int l = r->sphere_link[s];
        if (l < 0 || l >= L) return fail(ctx, VP_ERR_ARG, "sphere %d: link %d out of range", s, l);
        if (!finite_all(r->sphere_centre + 3 * s, 3) || !std::isfinite(r->sphere_radius[s]) || r->sphere_radius[s] < 0)
            return fail(ctx, VP_ERR_ARG, "sphere %d: bad centre or radius", s);
        order[s] = s;
    }
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return r->sphere_link[a] < r->sphere_link[b]; });
    // within a link of 4 or more spheres: along the principal axis of their
    // centres, so the first and second halves are compact (each gets its own
    // bounding sphere below)
    for (int i = 0; i < S;) {
        const int l = r->sphere_link[order[i]];
        int j = i;
        while (j < S && r->sphere_link[order[j]] == l) ++j;
        if (j - i >= 4) {
            double m[3] = {0, 0, 0}, C[3][3] = {{0}};
            for (int k = i; k < j; ++k)
                for (int a = 0; a < 3; ++a) m[a] += r->sphere_centre[3 * order[k] + a] / (j - i);
            for (int k = i; k < j; ++k)
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b)
                        C[a][b] += (r->sphere_centre[3 * order[k] + a] - m[a]) * (r->sphere_centre[3 * order[k] + b] - m[b]);
            double u[3] = {C[0][0] + 1e-12, C[1][1] + 2e-12, C[2][2] + 3e-12};  // power iteration
            for (int it = 0; it < 64; ++it) {
                double v[3];
                for (int a = 0; a < 3; ++a) v[a] = C[a][0] * u[0] + C[a][1] * u[1] + C[a][2] * u[2];
                const double n = norm3(v);
                if (!(n > 0)) break;
                for (int a = 0; a < 3; ++a) u[a] = v[a] / n;
            }
            auto proj = [&](int s) {
                const double *p = r->sphere_centre + 3 * s;
                return p[0] * u[0] + p[1] * u[1] + p[2] * u[2];
            };
            std::stable_sort(order.begin() + i, order.begin() + j, [&](int a, int b) { return proj(a) < proj(b); });
        }
        i = j;
    }
    std::vector<uint16_t> sorted_of(S);
    for (int i = 0; i < S; ++i) {
        const int s = order[i];
        sorted_of[s] = static_cast<uint16_t>(i);
        rp.perm[i] = static_cast<uint16_t>(s);
        const double *c = r->sphere_centre + 3 * s;
        rp.spheres[i] = float4{static_cast<float>(c[0]), static_cast<float>(c[1]), static_cast<float>(c[2]),
                               static_cast<float>(r->sphere_radius[s])};
    }
    for (int l = 0; l < L; ++l) {
        LinkC &K = rp.links[l];
        K.slot = -1;
        K.s0 = K.s1 = 0;
        K.g0 = K.g1 = 0;
        K.bs = float4{0.f, 0.f, 0.f, -1.f};
        K.sm = 0;
        K.pad = 0;
        rp.halves[l][0] = rp.halves[l][1] = float4{0.f, 0.f, 0.f, -1.f};
    }
    for (int i = 0; i < S;) {
        const int l = r->sphere_link[order[i]];
        int j = i;
        while (j < S && r->sphere_link[order[j]] == l) ++j;
        rp.links[l].s0 = static_cast<int16_t>(i);
        rp.links[l].s1 = static_cast<int16_t>(j);
        rp.links[l].sm = static_cast<int16_t>(j);
        i = j;
    }
    // bounding sphere of the sorted spheres [a, b) in their link's frame:
    // start from the better of two centres (the mean of the centres, the
    // middle of the box around the spheres), then take Badoiu-Clarkson steps
    // (move the centre 1/(k+1) of the way to the farthest surface point) and
    // keep the best centre seen.  The radius is recomputed exactly for each
    // centre, so the sphere encloses every sphere in double precision; the
    // float radius gets kCoarseEps on top.
    auto bound_spheres = [&](int a, int b, double c[3], int steps = 256) {
        double m[3] = {0, 0, 0}, lo[3], hi[3];
        for (int d = 0; d < 3; ++d) lo[d] = HUGE_VAL, hi[d] = -HUGE_VAL;
        for (int k = a; k < b; ++k) {
            const double *p = r->sphere_centre + 3 * order[k];
            const double rad = r->sphere_radius[order[k]];
            for (int d = 0; d < 3; ++d) {
                m[d] += p[d] / (b - a);
                lo[d] = std::min(lo[d], p[d] - rad);
                hi[d] = std::max(hi[d], p[d] + rad);
            }
        }
        auto radius_about = [&](const double *q) {
            double R = 0;
            for (int k = a; k < b; ++k) {
                const double *p = r->sphere_centre + 3 * order[k];
                const double d3[3] = {p[0] - q[0], p[1] - q[1], p[2] - q[2]};
                R = std::max(R, norm3(d3) + r->sphere_radius[order[k]]);
            }
            return R;
        };
        const double mid[3] = {0.5 * (lo[0] + hi[0]), 0.5 * (lo[1] + hi[1]), 0.5 * (lo[2] + hi[2])};
        const double Rm = radius_about(m), Rb = radius_about(mid);
        const double *best = Rb < Rm ? mid : m;
        double R = std::min(Rm, Rb), x[3];
        for (int d = 0; d < 3; ++d) c[d] = x[d] = best[d];
        for (int it = 1; it <= steps; ++it) {
            int far = a;
            double fd = -1, v[3] = {0, 0, 0};
            for (int k = a; k < b; ++k) {
                const double *p = r->sphere_centre + 3 * order[k];
                const double d3[3] = {p[0] - x[0], p[1] - x[1], p[2] - x[2]};
                const double dk = norm3(d3) + r->sphere_radius[order[k]];
                if (dk > fd) fd = dk, far = k, v[0] = d3[0], v[1] = d3[1], v[2] = d3[2];
            }
            const double n = norm3(v), rad = r->sphere_radius[order[far]];
            const double *p = r->sphere_centre + 3 * order[far];
            for (int d = 0; d < 3; ++d) {
                const double target = p[d] + (n > 0 ? v[d] / n * rad : 0.0);
                x[d] += (target - x[d]) / (it + 1);
            }
            const double Rx = radius_about(x);
            if (Rx < R) {
                R = Rx;
                for (int d = 0; d < 3; ++d) c[d] = x[d];
            }
        }
        return R;
    };
    auto half_sphere = [&](int a, int b) {
        double c[3];
        const double R = bound_spheres(a, b, c);
        return float4{static_cast<float>(c[0]), static_cast<float>(c[1]), static_cast<float>(c[2]),
                      static_cast<float>(R) + kCoarseEps};
    };
    // a link of 4 or more spheres splits, along the order above, where the two
    // halves' radii sum to the least (2 spheres at least on each side)
    for (int l = 0; l < L; ++l) {
        LinkC &K = rp.links[l];
        if (K.s1 - K.s0 < 4) continue;
        double best = HUGE_VAL, c[3];
        for (int k = K.s0 + 2; k <= K.s1 - 2; ++k) {
            const double sum = bound_spheres(K.s0, k, c, 32) + bound_spheres(k, K.s1, c, 32);
            if (sum < best) best = sum, K.sm = static_cast<int16_t>(k);
        }
    }
    for (int l = 0; l < L; ++l) {
        LinkC &K = rp.links[l];
        if (K.sm < K.s1) {
            rp.halves[l][0] = half_sphere(K.s0, K.sm);
            rp.halves[l][1] = half_sphere(K.sm, K.s1);
        }
    }

    // link bounding spheres (Sec. III-D mid-phase): a given sphere is checked
    // to contain its link's spheres; the derived bound replaces it where that
    // is tighter (the hierarchy only culls, so any enclosing sphere gives the
    // same verdicts)
    for (int l = 0; l < L; ++l) {
        LinkC &K = rp.links[l];
        if (K.s0 == K.s1) continue;
        double c[3];
        double R = bound_spheres(K.s0, K.s1, c);
        if (r->link_spheres) {
            const double *g = r->link_spheres + 4 * l;
            if (!finite_all(g, 4)) return fail(ctx, VP_ERR_ARG, "link sphere %d is not finite", l);
            double need = 0;
            for (int i = K.s0; i < K.s1; ++i) {
                const double *p = r->sphere_centre + 3 * order[i];
                const double d[3] = {p[0] - g[0], p[1] - g[1], p[2] - g[2]};
                need = std::max(need, norm3(d) + r->sphere_radius[order[i]]);
            }
            if (need > g[3] + 1e-9)
                return fail(ctx, VP_ERR_ARG, "link sphere %d does not contain its spheres (needs %.6g > %.6g)", l, need,
                            g[3]);
            if (g[3] <= R) {
                for (int d = 0; d < 3; ++d) c[d] = g[d];
                R = g[3];
            }
        }
        K.bs = float4{static_cast<float>(c[0]), static_cast<float>(c[1]), static_cast<float>(c[2]),
                      static_cast<float>(R) + kCoarseEps};
    }

    // self pairs grouped by (earlier link, later link), later link major
    struct PairRec {
        int la, lb, a, b;
    };
    std::vector<PairRec> prs(P);
    for (int p = 0; p < P; ++p) {
        int a = r->self_pairs[2 * p], b = r->self_pairs[2 * p + 1];
        if (a < 0 || a >= S || b < 0 || b >= S || a == b)
            return fail(ctx, VP_ERR_ARG, "self pair %d: bad sphere indices (%d, %d)", p, a, b);
        int la = r->sphere_link[a], lb = r->sphere_link[b];
        if (la > lb) {
            std::swap(a, b);
            std::swap(la, lb);
        }
        prs[p] = PairRec{la, lb, sorted_of[a], sorted_of[b]};
    }
    std::stable_sort(prs.begin(), prs.end(),
                     [](const PairRec &x, const PairRec &y) { return x.lb != y.lb ? x.lb < y.lb : x.la < y.la; });
    // link-pair groups (the later link lb is where the pair is checked) and
    // frame-stash slots for branch points (a joint whose parent is not the
    // previous joint)
    std::vector<int> slot_of(L, -1);
    int n_slots = 0;
    int ng = 0;
    for (int i = 0; i < P;) {
        int j = i;
        while (j < P && prs[j].la == prs[i].la && prs[j].lb == prs[i].lb) ++j;
        if (ng >= kMaxGroups) return fail(ctx, VP_ERR_CAPACITY, "too many link pairs with self pairs");
        GroupC &G = rp.groups[ng++];
        G.la = static_cast<int16_t>(prs[i].la);
        G.lb = static_cast<int16_t>(prs[i].lb);
        G.p0 = static_cast<int16_t>(i);
        G.p1 = static_cast<int16_t>(j);
        i = j;
    }
    for (int p = 0; p < P; ++p) rp.pairs[p] = PairC{static_cast<uint16_t>(prs[p].a), static_cast<uint16_t>(prs[p].b)};
    for (int j = 0; j < D; ++j) {
        const int pl = parent_link[j];
        if (pl != j && pl != 0 && slot_of[pl] < 0) slot_of[pl] = n_slots++;
    }
    // joint path from the base to each link
    std::vector<uint32_t> path(L, 0);
    for (int j = 0; j < D; ++j) path[j + 1] = path[parent_link[j]] | (1u << j);
    for (int l = 0; l < L; ++l) {
        rp.links[l].slot = static_cast<int16_t>(slot_of[l]);
        rp.links[l].path = static_cast<uint16_t>(path[l]);
    }
    for (int g = 0; g < ng;) {
        const int lb = rp.groups[g].lb;
        int h = g;
        while (h < ng && rp.groups[h].lb == lb) ++h;
        rp.links[lb].g0 = static_cast<int16_t>(g);
        rp.links[lb].g1 = static_cast<int16_t>(h);
        g = h;
    }
    for (int j = 0; j < D; ++j) {
        const int pl = parent_link[j];
        const int src = (pl == j) ? kParentPrev : (pl == 0 ? kParentBase : slot_of[pl]);
        rp.joints[j].meta |= (src & 0xFF) << kMetaParentShift;
        rp.joints[j].meta |= (pl & 0xFF) << kMetaParentLinkShift;
    }
    rp.n_groups = ng;
    for (int g = 0; g < kMaxGroups; ++g) rp.gorder[g] = static_cast<uint8_t>(g < ng ? g : 0);
    rp.n_gfront = ng;
    rp.n_slots = n_slots;
    rp.link_mask = 0;
    for (int l = 0; l < L; ++l)
        if (rp.links[l].s0 < rp.links[l].s1) rp.link_mask |= 1u << l;
    rp.simple = 1;
    for (int j = 0; j < D; ++j) {
        const int m = rp.joints[j].meta;
        if (!(m & kMetaOriginRotIdentity) || ((m >> kMetaAxisShift) & 3) == kAxisGeneral) rp.simple = 0;
    }

    ctx->robot = rp;
    ctx->sorted_of = sorted_of;
    ctx->robot_loaded = true;
    batched_invalidate(ctx->batched);
    if (ctx->fk_gen.kernel) {  // a generated FK belongs to the previous robot
        DeviceGuard g(ctx->device);
        fk_codegen_release(&ctx->fk_gen);
    }
    ctx->fk_mode = -1;
    ctx->fk_gen_failed = false;
    return VP_OK;
}

// ---------------------------------------------------------------------------
// environment

// FNV-1a over the packed environment's bytes (the tuning cache's key).
static uint64_t packed_hash(const std::vector<float4> &h) {
    uint64_t hsh = 1469598103934665603ull;
    const unsigned char *b = reinterpret_cast<const unsigned char *>(h.data());
    for (size_t i = 0; i < h.size() * 16; ++i) hsh = (hsh ^ b[i]) * 1099511628211ull;
    return hsh;
}

extern "C" vp_status vp_load_env(vp_ctx *ctx, const vp_env_desc *e) {
    if (!ctx) return VP_ERR_ARG;
    if (!e) return fail(ctx, VP_ERR_ARG, "environment descriptor is NULL");
    size_t n4 = 0;
    std::string msg;
    int rc = env_packed_float4(e, &n4, &msg);
    if (rc) return fail(ctx, rc == 2 ? VP_ERR_CAPACITY : VP_ERR_ARG, "%s", msg.c_str());
    std::vector<float4> h(n4);
    EnvView view{};
    rc = pack_env(e, h.data(), VP_MAX_ENV_BYTES / 16, &view, &msg);
    if (rc) return fail(ctx, rc == 2 ? VP_ERR_CAPACITY : VP_ERR_ARG, "%s", msg.c_str());
    DeviceGuard g(ctx->device);
    float4 *buf = nullptr;
    if (n4 > 0) {
        cudaError_t err = cudaMalloc(&buf, n4 * 16);
        if (err == cudaSuccess) err = cudaMemcpy(buf, h.data(), n4 * 16, cudaMemcpyHostToDevice);
        if (err != cudaSuccess) {
            if (buf) cudaFree(buf);
            return cuda_fail(ctx, err, "vp_load_env");
        }
    }
    if (ctx->env_buf) {
        cudaDeviceSynchronize();  // the old buffer may still be read by queued work
        cudaFree(ctx->env_buf);
    }
    ctx->env_buf = buf;
    view.data = buf;
    ctx->env = view;
    ctx->env_hash = packed_hash(h);
    ctx->env_host = std::move(h);
    ctx->env_loaded = true;
    batched_invalidate(ctx->batched);
    return VP_OK;
}

// ---------------------------------------------------------------------------
// compute calls

namespace {

// Launch shape of a plain-path validation kernel: the largest block (128,
// 64 or 32 threads) whose shared memory fits the opt-in limit, and where the
// environment lives -- in each block's shared memory, unless copying it
// there lowers the blocks per SM (then the kernel reads it in place, through
// L1; its loads are warp-uniform).  prep(smem, block, &bps) sets the
// kernel's shared-memory limit and reports its occupancy; it is called for
// the in-place size first and the staged size last, so the limit ends at the
// larger (prep also names the placement, for kernels with an instance per
// placement).  Returns false if no block fits.
template <class Prep>
bool plan_launch(vp_ctx *ctx, Prep prep, EnvView *view, int *block, size_t *smem, int *bps, cudaError_t *err) {
    *err = cudaSuccess;
    for (int b : {128, 64, 32}) {
        EnvView v0 = ctx->env, v1 = ctx->env;
        v0.staged = 0;
        v1.staged = 1;
        const size_t s0 = smem_bytes(v0, ctx->robot.n_links, b), s1 = smem_bytes(v1, ctx->robot.n_links, b);
        if (s0 > ctx->smem_optin) continue;
        int b0 = 0, b1 = 0;
        *err = prep(s0, b, false, &b0);
        if (*err == cudaSuccess && s1 <= ctx->smem_optin) *err = prep(s1, b, true, &b1);
        if (*err != cudaSuccess) return true;
        const bool staged = b1 >= 1 && b1 >= b0;
        *view = staged ? v1 : v0;
        *block = b;
        *smem = staged ? s1 : s0;
        *bps = staged ? b1 : b0;
        return true;
    }
    return false;
}

}  // namespace

extern "C" vp_status vp_fk_spheres(vp_ctx *ctx, const float *q, int64_t n, float *centres, void *stream) {
    if (!ctx) return VP_ERR_ARG;
    if (!ctx->robot_loaded) return fail(ctx, VP_ERR_NOT_LOADED, "robot not loaded");
    if (n < 0) return fail(ctx, VP_ERR_ARG, "n < 0");
    if (n == 0) return VP_OK;
    if (!q || !centres) return fail(ctx, VP_ERR_ARG, "NULL buffer");
    DeviceGuard g(ctx->device);
    if (ctx->fk_mode == -1 && !ctx->fk_gen.kernel && !ctx->fk_gen_failed) {
        // automatic: generate and compile the robot's FK on first use; if
        // that fails (no NVRTC), the table-driven kernel serves from now on
        std::string msg;
        ctx->fk_gen_failed = fk_codegen_build(ctx->robot, &ctx->fk_gen, &msg) != 0;
    }
    if (ctx->fk_mode == 1 || (ctx->fk_mode == -1 && ctx->fk_gen.kernel)) {
        const cudaError_t e =
            fk_codegen_launch(ctx->fk_gen, ctx->robot.n_spheres, q, n, centres, static_cast<cudaStream_t>(stream));
        return e == cudaSuccess ? VP_OK : cuda_fail(ctx, e, "vp_fk_spheres (generated)");
    }
    const int block = fk_configs_per_block(ctx->robot.n_spheres);
    const size_t smem = (static_cast<size_t>(ctx->robot.n_slots) * kFrameFloats + 3 * ctx->robot.n_spheres) * block *
                        sizeof(float);
    int bps = 0;
    cudaError_t e = prepare_fk(smem, block, &bps);
    if (e == cudaSuccess) {
        const int64_t grid = (n + block - 1) / block;
        e = launch_fk(ctx->robot, q, n, centres, static_cast<int>(grid), block, smem,
                      static_cast<cudaStream_t>(stream));
    }
    return e == cudaSuccess ? VP_OK : cuda_fail(ctx, e, "vp_fk_spheres");
}

extern "C" vp_status vp_validate_states(vp_ctx *ctx, const float *q, int64_t n, uint8_t *valid, void *stream) {
    vp_status s = check_loaded(ctx);
    if (s != VP_OK) return s;
    if (n < 0) return fail(ctx, VP_ERR_ARG, "n < 0");
    if (n == 0) return VP_OK;
    if (!q || !valid) return fail(ctx, VP_ERR_ARG, "NULL buffer");
    DeviceGuard g(ctx->device);
    int block = 0, bps = 0;
    size_t smem = 0;
    EnvView view;
    cudaError_t e = cudaSuccess;
    const int lmax = lmax_for(ctx->robot.n_links);
    if (!plan_launch(
            ctx, [lmax](size_t sm, int b, bool, int *o) { return prepare_states(lmax, sm, b, o); }, &view, &block, &smem,
            &bps, &e))
        return fail(ctx, VP_ERR_CAPACITY, "frame stash exceeds shared memory");
    view.order = batched_check_order(ctx->batched);
    if (e == cudaSuccess) {
        const int64_t need = (n + block - 1) / block;
        const int64_t grid =
            std::max<int64_t>(1, std::min<int64_t>(need, static_cast<int64_t>(std::max(bps, 1)) * ctx->num_sms));
        e = launch_states(ctx->robot, view, q, n, valid, ctx->status, static_cast<int>(grid), block, smem,
                          static_cast<cudaStream_t>(stream));
    }
    return e == cudaSuccess ? VP_OK : cuda_fail(ctx, e, "vp_validate_states");
}

extern "C" vp_status vp_edge_counts(vp_ctx *ctx, const float *q0, const float *q1, float resolution,
                                    int64_t n_edges, int32_t *counts, void *stream) {
    if (!ctx) return VP_ERR_ARG;
    if (!ctx->robot_loaded) return fail(ctx, VP_ERR_NOT_LOADED, "robot not loaded");
    if (n_edges < 0) return fail(ctx, VP_ERR_ARG, "n_edges < 0");
    if (!(resolution > 0.f) || !std::isfinite(resolution)) return fail(ctx, VP_ERR_ARG, "resolution must be > 0");
    if (n_edges == 0) return VP_OK;
    if (!q0 || !q1 || !counts) return fail(ctx, VP_ERR_ARG, "NULL buffer");
    DeviceGuard g(ctx->device);
    cudaError_t e = launch_counts(ctx->robot.n_joints, q0, q1, resolution, n_edges, counts,
                                  static_cast<cudaStream_t>(stream));
    return e == cudaSuccess ? VP_OK : cuda_fail(ctx, e, "vp_edge_counts");
}

static vp_status validate_edges_impl(vp_ctx *ctx, const float *q0, const float *q1, const int32_t *counts,
                                     float resolution, int64_t n_edges, uint8_t *valid, int mode,
                                     uint64_t *work, void *stream, BatchedState *slot = nullptr) {
    vp_status s = check_loaded(ctx);
    if (s != VP_OK) return s;
    if (n_edges < 0) return fail(ctx, VP_ERR_ARG, "n_edges < 0");
    if (!counts && (!(resolution > 0.f) || !std::isfinite(resolution)))
        return fail(ctx, VP_ERR_ARG, "resolution must be > 0 when counts is NULL");
    if (mode != VP_MODE_PLAIN && mode != VP_MODE_BATCHED && mode != VP_MODE_PER_EDGE)
        return fail(ctx, VP_ERR_ARG, "unknown mode %d", mode);
    if (n_edges == 0) return VP_OK;
    if (!q0 || !q1 || !valid) return fail(ctx, VP_ERR_ARG, "NULL buffer");
    DeviceGuard g(ctx->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const bool timed = ctx->timing && !work && mode != VP_MODE_PER_EDGE;
    if (timed) ctx->timed = true;
    if (mode == VP_MODE_BATCHED) {
        BatchedArgs a{&ctx->robot, &ctx->env, q0, q1, counts, resolution, n_edges, valid, ctx->status,
                      ctx->num_sms, ctx->smem_optin, st};
        a.env_hash = ctx->env_hash;
        if (timed) {
            a.ev_start = ctx->ev_start;
            a.ev_stop = ctx->ev_stop;
        }
        std::string msg;
        BatchedState &bs = slot ? *slot : ctx->batched;
        const int rc = work ? batched_work(bs, a, reinterpret_cast<unsigned long long *>(work), &msg)
                            : batched_validate(bs, a, &msg);
        if (rc == 0) return VP_OK;
        return fail(ctx, rc == 1 ? VP_ERR_CAPACITY : VP_ERR_CUDA, "batched: %s", msg.c_str());
    }
    int block = 0, bps = 0;
    size_t smem = 0;
    EnvView view;
    cudaError_t e = cudaSuccess;
    const bool stats = work != nullptr, simple = ctx->robot.simple != 0;
    const int lmax = lmax_for(ctx->robot.n_links);
    const int order = batched_check_order(ctx->batched);
    if (!plan_launch(
            ctx,
            [stats, lmax, simple, order](size_t sm, int b, bool staged, int *o) {
                return prepare_edges_plain(stats, lmax, simple, staged, sm, b, o, order);
            },
            &view, &block, &smem, &bps, &e))
        return fail(ctx, VP_ERR_CAPACITY, "frame stash exceeds shared memory");
    if (e != cudaSuccess) return cuda_fail(ctx, e, "vp_validate_edges (prepare)");
    if (bps < 1) return fail(ctx, VP_ERR_CAPACITY, "plain edge kernel cannot be resident");
    view.order = batched_check_order(ctx->batched);
    const int wpb = block / 32;
    if (mode == VP_MODE_PER_EDGE && !work) {
        const int D = ctx->robot.n_joints;
        const size_t smem32 = smem_bytes(view, ctx->robot.n_links, 32);
        for (int64_t i = 0; i < n_edges && e == cudaSuccess; ++i)
            e = launch_edges_plain(ctx->robot, view, q0 + i * D, q1 + i * D, counts ? counts + i : nullptr,
                                   resolution, 1, valid + i, ctx->status, nullptr, 1, 32, smem32, st);
        return e == cudaSuccess ? VP_OK : cuda_fail(ctx, e, "vp_validate_edges (per edge)");
    }
    const int64_t need = (n_edges + wpb - 1) / wpb;
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(need, static_cast<int64_t>(bps) * ctx->num_sms));
    if (timed) e = cudaEventRecord(ctx->ev_start, st);
    if (e == cudaSuccess)
        e = launch_edges_plain(ctx->robot, view, q0, q1, counts, resolution, n_edges, valid, ctx->status,
                               reinterpret_cast<unsigned long long *>(work), static_cast<int>(grid), block, smem, st);
    if (e == cudaSuccess && timed) e = cudaEventRecord(ctx->ev_stop, st);
    return e == cudaSuccess ? VP_OK : cuda_fail(ctx, e, "vp_validate_edges");
}

extern "C" vp_status vp_validate_edges(vp_ctx *ctx, const float *q0, const float *q1, const int32_t *counts,
                                       float resolution, int64_t n_edges, uint8_t *valid, int mode, void *stream) {
    return validate_edges_impl(ctx, q0, q1, counts, resolution, n_edges, valid, mode, nullptr, stream);
}

extern "C" vp_status vp_validate_edges_host(vp_ctx *ctx, const float *q0, const float *q1, const int32_t *counts,
                                            float resolution, int64_t n_edges, uint8_t *valid, int mode,
                                            void *stream) {
    vp_status s = check_loaded(ctx);
    if (s != VP_OK) return s;
    if (n_edges < 0) return fail(ctx, VP_ERR_ARG, "n_edges < 0");
    if (!counts && (!(resolution > 0.f) || !std::isfinite(resolution)))
        return fail(ctx, VP_ERR_ARG, "resolution must be > 0 when counts is NULL");
    if (mode != VP_MODE_PLAIN && mode != VP_MODE_BATCHED)
        return fail(ctx, VP_ERR_ARG, "vp_validate_edges_host: mode must be VP_MODE_PLAIN or VP_MODE_BATCHED");
    if (n_edges == 0) return VP_OK;
    if (!q0 || !q1 || !valid) return fail(ctx, VP_ERR_ARG, "NULL buffer");
    DeviceGuard g(ctx->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int D = ctx->robot.n_joints;
    const size_t nq = static_cast<size_t>(n_edges) * D, ne = static_cast<size_t>(n_edges);
    cudaError_t e = cudaSuccess;
    if (nq > ctx->hx_cap_q || ne > ctx->hx_cap_e) {  // grow the device copies (waits for queued work)
        e = cudaDeviceSynchronize();
        cudaFree(ctx->hx_q0);
        cudaFree(ctx->hx_q1);
        cudaFree(ctx->hx_counts);
        cudaFree(ctx->hx_valid);
        ctx->hx_q0 = ctx->hx_q1 = nullptr;
        ctx->hx_counts = nullptr;
        ctx->hx_valid = nullptr;
        ctx->hx_cap_q = ctx->hx_cap_e = 0;
        if (e == cudaSuccess) e = cudaMalloc(&ctx->hx_q0, nq * sizeof(float));
        if (e == cudaSuccess) e = cudaMalloc(&ctx->hx_q1, nq * sizeof(float));
        if (e == cudaSuccess) e = cudaMalloc(&ctx->hx_counts, ne * sizeof(int32_t));
        if (e == cudaSuccess) e = cudaMalloc(&ctx->hx_valid, ne);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "vp_validate_edges_host (device copies)");
        ctx->hx_cap_q = nq;
        ctx->hx_cap_e = ne;
    }
    if (!ctx->hx_in) e = cudaStreamCreateWithFlags(&ctx->hx_in, cudaStreamNonBlocking);
    if (e == cudaSuccess && !ctx->hx_out) e = cudaStreamCreateWithFlags(&ctx->hx_out, cudaStreamNonBlocking);
    for (cudaStream_t &cs : ctx->hx_cs)
        if (e == cudaSuccess && !cs) e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    for (cudaEvent_t &ev : ctx->hx_ev)
        if (e == cudaSuccess && !ev) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "vp_validate_edges_host (streams)");
    // chunks: the copies of chunk i+1 overlap the validation of chunk i, and
    // each chunk's verdicts go back as soon as they are known.  The plain
    // kernel takes chunks of about 2^19 edges (at most 8).  A batched chunk
    // runs on one of two compute streams with its own scratch, so its
    // persistent launch starts on the SMs the previous chunk's tail frees; a
    // large batch goes in doubling chunks (1/16, 1/16, 1/8, 1/4, 1/2), the
    // first copied in a sixteenth of the time of the whole.
    int64_t bounds[9] = {0};
    int n_chunks = 1;
    if (mode == VP_MODE_BATCHED) {
        if (n_edges >= (int64_t{1} << 20)) {
            const int64_t parts[5] = {1, 2, 4, 8, 16};  // bounds in sixteenths
            for (int c = 0; c < 5; ++c) bounds[c + 1] = n_edges * parts[c] / 16;
            n_chunks = 5;
        }
    } else {
        n_chunks = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(8, (n_edges + (1 << 19) - 1) >> 19)));
        for (int c = 1; c < n_chunks; ++c) bounds[c] = n_edges * c / n_chunks;
    }
    bounds[n_chunks] = n_edges;
    cudaEvent_t *ev_in = ctx->hx_ev, *ev_out = ctx->hx_ev + 8, ev_start = ctx->hx_ev[16], ev_done = ctx->hx_ev[17];
    // the copies wait for earlier work on the caller's stream (which may
    // still read the device copies)
    e = cudaEventRecord(ev_start, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->hx_in, ev_start, 0);
    const bool timing = ctx->timing;
    ctx->timing = false;  // the kernel-time hook times single-launch calls
    vp_status rs = VP_OK;
    for (int c = 0; c < n_chunks && e == cudaSuccess && rs == VP_OK; ++c) {
        const int64_t off = bounds[c], n = bounds[c + 1] - bounds[c];
        if (n <= 0) continue;
        const size_t qo = static_cast<size_t>(off) * D, qn = static_cast<size_t>(n) * D * sizeof(float);
        e = cudaMemcpyAsync(ctx->hx_q0 + qo, q0 + qo, qn, cudaMemcpyHostToDevice, ctx->hx_in);
        if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->hx_q1 + qo, q1 + qo, qn, cudaMemcpyHostToDevice, ctx->hx_in);
        if (e == cudaSuccess && counts)
            e = cudaMemcpyAsync(ctx->hx_counts + off, counts + off, n * sizeof(int32_t), cudaMemcpyHostToDevice,
                                ctx->hx_in);
        const bool batched = mode == VP_MODE_BATCHED;
        cudaStream_t cs = batched ? ctx->hx_cs[c & 1] : st;
        if (e == cudaSuccess) e = cudaEventRecord(ev_in[c], ctx->hx_in);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ev_in[c], 0);
        if (e != cudaSuccess) break;
        BatchedState *slot = nullptr;
        if (batched) {
            slot = &ctx->hx_slot[c & 1];
            batched_mirror(*slot, ctx->batched);
        }
        rs = validate_edges_impl(ctx, ctx->hx_q0 + qo, ctx->hx_q1 + qo, counts ? ctx->hx_counts + off : nullptr,
                                 resolution, n, ctx->hx_valid + off, mode, nullptr, cs, slot);
        if (rs != VP_OK) break;
        e = cudaEventRecord(ev_out[c], cs);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->hx_out, ev_out[c], 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(valid + off, ctx->hx_valid + off, n, cudaMemcpyDeviceToHost, ctx->hx_out);
    }
    ctx->timing = timing;
    if (rs != VP_OK) return rs;
    // the caller's stream completes only once every verdict is on the host
    if (e == cudaSuccess) e = cudaEventRecord(ev_done, ctx->hx_out);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ev_done, 0);
    return e == cudaSuccess ? VP_OK : cuda_fail(ctx, e, "vp_validate_edges_host");
}

extern "C" vp_status vp_validate_edges_work(vp_ctx *ctx, const float *q0, const float *q1, const int32_t *counts,
                                            float resolution, int64_t n_edges, uint8_t *valid, int mode,
                                            uint64_t *work, void *stream) {
    if (ctx && !work) return fail(ctx, VP_ERR_ARG, "work is NULL");
    if (ctx && mode == VP_MODE_PER_EDGE) return fail(ctx, VP_ERR_ARG, "no work counters for VP_MODE_PER_EDGE");
    return validate_edges_impl(ctx, q0, q1, counts, resolution, n_edges, valid, mode, work, stream);
}

extern "C" vp_status vp_collision_cost(vp_ctx *ctx, const float *q, int64_t n, float margin, float *cost,
                                       float *grad, void *stream) {
    vp_status s = check_loaded(ctx);
    if (s != VP_OK) return s;
    if (n < 0) return fail(ctx, VP_ERR_ARG, "n < 0");
    if (!std::isfinite(margin)) return fail(ctx, VP_ERR_ARG, "margin must be finite");
    if (n == 0) return VP_OK;
    if (!q || !cost) return fail(ctx, VP_ERR_ARG, "NULL buffer");
    DeviceGuard g(ctx->device);
    std::string msg;
    const int rc = cost_launch(ctx->robot, ctx->env, q, n, margin, cost, grad, ctx->status, ctx->num_sms,
                               ctx->smem_optin, static_cast<cudaStream_t>(stream), &msg);
    if (rc == 0) return VP_OK;
    return fail(ctx, rc == 1 ? VP_ERR_CAPACITY : VP_ERR_CUDA, "vp_collision_cost: %s", msg.c_str());
}

extern "C" vp_status vp_autotune(vp_ctx *ctx, const float *q0, const float *q1, const int32_t *counts,
                                 float resolution, int64_t n_edges, void *stream) {
    vp_status s = check_loaded(ctx);
    if (s != VP_OK) return s;
    if (n_edges <= 0) return fail(ctx, VP_ERR_ARG, "n_edges must be > 0");
    if (!q0 || !q1) return fail(ctx, VP_ERR_ARG, "NULL buffer");
    if (!counts && (!(resolution > 0.f) || !std::isfinite(resolution)))
        return fail(ctx, VP_ERR_ARG, "resolution must be > 0 when counts is NULL");
    DeviceGuard g(ctx->device);
    std::string msg;
    // the frequent-first order of the self-pair groups, counted on the
    // batch's first start configurations (a sample of its states)
    const int64_t n_sample = std::min<int64_t>(n_edges, 65536);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (ctx->robot.n_groups > 0 &&
        group_order(ctx->robot, q0, n_sample, st, ctx->robot.gorder, &ctx->robot.n_gfront, &msg) != 0)
        return fail(ctx, VP_ERR_CUDA, "vp_autotune: %s", msg.c_str());
    // the environment's visiting order: each kind's primitives most often
    // touched first, the kinds by their total (counted on the same sample)
    if (!ctx->env_host.empty()) {
        std::vector<unsigned> hits;
        if (prim_hits(ctx->robot, ctx->env, q0, n_sample, st, &hits, &msg) != 0)
            return fail(ctx, VP_ERR_CUDA, "vp_autotune: %s", msg.c_str());
        std::vector<float4> re;
        EnvView view = ctx->env;
        reorder_env(ctx->env_host, hits, &view, &re);
        if (re.size() != ctx->env_host.size() ||
            std::memcmp(re.data(), ctx->env_host.data(), re.size() * sizeof(float4)) != 0 ||
            view.kind_order != ctx->env.kind_order) {
            cudaError_t e = cudaDeviceSynchronize();  // queued work may still read the buffer
            if (e == cudaSuccess) e = cudaMemcpy(ctx->env_buf, re.data(), re.size() * 16, cudaMemcpyHostToDevice);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "vp_autotune (environment order)");
            ctx->env = view;
            ctx->env_hash = packed_hash(re);
            ctx->env_host = std::move(re);
        }
    }
    BatchedArgs a{&ctx->robot, &ctx->env, q0, q1, counts, resolution, n_edges, nullptr, ctx->status,
                  ctx->num_sms, ctx->smem_optin, st};
    a.env_hash = ctx->env_hash;
    const int rc = batched_autotune(ctx->batched, a, &msg);
    if (rc == 0) return VP_OK;
    return fail(ctx, rc == 1 ? VP_ERR_CAPACITY : VP_ERR_CUDA, "vp_autotune: %s", msg.c_str());
}

extern "C" vp_status vp_kernel_time(vp_ctx *ctx, int enable, float *last_ms) {
    if (!ctx) return VP_ERR_ARG;
    DeviceGuard g(ctx->device);
    if (enable && !ctx->ev_start) {
        cudaError_t e = cudaEventCreate(&ctx->ev_start);
        if (e == cudaSuccess) e = cudaEventCreate(&ctx->ev_stop);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "vp_kernel_time");
    }
    if (last_ms) {
        *last_ms = -1.f;
        if (ctx->timed && ctx->ev_stop) {
            cudaError_t e = cudaEventSynchronize(ctx->ev_stop);
            if (e == cudaSuccess) e = cudaEventElapsedTime(last_ms, ctx->ev_start, ctx->ev_stop);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "vp_kernel_time");
        }
    }
    ctx->timing = enable != 0;
    return VP_OK;
}

extern "C" vp_status vp_set_watchdog(vp_ctx *ctx, double seconds) {
    if (!ctx) return VP_ERR_ARG;
    if (!(seconds >= 0.0) || !std::isfinite(seconds) || seconds > 1e9)
        return fail(ctx, VP_ERR_ARG, "watchdog must be a finite number of seconds >= 0");
    ctx->batched.watchdog_ns = static_cast<unsigned long long>(seconds * 1e9);
    return VP_OK;
}

extern "C" vp_status vp_tiling(vp_ctx *ctx, int32_t *lanes, int n, int *n_buckets) {
    if (!ctx) return VP_ERR_ARG;
    if (n < 0 || (n > 0 && !lanes)) return fail(ctx, VP_ERR_ARG, "vp_tiling: bad output array");
    int G[16];
    const int nb = batched_tiling(ctx->batched, G, 16);
    for (int b = 0; b < n && b < nb; ++b) lanes[b] = G[b];
    if (n_buckets) *n_buckets = nb;
    return VP_OK;
}

extern "C" vp_status vp_set_tiling(vp_ctx *ctx, const int32_t *lanes, int n) {
    if (!ctx) return VP_ERR_ARG;
    if (n < 0 || n > 9 || (n > 0 && !lanes)) return fail(ctx, VP_ERR_ARG, "vp_set_tiling: n must be in [0, 9]");
    int G[9];
    for (int b = 0; b < n; ++b) {
        if (lanes[b] != 4 && lanes[b] != 8 && lanes[b] != 16 && lanes[b] != 32)
            return fail(ctx, VP_ERR_ARG, "vp_set_tiling: lanes per edge must be 4, 8, 16 or 32");
        G[b] = lanes[b];
    }
    batched_set_tiling(ctx->batched, G, n);
    return VP_OK;
}

extern "C" vp_status vp_set_screen_rounds(vp_ctx *ctx, int rounds) {
    if (!ctx) return VP_ERR_ARG;
    if (rounds < 0) return fail(ctx, VP_ERR_ARG, "vp_set_screen_rounds: rounds must be >= 0");
    batched_set_screen_rounds(ctx->batched, rounds);
    return VP_OK;
}

extern "C" vp_status vp_screen_rounds(vp_ctx *ctx, int *rounds) {
    if (!ctx || !rounds) return VP_ERR_ARG;
    *rounds = batched_screen_rounds(ctx->batched);
    return VP_OK;
}

vp_status vp_link_bounds(vp_ctx *ctx, int n_links, float *link_sphere, float *half_sphere, int32_t *sphere_half) {
    if (!ctx) return VP_ERR_ARG;
    if (!ctx->robot_loaded) return fail(ctx, VP_ERR_NOT_LOADED, "no robot loaded");
    const RobotParams &rp = ctx->robot;
    if (n_links != rp.n_links) return fail(ctx, VP_ERR_ARG, "n_links %d: the robot has %d links", n_links, rp.n_links);
    for (int l = 0; l < rp.n_links; ++l) {
        const LinkC &K = rp.links[l];
        const bool any = K.s0 < K.s1, split = K.sm < K.s1;
        if (link_sphere) {
            const float4 b = any ? K.bs : float4{0.f, 0.f, 0.f, -1.f};
            link_sphere[4 * l + 0] = b.x;
            link_sphere[4 * l + 1] = b.y;
            link_sphere[4 * l + 2] = b.z;
            link_sphere[4 * l + 3] = b.w;
        }
        if (half_sphere) {
            for (int h = 0; h < 2; ++h) {
                const float4 b = split ? rp.halves[l][h] : float4{0.f, 0.f, 0.f, -1.f};
                float *o = half_sphere + 8 * l + 4 * h;
                o[0] = b.x;
                o[1] = b.y;
                o[2] = b.z;
                o[3] = b.w;
            }
        }
        if (sphere_half)
            for (int i = K.s0; i < K.s1; ++i) sphere_half[rp.perm[i]] = split ? (i < K.sm ? 0 : 1) : -1;
    }
    return VP_OK;
}

extern "C" vp_status vp_set_check_order(vp_ctx *ctx, int order) {
    if (!ctx) return VP_ERR_ARG;
    if (order < 0 || order >= kOrderCount) return fail(ctx, VP_ERR_ARG, "vp_set_check_order: 0 to 5");
    batched_set_check_order(ctx->batched, order);
    return VP_OK;
}

extern "C" vp_status vp_check_order(vp_ctx *ctx, int *order) {
    if (!ctx || !order) return VP_ERR_ARG;
    *order = batched_check_order(ctx->batched);
    return VP_OK;
}

extern "C" vp_status vp_shortcut_paths(vp_ctx *ctx, float *paths, int32_t *lengths, int64_t P, int32_t W,
                                        const float *draws, int32_t T, float resolution, void *stream) {
    vp_status s = check_loaded(ctx);
    if (s != VP_OK) return s;
    if (P < 0 || W < 2 || T < 0) return fail(ctx, VP_ERR_ARG, "vp_shortcut_paths: need P >= 0, W >= 2, T >= 0");
    if (!(resolution > 0.f) || !std::isfinite(resolution))
        return fail(ctx, VP_ERR_ARG, "vp_shortcut_paths: resolution must be > 0");
    if (P == 0 || T == 0) return VP_OK;
    if (!paths || !lengths || !draws) return fail(ctx, VP_ERR_ARG, "vp_shortcut_paths: NULL buffer");
    DeviceGuard g(ctx->device);
    const int D = ctx->robot.n_joints;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSuccess;
    if (P > ctx->sc_cap || D != ctx->sc_dof) {  // grow the scratch (outside any capture)
        cudaStreamSynchronize(st);
        cudaFree(ctx->sc_q0);
        cudaFree(ctx->sc_q1);
        cudaFree(ctx->sc_ij);
        cudaFree(ctx->sc_ok);
        ctx->sc_q0 = ctx->sc_q1 = nullptr;
        ctx->sc_ij = nullptr;
        ctx->sc_ok = nullptr;
        ctx->sc_cap = 0;
        e = cudaMalloc(&ctx->sc_q0, P * D * sizeof(float));
        if (e == cudaSuccess) e = cudaMalloc(&ctx->sc_q1, P * D * sizeof(float));
        if (e == cudaSuccess) e = cudaMalloc(&ctx->sc_ij, P * sizeof(int2));
        if (e == cudaSuccess) e = cudaMalloc(&ctx->sc_ok, P);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "vp_shortcut_paths (scratch)");
        ctx->sc_cap = P;
        ctx->sc_dof = D;
    }
    for (int32_t t = 0; t < T; ++t) {
        e = shortcut_propose(paths, lengths, P, W, D, draws + static_cast<int64_t>(t) * P * 2, ctx->sc_q0,
                             ctx->sc_q1, ctx->sc_ij, st);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "vp_shortcut_paths (propose)");
        s = validate_edges_impl(ctx, ctx->sc_q0, ctx->sc_q1, nullptr, resolution, P, ctx->sc_ok, VP_MODE_BATCHED,
                                nullptr, stream);
        if (s != VP_OK) return s;
        e = shortcut_apply(paths, lengths, P, W, D, ctx->sc_ij, ctx->sc_ok, st);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "vp_shortcut_paths (apply)");
    }
    return VP_OK;
}

extern "C" vp_status vp_rrt_connect(vp_ctx *ctx, const float *start, const float *goal, int64_t B,
                                     const float *samples, int32_t T, float range, float resolution, int32_t cap,
                                     int32_t *status, int32_t *iters, float *path, int32_t *path_len,
                                     int32_t *tree_sizes, void *stream) {
    vp_status s = check_loaded(ctx);
    if (s != VP_OK) return s;
    if (B < 0 || T < 0 || cap < 2) return fail(ctx, VP_ERR_ARG, "vp_rrt_connect: need B >= 0, T >= 0, cap >= 2");
    if (!(range > 0.f) || !std::isfinite(range) || !(resolution > 0.f) || !std::isfinite(resolution))
        return fail(ctx, VP_ERR_ARG, "vp_rrt_connect: range and resolution must be > 0");
    if (B == 0) return VP_OK;
    if (!start || !goal || (T > 0 && !samples) || !status || !iters || !path || !path_len || !tree_sizes)
        return fail(ctx, VP_ERR_ARG, "vp_rrt_connect: NULL buffer");
    if (B > 0x7fffffff) return fail(ctx, VP_ERR_CAPACITY, "vp_rrt_connect: too many problems");
    DeviceGuard g(ctx->device);
    const int D = ctx->robot.n_joints;
    const size_t n_nodes = static_cast<size_t>(B) * 2 * cap * D, n_par = static_cast<size_t>(B) * 2 * cap;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSuccess;
    if (n_nodes > ctx->rrt_node_cap || n_par > ctx->rrt_parent_cap || !ctx->rrt_queue) {
        cudaStreamSynchronize(st);
        cudaFree(ctx->rrt_nodes);
        cudaFree(ctx->rrt_parent);
        ctx->rrt_nodes = nullptr;
        ctx->rrt_parent = nullptr;
        ctx->rrt_node_cap = ctx->rrt_parent_cap = 0;
        e = cudaMalloc(&ctx->rrt_nodes, n_nodes * sizeof(float));
        if (e == cudaSuccess) e = cudaMalloc(&ctx->rrt_parent, n_par * sizeof(int));
        if (e == cudaSuccess && !ctx->rrt_queue) e = cudaMalloc(&ctx->rrt_queue, 3 * sizeof(int));
        if (e != cudaSuccess) return cuda_fail(ctx, e, "vp_rrt_connect (scratch)");
        ctx->rrt_node_cap = n_nodes;
        ctx->rrt_parent_cap = n_par;
    }
    // problems the first phase sets aside: their indices, then where each stands
    const size_t n_idx = ((static_cast<size_t>(B) + 3) / 4) * 4;  // B indices, padded to 16 bytes
    const size_t n_pend = n_idx + static_cast<size_t>(B) * 4;      // then B int4
    if (n_pend > ctx->rrt_pending_cap) {
        cudaStreamSynchronize(st);
        cudaFree(ctx->rrt_pending);
        ctx->rrt_pending = nullptr;
        ctx->rrt_pending_cap = 0;
        e = cudaMalloc(&ctx->rrt_pending, n_pend * sizeof(int));
        if (e != cudaSuccess) return cuda_fail(ctx, e, "vp_rrt_connect (scratch)");
        ctx->rrt_pending_cap = n_pend;
    }
    // the int4 array starts at the first 16-byte boundary after the B indices
    int *save_base = ctx->rrt_pending + n_idx;
    RRTLaunch L{start, goal, samples, B, T, cap, range, resolution, ctx->rrt_nodes, ctx->rrt_parent, ctx->rrt_queue,
                ctx->rrt_pending, reinterpret_cast<int4 *>(save_base), status, iters, path, path_len, tree_sizes,
                ctx->batched.watchdog_ns};
    EnvView view = ctx->env;
    view.order = batched_check_order(ctx->batched);
    std::string msg;
    const int rc = rrt_launch(ctx->robot, view, L, ctx->status, ctx->num_sms, ctx->smem_optin, st, &msg);
    if (rc == 0) return VP_OK;
    return fail(ctx, rc == 1 ? VP_ERR_CAPACITY : VP_ERR_CUDA, "vp_rrt_connect: %s", msg.c_str());
}

extern "C" vp_status vp_fk_codegen(vp_ctx *ctx, int enable, double *compile_ms) {
    if (!ctx) return VP_ERR_ARG;
    if (!ctx->robot_loaded) return fail(ctx, VP_ERR_NOT_LOADED, "robot not loaded");
    DeviceGuard g(ctx->device);
    if (enable < -1 || enable > 1) return fail(ctx, VP_ERR_ARG, "vp_fk_codegen: enable must be -1, 0 or 1");
    if (enable != 1) {
        ctx->fk_mode = enable;
        if (compile_ms) *compile_ms = ctx->fk_gen.kernel ? ctx->fk_gen.compile_ms : 0.0;
        return VP_OK;
    }
    if (!ctx->fk_gen.kernel) {
        std::string msg;
        if (fk_codegen_build(ctx->robot, &ctx->fk_gen, &msg) != 0) return fail(ctx, VP_ERR_CUDA, "vp_fk_codegen: %s", msg.c_str());
    }
    ctx->fk_mode = 1;
    if (compile_ms) *compile_ms = ctx->fk_gen.compile_ms;
    return VP_OK;
}

extern "C" vp_status vp_nearest(vp_ctx *ctx, const float *points, int64_t M, const float *queries, int64_t N,
                                 int D, int64_t *index, float *dist2, void *stream) {
    if (!ctx) return VP_ERR_ARG;
    if (D < 1 || D > 16) return fail(ctx, VP_ERR_ARG, "vp_nearest: D must be in [1, 16]");
    if (M < 1) return fail(ctx, VP_ERR_ARG, "vp_nearest: no points");
    if (M >= 0xffffffffLL) return fail(ctx, VP_ERR_CAPACITY, "vp_nearest: at most 2^32 - 2 points");
    if (N < 0) return fail(ctx, VP_ERR_ARG, "vp_nearest: N < 0");
    if (N == 0) return VP_OK;
    if (!points || !queries || !index) return fail(ctx, VP_ERR_ARG, "vp_nearest: NULL buffer");
    if (reinterpret_cast<uintptr_t>(index) % 8) return fail(ctx, VP_ERR_ARG, "vp_nearest: index not 8-byte aligned");
    DeviceGuard g(ctx->device);
    std::string msg;
    const int rc = nn_launch(points, M, queries, N, D, index, dist2, ctx->num_sms, static_cast<cudaStream_t>(stream),
                             &msg);
    if (rc == 0) return VP_OK;
    return fail(ctx, rc == 1 ? VP_ERR_CAPACITY : VP_ERR_CUDA, "vp_nearest: %s", msg.c_str());
}

extern "C" vp_status vp_sync_status(vp_ctx *ctx, void *stream, uint32_t *bits) {
    if (!ctx) return VP_ERR_ARG;
    DeviceGuard g(ctx->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned h = 0;
    cudaError_t e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, ctx->status, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->status, 0, sizeof(unsigned), st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "vp_sync_status");
    if (bits) *bits = h;
    if (h & VP_DEVERR_TIMEOUT) return fail(ctx, VP_ERR_TIMEOUT, "device watchdog fired (status 0x%x)", h);
    if (h) return fail(ctx, VP_ERR_DEVICE, "device reported bad input (status 0x%x)", h);
    return VP_OK;
}

// ---------------------------------------------------------------------------
// robot packing without a context (used by the allocation-free entry point)

namespace vp {

// Packs `r` exactly as vp_load_robot does, through a context that owns no
// device resources (vp_load_robot itself touches no device memory).
vp_status pack_robot_host(const vp_robot_desc *r, RobotParams *out, std::string *err) {
    vp_ctx host_only;
    const vp_status s = vp_load_robot(&host_only, r);
    if (s == VP_OK)
        *out = host_only.robot;
    else if (err)
        *err = host_only.err;
    return s;
}

}  // namespace vp
