// Kernels of the plain path: edge validation (one warp per edge, raked
// states), state validation, FK sphere centres and edge state counts.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>
#include <vector>

#include "vp_validate.cuh"

namespace vp {

size_t smem_bytes(const EnvView &env, int n_links, int block) {
    const size_t warps = static_cast<size_t>((block + 31) / 32);
    return env_smem_bytes(env) + 16 + warps * 32 * sizeof(float) +
           static_cast<size_t>(n_links * kCentreFloats + (n_links - 1) * 2) * block * sizeof(float);
}

// One lane per configuration; lanes are independent (a warp stops once all
// its lanes collided).
template <int LMAX>
__global__ void VP_VALIDATION_BOUNDS(LMAX, 5) states_kernel(const __grid_constant__ RobotParams P, const EnvView env,
                                                     const float *__restrict__ q, const long long N,
                                                     uint8_t *__restrict__ valid, unsigned *status) {
    extern __shared__ __align__(16) unsigned char smem[];
    const SmemCarve sc = env.staged ? carve<true>(smem, env, P) : carve<false>(smem, env, P);
    if (!stage_env(sc.env, env, sc.bar, status)) return;
    const EnvSm es = env_views_rt(sc.env, env);
    const Stash &stash = sc.stash;
    const int lane = threadIdx.x & 31;
    const int D = P.n_joints;
    const long long step = static_cast<long long>(gridDim.x) * blockDim.x;
    for (long long base = static_cast<long long>(blockIdx.x) * blockDim.x + (threadIdx.x & ~31); base < N;
         base += step) {
        long long i = base + lane;
        const bool real = i < N;
        if (!real) i = N - 1;
        const float *qi = q + i * D;
        bool fin = true;
        for (int j = 0; j < D; ++j) fin &= isfinite(qi[j]);
        const WorkRef<false> w{nullptr, false};
        const bool c = pose_and_check<kStopAll, false, LMAX, false>(P, [qi](int j) { return qi[j]; }, es, stash, Ctl{kFull, false}, w);
        if (real) valid[i] = (c || !fin) ? 0 : 1;
    }
}

// FK sphere centres: one thread per configuration, a block of kFkConfigs
// consecutive configurations.  The centres go to shared memory first (in the
// caller's sphere order); the block's rows are one contiguous range of the
// output and leave in a single TMA bulk store (cp.async.bulk), whole 16-byte
// units of it when the output is 16-byte aligned, the rest by plain stores.
__global__ void __launch_bounds__(32) fk_kernel(const __grid_constant__ RobotParams P, const float *__restrict__ q,
                                                const long long N, float *__restrict__ out) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int cpb = blockDim.x;
    const int D = P.n_joints, S = P.n_spheres;
    float *buf = reinterpret_cast<float *>(smem);  // [cpb][3 S]
    Stash stash;
    stash.frames = buf + static_cast<size_t>(cpb) * 3 * S;
    stash.centres = nullptr;
    stash.motion = nullptr;
    stash.stride = cpb;
    const long long base = static_cast<long long>(blockIdx.x) * cpb;
    const long long i = base + threadIdx.x;
    if (i < N) {
        const float *qi = q + i * D;
        float *oi = buf + static_cast<size_t>(threadIdx.x) * 3 * S;
        Fr f;
        fr_identity(f);
        for (int l = 0; l <= D; ++l) {
            if (l > 0) {
                const JointC &J = P.joints[l - 1];
                const int pm = (J.meta >> kMetaParentShift) & 0xFF;
                if (pm == kParentBase)
                    fr_identity(f);
                else if (pm != kParentPrev)
                    stash.load_frame(pm, f);
                apply_joint(J, qi[l - 1], f);
                if (P.links[l].slot >= 0) stash.store_frame(P.links[l].slot, f);
            }
            const LinkC &L = P.links[l];
            for (int s = L.s0; s < L.s1; ++s) {
                const float4 sp = P.spheres[s];
                const float3 c = fr_apply(f, sp.x, sp.y, sp.z);
                float *o = oi + 3 * P.perm[s];
                o[0] = c.x;
                o[1] = c.y;
                o[2] = c.z;
            }
        }
    }
    const long long rows = min(static_cast<long long>(cpb), N - base);
    const long long count = rows * 3 * S;
    float *dst = out + base * 3 * S;
    const long long bulk = (reinterpret_cast<uintptr_t>(dst) & 15u) ? 0 : ((count * 4) & ~15ll);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // staged rows visible to the bulk copy
    __syncthreads();
    if (threadIdx.x == 0 && bulk > 0) {
        const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(buf));
        asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(sa),
                     "r"(static_cast<unsigned>(bulk))
                     : "memory");
        asm volatile("cp.async.bulk.commit_group;" ::: "memory");
    }
    for (long long e = bulk / 4 + threadIdx.x; e < count; e += cpb) dst[e] = buf[e];
    // shared memory stays allocated until the bulk copy has read it
    if (threadIdx.x == 0 && bulk > 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}

__global__ void counts_kernel(const int D, const float *__restrict__ q0, const float *__restrict__ q1,
                              const float res, const long long E, int32_t *__restrict__ counts) {
    const long long e = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e >= E) return;
    float dmax = 0.f;
    bool fin = true;
    for (int j = 0; j < D; ++j) {
        const float a = q0[e * D + j], b = q1[e * D + j];
        fin &= isfinite(a) && isfinite(b);
        if (fin) dmax = fmaxf(dmax, fabsf(b - a));
    }
    counts[e] = fin ? count_from_dmax(dmax, res) : -1;
}

// How often each self-pair group (link pair) collides: one configuration
// per thread, every link frame kept (in local memory), every group's sphere
// pairs tested until one collides; hits[g] counts the configurations in
// which group g has a colliding pair.  Feeds the frequent-first check order.
__global__ void group_hits_kernel(const __grid_constant__ RobotParams P, const float *__restrict__ q,
                                  const long long N, unsigned *__restrict__ hits) {
    const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int D = P.n_joints;
    const float *qi = q + i * D;
    for (int j = 0; j < D; ++j)
        if (!isfinite(qi[j])) return;
    Fr F[kMaxLinks];
    fr_identity(F[0]);
    for (int j = 0; j < D; ++j) {
        const JointC &J = P.joints[j];
        F[j + 1] = F[(J.meta >> kMetaParentLinkShift) & 0xFF];
        apply_joint(J, qi[j], F[j + 1]);
    }
    for (int g = 0; g < P.n_groups; ++g) {
        const GroupC G = P.groups[g];
        bool hit = false;
        for (int p = G.p0; p < G.p1 && !hit; ++p) {
            const PairC pr = P.pairs[p];
            const float4 sa = P.spheres[pr.a], sb = P.spheres[pr.b];
            const float3 a = fr_apply(F[G.la], sa.x, sa.y, sa.z);
            const float3 b = fr_apply(F[G.lb], sb.x, sb.y, sb.z);
            const float ex = a.x - b.x, ey = a.y - b.y, ez = a.z - b.z;
            const float r2 = sa.w + sb.w;
            hit = fmaf(ex, ex, fmaf(ey, ey, ez * ez)) < r2 * r2;
        }
        if (hit) atomicAdd(&hits[g], 1u);
    }
}

// How often each primitive collides: one configuration per thread, every
// link frame kept; for every primitive (packed order, kinds one after the
// other), each link's bounding sphere is tested and, where it touches, the
// link's spheres; hits[k] counts the configurations in which primitive k
// touches some sphere.  Feeds the environment's visiting order.
template <int KIND>
__device__ __forceinline__ void count_kind(const RobotParams &P, const Fr *F, const float4 *prims, int n,
                                           unsigned *hits) {
    using K = Kind<KIND>;
    for (int k = 0; k < n; ++k) {
        const float4 *o = prims + k * K::kWords;
        bool hit = false;
        for (int l = 0; l < P.n_links && !hit; ++l) {
            const LinkC &L = P.links[l];
            if (L.s0 >= L.s1 || !K::hit(fr_apply(F[l], L.bs.x, L.bs.y, L.bs.z), L.bs.w, o)) continue;
            for (int sp = L.s0; sp < L.s1 && !hit; ++sp) {
                const float4 c = P.spheres[sp];
                hit = K::hit(fr_apply(F[l], c.x, c.y, c.z), c.w, o);
            }
        }
        if (hit) atomicAdd(&hits[k], 1u);
    }
}

__global__ void prim_hits_kernel(const __grid_constant__ RobotParams P, const EnvView env, const float *__restrict__ q,
                                 const long long N, unsigned *__restrict__ hits) {
    const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int D = P.n_joints;
    const float *qi = q + i * D;
    for (int j = 0; j < D; ++j)
        if (!isfinite(qi[j])) return;
    Fr F[kMaxLinks];
    fr_identity(F[0]);
    for (int j = 0; j < D; ++j) {
        const JointC &J = P.joints[j];
        F[j + 1] = F[(J.meta >> kMetaParentLinkShift) & 0xFF];
        apply_joint(J, qi[j], F[j + 1]);
    }
    const EnvSm e = env_views<false>(nullptr, env);
    count_kind<0>(P, F, e.sph, e.ns, hits);
    count_kind<1>(P, F, e.cap, e.nc, hits + e.ns);
    count_kind<2>(P, F, e.box, e.nb, hits + e.ns + e.nc);
}

// ---------------------------------------------------------------------------
// launchers

template <class K>
static cudaError_t prepare(K kernel, size_t smem, int block, int *blocks_per_sm) {
    cudaError_t err = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (err != cudaSuccess) return err;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, kernel, block, smem);
}

const KernelSet &kernel_set(int lmax) {
    auto make = [](void (*f0)(KernelSet &), void (*f1)(KernelSet &), void (*f2)(KernelSet &)) {
        KernelSet s;
        f0(s);
        f1(s);
        f2(s);
        return s;
    };
    static const KernelSet s8 = make(kernel_set_fill_l8_f0, kernel_set_fill_l8_f1, kernel_set_fill_l8_f2);
    static const KernelSet s9 = make(kernel_set_fill_l9_f0, kernel_set_fill_l9_f1, kernel_set_fill_l9_f2);
    static const KernelSet s15 = make(kernel_set_fill_l15_f0, kernel_set_fill_l15_f1, kernel_set_fill_l15_f2);
    static const KernelSet s17 = make(kernel_set_fill_l17_f0, kernel_set_fill_l17_f1, kernel_set_fill_l17_f2);
    switch (lmax) {
        case 8: return s8;
        case 9: return s9;
        case 15: return s15;
        default: return s17;
    }
}

cudaError_t prepare_edges_plain(bool stats, int lmax, bool simple, bool staged, size_t smem, int block,
                                int *blocks_per_sm, int order) {
    // every family's attribute is set; the occupancy is that of the family of `order`
    cudaError_t e = cudaSuccess;
    for (int f = 0; f < kFamCount && e == cudaSuccess; ++f)
        if (f != family_of(order))
            e = cudaFuncSetAttribute(kernel_set(lmax).plain[f][stats][simple][staged],
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess) return e;
    return prepare(kernel_set(lmax).plain[family_of(order)][stats][simple][staged], smem, block, blocks_per_sm);
}

cudaError_t launch_edges_plain(const RobotParams &P, const EnvView &env, const float *q0, const float *q1,
                               const int32_t *counts, float res, int64_t E, uint8_t *valid, unsigned *status,
                               unsigned long long *work, int grid, int block, size_t smem, cudaStream_t st) {
    kernel_set(lmax_for(P.n_links))
        .plain[family_of(env.order)][work != nullptr][P.simple != 0][env.staged != 0]<<<grid, block, smem, st>>>(
            P, env, q0, q1, counts, res, E, valid, status, work);
    return cudaGetLastError();
}

using StatesKernel = void (*)(const RobotParams, const EnvView, const float *, const long long, uint8_t *,
                              unsigned *);
static StatesKernel states_kernel_for(int lmax) {
    switch (lmax) {
        case 8: return states_kernel<8>;
        case 9: return states_kernel<9>;
        case 15: return states_kernel<15>;
        default: return states_kernel<17>;
    }
}

cudaError_t prepare_states(int lmax, size_t smem, int block, int *blocks_per_sm) {
    return prepare(states_kernel_for(lmax), smem, block, blocks_per_sm);
}

cudaError_t launch_states(const RobotParams &P, const EnvView &env, const float *q, int64_t N, uint8_t *valid,
                          unsigned *status, int grid, int block, size_t smem, cudaStream_t st) {
    states_kernel_for(lmax_for(P.n_links))<<<grid, block, smem, st>>>(P, env, q, N, valid, status);
    return cudaGetLastError();
}

cudaError_t prepare_fk(size_t smem, int block, int *blocks_per_sm) {
    return prepare(fk_kernel, smem, block, blocks_per_sm);
}

// Configurations per FK block: 32 while a block's output rows fit in 48 KB
// of shared memory, else fewer.
int fk_configs_per_block(int n_spheres) {
    int c = 32;
    while (c > 4 && static_cast<size_t>(c) * 3 * n_spheres * sizeof(float) > 48 * 1024) c /= 2;
    return c;
}

cudaError_t launch_fk(const RobotParams &P, const float *q, int64_t N, float *centres, int grid, int block,
                      size_t smem, cudaStream_t st) {
    fk_kernel<<<grid, block, smem, st>>>(P, q, N, centres);
    return cudaGetLastError();
}

int group_order(const RobotParams &P, const float *q, int64_t N, cudaStream_t st, uint8_t *order, int *n_front,
                std::string *msg) {
    const int ng = P.n_groups;
    for (int g = 0; g < kMaxGroups; ++g) order[g] = static_cast<uint8_t>(g < ng ? g : 0);
    *n_front = ng;
    if (ng == 0 || N <= 0) return 0;
    unsigned *d_hits = nullptr;
    std::vector<unsigned> hits(static_cast<size_t>(ng), 0u);
    cudaError_t e = cudaMalloc(&d_hits, sizeof(unsigned) * ng);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_hits, 0, sizeof(unsigned) * ng, st);
    if (e == cudaSuccess) {
        const int block = 128;
        group_hits_kernel<<<static_cast<unsigned>((N + block - 1) / block), block, 0, st>>>(P, q, N, d_hits);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(hits.data(), d_hits, sizeof(unsigned) * ng, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (d_hits) cudaFree(d_hits);
    if (e != cudaSuccess) {
        *msg = std::string("group hit count: ") + cudaGetErrorString(e);
        return 2;
    }
    std::vector<int> idx(static_cast<size_t>(ng));
    for (int g = 0; g < ng; ++g) idx[g] = g;
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return hits[a] > hits[b]; });
    for (int g = 0; g < ng; ++g) order[g] = static_cast<uint8_t>(idx[g]);
    // the leading groups that hold three quarters of the counted collisions
    // go before the primitives (all of them when nothing collided)
    unsigned long long total = 0, run = 0;
    for (int g = 0; g < ng; ++g) total += hits[g];
    int front = ng;
    if (total > 0)
        for (int g = 0; g < ng; ++g) {
            run += hits[idx[g]];
            if (4 * run >= 3 * total) {
                front = g + 1;
                break;
            }
        }
    *n_front = front;
    return 0;
}

int prim_hits(const RobotParams &P, const EnvView &env, const float *q, int64_t N, cudaStream_t st,
              std::vector<unsigned> *hits, std::string *msg) {
    const int n = env.ns + env.nc + env.nb;
    hits->assign(static_cast<size_t>(n), 0u);
    if (n == 0 || N <= 0) return 0;
    unsigned *d_hits = nullptr;
    cudaError_t e = cudaMalloc(&d_hits, sizeof(unsigned) * n);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_hits, 0, sizeof(unsigned) * n, st);
    if (e == cudaSuccess) {
        EnvView v = env;
        v.staged = 0;
        const int block = 128;
        prim_hits_kernel<<<static_cast<unsigned>((N + block - 1) / block), block, 0, st>>>(P, v, q, N, d_hits);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(hits->data(), d_hits, sizeof(unsigned) * n, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (d_hits) cudaFree(d_hits);
    if (e != cudaSuccess) {
        *msg = std::string("primitive hit count: ") + cudaGetErrorString(e);
        return 2;
    }
    return 0;
}

cudaError_t launch_counts(int D, const float *q0, const float *q1, float res, int64_t E, int32_t *counts,
                          cudaStream_t st) {
    const int block = 256;
    const long long grid = (E + block - 1) / block;
    counts_kernel<<<static_cast<unsigned>(grid), block, 0, st>>>(D, q0, q1, res, E, counts);
    return cudaGetLastError();
}

}  // namespace vp
