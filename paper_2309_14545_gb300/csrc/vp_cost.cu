// Smooth penetration cost c(q) = sum_s sum_o max(0, r_s + m - d(c_s, o))^2
// and its gradient by a reverse-mode FK adjoint (an addition beside the
// paper's boolean check, which stays the judge of validity).
//
// One thread per configuration.  Forward: pose the links joint by joint; for
// each sphere accumulate the cost and g_s = dc/dc_s = sum_o -2 pen grad d;
// per link keep G = sum g_s and M = sum c_s x g_s.  Backward: sweep the links
// from the leaves to the base, adding each link's (G, M) into its parent's,
// so that each link holds the sums over the subtree its joint moves.  Then
// pose again (FK is a few hundred FMAs against thousands of ball tests) to
// get each joint's world axis a and origin p, and
//   dc/dq_j = a_j . (M_j - p_j x G_j)   (revolute)
//   dc/dq_j = a_j . G_j                 (prismatic).
// Keeping only (G, M) per link, not the axes and origins as well, halves the
// shared memory a thread holds, which sets how many warps an SM keeps.
#include <cuda_runtime.h>

#include <algorithm>

#include "vp_cost.h"
#include "vp_device.cuh"

namespace vp {

namespace {

constexpr int kLinkFloats = 6;  // G, M per link and lane

struct LinkStore {
    float *base;
    int stride;
    __device__ __forceinline__ float &at(int l, int k) const { return base[(l * kLinkFloats + k) * stride + threadIdx.x]; }
};

// Accumulate the penetration of ball (x, r) with every primitive: returns the
// cost and adds dcost/dx into g.
__device__ __forceinline__ float ball_cost(float3 x, float r, const EnvSm &env, float3 &g) {
    float c = 0.f;
    for (int o = 0; o < env.ns; ++o) {
        const float4 ob = env.sph[o];
        const float vx = x.x - ob.x, vy = x.y - ob.y, vz = x.z - ob.z;
        const float n2 = fmaf(vx, vx, fmaf(vy, vy, vz * vz));
        const float reach = r + ob.w;
        if (n2 < reach * reach) {  // pen = reach - |v| > 0
            const float n = sqrtf(n2);
            const float pen = reach - n;
            c = fmaf(pen, pen, c);
            if (n > 0.f) {
                const float s = -2.f * pen / n;
                g.x = fmaf(s, vx, g.x);
                g.y = fmaf(s, vy, g.y);
                g.z = fmaf(s, vz, g.z);
            }
        }
    }
    for (int o = 0; o < env.nc; ++o) {
        const float4 a = env.cap[2 * o], b = env.cap[2 * o + 1];
        const float wx = x.x - a.x, wy = x.y - a.y, wz = x.z - a.z;
        const float t = __saturatef(fmaf(wx, b.x, fmaf(wy, b.y, wz * b.z)) * b.w);
        const float vx = fmaf(-t, b.x, wx), vy = fmaf(-t, b.y, wy), vz = fmaf(-t, b.z, wz);
        const float n2 = fmaf(vx, vx, fmaf(vy, vy, vz * vz));
        const float reach = r + a.w;
        if (n2 < reach * reach) {
            const float n = sqrtf(n2);
            const float pen = reach - n;
            c = fmaf(pen, pen, c);
            if (n > 0.f) {
                const float s = -2.f * pen / n;
                g.x = fmaf(s, vx, g.x);
                g.y = fmaf(s, vy, g.y);
                g.z = fmaf(s, vz, g.z);
            }
        }
    }
    for (int o = 0; o < env.nb; ++o) {
        const float4 a0 = env.box[4 * o], a1 = env.box[4 * o + 1], a2 = env.box[4 * o + 2], h = env.box[4 * o + 3];
        const float y0 = fmaf(a0.x, x.x, fmaf(a0.y, x.y, fmaf(a0.z, x.z, a0.w)));
        const float y1 = fmaf(a1.x, x.x, fmaf(a1.y, x.y, fmaf(a1.z, x.z, a1.w)));
        const float y2 = fmaf(a2.x, x.x, fmaf(a2.y, x.y, fmaf(a2.z, x.z, a2.w)));
        const float e0 = fabsf(y0) - h.x, e1 = fabsf(y1) - h.y, e2 = fabsf(y2) - h.z;
        const float o0 = fmaxf(e0, 0.f), o1 = fmaxf(e1, 0.f), o2 = fmaxf(e2, 0.f);
        const float out2 = fmaf(o0, o0, fmaf(o1, o1, o2 * o2));
        if (out2 >= r * r) continue;  // d >= r: no penetration
        float d, gb0 = 0.f, gb1 = 0.f, gb2 = 0.f;
        if (out2 > 0.f) {
            const float n = sqrtf(out2);
            d = n;
            const float inv = 1.f / n;
            gb0 = copysignf(o0 * inv, y0);
            gb1 = copysignf(o1 * inv, y1);
            gb2 = copysignf(o2 * inv, y2);
        } else {
            // inside: distance to the nearest face
            if (e0 >= e1 && e0 >= e2) {
                d = e0;
                gb0 = copysignf(1.f, y0);
            } else if (e1 >= e2) {
                d = e1;
                gb1 = copysignf(1.f, y1);
            } else {
                d = e2;
                gb2 = copysignf(1.f, y2);
            }
        }
        const float pen = r - d;
        c = fmaf(pen, pen, c);
        const float s = -2.f * pen;
        // world gradient of d: sum_i gb_i a_i
        g.x = fmaf(s, fmaf(gb0, a0.x, fmaf(gb1, a1.x, gb2 * a2.x)), g.x);
        g.y = fmaf(s, fmaf(gb0, a0.y, fmaf(gb1, a1.y, gb2 * a2.y)), g.y);
        g.z = fmaf(s, fmaf(gb0, a0.z, fmaf(gb1, a1.z, gb2 * a2.z)), g.z);
    }
    return c;
}

template <bool STAGED>
__global__ void __launch_bounds__(128) cost_kernel(const __grid_constant__ RobotParams P, const EnvView env,
                                                   const float *__restrict__ q, const long long N, const float margin,
                                                   float *__restrict__ cost, float *__restrict__ grad,
                                                   unsigned *status) {
    extern __shared__ __align__(16) unsigned char smem[];
    size_t off = STAGED ? static_cast<size_t>(env_prim_float4(env)) * 16 : 0;  // no boxes: the cost has no cull
    float4 *env_sm = reinterpret_cast<float4 *>(smem);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + off);
    off += 16;
    const LinkStore ls{reinterpret_cast<float *>(smem + off), static_cast<int>(blockDim.x)};
    off += static_cast<size_t>(P.n_links) * kLinkFloats * blockDim.x * sizeof(float);
    Stash stash;
    stash.frames = reinterpret_cast<float *>(smem + off);
    stash.centres = nullptr;
    stash.motion = nullptr;
    stash.stride = static_cast<int>(blockDim.x);
    if (STAGED && !stage_env(env_sm, env, bar, status, env_prim_float4(env))) return;
    const EnvSm es = env_views<STAGED>(env_sm, env);
    const int D = P.n_joints;
    for (long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; i < N;
         i += static_cast<long long>(gridDim.x) * blockDim.x) {
        const float *qi = q + i * D;
        Fr f;
        fr_identity(f);
        float c = 0.f;
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
            float3 G = make_float3(0.f, 0.f, 0.f), M = make_float3(0.f, 0.f, 0.f);
            const LinkC &L = P.links[l];
            for (int s = L.s0; s < L.s1; ++s) {
                const float4 sp = P.spheres[s];
                const float3 x = fr_apply(f, sp.x, sp.y, sp.z);
                float3 gs = make_float3(0.f, 0.f, 0.f);
                c += ball_cost(x, sp.w + margin, es, gs);
                G.x += gs.x;
                G.y += gs.y;
                G.z += gs.z;
                M.x = fmaf(x.y, gs.z, fmaf(-x.z, gs.y, M.x));
                M.y = fmaf(x.z, gs.x, fmaf(-x.x, gs.z, M.y));
                M.z = fmaf(x.x, gs.y, fmaf(-x.y, gs.x, M.z));
            }
            if (grad != nullptr && l > 0) {
                ls.at(l, 0) = G.x;
                ls.at(l, 1) = G.y;
                ls.at(l, 2) = G.z;
                ls.at(l, 3) = M.x;
                ls.at(l, 4) = M.y;
                ls.at(l, 5) = M.z;
            }
        }
        cost[i] = c;
        if (grad == nullptr) continue;
        // subtree sums, leaves to base (joints are numbered parents first)
        for (int l = D; l >= 1; --l) {
            const int plink = (P.joints[l - 1].meta >> kMetaParentLinkShift) & 0xFF;
            if (plink >= 1)
                for (int k = 0; k < kLinkFloats; ++k) ls.at(plink, k) += ls.at(l, k);
        }
        // pose again for each joint's world axis and origin
        fr_identity(f);
        for (int l = 1; l <= D; ++l) {
            const JointC &J = P.joints[l - 1];
            const int pm = (J.meta >> kMetaParentShift) & 0xFF;
            if (pm == kParentBase)
                fr_identity(f);
            else if (pm != kParentPrev)
                stash.load_frame(pm, f);
            apply_joint(J, qi[l - 1], f);
            if (P.links[l].slot >= 0) stash.store_frame(P.links[l].slot, f);
            // the joint's world axis (R_after a = R_before a about its own axis)
            const float ax = fmaf(f.r0, J.ax[0], fmaf(f.r1, J.ax[1], f.r2 * J.ax[2]));
            const float ay = fmaf(f.r3, J.ax[0], fmaf(f.r4, J.ax[1], f.r5 * J.ax[2]));
            const float az = fmaf(f.r6, J.ax[0], fmaf(f.r7, J.ax[1], f.r8 * J.ax[2]));
            const float Gx = ls.at(l, 0), Gy = ls.at(l, 1), Gz = ls.at(l, 2);
            float gj;
            if (J.meta & kMetaPrismatic) {
                gj = fmaf(ax, Gx, fmaf(ay, Gy, az * Gz));
            } else {
                const float Mx = ls.at(l, 3), My = ls.at(l, 4), Mz = ls.at(l, 5);
                const float px = f.px, py = f.py, pz = f.pz;
                // M - p x G
                const float tx = Mx - fmaf(py, Gz, -pz * Gy);
                const float ty = My - fmaf(pz, Gx, -px * Gz);
                const float tz = Mz - fmaf(px, Gy, -py * Gx);
                gj = fmaf(ax, tx, fmaf(ay, ty, az * tz));
            }
            grad[i * D + (l - 1)] = gj;
        }
    }
}

}  // namespace

int cost_launch(const RobotParams &P, const EnvView &env, const float *q, int64_t n, float margin, float *cost,
                float *grad, unsigned *status, int num_sms, size_t smem_optin, cudaStream_t st, std::string *msg) {
    // largest block that fits; the environment in shared memory unless that
    // lowers the blocks per SM (then read in place, through L1)
    int block = 0, bps = 0;
    size_t smem = 0;
    EnvView view = env;
    cudaError_t e = cudaSuccess;
    for (int b : {128, 64, 32}) {
        const size_t rest = 16 + static_cast<size_t>(P.n_links * kLinkFloats + P.n_slots * kFrameFloats) * b *
                                     sizeof(float);
        EnvView vst = env;
        vst.staged = 1;
        const size_t m_st = static_cast<size_t>(env_prim_float4(vst)) * 16 + rest;
        if (rest > smem_optin) continue;
        const size_t m_max = m_st <= smem_optin ? m_st : rest;
        e = cudaFuncSetAttribute(cost_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 static_cast<int>(m_max));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(cost_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     static_cast<int>(rest));
        int b_in = 0, b_st = 0;
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b_in, cost_kernel<false>, b, rest);
        if (e == cudaSuccess && m_st <= smem_optin)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b_st, cost_kernel<true>, b, m_st);
        if (e != cudaSuccess) break;
        view.staged = (b_st >= 1 && b_st >= b_in) ? 1 : 0;
        smem = view.staged ? m_st : rest;
        bps = view.staged ? b_st : b_in;
        block = b;
        break;
    }
    if (e == cudaSuccess && !block) {
        *msg = "per-link adjoint storage exceeds shared memory";
        return 1;
    }
    if (e == cudaSuccess) {
        const int64_t need = (n + block - 1) / block;
        const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(need, static_cast<int64_t>(std::max(bps, 1)) * num_sms));
        (view.staged ? cost_kernel<true> : cost_kernel<false>)<<<static_cast<unsigned>(grid), block, smem, st>>>(
            P, view, q, n, margin, cost, grad, status);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        *msg = cudaGetErrorString(e);
        return 2;
    }
    return 0;
}

}  // namespace vp
