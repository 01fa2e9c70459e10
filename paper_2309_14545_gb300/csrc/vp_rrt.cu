// Batched RRT-Connect (Sec. III-E, "Bringing it Together": one of the two
// planners built on the vectorized primitives), device-resident: one warp
// solves one problem -- both trees in global memory, nearest-node scans over
// the warp's lanes, every edge checked by the same raked state check as
// vp_validate_edges -- and takes the next problem from a queue.
//
// The decisions that shape the trees -- which node is nearest, where the new
// node lies -- are FP32 with every operation rounded on its own (products,
// sums, differences, one square root and one division; no contraction), so
// a float32 reference taking the same steps builds the same trees wherever
// the edge verdicts agree.
//
// The kernel is a state machine with a single call site of the edge check
// (start and goal validity, EXTEND and CONNECT all pass through it), which
// keeps the inlined state check -- most of the code -- to one copy.
#include <cuda_runtime.h>

#include "vp_validate.cuh"

namespace vp {

namespace {

constexpr int kRRTThreads = 128;
constexpr int kRRTWarps = kRRTThreads / 32;
enum : int { kTrapped = 0, kAdvanced = 1, kReached = 2 };
enum : int { kCheckStart, kCheckGoal, kExtend, kConnect };

struct RRTArgs {
    const float *start, *goal, *samples;  // [B][D], [B][D], [B][T][D]
    long long B;
    int T, cap;
    float range, res;
    float *nodes;    // [B][2][cap][D] scratch
    int *parent;     // [B][2][cap] scratch
    int *queue;      // problem counter
    int *status;     // [B]: 1 solved, 0 not within T samples, -1 start or goal invalid
    int *iters;      // [B]: samples used
    float *path;     // [B][2 cap][D]
    int *path_len;   // [B]
    int *sizes;      // [B][2]
    unsigned long long watchdog_ns;
};

// A node index and the squared distance it was found at.
__device__ __forceinline__ unsigned long long pack_nd(float d2, int i) {
    return (static_cast<unsigned long long>(__float_as_uint(d2)) << 32) | static_cast<unsigned>(i);
}

template <int LMAX, bool SIMPLE, bool STAGED>
__global__ void VP_VALIDATION_BOUNDS(LMAX, 5)
    rrt_connect_kernel(const __grid_constant__ RobotParams P, const EnvView env, const RRTArgs a, unsigned *status) {
    extern __shared__ __align__(16) unsigned char smem[];
    const SmemCarve sc = carve<STAGED>(smem, env, P);
    // per warp: the target, the nearest node, the new node (16 floats each)
    __shared__ float s_vec[kRRTWarps][3][16];
    if (STAGED && !stage_env(sc.env, env, sc.bar, status)) return;
    const EnvSm es = env_views<STAGED>(sc.env, env);
    const Stash &stash = sc.stash;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int D = P.n_joints;
    float *wq0 = sc.warp_buf + wib * 32, *wdq = wq0 + 16;
    float *tgt = s_vec[wib][0], *nea = s_vec[wib][1], *nw = s_vec[wib][2];
    const uint64_t t_start = global_ns();
    while (true) {
        int b = 0;
        if (lane == 0) {
            b = (global_ns() - t_start >= a.watchdog_ns) ? -1 : atomicAdd(a.queue, 1);
            if (b < 0) atomicOr(status, VP_DEVERR_TIMEOUT);
        }
        b = __shfl_sync(kFull, b, 0);
        if (b < 0 || b >= a.B) break;
        float *tn[2] = {a.nodes + (static_cast<long long>(b) * 2) * a.cap * D,
                        a.nodes + (static_cast<long long>(b) * 2 + 1) * a.cap * D};
        int *tp[2] = {a.parent + (static_cast<long long>(b) * 2) * a.cap,
                      a.parent + (static_cast<long long>(b) * 2 + 1) * a.cap};
        const float *start = a.start + static_cast<long long>(b) * D, *goal = a.goal + static_cast<long long>(b) * D;
        if (lane < D) {
            tn[0][lane] = start[lane];
            tn[1][lane] = goal[lane];
        }
        if (lane == 0) tp[0][0] = tp[1][0] = -1;
        __syncwarp();
        int n[2] = {1, 1};
        int mode = kCheckStart, it = 0, ta = 0, t = 0, ia = -1, result = 0, meet = -1;
        bool done = false;
        while (!done) {
            // ---- what to check: (qa, qb) into the warp's interpolation buffers
            bool need = true;
            int near = -1, st_ok = kTrapped;
            if (mode == kCheckStart || mode == kCheckGoal) {
                const float *r = mode == kCheckStart ? start : goal;
                if (lane < D) {
                    nea[lane] = r[lane];
                    nw[lane] = r[lane];
                }
            } else {
                // nearest node of tree t to the target (lanes split the nodes)
                unsigned long long best = ~0ull;
                for (int i = lane; i < n[t]; i += 32) {
                    const float *x = tn[t] + static_cast<long long>(i) * D;
                    float acc = 0.f;
                    for (int d = 0; d < D; ++d) {
                        const float dx = __fsub_rn(x[d], tgt[d]);
                        acc = __fadd_rn(acc, __fmul_rn(dx, dx));
                    }
                    const unsigned long long v = pack_nd(acc, i);
                    best = v < best ? v : best;
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const unsigned long long w = __shfl_xor_sync(kFull, best, o);
                    best = w < best ? w : best;
                }
                near = static_cast<int>(best & 0xffffffffu);
                const float d2 = __uint_as_float(static_cast<unsigned>(best >> 32));
                if (lane < D) nea[lane] = tn[t][static_cast<long long>(near) * D + lane];
                __syncwarp();
                if (d2 == 0.f) {  // the target is already a node
                    need = false;
                    st_ok = kReached;
                } else if (n[t] == a.cap) {
                    need = false;
                    st_ok = kTrapped;
                    near = -1;
                } else {
                    const float dist = __fsqrt_rn(d2);
                    if (dist <= a.range) {
                        if (lane < D) nw[lane] = tgt[lane];
                        st_ok = kReached;
                    } else {
                        const float s = __fdiv_rn(a.range, dist);
                        if (lane < D) nw[lane] = __fadd_rn(nea[lane], __fmul_rn(s, __fsub_rn(tgt[lane], nea[lane])));
                        st_ok = kAdvanced;
                    }
                }
            }
            __syncwarp();
            // ---- the edge check (the only call site): raked states, as vp_validate_edges
            bool ok = true;
            if (need) {
                float dmax = 0.f;
                bool fin = true;
                for (int d = 0; d < D; ++d) {
                    const float x0 = nea[d], x1 = nw[d];
                    fin &= isfinite(x0) && isfinite(x1);
                    const float dq = x1 - x0;
                    if (fin) dmax = fmaxf(dmax, fabsf(dq));
                }
                if (lane < D) {
                    wq0[lane] = nea[lane];
                    wdq[lane] = nw[lane] - nea[lane];
                }
                __syncwarp();
                const int k = fin ? count_from_dmax(dmax, a.res) : -1;
                ok = k >= 2;
                if (ok) {
                    const int R = (k + 31) >> 5;
                    const float inv = __fdiv_rn(1.f, static_cast<float>(k - 1));
                    for (int r = 0; r < R; ++r) {
                        int i = lane * R + r;
                        if (i >= k) i = k - 1;
                        const float tt = static_cast<float>(i) * inv;
                        const WorkRef<false> w{nullptr, false};
                        const bool c = check_state<kFamPoseAll, kStopAny, false, LMAX, SIMPLE>(
                            P, [tt, wq0, wdq](int j) { return fmaf(tt, wdq[j], wq0[j]); }, es, stash,
                            Ctl{kFull, false}, w);
                        if (__any_sync(kFull, c)) {
                            ok = false;
                            break;
                        }
                    }
                }
                __syncwarp();
            }
            // ---- act on the outcome
            if (mode == kCheckStart || mode == kCheckGoal) {
                if (!ok) {
                    result = -1;
                    done = true;
                } else if (mode == kCheckStart) {
                    mode = kCheckGoal;
                } else {
                    mode = kExtend;
                    if (a.T == 0) done = true;
                    else if (lane < D) tgt[lane] = a.samples[(static_cast<long long>(b) * a.T) * D + lane];
                }
                __syncwarp();
                continue;
            }
            int s = st_ok, inew = near;
            if (need) {
                if (ok) {  // add the new node
                    inew = n[t];
                    if (lane < D) tn[t][static_cast<long long>(inew) * D + lane] = nw[lane];
                    if (lane == 0) tp[t][inew] = near;
                    ++n[t];
                } else {
                    s = kTrapped;
                }
            }
            __syncwarp();
            bool next = false;
            if (mode == kExtend) {
                if (s != kTrapped) {  // connect the other tree toward the new node
                    ia = inew;
                    if (lane < D) tgt[lane] = tn[t][static_cast<long long>(inew) * D + lane];
                    t = 1 - ta;
                    mode = kConnect;
                } else {
                    next = true;
                }
            } else {  // connect
                if (s == kReached) {
                    result = 1;
                    meet = inew;
                    done = true;
                } else if (s == kTrapped) {
                    next = true;
                }  // advanced: extend again toward the same node
            }
            if (next) {
                ++it;
                ta = 1 - ta;
                if (it == a.T) {
                    done = true;
                } else {
                    t = ta;
                    mode = kExtend;
                    if (lane < D) tgt[lane] = a.samples[(static_cast<long long>(b) * a.T + it) * D + lane];
                }
            }
            __syncwarp();
        }
        // ---- results: the path start ... goal through the meeting node
        int plen = 0;
        if (result == 1 && lane == 0) {
            // tree 0 holds the start: its chain from the meeting node, reversed,
            // then tree 1's chain past the meeting node (the same configuration)
            const int tx = 0, ty = 1;
            const int x0 = ta == 0 ? ia : meet, y0 = ta == 0 ? meet : ia;
            int lx = 0;
            for (int i = x0; i >= 0; i = tp[tx][i]) ++lx;
            float *out = a.path + static_cast<long long>(b) * 2 * a.cap * D;
            int pos = lx - 1;
            for (int i = x0; i >= 0; i = tp[tx][i], --pos)
                for (int d = 0; d < D; ++d) out[static_cast<long long>(pos) * D + d] = tn[tx][static_cast<long long>(i) * D + d];
            pos = lx;
            for (int i = tp[ty][y0]; i >= 0; i = tp[ty][i], ++pos)
                for (int d = 0; d < D; ++d) out[static_cast<long long>(pos) * D + d] = tn[ty][static_cast<long long>(i) * D + d];
            plen = pos;
        }
        if (lane == 0) {
            a.status[b] = result;
            a.iters[b] = result == -1 ? 0 : (result == 1 ? it + 1 : a.T);
            a.path_len[b] = plen;
            a.sizes[2 * b] = n[0];
            a.sizes[2 * b + 1] = n[1];
        }
        __syncwarp();
    }
}

using RRTKernel = void (*)(RobotParams, EnvView, RRTArgs, unsigned *);

template <int LMAX>
RRTKernel rrt_instance(bool simple, bool staged) {
    if (simple) return staged ? rrt_connect_kernel<LMAX, true, true> : rrt_connect_kernel<LMAX, true, false>;
    return staged ? rrt_connect_kernel<LMAX, false, true> : rrt_connect_kernel<LMAX, false, false>;
}

RRTKernel rrt_kernel_for(int lmax, bool simple, bool staged) {
    switch (lmax) {
        case 8: return rrt_instance<8>(simple, staged);
        case 9: return rrt_instance<9>(simple, staged);
        case 15: return rrt_instance<15>(simple, staged);
        default: return rrt_instance<17>(simple, staged);
    }
}

}  // namespace

int rrt_launch(const RobotParams &P, const EnvView &env_base, const RRTLaunch &L, unsigned *status, int num_sms,
               size_t smem_optin, cudaStream_t st, std::string *msg) {
    RRTArgs a;
    a.start = L.start;
    a.goal = L.goal;
    a.samples = L.samples;
    a.B = L.B;
    a.T = L.T;
    a.cap = L.cap;
    a.range = L.range;
    a.res = L.res;
    a.nodes = L.nodes;
    a.parent = L.parent;
    a.queue = L.queue;
    a.status = L.status;
    a.iters = L.iters;
    a.path = L.path;
    a.path_len = L.path_len;
    a.sizes = L.sizes;
    a.watchdog_ns = L.watchdog_ns;
    const int lmax = lmax_for(P.n_links);
    const bool simple = P.simple != 0;
    // environment in shared memory unless that lowers the blocks per SM
    EnvView vin = env_base, vst = env_base;
    vin.staged = 0;
    vst.staged = 1;
    const size_t m_in = smem_bytes(vin, P.n_links, kRRTThreads), m_st = smem_bytes(vst, P.n_links, kRRTThreads);
    if (m_in > smem_optin) {
        *msg = "frame stash exceeds shared memory";
        return 1;
    }
    const RRTKernel k_in = rrt_kernel_for(lmax, simple, false), k_st = rrt_kernel_for(lmax, simple, true);
    cudaError_t e = cudaFuncSetAttribute(k_in, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(m_in));
    int b_in = 0, b_st = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b_in, k_in, kRRTThreads, m_in);
    if (e == cudaSuccess && m_st <= smem_optin) {
        e = cudaFuncSetAttribute(k_st, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(m_st));
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b_st, k_st, kRRTThreads, m_st);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(a.queue, 0, sizeof(int), st);
    if (e == cudaSuccess) {
        const bool staged = b_st >= 1 && b_st >= b_in;
        const int bps = staged ? b_st : b_in;
        if (bps < 1) {
            *msg = "planner kernel cannot be resident";
            return 1;
        }
        const long long want = (a.B + kRRTWarps - 1) / kRRTWarps;
        const int grid = static_cast<int>(std::min<long long>(want, static_cast<long long>(bps) * num_sms));
        (staged ? k_st : k_in)<<<grid, kRRTThreads, staged ? m_st : m_in, st>>>(P, staged ? vst : vin, a, status);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        *msg = cudaGetErrorString(e);
        return 2;
    }
    return 0;
}

}  // namespace vp
