// Batched RRT-Connect (Sec. III-E, "Bringing it Together": one of the two
// planners built on the vectorized primitives), device-resident, in two
// phases:
//
//   1. one warp solves one problem -- both trees in global memory,
//      nearest-node scans over the warp's lanes, every edge checked by the
//      same raked state check as vp_validate_edges -- and takes the next
//      problem from a queue.  A problem still unsolved after its first
//      kPhase1Samples samples is set aside at that sample boundary (its
//      trees stay in global memory; its sample index, tree sizes and tree
//      roles are saved).
//   2. a team of four warps resumes each set-aside problem: warp 0 runs the
//      planner, and every nearest-node scan and edge check is shared by the
//      whole team (the scan's nodes split four ways; each edge state checked
//      by all four warps, each taking a quarter of the self-pair groups and
//      primitive batches, stopping together at the first collision).  The
//      launch's tail -- the few problems that need hundreds of samples --
//      runs on four warps' issue slots instead of one.
//
// Both phases take the same decisions in the same order (the team's scans
// and checks reduce to the same minimum and the same verdicts), so the
// split does not change any result.  The decisions that shape the trees --
// which node is nearest, where the new node lies -- are FP32 with every
// operation rounded on its own (products, sums, differences, one square
// root and one division; no contraction), so a float32 reference taking the
// same steps builds the same trees wherever the edge verdicts agree.
//
// The planner is a state machine with a single call site of the edge check
// (start and goal validity, EXTEND and CONNECT all pass through it), which
// keeps the inlined state check -- most of the code -- to one copy per
// kernel.
#include <cuda_runtime.h>

#include <algorithm>

#include "vp_validate.cuh"

namespace vp {

namespace {

constexpr int kRRTThreads = 128;
constexpr int kRRTWarps = kRRTThreads / 32;
constexpr int kPhase1Samples = 32;  // samples a problem gets in the first phase
enum : int { kTrapped = 0, kAdvanced = 1, kReached = 2 };
enum : int { kCheckStart, kCheckGoal, kExtend, kConnect };
enum : int { kUnsolved = 0, kSolved = 1, kInvalid = -1, kPaused = 2 };

struct RRTArgs {
    const float *start, *goal, *samples;  // [B][D], [B][D], [B][T][D]
    long long B;
    int T, cap;
    float range, res;
    float *nodes;    // [B][2][cap][D] scratch
    int *parent;     // [B][2][cap] scratch
    int *queue;      // problem counter (first phase)
    int *status;     // [B]: 1 solved, 0 not within T samples, -1 start or goal invalid
    int *iters;      // [B]: samples used
    float *path;     // [B][2 cap][D]
    int *path_len;   // [B]
    int *sizes;      // [B][2]
    int *pending;    // [B] problems set aside by the first phase (NULL: no second phase)
    int4 *save;      // [B] (sample index, tree sizes, tree roles) of a set-aside problem
    int *n_pending;  // how many were set aside
    int *queue2;     // problem counter (second phase)
    int t1;          // samples of the first phase
    unsigned long long watchdog_ns;
};

// A node index and the squared distance it was found at.
__device__ __forceinline__ unsigned long long pack_nd(float d2, int i) {
    return (static_cast<unsigned long long>(__float_as_uint(d2)) << 32) | static_cast<unsigned>(i);
}

// The packed (distance, index) minimum of tree nodes i = first, first +
// step, ... < n to the target (nodes [n][D], row-major), per thread.
__device__ __forceinline__ unsigned long long nearest_part(const float *nodes, int n, int D, const float *tgt,
                                                           int first, int step) {
    unsigned long long best = ~0ull;
    for (int i = first; i < n; i += step) {
        const float *x = nodes + static_cast<long long>(i) * D;
        float acc = 0.f;
        for (int d = 0; d < D; ++d) {
            const float dx = __fsub_rn(x[d], tgt[d]);
            acc = __fadd_rn(acc, __fmul_rn(dx, dx));
        }
        const unsigned long long v = pack_nd(acc, i);
        best = v < best ? v : best;
    }
    return best;
}

__device__ __forceinline__ unsigned long long warp_min_u64(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long w = __shfl_xor_sync(kFull, v, o);
        v = w < v ? w : v;
    }
    return v;
}

// Named barriers of the second phase's team (barrier 0 stays with
// __syncthreads): every thread of the block arrives at each, from whichever
// point of the code it has reached.
__device__ __forceinline__ void bar_sync(int id) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(kRRTThreads) : "memory");
}
__device__ __forceinline__ bool bar_or(int id, bool p) {
    unsigned r;
    asm volatile(
        "{\n .reg .pred pi, po;\n setp.ne.u32 pi, %1, 0;\n bar.red.or.pred po, %2, %3, pi;\n selp.u32 %0, 1, 0, po;\n}\n"
        : "=r"(r)
        : "r"(static_cast<unsigned>(p)), "r"(id), "r"(kRRTThreads)
        : "memory");
    return r != 0;
}

// Where one problem's planner stands between calls (a set-aside problem
// resumes from it).
struct PlanState {
    int n[2];        // tree sizes
    int mode, it, ta, t, ia, result, meet;
};

// The planner for problem b, run by one warp from state S until the problem
// is solved (result 1), shown infeasible (-1), out of samples (0) or, with
// it_stop < T, paused at the start of sample it_stop (result kPaused).
// Vectors live in tgt, nea, nw (D floats each, lanes < D write them);
// wq0/wdq receive each edge to check (its start and its difference).
// nearest(tree, n) returns the packed nearest node of tree's first n nodes
// to tgt; check(k) checks the edge in wq0/wdq at k states (true: valid).
template <class NearestF, class CheckF>
__device__ __forceinline__ void plan(const RRTArgs &a, long long b, int D, float *const tn[2], int *const tp[2],
                                     float *tgt, float *nea, float *nw, float *wq0, float *wdq, PlanState &S,
                                     int it_stop, NearestF nearest, CheckF check) {
    const int lane = threadIdx.x & 31;
    const float *start = a.start + b * D, *goal = a.goal + b * D;
    bool done = false;
    while (!done) {
        // ---- what to check: (nea -> nw)
        bool need = true;
        int near = -1, st_ok = kTrapped;
        if (S.mode == kCheckStart || S.mode == kCheckGoal) {
            const float *r = S.mode == kCheckStart ? start : goal;
            if (lane < D) {
                nea[lane] = r[lane];
                nw[lane] = r[lane];
            }
        } else {
            const unsigned long long best = nearest(tn[S.t], S.n[S.t]);
            near = static_cast<int>(best & 0xffffffffu);
            const float d2 = __uint_as_float(static_cast<unsigned>(best >> 32));
            if (lane < D) nea[lane] = tn[S.t][static_cast<long long>(near) * D + lane];
            __syncwarp();
            if (d2 == 0.f) {  // the target is already a node
                need = false;
                st_ok = kReached;
            } else if (S.n[S.t] == a.cap) {
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
            ok = k >= 2 && check(k);
            __syncwarp();
        }
        // ---- act on the outcome
        if (S.mode == kCheckStart || S.mode == kCheckGoal) {
            if (!ok) {
                S.result = kInvalid;
                done = true;
            } else if (S.mode == kCheckStart) {
                S.mode = kCheckGoal;
            } else {
                S.mode = kExtend;
                if (a.T == 0) done = true;
                else if (lane < D) tgt[lane] = a.samples[(b * a.T) * D + lane];
            }
            __syncwarp();
            continue;
        }
        int s = st_ok, inew = near;
        if (need) {
            if (ok) {  // add the new node
                inew = S.n[S.t];
                if (lane < D) tn[S.t][static_cast<long long>(inew) * D + lane] = nw[lane];
                if (lane == 0) tp[S.t][inew] = near;
                ++S.n[S.t];
            } else {
                s = kTrapped;
            }
        }
        __syncwarp();
        bool next = false;
        if (S.mode == kExtend) {
            if (s != kTrapped) {  // connect the other tree toward the new node
                S.ia = inew;
                if (lane < D) tgt[lane] = tn[S.t][static_cast<long long>(inew) * D + lane];
                S.t = 1 - S.ta;
                S.mode = kConnect;
            } else {
                next = true;
            }
        } else {  // connect
            if (s == kReached) {
                S.result = kSolved;
                S.meet = inew;
                done = true;
            } else if (s == kTrapped) {
                next = true;
            }  // advanced: extend again toward the same node
        }
        if (next) {
            ++S.it;
            S.ta = 1 - S.ta;
            if (S.it == a.T) {
                done = true;
            } else if (S.it == it_stop) {  // set aside at a sample boundary
                S.result = kPaused;
                done = true;
            } else {
                S.t = S.ta;
                S.mode = kExtend;
                if (lane < D) tgt[lane] = a.samples[(b * a.T + S.it) * D + lane];
            }
        }
        __syncwarp();
    }
}

// Results of a finished problem: the path start ... goal through the
// meeting node, status, samples used and tree sizes (one warp).
__device__ __forceinline__ void write_result(const RRTArgs &a, long long b, int D, float *const tn[2],
                                             int *const tp[2], const PlanState &S) {
    const int lane = threadIdx.x & 31;
    int plen = 0;
    if (S.result == kSolved && lane == 0) {
        // tree 0 holds the start: its chain from the meeting node, reversed,
        // then tree 1's chain past the meeting node (the same configuration)
        const int tx = 0, ty = 1;
        const int x0 = S.ta == 0 ? S.ia : S.meet, y0 = S.ta == 0 ? S.meet : S.ia;
        int lx = 0;
        for (int i = x0; i >= 0; i = tp[tx][i]) ++lx;
        float *out = a.path + b * 2 * a.cap * D;
        int pos = lx - 1;
        for (int i = x0; i >= 0; i = tp[tx][i], --pos)
            for (int d = 0; d < D; ++d) out[static_cast<long long>(pos) * D + d] = tn[tx][static_cast<long long>(i) * D + d];
        pos = lx;
        for (int i = tp[ty][y0]; i >= 0; i = tp[ty][i], ++pos)
            for (int d = 0; d < D; ++d) out[static_cast<long long>(pos) * D + d] = tn[ty][static_cast<long long>(i) * D + d];
        plen = pos;
    }
    if (lane == 0) {
        a.status[b] = S.result;
        a.iters[b] = S.result == kInvalid ? 0 : (S.result == kSolved ? S.it + 1 : a.T);
        a.path_len[b] = plen;
        a.sizes[2 * b] = S.n[0];
        a.sizes[2 * b + 1] = S.n[1];
    }
    __syncwarp();
}

__device__ __forceinline__ void tree_ptrs(const RRTArgs &a, long long b, int D, float *tn[2], int *tp[2]) {
    tn[0] = a.nodes + (b * 2) * a.cap * D;
    tn[1] = a.nodes + (b * 2 + 1) * a.cap * D;
    tp[0] = a.parent + (b * 2) * a.cap;
    tp[1] = a.parent + (b * 2 + 1) * a.cap;
}

// ---------------------------------------------------------------------------
// first phase: one warp per problem

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
    // the warp's own scan and raked check
    auto nearest = [&](const float *nodes, int n) {
        return warp_min_u64(nearest_part(nodes, n, D, tgt, lane, 32));
    };
    auto check = [&](int k) {
        const int R = (k + 31) >> 5;
        const float inv = __fdiv_rn(1.f, static_cast<float>(k - 1));
        for (int r = 0; r < R; ++r) {
            int i = lane * R + r;
            if (i >= k) i = k - 1;
            const float tt = static_cast<float>(i) * inv;
            const WorkRef<false> w{nullptr, false};
            const bool c = check_state<kFamPoseAll, kStopAny, false, LMAX, SIMPLE>(
                P, [tt, wq0, wdq](int j) { return fmaf(tt, wdq[j], wq0[j]); }, es, stash, Ctl{kFull, false}, w);
            if (__any_sync(kFull, c)) return false;
        }
        return true;
    };
    while (true) {
        int b = 0;
        if (lane == 0) {
            b = (global_ns() - t_start >= a.watchdog_ns) ? -1 : atomicAdd(a.queue, 1);
            if (b < 0) atomicOr(status, VP_DEVERR_TIMEOUT);
        }
        b = __shfl_sync(kFull, b, 0);
        if (b < 0 || b >= a.B) break;
        float *tn[2];
        int *tp[2];
        tree_ptrs(a, b, D, tn, tp);
        if (lane < D) {
            tn[0][lane] = a.start[static_cast<long long>(b) * D + lane];
            tn[1][lane] = a.goal[static_cast<long long>(b) * D + lane];
        }
        if (lane == 0) tp[0][0] = tp[1][0] = -1;
        __syncwarp();
        PlanState S{{1, 1}, kCheckStart, 0, 0, 0, -1, kUnsolved, -1};
        plan(a, b, D, tn, tp, tgt, nea, nw, wq0, wdq, S, a.pending ? a.t1 : a.T, nearest, check);
        if (S.result == kPaused) {  // to the second phase, with what it needs to resume
            if (lane == 0) {
                a.save[b] = make_int4(S.it, S.n[0], S.n[1], S.ta);
                a.pending[atomicAdd(a.n_pending, 1)] = b;
            }
            __syncwarp();
            continue;
        }
        write_result(a, b, D, tn, tp, S);
    }
}

// ---------------------------------------------------------------------------
// second phase: a team of four warps per set-aside problem

enum : int { kOpExit = 0, kOpNearest = 1, kOpCheck = 2 };

// Warp 0 runs the planner; at each nearest-node scan and edge check it
// posts the operation (barrier 1) and does its share beside warps 1-3,
// which do nothing but their shares (a scan ends at barrier 2, each raked
// round of a check at the OR-reduction of barrier 3).  Every thread of the
// block reaches every barrier the same number of times: warps 1-3 leave
// only on the exit operation warp 0 posts once its queue is empty.
template <int LMAX, bool SIMPLE, bool STAGED>
__global__ void VP_VALIDATION_BOUNDS(LMAX, 5)
    rrt_team_kernel(const __grid_constant__ RobotParams P, const EnvView env, const RRTArgs a, unsigned *status) {
    extern __shared__ __align__(16) unsigned char smem[];
    const SmemCarve sc = carve<STAGED>(smem, env, P);
    // target, nearest node, new node, edge start, edge difference
    __shared__ float s_vec[5][16];
    __shared__ const float *s_nodes;
    __shared__ int s_op, s_n, s_k;
    __shared__ volatile int s_flag;
    __shared__ unsigned long long s_best[kRRTWarps];
    if (STAGED && !stage_env(sc.env, env, sc.bar, status)) return;
    const EnvSm es = env_views<STAGED>(sc.env, env);
    const Stash &stash = sc.stash;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int D = P.n_joints;
    float *tgt = s_vec[0], *nea = s_vec[1], *nw = s_vec[2], *q0 = s_vec[3], *dq = s_vec[4];
    const Team team{wib, kRRTWarps, &s_flag};
    // a share of a scan: every thread a strided part of the nodes
    auto scan_part = [&]() {
        const unsigned long long v = warp_min_u64(nearest_part(s_nodes, s_n, D, tgt, threadIdx.x, kRRTThreads));
        if (lane == 0) s_best[wib] = v;
        bar_sync(2);
    };
    // a share of a raked check: every warp the same 32 states, a quarter of
    // the self-pair groups and primitive batches each
    auto check_part = [&]() -> bool {
        const int k = s_k;
        const int R = (k + 31) >> 5;
        const float inv = __fdiv_rn(1.f, static_cast<float>(k - 1));
        for (int r = 0; r < R; ++r) {
            int i = lane * R + r;
            if (i >= k) i = k - 1;
            const float tt = static_cast<float>(i) * inv;
            const WorkRef<false> w{nullptr, false};
            const auto qf = [tt, q0, dq](int j) { return fmaf(tt, dq[j], q0[j]); };
            const bool c = pose_and_check_all<kStopAny, false, LMAX, SIMPLE, decltype(qf), true>(
                P, qf, es, stash, Ctl{kFull, false}, w, team);
            if (bar_or(3, c)) return false;
        }
        return true;
    };
    if (wib != 0) {
        while (true) {
            bar_sync(1);
            const int op = s_op;
            if (op == kOpExit) return;
            if (op == kOpNearest)
                scan_part();
            else
                check_part();
        }
    }
    // warp 0: the planner
    auto nearest = [&](const float *nodes, int n) {
        if (lane == 0) {
            s_nodes = nodes;
            s_n = n;
            s_op = kOpNearest;
        }
        __syncwarp();
        bar_sync(1);
        scan_part();
        unsigned long long v = s_best[0];
        for (int w2 = 1; w2 < kRRTWarps; ++w2) v = s_best[w2] < v ? s_best[w2] : v;
        return v;
    };
    auto check = [&](int k) {
        if (lane == 0) {
            s_k = k;
            s_flag = 0;
            s_op = kOpCheck;
        }
        __syncwarp();
        bar_sync(1);
        return check_part();
    };
    const uint64_t t_start = global_ns();
    while (true) {
        int idx = 0;
        if (lane == 0) {
            idx = (global_ns() - t_start >= a.watchdog_ns) ? -1 : atomicAdd(a.queue2, 1);
            if (idx < 0) atomicOr(status, VP_DEVERR_TIMEOUT);
        }
        idx = __shfl_sync(kFull, idx, 0);
        if (idx < 0 || idx >= *a.n_pending) break;
        const long long b = a.pending[idx];
        float *tn[2];
        int *tp[2];
        tree_ptrs(a, b, D, tn, tp);
        const int4 sv = a.save[b];  // (sample index, tree sizes, tree roles)
        PlanState S{{sv.y, sv.z}, kExtend, sv.x, sv.w, sv.w, -1, kUnsolved, -1};
        if (lane < D) tgt[lane] = a.samples[(b * a.T + S.it) * D + lane];
        __syncwarp();
        plan(a, b, D, tn, tp, tgt, nea, nw, q0, dq, S, a.T, nearest, check);
        write_result(a, b, D, tn, tp, S);
    }
    if (lane == 0) s_op = kOpExit;
    __syncwarp();
    bar_sync(1);
}

using RRTKernel = void (*)(RobotParams, EnvView, RRTArgs, unsigned *);

template <int LMAX, bool TEAM>
RRTKernel rrt_instance(bool simple, bool staged) {
    if (TEAM) {
        if (simple) return staged ? rrt_team_kernel<LMAX, true, true> : rrt_team_kernel<LMAX, true, false>;
        return staged ? rrt_team_kernel<LMAX, false, true> : rrt_team_kernel<LMAX, false, false>;
    }
    if (simple) return staged ? rrt_connect_kernel<LMAX, true, true> : rrt_connect_kernel<LMAX, true, false>;
    return staged ? rrt_connect_kernel<LMAX, false, true> : rrt_connect_kernel<LMAX, false, false>;
}

template <bool TEAM>
RRTKernel rrt_kernel_for(int lmax, bool simple, bool staged) {
    switch (lmax) {
        case 8: return rrt_instance<8, TEAM>(simple, staged);
        case 9: return rrt_instance<9, TEAM>(simple, staged);
        case 15: return rrt_instance<15, TEAM>(simple, staged);
        default: return rrt_instance<17, TEAM>(simple, staged);
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
    a.queue = L.counters;
    a.n_pending = L.counters + 1;
    a.queue2 = L.counters + 2;
    a.status = L.status;
    a.iters = L.iters;
    a.path = L.path;
    a.path_len = L.path_len;
    a.sizes = L.sizes;
    // a second phase only when a problem can outlast the first one's samples
    const bool two = L.T > kPhase1Samples;
    a.pending = two ? L.pending : nullptr;
    a.save = two ? L.save : nullptr;
    a.t1 = kPhase1Samples;
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
    cudaError_t e = cudaMemsetAsync(L.counters, 0, 3 * sizeof(int), st);
    for (int phase = 0; phase < (two ? 2 : 1) && e == cudaSuccess; ++phase) {
        const RRTKernel k_in = phase ? rrt_kernel_for<true>(lmax, simple, false) : rrt_kernel_for<false>(lmax, simple, false);
        const RRTKernel k_st = phase ? rrt_kernel_for<true>(lmax, simple, true) : rrt_kernel_for<false>(lmax, simple, true);
        e = cudaFuncSetAttribute(k_in, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(m_in));
        int b_in = 0, b_st = 0;
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b_in, k_in, kRRTThreads, m_in);
        if (e == cudaSuccess && m_st <= smem_optin) {
            e = cudaFuncSetAttribute(k_st, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(m_st));
            if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b_st, k_st, kRRTThreads, m_st);
        }
        if (e != cudaSuccess) break;
        const bool staged = b_st >= 1 && b_st >= b_in;
        const int bps = staged ? b_st : b_in;
        if (bps < 1) {
            *msg = "planner kernel cannot be resident";
            return 1;
        }
        // first phase: a warp per problem; second: a block per set-aside
        // problem (as many blocks as can be resident; idle ones exit at once)
        const long long want = phase ? a.B : (a.B + kRRTWarps - 1) / kRRTWarps;
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
