// Batched edge validation for batches of uneven edge lengths.
//
// 1. bucket_count_kernel: state count k_e of every edge (explicit or from the
//    resolution), bucket = ceil(log2 k) class ([2,4], [5,8], ..., [257,512],
//    >512), block-aggregated histogram.  Malformed edges are answered here.
// 2. bucket_scatter_kernel: a permutation listing edges bucket by bucket,
//    longest bucket first (longest-processing-time order for the queue).
// 3. edges_batched_kernel: persistent; each warp pops work items from one
//    global counter.  A work item of bucket b packs 32/G_b edges into lane
//    groups of G_b lanes; the groups run the raked check in lockstep and the
//    warp leaves a state as soon as every group has a collision or is done.
// The three launches (plus the counter reset) are captured once into a CUDA
// graph per buffer set and replayed.  G_b comes from the autotuner, which
// times each bucket alone, at full occupancy, with every group size and keeps
// the fastest (cached per robot, environment and length profile).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "vp_batched.h"
#include "vp_device.cuh"
#include "vp_internal.h"

namespace vp {

namespace {

constexpr int kNB = 9;           // length buckets
constexpr int kBlock = 128;      // threads per block of the persistent kernel
constexpr int kCtrlHist = 0;     // ctrl[0..8]   edges per bucket
constexpr int kCtrlCursor = 16;  // ctrl[16..24] scatter cursors
constexpr int kCtrlQueue = 32;   // ctrl[32]     work-item counter
constexpr int kCtrlInts = 64;

struct BatchPlan {
    int G[kNB];            // lanes per edge, per bucket
    int edge_lo[kNB], edge_hi[kNB];  // bucket b's edges are perm[edge_lo[b], edge_hi[b]) (when !from_hist)
    int from_hist;         // 1: offsets from the histogram in ctrl (longest bucket first)
    unsigned long long watchdog_ns;  // time budget of one launch
};

__host__ __device__ __forceinline__ int bucket_of(int k) {
    // ceil(log2 k) - 2, clamped: [2,4] -> 0, [5,8] -> 1, ..., [257,512] -> 7, > 512 -> 8
    int c = 0;
    unsigned v = static_cast<unsigned>(k - 1);
    while (v) {
        ++c;
        v >>= 1;
    }
    return min(max(c - 2, 0), kNB - 1);
}

// Exclusive offsets of the buckets in processing order (longest first).
__device__ __forceinline__ void offsets_from_hist(const int *hist, int *off) {
    int acc = 0;
    for (int b = kNB - 1; b >= 0; --b) {
        off[b] = acc;
        acc += hist[b];
    }
    off[kNB] = acc;  // total; off[b] + hist[b] is bucket b's end
}

__device__ __forceinline__ int count_from_dmax_b(float dmax, float res) {
    const float steps = ceilf(__fdiv_rn(dmax, res));
    if (!(steps <= static_cast<float>(VP_MAX_STEPS))) return -1;
    return max(2, static_cast<int>(steps) + 1);
}

__global__ void bucket_count_kernel(const int D, const float *__restrict__ q0, const float *__restrict__ q1,
                                    const int32_t *__restrict__ counts, const float res, const long long E,
                                    int32_t *__restrict__ kbuf, uint8_t *__restrict__ valid, unsigned *status,
                                    int *ctrl) {
    __shared__ int hist[kNB];
    if (threadIdx.x < kNB) hist[threadIdx.x] = 0;
    __syncthreads();
    const long long e = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e < E) {
        float dmax = 0.f;
        bool fin = true;
        for (int j = 0; j < D; ++j) {
            const float a = q0[e * D + j], b = q1[e * D + j];
            fin &= isfinite(a) && isfinite(b);
            if (fin) dmax = fmaxf(dmax, fabsf(b - a));
        }
        int k = -1;
        if (counts != nullptr) {
            k = counts[e];
            if (k < 2) {
                atomicOr(status, VP_DEVERR_COUNT);
                k = -1;
            }
        } else if (fin) {
            k = count_from_dmax_b(dmax, res);
            if (k < 0) atomicOr(status, VP_DEVERR_LENGTH);
        }
        if (!fin) k = -1;
        kbuf[e] = k;
        if (k < 0)
            valid[e] = 0;
        else
            atomicAdd(&hist[bucket_of(k)], 1);
    }
    __syncthreads();
    if (threadIdx.x < kNB && hist[threadIdx.x]) atomicAdd(&ctrl[kCtrlHist + threadIdx.x], hist[threadIdx.x]);
}

__global__ void bucket_scatter_kernel(const long long E, const int32_t *__restrict__ kbuf,
                                      int2 *__restrict__ perm, int *ctrl) {
    __shared__ int cnt[kNB], base[kNB], off[kNB + 1];
    if (threadIdx.x == 0) offsets_from_hist(ctrl + kCtrlHist, off);
    if (threadIdx.x < kNB) cnt[threadIdx.x] = 0;
    __syncthreads();
    const long long e = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    int b = -1, r = 0, k = 0;
    if (e < E) {
        k = kbuf[e];
        if (k >= 2) {
            b = bucket_of(k);
            r = atomicAdd(&cnt[b], 1);
        }
    }
    __syncthreads();
    if (threadIdx.x < kNB && cnt[threadIdx.x])
        base[threadIdx.x] = atomicAdd(&ctrl[kCtrlCursor + threadIdx.x], cnt[threadIdx.x]);
    __syncthreads();
    if (b >= 0) perm[off[b] + base[b] + r] = make_int2(static_cast<int>(e), k);
}

// Persistent validation of bucketed edges; see the file comment.  STATS adds
// the work counters (VP_WORK_*) of the lanes that hold a state of a live edge.
template <bool STATS, int LMAX, bool SIMPLE>
__global__ void VP_VALIDATION_BOUNDS(LMAX, 6) edges_batched_kernel(
    const __grid_constant__ RobotParams P, const EnvView env, const float *__restrict__ q0,
    const float *__restrict__ q1, const int2 *__restrict__ perm, const BatchPlan plan, uint8_t *__restrict__ valid,
    unsigned *status, int *ctrl, unsigned long long *work) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_edge_lo[kNB], s_edge_hi[kNB], s_item_end[kNB];
    __shared__ int s_items;
    size_t off = static_cast<size_t>(env.n_float4) * 16;
    float4 *env_sm = reinterpret_cast<float4 *>(smem);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + off);
    off += 16;
    float *gbuf = reinterpret_cast<float *>(smem + off);  // [warps][8 groups][32]
    off += static_cast<size_t>(kBlock / 32) * 8 * 32 * sizeof(float);
    Stash stash;
    stash.frames = nullptr;
    stash.centres = reinterpret_cast<float *>(smem + off);
    off += static_cast<size_t>(P.n_links) * kCentreFloats * kBlock * sizeof(float);
    stash.motion = reinterpret_cast<float *>(smem + off);
    stash.stride = kBlock;

    if (threadIdx.x == 0) {
        int eo[kNB + 1];
        if (plan.from_hist) {
            offsets_from_hist(ctrl + kCtrlHist, eo);
            for (int b = 0; b < kNB; ++b) {
                s_edge_lo[b] = eo[b];
                s_edge_hi[b] = eo[b] + ctrl[kCtrlHist + b];
            }
        } else {
            for (int b = 0; b < kNB; ++b) {
                s_edge_lo[b] = plan.edge_lo[b];
                s_edge_hi[b] = plan.edge_hi[b];
            }
        }
        // work items in processing order: longest bucket first
        int items = 0;
        for (int b = kNB - 1; b >= 0; --b) {
            const int per = 32 / plan.G[b];
            items += max(0, s_edge_hi[b] - s_edge_lo[b] + per - 1) / per;
            s_item_end[b] = items;
        }
        s_items = items;
    }
    __syncthreads();
    if (!stage_env(env_sm, env.data, env.n_float4, bar, status)) return;
    const EnvSm es = env_in_smem(env_sm, env);
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int D = P.n_joints;
    float *wbuf = gbuf + wib * 8 * 32;
    const uint64_t t_start = global_ns();
    Work wk;
    if (STATS) {
#pragma unroll
        for (int i = 0; i < VP_WORK_N; ++i) wk.v[i] = 0;
    }

    while (true) {
        int item = 0;
        if (lane == 0) {
            if (global_ns() - t_start >= plan.watchdog_ns) {
                atomicOr(status, VP_DEVERR_TIMEOUT);
                item = -1;
            } else {
                item = atomicAdd(&ctrl[kCtrlQueue], 1);
            }
        }
        item = __shfl_sync(kFull, item, 0);
        if (item < 0 || item >= s_items) break;
        int b = kNB - 1;
        while (b > 0 && item >= s_item_end[b]) --b;
        const int first_item = (b == kNB - 1) ? 0 : s_item_end[b + 1];
        const int G = plan.G[b];
        const int per = 32 / G;
        const int g = lane / G, j = lane - g * G;
        const unsigned gmask = G == 32 ? kFull : (((1u << G) - 1u) << (g * G));
        const int slot = s_edge_lo[b] + (item - first_item) * per + g;
        const bool has_edge = g < per && slot < s_edge_hi[b];
        const int2 ek = has_edge ? perm[slot] : make_int2(0, 2);
        const int e = ek.x, k = ek.y;
        float *gq0 = wbuf + g * 32, *gdq = gq0 + 16;
        __syncwarp();
        if (has_edge) {
            for (int d = j; d < D; d += G) {
                const float a = q0[static_cast<long long>(e) * D + d];
                gq0[d] = a;
                gdq[d] = q1[static_cast<long long>(e) * D + d] - a;
            }
        } else {
            for (int d = j; d < 16; d += G) {
                gq0[d] = 0.f;
                gdq[d] = 0.f;
            }
        }
        __syncwarp();
        const int R = (k + G - 1) / G;
        const float inv = __fdiv_rn(1.f, static_cast<float>(k - 1));
        const int R_max = __reduce_max_sync(kFull, has_edge ? R : 0);
        bool done = !has_edge;
        for (int r = 0; r < R_max; ++r) {
            int i = j * R + r;
            const WorkRef<STATS> w{&wk, !done && i < k};
            if (i >= k) i = k - 1;
            const float t = static_cast<float>(i) * inv;
            const bool c = pose_and_check<kStopGroups, STATS, LMAX, SIMPLE>(
                P, [t, gq0, gdq](int jj) { return fmaf(t, gdq[jj], gq0[jj]); }, es, stash, Ctl{gmask, done}, w);
            const bool gcol = (__ballot_sync(kFull, c && !done) & gmask) != 0u;
            if (!done && (gcol || r == R - 1)) {
                if (j == 0) {
                    valid[e] = gcol ? 0 : 1;
                    if (STATS) wk.v[VP_WORK_EDGES_DONE] += 1;
                }
                done = true;
            }
            if (__all_sync(kFull, done)) break;
        }
        if constexpr (STATS) {
#pragma unroll
            for (int c = 0; c < VP_WORK_N; ++c) {
                const unsigned sum = __reduce_add_sync(kFull, wk.v[c]);
                if (lane == 0 && sum) atomicAdd(work + c, static_cast<unsigned long long>(sum));
                wk.v[c] = 0;
            }
        }
    }
}

size_t batched_smem(const EnvView &env, const RobotParams &P) {
    return static_cast<size_t>(env.n_float4) * 16 + 16 + static_cast<size_t>(kBlock / 32) * 8 * 32 * sizeof(float) +
           static_cast<size_t>(P.n_links * kCentreFloats + P.n_joints * 2) * kBlock * sizeof(float);
}

// The kernel instance for this robot's link count and counting mode.
using BatchedKernel = void (*)(const RobotParams, const EnvView, const float *, const float *, const int2 *,
                               const BatchPlan, uint8_t *, unsigned *, int *, unsigned long long *);
template <int LMAX>
BatchedKernel batched_instance(bool stats, bool simple) {
    if (stats) return edges_batched_kernel<true, LMAX, false>;
    return simple ? edges_batched_kernel<false, LMAX, true> : edges_batched_kernel<false, LMAX, false>;
}

BatchedKernel batched_kernel_for(const RobotParams &P, bool stats) {
    const bool simple = P.simple != 0;
    switch (lmax_for(P.n_links)) {
        case 8: return batched_instance<8>(stats, simple);
        case 9: return batched_instance<9>(stats, simple);
        case 15: return batched_instance<15>(stats, simple);
        default: return batched_instance<17>(stats, simple);
    }
}

// ---------------------------------------------------------------------------
// host side

struct TuneKey {
    std::vector<unsigned char> robot;
    int ns, nc, nb, sms;
    std::vector<int> profile;  // length histogram, coarse
    bool operator<(const TuneKey &o) const {
        return std::tie(robot, ns, nc, nb, sms, profile) < std::tie(o.robot, o.ns, o.nc, o.nb, o.sms, o.profile);
    }
};

std::mutex g_tune_mutex;
std::map<TuneKey, std::vector<int>> g_tune_cache;

struct Impl {
    int32_t *kbuf = nullptr;  // state count per edge (-1: answered in the bucketing pass)
    int2 *perm = nullptr;     // (edge, count) bucket by bucket, longest bucket first
    int *ctrl = nullptr;
    int64_t cap = 0;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t exec = nullptr;
    // graph key
    const void *k_q0 = nullptr, *k_q1 = nullptr, *k_counts = nullptr, *k_valid = nullptr;
    const void *k_ev = nullptr;
    unsigned long long k_watchdog = 0;
    int64_t k_E = -1;
    float k_res = 0.f;
    int G[kNB] = {4, 8, 16, 32, 32, 32, 32, 32, 32};
    bool tuned = false;
};

Impl *impl_of(BatchedState &st) {
    if (!st.impl) st.impl = new Impl();
    return static_cast<Impl *>(st.impl);
}

void drop_graph(Impl *im) {
    if (im->exec) cudaGraphExecDestroy(im->exec);
    im->exec = nullptr;
    im->k_E = -1;
}

int set_err(std::string *msg, const char *what, cudaError_t e) {
    *msg = std::string(what) + ": " + cudaGetErrorString(e);
    return 2;
}

int ensure_capacity(Impl *im, int64_t E, std::string *msg) {
    if (!im->ctrl) {
        cudaError_t e = cudaMalloc(&im->ctrl, kCtrlInts * sizeof(int));
        if (e != cudaSuccess) return set_err(msg, "cudaMalloc ctrl", e);
    }
    if (!im->cap_stream) {
        cudaError_t e = cudaStreamCreateWithFlags(&im->cap_stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return set_err(msg, "cudaStreamCreate", e);
    }
    if (E <= im->cap) return 0;
    drop_graph(im);
    if (im->kbuf) cudaFree(im->kbuf);
    if (im->perm) cudaFree(im->perm);
    im->kbuf = nullptr;
    im->perm = nullptr;
    im->cap = 0;
    const int64_t n = std::max<int64_t>(E, 1 << 16);
    cudaError_t e = cudaMalloc(&im->kbuf, n * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc(&im->perm, n * sizeof(int2));
    if (e != cudaSuccess) return set_err(msg, "cudaMalloc scratch", e);
    im->cap = n;
    return 0;
}

int prepare_kernel(const BatchedArgs &a, size_t *smem, int *grid, std::string *msg) {
    *smem = batched_smem(*a.env, *a.robot);
    if (*smem > a.smem_optin) {
        *msg = "environment and frame stash exceed shared memory";
        return 1;
    }
    const BatchedKernel k0 = batched_kernel_for(*a.robot, false), k1 = batched_kernel_for(*a.robot, true);
    cudaError_t e = cudaFuncSetAttribute(k0, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(*smem));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k1, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(*smem));
    int bps = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k0, kBlock, *smem);
    if (e != cudaSuccess) return set_err(msg, "batched kernel attributes", e);
    if (bps < 1) {
        *msg = "batched kernel cannot be resident";
        return 1;
    }
    *grid = bps * a.num_sms;
    return 0;
}

// Enqueue the whole pipeline on stream s (also used under capture).
cudaError_t enqueue(Impl *im, const BatchedArgs &a, const BatchPlan &plan, size_t smem, int grid, cudaStream_t s,
                    uint8_t *valid, unsigned long long *work = nullptr) {
    const int D = a.robot->n_joints;
    cudaError_t e = cudaMemsetAsync(im->ctrl, 0, kCtrlInts * sizeof(int), s);
    if (e != cudaSuccess) return e;
    const unsigned nb = static_cast<unsigned>((a.E + 255) / 256);
    bucket_count_kernel<<<nb, 256, 0, s>>>(D, a.q0, a.q1, a.counts, a.res, a.E, im->kbuf, valid, a.status, im->ctrl);
    bucket_scatter_kernel<<<nb, 256, 0, s>>>(a.E, im->kbuf, im->perm, im->ctrl);
    // external event-record nodes, so the events time the kernel when replayed from the graph
    if (a.ev_start) e = cudaEventRecordWithFlags(a.ev_start, s, cudaEventRecordExternal);
    if (e != cudaSuccess) return e;
    batched_kernel_for(*a.robot, work != nullptr)<<<grid, kBlock, smem, s>>>(*a.robot, *a.env, a.q0, a.q1, im->perm,
                                                                            plan, valid, a.status, im->ctrl, work);
    e = cudaGetLastError();
    if (e == cudaSuccess && a.ev_stop) e = cudaEventRecordWithFlags(a.ev_stop, s, cudaEventRecordExternal);
    return e;
}

// Host mirror of offsets_from_hist.
void offsets_host(const int *hist, int *off) {
    int acc = 0;
    for (int b = kNB - 1; b >= 0; --b) {
        off[b] = acc;
        acc += hist[b];
    }
    off[kNB] = acc;
}

BatchPlan plan_from(const Impl *im, unsigned long long watchdog_ns) {
    BatchPlan p;
    std::memset(&p, 0, sizeof(p));
    for (int b = 0; b < kNB; ++b) p.G[b] = im->G[b];
    p.from_hist = 1;
    p.watchdog_ns = watchdog_ns;
    return p;
}

}  // namespace

int batched_validate(BatchedState &st, const BatchedArgs &a, std::string *msg) {
    Impl *im = impl_of(st);
    int rc = ensure_capacity(im, a.E, msg);
    if (rc) return rc;
    size_t smem = 0;
    int grid = 0;
    rc = prepare_kernel(a, &smem, &grid, msg);
    if (rc) return rc;
    const bool same = im->exec && im->k_q0 == a.q0 && im->k_q1 == a.q1 && im->k_counts == a.counts &&
                      im->k_valid == a.valid && im->k_E == a.E && im->k_res == a.res && im->k_ev == a.ev_start &&
                      im->k_watchdog == st.watchdog_ns;
    if (!same) {
        drop_graph(im);
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(im->cap_stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return set_err(msg, "begin capture", e);
        cudaError_t e2 = enqueue(im, a, plan_from(im, st.watchdog_ns), smem, grid, im->cap_stream, a.valid);
        e = cudaStreamEndCapture(im->cap_stream, &graph);
        if (e2 != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return set_err(msg, "capture", e2);
        }
        if (e != cudaSuccess) return set_err(msg, "end capture", e);
        e = cudaGraphInstantiate(&im->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            im->exec = nullptr;
            return set_err(msg, "instantiate", e);
        }
        im->k_q0 = a.q0;
        im->k_q1 = a.q1;
        im->k_counts = a.counts;
        im->k_valid = a.valid;
        im->k_E = a.E;
        im->k_res = a.res;
        im->k_ev = a.ev_start;
        im->k_watchdog = st.watchdog_ns;
    }
    cudaError_t e = cudaGraphLaunch(im->exec, a.stream);
    return e == cudaSuccess ? 0 : set_err(msg, "graph launch", e);
}

int batched_work(BatchedState &st, const BatchedArgs &a, unsigned long long *work, std::string *msg) {
    Impl *im = impl_of(st);
    int rc = ensure_capacity(im, a.E, msg);
    if (rc) return rc;
    size_t smem = 0;
    int grid = 0;
    rc = prepare_kernel(a, &smem, &grid, msg);
    if (rc) return rc;
    const cudaError_t e = enqueue(im, a, plan_from(im, st.watchdog_ns), smem, grid, a.stream, a.valid, work);
    return e == cudaSuccess ? 0 : set_err(msg, "batched work", e);
}

// Tiling choice by coordinate descent on whole launches of the batch itself
// (its first 2^23 edges at most).  The batch's own size matters: the launch
// cannot end before its slowest work item, and an item of long edges at few
// lanes per edge runs many rounds in series, so a tiling that is best for a
// large batch can be worst for a small one.  The batch is bucketed once;
// then, in order of each bucket's share of the states, every lane-group size
// is tried for that bucket with the other buckets' choices held, timing the
// whole launch (all buckets back to back on one queue).  A bucket moves off
// its current size only for a 1% gain, so noise does not churn the choice;
// passes repeat (at most three) until none moves.
int batched_autotune(BatchedState &st, const BatchedArgs &a, std::string *msg) {
    Impl *im = impl_of(st);
    size_t smem = 0;
    int grid = 0;
    int rc = prepare_kernel(a, &smem, &grid, msg);
    if (rc) return rc;
    const int64_t S = std::min<int64_t>(a.E, int64_t{1} << 23);
    rc = ensure_capacity(im, S, msg);
    if (rc) return rc;
    cudaStream_t s = a.stream;
    uint8_t *tv = nullptr;
    cudaError_t e = cudaMalloc(&tv, S);
    if (e != cudaSuccess) return set_err(msg, "cudaMalloc tuning output", e);
    const unsigned nb = static_cast<unsigned>((S + 255) / 256);
    e = cudaMemsetAsync(im->ctrl, 0, kCtrlInts * sizeof(int), s);
    if (e == cudaSuccess) {
        bucket_count_kernel<<<nb, 256, 0, s>>>(a.robot->n_joints, a.q0, a.q1, a.counts, a.res, S, im->kbuf, tv,
                                               a.status, im->ctrl);
        bucket_scatter_kernel<<<nb, 256, 0, s>>>(S, im->kbuf, im->perm, im->ctrl);
        e = cudaGetLastError();
    }
    int hist[kNB] = {0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(hist, im->ctrl + kCtrlHist, sizeof(hist), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaFree(tv);
        return set_err(msg, "tuning bucket pass", e);
    }
    TuneKey key;
    key.robot.assign(reinterpret_cast<const unsigned char *>(a.robot),
                     reinterpret_cast<const unsigned char *>(a.robot) + sizeof(RobotParams));
    key.ns = a.env->ns;
    key.nc = a.env->nc;
    key.nb = a.env->nb;
    key.sms = a.num_sms;
    for (int b = 0; b < kNB; ++b)
        key.profile.push_back(hist[b] == 0 ? 0 : 1 + static_cast<int>((20 * static_cast<int64_t>(hist[b])) / S));
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            for (int b = 0; b < kNB; ++b) im->G[b] = it->second[b];
            im->tuned = true;
            drop_graph(im);
            cudaFree(tv);
            return 0;
        }
    }
    BatchPlan p;
    std::memset(&p, 0, sizeof(p));
    {
        int off[kNB + 1];
        offsets_host(hist, off);
        for (int b = 0; b < kNB; ++b) {
            p.edge_lo[b] = off[b];
            p.edge_hi[b] = off[b] + hist[b];
        }
    }
    p.from_hist = 0;
    p.watchdog_ns = st.watchdog_ns;
    const int defaults[kNB] = {4, 8, 16, 32, 32, 32, 32, 32, 32};
    for (int b = 0; b < kNB; ++b) p.G[b] = defaults[b];
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&t0);
    if (e == cudaSuccess) e = cudaEventCreate(&t1);
    // one timing: the best of two runs of the whole sample
    auto time_plan = [&](float *ms_out) {
        float best = 1e30f;
        for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
            e = cudaMemsetAsync(im->ctrl + kCtrlQueue, 0, sizeof(int), s);
            if (e != cudaSuccess) break;
            cudaEventRecord(t0, s);
            batched_kernel_for(*a.robot, false)<<<grid, kBlock, smem, s>>>(*a.robot, *a.env, a.q0, a.q1, im->perm,
                                                                           p, tv, a.status, im->ctrl, nullptr);
            cudaEventRecord(t1, s);
            e = cudaEventSynchronize(t1);
            if (e == cudaSuccess) e = cudaGetLastError();
            float ms = 0.f;
            if (e == cudaSuccess) cudaEventElapsedTime(&ms, t0, t1);
            best = std::min(best, ms);
        }
        *ms_out = best;
    };
    // buckets by their (approximate) share of the sample's states, largest first
    int order[kNB];
    for (int b = 0; b < kNB; ++b) order[b] = b;
    std::stable_sort(order, order + kNB, [&](int x, int y) {
        return static_cast<double>(hist[x]) * (1 << x) > static_cast<double>(hist[y]) * (1 << y);
    });
    float cur = 0.f;
    time_plan(&cur);  // warm-up
    time_plan(&cur);
    const int options[4] = {4, 8, 16, 32};
    bool moved = true;
    for (int pass = 0; pass < 3 && moved && e == cudaSuccess; ++pass) {
        moved = false;
        for (int oi = 0; oi < kNB && e == cudaSuccess; ++oi) {
            const int b = order[oi];
            if (hist[b] < 64) continue;  // too few to matter: keep the default
            const int keep = p.G[b];
            int best_g = keep;
            float best = cur;
            for (int G : options) {
                if (G == keep || e != cudaSuccess) continue;
                p.G[b] = G;
                float ms = 0.f;
                time_plan(&ms);
                if (ms < 0.99f * best) {
                    best = ms;
                    best_g = G;
                }
            }
            p.G[b] = best_g;
            moved = moved || best_g != keep;
            cur = best;
        }
    }
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    cudaFree(tv);
    if (e != cudaSuccess) return set_err(msg, "tuning runs", e);
    for (int b = 0; b < kNB; ++b) im->G[b] = p.G[b];
    im->tuned = true;
    drop_graph(im);
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        g_tune_cache[key] = std::vector<int>(im->G, im->G + kNB);
    }
    return 0;
}

void batched_invalidate(BatchedState &st) {
    if (!st.impl) return;
    Impl *im = static_cast<Impl *>(st.impl);
    drop_graph(im);
    im->tuned = false;
    const int defaults[kNB] = {4, 8, 16, 32, 32, 32, 32, 32, 32};
    for (int b = 0; b < kNB; ++b) im->G[b] = defaults[b];
}

void batched_release(BatchedState &st) {
    if (!st.impl) return;
    Impl *im = static_cast<Impl *>(st.impl);
    drop_graph(im);
    if (im->kbuf) cudaFree(im->kbuf);
    if (im->perm) cudaFree(im->perm);
    if (im->ctrl) cudaFree(im->ctrl);
    if (im->cap_stream) cudaStreamDestroy(im->cap_stream);
    delete im;
    st.impl = nullptr;
}

void batched_set_tiling(BatchedState &st, const int *G, int n) {
    Impl *im = impl_of(st);
    for (int b = 0; b < n && b < kNB; ++b) im->G[b] = G[b];
    im->tuned = true;
    drop_graph(im);
}

int batched_tiling(const BatchedState &st, int *G, int n) {
    const Impl *im = static_cast<const Impl *>(st.impl);
    const int defaults[kNB] = {4, 8, 16, 32, 32, 32, 32, 32, 32};
    for (int b = 0; b < n && b < kNB; ++b) G[b] = im ? im->G[b] : defaults[b];
    return kNB;
}

}  // namespace vp
