// Batched edge validation for batches of uneven edge lengths.
//
// 1. bucket_count_kernel: state count k_e of every edge (explicit or from the
//    resolution), bucket = ceil(log2 k) class ([2,4], [5,8], ..., [257,512],
//    >512), block-aggregated histogram.  Malformed counts (and, without
//    explicit counts, non-finite or over-long edges) are answered here; with
//    explicit counts the endpoints are read only once, by the edge kernel,
//    which answers a non-finite endpoint.
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
#include "vp_validate.cuh"

namespace vp {

namespace {

__global__ void bucket_count_kernel(const int D, const float *__restrict__ q0, const float *__restrict__ q1,
                                    const int32_t *__restrict__ counts, const float res, const long long E,
                                    int32_t *__restrict__ kbuf, uint8_t *__restrict__ valid, unsigned *status,
                                    int *ctrl) {
    __shared__ int hist[kNB];
    if (threadIdx.x < kNB) hist[threadIdx.x] = 0;
    __syncthreads();
    const long long e = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (e < E) {
        int k = -1;
        if (counts != nullptr) {
            // explicit counts: the endpoints are not read here (the edge
            // kernel checks that they are finite as it loads them)
            k = counts[e];
            if (k < 2) {
                atomicOr(status, VP_DEVERR_COUNT);
                k = -1;
            } else if (k > VP_MAX_STEPS + 1) {
                atomicOr(status, VP_DEVERR_LENGTH);
                k = -1;
            }
        } else {
            float dmax = 0.f;
            bool fin = true;
            for (int j = 0; j < D; ++j) {
                const float a = q0[e * D + j], b = q1[e * D + j];
                fin &= isfinite(a) && isfinite(b);
                if (fin) dmax = fmaxf(dmax, fabsf(b - a));
            }
            if (fin) {
                k = count_from_dmax(dmax, res);
                if (k < 0) atomicOr(status, VP_DEVERR_LENGTH);
            }
        }
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

BatchedKernel batched_kernel_for(const RobotParams &P, bool stats, bool staged, int order) {
    return kernel_set(lmax_for(P.n_links)).batched[family_of(order)][stats][P.simple != 0][staged];
}

SurvivorsKernel survivors_kernel_for(const RobotParams &P, bool stats, bool staged, int order) {
    return kernel_set(lmax_for(P.n_links)).survivors[family_of(order)][stats][P.simple != 0][staged];
}

size_t batched_smem(const EnvView &env, const RobotParams &P) {
    return env_smem_bytes(env) + 16 + static_cast<size_t>(kBlock / 32) * 8 * 32 * sizeof(float) +
           static_cast<size_t>(stash_floats(P.n_links)) * kBlock * sizeof(float);
}

// ---------------------------------------------------------------------------
// host side

struct TuneKey {
    std::vector<unsigned char> robot;
    int ns, nc, nb, sms;
    uint64_t env;              // contents of the environment: placement changes the best choice
    std::vector<int> profile;  // length histogram, coarse
    bool operator<(const TuneKey &o) const {
        return std::tie(robot, ns, nc, nb, sms, env, profile) <
               std::tie(o.robot, o.ns, o.nc, o.nb, o.sms, o.env, o.profile);
    }
};

std::mutex g_tune_mutex;
std::map<TuneKey, std::vector<int>> g_tune_cache;

struct Impl {
    int32_t *kbuf = nullptr;  // state count per edge (-1: answered in the bucketing pass)
    int2 *perm = nullptr;     // (edge, count) bucket by bucket, longest bucket first
    int2 *surv = nullptr;     // (edge, count) of the edges left to the second phase
    int2 *defer = nullptr;    // (edge, count) a two-pass order's first pass deferred, in perm's bucket ranges
    int *ctrl = nullptr;
    int64_t cap = 0;
    cudaStream_t cap_stream = nullptr;
    // replayable graphs, one per buffer set (a batch validated in chunks has
    // one per chunk), least recently used first out
    struct Graph {
        cudaGraphExec_t exec = nullptr;
        const void *q0 = nullptr, *q1 = nullptr, *counts = nullptr, *valid = nullptr, *ev = nullptr;
        unsigned long long watchdog = 0;
        int64_t E = -1;
        float res = 0.f;
        uint64_t used = 0;
    };
    std::vector<Graph> graphs;
    uint64_t clock = 0;
    int G[kNB] = {4, 8, 16, 32, 32, 32, 32, 32, 32};
    int screen_rounds = kDefaultScreenRounds;
    int order = 0;  // check order (kOrder* bits)
    bool tuned = false;
    uint64_t epoch = 0;          // graphs dropped so far (any change of robot, environment or tuning)
    uint64_t mirrored = ~0ull;   // the source's epoch this state last copied (batched_mirror)
};

Impl *impl_of(BatchedState &st) {
    if (!st.impl) st.impl = new Impl();
    return static_cast<Impl *>(st.impl);
}

constexpr size_t kMaxGraphs = 16;

void drop_graph(Impl *im) {
    for (auto &g : im->graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    im->graphs.clear();
    ++im->epoch;
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
    if (im->surv) cudaFree(im->surv);
    if (im->defer) cudaFree(im->defer);
    im->kbuf = nullptr;
    im->perm = nullptr;
    im->surv = nullptr;
    im->defer = nullptr;
    im->cap = 0;
    const int64_t n = std::max<int64_t>(E, 1 << 16);
    cudaError_t e = cudaMalloc(&im->kbuf, n * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc(&im->perm, n * sizeof(int2));
    if (e == cudaSuccess) e = cudaMalloc(&im->surv, n * sizeof(int2));
    if (e == cudaSuccess) e = cudaMalloc(&im->defer, n * sizeof(int2));
    if (e != cudaSuccess) return set_err(msg, "cudaMalloc scratch", e);
    im->cap = n;
    return 0;
}

// Shared memory, grid and environment placement of the persistent kernels:
// the environment goes into each block's shared memory unless that lowers
// the blocks per SM (then it is read in place, through L1).
int prepare_kernel(const BatchedArgs &a, EnvView *view, size_t *smem, int *grid, std::string *msg) {
    EnvView vin = *a.env, vst = *a.env;
    vin.staged = 0;
    vst.staged = 1;
    const size_t m_in = batched_smem(vin, *a.robot), m_st = batched_smem(vst, *a.robot);
    if (m_in > a.smem_optin) {
        *msg = "frame stash exceeds shared memory";
        return 1;
    }
    const size_t m_max = m_st <= a.smem_optin ? m_st : m_in;
    cudaError_t e = cudaSuccess;
    // every family of check orders (the tuner switches between them); the
    // grid fills the SMs for the family that keeps the most blocks resident
    // (blocks past another family's residency start late and find the queue
    // drained)
    int b_in = 0, b_st = 0;
    for (int fam = 0; fam < kFamCount; ++fam) {
        const int order = fam == kFamFrequent ? kOrderFrequent : (fam == kFamInterleave ? kOrderInterleave : 0);
        for (int stats = 0; stats < 2; ++stats)
            for (int staged = 0; staged < 2; ++staged) {
                const void *k[2] = {reinterpret_cast<const void *>(batched_kernel_for(*a.robot, stats, staged, order)),
                                    reinterpret_cast<const void *>(survivors_kernel_for(*a.robot, stats, staged, order))};
                const size_t m = staged ? m_max : m_in;
                for (const void *f : k)
                    if (e == cudaSuccess)
                        e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(m));
            }
        int bi = 0, bs = 0;
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bi, batched_kernel_for(*a.robot, false, false, order),
                                                              kBlock, m_in);
        if (e == cudaSuccess && m_st <= a.smem_optin)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bs, batched_kernel_for(*a.robot, false, true, order),
                                                              kBlock, m_st);
        b_in = std::max(b_in, bi);
        b_st = std::max(b_st, bs);
    }
    if (e != cudaSuccess) return set_err(msg, "batched kernel attributes", e);
    const bool staged = b_st >= 1 && b_st >= b_in;
    *view = staged ? vst : vin;
    *smem = staged ? m_st : m_in;
    const int bps = staged ? b_st : b_in;
    if (bps < 1) {
        *msg = "batched kernel cannot be resident";
        return 1;
    }
    *grid = bps * a.num_sms;
    return 0;
}

// The screening launch: one pass, or for the two-pass order the leading
// link pairs of every edge's first-round states, then the rest of the
// checks on the edges that left undecided (the first pass's list in place
// of perm).
cudaError_t launch_screening(Impl *im, const RobotParams &P, const EnvView &view, BatchPlan plan, const float *q0,
                             const float *q1, int grid, size_t smem, cudaStream_t s, uint8_t *valid,
                             unsigned *status, unsigned long long *work) {
    const BatchedKernel k = batched_kernel_for(P, work != nullptr, view.staged, view.order);
    if (view.order != kOrderTwoPass) {
        plan.pass = 0;
        k<<<grid, kBlock, smem, s>>>(P, view, q0, q1, im->perm, plan, valid, status, im->ctrl, im->surv, im->defer,
                                     work);
        return cudaGetLastError();
    }
    plan.pass = 1;
    k<<<grid, kBlock, smem, s>>>(P, view, q0, q1, im->perm, plan, valid, status, im->ctrl, im->surv, im->defer, work);
    plan.pass = 2;
    k<<<grid, kBlock, smem, s>>>(P, view, q0, q1, im->defer, plan, valid, status, im->ctrl, im->surv, im->defer,
                                 work);
    return cudaGetLastError();
}

// Enqueue the whole pipeline on stream s (also used under capture).
cudaError_t enqueue(Impl *im, const BatchedArgs &a, const EnvView &view, const BatchPlan &plan, size_t smem, int grid,
                    cudaStream_t s, uint8_t *valid, unsigned long long *work = nullptr) {
    const int D = a.robot->n_joints;
    cudaError_t e = cudaMemsetAsync(im->ctrl, 0, kCtrlInts * sizeof(int), s);
    if (e != cudaSuccess) return e;
    const unsigned nb = static_cast<unsigned>((a.E + 255) / 256);
    bucket_count_kernel<<<nb, 256, 0, s>>>(D, a.q0, a.q1, a.counts, a.res, a.E, im->kbuf, valid, a.status, im->ctrl);
    bucket_scatter_kernel<<<nb, 256, 0, s>>>(a.E, im->kbuf, im->perm, im->ctrl);
    // external event-record nodes, so the events time the kernel when replayed from the graph
    if (a.ev_start) e = cudaEventRecordWithFlags(a.ev_start, s, cudaEventRecordExternal);
    if (e != cudaSuccess) return e;
    e = launch_screening(im, *a.robot, view, plan, a.q0, a.q1, grid, smem, s, valid, a.status, work);
    if (e != cudaSuccess) return e;
    survivors_kernel_for(*a.robot, work != nullptr, view.staged, view.order)<<<grid, kBlock, smem, s>>>(*a.robot, view, a.q0, a.q1, im->surv,
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
    p.screen_rounds = im->screen_rounds;
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
    EnvView view;
    rc = prepare_kernel(a, &view, &smem, &grid, msg);
    if (rc) return rc;
    view.order = im->order;
    Impl::Graph *hit = nullptr;
    for (auto &g : im->graphs)
        if (g.q0 == a.q0 && g.q1 == a.q1 && g.counts == a.counts && g.valid == a.valid && g.E == a.E &&
            g.res == a.res && g.ev == a.ev_start && g.watchdog == st.watchdog_ns)
            hit = &g;
    if (!hit) {
        if (im->graphs.size() >= kMaxGraphs) {  // the least recently used makes room
            auto old = std::min_element(im->graphs.begin(), im->graphs.end(),
                                        [](const Impl::Graph &x, const Impl::Graph &y) { return x.used < y.used; });
            cudaGraphExecDestroy(old->exec);
            im->graphs.erase(old);
        }
        Impl::Graph ng;
        cudaGraph_t graph = nullptr;
        cudaError_t e = cudaStreamBeginCapture(im->cap_stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return set_err(msg, "begin capture", e);
        cudaError_t e2 = enqueue(im, a, view, plan_from(im, st.watchdog_ns), smem, grid, im->cap_stream, a.valid);
        e = cudaStreamEndCapture(im->cap_stream, &graph);
        if (e2 != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return set_err(msg, "capture", e2);
        }
        if (e != cudaSuccess) return set_err(msg, "end capture", e);
        e = cudaGraphInstantiate(&ng.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return set_err(msg, "instantiate", e);
        ng.q0 = a.q0;
        ng.q1 = a.q1;
        ng.counts = a.counts;
        ng.valid = a.valid;
        ng.E = a.E;
        ng.res = a.res;
        ng.ev = a.ev_start;
        ng.watchdog = st.watchdog_ns;
        im->graphs.push_back(ng);
        hit = &im->graphs.back();
    }
    hit->used = ++im->clock;
    cudaError_t e = cudaGraphLaunch(hit->exec, a.stream);
    return e == cudaSuccess ? 0 : set_err(msg, "graph launch", e);
}

int batched_work(BatchedState &st, const BatchedArgs &a, unsigned long long *work, std::string *msg) {
    Impl *im = impl_of(st);
    int rc = ensure_capacity(im, a.E, msg);
    if (rc) return rc;
    size_t smem = 0;
    int grid = 0;
    EnvView view;
    rc = prepare_kernel(a, &view, &smem, &grid, msg);
    if (rc) return rc;
    view.order = im->order;
    const cudaError_t e = enqueue(im, a, view, plan_from(im, st.watchdog_ns), smem, grid, a.stream, a.valid, work);
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
    EnvView view;
    int rc = prepare_kernel(a, &view, &smem, &grid, msg);
    if (rc) return rc;
    view.order = im->order;
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
    key.env = a.env_hash;
    for (int b = 0; b < kNB; ++b)
        key.profile.push_back(hist[b] == 0 ? 0 : 1 + static_cast<int>((20 * static_cast<int64_t>(hist[b])) / S));
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            for (int b = 0; b < kNB; ++b) im->G[b] = it->second[b];
            im->screen_rounds = it->second[kNB];
            im->order = it->second[kNB + 1];
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
    p.screen_rounds = kDefaultScreenRounds;
    view.order = 0;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&t0);
    if (e == cudaSuccess) e = cudaEventCreate(&t1);
    // one timing: the best of two runs of the whole sample
    auto time_plan = [&](float *ms_out) {
        float best = 1e30f;
        for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
            // the queues, the survivor count and the deferred counts
            e = cudaMemsetAsync(im->ctrl + kCtrlQueue, 0, kCtrlQueueInts * sizeof(int), s);
            if (e != cudaSuccess) break;
            cudaEventRecord(t0, s);
            launch_screening(im, *a.robot, view, p, a.q0, a.q1, grid, smem, s, tv, a.status, nullptr);
            survivors_kernel_for(*a.robot, false, view.staged, view.order)<<<grid, kBlock, smem, s>>>(*a.robot, view, a.q0, a.q1, im->surv,
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
    // check order (self pairs or primitives first; every link posed first,
    // or checks interleaved with posing; frequent pairs first, in one pass
    // or two) together with the screening rounds, the tiling held: the
    // two interact (a two-pass order wants a short screen), so one at a
    // time can stop short of the best pair
    auto tune_order = [&]() {
        const int keep_o = view.order, keep_r = p.screen_rounds;
        int best_o = keep_o, best_r = keep_r;
        float best = cur;
        for (int o = 0; o < kOrderCount && e == cudaSuccess; ++o)
            for (int R : {1, 2, 4, 8, 0}) {
                if ((o == keep_o && R == keep_r) || e != cudaSuccess) continue;
                view.order = o;
                p.screen_rounds = R;
                float ms = 0.f;
                time_plan(&ms);
                if (e == cudaSuccess && ms < 0.99f * best) {
                    best = ms;
                    best_o = o;
                    best_r = R;
                }
            }
        view.order = best_o;
        p.screen_rounds = best_r;
        cur = best;
    };
    tune_order();
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
    if (e == cudaSuccess) tune_order();
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    cudaFree(tv);
    if (e != cudaSuccess) return set_err(msg, "tuning runs", e);
    for (int b = 0; b < kNB; ++b) im->G[b] = p.G[b];
    im->screen_rounds = p.screen_rounds;
    im->order = view.order;
    im->tuned = true;
    drop_graph(im);
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        std::vector<int> v(im->G, im->G + kNB);
        v.push_back(im->screen_rounds);
        v.push_back(im->order);
        g_tune_cache[key] = v;
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
    im->screen_rounds = kDefaultScreenRounds;
    im->order = 0;
}

void batched_release(BatchedState &st) {
    if (!st.impl) return;
    Impl *im = static_cast<Impl *>(st.impl);
    drop_graph(im);
    if (im->kbuf) cudaFree(im->kbuf);
    if (im->perm) cudaFree(im->perm);
    if (im->surv) cudaFree(im->surv);
    if (im->ctrl) cudaFree(im->ctrl);
    if (im->cap_stream) cudaStreamDestroy(im->cap_stream);
    delete im;
    st.impl = nullptr;
}

void batched_mirror(BatchedState &dst, BatchedState &src) {
    dst.watchdog_ns = src.watchdog_ns;  // part of each graph's key
    Impl *d = impl_of(dst), *s = impl_of(src);
    bool same = d->mirrored == s->epoch && d->screen_rounds == s->screen_rounds && d->order == s->order;
    for (int b = 0; b < kNB; ++b) same = same && d->G[b] == s->G[b];
    if (same) return;
    for (int b = 0; b < kNB; ++b) d->G[b] = s->G[b];
    d->screen_rounds = s->screen_rounds;
    d->order = s->order;
    d->tuned = s->tuned;
    drop_graph(d);
    d->mirrored = s->epoch;
}

void batched_set_screen_rounds(BatchedState &st, int rounds) {
    Impl *im = impl_of(st);
    im->screen_rounds = rounds;
    im->tuned = true;
    drop_graph(im);
}

int batched_screen_rounds(const BatchedState &st) {
    const Impl *im = static_cast<const Impl *>(st.impl);
    return im ? im->screen_rounds : kDefaultScreenRounds;
}

void batched_set_check_order(BatchedState &st, int order) {
    Impl *im = impl_of(st);
    im->order = order;
    im->tuned = true;
    drop_graph(im);
}

int batched_check_order(const BatchedState &st) {
    const Impl *im = static_cast<const Impl *>(st.impl);
    return im ? im->order : 0;
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
