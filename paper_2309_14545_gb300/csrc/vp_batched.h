// Batched edge validation: persistent, length-bucketed work queue with a
// tuned tiling, replayed from a CUDA graph.
#pragma once

#include <cuda_runtime.h>

#include <string>

#include "vp_internal.h"
#include "vp_types.h"

namespace vp {

constexpr int kNB = 9;           // length buckets
constexpr int kBlock = 128;      // threads per block of the persistent kernel
constexpr int kCtrlHist = 0;     // ctrl[0..8]   edges per bucket
constexpr int kCtrlCursor = 16;  // ctrl[16..24] scatter cursors
constexpr int kCtrlQueue = 32;   // ctrl[32]     work-item counter
constexpr int kCtrlSurv = 33;    // ctrl[33]     edges left to the second phase
constexpr int kCtrlQueue2 = 34;  // ctrl[34]     second-phase work-item counter
constexpr int kCtrlQueueB = 35;  // ctrl[35]     work-item counter of a two-pass order's second pass
constexpr int kCtrlDefer = 36;   // ctrl[36..44] edges per bucket the first pass left undecided
constexpr int kCtrlQueueInts = 13;  // ctrl[32..44]: the counters each screening run starts from zero
constexpr int kCtrlInts = 64;
constexpr int kSplit = 16;       // second-phase work items per edge
constexpr int kDefaultScreenRounds = 0;

struct BatchPlan {
    int G[kNB];            // lanes per edge, per bucket
    int edge_lo[kNB], edge_hi[kNB];  // bucket b's edges are perm[edge_lo[b], edge_hi[b]) (when !from_hist)
    int from_hist;         // 1: offsets from the histogram in ctrl (longest bucket first)
    int screen_rounds;     // rounds a lane group spends on an edge before handing it on (0: no limit)
    int pass;              // 0: one screening pass; two-pass order: 1, the leading link pairs of the
                           // first-round states, undecided edges deferred by bucket; 2, the deferred edges
    unsigned long long watchdog_ns;  // time budget of one launch
};

// Kernel entry points, by link bound, counting mode, joint code and
// environment placement.
using PlainKernel = void (*)(RobotParams, EnvView, const float *, const float *, const int32_t *, float, long long,
                             uint8_t *, unsigned *, unsigned long long *);
using BatchedKernel = void (*)(RobotParams, EnvView, const float *, const float *, const int2 *, BatchPlan,
                               uint8_t *, unsigned *, int *, int2 *, int2 *, unsigned long long *);
using SurvivorsKernel = void (*)(RobotParams, EnvView, const float *, const float *, const int2 *, BatchPlan,
                                 uint8_t *, unsigned *, int *, unsigned long long *);
struct KernelSet {
    PlainKernel plain[3][2][2][2];  // [family][stats][simple][staged]
    BatchedKernel batched[3][2][2][2];
    SurvivorsKernel survivors[3][2][2][2];
};
// The instances of one link bound and family, each from its own compilation
// of vp_inst.cu.
#define VP_DECLARE_FILL(L)                    \
    void kernel_set_fill_l##L##_f0(KernelSet &); \
    void kernel_set_fill_l##L##_f1(KernelSet &); \
    void kernel_set_fill_l##L##_f2(KernelSet &);
VP_DECLARE_FILL(8)
VP_DECLARE_FILL(9)
VP_DECLARE_FILL(15)
VP_DECLARE_FILL(17)
#undef VP_DECLARE_FILL
// Every instance of link bound lmax (8, 9, 15 or 17).
const KernelSet &kernel_set(int lmax);

struct BatchedArgs {
    const RobotParams *robot;
    const EnvView *env;
    const float *q0, *q1;
    const int32_t *counts;
    float res;
    int64_t E;
    uint8_t *valid;
    unsigned *status;
    int num_sms;
    size_t smem_optin;
    cudaStream_t stream;
    cudaEvent_t ev_start = nullptr, ev_stop = nullptr;  // timing events around the persistent kernel
    uint64_t env_hash = 0;  // contents of the packed environment (tuning-cache key)
};

struct BatchedState {
    void *impl = nullptr;
    unsigned long long watchdog_ns = 60ull * 1000 * 1000 * 1000;  // persistent kernel time budget
};

// 0 = ok, 1 = capacity, 2 = CUDA error (message in *msg)
int batched_validate(BatchedState &st, const BatchedArgs &a, std::string *msg);
int batched_autotune(BatchedState &st, const BatchedArgs &a, std::string *msg);
// Batched validation without the graph, adding work counters into `work`.
int batched_work(BatchedState &st, const BatchedArgs &a, unsigned long long *work, std::string *msg);
void batched_invalidate(BatchedState &st);
// Make dst validate as src does (its tiling, screening rounds and check
// order), dropping dst's graphs whenever src's have been dropped since the
// last call (a new robot, environment or tuning).  Another state's scratch
// lets a second batch run beside the first, as the host-buffer call's chunks do.
void batched_mirror(BatchedState &dst, BatchedState &src);
void batched_release(BatchedState &st);
// Lanes per edge chosen for each length bucket; returns the bucket count.
int batched_tiling(const BatchedState &st, int *G, int n);
// Replace the first n buckets' lanes per edge (values already checked).
void batched_set_tiling(BatchedState &st, const int *G, int n);
// Check order of every validation kernel (kOrder* bits: primitives before
// self pairs, checks interleaved with posing), tuned along with the tiling.
void batched_set_check_order(BatchedState &st, int order);
int batched_check_order(const BatchedState &st);
// Screening rounds of the first phase (0: no limit, no second phase).
void batched_set_screen_rounds(BatchedState &st, int rounds);
int batched_screen_rounds(const BatchedState &st);

}  // namespace vp
