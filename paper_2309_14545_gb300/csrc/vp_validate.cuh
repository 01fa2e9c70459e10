// Validation kernel templates: the plain edge kernel (one warp per edge),
// the batched screening kernel and its second phase.  Each is instantiated
// per link bound LMAX and family of check orders FAM in its own translation
// unit (vp_inst.cu, compiled once per pair), for the counting mode STATS,
// the joint code SIMPLE and the environment placement STAGED (copied into
// shared memory, or read in place through L1; the host launches the
// instance matching EnvView::staged and sizes shared memory to match).
#pragma once

#include <cuda_runtime.h>

#include "vp_batched.h"
#include "vp_device.cuh"
#include "vp_internal.h"

namespace vp {

// State count of an edge from its largest joint displacement (float32, IEEE
// division): max(2, ceil(dmax / res) + 1); -1 past VP_MAX_STEPS.
__device__ __forceinline__ int count_from_dmax(float dmax, float res) {
    const float steps = ceilf(__fdiv_rn(dmax, res));
    if (!(steps <= static_cast<float>(VP_MAX_STEPS))) return -1;
    return max(2, static_cast<int>(steps) + 1);
}

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

struct SmemCarve {
    float4 *env;
    uint64_t *bar;
    float *warp_buf;
    Stash stash;
};

template <bool STAGED>
__device__ __forceinline__ SmemCarve carve(unsigned char *smem, const EnvView &env, const RobotParams &P) {
    SmemCarve c;
    size_t off = STAGED ? static_cast<size_t>(env.n_float4) * 16 : 0;
    c.env = reinterpret_cast<float4 *>(smem);
    c.bar = reinterpret_cast<uint64_t *>(smem + off);
    off += 16;
    c.warp_buf = reinterpret_cast<float *>(smem + off);
    off += static_cast<size_t>((blockDim.x + 31) / 32) * 32 * sizeof(float);
    c.stash = stash_at(smem + off, P.n_links, static_cast<int>(blockDim.x));
    return c;
}

template <bool STATS>
__device__ __forceinline__ void flush_work(Work &wk, unsigned long long *work, int lane) {
    if constexpr (STATS) {
#pragma unroll
        for (int i = 0; i < VP_WORK_N; ++i) {
            const unsigned s = __reduce_add_sync(kFull, wk.v[i]);
            if (lane == 0 && s) atomicAdd(work + i, static_cast<unsigned long long>(s));
            wk.v[i] = 0;
        }
    }
}

// One warp per edge.  Lane j of the warp checks states j*R + r in round r
// (R = ceil(k/32) rounds): the rake of Sec. III-D, 32 spread states per
// round.  Lanes past the end park on the last state.
template <bool STATS, int LMAX, bool SIMPLE, bool STAGED, int FAM>
__global__ void VP_VALIDATION_BOUNDS(LMAX, 5) edges_plain_kernel(const __grid_constant__ RobotParams P, const EnvView env,
                                                          const float *__restrict__ q0, const float *__restrict__ q1,
                                                          const int32_t *__restrict__ counts, const float res,
                                                          const long long E, uint8_t *__restrict__ valid,
                                                          unsigned *status, unsigned long long *work) {
    extern __shared__ __align__(16) unsigned char smem[];
    const SmemCarve sc = carve<STAGED>(smem, env, P);
    if (STAGED && !stage_env(sc.env, env, sc.bar, status)) return;
    const EnvSm es = env_views<STAGED>(sc.env, env);
    const Stash &stash = sc.stash;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    float *wq0 = sc.warp_buf + wib * 32;
    float *wdq = wq0 + 16;
    const int D = P.n_joints;
    Work wk;
    if (STATS) {
#pragma unroll
        for (int i = 0; i < VP_WORK_N; ++i) wk.v[i] = 0;
    }
    for (long long e = static_cast<long long>(blockIdx.x) * wpb + wib; e < E;
         e += static_cast<long long>(gridDim.x) * wpb) {
        float a = 0.f, b = 0.f;
        if (lane < D) {
            a = q0[e * D + lane];
            b = q1[e * D + lane];
        }
        const bool fin = isfinite(a) && isfinite(b);
        const float d = b - a;
        const bool all_fin = __all_sync(kFull, fin);
        const float dmax = __uint_as_float(__reduce_max_sync(kFull, __float_as_uint(fin ? fabsf(d) : 0.f)));
        if (lane < 16) {
            wq0[lane] = a;
            wdq[lane] = d;
        }
        __syncwarp();
        int k = 2;
        bool ok = all_fin;
        if (counts != nullptr) {
            k = counts[e];
            if (k < 2) {
                ok = false;
                if (lane == 0) atomicOr(status, VP_DEVERR_COUNT);
            } else if (k > VP_MAX_STEPS + 1) {  // as long as the longest edge a resolution may give
                ok = false;
                if (lane == 0) atomicOr(status, VP_DEVERR_LENGTH);
            }
        } else if (ok) {
            k = count_from_dmax(dmax, res);
            if (k < 0) {
                ok = false;
                if (lane == 0) atomicOr(status, VP_DEVERR_LENGTH);
            }
        }
        bool collided = !ok;
        if (ok) {
            const int R = (k + 31) >> 5;
            const float inv = __fdiv_rn(1.f, static_cast<float>(k - 1));
            for (int r = 0; r < R; ++r) {
                int i = lane * R + r;
                const bool real = i < k;
                if (!real) i = k - 1;
                const float t = static_cast<float>(i) * inv;
                const WorkRef<STATS> w{&wk, real};
                const bool c = check_state<FAM, kStopAny, STATS, LMAX, SIMPLE>(
                    P, [t, wq0, wdq](int j) { return fmaf(t, wdq[j], wq0[j]); }, es, stash, Ctl{kFull, false}, w);
                if (__any_sync(kFull, c)) {
                    collided = true;
                    break;
                }
            }
        }
        if (lane == 0) valid[e] = collided ? 0 : 1;
        if (STATS) {
            wk.v[VP_WORK_EDGES_DONE] += (lane == 0);
            flush_work<STATS>(wk, work, lane);
        }
        __syncwarp();
    }
}

// Persistent validation of bucketed edges; see the file comment.  STATS adds
// the work counters (VP_WORK_*) of the lanes that hold a state of a live edge.
template <bool STATS, int LMAX, bool SIMPLE, bool STAGED, int FAM>
__global__ void VP_VALIDATION_BOUNDS(LMAX, 6) edges_batched_kernel(
    const __grid_constant__ RobotParams P, const EnvView env, const float *__restrict__ q0,
    const float *__restrict__ q1, const int2 *__restrict__ perm, const BatchPlan plan, uint8_t *__restrict__ valid,
    unsigned *status, int *ctrl, int2 *__restrict__ surv, int2 *defer, unsigned long long *work) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_edge_lo[kNB], s_edge_hi[kNB], s_item_end[kNB];
    // the two-pass order is one of the frequent-first family's: the other
    // families' instances compile the single pass only
    const int pass = FAM == kFamFrequent ? plan.pass : 0;
    __shared__ int s_items;
    size_t off = STAGED ? static_cast<size_t>(env.n_float4) * 16 : 0;
    float4 *env_sm = reinterpret_cast<float4 *>(smem);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + off);
    off += 16;
    float *gbuf = reinterpret_cast<float *>(smem + off);  // [warps][8 groups][32]
    off += static_cast<size_t>(kBlock / 32) * 8 * 32 * sizeof(float);
    const Stash stash = stash_at(smem + off, P.n_links, kBlock);

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
        // a second pass takes the edges the first one deferred, which it
        // wrote from the start of each bucket's range (perm is that list)
        if (pass == 2)
            for (int b = 0; b < kNB; ++b) s_edge_hi[b] = s_edge_lo[b] + ctrl[kCtrlDefer + b];
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
    if (STAGED && !stage_env(env_sm, env, bar, status)) return;
    const EnvSm es = env_views<STAGED>(env_sm, env);
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
                item = atomicAdd(&ctrl[pass == 2 ? kCtrlQueueB : kCtrlQueue], 1);
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
        bool fin = true;
        if (has_edge) {
            for (int d = j; d < D; d += G) {
                const float a = q0[static_cast<long long>(e) * D + d];
                const float b = q1[static_cast<long long>(e) * D + d];
                fin &= isfinite(a) && isfinite(b);
                gq0[d] = a;
                gdq[d] = b - a;
            }
        } else {
            for (int d = j; d < 16; d += G) {
                gq0[d] = 0.f;
                gdq[d] = 0.f;
            }
        }
        __syncwarp();
        // an edge with a non-finite endpoint coordinate is invalid (its group
        // takes no state); with counts from the resolution the count pass has
        // answered it already
        const bool group_fin = (__ballot_sync(kFull, !fin) & gmask) == 0u;
        if (has_edge && !group_fin && j == 0) {
            valid[e] = 0;
            if (STATS) wk.v[VP_WORK_EDGES_DONE] += 1;
        }
        const int R = (k + G - 1) / G;
        const float inv = __fdiv_rn(1.f, static_cast<float>(k - 1));
        const int R_max = __reduce_max_sync(kFull, has_edge && group_fin ? R : 0);
        // the first of two passes checks the first round's states against
        // the leading link pairs only (check phase 0); the second checks the
        // rest of them on the same states (the bucket, and so the lanes per
        // edge, is the same), then goes on as a single pass does
        const int R_lim = pass == 1 ? min(R_max, 1)
                                         : (plan.screen_rounds > 0 ? min(R_max, plan.screen_rounds) : R_max);
        const int last_phase = pass == 1 ? 0 : 2;
        bool done = !has_edge || !group_fin;
        for (int r = 0; r < R_lim; ++r) {
            int i = j * R + r;
            const WorkRef<STATS> w{&wk, !done && i < k};
            if (i >= k) i = k - 1;
            const float t = static_cast<float>(i) * inv;
            const int first_phase = pass == 2 && r == 0 ? 1 : 0;
            const bool c = check_state<FAM, kStopGroups, STATS, LMAX, SIMPLE>(
                P, [t, gq0, gdq](int jj) { return fmaf(t, gdq[jj], gq0[jj]); }, es, stash, Ctl{gmask, done}, w,
                first_phase, last_phase);
            const bool gcol = (__ballot_sync(kFull, c && !done) & gmask) != 0u;
            if (!done && (gcol || (pass != 1 && r == R - 1))) {
                if (j == 0) {
                    valid[e] = gcol ? 0 : 1;
                    if (STATS) wk.v[VP_WORK_EDGES_DONE] += 1;
                }
                done = true;
            }
            if (__all_sync(kFull, done)) break;
        }
        // an edge the screening rounds left undecided goes to the second phase
        // (valid until one of its work items there finds a collision); one
        // the first of two passes left undecided, to the second pass
        if (!done && j == 0) {
            if (pass == 1) {
                defer[s_edge_lo[b] + atomicAdd(&ctrl[kCtrlDefer + b], 1)] = make_int2(e, k);
            } else {
                surv[atomicAdd(&ctrl[kCtrlSurv], 1)] = make_int2(e, k);
                valid[e] = 1;
                if (STATS) wk.v[VP_WORK_EDGES_DONE] += 1;
            }
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

// Second phase: the edges the screening rounds left undecided (mostly
// collision-free ones, which need every state checked).  Each is split into
// kSplit work items of consecutive rounds of a 32-lane raked pass over the
// edge (lane l, round r: state l R + r, R = ceil(k / 32)), so one long edge
// is spread over many warps instead of holding one lane group for all its
// rounds.  A collision clears the edge's verdict; items of an edge already
// found colliding are skipped.
template <bool STATS, int LMAX, bool SIMPLE, bool STAGED, int FAM>
__global__ void VP_VALIDATION_BOUNDS(LMAX, 6) survivors_kernel(
    const __grid_constant__ RobotParams P, const EnvView env, const float *__restrict__ q0,
    const float *__restrict__ q1, const int2 *__restrict__ surv, const BatchPlan plan, uint8_t *valid,
    unsigned *status, int *ctrl, unsigned long long *work) {
    const int n_items = ctrl[kCtrlSurv] * kSplit;  // written by the screening launch
    if (n_items == 0) return;
    extern __shared__ __align__(16) unsigned char smem[];
    size_t off = STAGED ? static_cast<size_t>(env.n_float4) * 16 : 0;
    float4 *env_sm = reinterpret_cast<float4 *>(smem);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + off);
    off += 16;
    float *gbuf = reinterpret_cast<float *>(smem + off);  // [warps][8 groups][32]
    off += static_cast<size_t>(kBlock / 32) * 8 * 32 * sizeof(float);
    const Stash stash = stash_at(smem + off, P.n_links, kBlock);
    if (STAGED && !stage_env(env_sm, env, bar, status)) return;
    const EnvSm es = env_views<STAGED>(env_sm, env);
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int D = P.n_joints;
    float *wq0 = gbuf + wib * 8 * 32, *wdq = wq0 + 16;
    volatile uint8_t *vvalid = valid;
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
                item = atomicAdd(&ctrl[kCtrlQueue2], 1);
            }
        }
        item = __shfl_sync(kFull, item, 0);
        if (item < 0 || item >= n_items) break;
        const int2 ek = surv[item / kSplit];
        const int e = ek.x, k = ek.y, c = item % kSplit;
        const int R = (k + 31) / 32, RC = (R + kSplit - 1) / kSplit;
        const int r0 = c * RC, r1 = min(R, r0 + RC);
        if (r0 >= r1) continue;
        __syncwarp();
        for (int d = lane; d < D; d += 32) {
            const float a = q0[static_cast<long long>(e) * D + d];
            wq0[d] = a;
            wdq[d] = q1[static_cast<long long>(e) * D + d] - a;
        }
        __syncwarp();
        const float inv = __fdiv_rn(1.f, static_cast<float>(k - 1));
        for (int r = r0; r < r1; ++r) {
            if (__shfl_sync(kFull, lane == 0 ? static_cast<int>(vvalid[e]) : 0, 0) == 0) break;  // decided elsewhere
            int i = lane * R + r;
            const WorkRef<STATS> w{&wk, i < k};
            if (i >= k) i = k - 1;
            const float t = static_cast<float>(i) * inv;
            const bool col = check_state<FAM, kStopAny, STATS, LMAX, SIMPLE>(
                P, [t, wq0, wdq](int jj) { return fmaf(t, wdq[jj], wq0[jj]); }, es, stash, Ctl{kFull, false}, w);
            if (__any_sync(kFull, col)) {
                if (lane == 0) vvalid[e] = 0;
                break;
            }
        }
        if constexpr (STATS) {
#pragma unroll
            for (int q = 0; q < VP_WORK_N; ++q) {
                const unsigned sum = __reduce_add_sync(kFull, wk.v[q]);
                if (lane == 0 && sum) atomicAdd(work + q, static_cast<unsigned long long>(sum));
                wk.v[q] = 0;
            }
        }
    }
}

// Every instance of one link bound and kernel family into s: [FAM][stats]
// [simple][staged] (the counting variant always takes the general joint
// code).
template <int LMAX, int FAM>
void fill_kernel_set(KernelSet &s) {
    s.plain[FAM][0][0][0] = edges_plain_kernel<false, LMAX, false, false, FAM>;
    s.plain[FAM][0][0][1] = edges_plain_kernel<false, LMAX, false, true, FAM>;
    s.plain[FAM][0][1][0] = edges_plain_kernel<false, LMAX, true, false, FAM>;
    s.plain[FAM][0][1][1] = edges_plain_kernel<false, LMAX, true, true, FAM>;
    s.plain[FAM][1][0][0] = s.plain[FAM][1][1][0] = edges_plain_kernel<true, LMAX, false, false, FAM>;
    s.plain[FAM][1][0][1] = s.plain[FAM][1][1][1] = edges_plain_kernel<true, LMAX, false, true, FAM>;
    s.batched[FAM][0][0][0] = edges_batched_kernel<false, LMAX, false, false, FAM>;
    s.batched[FAM][0][0][1] = edges_batched_kernel<false, LMAX, false, true, FAM>;
    s.batched[FAM][0][1][0] = edges_batched_kernel<false, LMAX, true, false, FAM>;
    s.batched[FAM][0][1][1] = edges_batched_kernel<false, LMAX, true, true, FAM>;
    s.batched[FAM][1][0][0] = s.batched[FAM][1][1][0] = edges_batched_kernel<true, LMAX, false, false, FAM>;
    s.batched[FAM][1][0][1] = s.batched[FAM][1][1][1] = edges_batched_kernel<true, LMAX, false, true, FAM>;
    s.survivors[FAM][0][0][0] = survivors_kernel<false, LMAX, false, false, FAM>;
    s.survivors[FAM][0][0][1] = survivors_kernel<false, LMAX, false, true, FAM>;
    s.survivors[FAM][0][1][0] = survivors_kernel<false, LMAX, true, false, FAM>;
    s.survivors[FAM][0][1][1] = survivors_kernel<false, LMAX, true, true, FAM>;
    s.survivors[FAM][1][0][0] = s.survivors[FAM][1][1][0] = survivors_kernel<true, LMAX, false, false, FAM>;
    s.survivors[FAM][1][0][1] = s.survivors[FAM][1][1][1] = survivors_kernel<true, LMAX, false, true, FAM>;
}

}  // namespace vp
