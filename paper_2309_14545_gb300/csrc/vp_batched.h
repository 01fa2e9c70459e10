// Batched edge validation: persistent, length-bucketed work queue with a
// tuned tiling, replayed from a CUDA graph.
#pragma once

#include <cuda_runtime.h>

#include <string>

#include "vp_types.h"

namespace vp {

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
void batched_release(BatchedState &st);
// Lanes per edge chosen for each length bucket; returns the bucket count.
int batched_tiling(const BatchedState &st, int *G, int n);
// Replace the first n buckets' lanes per edge (values already checked).
void batched_set_tiling(BatchedState &st, const int *G, int n);

}  // namespace vp
