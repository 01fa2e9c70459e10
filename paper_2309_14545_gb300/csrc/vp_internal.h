// Host-side launcher declarations shared by the C-ABI translation unit and
// the kernel translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "vp_types.h"

namespace vp {

// Shared-memory layout of the validation kernels (bytes):
//   [environment][mbarrier 16][per-warp edge data 128 x warps][stash]
struct SmemPlan {
    int block;          // threads per block
    size_t bytes;       // dynamic shared memory per block
    int blocks_per_sm;  // resident blocks per SM at this size
};

size_t smem_bytes(const EnvView &env, int n_frame_slots, int n_centre_slots, int block);

// Plain edge validation: one warp per edge, static grid-stride over edges.
cudaError_t launch_edges_plain(const RobotParams &P, const EnvView &env, const float *q0, const float *q1,
                               const int32_t *counts, float res, int64_t E, uint8_t *valid, unsigned *status,
                               unsigned long long *work, int grid, int block, size_t smem, cudaStream_t st);
cudaError_t prepare_edges_plain(bool stats, size_t smem, int block, int *blocks_per_sm);

cudaError_t launch_states(const RobotParams &P, const EnvView &env, const float *q, int64_t N, uint8_t *valid,
                          unsigned *status, int grid, int block, size_t smem, cudaStream_t st);
cudaError_t prepare_states(size_t smem, int block, int *blocks_per_sm);

cudaError_t launch_fk(const RobotParams &P, const float *q, int64_t N, float *centres, int grid, int block,
                      size_t smem, cudaStream_t st);
cudaError_t prepare_fk(size_t smem, int block, int *blocks_per_sm);

cudaError_t launch_counts(int D, const float *q0, const float *q1, float res, int64_t E, int32_t *counts,
                          cudaStream_t st);

}  // namespace vp
