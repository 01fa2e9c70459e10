// Host-side launcher declarations shared by the C-ABI translation unit and
// the kernel translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "vp_types.h"

namespace vp {

// Shared-memory layout of the validation kernels (bytes):
//   [environment][mbarrier 16][per-warp edge data 128 x warps][stash]
struct SmemPlan {
    int block;          // threads per block
    size_t bytes;       // dynamic shared memory per block
    int blocks_per_sm;  // resident blocks per SM at this size
};

// Validation kernels: environment, mbarrier, per-warp buffers, link centres.
size_t smem_bytes(const EnvView &env, int n_links, int block);

// Environment packing (host): float4 count, and the packed buffer with its
// view (data pointer left null).  0 = ok, 1 = bad argument, 2 = capacity.
int env_packed_float4(const vp_env_desc *e, size_t *n4, std::string *msg);
int pack_env(const vp_env_desc *e, float4 *out, size_t cap_float4, EnvView *view, std::string *msg);

// Link-count bound of the validation kernels' register-held link centres
// (instances exist for 8, 9, 15 and 17 links).
inline int lmax_for(int n_links) { return n_links <= 8 ? 8 : n_links <= 9 ? 9 : n_links <= 15 ? 15 : 17; }

// Plain edge validation: one warp per edge, static grid-stride over edges.
cudaError_t launch_edges_plain(const RobotParams &P, const EnvView &env, const float *q0, const float *q1,
                               const int32_t *counts, float res, int64_t E, uint8_t *valid, unsigned *status,
                               unsigned long long *work, int grid, int block, size_t smem, cudaStream_t st);
// Sets the shared-memory attribute of every family's instance; the
// occupancy returned is that of the family of check order `order`.
cudaError_t prepare_edges_plain(bool stats, int lmax, bool simple, bool staged, size_t smem, int block,
                                int *blocks_per_sm, int order);

cudaError_t launch_states(const RobotParams &P, const EnvView &env, const float *q, int64_t N, uint8_t *valid,
                          unsigned *status, int grid, int block, size_t smem, cudaStream_t st);
cudaError_t prepare_states(int lmax, size_t smem, int block, int *blocks_per_sm);

cudaError_t launch_fk(const RobotParams &P, const float *q, int64_t N, float *centres, int grid, int block,
                      size_t smem, cudaStream_t st);
cudaError_t prepare_fk(size_t smem, int block, int *blocks_per_sm);
int fk_configs_per_block(int n_spheres);

cudaError_t launch_counts(int D, const float *q0, const float *q1, float res, int64_t E, int32_t *counts,
                          cudaStream_t st);

// The frequent-first order of the self-pair groups: how often each group
// collides over configurations q [N][D] (device), most often first (ties in
// packed order) into order[kMaxGroups], and into *n_front the number of
// leading groups checked before the primitives (those that together hold
// three quarters of the collisions counted).  Synchronises st.  0 = ok,
// 2 = CUDA error (message in *msg).
int group_order(const RobotParams &P, const float *q, int64_t N, cudaStream_t st, uint8_t *order, int *n_front,
                std::string *msg);

// How often each packed primitive (spheres, capsules, cuboids, in packed
// order) touches a robot sphere over configurations q [N][D] (device).
// Synchronises st.  0 = ok, 2 = CUDA error.
int prim_hits(const RobotParams &P, const EnvView &env, const float *q, int64_t N, cudaStream_t st,
              std::vector<unsigned> *hits, std::string *msg);
// The packed environment `in` with each kind's primitives (and their world
// boxes) reordered most often hit first (ties keep their order), and the
// kinds visited in order of their total hits; *view gets the new kind order.
void reorder_env(const std::vector<float4> &in, const std::vector<unsigned> &hits, EnvView *view,
                 std::vector<float4> *out);

// Batched randomized shortcutting (vp_shortcut.cu): the propose and apply
// steps of one iteration.
cudaError_t shortcut_propose(const float *paths, const int32_t *lengths, int64_t P, int W, int D, const float *u,
                             float *q0c, float *q1c, int2 *ij, cudaStream_t st);
cudaError_t shortcut_apply(float *paths, int32_t *lengths, int64_t P, int W, int D, const int2 *ij, const uint8_t *ok,
                           cudaStream_t st);

// Per-robot FK compiled at run time (vp_codegen.cu).
struct FkCodegen {
    cudaLibrary_t lib = nullptr;
    cudaKernel_t kernel = nullptr;
    size_t source_bytes = 0;
    double compile_ms = 0.0;
};
std::string fk_source(const RobotParams &P);
int fk_codegen_build(const RobotParams &P, FkCodegen *out, std::string *msg);  // 0 = ok, 2 = failure
void fk_codegen_release(FkCodegen *g);
cudaError_t fk_codegen_launch(const FkCodegen &g, int n_spheres, const float *q, int64_t N, float *centres,
                              cudaStream_t st);

// Batched RRT-Connect (vp_rrt.cu): device buffers of one call.
struct RRTLaunch {
    const float *start, *goal, *samples;
    long long B;
    int T, cap;
    float range, res;
    float *nodes;
    int *parent;
    int *counters;   // 3 ints of scratch: the two phases' problem counters and the set-aside count
    int *pending;    // [B] scratch: problems the first phase set aside
    int4 *save;      // [B] scratch: where each set-aside problem stands
    int *status, *iters;
    float *path;
    int *path_len, *sizes;
    unsigned long long watchdog_ns;
};
// 0 = ok, 1 = capacity, 2 = CUDA error.
int rrt_launch(const RobotParams &P, const EnvView &env, const RRTLaunch &L, unsigned *status, int num_sms,
               size_t smem_optin, cudaStream_t st, std::string *msg);

// Batched l2 nearest neighbours (vp_nn.cu); 0 = ok, 1 = capacity, 2 = CUDA error.
int nn_launch(const float *points, int64_t M, const float *queries, int64_t N, int D, int64_t *index, float *dist2,
              int num_sms, cudaStream_t st, std::string *msg);

}  // namespace vp
