// Batched randomized shortcutting (Sec. III-E, "Bringing it Together": the
// planners' path simplification): per step, every path proposes one
// shortcut from the random numbers it is given, all proposals are validated
// in one batched edge-validation call, and the paths whose shortcut is valid
// drop the waypoints it skips.  These kernels are the propose and apply
// steps; vp_shortcut_paths (vp_api.cu) runs the loop.
#include <cuda_runtime.h>

#include "vp_internal.h"

namespace vp {

namespace {

// Path p's candidate (i, j) from (u0, u1): i = floor(u0 n), j = floor(u1 n)
// in float32 (round to nearest), clamped to n - 1, ordered; a candidate
// needs n >= 3 and j - i >= 2.  The edge rows go to q0c / q1c (waypoint 0
// twice when there is no candidate; its verdict is then ignored).
__global__ void shortcut_propose_kernel(const float *__restrict__ paths, const int32_t *__restrict__ lengths,
                                        long long P, int W, int D, const float *__restrict__ u,
                                        float *__restrict__ q0c, float *__restrict__ q1c, int2 *__restrict__ ij) {
    const long long p = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (p >= P) return;
    const int n = lengths[p];
    int i = -1, j = -1;
    if (n >= 3 && n <= W) {
        const float nf = static_cast<float>(n);
        int a = min(static_cast<int>(floorf(__fmul_rn(u[2 * p], nf))), n - 1);
        int b = min(static_cast<int>(floorf(__fmul_rn(u[2 * p + 1], nf))), n - 1);
        if (a > b) {
            const int t = a;
            a = b;
            b = t;
        }
        if (b - a >= 2) {
            i = a;
            j = b;
        }
    }
    const float *w = paths + p * W * D;
    const int ci = i >= 0 ? i : 0, cj = i >= 0 ? j : 0;
    for (int d = 0; d < D; ++d) {
        q0c[p * D + d] = w[ci * D + d];
        q1c[p * D + d] = w[cj * D + d];
    }
    ij[p] = make_int2(i, j);
}

// One warp per path: a valid shortcut (i, j) moves rows [j, n) to i + 1.
// Each pass reads its 32 elements before any lane writes, and later passes
// read only past everything written, so the overlapping move is safe.
__global__ void shortcut_apply_kernel(float *paths, int32_t *lengths, long long P, int W, int D,
                                      const int2 *__restrict__ ij, const uint8_t *__restrict__ ok) {
    const long long p = (static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (p >= P) return;
    const int2 c = ij[p];
    if (c.x < 0 || !ok[p]) return;
    const int n = lengths[p];
    float *w = paths + p * W * D;
    const int count = (n - c.y) * D;
    for (int e0 = 0; e0 < count; e0 += 32) {
        const int e = e0 + lane;
        const float v = e < count ? w[c.y * D + e] : 0.f;
        __syncwarp();
        if (e < count) w[(c.x + 1) * D + e] = v;
        __syncwarp();
    }
    if (lane == 0) lengths[p] = n - (c.y - c.x - 1);
}

}  // namespace

cudaError_t shortcut_propose(const float *paths, const int32_t *lengths, int64_t P, int W, int D, const float *u,
                             float *q0c, float *q1c, int2 *ij, cudaStream_t st) {
    shortcut_propose_kernel<<<static_cast<unsigned>((P + 255) / 256), 256, 0, st>>>(paths, lengths, P, W, D, u, q0c,
                                                                                    q1c, ij);
    return cudaGetLastError();
}

cudaError_t shortcut_apply(float *paths, int32_t *lengths, int64_t P, int W, int D, const int2 *ij, const uint8_t *ok,
                           cudaStream_t st) {
    shortcut_apply_kernel<<<static_cast<unsigned>((P * 32 + 255) / 256), 256, 0, st>>>(paths, lengths, P, W, D, ij,
                                                                                       ok);
    return cudaGetLastError();
}

}  // namespace vp
