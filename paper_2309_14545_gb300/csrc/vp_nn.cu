// Batched l2 nearest neighbours (Sec. III-E, "Bringing it Together": the
// planners' nearest-neighbour structure over a Euclidean configuration space,
// the l2 distance taken as a sum).  Brute force on the CUDA cores, FP32:
//
// * Each block holds a group of queries in registers (QPT per thread) and
//   streams a range of the points through shared memory in tiles; every
//   point of a tile is compared with every query of the block, so a point is
//   read from L2 once per block rather than once per query.
// * With few queries, several threads share a query and split the tile's
//   points between them (S threads per query), so the block stays busy.
// * The points are split over blocks (grid.y) to fill the GPU.  Each block's
//   best (distance, index) per query meets the others in one 64-bit atomicMin
//   on (float bits of the distance << 32 | index): non-negative float bits
//   order like the floats, and equal distances keep the lowest index.
// * With at most 16 queries the search reads every point once from memory
//   and is bound by that: a streaming kernel keeps the queries in shared
//   memory, lets each thread read its own points straight from memory
//   (consecutive lanes read consecutive rows) and keeps one best per query
//   in registers; a warp reduction precedes the atomicMin.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "vp_internal.h"

namespace vp {

namespace {

constexpr int kNNThreads = 128;
constexpr int kQPT = 4;     // queries per thread
constexpr int kTile = 128;  // points per shared-memory tile

template <int D>
__global__ void __launch_bounds__(kNNThreads) nn_kernel(const float *__restrict__ P, long long M,
                                                        const float *__restrict__ Q, long long N, int S,
                                                        long long chunk, unsigned long long *best) {
    constexpr int DP = (D + 3) / 4 * 4;  // padded row in shared memory (float4 loads)
    __shared__ __align__(16) float tile[kTile * DP];
    __shared__ unsigned long long sbest[kNNThreads * kQPT];
    const int groups = kNNThreads / S;  // queries groups of the block
    const int g = threadIdx.x / S, sub = threadIdx.x - g * S;
    const long long q0 = static_cast<long long>(blockIdx.x) * groups * kQPT + static_cast<long long>(g) * kQPT;
    const long long m0 = static_cast<long long>(blockIdx.y) * chunk;
    const long long m1 = min(M, m0 + chunk);

    float q[kQPT][D];
#pragma unroll
    for (int u = 0; u < kQPT; ++u)
#pragma unroll
        for (int d = 0; d < D; ++d) q[u][d] = (q0 + u < N) ? Q[(q0 + u) * D + d] : 0.f;
    float bd[kQPT];
    unsigned bi[kQPT];
#pragma unroll
    for (int u = 0; u < kQPT; ++u) {
        bd[u] = __int_as_float(0x7f800000);
        bi[u] = 0xffffffffu;
    }
    for (int i = threadIdx.x; i < kNNThreads * kQPT; i += kNNThreads) sbest[i] = ~0ull;

    for (long long base = m0; base < m1; base += kTile) {
        const int nt = static_cast<int>(min(static_cast<long long>(kTile), m1 - base));
        __syncthreads();
        for (int i = threadIdx.x; i < nt * D; i += kNNThreads) {
            const int j = i / D, d = i - j * D;
            tile[j * DP + d] = P[(base + j) * D + d];
        }
        __syncthreads();
        for (int j = sub; j < nt; j += S) {
            float p[DP];
#pragma unroll
            for (int c = 0; c < DP / 4; ++c) {
                const float4 v = reinterpret_cast<const float4 *>(tile + j * DP)[c];
                p[4 * c] = v.x;
                p[4 * c + 1] = v.y;
                p[4 * c + 2] = v.z;
                p[4 * c + 3] = v.w;
            }
            const unsigned idx = static_cast<unsigned>(base + j);
#pragma unroll
            for (int u = 0; u < kQPT; ++u) {
                float acc = 0.f;
#pragma unroll
                for (int d = 0; d < D; ++d) {
                    const float t = q[u][d] - p[d];
                    acc = fmaf(t, t, acc);
                }
                if (acc < bd[u]) {  // strict: the lower index wins among equal distances
                    bd[u] = acc;
                    bi[u] = idx;
                }
            }
        }
    }
    // the S threads of a query group, then the other blocks
    __syncthreads();
#pragma unroll
    for (int u = 0; u < kQPT; ++u)
        if (bi[u] != 0xffffffffu)
            atomicMin(&sbest[g * kQPT + u],
                      (static_cast<unsigned long long>(__float_as_uint(bd[u])) << 32) | bi[u]);
    __syncthreads();
    if (sub == 0) {
#pragma unroll
        for (int u = 0; u < kQPT; ++u) {
            const unsigned long long v = sbest[g * kQPT + u];
            if (q0 + u < N && v != ~0ull) atomicMin(&best[q0 + u], v);
        }
    }
}

__device__ __forceinline__ unsigned long long nn_pack(float d, unsigned i) {
    return (static_cast<unsigned long long>(__float_as_uint(d)) << 32) | i;
}

template <int D, int NQ>
__global__ void __launch_bounds__(kNNThreads) nn_stream_kernel(const float *__restrict__ P, long long M,
                                                               const float *__restrict__ Q, int N,
                                                               unsigned long long *best) {
    __shared__ float sq[NQ * D];
    for (int i = threadIdx.x; i < NQ * D; i += kNNThreads) sq[i] = (i < N * D) ? Q[i] : 0.f;
    __syncthreads();
    unsigned long long b[NQ];
#pragma unroll
    for (int u = 0; u < NQ; ++u) b[u] = ~0ull;
    const long long stride = static_cast<long long>(gridDim.x) * kNNThreads;
    // two points per step: both rows' loads are in flight before the arithmetic
    for (long long m = static_cast<long long>(blockIdx.x) * kNNThreads + threadIdx.x; m < M; m += 2 * stride) {
        const long long m2 = m + stride;
        const bool two = m2 < M;
        float p[D], p2[D];
#pragma unroll
        for (int d = 0; d < D; ++d) {
            p[d] = __ldg(P + m * D + d);
            p2[d] = two ? __ldg(P + m2 * D + d) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < NQ; ++u) {
            float acc = 0.f, acc2 = 0.f;
#pragma unroll
            for (int d = 0; d < D; ++d) {
                const float t = sq[u * D + d] - p[d], t2 = sq[u * D + d] - p2[d];
                acc = fmaf(t, t, acc);
                acc2 = fmaf(t2, t2, acc2);
            }
            const unsigned long long v = nn_pack(acc, static_cast<unsigned>(m));
            if (acc < __int_as_float(0x7f800000) && v < b[u]) b[u] = v;  // finite distances only
            const unsigned long long v2 = nn_pack(acc2, static_cast<unsigned>(m2));
            if (two && acc2 < __int_as_float(0x7f800000) && v2 < b[u]) b[u] = v2;
        }
    }
#pragma unroll
    for (int u = 0; u < NQ; ++u) {
        unsigned long long v = b[u];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
            v = w < v ? w : v;
        }
        if ((threadIdx.x & 31) == 0 && u < N && v != ~0ull) atomicMin(&best[u], v);
    }
}

// Unpack (distance bits, index) in place into the caller's index and
// distance arrays.
__global__ void nn_unpack_kernel(long long N, unsigned long long *packed, float *dist2) {
    const long long n = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const unsigned long long v = packed[n];
    if (dist2) dist2[n] = __uint_as_float(static_cast<unsigned>(v >> 32));
    reinterpret_cast<long long *>(packed)[n] = (v == ~0ull) ? -1 : static_cast<long long>(v & 0xffffffffull);
}

using NNKernel = void (*)(const float *, long long, const float *, long long, int, long long, unsigned long long *);

using NNStreamKernel = void (*)(const float *, long long, const float *, int, unsigned long long *);

template <int D>
NNStreamKernel nn_stream_for(int N) {
    if (N <= 1) return nn_stream_kernel<D, 1>;
    if (N <= 2) return nn_stream_kernel<D, 2>;
    if (N <= 4) return nn_stream_kernel<D, 4>;
    if (N <= 8) return nn_stream_kernel<D, 8>;
    return nn_stream_kernel<D, 16>;
}

NNStreamKernel nn_stream_kernel_for(int D, int N) {
    switch (D) {
        case 1: return nn_stream_for<1>(N);
        case 2: return nn_stream_for<2>(N);
        case 3: return nn_stream_for<3>(N);
        case 4: return nn_stream_for<4>(N);
        case 5: return nn_stream_for<5>(N);
        case 6: return nn_stream_for<6>(N);
        case 7: return nn_stream_for<7>(N);
        case 8: return nn_stream_for<8>(N);
        case 9: return nn_stream_for<9>(N);
        case 10: return nn_stream_for<10>(N);
        case 11: return nn_stream_for<11>(N);
        case 12: return nn_stream_for<12>(N);
        case 13: return nn_stream_for<13>(N);
        case 14: return nn_stream_for<14>(N);
        case 15: return nn_stream_for<15>(N);
        default: return nn_stream_for<16>(N);
    }
}

NNKernel nn_kernel_for(int D) {
    switch (D) {
        case 1: return nn_kernel<1>;
        case 2: return nn_kernel<2>;
        case 3: return nn_kernel<3>;
        case 4: return nn_kernel<4>;
        case 5: return nn_kernel<5>;
        case 6: return nn_kernel<6>;
        case 7: return nn_kernel<7>;
        case 8: return nn_kernel<8>;
        case 9: return nn_kernel<9>;
        case 10: return nn_kernel<10>;
        case 11: return nn_kernel<11>;
        case 12: return nn_kernel<12>;
        case 13: return nn_kernel<13>;
        case 14: return nn_kernel<14>;
        case 15: return nn_kernel<15>;
        default: return nn_kernel<16>;
    }
}

}  // namespace

int nn_launch(const float *points, int64_t M, const float *queries, int64_t N, int D, int64_t *index, float *dist2,
              int num_sms, cudaStream_t st, std::string *msg) {
    if (N == 0) return 0;
    unsigned long long *best = reinterpret_cast<unsigned long long *>(index);
    cudaError_t e = cudaMemsetAsync(best, 0xff, static_cast<size_t>(N) * sizeof(unsigned long long), st);
    if (e == cudaSuccess && N <= 16) {  // a few queries: one streaming pass over the points
        const long long blocks = std::min<long long>((M + kNNThreads - 1) / kNNThreads, 8LL * num_sms);
        nn_stream_kernel_for(D, static_cast<int>(N))<<<static_cast<unsigned>(blocks), kNNThreads, 0, st>>>(
            points, M, queries, static_cast<int>(N), best);
        e = cudaGetLastError();
        if (e == cudaSuccess) {
            nn_unpack_kernel<<<1, 256, 0, st>>>(N, best, dist2);
            e = cudaGetLastError();
        }
        if (e != cudaSuccess) {
            *msg = cudaGetErrorString(e);
            return 2;
        }
        return 0;
    }
    // threads per query: enough queries per block to reuse each tile, enough
    // blocks along the queries to spread them
    int S = 1;
    while (S < kNNThreads && (kNNThreads / S) * kQPT > 2 * N) S *= 2;
    const long long per_block = static_cast<long long>(kNNThreads / S) * kQPT;
    const long long qblocks = (N + per_block - 1) / per_block;
    const long long target = 8LL * num_sms;  // blocks to fill the GPU
    const long long tiles = (M + kTile - 1) / kTile;
    const long long mblocks = std::max(1LL, std::min({tiles, (target + qblocks - 1) / qblocks, 65535LL}));
    const long long chunk = ((M + mblocks - 1) / mblocks + kTile - 1) / kTile * kTile;
    const long long my = (M + chunk - 1) / chunk;
    if (e == cudaSuccess) {
        if (qblocks > 0x7fffffffLL) {
            *msg = "too many queries";
            return 1;
        }
        const dim3 grid(static_cast<unsigned>(qblocks), static_cast<unsigned>(my));
        nn_kernel_for(D)<<<grid, kNNThreads, 0, st>>>(points, M, queries, N, S, chunk, best);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        nn_unpack_kernel<<<static_cast<unsigned>((N + 255) / 256), 256, 0, st>>>(N, best, dist2);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        *msg = cudaGetErrorString(e);
        return 2;
    }
    return 0;
}

}  // namespace vp
