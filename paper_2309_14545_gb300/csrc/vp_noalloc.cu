// Edge validation for callers that cannot allocate device memory.
//
// A robot controller that re-plans inside its real-time loop, or a process
// whose device memory is fixed once at start-up, must not call cudaMalloc
// while it runs: an allocation can block, synchronise the device and take
// unbounded time.  Such a caller cannot create a vp_ctx either (vp_create
// and vp_load_env allocate).  vp_validate_edges_noalloc needs no context:
// it packs the robot into the kernel's parameter block on the host, stages
// the packed environment and the device status word in one file-scope
// static __device__ array, and runs the plain edge kernel on the caller's
// buffers.  The paper has no counterpart to this entry point.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>

#include "vp_internal.h"

namespace vp {
vp_status pack_robot_host(const vp_robot_desc *r, RobotParams *out, std::string *err);
}

using namespace vp;

namespace {

constexpr size_t kStatusBytes = 256;  // status word, padded so the environment starts 256-aligned
constexpr size_t kScratchBytes = kStatusBytes + VP_NOALLOC_MAX_ENV_BYTES;
constexpr int kMaxDevices = 64;

// The scratch every call shares: [status word | packed environment].  Each
// device that loads the library holds one copy until the process exits.
// In host code this name is only a stand-in; its device address comes from
// cudaGetSymbolAddress (see device_scratch).
static __device__ __align__(256) unsigned char vp_noalloc_scratch[kScratchBytes];

struct DeviceSetup {
    bool done = false;
    unsigned char *scratch = nullptr;  // device address of vp_noalloc_scratch
    int num_sms = 0;
    size_t smem_optin = 0;
};

std::mutex g_setup_mutex;
DeviceSetup g_setup[kMaxDevices];

// Per-thread host staging for the packed environment (no heap use).
thread_local float4 t_env_host[VP_NOALLOC_MAX_ENV_BYTES / 16];

void set_msg(char *buf, int32_t len, const char *fmt, ...) {
    if (!buf || len <= 0) return;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, static_cast<size_t>(len), fmt, ap);
    va_end(ap);
}

// Once per device, with that device current: look up the array's device
// address and the launch limits.
vp_status device_scratch(int dev, DeviceSetup **out, char *msg, int32_t msg_len) {
    if (dev < 0 || dev >= kMaxDevices) {
        set_msg(msg, msg_len, "device index out of range");
        return VP_ERR_ARG;
    }
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    DeviceSetup &s = g_setup[dev];
    if (!s.done) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, vp_noalloc_scratch);
        int sms = 0, smem = 0;
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (e != cudaSuccess) {
            set_msg(msg, msg_len, "scratch set-up failed: %s", cudaGetErrorString(e));
            return VP_ERR_CUDA;
        }
        s.scratch = static_cast<unsigned char *>(ptr);
        s.num_sms = sms;
        s.smem_optin = static_cast<size_t>(smem);
        s.done = true;
    }
    *out = &s;
    return VP_OK;
}

bool finite_n(const double *p, int n) {
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(p[i])) return false;
    return true;
}

// Pack the environment into t_env_host in the kernel's float4 layout;
// returns the float4 count or -1 (message set).
int pack_env(const vp_env_desc *e, char *msg, int32_t msg_len, vp_status *st) {
    const int ns = e->n_spheres, nc = e->n_capsules, nb = e->n_cuboids;
    *st = VP_ERR_ARG;
    if (ns < 0 || nc < 0 || nb < 0) {
        set_msg(msg, msg_len, "negative primitive count");
        return -1;
    }
    if ((ns && !e->spheres) || (nc && !e->capsules) || (nb && !e->cuboids)) {
        set_msg(msg, msg_len, "primitive table pointer is NULL");
        return -1;
    }
    const double n4 = static_cast<double>(ns) + 2.0 * nc + 4.0 * nb;
    if (n4 * 16 > VP_NOALLOC_MAX_ENV_BYTES) {
        set_msg(msg, msg_len, "environment packs to %.0f bytes, more than the %d-byte static scratch", n4 * 16,
                VP_NOALLOC_MAX_ENV_BYTES);
        *st = VP_ERR_CAPACITY;
        return -1;
    }
    float4 *h = t_env_host;
    int k = 0;
    for (int i = 0; i < ns; ++i) {
        const double *p = e->spheres + 4 * i;
        if (!finite_n(p, 4) || p[3] < 0) {
            set_msg(msg, msg_len, "malformed sphere");
            return -1;
        }
        h[k++] = float4{float(p[0]), float(p[1]), float(p[2]), float(p[3])};
    }
    for (int i = 0; i < nc; ++i) {
        const double *p = e->capsules + 7 * i;
        if (!finite_n(p, 7) || p[6] < 0) {
            set_msg(msg, msg_len, "malformed capsule");
            return -1;
        }
        const double u[3] = {p[3] - p[0], p[4] - p[1], p[5] - p[2]};
        const double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
        h[k++] = float4{float(p[0]), float(p[1]), float(p[2]), float(p[6])};
        h[k++] = float4{float(u[0]), float(u[1]), float(u[2]), uu > 0 ? float(1.0 / uu) : 0.f};
    }
    for (int i = 0; i < nb; ++i) {
        const double *p = e->cuboids + 15 * i;
        if (!finite_n(p, 15) || p[12] < 0 || p[13] < 0 || p[14] < 0) {
            set_msg(msg, msg_len, "malformed cuboid");
            return -1;
        }
        const double *c = p, *R = p + 3;
        for (int a = 0; a < 3; ++a) {
            const double ax[3] = {R[0 * 3 + a], R[1 * 3 + a], R[2 * 3 + a]};
            const double off = ax[0] * c[0] + ax[1] * c[1] + ax[2] * c[2];
            h[k++] = float4{float(ax[0]), float(ax[1]), float(ax[2]), float(-off)};
        }
        h[k++] = float4{float(p[12]), float(p[13]), float(p[14]), 0.f};
    }
    *st = VP_OK;
    return k;
}

}  // namespace

extern "C" vp_status vp_validate_edges_noalloc(const vp_robot_desc *robot, const vp_env_desc *env,
                                               const float *q0, const float *q1, const int32_t *counts,
                                               float resolution, int64_t n_edges, uint8_t *valid, void *stream,
                                               char *errbuf, int32_t errbuf_len) {
    if (errbuf && errbuf_len > 0) errbuf[0] = '\0';
    if (!robot || !env) {
        set_msg(errbuf, errbuf_len, "robot or environment descriptor is NULL");
        return VP_ERR_ARG;
    }
    if (n_edges < 0) {
        set_msg(errbuf, errbuf_len, "n_edges < 0");
        return VP_ERR_ARG;
    }
    if (!counts && (!(resolution > 0.f) || !std::isfinite(resolution))) {
        set_msg(errbuf, errbuf_len, "resolution must be > 0 when counts is NULL");
        return VP_ERR_ARG;
    }
    if (n_edges > 0 && (!q0 || !q1 || !valid)) {
        set_msg(errbuf, errbuf_len, "NULL buffer");
        return VP_ERR_ARG;
    }
    RobotParams rp;
    std::string perr;
    vp_status st = pack_robot_host(robot, &rp, &perr);
    if (st != VP_OK) {
        set_msg(errbuf, errbuf_len, "robot: %s", perr.c_str());
        return st;
    }
    const int n4 = pack_env(env, errbuf, errbuf_len, &st);
    if (n4 < 0) return st;
    if (n_edges == 0) return VP_OK;

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        set_msg(errbuf, errbuf_len, "no current device: %s", cudaGetErrorString(e));
        return VP_ERR_CUDA;
    }
    DeviceSetup *ds = nullptr;
    st = device_scratch(dev, &ds, errbuf, errbuf_len);
    if (st != VP_OK) return st;

    unsigned *status = reinterpret_cast<unsigned *>(ds->scratch);
    float4 *env_dev = reinterpret_cast<float4 *>(ds->scratch + kStatusBytes);
    const EnvView ev{env_dev, env->n_spheres, env->n_capsules, env->n_cuboids, n4};
    int block = 0;
    size_t smem = 0;
    for (int b : {128, 64, 32}) {
        const size_t s = smem_bytes(ev, rp.n_slots, rp.n_cslots, b);
        if (s <= ds->smem_optin) {
            block = b;
            smem = s;
            break;
        }
    }
    if (block == 0) {
        set_msg(errbuf, errbuf_len, "environment and frame stash exceed shared memory");
        return VP_ERR_CAPACITY;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int bps = 0;
    e = prepare_edges_plain(false, smem, block, &bps);
    // the array keeps the previous call's contents: restage the environment
    // and clear the status word on every call
    if (e == cudaSuccess && n4 > 0)
        e = cudaMemcpyAsync(env_dev, t_env_host, static_cast<size_t>(n4) * 16, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, sizeof(unsigned), s);
    if (e == cudaSuccess) {
        const int wpb = block / 32;
        const int64_t need = (n_edges + wpb - 1) / wpb;
        const int64_t cap = static_cast<int64_t>(bps > 0 ? bps : 1) * ds->num_sms;
        const int grid = static_cast<int>(need < cap ? need : cap);
        e = launch_edges_plain(rp, ev, q0, q1, counts, resolution, n_edges, valid, status, nullptr, grid, block,
                               smem, s);
    }
    unsigned bits = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bits, status, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        set_msg(errbuf, errbuf_len, "CUDA: %s", cudaGetErrorString(e));
        return VP_ERR_CUDA;
    }
    if (bits & VP_DEVERR_TIMEOUT) {
        set_msg(errbuf, errbuf_len, "device watchdog fired");
        return VP_ERR_TIMEOUT;
    }
    if (bits) {
        set_msg(errbuf, errbuf_len, "device reported bad input (status bits 0x%x)", bits);
        return VP_ERR_DEVICE;
    }
    return VP_OK;
}
