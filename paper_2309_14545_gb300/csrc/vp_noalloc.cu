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

// Per-thread host staging for the packed environment.
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
    EnvView ev{};
    std::string emsg;
    const int prc = pack_env(env, t_env_host, VP_NOALLOC_MAX_ENV_BYTES / 16, &ev, &emsg);
    if (prc) {
        if (prc == 2) emsg += " (the static scratch holds " + std::to_string(VP_NOALLOC_MAX_ENV_BYTES) + " bytes)";
        set_msg(errbuf, errbuf_len, "%s", emsg.c_str());
        return prc == 2 ? VP_ERR_CAPACITY : VP_ERR_ARG;
    }
    const int n4 = ev.n_float4;
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
    ev.data = env_dev;
    int block = 0;
    size_t smem = 0;
    for (int b : {128, 64, 32}) {
        const size_t s = smem_bytes(ev, rp.n_links, b);
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
    e = prepare_edges_plain(false, lmax_for(rp.n_links), rp.simple != 0, ev.staged != 0, smem, block, &bps,
                            ev.order);
    if (e == cudaSuccess && bps < 1) {  // the same status the context path reports
        set_msg(errbuf, errbuf_len, "plain edge kernel cannot be resident");
        return VP_ERR_CAPACITY;
    }
    // the array keeps the previous call's contents: restage the environment
    // and clear the status word on every call
    if (e == cudaSuccess && n4 > 0)
        e = cudaMemcpyAsync(env_dev, t_env_host, static_cast<size_t>(n4) * 16, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, sizeof(unsigned), s);
    if (e == cudaSuccess) {
        const int wpb = block / 32;
        const int64_t need = (n_edges + wpb - 1) / wpb;
        const int64_t cap = static_cast<int64_t>(bps) * ds->num_sms;
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
