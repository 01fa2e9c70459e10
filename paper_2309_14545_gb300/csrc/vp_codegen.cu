// Per-robot FK by code generation (the tracing-compiler idea of Sec. III-B,
// "Vectorized Forward Kinematics": the robot's kinematic chain compiled into
// straight-line code with its constants folded in, instead of interpreting
// a table).  The generator writes a CUDA kernel for the loaded robot -- one
// configuration per thread, every joint and sphere unrolled, every fixed
// transform and sphere offset a literal, terms with a zero coefficient left
// out (exact for finite frames) -- and compiles it with NVRTC for the
// running device.  It computes what the table-driven FK kernel computes, in
// the same order of operations.
#include <cuda_runtime.h>
#include <dlfcn.h>
#include <nvrtc.h>

#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "vp_internal.h"

namespace vp {

namespace {

std::string lit(float v) {  // the exact float as a literal
    if (v == 0.f) return "0.f";
    unsigned bits = 0;
    std::memcpy(&bits, &v, sizeof(bits));
    char b[64];
    snprintf(b, sizeof(b), "__int_as_float(0x%08x)", bits);
    return b;
}

// sum_i a_i k_i + add, nested as fmaf(a0, k0, fmaf(a1, k1, ... add)) with the
// zero-coefficient terms dropped; `add` empty means no addend (the last
// surviving term is then a plain product).
std::string fma_sum(const std::vector<std::pair<std::string, float>> &terms, const std::string &add) {
    std::vector<std::pair<std::string, float>> t;
    for (const auto &x : terms)
        if (x.second != 0.f) t.push_back(x);
    std::string e = add;
    for (int i = static_cast<int>(t.size()) - 1; i >= 0; --i) {
        if (e.empty())
            e = "(" + t[i].first + " * " + lit(t[i].second) + ")";
        else
            e = "fmaf(" + t[i].first + ", " + lit(t[i].second) + ", " + e + ")";
    }
    return e.empty() ? "0.f" : e;
}

std::string fv(int l, const char *c) { return "L" + std::to_string(l) + "_" + c; }

// NVRTC, opened on first use (the library does not link it, so it loads
// where NVRTC is absent and only code generation then fails).
struct Nvrtc {
    decltype(&nvrtcCreateProgram) create = nullptr;
    decltype(&nvrtcCompileProgram) compile = nullptr;
    decltype(&nvrtcGetProgramLogSize) log_size = nullptr;
    decltype(&nvrtcGetProgramLog) log = nullptr;
    decltype(&nvrtcGetCUBINSize) cubin_size = nullptr;
    decltype(&nvrtcGetCUBIN) cubin = nullptr;
    decltype(&nvrtcDestroyProgram) destroy = nullptr;
    bool ok = false;
};

const Nvrtc &nvrtc() {
    static Nvrtc n;
    static std::once_flag once;
    std::call_once(once, [] {
        std::vector<std::string> names = {"libnvrtc.so.13", "libnvrtc.so"};
        if (const char *h = std::getenv("CUDA_HOME")) names.push_back(std::string(h) + "/lib64/libnvrtc.so");
        names.push_back("/usr/local/cuda/lib64/libnvrtc.so");
        void *lib = nullptr;
        for (const auto &nm : names)
            if ((lib = dlopen(nm.c_str(), RTLD_NOW | RTLD_LOCAL))) break;
        if (!lib) return;
        n.create = reinterpret_cast<decltype(n.create)>(dlsym(lib, "nvrtcCreateProgram"));
        n.compile = reinterpret_cast<decltype(n.compile)>(dlsym(lib, "nvrtcCompileProgram"));
        n.log_size = reinterpret_cast<decltype(n.log_size)>(dlsym(lib, "nvrtcGetProgramLogSize"));
        n.log = reinterpret_cast<decltype(n.log)>(dlsym(lib, "nvrtcGetProgramLog"));
        n.cubin_size = reinterpret_cast<decltype(n.cubin_size)>(dlsym(lib, "nvrtcGetCUBINSize"));
        n.cubin = reinterpret_cast<decltype(n.cubin)>(dlsym(lib, "nvrtcGetCUBIN"));
        n.destroy = reinterpret_cast<decltype(n.destroy)>(dlsym(lib, "nvrtcDestroyProgram"));
        n.ok = n.create && n.compile && n.log_size && n.log && n.cubin_size && n.cubin && n.destroy;
    });
    return n;
}

}  // namespace

std::string fk_source(const RobotParams &P) {
    static const char *R[9] = {"r0", "r1", "r2", "r3", "r4", "r5", "r6", "r7", "r8"};
    const int D = P.n_joints, S = P.n_spheres;
    std::string s;
    // one configuration per thread; rows staged in shared memory, then the
    // block's rows (one contiguous range of the output) leave in a single
    // TMA bulk store, so the warp does not spend hundreds of load/store
    // instructions on the write-out
    s += "extern \"C\" __global__ void __launch_bounds__(32) fk_gen(const float *__restrict__ q, long long N,\n"
         "                                                         float *__restrict__ out) {\n"
         "    extern __shared__ __align__(16) float buf[];\n"
         "    const long long base = (long long)blockIdx.x * blockDim.x;\n"
         "    const long long i = base + threadIdx.x;\n"
         "    if (i < N) {\n";
    s += "    const float *qi = q + i * " + std::to_string(D) + ";\n";
    s += "    float *oi = buf + threadIdx.x * " + std::to_string(3 * S) + ";\n";
    // link 0: the base, identity
    for (int k = 0; k < 9; ++k) s += "    const float " + fv(0, R[k]) + " = " + ((k % 4 == 0) ? "1.f" : "0.f") + ";\n";
    s += "    const float L0_px = 0.f, L0_py = 0.f, L0_pz = 0.f;\n";
    auto spheres_of = [&](int l) {
        const LinkC &L = P.links[l];
        for (int k = L.s0; k < L.s1; ++k) {
            const float4 c = P.spheres[k];
            const int o = 3 * P.perm[k];
            const char *pc[3] = {"px", "py", "pz"};
            for (int a = 0; a < 3; ++a)
                s += "    oi[" + std::to_string(o + a) + "] = " +
                     fma_sum({{fv(l, R[3 * a]), c.x}, {fv(l, R[3 * a + 1]), c.y}, {fv(l, R[3 * a + 2]), c.z}},
                             fv(l, pc[a])) +
                     ";\n";
        }
    };
    spheres_of(0);
    for (int j = 0; j < D; ++j) {
        const JointC &J = P.joints[j];
        const int l = j + 1;
        const int src = (J.meta >> kMetaParentShift) & 0xFF;
        const int pl = src == kParentPrev ? l - 1 : (src == kParentBase ? 0 : (J.meta >> kMetaParentLinkShift) & 0xFF);
        const std::string sj = std::to_string(j);
        s += "    // joint " + sj + ": link " + std::to_string(pl) + " -> link " + std::to_string(l) + "\n";
        // origin translation in the parent frame
        const char *pc[3] = {"px", "py", "pz"};
        const float t[3] = {J.o[3], J.o[7], J.o[11]};
        for (int a = 0; a < 3; ++a)
            s += "    float " + fv(l, pc[a]) + " = " +
                 fma_sum({{fv(pl, R[3 * a]), t[0]}, {fv(pl, R[3 * a + 1]), t[1]}, {fv(pl, R[3 * a + 2]), t[2]}},
                         fv(pl, pc[a])) +
                 ";\n";
        // origin rotation: R <- R_parent O (or R_parent itself)
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) {
                std::string e;
                if (J.meta & kMetaOriginRotIdentity)
                    e = fv(pl, R[3 * r + c]);
                else
                    e = fma_sum({{fv(pl, R[3 * r]), J.o[c]}, {fv(pl, R[3 * r + 1]), J.o[4 + c]},
                                 {fv(pl, R[3 * r + 2]), J.o[8 + c]}},
                                "");
                s += "    float " + fv(l, R[3 * r + c]) + " = " + e + ";\n";
            }
        if (J.meta & kMetaPrismatic) {
            s += "    {\n        const float qj = qi[" + sj + "];\n";
            s += "        const float ax = " + lit(J.ax[0]) + " * qj, ay = " + lit(J.ax[1]) + " * qj, az = " +
                 lit(J.ax[2]) + " * qj;\n";
            for (int a = 0; a < 3; ++a)
                s += "        " + fv(l, pc[a]) + " = fmaf(" + fv(l, R[3 * a]) + ", ax, fmaf(" + fv(l, R[3 * a + 1]) +
                     ", ay, fmaf(" + fv(l, R[3 * a + 2]) + ", az, " + fv(l, pc[a]) + ")));\n";
            s += "    }\n";
        } else {
            s += "    {\n        float sj, cj;\n        sincosf(qi[" + sj + "], &sj, &cj);\n";
            const int axis = (J.meta >> kMetaAxisShift) & 3;
            auto rot2 = [&](int i0, int i1, bool plus_first) {
                // columns i0, i1: c_i0' = c c_i0 +- s c_i1, c_i1' = c c_i1 -+ s c_i0
                for (int r = 0; r < 3; ++r) {
                    const std::string a = fv(l, R[3 * r + i0]), b = fv(l, R[3 * r + i1]);
                    s += "        { const float a = " + a + ";\n";
                    s += "          " + a + " = fmaf(cj, a, " + (plus_first ? "" : "-") + "sj * " + b + ");\n";
                    s += "          " + b + " = fmaf(cj, " + b + ", " + (plus_first ? "-" : "") + "sj * a); }\n";
                }
            };
            if (axis == kAxisZ)
                rot2(0, 1, true);
            else if (axis == kAxisY)
                rot2(0, 2, false);
            else if (axis == kAxisX)
                rot2(1, 2, true);
            else {
                s += "        const float x = " + lit(J.ax[0]) + ", y = " + lit(J.ax[1]) + ", z = " + lit(J.ax[2]) +
                     ", v = 1.f - cj;\n";
                s += "        const float m00 = fmaf(v * x, x, cj), m01 = fmaf(v * x, y, -sj * z), "
                     "m02 = fmaf(v * x, z, sj * y);\n";
                s += "        const float m10 = fmaf(v * y, x, sj * z), m11 = fmaf(v * y, y, cj), "
                     "m12 = fmaf(v * y, z, -sj * x);\n";
                s += "        const float m20 = fmaf(v * z, x, -sj * y), m21 = fmaf(v * z, y, sj * x), "
                     "m22 = fmaf(v * z, z, cj);\n";
                for (int r = 0; r < 3; ++r) {
                    const std::string g0 = fv(l, R[3 * r]), g1 = fv(l, R[3 * r + 1]), g2 = fv(l, R[3 * r + 2]);
                    s += "        { const float g0 = " + g0 + ", g1 = " + g1 + ", g2 = " + g2 + ";\n";
                    s += "          " + g0 + " = fmaf(g0, m00, fmaf(g1, m10, g2 * m20));\n";
                    s += "          " + g1 + " = fmaf(g0, m01, fmaf(g1, m11, g2 * m21));\n";
                    s += "          " + g2 + " = fmaf(g0, m02, fmaf(g1, m12, g2 * m22)); }\n";
                }
            }
            s += "    }\n";
        }
        spheres_of(l);
    }
    s += "    }\n"
         "    const long long rows = min((long long)blockDim.x, N - base);\n";
    s += "    const long long count = rows * " + std::to_string(3 * S) + ";\n";
    s += "    float *dst = out + base * " + std::to_string(3 * S) + ";\n";
    // the bulk copy wants 16-byte aligned addresses and a multiple of 16
    // bytes: the whole rows when the output is aligned, else nothing; the
    // last few floats of a ragged range go by plain stores
    s += "    const long long bulk = (reinterpret_cast<unsigned long long>(dst) & 15ull) ? 0 : ((count * 4) & ~15ll);\n"
         "    asm volatile(\"fence.proxy.async.shared::cta;\" ::: \"memory\");\n"
         "    __syncthreads();\n"
         "    if (threadIdx.x == 0 && bulk > 0) {\n"
         "        unsigned sa;\n"
         "        asm volatile(\"{ .reg .u64 t; cvta.to.shared.u64 t, %1; cvt.u32.u64 %0, t; }\" : \"=r\"(sa) : \"l\"(buf));\n"
         "        asm volatile(\"cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;\"\n"
         "                     :: \"l\"(dst), \"r\"(sa), \"r\"((unsigned)bulk) : \"memory\");\n"
         "        asm volatile(\"cp.async.bulk.commit_group;\" ::: \"memory\");\n"
         "    }\n"
         "    for (long long e = bulk / 4 + threadIdx.x; e < count; e += blockDim.x) dst[e] = buf[e];\n"
         "    if (threadIdx.x == 0 && bulk > 0) asm volatile(\"cp.async.bulk.wait_group.read 0;\" ::: \"memory\");\n"
         "}\n";
    return s;
}

// Compile the generated source for the current device and load it.
int fk_codegen_build(const RobotParams &P, FkCodegen *out, std::string *msg) {
    const auto t0 = std::chrono::steady_clock::now();
    const std::string src = fk_source(P);
    int dev = 0, major = 0, minor = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    const Nvrtc &nv = nvrtc();
    if (!nv.ok) {
        *msg = "NVRTC (libnvrtc.so) not found";
        return 2;
    }
    nvrtcProgram prog;
    if (nv.create(&prog, src.c_str(), "vp_fk_gen.cu", 0, nullptr, nullptr) != NVRTC_SUCCESS) {
        *msg = "nvrtcCreateProgram failed";
        return 2;
    }
    const std::string arch = "--gpu-architecture=sm_" + std::to_string(major) + std::to_string(minor) +
                             ((major >= 9) ? "a" : "");
    const char *opts[] = {arch.c_str(), "--std=c++17", "-default-device"};
    nvrtcResult r = nv.compile(prog, 3, opts);
    if (r != NVRTC_SUCCESS) {
        size_t n = 0;
        nv.log_size(prog, &n);
        std::string log(n, '\0');
        if (n) nv.log(prog, &log[0]);
        nv.destroy(&prog);
        *msg = "NVRTC: " + log.substr(0, 600);
        return 2;
    }
    size_t n = 0;
    nv.cubin_size(prog, &n);
    std::vector<char> cubin(n);
    nv.cubin(prog, cubin.data());
    nv.destroy(&prog);
    cudaLibrary_t lib = nullptr;
    cudaError_t e = cudaLibraryLoadData(&lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
    cudaKernel_t k = nullptr;
    if (e == cudaSuccess) e = cudaLibraryGetKernel(&k, lib, "fk_gen");
    if (e != cudaSuccess) {
        if (lib) cudaLibraryUnload(lib);
        *msg = std::string("loading the generated FK: ") + cudaGetErrorString(e);
        return 2;
    }
    out->lib = lib;
    out->kernel = k;
    out->source_bytes = src.size();
    out->compile_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return 0;
}

void fk_codegen_release(FkCodegen *g) {
    if (g->lib) cudaLibraryUnload(g->lib);
    g->lib = nullptr;
    g->kernel = nullptr;
}

cudaError_t fk_codegen_launch(const FkCodegen &g, int n_spheres, const float *q, int64_t N, float *centres,
                              cudaStream_t st) {
    long long n = N;
    void *args[] = {const_cast<float **>(&q), &n, &centres};
    const int cpb = fk_configs_per_block(n_spheres);  // output rows of a block fit in 48 KB
    const unsigned grid = static_cast<unsigned>((N + cpb - 1) / cpb);
    return cudaLaunchKernel(reinterpret_cast<const void *>(g.kernel), dim3(grid), dim3(cpb), args,
                            static_cast<size_t>(cpb) * 3 * n_spheres * sizeof(float), st);
}

}  // namespace vp
