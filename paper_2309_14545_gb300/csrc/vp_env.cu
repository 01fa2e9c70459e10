// Host packing of an environment descriptor into the kernels' float4 layout,
// shared by vp_load_env and the allocation-free entry point.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <vector>

#include "vp_internal.h"

namespace vp {

namespace {

bool finite_n(const double *p, int n) {
    for (int i = 0; i < n; ++i)
        if (!std::isfinite(p[i])) return false;
    return true;
}

}  // namespace

int env_packed_float4(const vp_env_desc *e, size_t *n4, std::string *msg) {
    const int ns = e->n_spheres, nc = e->n_capsules, nb = e->n_cuboids;
    if (ns < 0 || nc < 0 || nb < 0) {
        *msg = "negative primitive count";
        return 1;
    }
    if ((ns && !e->spheres) || (nc && !e->capsules) || (nb && !e->cuboids)) {
        *msg = "primitive table pointer is NULL";
        return 1;
    }
    const size_t n = static_cast<size_t>(ns) + nc + nb;
    if (n >= (1u << 24)) {
        *msg = "too many primitives";
        return 2;
    }
    *n4 = 3 * static_cast<size_t>(ns) + 4 * static_cast<size_t>(nc) + 6 * static_cast<size_t>(nb);
    return 0;
}

namespace {

// float nearest to x on the side away from the box (outward rounding)
float round_down(double x) {
    float f = static_cast<float>(x);
    if (static_cast<double>(f) > x) f = std::nextafter(f, -INFINITY);
    return f;
}
float round_up(double x) {
    float f = static_cast<float>(x);
    if (static_cast<double>(f) < x) f = std::nextafter(f, INFINITY);
    return f;
}

// A primitive's world box [lo, hi] grown by the rounding margin, as floats.
void put_box(float4 *out, const double lo[3], const double hi[3]) {
    double m = 0.0;
    for (int a = 0; a < 3; ++a) m = std::max(m, std::max(std::fabs(lo[a]), std::fabs(hi[a])));
    const double g = kBoxMarginAbs + kBoxMarginRel * (1.0 + m);
    out[0] = float4{round_down(lo[0] - g), round_down(lo[1] - g), round_down(lo[2] - g), 0.f};
    out[1] = float4{round_up(hi[0] + g), round_up(hi[1] + g), round_up(hi[2] + g), 0.f};
}

}  // namespace

int pack_env(const vp_env_desc *e, float4 *out, size_t cap_float4, EnvView *view, std::string *msg) {
    size_t n4 = 0;
    int rc = env_packed_float4(e, &n4, msg);
    if (rc) return rc;
    if (n4 > cap_float4) {
        char b[160];
        snprintf(b, sizeof(b), "environment packs to %zu bytes, more than the %zu-byte limit", n4 * 16,
                 cap_float4 * 16);
        *msg = b;
        return 2;
    }
    const int ns = e->n_spheres, nc = e->n_capsules, nb = e->n_cuboids;
    // validate, then order each kind largest bounding radius first (large
    // primitives are the likeliest to end a colliding state early)
    std::vector<std::pair<double, int>> os, oc, ob;
    for (int i = 0; i < ns; ++i) {
        const double *p = e->spheres + 4 * i;
        if (!finite_n(p, 4) || p[3] < 0) {
            *msg = "sphere " + std::to_string(i) + " is malformed";
            return 1;
        }
        os.push_back({p[3], i});
    }
    for (int i = 0; i < nc; ++i) {
        const double *p = e->capsules + 7 * i;
        if (!finite_n(p, 7) || p[6] < 0) {
            *msg = "capsule " + std::to_string(i) + " is malformed";
            return 1;
        }
        const double u[3] = {p[3] - p[0], p[4] - p[1], p[5] - p[2]};
        oc.push_back({0.5 * std::sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]) + p[6], i});
    }
    for (int i = 0; i < nb; ++i) {
        const double *p = e->cuboids + 15 * i;
        if (!finite_n(p, 15) || p[12] < 0 || p[13] < 0 || p[14] < 0) {
            *msg = "cuboid " + std::to_string(i) + " is malformed";
            return 1;
        }
        ob.push_back({std::sqrt(p[12] * p[12] + p[13] * p[13] + p[14] * p[14]), i});
    }
    auto by_size = [](const std::pair<double, int> &a, const std::pair<double, int> &b) { return a.first > b.first; };
    std::stable_sort(os.begin(), os.end(), by_size);
    std::stable_sort(oc.begin(), oc.end(), by_size);
    std::stable_sort(ob.begin(), ob.end(), by_size);
    size_t k = 0;
    for (const auto &it : os) {
        const double *p = e->spheres + 4 * it.second;
        out[k++] = float4{float(p[0]), float(p[1]), float(p[2]), float(p[3])};
    }
    for (const auto &it : oc) {
        const double *p = e->capsules + 7 * it.second;
        const double u[3] = {p[3] - p[0], p[4] - p[1], p[5] - p[2]};
        const double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
        out[k++] = float4{float(p[0]), float(p[1]), float(p[2]), float(p[6])};
        out[k++] = float4{float(u[0]), float(u[1]), float(u[2]), uu > 0 ? float(1.0 / uu) : 0.f};
    }
    for (const auto &it : ob) {
        const double *p = e->cuboids + 15 * it.second;
        const double *c = p, *R = p + 3;
        for (int a = 0; a < 3; ++a) {
            // box axis a = column a of R
            const double ax[3] = {R[0 * 3 + a], R[1 * 3 + a], R[2 * 3 + a]};
            const double off = ax[0] * c[0] + ax[1] * c[1] + ax[2] * c[2];
            out[k++] = float4{float(ax[0]), float(ax[1]), float(ax[2]), float(-off)};
        }
        out[k++] = float4{float(p[12]), float(p[13]), float(p[14]), 0.f};
    }
    // world boxes, same kinds and order
    for (const auto &it : os) {
        const double *p = e->spheres + 4 * it.second;
        const double lo[3] = {p[0] - p[3], p[1] - p[3], p[2] - p[3]};
        const double hi[3] = {p[0] + p[3], p[1] + p[3], p[2] + p[3]};
        put_box(out + k, lo, hi);
        k += 2;
    }
    for (const auto &it : oc) {
        const double *p = e->capsules + 7 * it.second;
        double lo[3], hi[3];
        for (int a = 0; a < 3; ++a) {
            lo[a] = std::min(p[a], p[3 + a]) - p[6];
            hi[a] = std::max(p[a], p[3 + a]) + p[6];
        }
        put_box(out + k, lo, hi);
        k += 2;
    }
    for (const auto &it : ob) {
        const double *p = e->cuboids + 15 * it.second;
        const double *c = p, *R = p + 3, *h = p + 12;
        double lo[3], hi[3];
        for (int a = 0; a < 3; ++a) {  // world axis a: |R_a0| h0 + |R_a1| h1 + |R_a2| h2
            const double ext = std::fabs(R[3 * a]) * h[0] + std::fabs(R[3 * a + 1]) * h[1] +
                               std::fabs(R[3 * a + 2]) * h[2];
            lo[a] = c[a] - ext;
            hi[a] = c[a] + ext;
        }
        put_box(out + k, lo, hi);
        k += 2;
    }
    // kinds visited in order of their largest member
    const double top[3] = {os.empty() ? -1.0 : os[0].first, oc.empty() ? -1.0 : oc[0].first,
                           ob.empty() ? -1.0 : ob[0].first};
    int kinds[3] = {2, 1, 0};
    std::stable_sort(kinds, kinds + 3, [&](int a, int b) { return top[a] > top[b]; });
    view->data = nullptr;
    view->ns = ns;
    view->nc = nc;
    view->nb = nb;
    view->n_float4 = static_cast<int>(n4);
    view->kind_order = kinds[0] | (kinds[1] << 4) | (kinds[2] << 8);
    view->staged = 1;
    view->order = 0;
    return 0;
}

void reorder_env(const std::vector<float4> &in, const std::vector<unsigned> &hits, EnvView *view,
                 std::vector<float4> *out) {
    const int n[3] = {view->ns, view->nc, view->nb};
    const int words[3] = {1, 2, 4};
    int first[3], word0[3], box0[3];  // first primitive index, first data word, first box word of each kind
    first[0] = 0;
    first[1] = n[0];
    first[2] = n[0] + n[1];
    word0[0] = 0;
    word0[1] = n[0];
    word0[2] = n[0] + 2 * n[1];
    const int data_words = n[0] + 2 * n[1] + 4 * n[2];
    box0[0] = data_words;
    box0[1] = data_words + 2 * n[0];
    box0[2] = data_words + 2 * (n[0] + n[1]);
    *out = in;
    unsigned long long total[3] = {0, 0, 0};
    for (int kind = 0; kind < 3; ++kind) {
        std::vector<int> idx(static_cast<size_t>(n[kind]));
        for (int k = 0; k < n[kind]; ++k) {
            idx[k] = k;
            total[kind] += hits[first[kind] + k];
        }
        std::stable_sort(idx.begin(), idx.end(),
                         [&](int a, int b) { return hits[first[kind] + a] > hits[first[kind] + b]; });
        for (int k = 0; k < n[kind]; ++k) {
            const int src = idx[k];
            for (int w = 0; w < words[kind]; ++w)
                (*out)[word0[kind] + k * words[kind] + w] = in[word0[kind] + src * words[kind] + w];
            for (int w = 0; w < 2; ++w) (*out)[box0[kind] + 2 * k + w] = in[box0[kind] + 2 * src + w];
        }
    }
    // kinds by their total hits (ties keep the previous order)
    int kinds[3] = {view->kind_order & 15, (view->kind_order >> 4) & 15, (view->kind_order >> 8) & 15};
    std::stable_sort(kinds, kinds + 3, [&](int a, int b) { return total[a] > total[b]; });
    view->kind_order = kinds[0] | (kinds[1] << 4) | (kinds[2] << 8);
}

}  // namespace vp
