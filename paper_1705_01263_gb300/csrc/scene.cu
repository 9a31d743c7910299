// rt_scene_create / rt_scene_destroy / rt_scene_info: host preprocessing of a
// scene and its upload to device memory (paper Sec. 2.1.1: one flux value per
// emitting triangle computed in a preprocess; Sec. 2.1.2: the environment
// hierarchy built in a preprocess; Sec. 5.6: the whole scene resides in the
// memory of each device).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.h"

namespace rtg {
namespace {

template <class T>
rt_status upload(rt_scene *s, const T *host, size_t count, const T **dev_out, const T **host_out) {
    *dev_out = nullptr;
    if (host_out) *host_out = nullptr;
    if (count == 0 || host == nullptr) return RT_OK;
    if (host_out && s->host_only) {
        std::vector<uint8_t> keep(count * sizeof(T));
        std::memcpy(keep.data(), host, keep.size());
        s->host_keep.push_back(std::move(keep));
        *host_out = (const T *)s->host_keep.back().data();
    }
    if (s->host_only) return RT_OK;
    void *d = nullptr;
    cudaError_t e = cudaMalloc(&d, count * sizeof(T));
    if (e != cudaSuccess) {
        set_error("cudaMalloc failed for scene data");
        return e == cudaErrorMemoryAllocation ? RT_OOM : RT_CUDA_ERROR;
    }
    s->dev_allocs.push_back(d);
    s->device_bytes += (int64_t)(count * sizeof(T));
    RT_CUDA_TRY(cudaMemcpy(d, host, count * sizeof(T), cudaMemcpyHostToDevice));
    *dev_out = (const T *)d;
    return RT_OK;
}

#define RT_TRY(expr)                       \
    do {                                   \
        rt_status _s = (expr);             \
        if (_s != RT_OK) return _s;        \
    } while (0)

double lum3(const float *c) { return 0.2126 * c[0] + 0.7152 * c[1] + 0.0722 * c[2]; }

// Mean luminance of a textured emitter over its triangle, by stratified
// supersampling of the UV footprint (16 x 16 strata, nearest texel).
double textured_mean(const rt_scene_desc *d, int64_t t, int32_t tex) {
    const uint32_t *id = d->indices + 3 * t;
    double acc = 0.0;
    const int n = 16;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double u1 = (i + 0.5) / n, u2 = (j + 0.5) / n;
            double su = std::sqrt(u1);
            double b1 = su * (1.0 - u2), b2 = su * u2, b0 = 1.0 - su;
            double u = b0 * d->uvs[2 * id[0]] + b1 * d->uvs[2 * id[1]] + b2 * d->uvs[2 * id[2]];
            double v = b0 * d->uvs[2 * id[0] + 1] + b1 * d->uvs[2 * id[1] + 1] + b2 * d->uvs[2 * id[2] + 1];
            int x = (int)std::floor(std::min(1.0, std::max(0.0, u)) * d->tex_width);
            int y = (int)std::floor(std::min(1.0, std::max(0.0, v)) * d->tex_height);
            x = std::min(x, d->tex_width - 1);
            y = std::min(y, d->tex_height - 1);
            acc += lum3(d->textures + 3 * (((size_t)tex * d->tex_height + y) * d->tex_width + x));
        }
    return acc / (n * n);
}

// Vose's alias method in double precision; thresholds stored as float.
void build_alias(const std::vector<double> &w, std::vector<float2> &out) {
    size_t n = w.size();
    double sum = 0.0;
    for (double x : w) sum += x;
    std::vector<double> p(n);
    std::vector<uint32_t> small, large;
    out.assign(n, make_float2(1.f, 0.f));
    for (size_t i = 0; i < n; ++i) {
        p[i] = w[i] * (double)n / sum;
        uint32_t self = (uint32_t)i;
        float bits;
        std::memcpy(&bits, &self, 4);
        out[i] = make_float2(1.f, bits);
        (p[i] < 1.0 ? small : large).push_back((uint32_t)i);
    }
    while (!small.empty() && !large.empty()) {
        uint32_t s = small.back(); small.pop_back();
        uint32_t g = large.back(); large.pop_back();
        float bits;
        std::memcpy(&bits, &g, 4);
        out[s] = make_float2((float)p[s], bits);
        p[g] = (p[g] + p[s]) - 1.0;
        (p[g] < 1.0 ? small : large).push_back(g);
    }
}

}  // namespace
}  // namespace rtg

using namespace rtg;

namespace rtg {
rt_status scene_create(const rt_scene_desc *d, rt_scene **out, bool host_only);
}

extern "C" rt_status rt_scene_create(const rt_scene_desc *d, rt_scene **out) {
    return scene_create(d, out, false);
}

/* Host-only copy of the scene for the CPU test hooks (no device memory). */
extern "C" rt_status rt_debug_scene_create_host(const rt_scene_desc *d, rt_scene **out) {
    return scene_create(d, out, true);
}

rt_status rtg::scene_create(const rt_scene_desc *d, rt_scene **out, bool host_only) {
    if (!d || !out) { set_error("rt_scene_create: null argument"); return RT_INVALID_ARG; }
    *out = nullptr;
    if (d->num_triangles < 0 || d->num_vertices < 0 || (d->num_triangles > 0 && (!d->vertices || !d->indices ||
                                                                                   !d->tri_material))) {
        set_error("rt_scene_create: missing geometry arrays");
        return RT_INVALID_ARG;
    }
    if (d->num_instances > 0) {
        set_error("rt_scene_create: instanced scenes are not supported by this build");
        return RT_NOT_SUPPORTED;
    }
    if (d->num_materials <= 0 || !d->albedo || !d->roughness || !d->ggx_weight || !d->emission) {
        set_error("rt_scene_create: material arrays missing");
        return RT_INVALID_ARG;
    }
    const int64_t T = d->num_triangles, V = d->num_vertices;
    for (int64_t t = 0; t < T; ++t) {
        for (int k = 0; k < 3; ++k)
            if ((int64_t)d->indices[3 * t + k] >= V) { set_error("rt_scene_create: vertex index out of range"); return RT_INVALID_ARG; }
        if ((int32_t)d->tri_material[t] >= d->num_materials) { set_error("rt_scene_create: material index out of range"); return RT_INVALID_ARG; }
    }
    bool any_tex = false;
    if (d->emission_tex)
        for (int32_t m = 0; m < d->num_materials; ++m)
            if (d->emission_tex[m] >= 0) {
                any_tex = true;
                if (d->emission_tex[m] >= d->num_textures || !d->textures || !d->uvs) {
                    set_error("rt_scene_create: emission texture index out of range or uvs missing");
                    return RT_INVALID_ARG;
                }
            }
    if (d->env) {
        int32_t W = d->env_width, H = d->env_height;
        if (W < 2 || H < 1 || W != 2 * H || (W & (W - 1)) != 0) {
            set_error("rt_scene_create: environment must be W x H with W = 2H a power of two");
            return RT_INVALID_ARG;
        }
    }
    rt_scene *s = new rt_scene();
    s->host_only = host_only;
    auto fail = [&](rt_status st) { rt_scene_destroy(s); return st; };
    DevScene &D = s->dev, &Hs = s->host;
    s->num_triangles = T;

    // ---- BVH
    Bvh8 bvh;
    build_bvh8(d->vertices, d->indices, nullptr, T, bvh);
    s->num_nodes = bvh.num_nodes();
    s->num_leaf_tris = bvh.num_tris();
    s->bvh_depth = bvh.depth;
    rt_status st;
    if ((st = upload(s, (const uint4 *)bvh.nodes.data(), bvh.nodes.size() / 4, &D.nodes, &Hs.nodes)) != RT_OK) return fail(st);
    if ((st = upload(s, (const float4 *)bvh.tris.data(), bvh.tris.size() / 4, &D.tris, &Hs.tris)) != RT_OK) return fail(st);
    D.bb_lo = Hs.bb_lo = make_float3(bvh.lo[0], bvh.lo[1], bvh.lo[2]);
    D.bb_hi = Hs.bb_hi = make_float3(bvh.hi[0], bvh.hi[1], bvh.hi[2]);

    // ---- shading arrays
    if ((st = upload(s, d->vertices, (size_t)V * 3, &D.vertices, &Hs.vertices)) != RT_OK) return fail(st);
    if (d->normals && (st = upload(s, d->normals, (size_t)V * 3, &D.normals, &Hs.normals)) != RT_OK) return fail(st);
    if (d->uvs && (st = upload(s, d->uvs, (size_t)V * 2, &D.uvs, &Hs.uvs)) != RT_OK) return fail(st);
    if ((st = upload(s, d->indices, (size_t)T * 3, &D.indices, &Hs.indices)) != RT_OK) return fail(st);
    if ((st = upload(s, d->tri_material, (size_t)T, &D.tri_material, &Hs.tri_material)) != RT_OK) return fail(st);
    std::vector<float4> ma(d->num_materials), mb(d->num_materials);
    std::vector<int32_t> mt(d->num_materials, -1);
    for (int32_t m = 0; m < d->num_materials; ++m) {
        ma[m] = make_float4(d->albedo[3 * m], d->albedo[3 * m + 1], d->albedo[3 * m + 2], d->roughness[m]);
        mb[m] = make_float4(d->emission[3 * m], d->emission[3 * m + 1], d->emission[3 * m + 2], d->ggx_weight[m]);
        if (d->emission_tex) mt[m] = d->emission_tex[m];
    }
    if ((st = upload(s, ma.data(), ma.size(), &D.mat_a, &Hs.mat_a)) != RT_OK) return fail(st);
    if ((st = upload(s, mb.data(), mb.size(), &D.mat_b, &Hs.mat_b)) != RT_OK) return fail(st);
    if ((st = upload(s, mt.data(), mt.size(), &D.mat_tex, &Hs.mat_tex)) != RT_OK) return fail(st);
    if (any_tex) {
        D.tex_w = Hs.tex_w = d->tex_width;
        D.tex_h = Hs.tex_h = d->tex_height;
        if ((st = upload(s, d->textures, (size_t)d->num_textures * d->tex_width * d->tex_height * 3, &D.textures,
                         &Hs.textures)) != RT_OK)
            return fail(st);
    }

    // ---- environment pyramid: weights = luminance x exact texel solid angle
    double env_sum = 0.0;
    if (d->env) {
        const int32_t W = d->env_width, H = d->env_height;
        int levels = 0;
        for (int32_t w = W; w >= 2; w /= 2) ++levels;
        if (levels > 16) { set_error("environment too large"); return fail(RT_INVALID_ARG); }
        std::vector<std::vector<double>> lv(levels);
        lv[0].resize((size_t)W * H);
        for (int32_t y = 0; y < H; ++y) {
            double om = (2.0 * M_PI / W) * (std::cos(M_PI * y / H) - std::cos(M_PI * (y + 1) / H));
            for (int32_t x = 0; x < W; ++x) {
                double w = lum3(d->env + 3 * ((size_t)y * W + x)) * om;
                lv[0][(size_t)y * W + x] = w;
                env_sum += w;
            }
        }
        for (int l = 1; l < levels; ++l) {
            int32_t pw = W >> (l - 1), ph = std::max(1, H >> (l - 1));
            int32_t lw = W >> l, lh = std::max(1, H >> l);
            lv[l].assign((size_t)lw * lh, 0.0);
            for (int32_t y = 0; y < ph; ++y)
                for (int32_t x = 0; x < pw; ++x) lv[l][(size_t)(y / 2) * lw + x / 2] += lv[l - 1][(size_t)y * pw + x];
        }
        std::vector<float> pyr;
        std::vector<int64_t> off(levels);
        for (int l = 0; l < levels; ++l) {
            off[l] = (int64_t)pyr.size();
            for (double v : lv[l]) pyr.push_back((float)v);
        }
        std::vector<float4> env4((size_t)W * H);
        for (size_t i = 0; i < env4.size(); ++i) {
            const float *c = d->env + 3 * i;
            env4[i] = make_float4(c[0], c[1], c[2], env_sum > 0.0 ? (float)(lum3(c) / env_sum) : 0.f);
        }
        D.env_w = Hs.env_w = W;
        D.env_h = Hs.env_h = H;
        D.env_levels = Hs.env_levels = levels;
        for (int l = 0; l < levels; ++l) D.env_off_h[l] = Hs.env_off_h[l] = off[l];
        if ((st = upload(s, env4.data(), env4.size(), &D.env, &Hs.env)) != RT_OK) return fail(st);
        if ((st = upload(s, pyr.data(), pyr.size(), &D.env_pyr, &Hs.env_pyr)) != RT_OK) return fail(st);
        if ((st = upload(s, off.data(), off.size(), &D.env_off, &Hs.env_off)) != RT_OK) return fail(st);
    }

    // ---- emitters: flux per triangle, alias table, per-triangle area pdf
    std::vector<double> flux;
    std::vector<uint32_t> light_tri;
    std::vector<double> area(T);
    for (int64_t t = 0; t < T; ++t) {
        const float *p0 = d->vertices + 3 * (size_t)d->indices[3 * t], *p1 = d->vertices + 3 * (size_t)d->indices[3 * t + 1],
                    *p2 = d->vertices + 3 * (size_t)d->indices[3 * t + 2];
        double e1[3] = {(double)p1[0] - p0[0], (double)p1[1] - p0[1], (double)p1[2] - p0[2]};
        double e2[3] = {(double)p2[0] - p0[0], (double)p2[1] - p0[1], (double)p2[2] - p0[2]};
        double c[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
        area[t] = 0.5 * std::sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
        uint32_t m = d->tri_material[t];
        double L = lum3(d->emission + 3 * m);
        if (!(L > 0.0) || !(area[t] > 0.0)) continue;
        int32_t tex = d->emission_tex ? d->emission_tex[m] : -1;
        if (tex >= 0) L *= textured_mean(d, t, tex);
        if (!(L > 0.0)) continue;
        flux.push_back(L * area[t]);
        light_tri.push_back((uint32_t)t);
    }
    double flux_sum = 0.0;
    for (double f : flux) flux_sum += f;
    const bool has_env = d->env && env_sum > 0.0;
    const float p_env = has_env ? (flux.empty() ? 1.f : 0.5f) : 0.f;
    D.p_env = Hs.p_env = p_env;
    std::vector<float> lpa((size_t)std::max<int64_t>(T, 1), 0.f);
    for (size_t i = 0; i < flux.size(); ++i)
        lpa[light_tri[i]] = (float)((1.0 - p_env) * (flux[i] / flux_sum) / area[light_tri[i]]);
    if ((st = upload(s, lpa.data(), (size_t)T, &D.tri_light_pdf_area, &Hs.tri_light_pdf_area)) != RT_OK) return fail(st);
    if (!flux.empty()) {
        std::vector<float2> alias;
        build_alias(flux, alias);
        D.num_lights = Hs.num_lights = (uint32_t)flux.size();
        if ((st = upload(s, alias.data(), alias.size(), &D.alias, &Hs.alias)) != RT_OK) return fail(st);
        if ((st = upload(s, light_tri.data(), light_tri.size(), &D.light_tri, &Hs.light_tri)) != RT_OK) return fail(st);
    }
    *out = s;
    return RT_OK;
}

extern "C" rt_status rt_scene_destroy(rt_scene *s) {
    if (!s) return RT_OK;
    for (void *p : s->dev_allocs) cudaFree(p);
    delete s;
    return RT_OK;
}

extern "C" rt_status rt_scene_info(const rt_scene *s, int64_t *nodes, int64_t *leaf_tris, int64_t *bytes) {
    if (!s) { set_error("rt_scene_info: null scene"); return RT_INVALID_ARG; }
    if (nodes) *nodes = s->num_nodes;
    if (leaf_tris) *leaf_tris = s->num_leaf_tris;
    if (bytes) *bytes = s->device_bytes;
    return RT_OK;
}
