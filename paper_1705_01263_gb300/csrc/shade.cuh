// One path vertex of the consistent QMC estimator: state setup with
// shading-normal adaptation (Sec. 2.2 stage 1, Appendix A.3), emitter hit and
// environment miss weighted by MIS (Sec. 2), next event estimation with
// alias-table triangle selection and the environment pyramid (Sec. 2.1.1,
// Sec. 2.1.2), and sampling of the layered BSDF (Sec. 2.2 stage 4).
//
// Readings of the paper fixed here (the FP64 oracle takes the same ones):
//  - max_depth D counts scattering vertices: vertices 1..D do NEE and sample
//    a continuation; vertex D+1 only contributes its emission;
//  - MIS = power heuristic between light sampling and BSDF sampling;
//  - dimensions: 0, 1 in-pixel offset; vertex v uses 2 + 7(v-1) + {0 light
//    select, 1-2 light point, 3 lobe select, 4-5 direction, 6 roulette};
//  - the environment is chosen in NEE with probability p_env (0.5 when both
//    the environment and triangle emitters exist);
//  - a direction below the geometric tangent plane carries nothing; the BSDF
//    vanishes outside the shading hemisphere;
//  - a shadow ray to a triangle runs from the offset origin and stops at
//    (1 - 1e-4) of its distance from there.
#pragma once

#include "guide.cuh"
#include "halton.cuh"
#include "traverse.cuh"

namespace rtg {

struct CameraView {
    V3 eye, fwd, right, up;
    float tan_half, aspect;
    uint32_t W, H;
};

CameraView make_camera(const rt_camera &c);   // host: basis from eye/look-at/up

struct RenderParams {
    DevScene sc;
    CameraView cam;
    Enum en;
    const HaltonDim *dims;   // per dimension (index >= 2 used)
    uint32_t max_depth;
    float sigma;             // > 0 Gaussian, <= 0 box
    int32_t mis_mode;        // 0 power, 1 balance, 2 NEE only, 3 BSDF only
    int32_t rr;
};

// State of one camera path between two vertices.
struct PathState {
    V3 o, d;          // pending ray
    V3 beta;          // throughput
    float prev_pdf;   // pdf of the direction that produced the pending ray
    V3 L;             // radiance gathered so far
    uint64_t index;   // QMC sequence index
    uint32_t pixel;
    uint32_t depth;   // vertex number the pending ray will create (1 = camera ray)
    uint32_t prev_cell;  // normal cell of the vertex that emitted the pending ray (environment pdf)
    uint32_t prev_n;     // its geometric normal, octahedral 16:16 code (light hierarchy pdf)
};

struct ShadowRay {
    V3 o, d;
    float tmax;
    V3 contrib;
};

RT_HD float dim_value(const RenderParams &P, uint64_t idx, int dim) {
    return u32_to_unit(radical_inverse(idx, P.dims[dim]));
}

// ---------------------------------------------------------------- camera
RT_HD void camera_ray(const CameraView &c, float sx, float sy, V3 &o, V3 &d) {
    float nx = (2.f * sx / (float)c.W - 1.f) * c.tan_half * c.aspect;
    float ny = (1.f - 2.f * sy / (float)c.H) * c.tan_half;
    d = normalize(c.fwd + nx * c.right + ny * c.up);
    o = c.eye;
}

// Filter importance sampling (Appendix A.1): Gaussian offset by Box-Muller
// of the in-pixel sample; the sample credits its own pixel.
RT_HD void filter_offset(float sigma, float u0, float u1, float &dx, float &dy) {
    if (!(sigma > 0.f)) { dx = u0 - 0.5f; dy = u1 - 0.5f; return; }
    float r = sigma * sqrtf(-2.f * logf(1.f - u0));
    float s, c;
#ifdef __CUDA_ARCH__
    sincosf(2.f * kPi * u1, &s, &c);
#else
    s = sinf(2.f * kPi * u1); c = cosf(2.f * kPi * u1);
#endif
    dx = r * c;
    dy = r * s;
}

RT_HD void raygen(const RenderParams &P, uint32_t pixel, uint32_t j, PathState &s) {
    uint32_t x = pixel % P.cam.W, y = pixel / P.cam.W;
    uint64_t idx = pixel_base_index(P.en, x, y) + (uint64_t)j * P.en.period;
    float u0 = u32_to_unit(dim0_bits(P.en, idx)), u1 = u32_to_unit(dim1_bits(P.en, idx));
    float dx, dy;
    filter_offset(P.sigma, u0, u1, dx, dy);
    camera_ray(P.cam, (float)x + 0.5f + dx, (float)y + 0.5f + dy, s.o, s.d);
    s.beta = v3(1.f, 1.f, 1.f);
    s.prev_pdf = 0.f;
    s.L = v3(0.f, 0.f, 0.f);
    s.index = idx;
    s.pixel = pixel;
    s.depth = 1;
    s.prev_cell = 0;
    s.prev_n = 0;
}

// ------------------------------------------------------------------ BSDF
RT_HD void onb(V3 n, V3 &t, V3 &b) {
    float sign = n.z >= 0.f ? 1.f : -1.f;
    float a = -1.f / (sign + n.z);
    float bb = n.x * n.y * a;
    t = v3(1.f + sign * n.x * n.x * a, sign * bb, -sign * n.x);
    b = v3(bb, sign + n.y * n.y * a, -n.y);
}

RT_HD V3 adapt_shading_normal(V3 ns, V3 ng, V3 wo) {
    float c = dot(wo, ns);
    V3 r = 2.f * c * ns - wo;
    float a = dot(r, ng);
    if (a >= kAdaptEps) return ns;
    const float e = kAdaptEps;
    float sq = e * sqrtf(fmaxf(0.f, (1.f - a * a) / (1.f - e * e)));
    float t = sq - a;
    V3 rp = r + t * ng;
    float lr = length(rp);
    if (!(lr > 1e-12f)) return ng;
    rp = rp * (1.f / lr);
    V3 h = wo + rp;
    float lh = length(h);
    if (!(lh > 1e-12f)) return ng;
    return h * (1.f / lh);
}

RT_HD float ggx_D(float a2, float ch) {
    if (ch <= 0.f) return 0.f;
    float k = ch * ch * (a2 - 1.f) + 1.f;
    return a2 / (kPi * k * k);
}
RT_HD float ggx_lambda(float a2, float c) {
    float c2 = c * c;
    float t2 = fmaxf(0.f, 1.f - c2) / c2;
    return 0.5f * (-1.f + sqrtf(1.f + a2 * t2));
}
RT_HD float schlick(float c) {
    float m = 1.f - fmaxf(0.f, fminf(1.f, c));
    float m2 = m * m;
    return kF0 + (1.f - kF0) * m2 * m2 * m;
}

struct Material {
    V3 albedo;
    float alpha;   // roughness^2, >= 1e-4
    float w;       // GGX weight
};

RT_HD void bsdf_eval(const Material &m, V3 ns, V3 wo, V3 wi, V3 &f, float &pdf) {
    float co = dot(wo, ns), ci = dot(wi, ns);
    f = v3(0.f, 0.f, 0.f);
    pdf = 0.f;
    if (co <= 0.f || ci <= 0.f) return;
    float a2 = m.alpha * m.alpha;
    V3 h = normalize(wo + wi);
    float ch = dot(h, ns), cih = dot(wi, h);
    float D = ggx_D(a2, ch);
    float lo = ggx_lambda(a2, co);
    float G2 = 1.f / (1.f + lo + ggx_lambda(a2, ci));
    float spec = D * G2 * schlick(cih) / (4.f * co * ci);
    float kd = (1.f - m.w) * kInvPi;
    f = v3(m.w * spec + kd * m.albedo.x, m.w * spec + kd * m.albedo.y, m.w * spec + kd * m.albedo.z);
    float pdf_spec = D / ((1.f + lo) * 4.f * co);
    pdf = m.w * pdf_spec + (1.f - m.w) * ci * kInvPi;
}

RT_HD V3 ggx_vndf(float alpha, V3 v, float u1, float u2) {
    V3 vh = normalize(v3(alpha * v.x, alpha * v.y, v.z));
    float lensq = vh.x * vh.x + vh.y * vh.y;
    V3 T1 = lensq > 0.f ? v3(-vh.y, vh.x, 0.f) * (1.f / sqrtf(lensq)) : v3(1.f, 0.f, 0.f);
    V3 T2 = cross(vh, T1);
    float r = sqrtf(u1), phi = 2.f * kPi * u2;
    float sp, cp;
#ifdef __CUDA_ARCH__
    sincosf(phi, &sp, &cp);
#else
    sp = sinf(phi); cp = cosf(phi);
#endif
    float t1 = r * cp, t2 = r * sp;
    float s = 0.5f * (1.f + vh.z);
    t2 = (1.f - s) * sqrtf(fmaxf(0.f, 1.f - t1 * t1)) + s * t2;
    float tz = sqrtf(fmaxf(0.f, 1.f - t1 * t1 - t2 * t2));
    V3 nh = t1 * T1 + t2 * T2 + tz * vh;
    return normalize(v3(alpha * nh.x, alpha * nh.y, fmaxf(0.f, nh.z)));
}

RT_HD bool bsdf_sample(const Material &m, V3 ns, V3 wo, float u_lobe, float u1, float u2, V3 &wi, V3 &f,
                       float &pdf) {
    V3 t, b;
    onb(ns, t, b);
    float co = dot(wo, ns);
    if (co <= 0.f) return false;
    V3 local;
    if (u_lobe < m.w) {
        V3 vl = v3(dot(wo, t), dot(wo, b), co);
        V3 h = ggx_vndf(m.alpha, vl, u1, u2);
        local = 2.f * dot(vl, h) * h - vl;
    } else {
        float r = sqrtf(u1), phi = 2.f * kPi * u2;
        float sp, cp;
#ifdef __CUDA_ARCH__
        sincosf(phi, &sp, &cp);
#else
        sp = sinf(phi); cp = cosf(phi);
#endif
        local = v3(r * cp, r * sp, sqrtf(fmaxf(0.f, 1.f - u1)));
    }
    wi = normalize(local.x * t + local.y * b + local.z * ns);
    bsdf_eval(m, ns, wo, wi, f, pdf);
    return pdf > 0.f;
}

RT_HD Material load_material(const DevScene &sc, uint32_t mid) {
    float4 a = ldg(sc.mat_a + mid);
    float4 b = ldg(sc.mat_b + mid);
    Material m;
    m.albedo = v3(a.x, a.y, a.z);
    m.alpha = fmaxf(a.w * a.w, 1e-4f);
    m.w = b.w;
    return m;
}

// --------------------------------------------------------------- lights
RT_HD float mis_weight(int mode, float pa, float pb) {
    if (mode == 1) return pa / (pa + pb);
    float a = pa * pa, b = pb * pb;
    return a / (a + b);
}

// Instance transforms (rows 0..2 world->object, rows 3..5 object->world).
RT_HD V3 xf_point(const float4 *xf, uint32_t inst, V3 p) {
    const float4 a = ldg(xf + 6 * (size_t)inst + 3), b = ldg(xf + 6 * (size_t)inst + 4), c = ldg(xf + 6 * (size_t)inst + 5);
    return v3(a.x * p.x + a.y * p.y + a.z * p.z + a.w, b.x * p.x + b.y * p.y + b.z * p.z + b.w,
              c.x * p.x + c.y * p.y + c.z * p.z + c.w);
}
// Normals map with the inverse transpose of object->world, i.e. the
// transpose of the world->object linear part.
RT_HD V3 xf_normal(const float4 *xf, uint32_t inst, V3 n) {
    const float4 a = ldg(xf + 6 * (size_t)inst), b = ldg(xf + 6 * (size_t)inst + 1), c = ldg(xf + 6 * (size_t)inst + 2);
    return v3(a.x * n.x + b.x * n.y + c.x * n.z, a.y * n.x + b.y * n.y + c.y * n.z, a.z * n.x + b.z * n.y + c.z * n.z);
}

// World-space vertex k of triangle prim (of instance inst in two-level scenes).
RT_HD V3 tri_vertex(const DevScene &sc, uint32_t inst, uint32_t prim, int k) {
    uint32_t vi = ldg(sc.indices + 3 * (size_t)prim + k);
    const float *v = sc.vertices + 3 * (size_t)vi;
    V3 p = v3(ldg(v), ldg(v + 1), ldg(v + 2));
    return sc.two_level ? xf_point(sc.inst_xf, inst, p) : p;
}

RT_HD V3 tri_emission(const DevScene &sc, uint32_t prim, uint32_t mid, float b1, float b2) {
    float4 e = ldg(sc.mat_b + mid);
    V3 Le = v3(e.x, e.y, e.z);
    int32_t tex = ldg(sc.mat_tex + mid);
    if (tex < 0) return Le;
    float b0 = 1.f - b1 - b2;
    uint32_t i0 = ldg(sc.indices + 3 * (size_t)prim), i1 = ldg(sc.indices + 3 * (size_t)prim + 1),
             i2 = ldg(sc.indices + 3 * (size_t)prim + 2);
    float u = b0 * ldg(sc.uvs + 2 * (size_t)i0) + b1 * ldg(sc.uvs + 2 * (size_t)i1) + b2 * ldg(sc.uvs + 2 * (size_t)i2);
    float v = b0 * ldg(sc.uvs + 2 * (size_t)i0 + 1) + b1 * ldg(sc.uvs + 2 * (size_t)i1 + 1) +
              b2 * ldg(sc.uvs + 2 * (size_t)i2 + 1);
    int x = (int)floorf(fminf(1.f, fmaxf(0.f, u)) * (float)sc.tex_w);
    int y = (int)floorf(fminf(1.f, fmaxf(0.f, v)) * (float)sc.tex_h);
    x = x >= sc.tex_w ? sc.tex_w - 1 : x;
    y = y >= sc.tex_h ? sc.tex_h - 1 : y;
    const float *t = sc.textures + 3 * (((size_t)tex * sc.tex_h + y) * sc.tex_w + x);
    return v3(Le.x * ldg(t), Le.y * ldg(t + 1), Le.z * ldg(t + 2));
}

RT_HD V3 tri_emission(const DevScene &sc, uint32_t prim, float b1, float b2) {
    return tri_emission(sc, prim, ldg(sc.tri_material + prim), b1, b2);
}

// Equirectangular texel of a direction (row 0 looks at +y).
RT_HD int env_texel(const DevScene &sc, V3 w) {
    float cy = fmaxf(-1.f, fminf(1.f, w.y));
    float th = acosf(cy);
    float ph = atan2f(w.z, w.x);
    if (ph < 0.f) ph += 2.f * kPi;
    int x = (int)floorf(ph * (1.f / (2.f * kPi)) * (float)sc.env_w);
    int y = (int)floorf(th * kInvPi * (float)sc.env_h);
    x = x < 0 ? 0 : (x >= sc.env_w ? sc.env_w - 1 : x);
    y = y < 0 ? 0 : (y >= sc.env_h ? sc.env_h - 1 : y);
    return y * sc.env_w + x;
}

RT_HD float envw(const DevScene &sc, int level, int x, int y) {
    int w = sc.env_w >> level;
    return ldg(sc.env_pyr + sc.env_off_h[level] + (int64_t)y * w + x);
}

RT_HD int choose2(float a, float b, float &u) {
    float p = a / (a + b);
    if (u < p) { u = u / p; return 0; }
    u = (u - p) / (1.f - p);
    if (u >= 1.f) u = 0.99999994f;
    return 1;
}

// Pyramid descent (Sec. 2.1.2): column by u then row by v at each level,
// rescaling each, from the top pair down to a texel. The weights come in
// blocks of two levels (DevScene::env_dq; a normal cell's own blocks where
// its children are reweighted, cellq non-null), so one load serves two
// choices; the choices and the values they use are those of a level-by-level
// walk over the stored weights.
RT_HD void env_descend(const DevScene &sc, const float4 *cellq, float top0, float top1, float &u, float &v, int &x,
                       int &y) {
    int l = sc.env_levels - 1;
    x = choose2(top0, top1, u);
    y = 0;
    while (l >= 1) {
        const int64_t node = (int64_t)y * (sc.env_w >> l) + x;
        const bool own = cellq && sc.env_ndqoff_h[l] >= 0;
        const float4 *B = own ? cellq + sc.env_ndqoff_h[l] : sc.env_dq + sc.env_dqoff_h[l];
        if (l >= 2) {
            B += 5 * node;
            const float4 q = ldg(B), g0 = ldg(B + 1), g1 = ldg(B + 2), g2 = ldg(B + 3), g3 = ldg(B + 4);
            int dx = choose2(q.x + q.z, q.y + q.w, u);
            int dy = choose2(dx ? q.y : q.x, dx ? q.w : q.z, v);
            x = 2 * x + dx;
            y = 2 * y + dy;
            const int k = 2 * dy + dx;
            const float4 g = k == 0 ? g0 : (k == 1 ? g1 : (k == 2 ? g2 : g3));
            dx = choose2(g.x + g.z, g.y + g.w, u);
            dy = choose2(dx ? g.y : g.x, dx ? g.w : g.z, v);
            x = 2 * x + dx;
            y = 2 * y + dy;
            l -= 2;
        } else {
            const float4 q = ldg(B + node);
            const int dx = choose2(q.x + q.z, q.y + q.w, u);
            const int dy = choose2(dx ? q.y : q.x, dx ? q.w : q.z, v);
            x = 2 * x + dx;
            y = 2 * y + dy;
            l -= 1;
        }
    }
}

// Direction uniform in (phi, cos theta) inside texel (x, y), by the
// remaining fractions u, v.
RT_HD V3 env_texel_dir(const DevScene &sc, int x, int y, float u, float v) {
    float phi = 2.f * kPi * ((float)x + u) / (float)sc.env_w;
    float c0 = cosf(kPi * (float)y / (float)sc.env_h), c1 = cosf(kPi * (float)(y + 1) / (float)sc.env_h);
    float ct = c0 - v * (c0 - c1);
    float st = sqrtf(fmaxf(0.f, 1.f - ct * ct));
    float sp, cp;
#ifdef __CUDA_ARCH__
    sincosf(phi, &sp, &cp);
#else
    sp = sinf(phi); cp = cosf(phi);
#endif
    return v3(st * cp, ct, st * sp);
}

RT_HD V3 env_sample(const DevScene &sc, float u, float v) {
    const int top = sc.env_levels - 1;
    int x, y;
    env_descend(sc, nullptr, envw(sc, top, 0, 0), envw(sc, top, 1, 0), u, v, x, y);
    return env_texel_dir(sc, x, y, u, v);
}

// Normal-oriented top levels of the pyramid (Sec. 2.1.2). The unit sphere of
// geometric normals is cut into kEnvCellSide^2 cells of the octahedral map
// (plane (x, z); the lower hemisphere folded over the diagonals); for each
// cell the scene holds its own copy of the top pyramid levels, built on the
// host: the finest of them weights each region by a bound of the clamped
// cosine between the cell's normals and the region's directions, the coarser
// ones are sums. A descent for a vertex of cell c follows that copy down to
// the finest reweighted level and the plain pyramid below it.
constexpr int kEnvCellSide = 8;   // the scene's tables hold the top five levels for each of the 64 cells

RT_HD uint32_t env_cell(V3 n) {
    float a = fabsf(n.x) + fabsf(n.y) + fabsf(n.z);
    if (!(a > 0.f)) return 0u;
    float px = n.x / a, pz = n.z / a;
    if (n.y < 0.f) {
        float fx = (1.f - fabsf(pz)) * (px >= 0.f ? 1.f : -1.f);
        float fz = (1.f - fabsf(px)) * (pz >= 0.f ? 1.f : -1.f);
        px = fx;
        pz = fz;
    }
    int i = (int)floorf((px + 1.f) * (0.5f * kEnvCellSide));
    int j = (int)floorf((pz + 1.f) * (0.5f * kEnvCellSide));
    i = i < 0 ? 0 : (i >= kEnvCellSide ? kEnvCellSide - 1 : i);
    j = j < 0 ? 0 : (j >= kEnvCellSide ? kEnvCellSide - 1 : j);
    return (uint32_t)(j * kEnvCellSide + i);
}

// Solid-angle pdf factor of finest texel `tx` for normal cell `cell`
// relative to the plain pyramid's pdf (texel luminance / total weight).
RT_HD float env_cell_factor(const DevScene &sc, uint32_t cell, int tx) {
    if (!sc.env_nw) return 1.f;
    const int x = tx % sc.env_w, y = tx / sc.env_w, ls = sc.env_lstar;
    return ldg(sc.env_nfac + (size_t)cell * (size_t)sc.env_nregions + (size_t)((y >> ls) * (sc.env_w >> ls) + (x >> ls)));
}

// Descent for a vertex of normal cell `cell`; a cell whose reweighted total
// vanishes (env_nscale 0) descends the plain pyramid.
RT_HD V3 env_sample_cell(const DevScene &sc, uint32_t cell, float u, float v) {
    if (!sc.env_nw || !(ldg(sc.env_nscale + cell) > 0.f)) return env_sample(sc, u, v);
    const float *blk = sc.env_nw + (size_t)cell * (size_t)sc.env_nstride;
    const int top = sc.env_levels - 1;
    int x, y;
    env_descend(sc, sc.env_ndq + (size_t)cell * (size_t)sc.env_ndqstride, ldg(blk + sc.env_noff_h[top]),
                ldg(blk + sc.env_noff_h[top] + 1), u, v, x, y);
    return env_texel_dir(sc, x, y, u, v);
}

// Ray origin moved off the surface along n by an offset that grows with the
// magnitude of the position (integer-ULP offset as in Waechter and Binder,
// "A fast and robust method for avoiding self-intersection", 2019).
RT_HD V3 offset_origin(V3 p, V3 n) {
    const float kOrigin = 1.f / 32.f, kFloatScale = 1.f / 65536.f, kIntScale = 256.f;
    float pc[3] = {p.x, p.y, p.z}, nc[3] = {n.x, n.y, n.z}, out[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        int of = (int)(kIntScale * nc[a]);
        int bits = (int)as_uint(pc[a]);
        float pi = as_float((uint32_t)(bits + (pc[a] < 0.f ? -of : of)));
        out[a] = fabsf(pc[a]) < kOrigin ? pc[a] + kFloatScale * nc[a] : pi;
    }
    return v3(out[0], out[1], out[2]);
}

// --------------------------------------------------------------- shading
// Local frame of a hit (Sec. 2.2 stage 1): position from barycentrics,
// geometric normal turned towards wo, interpolated shading normal on the same
// side, adapted so the perfect reflection stays above the tangent plane
// (Appendix A.3).
struct Vertex {
    V3 x, ng, ns, wo;
    V3 nsr;           // shading normal before the adaptation (on ng's side)
    float cog;        // cos between wo and the unflipped geometric normal
};

RT_HD void setup_vertex(const DevScene &sc, const PathState &s, const Hit &h, Vertex &vx) {
    const uint32_t prim = h.prim;
    const uint32_t i0 = ldg(sc.indices + 3 * (size_t)prim), i1 = ldg(sc.indices + 3 * (size_t)prim + 1),
                   i2 = ldg(sc.indices + 3 * (size_t)prim + 2);
    // positions and vertex normals are independent loads: issued together
    const float *p0 = sc.vertices + 3 * (size_t)i0, *p1 = sc.vertices + 3 * (size_t)i1,
                *p2 = sc.vertices + 3 * (size_t)i2;
    V3 v0 = v3(ldg(p0), ldg(p0 + 1), ldg(p0 + 2)), v1 = v3(ldg(p1), ldg(p1 + 1), ldg(p1 + 2)),
       v2 = v3(ldg(p2), ldg(p2 + 1), ldg(p2 + 2));
    V3 m0 = v3(0.f, 0.f, 0.f), m1 = m0, m2 = m0;
    if (sc.normals) {
        const float *n0 = sc.normals + 3 * (size_t)i0, *n1 = sc.normals + 3 * (size_t)i1,
                    *n2 = sc.normals + 3 * (size_t)i2;
        m0 = v3(ldg(n0), ldg(n0 + 1), ldg(n0 + 2));
        m1 = v3(ldg(n1), ldg(n1 + 1), ldg(n1 + 2));
        m2 = v3(ldg(n2), ldg(n2 + 1), ldg(n2 + 2));
    }
    if (sc.two_level) {
        v0 = xf_point(sc.inst_xf, h.inst, v0);
        v1 = xf_point(sc.inst_xf, h.inst, v1);
        v2 = xf_point(sc.inst_xf, h.inst, v2);
    }
    float b0 = 1.f - h.b1 - h.b2;
    vx.x = b0 * v0 + h.b1 * v1 + h.b2 * v2;
    V3 ng = normalize(cross(v1 - v0, v2 - v0));
    vx.wo = -s.d;
    vx.cog = dot(vx.wo, ng);
    if (vx.cog < 0.f) ng = -ng;
    V3 ns = ng;
    if (sc.normals) {
        ns = b0 * m0 + h.b1 * m1 + h.b2 * m2;
        if (sc.two_level) ns = xf_normal(sc.inst_xf, h.inst, ns);
        ns = normalize(ns);
        if (dot(ns, ng) < 0.f) ns = -ns;
    }
    vx.ng = ng;
    vx.nsr = ns;
    vx.ns = adapt_shading_normal(ns, ng, vx.wo);
}

// Training record of a guided vertex: network input, sampled direction and
// the throughput on arrival (the radiance that comes back through wi is
// known only when the path ends).
struct GuideRecord {
    float feat[7];
    V3 wi;
    V3 beta;
};

// ------------------------------------------------------- light hierarchy
// Octahedral 16:16 code of a unit vector (plane (x, y), lower hemisphere
// folded over the diagonals, 16 bits per coordinate) and back: the path
// state keeps the previous vertex's geometric normal in one 32-bit word.
RT_HD uint32_t oct_encode(V3 n) {
    float a = fabsf(n.x) + fabsf(n.y) + fabsf(n.z);
    float px = a > 0.f ? n.x / a : 0.f, py = a > 0.f ? n.y / a : 0.f;
    if (n.z < 0.f) {
        float fx = (1.f - fabsf(py)) * (px >= 0.f ? 1.f : -1.f);
        float fy = (1.f - fabsf(px)) * (py >= 0.f ? 1.f : -1.f);
        px = fx;
        py = fy;
    }
    uint32_t ux = (uint32_t)rintf(fminf(fmaxf(px * 0.5f + 0.5f, 0.f), 1.f) * 65535.f);
    uint32_t uy = (uint32_t)rintf(fminf(fmaxf(py * 0.5f + 0.5f, 0.f), 1.f) * 65535.f);
    return ux | (uy << 16);
}

RT_HD V3 oct_decode(uint32_t c) {
    float px = (float)(c & 0xffffu) * (2.f / 65535.f) - 1.f, py = (float)(c >> 16) * (2.f / 65535.f) - 1.f;
    float z = 1.f - fabsf(px) - fabsf(py);
    if (z < 0.f) {
        float fx = (1.f - fabsf(py)) * (px >= 0.f ? 1.f : -1.f);
        float fy = (1.f - fabsf(px)) * (py >= 0.f ? 1.f : -1.f);
        px = fx;
        py = fy;
    }
    return normalize(v3(px, py, z));
}

// Estimated contribution of a light-hierarchy node to point x of normal n
// (Sec. 2.1.1): its directional value for the region the point lies in,
// seen from the box centre, times a bound of the surface cosine over the
// box's bounding sphere, over the squared distance to the centre; inside the
// sphere the largest directional value over the squared radius. The node
// comes as its three float4 of a descent record: (centre, r), (I0..I3),
// (I4, I5, flux, link).
RT_HD float lb_estimate(float4 a, float4 b, float4 c, V3 x, V3 n) {
    if (!(c.z > 0.f)) return 0.f;
    const V3 v = x - v3(a.x, a.y, a.z);
    const float d2 = dot(v, v), r = a.w;
    if (d2 <= r * r) return fmaxf(fmaxf(fmaxf(b.x, b.y), fmaxf(b.z, b.w)), fmaxf(c.x, c.y)) / (r * r);
    const float d = sqrtf(d2);
    const V3 w = v * (1.f / d);
    const float ax = fabsf(w.x), ay = fabsf(w.y), az = fabsf(w.z);
    float I;
    if (az > fmaxf(ax, ay)) I = w.z < 0.f ? c.y : c.x;
    else if (ay > ax) I = w.y < 0.f ? b.w : b.z;
    else I = w.x < 0.f ? b.y : b.x;
    // kappa(angle(n, -w) - asin(r / d)) through cosines: 1 inside the cone,
    // cos of the gap up to 90 degrees, 0 beyond
    const float ca = -dot(n, w), sa = sqrtf(fmaxf(0.f, 1.f - ca * ca));
    const float sb = r / d, cb = sqrtf(fmaxf(0.f, 1.f - sb * sb));
    const float cs = ca >= cb ? 1.f : fmaxf(0.f, ca * cb + sa * sb);
    return I * cs / d2;
}

// One step of the descent at record R: the two children's data (loaded
// together) and the probability of the first child: a child without flux is
// never chosen, else the share of the estimates (of the fluxes when both
// vanish) clamped to [0.1, 0.9].
struct LbStep {
    float4 c0, c1;   // (I4, I5, flux, link) of each child
    float p_left;
};

RT_HD LbStep lb_step(const float4 *R, V3 x, V3 n) {
    const float4 a0 = ldg(R), b0 = ldg(R + 1), c0 = ldg(R + 2), a1 = ldg(R + 3), b1 = ldg(R + 4), c1 = ldg(R + 5);
    LbStep st;
    st.c0 = c0;
    st.c1 = c1;
    const float fl = c0.z, fr = c1.z;
    if (!(fl > 0.f)) st.p_left = 0.f;
    else if (!(fr > 0.f)) st.p_left = 1.f;
    else {
        const float el = lb_estimate(a0, b0, c0, x, n), er = lb_estimate(a1, b1, c1, x, n);
        const float p = el + er > 0.f ? el / (el + er) : fl / (fl + fr);
        st.p_left = fminf(fmaxf(p, 0.1f), 0.9f);
    }
    return st;
}

constexpr int kLbMaxDepth = 64;

// Emitter drawn with u from point x of normal n, and its probability P (0
// when the descent does not end in a leaf within kLbMaxDepth levels). Not
// inlined, like lb_prob: the shading kernels then keep the registers of the
// scenes without a hierarchy.
RT_HD __noinline__ uint32_t lb_sample(const DevScene &sc, V3 x, V3 n, float u, float &P) {
    uint32_t rec = 0;
    P = 1.f;
    for (int depth = 0; depth < kLbMaxDepth; ++depth) {
        const LbStep st = lb_step(sc.lb_rec + 7 * (size_t)rec, x, n);
        const bool left = u < st.p_left;
        if (left) {
            u = u / st.p_left;
            P *= st.p_left;
        } else {
            u = (u - st.p_left) / (1.f - st.p_left);
            if (u >= 1.f) u = 0.99999994f;
            P *= 1.f - st.p_left;
        }
        const float4 c = left ? st.c0 : st.c1;
        const uint32_t link = as_uint(c.w);
        if (link & 0x80000000u) {
            const uint32_t first = (link & 0x7fffffffu) >> 3, count = link & 7u;
            const float target = u * c.z;
            float cum = 0.f;
            uint32_t pick = ldg(sc.lb_perm + first + count - 1);
            float fpick = 0.f;
            for (uint32_t i = 0; i < count; ++i) {
                const uint32_t e = ldg(sc.lb_perm + first + i);
                const float f = ldg(sc.lb_eflux + e);
                cum += f;
                if (target < cum || i + 1 == count) { pick = e; fpick = f; break; }
            }
            P *= fpick / c.z;
            return pick;
        }
        rec = link;
    }
    P = 0.f;
    return 0u;
}

// Probability that the descent from x (normal n) draws emitter e: the same
// branch probabilities along the path from e's leaf up to the root.
RT_HD __noinline__ float lb_prob(const DevScene &sc, V3 x, V3 n, uint32_t e) {
    const uint32_t up = ldg(sc.lb_up + e);
    uint32_t rec = up >> 1, side = up & 1u;
    float P = ldg(sc.lb_eflux + e);
    bool first = true;
    for (int depth = 0; depth < kLbMaxDepth; ++depth) {
        const float4 *R = sc.lb_rec + 7 * (size_t)rec;
        const float4 info = ldg(R + 6);
        const LbStep st = lb_step(R, x, n);
        if (first) {
            P /= side ? st.c1.z : st.c0.z;   // the emitter's share of its leaf
            first = false;
        }
        P *= side ? 1.f - st.p_left : st.p_left;
        const uint32_t parent = as_uint(info.x);
        if (parent == 0xffffffffu) break;
        rec = parent;
        side = as_uint(info.y);
    }
    return P;
}

// Area of emitter e (world space).
RT_HD float emitter_area(const DevScene &sc, uint32_t e) {
    const float4 *LV = sc.light_v + 3 * (size_t)e;
    const V3 a = f4xyz(ldg(LV)), b = f4xyz(ldg(LV + 1)), c = f4xyz(ldg(LV + 2));
    return 0.5f * length(cross(b - a, c - a));
}

// NEE light pick of a vertex: the sample's light-selection and light-point
// dimensions and, for a triangle emitter, its world-space vertices, material
// and light pdf. It needs only the sample index, so the shading kernels issue
// its loads before the vertex is set up, overlapping their latencies.
struct NeePick {
    float us, ua, ub;
    uint32_t lt, lmid;
    float lpa;
    V3 l0, l1, l2;
};

// kLb false: compiled without the light hierarchy (scenes that have none).
template <bool kLb = true>
RT_HD NeePick nee_pick(const RenderParams &P, uint64_t index, int base) {
    const DevScene &sc = P.sc;
    NeePick k;
    k.us = dim_value(P, index, base);
    k.ua = dim_value(P, index, base + 1);
    k.ub = dim_value(P, index, base + 2);
    k.lt = 0;
    k.lmid = 0;
    k.lpa = 0.f;
    k.l0 = k.l1 = k.l2 = v3(0.f, 0.f, 0.f);
    if (!(k.us < sc.p_env) && !(kLb && sc.lb_rec)) {
        float u2 = (k.us - sc.p_env) / (1.f - sc.p_env);
        float xn = u2 * (float)sc.num_lights;
        uint32_t bin = (uint32_t)xn;
        if (bin >= sc.num_lights) bin = sc.num_lights - 1;
        float frac = xn - (float)bin;
        float2 al = ldg(sc.alias + bin);
        uint32_t li = frac < al.x ? bin : as_uint(al.y);
        k.lt = ldg(sc.light_tri + li);
        const float4 *LV = sc.light_v + 3 * (size_t)li;
        k.l0 = f4xyz(ldg(LV));
        k.l1 = f4xyz(ldg(LV + 1));
        k.l2 = f4xyz(ldg(LV + 2));
        k.lpa = ldg(sc.tri_light_pdf_area + k.lt);
        k.lmid = ldg(sc.tri_material + k.lt);
    }
    return k;
}

// Next-event estimation and the continuation of vertex `vx` (material m) of
// path s, vertex number s.depth: the scattering half of shade(), shared with
// the probe vertex. Returns bit 0 when the path continues and bit 1 when `sh`
// holds a shadow ray (see shade()).
// `mix` holds the decoded guiding mixture of a guided vertex (thread-local
// storage by default; the guided kernels pass shared-memory storage).
template <bool kLb = true, class Mix = Mixture>
RT_HD int scatter(const RenderParams &P, PathState &s, const Vertex &vx, const Material &m, bool nee,
                  const NeePick &pk, ShadowRay &sh, const __nv_bfloat16 *graw, float alpha, GuideRecord *rec, float3 glo,
                  float3 ghi, Mix mix = Mix()) {
    const DevScene &sc = P.sc;
    const int mode = P.mis_mode;
    const uint32_t v = s.depth;
    const int base = 2 + 7 * (int)(v - 1);
    const V3 x = vx.x, ng = vx.ng, ns = vx.ns, wo = vx.wo;
    const bool guided = graw != nullptr && alpha > 0.f;
    if (guided) decode_mixture(graw, mix);
    V3 xo = offset_origin(x, ng);
    int ret = 0;
    // next-event estimation
    if (nee) {
        const float us = pk.us, ua = pk.ua, ub = pk.ub;
        V3 wi = v3(0.f, 0.f, 1.f), Le = v3(0.f, 0.f, 0.f), sdir = wi;
        float pdf_l = 0.f, tmax = INFINITY;
        if (us < sc.p_env) {
            const uint32_t cell = env_cell(ng);
            wi = env_sample_cell(sc, cell, ua, ub);
            sdir = wi;
            const int tx = env_texel(sc, wi);
            float4 e = ldg(sc.env + tx);
            Le = v3(e.x, e.y, e.z);
            pdf_l = sc.p_env * e.w * env_cell_factor(sc, cell, tx);
        } else {
            V3 l0 = pk.l0, l1 = pk.l1, l2 = pk.l2;
            uint32_t lt = pk.lt, lmid = pk.lmid;
            float lpa = pk.lpa;
            if (kLb && sc.lb_rec) {
                // the light hierarchy draws the emitter from the offset
                // origin and the normal as the path state keeps it, so that
                // an emitter hit by the continuation gets the same number
                float P;
                const uint32_t li = lb_sample(sc, xo, oct_decode(oct_encode(ng)), (us - sc.p_env) / (1.f - sc.p_env), P);
                const float4 *LV = sc.light_v + 3 * (size_t)li;
                l0 = f4xyz(ldg(LV));
                l1 = f4xyz(ldg(LV + 1));
                l2 = f4xyz(ldg(LV + 2));
                lt = ldg(sc.light_tri + li);
                lmid = ldg(sc.tri_material + lt);
                lpa = (1.f - sc.p_env) * P / (0.5f * length(cross(l1 - l0, l2 - l0)));
            }
            float sq = sqrtf(ua);
            float lb1 = sq * (1.f - ub), lb2 = sq * ub;
            V3 y = (1.f - sq) * l0 + lb1 * l1 + lb2 * l2;
            V3 dv = y - x;
            float dist = length(dv);
            if (dist > 0.f) {
                wi = dv * (1.f / dist);
                V3 lng = normalize(cross(l1 - l0, l2 - l0));
                float cl = -dot(wi, lng);
                if (cl > 0.f) {
                    pdf_l = lpa * dist * dist / cl;
                    Le = tri_emission(sc, lt, lmid, lb1, lb2);
                    // The shadow segment runs from the offset origin: its own
                    // length bounds the test, so that the sampled triangle
                    // itself is never reached (from x, a receiver close to the
                    // emitter at a grazing angle would see the offset eat the
                    // margin and occlude itself).
                    V3 sv = y - xo;
                    float sl = length(sv);
                    if (sl > 0.f) {
                        sdir = sv * (1.f / sl);
                        tmax = sl * (1.f - kShadowEps);
                    } else {
                        pdf_l = 0.f;
                    }
                }
            }
        }
        if (pdf_l > 0.f && dot(wi, ng) > 0.f) {
            V3 f;
            float pdf_b;
            bsdf_eval(m, ns, wo, wi, f, pdf_b);
            if (guided) pdf_b = alpha * mixture_pdf(mix, wi) + (1.f - alpha) * pdf_b;
            if (pdf_b > 0.f && (!guided || f.x > 0.f || f.y > 0.f || f.z > 0.f)) {
                float w = mode == 2 ? 1.f : mis_weight(mode, pdf_l, pdf_b);
                float k = dot(wi, ns) * w / pdf_l;
                sh.o = xo;
                sh.d = sdir;
                sh.tmax = tmax;
                sh.contrib = mul(mul(s.beta, f), Le) * k;
                ret |= 2;
            }
        }
    }
    // continuation
    V3 wi, f;
    float pdf;
    float u3 = dim_value(P, s.index, base + 3), u4 = dim_value(P, s.index, base + 4),
          u5 = dim_value(P, s.index, base + 5);
    if (guided) {
        if (u3 < alpha) {
            wi = mixture_sample(mix, u3 / alpha, u4, u5);
        } else {
            V3 fb;
            float pb;
            if (!bsdf_sample(m, ns, wo, (u3 - alpha) / (1.f - alpha), u4, u5, wi, fb, pb)) return ret;
        }
        bsdf_eval(m, ns, wo, wi, f, pdf);
        pdf = alpha * mixture_pdf(mix, wi) + (1.f - alpha) * pdf;
        if (!(pdf > 0.f) || (f.x <= 0.f && f.y <= 0.f && f.z <= 0.f)) return ret;
    } else if (!bsdf_sample(m, ns, wo, u3, u4, u5, wi, f, pdf)) {
        return ret;
    }
    if (dot(wi, ng) <= 0.f) return ret;
    float ci = dot(wi, ns);
    V3 beta_in = s.beta;
    s.beta = mul(s.beta, f) * (ci / pdf);
    if (P.rr && v >= 3) {
        float q = fmaxf(0.05f, 1.f - maxc(s.beta));
        if (dim_value(P, s.index, base + 6) < q) return ret;
        s.beta = s.beta * (1.f / (1.f - q));
    }
    if (s.beta.x == 0.f && s.beta.y == 0.f && s.beta.z == 0.f) return ret;
    if (rec) {
        guide_features(x, wo, ns, glo, ghi, rec->feat);
        rec->wi = wi;
        rec->beta = beta_in;
    }
    s.prev_pdf = pdf;
    s.prev_cell = env_cell(ng);
    s.prev_n = oct_encode(ng);
    s.o = xo;
    s.d = wi;
    s.depth = v + 1;
    return ret | 1;
}


// Shade the hit of the pending ray of `s`. Returns bit 0 when the path
// continues (new pending ray in s.o, s.d) and bit 1 when `sh` holds a shadow
// ray whose unoccluded contribution must be added to s.L. With `graw` (the
// guiding network's 40 outputs for this vertex, BF16) the continuation is drawn
// from the one-sample MIS mixture alpha * vMF-mixture + (1 - alpha) * BSDF
// and every pdf used for MIS is that mixture's; with `rec` the vertex's
// training record is filled when the path continues.
template <bool kLb = true, class Mix = Mixture>
RT_HD int shade(const RenderParams &P, PathState &s, const Hit &h, ShadowRay &sh, const __nv_bfloat16 *graw = nullptr,
                float alpha = 0.f, GuideRecord *rec = nullptr, float3 glo = float3{0.f, 0.f, 0.f},
                float3 ghi = float3{1.f, 1.f, 1.f}, Mix mix = Mix()) {
    const DevScene &sc = P.sc;
    const int mode = P.mis_mode;
    const uint32_t v = s.depth;
    if (h.prim == RT_MISS) {
        if (sc.env_w > 0) {
            int tx = env_texel(sc, s.d);
            float4 e = ldg(sc.env + tx);
            float w = 1.f;
            if (v > 1) {
                if (mode == 3) w = 1.f;
                else if (mode == 2) w = 0.f;
                else w = sc.p_env > 0.f
                             ? mis_weight(mode, s.prev_pdf, sc.p_env * e.w * env_cell_factor(sc, s.prev_cell, tx))
                             : 1.f;
            }
            s.L = s.L + mul(s.beta, v3(e.x, e.y, e.z)) * w;
        }
        return 0;
    }
    const uint32_t prim = h.prim;
    // Loads that need only the hit record and the sample index go out before
    // the vertex is set up, so that their latencies overlap with its loads:
    // the hit triangle's material and light pdf, and the NEE light pick.
    const uint32_t mid = ldg(sc.tri_material + prim);
    const float lpa = ldg(sc.tri_light_pdf_area + prim);
    const bool last = v == P.max_depth + 1;
    const bool nee = !last && (sc.num_lights > 0 || sc.p_env > 0.f) && mode != 3;
    NeePick pk;
    if (nee) pk = nee_pick<kLb>(P, s.index, 2 + 7 * (int)(v - 1));
    Vertex vx;
    setup_vertex(sc, s, h, vx);
    if (vx.cog > 0.f && lpa > 0.f) {
        V3 Le = tri_emission(sc, prim, mid, h.b1, h.b2);
        float w = 1.f;
        if (v > 1) {
            if (mode == 3) w = 1.f;
            else if (mode == 2) w = 0.f;
            else {
                float pa = lpa;
                if (kLb && sc.lb_rec) {
                    // the hierarchy's probability of this emitter from the
                    // previous vertex (offset origin s.o, its stored normal)
                    const uint32_t li = ldg(sc.lb_inst_base + h.inst) + ldg(sc.lb_tri_rank + prim);
                    pa = (1.f - sc.p_env) * lb_prob(sc, s.o, oct_decode(s.prev_n), li) / emitter_area(sc, li);
                }
                w = mis_weight(mode, s.prev_pdf, pa * h.t * h.t / vx.cog);
            }
        }
        s.L = s.L + mul(s.beta, Le) * w;
    }
    if (last) return 0;
    const Material m = load_material(sc, mid);
    return scatter<kLb, Mix>(P, s, vx, m, nee, pk, sh, graw, alpha, rec, glo, ghi, mix);
}

// Vertex 1 of an irradiance-probe path (Sec. 4.2): a virtual white
// Lambertian point at `pos` facing `nrm` (albedo 1, geometric and shading
// normal nrm, wo = nrm) that emits nothing, so its outgoing radiance is E / pi;
// the caller starts the path with throughput pi, so that the path's radiance
// estimates the irradiance E. Everything after it is a camera path's.
RT_HD int probe_vertex(const RenderParams &P, PathState &s, V3 pos, V3 nrm, ShadowRay &sh) {
    const DevScene &sc = P.sc;
    const bool nee = (sc.num_lights > 0 || sc.p_env > 0.f) && P.mis_mode != 3;
    NeePick pk;
    if (nee) pk = nee_pick(P, s.index, 2 + 7 * (int)(s.depth - 1));
    Vertex vx;
    vx.x = pos;
    vx.ng = nrm;
    vx.ns = nrm;
    vx.nsr = nrm;
    vx.wo = nrm;
    vx.cog = 1.f;
    Material m;
    m.albedo = v3(1.f, 1.f, 1.f);
    m.alpha = 1.f;
    m.w = 0.f;
    return scatter(P, s, vx, m, nee, pk, sh, nullptr, 0.f, nullptr, float3{0.f, 0.f, 0.f}, float3{1.f, 1.f, 1.f});
}

// Whole path in one thread: the megakernel body (Sec. 3.1 hybrid scheme)
// and the host debug path.
#pragma nv_exec_check_disable
template <class TraceClosest, class TraceAny>
RT_HD void finish_path(const RenderParams &P, PathState &s, TraceClosest closest, TraceAny any,
                       uint32_t &ext_rays, uint32_t &shadow_rays) {
    for (;;) {
        Hit h;
        closest(s.o, s.d, h);
        ++ext_rays;
        ShadowRay sh;
        int r = shade(P, s, h, sh);
        if (r & 2) {
            ++shadow_rays;
            if (!any(sh.o, sh.d, sh.tmax)) s.L = s.L + sh.contrib;
        }
        if (!(r & 1)) break;
    }
}

}  // namespace rtg
