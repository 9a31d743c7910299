// Two-way path tracing (paper Sec. 2): the forward path tracer and a light
// tracer run as separate stages with the same number of paths per iteration
// and are combined by multiple importance sampling. The light tracer starts
// on the environment with next-event estimation's probability p_env (a
// direction from the plain pyramid) or on a triangle emitter in proportion to
// its flux, aims the photon at a cluster of objects picked for the camera's
// view (Sec. 2.1.3, aiming.cuh) or, as an A/B option, emits uniformly over
// the scene's bound, and connects every vertex of a light path to the
// pinhole camera, adding the connection to the pixels whose filter reaches
// the image point.
//
// Techniques for a path x0 (eye) .. xk (triangle emitter, or a direction
// towards the environment), k >= 2, through pixel j: the camera path's
// BSDF-sampled hit of xk, next-event estimation at x(k-1), and the light path
// xk .. x1 connected to x0; one camera path per pixel against W H light
// paths per iteration; power or balance heuristic. Paths with k = 1 (an
// emitter or the sky seen directly) keep the path tracer's weights.
//
// Neither side stores its path. Each keeps two numbers between vertices:
//  - camera side: Pi, the product over the finished vertices x1 .. x(v-1)
//    of (light-tracer density / camera density) in area measure, and
//    c = |cos(ng, wi)| / C_v of the current vertex (C_v its camera density,
//    wi its continuation); the light tracer's density of x_v needs the
//    direction from x(v+1), so its ratio is finished one vertex later with
//    the reverse BSDF pdf there;
//  - light side: S, the sum over the two camera techniques of the product
//    of (camera density / light-tracer density)^beta over the finished
//    vertices, and pend = |cos(ng, wo)| / L_i of the current vertex (L_i
//    its light-tracer density, wo the direction it leaves to); the camera
//    density of x(i+1) needs the BSDF pdf at x_i with its camera-side
//    direction, known once x_i chooses where to go (the eye or a sample).
// The pixel-dependent factor of x1 enters last.
#include <algorithm>
#include <vector>
#include "internal.h"
#include "shade.cuh"
#include "aiming.cuh"

namespace rtg {

struct TwParams {
    float nL;         // light paths per iteration (W H): the light tracer's sample count
    float f2;         // focal length in pixels, squared
    float R;          // splat radius in pixels (3 sigma); <= 0: box filter
    int base;         // first light-path sample dimension
    int lt_mode;      // 0: MIS; 1: the light tracer alone wherever it makes the path
    V3 bc;            // the scene's bounding sphere: centre,
    float br;         // radius (half the diagonal of its box),
    float inv_disk;   // 1 / (pi br^2): area density of an environment photon's disk (uniform emission)
    int aim;          // photon aiming (Sec. 2.1.3) instead of uniform emission
    float4 aim_eye;   // eye position and the solid angle of the camera's view cone
};

// Density per unit area across w of an environment photon's line through x:
// aimed (the clusters whose spheres the line meets) or uniform over the
// scene's bounding sphere.
RT_D float tw_env_across(const DevScene &sc, const TwParams &T, V3 x, V3 w) {
    return T.aim ? aim_env_density(sc, T.aim_eye, x, w) : T.inv_disk;
}

// Solid-angle density of a triangle photon from y (emitter normal ny) along
// w: aimed, or cosine-distributed.
RT_D float tw_emit_dir(const DevScene &sc, const TwParams &T, V3 y, V3 ny, V3 w) {
    if (T.aim) return aim_dir_density(sc, T.aim_eye, y, ny, w);
    return fmaxf(dot(w, ny), 0.f) * (1.f / kPi);
}

struct TwCounters {
    unsigned long long ext_rays, shadow_rays;
};

// Heuristic weight of a technique whose density is 1 against two others
// (already scaled by sample counts, relative to it).
RT_HD float tw_weight(int mode, float a, float b) {
    a = fminf(a, 1e30f);
    b = fminf(b, 1e30f);
    if (mode == 1) return 1.f / (1.f + a + b);
    return 1.f / (1.f + a * a + b * b);
}

// Solid-angle pdf of the BSDF sampler at a vertex (geometric normal ng,
// shading normal nsr before adaptation, either side) given wo, for wi:
// normals turned to wo, shading normal adapted for wo (Appendix A.3), zero
// below the geometric tangent plane.
RT_HD float tw_dir_pdf(const Material &m, V3 ng, V3 nsr, V3 wo, V3 wi) {
    if (dot(wo, ng) < 0.f) ng = -ng;
    if (!(dot(wi, ng) > 0.f)) return 0.f;
    if (dot(nsr, ng) < 0.f) nsr = -nsr;
    V3 ns = adapt_shading_normal(nsr, ng, wo);
    V3 f;
    float pdf;
    bsdf_eval(m, ns, wo, wi, f, pdf);
    return pdf;
}

// Image point (pixels) of x and the cosine to the optical axis.
RT_HD bool tw_project(const CameraView &c, V3 x, float &sx, float &sy, float &cz) {
    V3 d = normalize(x - c.eye);
    cz = dot(d, c.fwd);
    if (!(cz > 0.f)) return false;
    float nx = dot(d, c.right) / cz, ny = dot(d, c.up) / cz;
    sx = 0.5f * (float)c.W * (1.f + nx / (c.tan_half * c.aspect));
    sy = 0.5f * (float)c.H * (1.f - ny / c.tan_half);
    return true;
}

// Filter density per pixel^2 at offset (dx, dy) from a pixel centre; `ok`:
// the light tracer connects to that pixel.
RT_HD float tw_filter(float sigma, float R, float dx, float dy, bool &ok) {
    if (!(sigma > 0.f)) {
        ok = dx >= -0.5f && dx < 0.5f && dy >= -0.5f && dy < 0.5f;
        return ok ? 1.f : 0.f;
    }
    float r2 = dx * dx + dy * dy;
    ok = r2 <= R * R;
    return expf(-r2 / (2.f * sigma * sigma)) / (2.f * kPi * sigma * sigma);
}

// ------------------------------------------------------------ camera stage
// One camera path (pixel, iteration j): the path tracer of shade()/scatter()
// without guiding, with the light tracer as a third technique in the weights
// of emitter and environment hits and of next-event samples.
RT_D V3 tw_camera_path(const RenderParams &P, const TwParams &T, uint32_t pixel, uint32_t j, uint32_t &ext,
                       uint32_t &shadow) {
    const DevScene &sc = P.sc;
    const int mode = P.mis_mode;
    PathState s;
    raygen(P, pixel, j, s);
    const float px = (float)(pixel % P.cam.W) + 0.5f, py = (float)(pixel / P.cam.W) + 0.5f;
    float Pi = 1.f, cprev = 0.f;
    for (;;) {
        Hit h;
        {
            Ray r{s.o, s.d, 0.f, INFINITY};
            h.prim = RT_MISS; h.inst = 0; h.t = INFINITY; h.b1 = h.b2 = 0.f;
            trace_scene<false>(sc, r, h);
        }
        ++ext;
        const uint32_t v = s.depth;
        if (h.prim == RT_MISS) {
            if (sc.env_w > 0) {
                int tx = env_texel(sc, s.d);
                float4 e = ldg(sc.env + tx);
                float w = 1.f;
                if (v > 1 && sc.p_env > 0.f) {
                    const float pn = sc.p_env * e.w * env_cell_factor(sc, s.prev_cell, tx);
                    // light tracer / hit: x(v-1)'s factor, |cos| / (pi r^2) over
                    // its camera density, times the photon's direction pdf
                    // over the continuation's
                    const float r_lt =
                        Pi > 0.f ? T.nL * Pi * cprev * tw_env_across(sc, T, s.o, s.d) * sc.p_env * e.w / s.prev_pdf : 0.f;
                    if (T.lt_mode == 1) w = r_lt > 0.f ? 0.f : mis_weight(mode, s.prev_pdf, pn);
                    else w = tw_weight(mode, pn / s.prev_pdf, r_lt);
                }
                s.L = s.L + mul(s.beta, v3(e.x, e.y, e.z)) * w;
            }
            break;
        }
        const uint32_t prim = h.prim;
        const uint32_t mid = ldg(sc.tri_material + prim);
        const float lpa = ldg(sc.tri_light_pdf_area + prim);
        Vertex vx;
        setup_vertex(sc, s, h, vx);
        const float cA = fabsf(vx.cog);
        const float t2 = h.t * h.t;
        // camera density of this vertex (area measure)
        float Cd;
        if (v == 1) {
            float sx, sy, cz;
            bool ok = false;
            Cd = 0.f;
            if (tw_project(P.cam, vx.x, sx, sy, cz)) {
                float g = tw_filter(P.sigma, T.R, sx - px, sy - py, ok);
                Cd = g * T.f2 * cA / (cz * cz * cz * t2);
            }
            if (!ok || !(Cd > 0.f)) Pi = 0.f;
        } else {
            Cd = s.prev_pdf * cA / t2;
        }
        if (vx.cog > 0.f && lpa > 0.f) {
            V3 Le = tri_emission(sc, prim, mid, h.b1, h.b2);
            float w = 1.f;
            if (v > 1) {
                float pa = lpa;   // next-event estimation's area pdf of this point
                if (sc.lb_rec) {
                    // the light hierarchy's, from the previous vertex (its
                    // offset origin and stored normal), as in shade()
                    const uint32_t li = ldg(sc.lb_inst_base + h.inst) + ldg(sc.lb_tri_rank + prim);
                    pa = (1.f - sc.p_env) * lb_prob(sc, s.o, oct_decode(s.prev_n), li) / emitter_area(sc, li);
                }
                const float r_nee = pa * t2 / (s.prev_pdf * vx.cog);
                // light tracer / hit: the factor of x_v, q(y -> x_(v-1)) c / t^2
                // (q the emission's direction density), times the emitter's,
                // pA_lt t^2 / (prev_pdf cos_y)
                const float pa_lt = lpa;   // the light tracer's area pdf (alias table, 1 - p_env)
                float r_lt = 0.f;
                if (Pi > 0.f) {
                    const float qd = tw_emit_dir(sc, T, vx.x, vx.ng, vx.wo);
                    r_lt = T.nL * Pi * cprev * pa_lt * qd / (vx.cog * s.prev_pdf);
                }
                if (T.lt_mode == 1) w = r_lt > 0.f ? 0.f : mis_weight(mode, s.prev_pdf, pa * t2 / vx.cog);
                else w = tw_weight(mode, r_nee, r_lt);
            }
            s.L = s.L + mul(s.beta, Le) * w;
        }
        if (v == P.max_depth + 1) break;
        const Material m = load_material(sc, mid);
        const V3 x = vx.x, ng = vx.ng, ns = vx.ns, wo = vx.wo;
        const int base = 2 + 7 * (int)(v - 1);
        const V3 xo = offset_origin(x, ng);
        // next-event estimation
        if ((sc.num_lights > 0 || sc.p_env > 0.f) && mode != 3) {
            NeePick pk = nee_pick<false>(P, s.index, base);
            const float us = pk.us, ua = pk.ua, ub = pk.ub;
            V3 wi = v3(0.f, 0.f, 1.f), Le = v3(0.f, 0.f, 0.f), sdir = wi;
            float pdf_l = 0.f, tmax = INFINITY, cl = 0.f, dist = 0.f, lt_over_nee = 0.f, env_pw = 0.f;
            bool tri = false;
            V3 ly = v3(0.f, 0.f, 0.f), lnrm = v3(0.f, 0.f, 1.f);   // sampled light point and its normal
            if (us < sc.p_env) {
                const uint32_t cell = env_cell(ng);
                wi = env_sample_cell(sc, cell, ua, ub);
                sdir = wi;
                const int tx = env_texel(sc, wi);
                float4 e = ldg(sc.env + tx);
                Le = v3(e.x, e.y, e.z);
                pdf_l = sc.p_env * e.w * env_cell_factor(sc, cell, tx);
                env_pw = e.w;
            } else {
                V3 l0 = pk.l0, l1 = pk.l1, l2 = pk.l2;
                uint32_t lt = pk.lt, lmid = pk.lmid;
                float lpa_n = pk.lpa;
                if (sc.lb_rec) {
                    float Pp;
                    const uint32_t li =
                        lb_sample(sc, xo, oct_decode(oct_encode(ng)), (us - sc.p_env) / (1.f - sc.p_env), Pp);
                    const float4 *LV = sc.light_v + 3 * (size_t)li;
                    l0 = f4xyz(ldg(LV));
                    l1 = f4xyz(ldg(LV + 1));
                    l2 = f4xyz(ldg(LV + 2));
                    lt = ldg(sc.light_tri + li);
                    lmid = ldg(sc.tri_material + lt);
                    lpa_n = (1.f - sc.p_env) * Pp / (0.5f * length(cross(l1 - l0, l2 - l0)));
                }
                float sq = sqrtf(ua);
                float lb1 = sq * (1.f - ub), lb2 = sq * ub;
                V3 y = (1.f - sq) * l0 + lb1 * l1 + lb2 * l2;
                V3 dv = y - x;
                dist = length(dv);
                if (dist > 0.f) {
                    wi = dv * (1.f / dist);
                    V3 lng = normalize(cross(l1 - l0, l2 - l0));
                    ly = y;
                    lnrm = lng;
                    cl = -dot(wi, lng);
                    if (cl > 0.f) {
                        pdf_l = lpa_n * dist * dist / cl;
                        Le = tri_emission(sc, lt, lmid, lb1, lb2);
                        V3 sv = y - xo;
                        float sl = length(sv);
                        if (sl > 0.f) {
                            sdir = sv * (1.f / sl);
                            tmax = sl * (1.f - kShadowEps);
                            tri = true;
                            // the light tracer's area pdf of the point (alias
                            // table) over next-event estimation's
                            lt_over_nee = ldg(sc.tri_light_pdf_area + lt) / lpa_n;
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
                if (pdf_b > 0.f) {
                    float w = mode == 2 ? 1.f : mis_weight(mode, pdf_l, pdf_b);
                    if (tri) {
                        float r_lt = 0.f;
                        if (Pi > 0.f) {
                            // x(v-1): reverse pdf at x_v from the light point
                            float fv1 = 1.f;
                            if (v >= 2) fv1 = tw_dir_pdf(m, ng, vx.nsr, wi, wo) * cprev / t2;
                            // x_v: the emission's direction density from y
                            // towards x_v, cos at x_v towards y
                            const float fv = tw_emit_dir(sc, T, ly, lnrm, -wi) * dot(wi, ng) / (dist * dist * Cd);
                            r_lt = T.nL * Pi * fv1 * fv * lt_over_nee;
                        }
                        if (T.lt_mode == 1) w = r_lt > 0.f ? 0.f : w;
                        else w = tw_weight(mode, pdf_b / pdf_l, r_lt);
                    } else {
                        // an environment direction: x_v's factor |cos| / (pi r^2)
                        // over its camera density, the photon's direction pdf
                        // over NEE's
                        float r_lt = 0.f;
                        if (Pi > 0.f) {
                            float fv1 = 1.f;
                            if (v >= 2) fv1 = tw_dir_pdf(m, ng, vx.nsr, wi, wo) * cprev / t2;
                            r_lt = T.nL * Pi * fv1 * (dot(wi, ng) * tw_env_across(sc, T, vx.x, wi) / Cd) * sc.p_env *
                                   env_pw / pdf_l;
                        }
                        if (T.lt_mode == 1) w = r_lt > 0.f ? 0.f : w;
                        else w = tw_weight(mode, pdf_b / pdf_l, r_lt);
                    }
                    const float k = dot(wi, ns) * w / pdf_l;
                    V3 contrib = mul(mul(s.beta, f), Le) * k;
                    if (contrib.x > 0.f || contrib.y > 0.f || contrib.z > 0.f) {
                        Ray r{xo, sdir, 0.f, tmax};
                        Hit hs;
                        hs.prim = RT_MISS; hs.t = INFINITY;
                        trace_scene<true>(sc, r, hs);
                        ++shadow;
                        if (hs.prim == RT_MISS) s.L = s.L + contrib;
                    }
                }
            }
        }
        // continuation
        V3 wi, f;
        float pdf;
        if (!bsdf_sample(m, ns, wo, dim_value(P, s.index, base + 3), dim_value(P, s.index, base + 4),
                         dim_value(P, s.index, base + 5), wi, f, pdf))
            break;
        if (dot(wi, ng) <= 0.f) break;
        if (Pi > 0.f && v >= 2) Pi = fminf(Pi * tw_dir_pdf(m, ng, vx.nsr, wi, wo) * cprev / t2, 1e30f);
        cprev = dot(wi, ng) / Cd;
        s.beta = mul(s.beta, f) * (dot(wi, ns) / pdf);
        if (P.rr && v >= 3) {
            float q = fmaxf(0.05f, 1.f - maxc(s.beta));
            if (dim_value(P, s.index, base + 6) < q) break;
            s.beta = s.beta * (1.f / (1.f - q));
        }
        if (s.beta.x == 0.f && s.beta.y == 0.f && s.beta.z == 0.f) break;
        s.prev_pdf = pdf;
        s.prev_cell = env_cell(ng);
        s.prev_n = oct_encode(ng);
        s.o = xo;
        s.d = wi;
        s.depth = v + 1;
    }
    return s.L;
}

__global__ void __launch_bounds__(128) k_tw_camera(RenderParams P, TwParams T, double *sum, double *sum2,
                                                   uint32_t *count, uint32_t j0, uint64_t n, TwCounters *ctr) {
    const uint32_t WH = P.cam.W * P.cam.H;
    uint32_t ext = 0, shadow = 0;
    for (uint64_t task = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; task < n;
         task += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t pixel = (uint32_t)(task % WH), j = j0 + (uint32_t)(task / WH);
        V3 L = tw_camera_path(P, T, pixel, j, ext, shadow);
        double *sp = sum + 3 * (size_t)pixel, *sq = sum2 + 3 * (size_t)pixel;
        atomicAdd(sp, (double)L.x);
        atomicAdd(sp + 1, (double)L.y);
        atomicAdd(sp + 2, (double)L.z);
        atomicAdd(sq, (double)L.x * L.x);
        atomicAdd(sq + 1, (double)L.y * L.y);
        atomicAdd(sq + 2, (double)L.z * L.z);
        atomicAdd(count + pixel, 1u);
    }
    ext = __reduce_add_sync(0xFFFFFFFFu, ext);
    shadow = __reduce_add_sync(0xFFFFFFFFu, shadow);
    if (lane_id() == 0) {
        atomicAdd(&ctr->ext_rays, (unsigned long long)ext);
        atomicAdd(&ctr->shadow_rays, (unsigned long long)shadow);
    }
}

// ------------------------------------------------------------- light stage
// Light path m (iteration m / (W H)): the environment with next-event
// estimation's probability, else an emitter by the alias table and a point
// uniform on it; with photon aiming (Sec. 2.1.3) a cluster picked through
// the cluster hierarchy with the eye's view, then a uniform point of that
// cluster's disk across the environment direction, or a direction uniform in
// the cone its sphere subtends from the emitter point; without, a point of
// the disk across the scene's bounding sphere or a cosine direction. At
// vertex t = 1..D a connection to the eye, then (t < D) a BSDF sample with
// the arriving direction as wo. Sample dimensions from T.base: {0: emitter,
// 1,2: point (environment: direction), 3,4: direction (environment: disk
// point), 5: cluster}, vertex t: T.base + 6 + 3 (t - 1) + {0: lobe, 1,2:
// direction}.
RT_D void tw_light_path(const RenderParams &P, const TwParams &T, uint64_t m, double *splat, uint32_t &ext,
                        uint32_t &shadow) {
    const DevScene &sc = P.sc;
    const CameraView &cam = P.cam;
    const int mode = P.mis_mode;
    const float beta_exp = mode == 1 ? 1.f : 2.f;
    // emission: the environment with next-event estimation's probability
    // p_env, else a triangle emitter by flux
    const float us = dim_value(P, m, T.base);
    const float ua = dim_value(P, m, T.base + 1), ub = dim_value(P, m, T.base + 2);
    const float u3 = dim_value(P, m, T.base + 3), u4 = dim_value(P, m, T.base + 4);
    const float uc = dim_value(P, m, T.base + 5);
    const bool aim = T.aim != 0;
    float sphi, cphi;
    sincosf(2.f * kPi * u4, &sphi, &cphi);
    const bool env = us < sc.p_env;
    V3 beta, o, dir;
    float pa;            // the light tracer's pdf of the emission: area (triangle) or solid angle (environment)
    float q_prev = 0.f;  // pdf of the direction that made the pending ray (triangle emission)
    float pend = 0.f;    // |cos| at the previous vertex toward this one over its light density
    uint32_t li = 0, lt = 0;
    float env_pw = 0.f;
    if (env) {
        // a direction w from the plain pyramid, a uniform point of the disk
        // of radius br across the bounding sphere, travelling along -w
        const V3 w = env_sample(sc, ua, ub);
        const float4 e = ldg(sc.env + env_texel(sc, w));
        env_pw = e.w;
        if (!(env_pw > 0.f)) return;
        pa = sc.p_env * env_pw;
        V3 t1, t2;
        onb(w, t1, t2);
        if (aim) {
            // a uniform point of the chosen cluster's disk across w, moved
            // back along w outside the scene; the line density at the first
            // hit completes the throughput there
            const float4 sph = aim_sample(sc, T.aim_eye, false, w, w, uc);
            const float r = sph.w * sqrtf(u3);
            const V3 p = v3(sph.x, sph.y, sph.z) + (r * cphi) * t1 + (r * sphi) * t2;
            o = p + (length(p - T.bc) + T.br) * w;
            beta = v3(e.x, e.y, e.z) * (1.f / pa);
        } else {
            const float r = T.br * sqrtf(u3);
            o = T.bc + (2.f * T.br) * w + (r * cphi) * t1 + (r * sphi) * t2;
            beta = v3(e.x, e.y, e.z) * (1.f / (pa * T.inv_disk));
        }
        dir = -w;
    } else {
        float u2 = (us - sc.p_env) / (1.f - sc.p_env);
        float xn = u2 * (float)sc.num_lights;
        uint32_t bin = (uint32_t)xn;
        if (bin >= sc.num_lights) bin = sc.num_lights - 1;
        const float frac = xn - (float)bin;
        const float2 al = ldg(sc.alias + bin);
        li = frac < al.x ? bin : as_uint(al.y);
        lt = ldg(sc.light_tri + li);
        const float4 *LV = sc.light_v + 3 * (size_t)li;
        const V3 l0 = f4xyz(ldg(LV)), l1 = f4xyz(ldg(LV + 1)), l2 = f4xyz(ldg(LV + 2));
        const float sq = sqrtf(ua);
        const float lb1 = sq * (1.f - ub), lb2 = sq * ub;
        const V3 y = (1.f - sq) * l0 + lb1 * l1 + lb2 * l2;
        const V3 lng = normalize(cross(l1 - l0, l2 - l0));
        pa = ldg(sc.tri_light_pdf_area + lt);   // (1 - p_env) x flux share / area
        const V3 Le = tri_emission(sc, lt, ldg(sc.tri_material + lt), lb1, lb2);
        if (aim) {
            const float4 sph = aim_sample(sc, T.aim_eye, true, y, lng, uc);
            dir = aim_cone_sample(sph, y, u3, u4);
            const float ce = dot(dir, lng);
            if (!(ce > 0.f)) return;   // behind the one-sided emitter: no power
            const float qd = aim_dir_density(sc, T.aim_eye, y, lng, dir);
            if (!(qd > 0.f)) return;
            beta = Le * (ce / (pa * qd));
            q_prev = qd;
            pend = ce / pa;
        } else {
            const float ce = sqrtf(fmaxf(0.f, 1.f - u3));
            if (!(ce > 0.f)) return;
            V3 t1, t2;
            onb(lng, t1, t2);
            const float rr = sqrtf(u3);
            dir = normalize(rr * cphi * t1 + rr * sphi * t2 + ce * lng);
            beta = Le * (kPi / pa);
            q_prev = ce / kPi;
            pend = ce / pa;
        }
        o = offset_origin(y, lng);
    }
    float S = 0.f;               // sum over camera techniques of prod (C / L)^beta, finished vertices
    for (uint32_t t = 1; t <= P.max_depth; ++t) {
        Hit h;
        {
            Ray r{o, dir, 0.f, INFINITY};
            h.prim = RT_MISS; h.inst = 0; h.t = INFINITY; h.b1 = h.b2 = 0.f;
            trace_scene<false>(sc, r, h);
        }
        ++ext;
        if (h.prim == RT_MISS) return;
        PathState ps;
        ps.d = dir;
        Vertex vx;
        setup_vertex(sc, ps, h, vx);   // ng, nsr turned to the arriving side; ns adapted for it
        const V3 x = vx.x, ng = vx.ng, wi = vx.wo;
        const float cwi = fabsf(vx.cog);
        const float t2 = h.t * h.t;
        // light-tracer density of x (given the direction, for an environment photon)
        float across = T.inv_disk;
        if (t == 1 && env && aim) {
            across = aim_env_density(sc, T.aim_eye, x, -dir);
            if (!(across > 0.f)) return;
            beta = beta * (1.f / across);
        }
        const float Ld = (t == 1 && env) ? cwi * across : q_prev * cwi / t2;
        // factor that turns the BSDF pdf at x towards the previous vertex into
        // (camera density / light density) of that vertex
        const float gfac = (t == 1 && env) ? 1.f / pa : pend / t2;
        const Material mat = load_material(sc, ldg(sc.tri_material + h.prim));
        const V3 xo = offset_origin(x, ng);
        // p_light of the emitter from x (next-event estimation's area pdf)
        float G_nee = 0.f;
        if (t == 1 && env) {
            // next-event estimation's solid-angle pdf of the photon's direction from x
            const uint32_t cell = env_cell(ng);
            G_nee = sc.p_env * env_pw * env_cell_factor(sc, cell, env_texel(sc, wi)) / pa;
        } else if (t == 1) {
            // next-event estimation's area pdf of the emission point from x
            float pl = ldg(sc.tri_light_pdf_area + lt);
            if (sc.lb_rec) pl = (1.f - sc.p_env) * lb_prob(sc, xo, oct_decode(oct_encode(ng)), li) / emitter_area(sc, li);
            G_nee = pl / pa;
        }
        // connection to the eye
        const V3 te = cam.eye - x;
        const float re2 = dot(te, te);
        const V3 we = te * (1.f / sqrtf(re2));
        float sx, sy, cz;
        if (dot(we, ng) > 0.f && tw_project(cam, x, sx, sy, cz) && sx > -T.R - 2.f && sx < (float)cam.W + T.R + 2.f &&
            sy > -T.R - 2.f && sy < (float)cam.H + T.R + 2.f) {
            const V3 nsa = adapt_shading_normal(vx.nsr, ng, we);
            V3 f;
            float b_i;
            bsdf_eval(mat, nsa, we, wi, f, b_i);
            if (f.x > 0.f || f.y > 0.f || f.z > 0.f) {
                const V3 sv = cam.eye - xo;
                const float sl = length(sv);
                bool vis = false;
                if (sl > 0.f) {
                    Ray r{xo, sv * (1.f / sl), 0.f, sl * (1.f - kShadowEps)};
                    Hit hs;
                    hs.prim = RT_MISS; hs.t = INFINITY;
                    trace_scene<true>(sc, r, hs);
                    ++shadow;
                    vis = hs.prim == RT_MISS;
                }
                if (vis) {
                    const float G = b_i * gfac;
                    const float Sc = t == 1 ? powf(G, beta_exp) + powf(G_nee, beta_exp) : S * powf(G, beta_exp);
                    const float c1 = dot(we, ng);
                    const V3 base_c = mul(beta, f) * (fabsf(dot(wi, nsa)) / cwi);
                    const float We0 = T.f2 * c1 / (cz * cz * cz * re2);
                    int x0, x1, y0, y1;
                    if (T.R > 0.f) {
                        x0 = (int)floorf(sx - 0.5f - T.R); x1 = (int)ceilf(sx - 0.5f + T.R);
                        y0 = (int)floorf(sy - 0.5f - T.R); y1 = (int)ceilf(sy - 0.5f + T.R);
                    } else {
                        x0 = x1 = (int)floorf(sx);
                        y0 = y1 = (int)floorf(sy);
                    }
                    x0 = max(x0, 0); y0 = max(y0, 0);
                    x1 = min(x1, (int)cam.W - 1); y1 = min(y1, (int)cam.H - 1);
                    for (int yy = y0; yy <= y1; ++yy)
                        for (int xx = x0; xx <= x1; ++xx) {
                            bool ok;
                            const float g = tw_filter(P.sigma, T.R, sx - ((float)xx + 0.5f), sy - ((float)yy + 0.5f), ok);
                            if (!ok) continue;
                            const float We = g * We0;   // also the camera density of x through this pixel
                            float w = 1.f;
                            if (T.lt_mode == 0) {
                                const float g1 = We / (Ld * T.nL);
                                const float rsum = fminf(Sc * powf(g1, beta_exp), 1e30f);
                                w = 1.f / (1.f + rsum);
                            }
                            const V3 c = base_c * (w * We / T.nL);
                            double *dst = splat + 3 * ((size_t)yy * cam.W + (size_t)xx);
                            atomicAdd(dst, (double)c.x);
                            atomicAdd(dst + 1, (double)c.y);
                            atomicAdd(dst + 2, (double)c.z);
                        }
                }
            }
        }
        if (t == P.max_depth) return;
        // continuation: the BSDF sampler with the arriving direction as wo
        const int bb = T.base + 6 + 3 * (int)(t - 1);
        V3 wn, fs;
        float q;
        if (!bsdf_sample(mat, vx.ns, wi, dim_value(P, m, bb), dim_value(P, m, bb + 1), dim_value(P, m, bb + 2), wn,
                         fs, q))
            return;
        if (!(dot(wn, ng) > 0.f)) return;
        const V3 nsn = adapt_shading_normal(vx.nsr, ng, wn);
        V3 fc;
        float b_n;
        bsdf_eval(mat, nsn, wn, wi, fc, b_n);
        const float G = b_n * gfac;
        S = t == 1 ? powf(G, beta_exp) + powf(G_nee, beta_exp) : S * powf(G, beta_exp);
        S = fminf(S, 1e30f);
        beta = mul(beta, fc) * (fabsf(dot(wi, nsn)) / cwi * dot(wn, ng) / q);
        if (beta.x == 0.f && beta.y == 0.f && beta.z == 0.f) return;
        pend = dot(wn, ng) / Ld;
        q_prev = q;
        o = xo;
        dir = wn;
    }
}

__global__ void __launch_bounds__(128) k_tw_light(RenderParams P, TwParams T, double *splat, uint64_t m0, uint64_t n,
                                                  TwCounters *ctr) {
    uint32_t ext = 0, shadow = 0;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        tw_light_path(P, T, m0 + i, splat, ext, shadow);
    ext = __reduce_add_sync(0xFFFFFFFFu, ext);
    shadow = __reduce_add_sync(0xFFFFFFFFu, shadow);
    if (lane_id() == 0) {
        atomicAdd(&ctr->ext_rays, (unsigned long long)ext);
        atomicAdd(&ctr->shadow_rays, (unsigned long long)shadow);
    }
}

}  // namespace rtg

using namespace rtg;

extern "C" rt_status rt_render_two_way(const rt_scene *s, const rt_camera *cam, uint32_t spp, uint32_t max_depth,
                                       rt_film *film, const rt_render_opts *opts_in, int32_t lt_mode,
                                       double *lt_splat, rt_stats *stats, void *stream) {
    if (!s || !cam || !film) { set_error("rt_render_two_way: null argument"); return RT_INVALID_ARG; }
    if (s->host_only) { set_error("rt_render_two_way: scene has no device copy"); return RT_INVALID_ARG; }
    if (cam->width != film->W || cam->height != film->H) {
        set_error("rt_render_two_way: camera and film sizes differ");
        return RT_INVALID_ARG;
    }
    if (max_depth < 1 || max_depth > (uint32_t)kMaxDepth) {
        set_error("rt_render_two_way: max_depth must be in [1, 64]");
        return RT_INVALID_ARG;
    }
    rt_render_opts o{};
    if (opts_in) o = *opts_in;
    if (o.mis_mode != 0 && o.mis_mode != 1) {
        set_error("rt_render_two_way: mis_mode must be 0 (power) or 1 (balance)");
        return RT_INVALID_ARG;
    }
    if (lt_mode < 0 || lt_mode > 1) { set_error("rt_render_two_way: lt_mode must be 0 or 1"); return RT_INVALID_ARG; }
    if (o.lt_emission < 0 || o.lt_emission > 1) {
        set_error("rt_render_two_way: lt_emission must be 0 (photon aiming) or 1 (uniform)");
        return RT_INVALID_ARG;
    }
    if (o.guide) { set_error("rt_render_two_way: guiding is not combined with light tracing"); return RT_NOT_SUPPORTED; }
    const uint64_t WH = (uint64_t)cam->width * cam->height;
    if (film->next_task % WH) {
        set_error("rt_render_two_way: the film must hold whole passes");
        return RT_INVALID_ARG;
    }
    if (stats) *stats = rt_stats{};
    if (spp == 0) return RT_OK;
    const uint64_t j0 = film->next_task / WH;
    if (j0 + spp > 0xFFFFFFFFull) { set_error("rt_render_two_way: iteration index overflow"); return RT_INVALID_ARG; }
    cudaStream_t st = (cudaStream_t)stream;
    const int base = 2 + 7 * (int)(max_depth + 1);
    const int ndims = base + 6 + 3 * (int)max_depth;
    std::vector<HaltonDim> dims = make_dims(o.seed, ndims);
    // the dimension table and counters live for this call only; every exit
    // path, the error returns included, releases them on the stream
    struct Scoped {
        void *p = nullptr;
        cudaStream_t st;
        ~Scoped() { if (p) cudaFreeAsync(p, st); }
    } dd_mem{nullptr, st}, ctr_mem{nullptr, st};
    RT_CUDA_TRY(cudaMallocAsync(&dd_mem.p, dims.size() * sizeof(HaltonDim), st));
    RT_CUDA_TRY(cudaMallocAsync(&ctr_mem.p, sizeof(TwCounters), st));
    HaltonDim *dd = (HaltonDim *)dd_mem.p;
    TwCounters *ctr = (TwCounters *)ctr_mem.p;
    RT_CUDA_TRY(cudaMemcpyAsync(dd, dims.data(), dims.size() * sizeof(HaltonDim), cudaMemcpyHostToDevice, st));
    RT_CUDA_TRY(cudaMemsetAsync(ctr, 0, sizeof(TwCounters), st));
    RenderParams P;
    P.sc = s->dev;
    P.cam = make_camera(*cam);
    P.en = make_enum(cam->width, cam->height);
    P.dims = dd;
    P.max_depth = max_depth;
    P.sigma = o.filter_sigma == 0.f ? 0.5f : o.filter_sigma;
    P.mis_mode = o.mis_mode;
    P.rr = o.rr_enable;
    TwParams T;
    T.nL = (float)WH;
    const float f = (float)cam->height / (2.f * P.cam.tan_half);
    T.f2 = f * f;
    T.R = P.sigma > 0.f ? 3.f * P.sigma : 0.f;
    T.base = base;
    T.lt_mode = lt_mode;
    {
        const float3 lo = s->dev.bb_lo, hi = s->dev.bb_hi;
        const double dx = (double)hi.x - lo.x, dy = (double)hi.y - lo.y, dz = (double)hi.z - lo.z;
        const double r = 0.5 * std::sqrt(dx * dx + dy * dy + dz * dz);
        T.bc = v3((float)(0.5 * ((double)lo.x + hi.x)), (float)(0.5 * ((double)lo.y + hi.y)),
                  (float)(0.5 * ((double)lo.z + hi.z)));
        T.br = r > 0.0 ? (float)r : 1.f;
        T.inv_disk = (float)(1.0 / (3.14159265358979323846 * (double)T.br * T.br));
    }
    // photon aiming: on unless uniform emission is asked for (A/B); the eye
    // and the solid angle of the view cone through the image corners
    T.aim = (o.lt_emission == 0 && s->dev.pa_nnodes > 0) ? 1 : 0;
    {
        const double th = std::tan(0.5 * (double)cam->vfov_deg * 3.14159265358979323846 / 180.0);
        const double asp = (double)cam->width / (double)cam->height;
        const double tc = th * std::sqrt(1.0 + asp * asp);
        const double om = 2.0 * 3.14159265358979323846 * (1.0 - 1.0 / std::sqrt(1.0 + tc * tc));
        T.aim_eye = make_float4(cam->eye[0], cam->eye[1], cam->eye[2], (float)om);
    }
    const uint64_t n = (uint64_t)spp * WH;
    // One path per thread: with several paths per thread the lanes of a warp
    // drift apart (each starts its next path whenever its last one ends) and
    // the warp runs their different phases one after another.
    const int grid = (int)std::min<uint64_t>((n + 127) / 128, 0x7FFFFFFFull);
    k_tw_camera<<<grid, 128, 0, st>>>(P, T, film->sum, film->sum2, film->count, (uint32_t)j0, n, ctr);
    RT_CUDA_TRY(cudaGetLastError());
    if (P.sc.num_lights > 0 || P.sc.p_env > 0.f) {
        double *dst = lt_splat ? lt_splat : film->sum;
        k_tw_light<<<grid, 128, 0, st>>>(P, T, dst, j0 * WH, n, ctr);
        RT_CUDA_TRY(cudaGetLastError());
    }
    TwCounters hc{};
    RT_CUDA_TRY(cudaMemcpyAsync(&hc, ctr, sizeof(TwCounters), cudaMemcpyDeviceToHost, st));
    dd_mem.p = ctr_mem.p = nullptr;
    RT_CUDA_TRY(cudaFreeAsync(dd, st));
    RT_CUDA_TRY(cudaFreeAsync(ctr, st));
    RT_CUDA_TRY(cudaStreamSynchronize(st));
    film->next_task += n;
    if (stats) {
        stats->paths = n;
        stats->extension_rays = hc.ext_rays;
        stats->shadow_rays = hc.shadow_rays;
        stats->waves = 1;
        stats->kernel_launches = (P.sc.num_lights > 0 || P.sc.p_env > 0.f) ? 2 : 1;
    }
    return RT_OK;
}
