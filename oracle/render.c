/*
 * Oracle: the camera-path estimator with next-event estimation and multiple
 * importance sampling, written out sample by sample in FP64 (paper Sec. 2
 * "forward path tracer ... next event estimation ... combined using MIS",
 * Sec. 2.1 light importance sampling, Appendix A.1 filter importance
 * sampling, Appendix A.2 QMC sample enumeration, Appendix A.4 per-pixel
 * sample counts).
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Readings fixed where the paper is silent:
 *   - max_depth D = number of scattering vertices; vertices 1..D do NEE and
 *     sample a continuation, vertex D+1 only adds its emission;
 *   - MIS = power heuristic (beta = 2) between NEE and BSDF sampling;
 *   - Gaussian filter sigma = 0.5 px (3 sigma covers a 3 x 3 pixel block),
 *     Box-Muller on the in-pixel offset, the sample credits its own pixel;
 *   - dimensions: 0,1 in-pixel offset; bounce v (1-based) uses dimensions
 *     2 + 7(v-1) + {0: light select, 1,2: light point, 3: lobe select,
 *     4,5: direction, 6: Russian roulette};
 *   - a continuation or light direction below the geometric tangent plane
 *     (seen from wo) carries nothing; the BSDF is zero outside the shading
 *     hemisphere; a shadow ray to a triangle runs from the offset origin to
 *     the light point and stops at (1 - 1e-4) of that length; ray origins
 *     move off the surface along the geometric normal.
 */
#include "oracle.h"
#include "oracle_internal.h"
#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#define OR_PI 3.14159265358979323846
#define OR_SHADOW_EPS 1e-4

static double dot3(const double a[3], const double b[3]) {
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}
static void normalize3(double a[3]) {
    double l = sqrt(dot3(a, a));
    if (l > 0.0) { a[0] /= l; a[1] /= l; a[2] /= l; }
}
static void cross3(const double a[3], const double b[3], double c[3]) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

void or_camera_ray(const or_camera *c, double sx, double sy, double o[3],
                   double d[3]) {
    double fwd[3] = {c->look_at[0] - c->eye[0], c->look_at[1] - c->eye[1], c->look_at[2] - c->eye[2]};
    normalize3(fwd);
    double right[3], up[3];
    cross3(fwd, c->up, right);
    normalize3(right);
    cross3(right, fwd, up);
    double th = tan(0.5 * c->vfov_deg * OR_PI / 180.0);
    double asp = (double)c->width / (double)c->height;
    double nx = (2.0 * sx / (double)c->width - 1.0) * th * asp;
    double ny = (1.0 - 2.0 * sy / (double)c->height) * th;
    for (int a = 0; a < 3; ++a) {
        o[a] = c->eye[a];
        d[a] = fwd[a] + nx * right[a] + ny * up[a];
    }
    normalize3(d);
}

void or_filter_offset(double sigma, double u0, double u1, double *dx, double *dy) {
    if (!(sigma > 0.0)) { *dx = u0 - 0.5; *dy = u1 - 0.5; return; }
    double r = sigma * sqrt(-2.0 * log(1.0 - u0));
    double phi = 2.0 * OR_PI * u1;
    *dx = r * cos(phi);
    *dy = r * sin(phi);
}

static double mis_weight(int mode, double pa, double pb) {
    if (mode == 1) return pa / (pa + pb);
    double a = pa * pa, b = pb * pb;
    return a / (a + b);
}

void or_offset_origin(const double x[3], const double n[3], double out[3]) {
    double m = fmax(1.0, fmax(fabs(x[0]), fmax(fabs(x[1]), fabs(x[2]))));
    for (int a = 0; a < 3; ++a) out[a] = x[a] + n[a] * 1e-9 * m;
}

typedef struct {
    const or_scene *s;
    const or_camera *cam;
    const or_render_opts *opts;
    uint32_t k, l;
    uint32_t *factors; /* per dimension */
    int ndims;
    uint32_t D;
    /* two-way path tracing: the light tracer is a third MIS technique */
    int tw;            /* 1 + lt_mode of or_render_two_way, 0 = off */
    or_tw_cam tc;
} ctx_t;

/* Weight of a camera technique (density `mine`, the other camera technique
 * `other`) for a path the light tracer makes with density p_lt; W H light
 * paths per iteration against one camera path per pixel. */
static double tw_camera_weight(const ctx_t *c, double mine, double other, double p_lt) {
    double nl = (double)c->cam->width * (double)c->cam->height * p_lt;
    if (c->tw == 3) nl = 0.0;
    if (c->tw == 2) return nl > 0.0 ? 0.0 : or_tw_weight(c->opts->mis_mode, mine, other, 0.0);
    return or_tw_weight(c->opts->mis_mode, mine, other, nl);
}

static double dimv(const ctx_t *c, uint64_t idx, int dim) {
    return or_sample_dim(idx, dim, c->k, c->l, c->factors);
}

/* Radiance of one camera path (sequence index idx through pixel px, py), or,
 * with probe_x and probe_n given, the irradiance estimate of one probe path
 * (Sec. 4.2, alternate outputs: irradiance at a point from the hemisphere
 * around a normal). Reading: the probe is vertex 1, a virtual white
 * Lambertian surface point (albedo 1, geometric and shading normal probe_n,
 * wo = probe_n) that emits nothing; its outgoing radiance is E / pi, so the
 * path's radiance times pi estimates E. The vertices after it are those of a
 * camera path, with the same dimension allocation. */
static void path_radiance(const ctx_t *c, uint64_t idx, uint32_t px,
                          uint32_t py, const double *probe_x, const double *probe_n,
                          double L[3], uint64_t *rays) {
    const or_scene *s = c->s;
    int mode = c->opts->mis_mode;
    L[0] = L[1] = L[2] = 0.0;
    double o[3] = {0.0, 0.0, 0.0}, d[3] = {0.0, 0.0, 1.0};
    if (!probe_x) {
        double dx, dy;
        or_filter_offset(c->opts->filter_sigma, dimv(c, idx, 0), dimv(c, idx, 1), &dx, &dy);
        or_camera_ray(c->cam, (double)px + 0.5 + dx, (double)py + 0.5 + dy, o, d);
    }
    double beta[3] = {1.0, 1.0, 1.0};
    double prev_pdf = 0.0;
    /* two-way: the camera path's vertices, x[0] the eye */
    or_tw_vertex X[68];
    if (c->tw) {
        memset(&X[0], 0, sizeof X[0]);
        for (int a = 0; a < 3; ++a) X[0].x[a] = o[a];
    }
    double prev_ng[3] = {0.0, 1.0, 0.0};   /* geometric normal of the previous vertex (env pdf) */
    int has_tris = s->nlights > 0, has_env = s->p_env > 0.0;
    for (uint32_t v = 1; v <= c->D + 1; ++v) {
        const int at_probe = probe_x && v == 1;
        uint32_t prim = 0; double t = 0.0, b1 = 0.0, b2 = 0.0;
        if (!at_probe) {
            or_trace_one(s, o, d, 0.0, INFINITY, 0, &prim, &t, &b1, &b2);
            ++*rays;
        }
        if (prim == OR_MISS) {
            if (s->d.env) {
                double Le[3];
                or_env_lookup(s, d, Le);
                double w = 1.0;
                if (v > 1) {
                    if (mode == 3) w = 1.0;
                    else if (mode == 2) w = 0.0;
                    else w = has_env ? mis_weight(mode, prev_pdf, s->p_env * or_env_pdf_n(s, prev_ng, d)) : 1.0;
                    if (c->tw && has_env) {
                        double ph, pn, pl;
                        memset(&X[v], 0, sizeof X[v]);
                        X[v].prim = OR_MISS;
                        for (int a = 0; a < 3; ++a) X[v].x[a] = d[a];
                        or_tw_pdfs(s, &c->tc, X, (int)v, px, py, &ph, &pn, &pl);
                        w = tw_camera_weight(c, ph, pn, pl);
                        if (c->tw == 4 && pl > 0.0) L[0] += 1.0;   /* density check: count the hit */
                    }
                }
                if (c->tw == 4) w = 0.0;
                for (int a = 0; a < 3; ++a) L[a] += beta[a] * Le[a] * w;
            }
            break;
        }
        double x[3], ng[3], wo[3], cog;
        double b0 = 1.0 - b1 - b2;
        if (at_probe) {
            for (int a = 0; a < 3; ++a) { x[a] = probe_x[a]; ng[a] = probe_n[a]; wo[a] = probe_n[a]; }
            cog = 1.0;
        } else {
            const double *vv = s->v64 + 9 * (size_t)prim;
            for (int a = 0; a < 3; ++a) x[a] = b0 * vv[a] + b1 * vv[3 + a] + b2 * vv[6 + a];
            for (int a = 0; a < 3; ++a) { ng[a] = s->ng[3 * prim + a]; wo[a] = -d[a]; }
            cog = dot3(wo, ng);
        }
        uint32_t m = at_probe ? 0u : s->d.tri_material[prim];
        if (c->tw) or_tw_vertex_at(s, prim, b1, b2, &X[v]);
        if (!at_probe && cog > 0.0 && s->tri_light_pdf_area[prim] > 0.0) {
            double Le[3];
            or_tri_emission(s, prim, b1, b2, Le);
            double w = 1.0;
            if (v > 1) {
                if (mode == 3) w = 1.0;
                else if (mode == 2) w = 0.0;
                else if (c->tw) {
                    double ph, pn, pl;
                    or_tw_pdfs(s, &c->tc, X, (int)v, px, py, &ph, &pn, &pl);
                    w = tw_camera_weight(c, ph, pn, pl);
                    if (c->tw == 4) {   /* density check: count the hit */
                        if (pl > 0.0) L[0] += 1.0;
                        w = 0.0;
                    }
                } else {
                    /* the light hierarchy's probability of this emitter from
                     * the previous vertex (its offset origin o and normal) */
                    double pa = s->lb_nodes ? (1.0 - s->p_env) * or_lb_prob(s, o, prev_ng, s->light_of_tri[prim]) /
                                                  s->area[prim]
                                            : s->tri_light_pdf_area[prim];
                    w = mis_weight(mode, prev_pdf, pa * t * t / cog);
                }
            }
            if (c->tw == 4 && v == 1) w = 0.0;
            for (int a = 0; a < 3; ++a) L[a] += beta[a] * Le[a] * w;
        }
        if (v == c->D + 1) break;
        if (cog < 0.0) { ng[0] = -ng[0]; ng[1] = -ng[1]; ng[2] = -ng[2]; }
        double ns[3] = {ng[0], ng[1], ng[2]};
        if (s->d.normals && !at_probe) {
            const uint32_t *id = s->d.indices + 3 * (size_t)prim;
            for (int a = 0; a < 3; ++a)
                ns[a] = b0 * s->d.normals[3 * (size_t)id[0] + a] + b1 * s->d.normals[3 * (size_t)id[1] + a] +
                        b2 * s->d.normals[3 * (size_t)id[2] + a];
            normalize3(ns);
            if (dot3(ns, ng) < 0.0) { ns[0] = -ns[0]; ns[1] = -ns[1]; ns[2] = -ns[2]; }
        }
        double nsa[3];
        or_adapt_shading_normal(ns, ng, wo, nsa);
        double albedo[3] = {s->d.albedo[3 * m], s->d.albedo[3 * m + 1], s->d.albedo[3 * m + 2]};
        double rough = s->d.roughness[m], gw = s->d.ggx_weight[m];
        if (at_probe) { albedo[0] = albedo[1] = albedo[2] = 1.0; gw = 0.0; }
        int base = 2 + 7 * (int)(v - 1);
        double xo[3];
        or_offset_origin(x, ng, xo);
        /* next-event estimation */
        if ((has_tris || has_env) && mode != 3) {
            double us = dimv(c, idx, base), ua = dimv(c, idx, base + 1), ub = dimv(c, idx, base + 2);
            double wi[3], Le[3], sdir[3], pdf_l = 0.0, tmax = INFINITY;
            int64_t tw_li = -1;
            if (us < s->p_env) {
                double pe;
                or_env_sample_n(s, ng, ua, ub, wi, &pe);
                for (int a = 0; a < 3; ++a) sdir[a] = wi[a];
                or_env_lookup(s, wi, Le);
                pdf_l = s->p_env * or_env_pdf_n(s, ng, wi);
            } else {
                double u2 = (us - s->p_env) / (1.0 - s->p_env);
                if (u2 >= 1.0) u2 = nextafter(1.0, 0.0);
                double psel = 0.0;
                int64_t li = s->lb_nodes ? or_lb_sample(s, xo, ng, u2, &psel)
                                         : or_alias_sample(s->alias_prob, s->alias_idx, s->nlights, u2);
                uint32_t lt = (uint32_t)s->light_tri[li];
                tw_li = li;
                const double *lv = s->v64 + 9 * (size_t)lt;
                double sq = sqrt(ua);
                double lb1 = sq * (1.0 - ub), lb2 = sq * ub, lb0 = 1.0 - sq;
                double y[3];
                for (int a = 0; a < 3; ++a) y[a] = lb0 * lv[a] + lb1 * lv[3 + a] + lb2 * lv[6 + a];
                double dv[3] = {y[0] - x[0], y[1] - x[1], y[2] - x[2]};
                double dist = sqrt(dot3(dv, dv));
                if (dist > 0.0) {
                    for (int a = 0; a < 3; ++a) wi[a] = dv[a] / dist;
                    const double *lng = s->ng + 3 * (size_t)lt;
                    double cl = -dot3(wi, lng);
                    if (cl > 0.0) {
                        double pa = s->lb_nodes ? (1.0 - s->p_env) * psel / s->area[lt] : s->tri_light_pdf_area[lt];
                        pdf_l = pa * dist * dist / cl;
                        or_tri_emission(s, lt, lb1, lb2, Le);
                        /* the shadow segment: offset origin -> light point */
                        double sv[3] = {y[0] - xo[0], y[1] - xo[1], y[2] - xo[2]};
                        double sl = sqrt(dot3(sv, sv));
                        if (sl > 0.0) {
                            for (int a = 0; a < 3; ++a) sdir[a] = sv[a] / sl;
                            tmax = sl * (1.0 - OR_SHADOW_EPS);
                        } else {
                            pdf_l = 0.0;
                        }
                    }
                }
            }
            if (c->tw == 4 && pdf_l > 0.0 && dot3(wi, ng) > 0.0) {
                /* density check: count next-event samples that make a
                 * visible path the light tracer could make */
                double sq = sqrt(ua), ph, pn, pl;
                if (tw_li >= 0) {
                    or_tw_vertex_at(s, (uint32_t)s->light_tri[tw_li], sq * (1.0 - ub), sq * ub, &X[v + 1]);
                } else {
                    memset(&X[v + 1], 0, sizeof X[v + 1]);
                    X[v + 1].prim = OR_MISS;
                    for (int a = 0; a < 3; ++a) X[v + 1].x[a] = wi[a];
                }
                or_tw_pdfs(s, &c->tc, X, (int)v + 1, px, py, &ph, &pn, &pl);
                if (pl > 0.0) {
                    uint32_t sp; double st, sb1, sb2;
                    or_trace_one(s, xo, sdir, 0.0, tmax, 1, &sp, &st, &sb1, &sb2);
                    ++*rays;
                    if (sp == OR_MISS) L[1] += 1.0;
                }
            } else if (c->tw != 4 && pdf_l > 0.0 && dot3(wi, ng) > 0.0) {
                double f[3], pdf_b;
                or_bsdf_eval(albedo, rough, gw, nsa, wo, wi, f, &pdf_b);
                if (pdf_b > 0.0) {
                    double w = mode == 2 ? 1.0 : mis_weight(mode, pdf_l, pdf_b);
                    if (c->tw) {
                        double sq = sqrt(ua), ph, pn, pl;
                        if (us >= s->p_env) {
                            or_tw_vertex_at(s, (uint32_t)s->light_tri[tw_li], sq * (1.0 - ub), sq * ub, &X[v + 1]);
                        } else {
                            memset(&X[v + 1], 0, sizeof X[v + 1]);
                            X[v + 1].prim = OR_MISS;
                            for (int a = 0; a < 3; ++a) X[v + 1].x[a] = wi[a];
                        }
                        or_tw_pdfs(s, &c->tc, X, (int)v + 1, px, py, &ph, &pn, &pl);
                        w = tw_camera_weight(c, pn, ph, pl);
                    }
                    double ci = dot3(wi, nsa);
                    uint32_t sp; double st, sb1, sb2;
                    or_trace_one(s, xo, sdir, 0.0, tmax, 1, &sp, &st, &sb1, &sb2);
                    ++*rays;
                    if (sp == OR_MISS)
                        for (int a = 0; a < 3; ++a) L[a] += beta[a] * f[a] * ci * Le[a] * w / pdf_l;
                }
            }
        }
        /* continuation */
        double wi[3], f[3], pdf;
        if (!or_bsdf_sample(albedo, rough, gw, nsa, wo, dimv(c, idx, base + 3),
                            dimv(c, idx, base + 4), dimv(c, idx, base + 5), wi, f, &pdf))
            break;
        if (dot3(wi, ng) <= 0.0) break;
        double ci = dot3(wi, nsa);
        for (int a = 0; a < 3; ++a) beta[a] *= f[a] * ci / pdf;
        if (c->opts->rr_enable && v >= 3) {
            double mx = fmax(beta[0], fmax(beta[1], beta[2]));
            double q = fmax(0.05, 1.0 - mx);
            if (dimv(c, idx, base + 6) < q) break;
            for (int a = 0; a < 3; ++a) beta[a] /= (1.0 - q);
        }
        if (beta[0] == 0.0 && beta[1] == 0.0 && beta[2] == 0.0) break;
        prev_pdf = pdf;
        for (int a = 0; a < 3; ++a) { o[a] = xo[a]; d[a] = wi[a]; prev_ng[a] = ng[a]; }
    }
}

static void ctx_init(ctx_t *c, const or_scene *s, const or_camera *cam,
                     uint32_t D, const or_render_opts *opts) {
    c->s = s; c->cam = cam; c->opts = opts; c->D = D;
    uint64_t p2, p3;
    or_enum_params(cam->width, cam->height, &c->k, &c->l, &p2, &p3);
    c->ndims = 2 + 7 * (int)(D + 1);
    c->tw = 0;
    c->factors = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)c->ndims);
    for (int d = 0; d < c->ndims; ++d)
        c->factors[d] = d < 2 ? 1u : or_scramble_factor(opts->seed, or_prime(d));
}

typedef struct {
    const ctx_t *c;
    uint32_t iter0, spp;
    double *sum, *sum2;
    uint32_t *count;
    uint32_t row0, row1;
    uint64_t rays;
} job_t;

static void *render_rows(void *arg) {
    job_t *j = (job_t *)arg;
    const ctx_t *c = j->c;
    uint32_t W = c->cam->width, H = c->cam->height;
    uint32_t k, l; uint64_t p2, p3;
    or_enum_params(W, H, &k, &l, &p2, &p3);
    for (uint32_t y = j->row0; y < j->row1; ++y)
        for (uint32_t x = 0; x < W; ++x) {
            uint64_t i0 = or_pixel_base_index(W, H, x, y);
            size_t p = (size_t)y * W + x;
            for (uint32_t s = j->iter0; s < j->iter0 + j->spp; ++s) {
                uint64_t idx = i0 + (uint64_t)s * p2 * p3;
                double L[3];
                path_radiance(c, idx, x, y, NULL, NULL, L, &j->rays);
                for (int a = 0; a < 3; ++a) {
                    j->sum[3 * p + a] += L[a];
                    j->sum2[3 * p + a] += L[a] * L[a];
                }
                j->count[p] += 1;
            }
        }
    return NULL;
}

void or_render(const or_scene *s, const or_camera *cam, uint32_t iter0,
               uint32_t spp, uint32_t max_depth, const or_render_opts *opts,
               double *sum, double *sum2, uint32_t *count, uint64_t *rays_traced) {
    ctx_t c;
    ctx_init(&c, s, cam, max_depth, opts);
    int nth = opts->threads > 0 ? opts->threads : (int)sysconf(_SC_NPROCESSORS_ONLN);
    if (nth < 1) nth = 1;
    uint32_t H = cam->height;
    if ((uint32_t)nth > H) nth = (int)H;
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nth);
    job_t *jobs = (job_t *)calloc((size_t)nth, sizeof(job_t));
    /* interleave rows in blocks so that threads get similar work */
    uint32_t rows_per = (H + (uint32_t)nth - 1) / (uint32_t)nth;
    for (int t = 0; t < nth; ++t) {
        jobs[t].c = &c; jobs[t].iter0 = iter0; jobs[t].spp = spp;
        jobs[t].sum = sum; jobs[t].sum2 = sum2; jobs[t].count = count;
        jobs[t].row0 = (uint32_t)t * rows_per;
        jobs[t].row1 = jobs[t].row0 + rows_per > H ? H : jobs[t].row0 + rows_per;
        if (jobs[t].row0 > H) jobs[t].row0 = H;
        pthread_create(&th[t], NULL, render_rows, &jobs[t]);
    }
    uint64_t rays = 0;
    for (int t = 0; t < nth; ++t) { pthread_join(th[t], NULL); rays += jobs[t].rays; }
    if (rays_traced) *rays_traced = rays;
    free(th); free(jobs); free(c.factors);
}

void or_render_pixels(const or_scene *s, const or_camera *cam,
                      const uint32_t *px, const uint32_t *py,
                      const uint32_t *sample_j, int64_t n, uint32_t max_depth,
                      const or_render_opts *opts, double *L) {
    ctx_t c;
    ctx_init(&c, s, cam, max_depth, opts);
    uint32_t k, l; uint64_t p2, p3;
    or_enum_params(cam->width, cam->height, &k, &l, &p2, &p3);
    uint64_t rays = 0;
    for (int64_t r = 0; r < n; ++r) {
        uint64_t i0 = or_pixel_base_index(cam->width, cam->height, px[r], py[r]);
        path_radiance(&c, i0 + (uint64_t)sample_j[r] * p2 * p3, px[r], py[r], NULL, NULL, L + 3 * r, &rays);
    }
    free(c.factors);
}

/* Irradiance probes: probe p (position pos[3p..], unit normal nrm[3p..]) is
 * the pixel (p, 0) of an n x 1 image for the sample enumeration; iterations
 * [iter0, iter0 + spp); per probe the sums of E = pi L, of E^2 and the
 * sample count. */
void or_render_probes(const or_scene *s, const double *pos, const double *nrm, uint32_t n,
                      uint32_t iter0, uint32_t spp, uint32_t max_depth,
                      const or_render_opts *opts, double *sum, double *sum2,
                      uint32_t *count, uint64_t *rays_traced) {
    or_camera cam;
    memset(&cam, 0, sizeof cam);
    cam.width = n;
    cam.height = 1;
    ctx_t c;
    ctx_init(&c, s, &cam, max_depth, opts);
    uint32_t k, l; uint64_t p2, p3;
    or_enum_params(n, 1, &k, &l, &p2, &p3);
    uint64_t rays = 0;
    for (uint32_t p = 0; p < n; ++p) {
        uint64_t i0 = or_pixel_base_index(n, 1, p, 0);
        for (uint32_t j = iter0; j < iter0 + spp; ++j) {
            double L[3];
            path_radiance(&c, i0 + (uint64_t)j * p2 * p3, p, 0, pos + 3 * (size_t)p, nrm + 3 * (size_t)p, L, &rays);
            for (int a = 0; a < 3; ++a) {
                double e = OR_PI * L[a];
                sum[3 * (size_t)p + a] += e;
                sum2[3 * (size_t)p + a] += e * e;
            }
            count[p] += 1;
        }
    }
    if (rays_traced) *rays_traced = rays;
    free(c.factors);
}

void or_render_two_way(const or_scene *s, const or_camera *cam, uint32_t iter0, uint32_t spp,
                       uint32_t max_depth, const or_render_opts *opts, int32_t lt_mode, double *sum,
                       double *sum2, uint32_t *count, double *splat, uint64_t *rays_traced) {
    ctx_t c;
    ctx_init(&c, s, cam, max_depth, opts);
    c.tw = 1 + lt_mode;
    or_tw_cam_init(s, cam, opts->filter_sigma, &c.tc);
    c.tc.aim = opts->lt_aim;
    int nth = opts->threads > 0 ? opts->threads : (int)sysconf(_SC_NPROCESSORS_ONLN);
    if (nth < 1) nth = 1;
    uint32_t H = cam->height;
    if ((uint32_t)nth > H) nth = (int)H;
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nth);
    job_t *jobs = (job_t *)calloc((size_t)nth, sizeof(job_t));
    uint32_t rows_per = (H + (uint32_t)nth - 1) / (uint32_t)nth;
    for (int t = 0; t < nth; ++t) {
        jobs[t].c = &c; jobs[t].iter0 = iter0; jobs[t].spp = spp;
        jobs[t].sum = sum; jobs[t].sum2 = sum2; jobs[t].count = count;
        jobs[t].row0 = (uint32_t)t * rows_per;
        jobs[t].row1 = jobs[t].row0 + rows_per > H ? H : jobs[t].row0 + rows_per;
        if (jobs[t].row0 > H) jobs[t].row0 = H;
        pthread_create(&th[t], NULL, render_rows, &jobs[t]);
    }
    uint64_t rays = 0;
    for (int t = 0; t < nth; ++t) { pthread_join(th[t], NULL); rays += jobs[t].rays; }
    free(th); free(jobs); free(c.factors);
    if (lt_mode != 2) {
        uint64_t lr = 0;
        or_light_trace(s, cam, iter0, spp, max_depth, opts, lt_mode, splat, &lr);
        rays += lr;
    }
    if (rays_traced) *rays_traced = rays;
}
