/*
 * Oracle: two-way path tracing (paper Sec. 2): the forward path tracer and a
 * light tracer run as separate stages with the same number of paths and are
 * combined by multiple importance sampling. The light tracer starts paths on
 * the triangle emitters, chosen in proportion to their flux (Sec. 2.1.3, the
 * emission that photon aiming improves on), and connects every vertex of a
 * light path to the camera.
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Every path pdf here is the plain product over the path's stored vertices,
 * one factor per vertex in area measure, evaluated from the vertex list each
 * time a contribution is made; no running ratio is kept.
 *
 * Readings fixed where the paper is silent:
 *   - techniques for a path x0 (pinhole) .. xk (triangle emitter) with
 *     k >= 2 seen through pixel j: the camera path reaching xk by its
 *     BSDF-sampled continuation ("hit"), next-event estimation at x(k-1)
 *     ("nee"), and the light path x(k) .. x1 connected to x0 ("lt"); paths
 *     with k = 1 (an emitter or the environment seen directly) have no
 *     light-tracer technique; for a path ending in the environment xk is a
 *     direction and its densities are solid angles at x(k-1);
 *   - one camera path per pixel and iteration against W x H light paths per
 *     iteration: the sample counts in the heuristic are 1 and W H; the same
 *     power (beta 2) or balance heuristic as the two-technique path tracer;
 *   - pixel measurement: the Gaussian filter of the camera samples (sigma
 *     px, the sample credits its own pixel), so the camera technique's
 *     density of x1 through pixel j is g(u - c_j) f^2 |cos_1| / (cos^3 theta
 *     r^2) with u the image point of x1, c_j the pixel centre, f the focal
 *     length in pixels, theta the angle to the optical axis; the light
 *     tracer adds its connection to every pixel whose centre lies within
 *     3 sigma of u (the box filter: the pixel that holds u) and its density
 *     is zero for the other pixels, so the truncation costs no bias;
 *   - light path: the environment with next-event estimation's probability
 *     p_env, else a triangle emitter by the alias table (flux proportional),
 *     point uniform on the triangle (the same warp as NEE), direction
 *     cosine-distributed about the emitter's normal; an environment photon
 *     takes a direction w from the plain pyramid and a uniform point of the
 *     disk of radius r across the scene's bounding sphere (centre and half
 *     diagonal of its vertices' box; Sec. 2.1.3 names uniform aiming at a
 *     bound of the whole scene as the usual practice) and travels along
 *     -w, so its first hit has area density p_env p(w) |cos| / (pi r^2); at a vertex
 *     the next direction is drawn by the BSDF sampler with the arriving
 *     direction in the role of wo (its adapted shading normal too); the
 *     throughput takes the adjoint's shading-normal factor |wi.ns| / |wi.ng|
 *     of the vertex's shading normal as the camera side adapts it; no
 *     Russian roulette; vertices 1..D (the path tracer's depth) connect;
 *   - a direction below the geometric tangent plane of the side it leaves
 *     from ends the path, as in the path tracer; the connection ray runs from
 *     the offset origin to the eye and stops at (1 - 1e-4) of that length;
 *   - lt_mode 3 (a check of the densities, not an image): the camera stage
 *     counts per pixel its BSDF-sampled emitter hits (channel 0) and its
 *     unoccluded next-event samples on triangles (channel 1) on paths the
 *     light tracer can make, the light stage adds p_hit / (W H p_lt) and
 *     p_nee / (W H p_lt) at each connection; both estimate the same numbers
 *     only if every density is the density of the sampler it names;
 *   - sample dimensions of light path m = iteration * W H + i (i < W H):
 *     base = 2 + 7 (D + 1) (after the camera path's), base + {0: emitter,
 *     1,2: point (environment: direction), 3,4: direction (environment:
 *     disk point), 5: cluster of photon aiming}, then vertex t (1-based)
 *     base + 6 + 3 (t - 1) + {0: lobe, 1,2: direction};
 *   - photon aiming (Sec. 2.1.3, photon_aiming.c; lt_aim): an environment
 *     photon's disk is that of the chosen cluster, its first hit's area
 *     density p_env p(w) |cos| D(x, w) with D the line density of
 *     or_pa_env_density; a triangle photon's direction is drawn in the
 *     chosen cluster's cone, its solid-angle density or_pa_dir_density
 *     replacing the cosine distribution's cos / pi.
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
static double dist2(const double a[3], const double b[3]) {
    double d[3] = {a[0] - b[0], a[1] - b[1], a[2] - b[2]};
    return dot3(d, d);
}
/* unit vector from a to b */
static void unit_to(const double a[3], const double b[3], double out[3]) {
    for (int i = 0; i < 3; ++i) out[i] = b[i] - a[i];
    normalize3(out);
}

void or_tw_cam_init(const or_scene *s, const or_camera *c, double sigma, or_tw_cam *tc) {
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = 0; i < 3 * s->nt; ++i)
        for (int a = 0; a < 3; ++a) {
            double v = s->v64[3 * i + a];
            if (v < lo[a]) lo[a] = v;
            if (v > hi[a]) hi[a] = v;
        }
    if (s->nt > 0) {
        for (int a = 0; a < 3; ++a) tc->bc[a] = 0.5 * (lo[a] + hi[a]);
        tc->br = 0.5 * sqrt(dist2(lo, hi));
    } else {
        tc->bc[0] = tc->bc[1] = tc->bc[2] = 0.0;
        tc->br = 1.0;
    }
    for (int a = 0; a < 3; ++a) tc->eye[a] = c->eye[a];
    double fwd[3] = {c->look_at[0] - c->eye[0], c->look_at[1] - c->eye[1], c->look_at[2] - c->eye[2]};
    normalize3(fwd);
    double right[3], up[3];
    cross3(fwd, c->up, right);
    normalize3(right);
    cross3(right, fwd, up);
    for (int a = 0; a < 3; ++a) { tc->fwd[a] = fwd[a]; tc->right[a] = right[a]; tc->up[a] = up[a]; }
    tc->th = tan(0.5 * c->vfov_deg * OR_PI / 180.0);
    tc->asp = (double)c->width / (double)c->height;
    /* pixel pitch on the plane at unit distance is 2 th / H */
    tc->f = (double)c->height / (2.0 * tc->th);
    tc->W = c->width;
    tc->H = c->height;
    tc->sigma = sigma;
    /* view cone: around the optical axis, through the image corners */
    double tan_c = tc->th * sqrt(1.0 + tc->asp * tc->asp);
    double cos_c = 1.0 / sqrt(1.0 + tan_c * tan_c);
    for (int a = 0; a < 3; ++a) tc->aim_eye[a] = tc->eye[a];
    tc->aim_eye[3] = 2.0 * OR_PI * (1.0 - cos_c);
}

/* Photon aiming's eye vector of a camera: position and the solid angle of
 * its view cone. */
void or_pa_eye(const or_scene *s, const or_camera *c, double out[4]) {
    or_tw_cam tc;
    or_tw_cam_init(s, c, 0.5, &tc);
    for (int a = 0; a < 4; ++a) out[a] = tc.aim_eye[a];
}

void or_tw_vertex_at(const or_scene *s, uint32_t prim, double b1, double b2, or_tw_vertex *v) {
    const double *vv = s->v64 + 9 * (size_t)prim;
    double b0 = 1.0 - b1 - b2;
    for (int a = 0; a < 3; ++a) {
        v->x[a] = b0 * vv[a] + b1 * vv[3 + a] + b2 * vv[6 + a];
        v->ng[a] = s->ng[3 * (size_t)prim + a];
        v->ns[a] = v->ng[a];
    }
    if (s->d.normals) {
        const uint32_t *id = s->d.indices + 3 * (size_t)prim;
        for (int a = 0; a < 3; ++a)
            v->ns[a] = b0 * s->d.normals[3 * (size_t)id[0] + a] + b1 * s->d.normals[3 * (size_t)id[1] + a] +
                       b2 * s->d.normals[3 * (size_t)id[2] + a];
        normalize3(v->ns);
    }
    v->prim = prim;
}

/* Image point of x seen from the eye: (sx, sy) in pixels and cos theta. */
static int project(const or_tw_cam *tc, const double x[3], double *sx, double *sy, double *cz) {
    double d[3];
    unit_to(tc->eye, x, d);
    *cz = dot3(d, tc->fwd);
    if (!(*cz > 0.0)) return 0;
    double nx = dot3(d, tc->right) / *cz, ny = dot3(d, tc->up) / *cz;
    *sx = 0.5 * (double)tc->W * (1.0 + nx / (tc->th * tc->asp));
    *sy = 0.5 * (double)tc->H * (1.0 - ny / tc->th);
    return 1;
}

/* Filter density of image offset (dx, dy) from a pixel centre, per pixel^2,
 * and whether the light tracer connects to that pixel. */
static double filter_density(double sigma, double dx, double dy, int *lt_ok) {
    if (!(sigma > 0.0)) {
        int in = dx >= -0.5 && dx < 0.5 && dy >= -0.5 && dy < 0.5;
        *lt_ok = in;
        return in ? 1.0 : 0.0;
    }
    double r2 = dx * dx + dy * dy;
    double R = 3.0 * sigma;
    *lt_ok = r2 <= R * R;
    return exp(-r2 / (2.0 * sigma * sigma)) / (2.0 * OR_PI * sigma * sigma);
}

/* Camera density (area measure) of x1 through pixel (px, py). */
static double cam_density(const or_tw_cam *tc, const or_tw_vertex *x1, uint32_t px, uint32_t py, int *lt_ok) {
    double sx, sy, cz;
    *lt_ok = 0;
    if (!project(tc, x1->x, &sx, &sy, &cz)) return 0.0;
    double g = filter_density(tc->sigma, sx - ((double)px + 0.5), sy - ((double)py + 0.5), lt_ok);
    double w[3];
    unit_to(x1->x, tc->eye, w);
    double c1 = fabs(dot3(w, x1->ng));
    return g * tc->f * tc->f * c1 / (cz * cz * cz * dist2(tc->eye, x1->x));
}

/* |cos| between v's geometric normal and the direction to point p */
static double cos_to(const or_tw_vertex *v, const double p[3]) {
    double w[3];
    unit_to(v->x, p, w);
    return fabs(dot3(w, v->ng));
}

/* Solid-angle pdf with which the BSDF sampler at v, given the direction to
 * point a as wo, draws the direction to point b: geometric normal turned to
 * wo, shading normal to its side and adapted for wo (Appendix A.3); zero
 * below the geometric tangent plane. */
static double dir_pdf_w(const or_scene *s, const or_tw_vertex *v, const double wo[3], const double wi[3]) {
    double ng[3] = {v->ng[0], v->ng[1], v->ng[2]};
    if (dot3(wo, ng) < 0.0) { ng[0] = -ng[0]; ng[1] = -ng[1]; ng[2] = -ng[2]; }
    if (!(dot3(wi, ng) > 0.0)) return 0.0;
    double ns[3] = {v->ns[0], v->ns[1], v->ns[2]};
    if (dot3(ns, ng) < 0.0) { ns[0] = -ns[0]; ns[1] = -ns[1]; ns[2] = -ns[2]; }
    double nsa[3];
    or_adapt_shading_normal(ns, ng, wo, nsa);
    uint32_t m = s->d.tri_material[v->prim];
    double albedo[3] = {s->d.albedo[3 * m], s->d.albedo[3 * m + 1], s->d.albedo[3 * m + 2]};
    double f[3], pdf;
    or_bsdf_eval(albedo, s->d.roughness[m], s->d.ggx_weight[m], nsa, wo, wi, f, &pdf);
    return pdf;
}

/* the same, towards points a (wo) and b (wi); an environment vertex holds
 * its direction instead of a point */
static void toward(const or_tw_vertex *v, const or_tw_vertex *p, double w[3]) {
    if (p->prim == OR_MISS) { w[0] = p->x[0]; w[1] = p->x[1]; w[2] = p->x[2]; }
    else unit_to(v->x, p->x, w);
}
static double dir_pdf(const or_scene *s, const or_tw_vertex *v, const or_tw_vertex *a, const or_tw_vertex *b) {
    double wo[3], wi[3];
    toward(v, a, wo);
    toward(v, b, wi);
    return dir_pdf_w(s, v, wo, wi);
}

/* Area pdf with which next-event estimation at x(k-1) (wo towards x(k-2))
 * picks the point of emitter triangle xk->prim. */
static double nee_density(const or_scene *s, const or_tw_vertex *xm, const double toward[3], const or_tw_vertex *xk) {
    if (!s->lb_nodes) return s->tri_light_pdf_area[xk->prim];
    double wo[3];
    unit_to(xm->x, toward, wo);
    double ng[3] = {xm->ng[0], xm->ng[1], xm->ng[2]};
    if (dot3(wo, ng) < 0.0) { ng[0] = -ng[0]; ng[1] = -ng[1]; ng[2] = -ng[2]; }
    double xo[3];
    or_offset_origin(xm->x, ng, xo);
    return (1.0 - s->p_env) * or_lb_prob(s, xo, ng, s->light_of_tri[xk->prim]) / s->area[xk->prim];
}

/* Area pdf of the light tracer's emission point on triangle prim: the
 * triangle emitters are chosen with probability 1 - p_env (the environment
 * with p_env, as in next-event estimation), then by flux. */
static double lt_point_density(const or_scene *s, uint32_t prim) {
    return (1.0 - s->p_env) * s->light_prob[s->light_of_tri[prim]] / s->area[prim];
}

/* Solid-angle pdf with which next-event estimation at xm (wo towards point
 * `from`) picks environment direction w. */
static double env_nee_density(const or_scene *s, const or_tw_vertex *xm, const double from[3], const double w[3]) {
    double wo[3];
    unit_to(xm->x, from, wo);
    double ng[3] = {xm->ng[0], xm->ng[1], xm->ng[2]};
    if (dot3(wo, ng) < 0.0) { ng[0] = -ng[0]; ng[1] = -ng[1]; ng[2] = -ng[2]; }
    return s->p_env * or_env_pdf_n(s, ng, w);
}

void or_tw_pdfs(const or_scene *s, const or_tw_cam *tc, const or_tw_vertex *x, int k, uint32_t px, uint32_t py,
                double *p_hit, double *p_nee, double *p_lt) {
    *p_hit = *p_nee = *p_lt = 0.0;
    if (k < 2) return;
    const or_tw_vertex *xk = &x[k];
    const int env = xk->prim == OR_MISS;   /* xk: a direction towards the environment */
    double cy = 0.0;
    if (!env) {
        double w[3];
        unit_to(xk->x, x[k - 1].x, w);
        cy = dot3(w, xk->ng);   /* the emitter radiates on its normal's side */
        if (!(cy > 0.0)) return;
    }
    int lt_ok;
    double pc = cam_density(tc, &x[1], px, py, &lt_ok);
    /* camera techniques: the shared prefix x1 .. x(k-1) */
    double pre = pc;
    for (int i = 1; i <= k - 2; ++i)
        pre *= dir_pdf(s, &x[i], &x[i - 1], &x[i + 1]) * cos_to(&x[i + 1], x[i].x) / dist2(x[i].x, x[i + 1].x);
    if (env) {
        /* solid angle at x(k-1): the continuation's pdf, NEE's environment pdf */
        *p_hit = pre * dir_pdf(s, &x[k - 1], &x[k - 2], xk);
        *p_nee = pre * env_nee_density(s, &x[k - 1], x[k - 2].x, xk->x);
    } else {
        *p_hit = pre * dir_pdf(s, &x[k - 1], &x[k - 2], xk) * cy / dist2(x[k - 1].x, xk->x);
        *p_nee = pre * nee_density(s, &x[k - 1], x[k - 2].x, xk);
    }
    /* light tracer: emission point and cosine direction (a triangle), or a
     * direction and a point of the disk of the scene's bounding sphere
     * across it (the environment); then BSDF samples with the arriving
     * direction as wo, down to x1 */
    if (!lt_ok) return;
    double pl;
    if (env) {
        /* per unit area across w: uniform over the scene's bound, or aimed
         * at the clusters whose spheres the photon's line meets */
        double across = tc->aim ? or_pa_env_density(s, tc->aim_eye, x[k - 1].x, xk->x) : 1.0 / (OR_PI * tc->br * tc->br);
        pl = s->p_env * or_env_pdf(s, xk->x) * fabs(dot3(x[k - 1].ng, xk->x)) * across;
    } else {
        /* per solid angle at the emitter: cosine, or aimed at the clusters
         * whose cones hold the direction */
        double pw;
        if (tc->aim) {
            double w[3];
            unit_to(xk->x, x[k - 1].x, w);
            pw = or_pa_dir_density(s, tc->aim_eye, xk->x, xk->ng, w);
        } else {
            pw = cy / OR_PI;
        }
        pl = lt_point_density(s, xk->prim) * pw * cos_to(&x[k - 1], xk->x) / dist2(x[k - 1].x, xk->x);
    }
    for (int i = k - 1; i >= 2; --i)
        pl *= dir_pdf(s, &x[i], &x[i + 1], &x[i - 1]) * cos_to(&x[i - 1], x[i].x) / dist2(x[i].x, x[i - 1].x);
    *p_lt = pl;
}

double or_tw_weight(int mode, double mine, double other1, double other2) {
    if (mode == 1) {
        double d = mine + other1 + other2;
        return d > 0.0 ? mine / d : 0.0;
    }
    double d = mine * mine + other1 * other1 + other2 * other2;
    return d > 0.0 ? mine * mine / d : 0.0;
}

/* ------------------------------------------------------- light tracer */
typedef struct {
    const or_scene *s;
    or_tw_cam tc;
    uint32_t D, k, l;
    const uint32_t *factors;
    int base;
    int mode;
    int lt_mode;       /* 0 MIS, 1 light tracer alone for k >= 2 */
    double *splat;     /* this worker's H x W x 3 */
    uint64_t m0, m1;   /* light paths [m0, m1) */
    uint64_t rays;
} lt_job;

static double ltdim(const lt_job *j, uint64_t m, int dim) {
    return or_sample_dim(m, dim, j->k, j->l, j->factors);
}

static void light_path(lt_job *j, uint64_t m, or_tw_vertex *V, or_tw_vertex *X) {
    const or_scene *s = j->s;
    const or_tw_cam *tc = &j->tc;
    if (s->nlights <= 0 && !(s->p_env > 0.0)) return;
    const double nL = (double)tc->W * (double)tc->H;
    double us = ltdim(j, m, j->base), ua = ltdim(j, m, j->base + 1), ub = ltdim(j, m, j->base + 2);
    double u3 = ltdim(j, m, j->base + 3), u4 = ltdim(j, m, j->base + 4), uc = ltdim(j, m, j->base + 5);
    double beta[3], o[3], dir[3];
    int env_photon = 0;
    double env_k = 0.0;   /* aimed environment photon: Le / (p_env pw), divided by the line density at the hit */
    if (us < s->p_env) {
        /* environment photon: a direction from the plain pyramid, then a
         * uniform point of the disk of radius br across the bounding sphere,
         * travelling back along the direction */
        double w[3], pw;
        int32_t tx, ty;
        or_env_sample(s, ua, ub, w, &pw, &tx, &ty);
        if (!(pw > 0.0)) return;
        double Le[3];
        or_env_lookup(s, w, Le);
        memset(&V[0], 0, sizeof V[0]);
        V[0].prim = OR_MISS;
        for (int a = 0; a < 3; ++a) V[0].x[a] = w[a];
        double t1[3], t2[3];
        or_onb(w, t1, t2);
        if (tc->aim && s->pa_nclusters > 0) {
            /* a cluster by the hierarchy, a uniform point of the disk of
             * its sphere across w, moved back along w outside the scene */
            int32_t c = or_pa_sample(s, tc->aim_eye, NULL, NULL, uc, NULL);
            const double *cc = s->pa_cc + 4 * c;
            double r = cc[3] * sqrt(u3), phi = 2.0 * OR_PI * u4;
            double p[3];
            for (int a = 0; a < 3; ++a) p[a] = cc[a] + r * cos(phi) * t1[a] + r * sin(phi) * t2[a];
            double back = sqrt(dist2(p, tc->bc)) + tc->br;
            for (int a = 0; a < 3; ++a) { o[a] = p[a] + back * w[a]; dir[a] = -w[a]; }
            env_photon = 1;
            env_k = 1.0 / (s->p_env * pw);
            for (int a = 0; a < 3; ++a) beta[a] = Le[a];
        } else {
            double r = tc->br * sqrt(u3), phi = 2.0 * OR_PI * u4;
            for (int a = 0; a < 3; ++a) {
                o[a] = tc->bc[a] + 2.0 * tc->br * w[a] + r * cos(phi) * t1[a] + r * sin(phi) * t2[a];
                dir[a] = -w[a];
            }
            /* Le / (p_env pw |cos| / (pi br^2)) with |cos| taken at the hit */
            double k = OR_PI * tc->br * tc->br / (s->p_env * pw);
            for (int a = 0; a < 3; ++a) beta[a] = Le[a] * k;
        }
    } else {
        double u2 = (us - s->p_env) / (1.0 - s->p_env);
        if (u2 >= 1.0) u2 = nextafter(1.0, 0.0);
        int64_t e = or_alias_sample(s->alias_prob, s->alias_idx, s->nlights, u2);
        uint32_t lt = (uint32_t)s->light_tri[e];
        double sq = sqrt(ua);
        double b1 = sq * (1.0 - ub), b2 = sq * ub;
        or_tw_vertex_at(s, lt, b1, b2, &V[0]);
        double Le[3];
        or_tri_emission(s, lt, b1, b2, Le);
        double pa = lt_point_density(s, lt);
        if (tc->aim && s->pa_nclusters > 0) {
            /* a cluster by the hierarchy (seen from the emitter point), a
             * direction uniform in the cone its sphere subtends */
            int32_t c = or_pa_sample(s, tc->aim_eye, V[0].x, V[0].ng, uc, NULL);
            or_pa_cone_sample(s, c, V[0].x, u3, u4, dir);
            double cy = dot3(dir, V[0].ng);
            if (!(cy > 0.0)) return;   /* behind the one-sided emitter: no power */
            double pw = or_pa_dir_density(s, tc->aim_eye, V[0].x, V[0].ng, dir);
            if (!(pw > 0.0)) return;
            /* Le cos / (pa pw) */
            for (int a = 0; a < 3; ++a) beta[a] = Le[a] * cy / (pa * pw);
        } else {
            double t1[3], t2[3];
            or_onb(V[0].ng, t1, t2);
            double r = sqrt(u3), phi = 2.0 * OR_PI * u4, cz = sqrt(fmax(0.0, 1.0 - u3));
            if (!(cz > 0.0)) return;
            for (int a = 0; a < 3; ++a) dir[a] = r * cos(phi) * t1[a] + r * sin(phi) * t2[a] + cz * V[0].ng[a];
            normalize3(dir);
            /* Le cos / (pa cos / pi) */
            for (int a = 0; a < 3; ++a) beta[a] = Le[a] * OR_PI / pa;
        }
        or_offset_origin(V[0].x, V[0].ng, o);
    }
    for (uint32_t t = 1; t <= j->D; ++t) {
        uint32_t prim; double th, hb1, hb2;
        or_trace_one(s, o, dir, 0.0, INFINITY, 0, &prim, &th, &hb1, &hb2);
        ++j->rays;
        if (prim == OR_MISS) return;
        or_tw_vertex_at(s, prim, hb1, hb2, &V[t]);
        const or_tw_vertex *v = &V[t];
        if (t == 1 && env_photon) {
            /* Le |cos| / (p_env pw |cos| D): the line density D at the hit */
            double D = or_pa_env_density(s, tc->aim_eye, v->x, V[0].x);
            if (!(D > 0.0)) return;
            for (int a = 0; a < 3; ++a) beta[a] *= env_k / D;
        }
        double wi[3] = {-dir[0], -dir[1], -dir[2]};
        double ngf[3] = {v->ng[0], v->ng[1], v->ng[2]};
        if (dot3(wi, ngf) < 0.0) { ngf[0] = -ngf[0]; ngf[1] = -ngf[1]; ngf[2] = -ngf[2]; }
        double nsf[3] = {v->ns[0], v->ns[1], v->ns[2]};
        if (dot3(nsf, ngf) < 0.0) { nsf[0] = -nsf[0]; nsf[1] = -nsf[1]; nsf[2] = -nsf[2]; }
        double cwi_g = fabs(dot3(wi, v->ng));
        uint32_t mt = s->d.tri_material[prim];
        double albedo[3] = {s->d.albedo[3 * mt], s->d.albedo[3 * mt + 1], s->d.albedo[3 * mt + 2]};
        double rough = s->d.roughness[mt], gw = s->d.ggx_weight[mt];
        double xo[3];
        or_offset_origin(v->x, ngf, xo);
        /* connection to the pinhole */
        double we[3];
        unit_to(v->x, tc->eye, we);
        double sx, sy, czc;
        double mg = 3.0 * tc->sigma + 2.0;   /* image points beyond the splat window reach no pixel */
        if (dot3(we, ngf) > 0.0 && project(tc, v->x, &sx, &sy, &czc) && sx > -mg && sx < (double)tc->W + mg &&
            sy > -mg && sy < (double)tc->H + mg) {
            double nsa[3], f[3], pdf;
            or_adapt_shading_normal(nsf, ngf, we, nsa);
            or_bsdf_eval(albedo, rough, gw, nsa, we, wi, f, &pdf);
            if (f[0] > 0.0 || f[1] > 0.0 || f[2] > 0.0 || j->lt_mode == 3) {
                double seg[3] = {tc->eye[0] - xo[0], tc->eye[1] - xo[1], tc->eye[2] - xo[2]};
                double sl = sqrt(dot3(seg, seg));
                uint32_t sp = OR_MISS; double st, sb1, sb2;
                if (sl > 0.0) {
                    for (int a = 0; a < 3; ++a) seg[a] /= sl;
                    or_trace_one(s, xo, seg, 0.0, sl * (1.0 - OR_SHADOW_EPS), 1, &sp, &st, &sb1, &sb2);
                    ++j->rays;
                }
                if (sl > 0.0 && sp == OR_MISS) {
                    /* the path in camera order: eye, V[t], V[t-1], ..., V[0] */
                    int k = (int)t + 1;
                    memset(&X[0], 0, sizeof X[0]);
                    for (int a = 0; a < 3; ++a) X[0].x[a] = tc->eye[a];
                    for (int i = 1; i <= k; ++i) X[i] = V[k - i];
                    double shade_f = fabs(dot3(wi, nsa)) / cwi_g;
                    double c1 = fabs(dot3(we, v->ng));
                    double r2 = dist2(tc->eye, v->x);
                    int x0 = (int)floor(sx - 0.5 - 3.0 * tc->sigma), x1 = (int)ceil(sx - 0.5 + 3.0 * tc->sigma);
                    int y0 = (int)floor(sy - 0.5 - 3.0 * tc->sigma), y1 = (int)ceil(sy - 0.5 + 3.0 * tc->sigma);
                    if (!(tc->sigma > 0.0)) { x0 = x1 = (int)floor(sx); y0 = y1 = (int)floor(sy); }
                    for (int py = y0; py <= y1; ++py)
                        for (int px = x0; px <= x1; ++px) {
                            if (px < 0 || py < 0 || px >= (int)tc->W || py >= (int)tc->H) continue;
                            int ok;
                            double g = filter_density(tc->sigma, sx - ((double)px + 0.5), sy - ((double)py + 0.5), &ok);
                            if (!ok) continue;
                            double We = g * tc->f * tc->f * c1 / (czc * czc * czc * r2);
                            double w = 1.0;
                            if (j->lt_mode == 0) {
                                double ph, pn, pl;
                                or_tw_pdfs(s, tc, X, k, (uint32_t)px, (uint32_t)py, &ph, &pn, &pl);
                                w = or_tw_weight(j->mode, nL * pl, ph, pn);
                            }
                            double *sp3 = j->splat + 3 * ((size_t)py * tc->W + (size_t)px);
                            if (j->lt_mode == 3) {
                                /* density check: the camera techniques' densities over the
                                 * light tracer's; their mean counts the camera's samples */
                                double ph, pn, pl;
                                or_tw_pdfs(s, tc, X, k, (uint32_t)px, (uint32_t)py, &ph, &pn, &pl);
                                if (pl > 0.0) { sp3[0] += ph / (nL * pl); sp3[1] += pn / (nL * pl); }
                                continue;
                            }
                            for (int a = 0; a < 3; ++a) sp3[a] += w * beta[a] * f[a] * shade_f * We / nL;
                        }
                }
            }
        }
        if (t == j->D) return;
        /* continuation: BSDF sampling with the arriving direction as wo */
        int bb = j->base + 6 + 3 * (int)(t - 1);
        double nsl[3], wn[3], fs[3], q;
        or_adapt_shading_normal(nsf, ngf, wi, nsl);
        if (!or_bsdf_sample(albedo, rough, gw, nsl, wi, ltdim(j, m, bb), ltdim(j, m, bb + 1), ltdim(j, m, bb + 2),
                            wn, fs, &q))
            return;
        if (!(dot3(wn, ngf) > 0.0)) return;
        double nsn[3], fc[3], pc;
        or_adapt_shading_normal(nsf, ngf, wn, nsn);
        or_bsdf_eval(albedo, rough, gw, nsn, wn, wi, fc, &pc);
        double k2 = fabs(dot3(wi, nsn)) / cwi_g * fabs(dot3(wn, v->ng)) / q;
        for (int a = 0; a < 3; ++a) beta[a] *= fc[a] * k2;
        if (beta[0] == 0.0 && beta[1] == 0.0 && beta[2] == 0.0) return;
        for (int a = 0; a < 3; ++a) { o[a] = xo[a]; dir[a] = wn[a]; }
    }
}

static void *lt_rows(void *arg) {
    lt_job *j = (lt_job *)arg;
    or_tw_vertex *V = (or_tw_vertex *)malloc(sizeof(or_tw_vertex) * (j->D + 2));
    or_tw_vertex *X = (or_tw_vertex *)malloc(sizeof(or_tw_vertex) * (j->D + 2));
    for (uint64_t m = j->m0; m < j->m1; ++m) light_path(j, m, V, X);
    free(V); free(X);
    return NULL;
}

void or_light_trace(const or_scene *s, const or_camera *cam, uint32_t iter0, uint32_t spp, uint32_t D,
                    const or_render_opts *opts, int lt_mode, double *splat, uint64_t *rays_traced) {
    uint32_t W = cam->width, H = cam->height;
    uint32_t k, l; uint64_t p2, p3;
    or_enum_params(W, H, &k, &l, &p2, &p3);
    int base = 2 + 7 * (int)(D + 1);
    int ndims = base + 6 + 3 * (int)D;
    uint32_t *factors = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)ndims);
    for (int d = 0; d < ndims; ++d) factors[d] = d < 2 ? 1u : or_scramble_factor(opts->seed, or_prime(d));
    int nth = opts->threads > 0 ? opts->threads : (int)sysconf(_SC_NPROCESSORS_ONLN);
    if (nth < 1) nth = 1;
    uint64_t WH = (uint64_t)W * H, m0 = (uint64_t)iter0 * WH, n = (uint64_t)spp * WH;
    if ((uint64_t)nth > n) nth = n ? (int)n : 1;
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nth);
    lt_job *jobs = (lt_job *)calloc((size_t)nth, sizeof(lt_job));
    for (int t = 0; t < nth; ++t) {
        lt_job *j = &jobs[t];
        j->s = s;
        or_tw_cam_init(s, cam, opts->filter_sigma, &j->tc);
        j->tc.aim = opts->lt_aim;
        j->D = D; j->k = k; j->l = l; j->factors = factors; j->base = base;
        j->mode = opts->mis_mode;
        j->lt_mode = lt_mode;
        j->splat = (double *)calloc((size_t)WH * 3, sizeof(double));
        j->m0 = m0 + n * (uint64_t)t / (uint64_t)nth;
        j->m1 = m0 + n * (uint64_t)(t + 1) / (uint64_t)nth;
        pthread_create(&th[t], NULL, lt_rows, j);
    }
    uint64_t rays = 0;
    for (int t = 0; t < nth; ++t) {
        pthread_join(th[t], NULL);
        for (size_t i = 0; i < (size_t)WH * 3; ++i) splat[i] += jobs[t].splat[i];
        rays += jobs[t].rays;
        free(jobs[t].splat);
    }
    if (rays_traced) *rays_traced = rays;
    free(th); free(jobs); free(factors);
}
