/*
 * Oracle: scene set-up and light importance sampling in FP64 (paper
 * Sec. 2.1.1 "geometric light sources": triangles only, one flux value per
 * triangle integrated in a preprocess; Sec. 2.1.2 "environment light": an
 * equirectangular finest level, coarser levels by downsampling, values scaled
 * by their area on the unit sphere, probabilistic descent by intensity).
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Triangle selection uses Walker's alias table built by Vose's method (the
 * synthetic many-light workload asks for it); the paper's light BVH is not
 * built here. Readings fixed where the paper is silent:
 *   - flux_t = luminance(emission) * area_t (the pi of a Lambertian emitter
 *     cancels in the normalisation); luminance = Rec. 709 weights;
 *   - environment chosen with probability 0.5 when both kinds of light exist;
 *   - environment weights = luminance * exact texel solid angle
 *     (2 pi / W) * (cos theta0 - cos theta1); the map must be W x H with
 *     W = 2H a power of two, top level 2 x 1, each coarser texel the sum of
 *     its 2 x 2 children; the descent picks a column with u and then a row
 *     with v, rescaling each, and places the direction uniformly in
 *     (phi, cos theta) inside the final texel, so pdf = lum(texel) / sum(w).
 */
#include "oracle.h"
#include "oracle_internal.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define OR_PI 3.14159265358979323846

/* ------------------------------------------------------------ alias table */
void or_alias_build(const double *w, int64_t n, double *prob, int64_t *alias) {
    double sum = 0.0;
    for (int64_t i = 0; i < n; ++i) sum += w[i];
    double *p = (double *)malloc(sizeof(double) * (size_t)n);
    int64_t *small = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    int64_t *large = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    int64_t ns = 0, nl = 0;
    for (int64_t i = 0; i < n; ++i) {
        p[i] = w[i] * (double)n / sum;
        alias[i] = i;
        if (p[i] < 1.0) small[ns++] = i; else large[nl++] = i;
    }
    while (ns > 0 && nl > 0) {
        int64_t s = small[--ns], g = large[--nl];
        prob[s] = p[s];
        alias[s] = g;
        p[g] = (p[g] + p[s]) - 1.0;
        if (p[g] < 1.0) small[ns++] = g; else large[nl++] = g;
    }
    while (nl > 0) { int64_t g = large[--nl]; prob[g] = 1.0; alias[g] = g; }
    while (ns > 0) { int64_t s = small[--ns]; prob[s] = 1.0; alias[s] = s; }
    free(p); free(small); free(large);
}

int64_t or_alias_sample(const double *prob, const int64_t *alias, int64_t n,
                        double u) {
    double x = u * (double)n;
    int64_t bin = (int64_t)floor(x);
    if (bin >= n) bin = n - 1;
    double frac = x - (double)bin;
    return frac < prob[bin] ? bin : alias[bin];
}

/* ----------------------------------------------------- environment pyramid */
static double texel_solid_angle(int32_t W, int32_t H, int32_t y) {
    double th0 = OR_PI * (double)y / (double)H, th1 = OR_PI * (double)(y + 1) / (double)H;
    return (2.0 * OR_PI / (double)W) * (cos(th0) - cos(th1));
}

static void build_env(or_scene *s) {
    s->env_levels = 0; s->env_wsum = 0.0;
    if (!s->d.env) return;
    int32_t W = s->d.env_w, H = s->d.env_h;
    int levels = 0;
    for (int32_t w = W; w >= 2; w /= 2) ++levels;
    s->env_levels = levels;
    s->env_w = (double **)calloc((size_t)levels, sizeof(double *));
    s->env_lw = (int32_t *)calloc((size_t)levels, sizeof(int32_t));
    s->env_lh = (int32_t *)calloc((size_t)levels, sizeof(int32_t));
    s->env_lw[0] = W; s->env_lh[0] = H;
    s->env_w[0] = (double *)malloc(sizeof(double) * (size_t)W * (size_t)H);
    double sum = 0.0;
    for (int32_t y = 0; y < H; ++y) {
        double om = texel_solid_angle(W, H, y);
        for (int32_t x = 0; x < W; ++x) {
            const float *L = s->d.env + 3 * ((size_t)y * W + x);
            double c[3] = {L[0], L[1], L[2]};
            double wv = or_luminance(c) * om;
            s->env_w[0][(size_t)y * W + x] = wv;
            sum += wv;
        }
    }
    s->env_wsum = sum;
    for (int l = 1; l < levels; ++l) {
        int32_t lw = s->env_lw[l - 1] / 2, lh = s->env_lh[l - 1] / 2;
        if (lh < 1) lh = 1;
        s->env_lw[l] = lw; s->env_lh[l] = lh;
        s->env_w[l] = (double *)calloc((size_t)lw * (size_t)lh, sizeof(double));
        int32_t pw = s->env_lw[l - 1], ph = s->env_lh[l - 1];
        for (int32_t y = 0; y < ph; ++y)
            for (int32_t x = 0; x < pw; ++x)
                s->env_w[l][(size_t)(y / 2) * lw + x / 2] += s->env_w[l - 1][(size_t)y * pw + x];
    }
}

static double envw(const or_scene *s, int l, int32_t x, int32_t y) {
    return s->env_w[l][(size_t)y * s->env_lw[l] + x];
}

/* ------------------------------------- normal-oriented top levels (2.1.2) */
#define OR_ENV_CELL_SIDE 8        /* 8 x 8 octahedral cells of the normal */
#define OR_ENV_NORMAL_LEVELS 5    /* reweighted top levels of the pyramid */

static void or_normalize(double a[3]) {
    double l = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
    if (l > 0.0) { a[0] /= l; a[1] /= l; a[2] /= l; }
}

static double angle_between(const double a[3], const double b[3]) {
    double c = a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
    if (c > 1.0) c = 1.0;
    if (c < -1.0) c = -1.0;
    return acos(c);
}

/* Octahedral map of the unit sphere onto [-1, 1]^2 (plane x, z; the lower
 * hemisphere y < 0 folded over the diagonals) and back. */
static void oct_decode(double px, double pz, double n[3]) {
    double y = 1.0 - fabs(px) - fabs(pz);
    if (y < 0.0) {
        double ox = (1.0 - fabs(pz)) * (px >= 0.0 ? 1.0 : -1.0);
        double oz = (1.0 - fabs(px)) * (pz >= 0.0 ? 1.0 : -1.0);
        px = ox; pz = oz;
    }
    n[0] = px; n[1] = y; n[2] = pz;
    or_normalize(n);
}

int or_env_normal_cell(const double n[3]) {
    double sum = fabs(n[0]) + fabs(n[1]) + fabs(n[2]);
    if (!(sum > 0.0)) return 0;
    double px = n[0] / sum, pz = n[2] / sum;
    if (n[1] < 0.0) {
        double ox = (1.0 - fabs(pz)) * (px >= 0.0 ? 1.0 : -1.0);
        double oz = (1.0 - fabs(px)) * (pz >= 0.0 ? 1.0 : -1.0);
        px = ox; pz = oz;
    }
    int i = (int)floor((px + 1.0) * 0.5 * OR_ENV_CELL_SIDE);
    int j = (int)floor((pz + 1.0) * 0.5 * OR_ENV_CELL_SIDE);
    if (i < 0) i = 0;
    if (i >= OR_ENV_CELL_SIDE) i = OR_ENV_CELL_SIDE - 1;
    if (j < 0) j = 0;
    if (j >= OR_ENV_CELL_SIDE) j = OR_ENV_CELL_SIDE - 1;
    return j * OR_ENV_CELL_SIDE + i;
}

/* Centre direction of a set given on a 17 x 17 parameter grid and the
 * largest angle from it to the set: the largest angle to a grid point plus
 * the largest angle across a grid square's diagonal (every point of the set
 * lies within that of a grid point). */
static void cone_of_grid(double pts[17][17][3], double centre[3], double *radius) {
    double far = 0.0, step = 0.0;
    for (int a = 0; a < 17; ++a)
        for (int b = 0; b < 17; ++b) {
            double t = angle_between(centre, pts[a][b]);
            if (t > far) far = t;
            if (a < 16 && b < 16) {
                double d1 = angle_between(pts[a][b], pts[a + 1][b + 1]);
                double d2 = angle_between(pts[a + 1][b], pts[a][b + 1]);
                if (d1 > step) step = d1;
                if (d2 > step) step = d2;
            }
        }
    *radius = far + step;
}

static void cell_cone(int cell, double centre[3], double *radius) {
    int i = cell % OR_ENV_CELL_SIDE, j = cell / OR_ENV_CELL_SIDE;
    double pts[17][17][3];
    for (int a = 0; a < 17; ++a)
        for (int b = 0; b < 17; ++b) {
            double u = (i + a / 16.0) / OR_ENV_CELL_SIDE, v = (j + b / 16.0) / OR_ENV_CELL_SIDE;
            oct_decode(2.0 * u - 1.0, 2.0 * v - 1.0, pts[a][b]);
        }
    oct_decode(2.0 * (i + 0.5) / OR_ENV_CELL_SIDE - 1.0, 2.0 * (j + 0.5) / OR_ENV_CELL_SIDE - 1.0, centre);
    cone_of_grid(pts, centre, radius);
}

static void dir_of(double theta, double phi, double d[3]) {
    d[0] = sin(theta) * cos(phi); d[1] = cos(theta); d[2] = sin(theta) * sin(phi);
}

/* Region (x, y) of a level of lw x lh nodes: phi in [2 pi x / lw, ...),
 * theta in [pi y / lh, ...). */
static void region_cone(int32_t lw, int32_t lh, int32_t x, int32_t y, double centre[3], double *radius) {
    double pts[17][17][3];
    double t0 = OR_PI * y / lh, t1 = OR_PI * (y + 1) / lh;
    double p0 = 2.0 * OR_PI * x / lw, p1 = 2.0 * OR_PI * (x + 1) / lw;
    for (int a = 0; a < 17; ++a)
        for (int b = 0; b < 17; ++b) dir_of(t0 + (t1 - t0) * a / 16.0, p0 + (p1 - p0) * b / 16.0, pts[a][b]);
    dir_of(0.5 * (t0 + t1), 0.5 * (p0 + p1), centre);
    cone_of_grid(pts, centre, radius);
}

/* Per normal cell, the finest reweighted level holds w x kappa, kappa the
 * cone bound of the clamped cosine between the cell's normals and the
 * region's directions (1 when the cones overlap, 0 when every pair is at
 * least 90 degrees apart); the coarser reweighted levels are sums of their
 * children, so the descent is proportional to the reweighted energy below. */
static void build_env_normal_levels(or_scene *s) {
    s->env_nw = NULL;
    if (!s->d.env || s->d.env_plain || !(s->env_wsum > 0.0)) return;
    int top = s->env_levels - 1;
    int nl = OR_ENV_NORMAL_LEVELS < s->env_levels ? OR_ENV_NORMAL_LEVELS : s->env_levels;
    s->env_lstar = top - nl + 1;
    int64_t off = 0;
    for (int l = top; l >= s->env_lstar; --l) {
        s->env_noff[l] = off;
        off += (int64_t)s->env_lw[l] * s->env_lh[l];
    }
    s->env_nstride = off;
    int ncell = OR_ENV_CELL_SIDE * OR_ENV_CELL_SIDE;
    s->env_nw = (double *)calloc((size_t)ncell * (size_t)off, sizeof(double));
    const int ls = s->env_lstar;
    const int32_t lw = s->env_lw[ls], lh = s->env_lh[ls];
    double *rc = (double *)malloc(sizeof(double) * 3 * (size_t)lw * lh);
    double *rb = (double *)malloc(sizeof(double) * (size_t)lw * lh);
    for (int32_t y = 0; y < lh; ++y)
        for (int32_t x = 0; x < lw; ++x) region_cone(lw, lh, x, y, rc + 3 * ((size_t)y * lw + x), rb + (size_t)y * lw + x);
    for (int c = 0; c < ncell; ++c) {
        double nc[3], alpha;
        cell_cone(c, nc, &alpha);
        double *blk = s->env_nw + (size_t)c * (size_t)off;
        for (int32_t y = 0; y < lh; ++y)
            for (int32_t x = 0; x < lw; ++x) {
                size_t i = (size_t)y * lw + x;
                double ang = angle_between(nc, rc + 3 * i) - alpha - rb[i];
                double kappa = ang <= 0.0 ? 1.0 : (ang >= 0.5 * OR_PI ? 0.0 : cos(ang));
                blk[s->env_noff[ls] + i] = s->env_w[ls][i] * kappa;
            }
        for (int l = ls + 1; l <= top; ++l) {
            int32_t pw = s->env_lw[l - 1], ph = s->env_lh[l - 1], qw = s->env_lw[l];
            for (int32_t y = 0; y < ph; ++y)
                for (int32_t x = 0; x < pw; ++x)
                    blk[s->env_noff[l] + (size_t)(y / 2) * qw + x / 2] += blk[s->env_noff[l - 1] + (size_t)y * pw + x];
        }
    }
    free(rc);
    free(rb);
}

void or_env_lookup(const or_scene *s, const double wi[3], double L[3]) {
    L[0] = L[1] = L[2] = 0.0;
    if (!s->d.env) return;
    int32_t W = s->d.env_w, H = s->d.env_h;
    double cy = fmax(-1.0, fmin(1.0, wi[1]));
    double theta = acos(cy);
    double phi = atan2(wi[2], wi[0]);
    if (phi < 0.0) phi += 2.0 * OR_PI;
    int32_t x = (int32_t)floor(phi / (2.0 * OR_PI) * W);
    int32_t y = (int32_t)floor(theta / OR_PI * H);
    if (x >= W) x = W - 1;
    if (x < 0) x = 0;
    if (y >= H) y = H - 1;
    if (y < 0) y = 0;
    const float *p = s->d.env + 3 * ((size_t)y * W + x);
    L[0] = p[0]; L[1] = p[1]; L[2] = p[2];
}

double or_env_pdf(const or_scene *s, const double wi[3]) {
    if (!s->d.env || !(s->env_wsum > 0.0)) return 0.0;
    double L[3];
    or_env_lookup(s, wi, L);
    return or_luminance(L) / s->env_wsum;
}

static int choose(double a, double b, double *u) {
    double p = a / (a + b);
    if (*u < p) { *u = *u / p; return 0; }
    *u = (*u - p) / (1.0 - p);
    if (*u >= 1.0) *u = nextafter(1.0, 0.0);
    return 1;
}

void or_env_sample(const or_scene *s, double u, double v, double wi[3],
                   double *pdf, int32_t *tx, int32_t *ty) {
    int top = s->env_levels - 1;
    int32_t x = choose(envw(s, top, 0, 0), envw(s, top, 1, 0), &u), y = 0;
    for (int l = top - 1; l >= 0; --l) {
        double left = envw(s, l, 2 * x, 2 * y) + envw(s, l, 2 * x, 2 * y + 1);
        double right = envw(s, l, 2 * x + 1, 2 * y) + envw(s, l, 2 * x + 1, 2 * y + 1);
        x = 2 * x + choose(left, right, &u);
        y = 2 * y + choose(envw(s, l, x, 2 * y), envw(s, l, x, 2 * y + 1), &v);
    }
    int32_t W = s->d.env_w, H = s->d.env_h;
    double phi = 2.0 * OR_PI * ((double)x + u) / (double)W;
    double c0 = cos(OR_PI * (double)y / (double)H), c1 = cos(OR_PI * (double)(y + 1) / (double)H);
    double ct = c0 - v * (c0 - c1);
    double st = sqrt(fmax(0.0, 1.0 - ct * ct));
    wi[0] = st * cos(phi); wi[1] = ct; wi[2] = st * sin(phi);
    const float *p = s->d.env + 3 * ((size_t)y * W + x);
    double L[3] = {p[0], p[1], p[2]};
    *pdf = or_luminance(L) / s->env_wsum;
    if (tx) *tx = x;
    if (ty) *ty = y;
}

/* Weight of node (x, y) of level l for normal cell c: reweighted at the
 * normal-oriented levels, plain below them. */
static double envw_n(const or_scene *s, int c, int l, int32_t x, int32_t y) {
    if (!s->env_nw || l < s->env_lstar) return envw(s, l, x, y);
    return s->env_nw[(size_t)c * (size_t)s->env_nstride + (size_t)s->env_noff[l] + (size_t)y * s->env_lw[l] + x];
}

static int choose_p(double p, double *u) {
    if (*u < p) { *u = *u / p; return 0; }
    *u = (*u - p) / (1.0 - p);
    if (*u >= 1.0) *u = nextafter(1.0, 0.0);
    return 1;
}

/* Solid-angle pdf of a direction in finest texel (x0, y0) for normal cell c.
 * The descent reaches region R of the finest reweighted level with
 * probability W_c(R) / W_c(total) and then the texel with the plain share
 * w(texel) / w(R); with W_c(R) = w(R) kappa_c(R) this is kappa_c(R) w(texel)
 * / W_c(total), over the texel's solid angle. A cell whose reweighted total
 * vanishes (nothing lit above any of its normals) uses the plain pyramid. */
static double texel_pdf_n(const or_scene *s, int c, int32_t x0, int32_t y0) {
    int top = s->env_levels - 1;
    int32_t W = s->d.env_w, H = s->d.env_h;
    double total = envw_n(s, c, top, 0, 0) + envw_n(s, c, top, 1, 0);
    if (!(total > 0.0)) return envw(s, 0, x0, y0) / s->env_wsum / texel_solid_angle(W, H, y0);
    int ls = s->env_lstar;
    double region = envw(s, ls, x0 >> ls, y0 >> ls);
    if (!(region > 0.0)) return 0.0;
    double P = envw_n(s, c, ls, x0 >> ls, y0 >> ls) / total;
    return P * envw(s, 0, x0, y0) / region / texel_solid_angle(W, H, y0);
}

static void env_texel_of(const or_scene *s, const double wi[3], int32_t *x, int32_t *y) {
    int32_t W = s->d.env_w, H = s->d.env_h;
    double cy = fmax(-1.0, fmin(1.0, wi[1]));
    double theta = acos(cy);
    double phi = atan2(wi[2], wi[0]);
    if (phi < 0.0) phi += 2.0 * OR_PI;
    *x = (int32_t)floor(phi / (2.0 * OR_PI) * W);
    *y = (int32_t)floor(theta / OR_PI * H);
    if (*x >= W) *x = W - 1;
    if (*x < 0) *x = 0;
    if (*y >= H) *y = H - 1;
    if (*y < 0) *y = 0;
}

double or_env_pdf_n(const or_scene *s, const double ng[3], const double wi[3]) {
    if (!s->env_nw) return or_env_pdf(s, wi);
    int32_t x, y;
    env_texel_of(s, wi, &x, &y);
    return texel_pdf_n(s, or_env_normal_cell(ng), x, y);
}

void or_env_sample_n(const or_scene *s, const double ng[3], double u, double v, double wi[3], double *pdf) {
    int c = or_env_normal_cell(ng);
    int top = s->env_levels - 1;
    if (!s->env_nw || !(envw_n(s, c, top, 0, 0) + envw_n(s, c, top, 1, 0) > 0.0)) {
        or_env_sample(s, u, v, wi, pdf, NULL, NULL);
        if (s->env_nw) *pdf = or_env_pdf_n(s, ng, wi);
        return;
    }
    /* reweighted choices down to the finest reweighted level, plain below */
    double a = envw_n(s, c, top, 0, 0), b = envw_n(s, c, top, 1, 0);
    int32_t x = choose_p(a / (a + b), &u), y = 0;
    for (int l = top - 1; l >= 0; --l) {
        double ln = envw_n(s, c, l, 2 * x, 2 * y) + envw_n(s, c, l, 2 * x, 2 * y + 1);
        double rn = envw_n(s, c, l, 2 * x + 1, 2 * y) + envw_n(s, c, l, 2 * x + 1, 2 * y + 1);
        x = 2 * x + choose_p(ln / (ln + rn), &u);
        double t0 = envw_n(s, c, l, x, 2 * y), t1 = envw_n(s, c, l, x, 2 * y + 1);
        y = 2 * y + choose_p(t0 / (t0 + t1), &v);
    }
    int32_t W = s->d.env_w, H = s->d.env_h;
    double phi = 2.0 * OR_PI * ((double)x + u) / (double)W;
    double c0 = cos(OR_PI * (double)y / (double)H), c1 = cos(OR_PI * (double)(y + 1) / (double)H);
    double ct = c0 - v * (c0 - c1);
    double st = sqrt(fmax(0.0, 1.0 - ct * ct));
    wi[0] = st * cos(phi); wi[1] = ct; wi[2] = st * sin(phi);
    *pdf = texel_pdf_n(s, c, x, y);
}

void or_env_texel_probs_n(const or_scene *s, int cell, double *texel_prob) {
    int32_t W = s->d.env_w, H = s->d.env_h;
    for (int32_t y = 0; y < H; ++y)
        for (int32_t x = 0; x < W; ++x) {
            double pdf = s->env_nw ? texel_pdf_n(s, cell, x, y)
                                   : envw(s, 0, x, y) / s->env_wsum / texel_solid_angle(W, H, y);
            texel_prob[(size_t)y * W + x] = pdf * texel_solid_angle(W, H, y);
        }
}

/* Probability of every finest texel under the descent: the product of the
 * conditional choices along its path, accumulated top-down. */
void or_env_pyramid_probs(const float *env, int32_t W, int32_t H,
                          double *texel_prob) {
    or_scene_desc d;
    memset(&d, 0, sizeof d);
    d.env = env; d.env_w = W; d.env_h = H;
    or_scene *s = or_scene_create(&d);
    int top = s->env_levels - 1;
    double *cur = (double *)malloc(sizeof(double) * 2);
    double a = envw(s, top, 0, 0), b = envw(s, top, 1, 0);
    cur[0] = a / (a + b); cur[1] = b / (a + b);
    int32_t cw = 2, ch = 1;
    for (int l = top - 1; l >= 0; --l) {
        int32_t nw = s->env_lw[l], nh = s->env_lh[l];
        double *nxt = (double *)calloc((size_t)nw * (size_t)nh, sizeof(double));
        for (int32_t y = 0; y < ch; ++y)
            for (int32_t x = 0; x < cw; ++x) {
                double P = cur[(size_t)y * cw + x];
                if (P == 0.0) continue;
                double left = envw(s, l, 2 * x, 2 * y) + envw(s, l, 2 * x, 2 * y + 1);
                double right = envw(s, l, 2 * x + 1, 2 * y) + envw(s, l, 2 * x + 1, 2 * y + 1);
                for (int cx = 0; cx < 2; ++cx) {
                    double pc = (cx == 0 ? left : right) / (left + right);
                    int32_t X = 2 * x + cx;
                    double t0 = envw(s, l, X, 2 * y), t1 = envw(s, l, X, 2 * y + 1);
                    if (t0 + t1 == 0.0) continue;
                    nxt[(size_t)(2 * y) * nw + X] += P * pc * t0 / (t0 + t1);
                    nxt[(size_t)(2 * y + 1) * nw + X] += P * pc * t1 / (t0 + t1);
                }
            }
        free(cur); cur = nxt; cw = nw; ch = nh;
    }
    memcpy(texel_prob, cur, sizeof(double) * (size_t)W * (size_t)H);
    free(cur);
    or_scene_destroy(s);
}

/* ------------------------------------------------------------- emitters */
static void material_emission_avg(const or_scene *s, uint32_t m, double Le[3]) {
    const float *e = s->d.emission + 3 * m;
    Le[0] = e[0]; Le[1] = e[1]; Le[2] = e[2];
}

static double tex_lum(const or_scene *s, int32_t tex, int32_t x, int32_t y) {
    const float *p = s->d.textures + 3 * (((size_t)tex * s->d.tex_h + y) * s->d.tex_w + x);
    double c[3] = {p[0], p[1], p[2]};
    return or_luminance(c);
}

/* Area of the polygon obtained by clipping a 2D triangle to [x0,x1]x[y0,y1]
 * (Sutherland-Hodgman against the four half-planes, then the shoelace sum). */
static double clip_area(const double tri[3][2], double x0, double x1, double y0,
                        double y1) {
    double poly[16][2], tmp[16][2];
    int n = 3;
    for (int i = 0; i < 3; ++i) { poly[i][0] = tri[i][0]; poly[i][1] = tri[i][1]; }
    for (int side = 0; side < 4; ++side) {
        int m = 0;
        for (int i = 0; i < n; ++i) {
            const double *a = poly[i], *b = poly[(i + 1) % n];
            double da, db;
            switch (side) {
                case 0: da = a[0] - x0; db = b[0] - x0; break;
                case 1: da = x1 - a[0]; db = x1 - b[0]; break;
                case 2: da = a[1] - y0; db = b[1] - y0; break;
                default: da = y1 - a[1]; db = y1 - b[1]; break;
            }
            if (da >= 0.0) { tmp[m][0] = a[0]; tmp[m][1] = a[1]; ++m; }
            if ((da >= 0.0) != (db >= 0.0)) {
                double t = da / (da - db);
                tmp[m][0] = a[0] + t * (b[0] - a[0]);
                tmp[m][1] = a[1] + t * (b[1] - a[1]);
                ++m;
            }
        }
        n = m;
        for (int i = 0; i < n; ++i) { poly[i][0] = tmp[i][0]; poly[i][1] = tmp[i][1]; }
        if (n == 0) return 0.0;
    }
    double acc = 0.0;
    for (int i = 0; i < n; ++i) {
        const double *a = poly[i], *b = poly[(i + 1) % n];
        acc += a[0] * b[1] - b[0] * a[1];
    }
    return 0.5 * fabs(acc);
}

/* Mean luminance of a textured emitter over its triangle: nearest-texel
 * emission integrated exactly over the triangle's UV footprint. */
static double textured_mean_lum(const or_scene *s, int64_t t, int32_t tex) {
    const uint32_t *id = s->d.indices + 3 * t;
    int32_t tw = s->d.tex_w, th = s->d.tex_h;
    double tri[3][2];
    for (int k = 0; k < 3; ++k) {
        tri[k][0] = fmin(1.0, fmax(0.0, (double)s->d.uvs[2 * id[k]])) * tw;
        tri[k][1] = fmin(1.0, fmax(0.0, (double)s->d.uvs[2 * id[k] + 1])) * th;
    }
    double auv = 0.5 * fabs((tri[1][0] - tri[0][0]) * (tri[2][1] - tri[0][1]) -
                            (tri[2][0] - tri[0][0]) * (tri[1][1] - tri[0][1]));
    if (!(auv > 0.0)) {
        int32_t x = (int32_t)fmin(tw - 1, floor(tri[0][0]));
        int32_t y = (int32_t)fmin(th - 1, floor(tri[0][1]));
        return tex_lum(s, tex, x, y);
    }
    double acc = 0.0;
    int32_t xa = (int32_t)floor(fmin(tri[0][0], fmin(tri[1][0], tri[2][0])));
    int32_t xb = (int32_t)floor(fmax(tri[0][0], fmax(tri[1][0], tri[2][0])));
    int32_t ya = (int32_t)floor(fmin(tri[0][1], fmin(tri[1][1], tri[2][1])));
    int32_t yb = (int32_t)floor(fmax(tri[0][1], fmax(tri[1][1], tri[2][1])));
    for (int32_t y = ya; y <= yb; ++y)
        for (int32_t x = xa; x <= xb; ++x) {
            int32_t cx = x < 0 ? 0 : (x >= tw ? tw - 1 : x);
            int32_t cy = y < 0 ? 0 : (y >= th ? th - 1 : y);
            double a = clip_area(tri, x, x + 1, y, y + 1);
            if (a > 0.0) acc += a * tex_lum(s, tex, cx, cy);
        }
    return acc / auv;
}

void or_tri_emission(const or_scene *s, uint32_t prim, double b1, double b2,
                     double Le[3]) {
    uint32_t m = s->d.tri_material[prim];
    material_emission_avg(s, m, Le);
    int32_t tex = s->d.emission_tex ? s->d.emission_tex[m] : -1;
    if (tex < 0) return;
    const uint32_t *id = s->d.indices + 3 * (size_t)prim;
    double b0 = 1.0 - b1 - b2;
    double u = b0 * s->d.uvs[2 * id[0]] + b1 * s->d.uvs[2 * id[1]] + b2 * s->d.uvs[2 * id[2]];
    double v = b0 * s->d.uvs[2 * id[0] + 1] + b1 * s->d.uvs[2 * id[1] + 1] + b2 * s->d.uvs[2 * id[2] + 1];
    int32_t tw = s->d.tex_w, th = s->d.tex_h;
    int32_t x = (int32_t)floor(fmin(1.0, fmax(0.0, u)) * tw);
    int32_t y = (int32_t)floor(fmin(1.0, fmax(0.0, v)) * th);
    if (x >= tw) x = tw - 1;
    if (y >= th) y = th - 1;
    const float *p = s->d.textures + 3 * (((size_t)tex * th + y) * tw + x);
    for (int c = 0; c < 3; ++c) Le[c] *= p[c];
}

void or_build_lights(or_scene *s) {
    s->tri_light_pdf_area = (double *)calloc((size_t)(s->nt > 0 ? s->nt : 1), sizeof(double));
    int64_t nl = 0;
    double *flux = (double *)malloc(sizeof(double) * (size_t)(s->nt > 0 ? s->nt : 1));
    int64_t *ids = (int64_t *)malloc(sizeof(int64_t) * (size_t)(s->nt > 0 ? s->nt : 1));
    double total = 0.0;
    for (int64_t t = 0; t < s->nt; ++t) {
        uint32_t m = s->d.tri_material[t];
        double Le[3];
        material_emission_avg(s, m, Le);
        double lum = or_luminance(Le);
        if (!(lum > 0.0) || !(s->area[t] > 0.0)) continue;
        int32_t tex = s->d.emission_tex ? s->d.emission_tex[m] : -1;
        if (tex >= 0) lum *= textured_mean_lum(s, t, tex);
        if (!(lum > 0.0)) continue;
        flux[nl] = lum * s->area[t];
        ids[nl] = t;
        total += flux[nl];
        ++nl;
    }
    s->nlights = nl;
    s->flux_sum = total;
    s->light_flux = (double *)malloc(sizeof(double) * (size_t)(nl > 0 ? nl : 1));
    for (int64_t i = 0; i < nl; ++i) s->light_flux[i] = flux[i];
    s->light_of_tri = (int64_t *)malloc(sizeof(int64_t) * (size_t)(s->nt > 0 ? s->nt : 1));
    for (int64_t t = 0; t < s->nt; ++t) s->light_of_tri[t] = -1;
    for (int64_t i = 0; i < nl; ++i) s->light_of_tri[ids[i]] = i;
    s->light_tri = ids;
    s->light_prob = flux;
    s->alias_prob = (double *)malloc(sizeof(double) * (size_t)(nl > 0 ? nl : 1));
    s->alias_idx = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nl > 0 ? nl : 1));
    if (nl > 0) or_alias_build(flux, nl, s->alias_prob, s->alias_idx);
    int has_env = s->d.env && s->env_wsum > 0.0;
    s->p_env = has_env ? (nl > 0 ? 0.5 : 1.0) : 0.0;
    for (int64_t i = 0; i < nl; ++i) {
        s->light_prob[i] = flux[i] / total;
        s->tri_light_pdf_area[ids[i]] = (1.0 - s->p_env) * s->light_prob[i] / s->area[ids[i]];
    }
}

double or_scene_light_pdf_area(const or_scene *s, uint32_t prim) {
    return s->tri_light_pdf_area[prim];
}
double or_scene_env_select_prob(const or_scene *s) { return s->p_env; }

/* ----------------------------------------------------------- scene object */
or_scene *or_scene_create(const or_scene_desc *d) {
    or_scene *s = (or_scene *)calloc(1, sizeof(or_scene));
    s->d = *d;
    s->nt = d->nt;
    size_t nt = (size_t)(d->nt > 0 ? d->nt : 1);
    s->v64 = (double *)malloc(sizeof(double) * 9 * nt);
    s->ng = (double *)malloc(sizeof(double) * 3 * nt);
    s->area = (double *)malloc(sizeof(double) * nt);
    for (int64_t t = 0; t < d->nt; ++t) {
        for (int k = 0; k < 3; ++k)
            for (int a = 0; a < 3; ++a)
                s->v64[9 * t + 3 * k + a] = d->vertices[3 * (size_t)d->indices[3 * t + k] + a];
        const double *v = s->v64 + 9 * t;
        double e1[3] = {v[3] - v[0], v[4] - v[1], v[5] - v[2]};
        double e2[3] = {v[6] - v[0], v[7] - v[1], v[8] - v[2]};
        double c[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2],
                       e1[0] * e2[1] - e1[1] * e2[0]};
        double l = sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
        s->area[t] = 0.5 * l;
        for (int a = 0; a < 3; ++a) s->ng[3 * t + a] = l > 0.0 ? c[a] / l : 0.0;
    }
    or_build_bvh(s);
    build_env(s);
    build_env_normal_levels(s);
    if (d->tri_material) {
        or_build_lights(s);
        or_build_light_bvh(s);
    }
    or_build_photon_aiming(s);
    return s;
}

void or_scene_destroy(or_scene *s) {
    if (!s) return;
    free(s->v64); free(s->ng); free(s->area); free(s->nodes); free(s->bvh_prims);
    free(s->light_tri); free(s->light_prob); free(s->alias_prob); free(s->alias_idx);
    free(s->tri_light_pdf_area);
    free(s->light_flux); free(s->light_of_tri);
    free(s->lb_nodes); free(s->lb_perm); free(s->lb_leaf_of);
    for (int l = 0; l < s->env_levels; ++l) free(s->env_w[l]);
    free(s->env_w); free(s->env_lw); free(s->env_lh); free(s->env_nw);
    free(s->pa_cc); free(s->pa_nodes); free(s->pa_obj_cluster);
    free(s);
}
