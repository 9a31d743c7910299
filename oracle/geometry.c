/*
 * Oracle: scene set-up and ray casting in FP64 (paper Sec. 2.3 "watertight
 * ray traversal and triangle intersection", Sec. 3.1 rays -> hits).
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Intersection is the watertight test of Woop, Benthin and Wald (JCGT 2013)
 * evaluated in double precision on the FP32 input vertices. Closest hit =
 * smallest t in (tmin, tmax); equal t -> the lower primitive index. Rays are
 * cast either against every triangle (brute force) or through a plain binary
 * BVH with median splits whose boxes are padded so that it can never reject
 * a triangle the brute-force loop would accept.
 */
#include "oracle.h"
#include "oracle_internal.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------ watertight intersection */
int or_intersect_tri(const double o[3], const double d[3], double tmin,
                     double tmax, const double v0[3], const double v1[3],
                     const double v2[3], double *t_out, double *b1, double *b2) {
    int kz = 0;
    if (fabs(d[1]) > fabs(d[kz])) kz = 1;
    if (fabs(d[2]) > fabs(d[kz])) kz = 2;
    int kx = (kz + 1) % 3, ky = (kx + 1) % 3;
    if (d[kz] < 0.0) { int tmp = kx; kx = ky; ky = tmp; }
    double Sx = d[kx] / d[kz], Sy = d[ky] / d[kz], Sz = 1.0 / d[kz];
    double A[3], B[3], C[3];
    for (int a = 0; a < 3; ++a) { A[a] = v0[a] - o[a]; B[a] = v1[a] - o[a]; C[a] = v2[a] - o[a]; }
    double Ax = A[kx] - Sx * A[kz], Ay = A[ky] - Sy * A[kz];
    double Bx = B[kx] - Sx * B[kz], By = B[ky] - Sy * B[kz];
    double Cx = C[kx] - Sx * C[kz], Cy = C[ky] - Sy * C[kz];
    double U = Cx * By - Cy * Bx;
    double V = Ax * Cy - Ay * Cx;
    double W = Bx * Ay - By * Ax;
    if ((U < 0.0 || V < 0.0 || W < 0.0) && (U > 0.0 || V > 0.0 || W > 0.0))
        return 0;
    double det = U + V + W;
    if (det == 0.0) return 0;
    double Az = Sz * A[kz], Bz = Sz * B[kz], Cz = Sz * C[kz];
    double T = U * Az + V * Bz + W * Cz;
    double t = T / det;
    if (!(t > tmin && t < tmax)) return 0;
    *t_out = t;
    *b1 = V / det;
    *b2 = W / det;
    return 1;
}

/* ------------------------------------------------------------ binary BVH */
typedef struct { double lo[3], hi[3]; int64_t left, right, first, count; } bnode;

static void tri_bounds(const or_scene *s, int64_t t, double lo[3], double hi[3]) {
    const double *v = s->v64 + 9 * t;
    for (int a = 0; a < 3; ++a) {
        lo[a] = fmin(v[a], fmin(v[3 + a], v[6 + a]));
        hi[a] = fmax(v[a], fmax(v[3 + a], v[6 + a]));
    }
}

typedef struct { double key; int64_t prim; } keyed;

static int cmp_keyed(const void *a, const void *b) {
    const keyed *x = (const keyed *)a, *y = (const keyed *)b;
    if (x->key < y->key) return -1;
    if (x->key > y->key) return 1;
    return (x->prim > y->prim) - (x->prim < y->prim);
}

static int64_t build_rec(or_scene *s, int64_t first, int64_t count) {
    int64_t id = s->nnodes++;
    bnode *n = &((bnode *)s->nodes)[id];
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    double clo[3] = {INFINITY, INFINITY, INFINITY}, chi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = first; i < first + count; ++i) {
        double tl[3], th[3];
        tri_bounds(s, s->bvh_prims[i], tl, th);
        for (int a = 0; a < 3; ++a) {
            lo[a] = fmin(lo[a], tl[a]); hi[a] = fmax(hi[a], th[a]);
            double c = 0.5 * (tl[a] + th[a]);
            clo[a] = fmin(clo[a], c); chi[a] = fmax(chi[a], c);
        }
    }
    double ext = 0.0;
    for (int a = 0; a < 3; ++a) ext = fmax(ext, fmax(fabs(lo[a]), fabs(hi[a])));
    double pad = 1e-9 * (ext + 1.0);
    for (int a = 0; a < 3; ++a) { n->lo[a] = lo[a] - pad; n->hi[a] = hi[a] + pad; }
    if (count <= 4) {
        n->left = n->right = -1; n->first = first; n->count = count;
        return id;
    }
    int axis = 0;
    for (int a = 1; a < 3; ++a)
        if (chi[a] - clo[a] > chi[axis] - clo[axis]) axis = a;
    /* median split: sort the range by centroid along the axis */
    keyed *tmp = (keyed *)malloc(sizeof(keyed) * (size_t)count);
    for (int64_t i = 0; i < count; ++i) {
        double tl[3], th[3];
        tri_bounds(s, s->bvh_prims[first + i], tl, th);
        tmp[i].key = 0.5 * (tl[axis] + th[axis]);
        tmp[i].prim = s->bvh_prims[first + i];
    }
    qsort(tmp, (size_t)count, sizeof(keyed), cmp_keyed);
    for (int64_t i = 0; i < count; ++i) s->bvh_prims[first + i] = tmp[i].prim;
    free(tmp);
    int64_t mid = first + count / 2;
    n->first = -1; n->count = 0;
    int64_t l = build_rec(s, first, mid - first);
    int64_t r = build_rec(s, mid, first + count - mid);
    n = &((bnode *)s->nodes)[id];
    n->left = l; n->right = r;
    return id;
}

void or_build_bvh(or_scene *s) {
    s->bvh_prims = (int64_t *)malloc(sizeof(int64_t) * (size_t)(s->nt > 0 ? s->nt : 1));
    for (int64_t i = 0; i < s->nt; ++i) s->bvh_prims[i] = i;
    s->nodes = malloc(sizeof(bnode) * (size_t)(2 * s->nt + 1));
    s->nnodes = 0;
    if (s->nt > 0) build_rec(s, 0, s->nt);
}

int64_t or_bvh_node_count(const or_scene *s) { return s->nnodes; }

static int box_hit(const bnode *n, const double o[3], const double d[3],
                   double tmin, double tmax) {
    double t0 = tmin, t1 = tmax;
    for (int a = 0; a < 3; ++a) {
        if (d[a] == 0.0) {
            if (o[a] < n->lo[a] || o[a] > n->hi[a]) return 0;
            continue;
        }
        double inv = 1.0 / d[a];
        double ta = (n->lo[a] - o[a]) * inv, tb = (n->hi[a] - o[a]) * inv;
        if (ta > tb) { double tmp = ta; ta = tb; tb = tmp; }
        if (ta > t0) t0 = ta;
        if (tb < t1) t1 = tb;
        if (t0 > t1) return 0;
    }
    return 1;
}

/* Closest (or any) hit through the BVH. Ties in t go to the lower prim. */
static void trace_bvh(const or_scene *s, const double o[3], const double d[3],
                      double tmin, double tmax, int any_hit, uint32_t *prim,
                      double *t, double *b1, double *b2) {
    *prim = OR_MISS; *t = INFINITY; *b1 = *b2 = 0.0;
    if (s->nnodes == 0) return;
    const bnode *nodes = (const bnode *)s->nodes;
    int64_t stack[256]; int sp = 0;
    stack[sp++] = 0;
    double best = tmax;
    while (sp > 0) {
        const bnode *n = &nodes[stack[--sp]];
        /* best is inclusive here so that an equal-t triangle is still seen */
        if (!box_hit(n, o, d, tmin, best)) continue;
        if (n->left < 0) {
            for (int64_t i = n->first; i < n->first + n->count; ++i) {
                int64_t tri = s->bvh_prims[i];
                const double *v = s->v64 + 9 * tri;
                double th, u1, u2;
                /* accept t <= best: strict t < best is checked after */
                if (or_intersect_tri(o, d, tmin, nextafter(best, INFINITY), v, v + 3, v + 6, &th, &u1, &u2)) {
                    if (th < best || (th == best && (uint32_t)tri < *prim)) {
                        if (th == tmax) continue;
                        best = th; *t = th; *prim = (uint32_t)tri; *b1 = u1; *b2 = u2;
                        if (any_hit) return;
                    }
                }
            }
        } else {
            stack[sp++] = n->left;
            stack[sp++] = n->right;
        }
    }
}

static void trace_brute(const or_scene *s, const double o[3], const double d[3],
                        double tmin, double tmax, int any_hit, uint32_t *prim,
                        double *t, double *b1, double *b2) {
    *prim = OR_MISS; *t = INFINITY; *b1 = *b2 = 0.0;
    double best = tmax;
    for (int64_t tri = 0; tri < s->nt; ++tri) {
        const double *v = s->v64 + 9 * tri;
        double th, u1, u2;
        if (or_intersect_tri(o, d, tmin, best, v, v + 3, v + 6, &th, &u1, &u2)) {
            best = th; *t = th; *prim = (uint32_t)tri; *b1 = u1; *b2 = u2;
            if (any_hit) return;
        }
    }
}

void or_trace_one(const or_scene *s, const double o[3], const double d[3],
                  double tmin, double tmax, int any_hit, uint32_t *prim,
                  double *t, double *b1, double *b2) {
    if (s->nt <= 64) trace_brute(s, o, d, tmin, tmax, any_hit, prim, t, b1, b2);
    else trace_bvh(s, o, d, tmin, tmax, any_hit, prim, t, b1, b2);
}

void or_trace(const or_scene *s, const float *rays, int64_t n, int any_hit,
              int use_bvh, uint32_t *prim, double *t, double *b1, double *b2) {
    for (int64_t r = 0; r < n; ++r) {
        const float *ry = rays + 8 * r;
        double o[3] = {ry[0], ry[1], ry[2]}, d[3] = {ry[3], ry[4], ry[5]};
        if (use_bvh)
            trace_bvh(s, o, d, ry[6], ry[7], any_hit, &prim[r], &t[r], &b1[r], &b2[r]);
        else
            trace_brute(s, o, d, ry[6], ry[7], any_hit, &prim[r], &t[r], &b1[r], &b2[r]);
    }
}
