/*
 * Oracle: photon aiming for the light-tracing stage (paper Sec. 2.1.3).
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * The section gives the ingredients, not the formulas: objects are grouped
 * into clusters bottom-up, merging nearby clusters of similar size, with a
 * criterion that makes the result independent of the merge order; a photon
 * picks a cluster by descending a bounding-volume hierarchy over the
 * clusters, each step choosing a child in proportion to an optimistic
 * estimate of the screen-space photon density it would receive, and is then
 * aimed uniformly at the chosen cluster's bounding volume; the density for
 * MIS sums over every cluster whose volume the emission ray passes.
 *
 * Readings fixed here (the same on the CUDA side):
 *   - objects: the connected components of the triangle mesh (triangles
 *     sharing a vertex index); bounding sphere = centre and half diagonal of
 *     the component's box;
 *   - clusters: connected components of the graph that links two objects
 *     a, b when they are similar, r_a <= 2 r_b and r_b <= 2 r_a (neither is
 *     much larger than the other), and nearby, their boxes intersect
 *     (touching counts); merging linked objects in any order gives the same
 *     clusters;
 *     a cluster's sphere = centre and half diagonal of its box;
 *   - hierarchy: binary, a set of clusters split at its median cluster
 *     along the longest axis of their centres' box (ordered by centre, then
 *     index), one cluster per leaf; a node's sphere is centred on its box
 *     and encloses every cluster sphere below it;
 *   - estimate of a node for a photon: the solid angle under which the eye
 *     sees the node's sphere, 2 pi (1 - sqrt(1 - r^2/d^2)), 4 pi when the
 *     eye is inside, capped at the solid angle of the camera's view cone
 *     (the cone around the optical axis through the image corners): the
 *     optimistic bound of the screen area a cluster of that size can take.
 *     Aiming uniformly at a sphere of radius r puts 1/(pi r^2) photons per
 *     unit area on it and a pixel at distance d covers an area proportional
 *     to d^2, so clusters chosen in proportion to r^2/d^2 receive about as
 *     many photons per pixel; the cap keeps a cluster around the eye (a
 *     ground plane) from taking photons that its huge sphere mostly sends
 *     out of view. For a photon from a triangle emitter the estimate is zero
 *     when the node's sphere lies wholly behind the emitter's plane. A child
 *     is chosen with probability proportional to its estimate (one half each
 *     when both vanish);
 *   - aiming: an environment photon of direction w (from the plain pyramid)
 *     starts at a uniform point of the disk of the chosen cluster's sphere
 *     across w, moved back along w outside the scene's bounding sphere, and
 *     travels along -w; a triangle photon from point y leaves in a direction
 *     uniform in the cone from y that the chosen sphere subtends (uniform
 *     over all directions when y is inside it);
 *   - densities: an environment photon's line through a point x has
 *     density sum over clusters c whose sphere the line meets of P_c / (pi
 *     r_c^2) per unit area across w; a triangle photon's direction has
 *     solid-angle density sum over clusters c whose cone holds it of P_c(y)
 *     / (2 pi (1 - cos theta_c)).
 */
#include "oracle.h"
#include "oracle_internal.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define OR_PI 3.14159265358979323846

static int32_t uf_find(int32_t *p, int32_t a) {
    while (p[a] != a) {
        p[a] = p[p[a]];
        a = p[a];
    }
    return a;
}
static void uf_union(int32_t *p, int32_t a, int32_t b) {
    a = uf_find(p, a);
    b = uf_find(p, b);
    if (a == b) return;
    if (a < b) p[b] = a; else p[a] = b;
}

typedef struct {
    double lo[3], hi[3];
    double c[3], r;
} pa_box;

static void box_empty(pa_box *b) {
    for (int a = 0; a < 3; ++a) { b->lo[a] = INFINITY; b->hi[a] = -INFINITY; }
}
static void box_grow_pt(pa_box *b, const double p[3]) {
    for (int a = 0; a < 3; ++a) {
        if (p[a] < b->lo[a]) b->lo[a] = p[a];
        if (p[a] > b->hi[a]) b->hi[a] = p[a];
    }
}
static void box_grow(pa_box *b, const pa_box *o) {
    box_grow_pt(b, o->lo);
    box_grow_pt(b, o->hi);
}
static void box_sphere(pa_box *b) {
    double d2 = 0.0;
    for (int a = 0; a < 3; ++a) {
        b->c[a] = 0.5 * (b->lo[a] + b->hi[a]);
        double e = b->hi[a] - b->lo[a];
        d2 += e * e;
    }
    b->r = 0.5 * sqrt(d2);
}

/* recursive median split over clusters idx[0..n) */
typedef struct {
    or_scene *s;
    const pa_box *cb;   /* cluster boxes */
    int32_t *idx;
    int axis;
} pa_build_ctx;

static pa_build_ctx *g_sort_ctx;   /* qsort has no context argument; the build is single-threaded */
static int cmp_centre(const void *pa, const void *pb) {
    int32_t a = *(const int32_t *)pa, b = *(const int32_t *)pb;
    double ca = g_sort_ctx->cb[a].c[g_sort_ctx->axis], cbv = g_sort_ctx->cb[b].c[g_sort_ctx->axis];
    if (ca < cbv) return -1;
    if (ca > cbv) return 1;
    return a < b ? -1 : (a > b ? 1 : 0);
}

static int32_t build_node(pa_build_ctx *x, int32_t *idx, int32_t n) {
    or_scene *s = x->s;
    int32_t id = s->pa_nnodes++;
    or_pa_node *nd = &s->pa_nodes[id];
    pa_box nb;
    box_empty(&nb);
    for (int32_t i = 0; i < n; ++i) box_grow(&nb, &x->cb[idx[i]]);
    box_sphere(&nb);
    double r = 0.0;
    for (int32_t i = 0; i < n; ++i) {
        const pa_box *c = &x->cb[idx[i]];
        double d = sqrt((c->c[0] - nb.c[0]) * (c->c[0] - nb.c[0]) + (c->c[1] - nb.c[1]) * (c->c[1] - nb.c[1]) +
                        (c->c[2] - nb.c[2]) * (c->c[2] - nb.c[2]));
        if (d + c->r > r) r = d + c->r;
    }
    for (int a = 0; a < 3; ++a) nd->c[a] = nb.c[a];
    nd->r = r;
    if (n == 1) {
        nd->left = nd->right = -1;
        nd->cluster = idx[0];
        return id;
    }
    nd->cluster = -1;
    pa_box cen;
    box_empty(&cen);
    for (int32_t i = 0; i < n; ++i) box_grow_pt(&cen, x->cb[idx[i]].c);
    int axis = 0;
    double ext = cen.hi[0] - cen.lo[0];
    for (int a = 1; a < 3; ++a)
        if (cen.hi[a] - cen.lo[a] > ext) { ext = cen.hi[a] - cen.lo[a]; axis = a; }
    x->axis = axis;
    g_sort_ctx = x;
    qsort(idx, (size_t)n, sizeof(int32_t), cmp_centre);
    int32_t h = n / 2;
    int32_t l = build_node(x, idx, h);
    int32_t rr = build_node(x, idx + h, n - h);
    s->pa_nodes[id].left = l;
    s->pa_nodes[id].right = rr;
    return id;
}

void or_build_photon_aiming(or_scene *s) {
    s->pa_nclusters = 0;
    s->pa_nnodes = 0;
    if (s->nt <= 0) return;
    int64_t nv = s->d.nv;
    /* objects: components over shared vertex indices */
    int32_t *vp = (int32_t *)malloc(sizeof(int32_t) * (size_t)nv);
    for (int64_t i = 0; i < nv; ++i) vp[i] = (int32_t)i;
    for (int64_t t = 0; t < s->nt; ++t) {
        const uint32_t *id = s->d.indices + 3 * (size_t)t;
        uf_union(vp, (int32_t)id[0], (int32_t)id[1]);
        uf_union(vp, (int32_t)id[0], (int32_t)id[2]);
    }
    int32_t *obj_of_root = (int32_t *)malloc(sizeof(int32_t) * (size_t)nv);
    for (int64_t i = 0; i < nv; ++i) obj_of_root[i] = -1;
    int32_t nobj = 0;
    /* number objects in the order of their first triangle */
    int32_t *tri_obj = (int32_t *)malloc(sizeof(int32_t) * (size_t)s->nt);
    for (int64_t t = 0; t < s->nt; ++t) {
        int32_t r = uf_find(vp, (int32_t)s->d.indices[3 * (size_t)t]);
        if (obj_of_root[r] < 0) obj_of_root[r] = nobj++;
        tri_obj[t] = obj_of_root[r];
    }
    pa_box *ob = (pa_box *)malloc(sizeof(pa_box) * (size_t)nobj);
    for (int32_t o = 0; o < nobj; ++o) box_empty(&ob[o]);
    for (int64_t t = 0; t < s->nt; ++t)
        for (int k = 0; k < 3; ++k) box_grow_pt(&ob[tri_obj[t]], s->v64 + 9 * (size_t)t + 3 * k);
    for (int32_t o = 0; o < nobj; ++o) box_sphere(&ob[o]);
    /* clusters: components of the similar-and-nearby graph */
    int32_t *op = (int32_t *)malloc(sizeof(int32_t) * (size_t)nobj);
    for (int32_t o = 0; o < nobj; ++o) op[o] = o;
    for (int32_t a = 0; a < nobj; ++a)
        for (int32_t b = a + 1; b < nobj; ++b) {
            double ra = ob[a].r, rb = ob[b].r;
            if (!(ra <= 2.0 * rb && rb <= 2.0 * ra)) continue;
            int apart = 0;
            for (int k = 0; k < 3; ++k)
                if (ob[a].lo[k] > ob[b].hi[k] || ob[b].lo[k] > ob[a].hi[k]) apart = 1;
            if (!apart) uf_union(op, a, b);
        }
    int32_t *cl_of_root = (int32_t *)malloc(sizeof(int32_t) * (size_t)nobj);
    for (int32_t o = 0; o < nobj; ++o) cl_of_root[o] = -1;
    int32_t ncl = 0;
    int32_t *obj_cl = (int32_t *)malloc(sizeof(int32_t) * (size_t)nobj);
    for (int32_t o = 0; o < nobj; ++o) {
        int32_t r = uf_find(op, o);
        if (cl_of_root[r] < 0) cl_of_root[r] = ncl++;
        obj_cl[o] = cl_of_root[r];
    }
    pa_box *cb = (pa_box *)malloc(sizeof(pa_box) * (size_t)ncl);
    for (int32_t c = 0; c < ncl; ++c) box_empty(&cb[c]);
    for (int32_t o = 0; o < nobj; ++o) box_grow(&cb[obj_cl[o]], &ob[o]);
    for (int32_t c = 0; c < ncl; ++c) box_sphere(&cb[c]);
    s->pa_nclusters = ncl;
    s->pa_nobjects = nobj;
    s->pa_cc = (double *)malloc(sizeof(double) * 4 * (size_t)ncl);
    for (int32_t c = 0; c < ncl; ++c) {
        for (int a = 0; a < 3; ++a) s->pa_cc[4 * c + a] = cb[c].c[a];
        s->pa_cc[4 * c + 3] = cb[c].r;
    }
    s->pa_obj_cluster = obj_cl;
    s->pa_nodes = (or_pa_node *)calloc(2 * (size_t)ncl, sizeof(or_pa_node));
    int32_t *idx = (int32_t *)malloc(sizeof(int32_t) * (size_t)ncl);
    for (int32_t c = 0; c < ncl; ++c) idx[c] = c;
    pa_build_ctx x = {s, cb, idx, 0};
    build_node(&x, idx, ncl);
    free(idx); free(cb); free(cl_of_root); free(op); free(ob); free(tri_obj); free(obj_of_root); free(vp);
}

/* Estimate of a node: solid angle of its sphere seen from the eye; zero for
 * a triangle photon (front != NULL: emitter point y, normal n) when the
 * sphere is wholly behind the emitter's plane. */
static double node_weight(const or_pa_node *n, const double eye[4], const double *y, const double *ny) {
    if (y) {
        double s = (n->c[0] - y[0]) * ny[0] + (n->c[1] - y[1]) * ny[1] + (n->c[2] - y[2]) * ny[2];
        if (!(s > -n->r)) return 0.0;
    }
    double dx = n->c[0] - eye[0], dy = n->c[1] - eye[1], dz = n->c[2] - eye[2];
    double d2 = dx * dx + dy * dy + dz * dz, r2 = n->r * n->r;
    double om = 4.0 * OR_PI;
    if (d2 > r2) {
        double x = r2 / d2;
        om = 2.0 * OR_PI * x / (1.0 + sqrt(1.0 - x));   /* 2 pi (1 - sqrt(1 - x)) */
    }
    return om < eye[3] ? om : eye[3];                   /* at most the screen's solid angle */
}

double or_pa_p_left(const or_scene *s, int32_t node, const double eye[4], const double *y, const double *ny) {
    const or_pa_node *n = &s->pa_nodes[node];
    double wl = node_weight(&s->pa_nodes[n->left], eye, y, ny);
    double wr = node_weight(&s->pa_nodes[n->right], eye, y, ny);
    if (!(wl + wr > 0.0)) return 0.5;
    return wl / (wl + wr);
}

int32_t or_pa_sample(const or_scene *s, const double eye[4], const double *y, const double *ny, double u,
                     double *prob) {
    int32_t node = 0;
    double p = 1.0;
    while (s->pa_nodes[node].cluster < 0) {
        double pl = or_pa_p_left(s, node, eye, y, ny);
        if (u < pl) {
            u = u / pl;
            p *= pl;
            node = s->pa_nodes[node].left;
        } else {
            u = (u - pl) / (1.0 - pl);
            p *= 1.0 - pl;
            node = s->pa_nodes[node].right;
        }
        if (u >= 1.0) u = nextafter(1.0, 0.0);
    }
    if (prob) *prob = p;
    return s->pa_nodes[node].cluster;
}

/* every cluster's probability, by the plain product down the tree */
static void probs_rec(const or_scene *s, int32_t node, double p, const double eye[4], const double *y,
                      const double *ny, double *P) {
    const or_pa_node *n = &s->pa_nodes[node];
    if (n->cluster >= 0) { P[n->cluster] = p; return; }
    double pl = or_pa_p_left(s, node, eye, y, ny);
    probs_rec(s, n->left, p * pl, eye, y, ny, P);
    probs_rec(s, n->right, p * (1.0 - pl), eye, y, ny, P);
}
void or_pa_probs(const or_scene *s, const double eye[4], const double *y, const double *ny, double *P) {
    if (s->pa_nclusters > 0) probs_rec(s, 0, 1.0, eye, y, ny, P);
}

/* Density across w of the environment photon's line through x: the sum over
 * clusters whose sphere the line meets of P_c / (pi r_c^2). */
double or_pa_env_density(const or_scene *s, const double eye[4], const double x[3], const double w[3]) {
    int32_t n = s->pa_nclusters;
    if (n <= 0) return 0.0;
    double *P = (double *)malloc(sizeof(double) * (size_t)n);
    or_pa_probs(s, eye, NULL, NULL, P);
    double sum = 0.0;
    for (int32_t c = 0; c < n; ++c) {
        const double *cc = s->pa_cc + 4 * c;
        double v[3] = {cc[0] - x[0], cc[1] - x[1], cc[2] - x[2]};
        double t = v[0] * w[0] + v[1] * w[1] + v[2] * w[2];
        double q2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2] - t * t;   /* squared distance of the centre to the line */
        if (q2 <= cc[3] * cc[3]) sum += P[c] / (OR_PI * cc[3] * cc[3]);
    }
    free(P);
    return sum;
}

/* Solid-angle density of a triangle photon from y (emitter normal ny)
 * leaving in direction w: the sum over clusters whose cone from y holds w
 * of P_c(y) / (2 pi (1 - cos theta_c)), or P_c(y) / (4 pi) when y is inside
 * the cluster's sphere. */
double or_pa_dir_density(const or_scene *s, const double eye[4], const double y[3], const double ny[3],
                         const double w[3]) {
    int32_t n = s->pa_nclusters;
    if (n <= 0) return 0.0;
    double *P = (double *)malloc(sizeof(double) * (size_t)n);
    or_pa_probs(s, eye, y, ny, P);
    double sum = 0.0;
    for (int32_t c = 0; c < n; ++c) {
        if (!(P[c] > 0.0)) continue;
        const double *cc = s->pa_cc + 4 * c;
        double v[3] = {cc[0] - y[0], cc[1] - y[1], cc[2] - y[2]};
        double d2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2], r2 = cc[3] * cc[3];
        if (d2 <= r2) { sum += P[c] / (4.0 * OR_PI); continue; }
        double d = sqrt(d2);
        double cmax = sqrt(1.0 - r2 / d2);
        double cw = (v[0] * w[0] + v[1] * w[1] + v[2] * w[2]) / d;
        /* 1 - cmax without cancellation: (r^2/d^2) / (1 + cmax) */
        if (cw >= cmax) sum += P[c] / (2.0 * OR_PI * (r2 / d2) / (1.0 + cmax));
    }
    free(P);
    return sum;
}

/* A direction uniform in the cone from y subtending cluster c's sphere
 * (uniform over all directions when y is inside it). */
void or_pa_cone_sample(const or_scene *s, int32_t c, const double y[3], double u1, double u2, double w[3]) {
    const double *cc = s->pa_cc + 4 * c;
    double v[3] = {cc[0] - y[0], cc[1] - y[1], cc[2] - y[2]};
    double d2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2], r2 = cc[3] * cc[3];
    double ct;
    double axis[3] = {0.0, 0.0, 1.0};
    if (d2 <= r2) {
        ct = 1.0 - 2.0 * u1;
    } else {
        double d = sqrt(d2);
        for (int a = 0; a < 3; ++a) axis[a] = v[a] / d;
        double one_minus = (r2 / d2) / (1.0 + sqrt(1.0 - r2 / d2));   /* 1 - cos theta_max */
        ct = 1.0 - u1 * one_minus;
    }
    double st = sqrt(fmax(0.0, 1.0 - ct * ct)), phi = 2.0 * OR_PI * u2;
    double t1[3], t2[3];
    or_onb(axis, t1, t2);
    for (int a = 0; a < 3; ++a) w[a] = st * cos(phi) * t1[a] + st * sin(phi) * t2[a] + ct * axis[a];
    double l = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
    for (int a = 0; a < 3; ++a) w[a] /= l;
}

/* Cluster spheres (n x 4), the cluster of every object and the number of
 * objects; returns the number of clusters (any output may be NULL). */
int32_t or_pa_info(const or_scene *s, double *spheres, int32_t *obj_cluster, int32_t *n_objects) {
    if (spheres) memcpy(spheres, s->pa_cc, sizeof(double) * 4 * (size_t)s->pa_nclusters);
    if (obj_cluster) memcpy(obj_cluster, s->pa_obj_cluster, sizeof(int32_t) * (size_t)s->pa_nobjects);
    if (n_objects) *n_objects = s->pa_nobjects;
    return s->pa_nclusters;
}
