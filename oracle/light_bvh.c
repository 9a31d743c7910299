/*
 * Oracle: probabilistic light hierarchy (paper Sec. 2.1.1): a bounding volume
 * hierarchy over the triangle emitters, traversed probabilistically from a
 * shading point; at each node the two children's estimated contributions
 * drive the choice, clamped so that no child with emitting geometry is left
 * out; in a leaf the emitter is chosen by flux; the same choices, made
 * deterministically along the emitter's unique path, give the probability
 * that MIS needs when a path hits an emitter. Directional emission is
 * represented per node by one value per region of the sphere.
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Readings fixed where the paper is silent:
 *   - binary tree; a node with at most OR_LB_LEAF emitters is a leaf; a larger
 *     one is split at its median emitter (count / 2 to the left) after
 *     ordering its emitters by centroid along the longest axis of their
 *     centroid bounds (ties of extent: the lower axis; ties of coordinate:
 *     the lower emitter index); centroid = (v0 + v1 + v2) / 3;
 *   - node: bounds of its emitters' vertices, flux = sum of emitter fluxes
 *     (luminance x area, the alias table's weights), and six directional
 *     values, one per face region of the cube (directions whose largest
 *     component in magnitude is +x, -x, +y, -y, +z, -z):
 *     I_k = sum_e flux_e kappa(angle(n_e, a_k) - theta_f), a_k the face axis,
 *     theta_f = acos(1 / sqrt 3) the angle from a face axis to its corners,
 *     kappa(g) = 1 for g <= 0, cos g below 90 degrees, 0 beyond: an upper
 *     bound of flux_e max(0, n_e . w) over the region (one-sided emitters);
 *   - estimate of a node with flux > 0 for a shading point x of normal n
 *     (the paper's flux over squared distance to the box centre times a
 *     conservative cosine): c = box centre, r = half its diagonal,
 *     v = x - c; inside the sphere (|v| <= r) e = max_k I_k / r^2; outside,
 *     with w = v / |v| and region k of w, e = I_k kappa(angle(n, -w) -
 *     asin(r / |v|)) / |v|^2;
 *   - child choice: a child without flux is never chosen; otherwise
 *     p_left = e_L / (e_L + e_R) (flux_L / (flux_L + flux_R) when both
 *     estimates vanish), clamped to [OR_LB_PMIN, 1 - OR_LB_PMIN];
 *   - one uniform number drives the descent: it picks a side against p and is
 *     rescaled to [0, 1) inside the chosen side, then picks the emitter of the
 *     leaf against the leaf's cumulative fluxes;
 *   - the estimates use the point and geometric normal of the vertex doing
 *     NEE (its offset ray origin, the origin of its continuation ray), so the
 *     probability is known again at the emitter the continuation hits.
 */
#include "oracle.h"
#include "oracle_internal.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define OR_PI 3.14159265358979323846

static double lb_kappa(double g) {
    if (g <= 0.0) return 1.0;
    if (g >= 0.5 * OR_PI) return 0.0;
    return cos(g);
}

static double lb_angle(const double a[3], const double b[3]) {
    double c = a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
    if (c > 1.0) c = 1.0;
    if (c < -1.0) c = -1.0;
    return acos(c);
}

int or_lb_region(const double w[3]) {
    int a = 0;
    if (fabs(w[1]) > fabs(w[a])) a = 1;
    if (fabs(w[2]) > fabs(w[a])) a = 2;
    return 2 * a + (w[a] < 0.0 ? 1 : 0);
}

/* emitter e's centroid coordinate along axis a */
static double lb_centroid(const or_scene *s, int64_t e, int a) {
    const double *v = s->v64 + 9 * (size_t)s->light_tri[e];
    return (v[a] + v[3 + a] + v[6 + a]) / 3.0;
}

static const or_scene *g_sort_scene;
static int g_sort_axis;

static int lb_cmp(const void *pa, const void *pb) {
    int64_t a = *(const int64_t *)pa, b = *(const int64_t *)pb;
    double ca = lb_centroid(g_sort_scene, a, g_sort_axis), cb = lb_centroid(g_sort_scene, b, g_sort_axis);
    if (ca < cb) return -1;
    if (ca > cb) return 1;
    return a < b ? -1 : (a > b ? 1 : 0);
}

static int32_t lb_build(or_scene *s, int64_t first, int64_t count, int32_t parent) {
    int32_t id = (int32_t)s->lb_n++;
    or_lb_node *nd = &s->lb_nodes[id];
    memset(nd, 0, sizeof *nd);
    nd->parent = parent;
    nd->first = first;
    nd->count = count;
    nd->left = nd->right = -1;
    for (int a = 0; a < 3; ++a) { nd->lo[a] = INFINITY; nd->hi[a] = -INFINITY; }
    double clo[3] = {INFINITY, INFINITY, INFINITY}, chi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = first; i < first + count; ++i) {
        int64_t e = s->lb_perm[i];
        int64_t t = s->light_tri[e];
        const double *v = s->v64 + 9 * (size_t)t;
        for (int k = 0; k < 3; ++k)
            for (int a = 0; a < 3; ++a) {
                if (v[3 * k + a] < nd->lo[a]) nd->lo[a] = v[3 * k + a];
                if (v[3 * k + a] > nd->hi[a]) nd->hi[a] = v[3 * k + a];
            }
        for (int a = 0; a < 3; ++a) {
            double c = lb_centroid(s, e, a);
            if (c < clo[a]) clo[a] = c;
            if (c > chi[a]) chi[a] = c;
        }
        double fl = s->light_flux[e];
        nd->flux += fl;
        const double *n = s->ng + 3 * (size_t)t;
        for (int k = 0; k < 6; ++k) {
            double ax[3] = {0.0, 0.0, 0.0};
            ax[k / 2] = (k & 1) ? -1.0 : 1.0;
            nd->I[k] += fl * lb_kappa(lb_angle(n, ax) - acos(1.0 / sqrt(3.0)));
        }
    }
    for (int a = 0; a < 3; ++a) nd->c[a] = 0.5 * (nd->lo[a] + nd->hi[a]);
    double dx = nd->hi[0] - nd->lo[0], dy = nd->hi[1] - nd->lo[1], dz = nd->hi[2] - nd->lo[2];
    nd->r = 0.5 * sqrt(dx * dx + dy * dy + dz * dz);
    if (count <= OR_LB_LEAF) {
        for (int64_t i = first; i < first + count; ++i) s->lb_leaf_of[s->lb_perm[i]] = id;
        return id;
    }
    int axis = 0;
    for (int a = 1; a < 3; ++a)
        if (chi[a] - clo[a] > chi[axis] - clo[axis]) axis = a;
    g_sort_scene = s;
    g_sort_axis = axis;
    qsort(s->lb_perm + first, (size_t)count, sizeof(int64_t), lb_cmp);
    int64_t half = count / 2;
    int32_t l = lb_build(s, first, half, id);
    int32_t r = lb_build(s, first + half, count - half, id);
    s->lb_nodes[id].left = l;
    s->lb_nodes[id].right = r;
    s->lb_nodes[id].count = 0;
    return id;
}

void or_build_light_bvh(or_scene *s) {
    s->lb_nodes = NULL;
    s->lb_n = 0;
    if (!s->d.light_bvh || s->nlights <= 0) return;
    int64_t n = s->nlights;
    s->lb_nodes = (or_lb_node *)calloc((size_t)(2 * n), sizeof(or_lb_node));
    s->lb_perm = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    s->lb_leaf_of = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    for (int64_t i = 0; i < n; ++i) s->lb_perm[i] = i;
    lb_build(s, 0, n, -1);
}

/* Estimated contribution of node `id` to point x of normal n. */
double or_lb_estimate(const or_scene *s, int32_t id, const double x[3], const double n[3]) {
    const or_lb_node *nd = &s->lb_nodes[id];
    if (!(nd->flux > 0.0)) return 0.0;
    double v[3] = {x[0] - nd->c[0], x[1] - nd->c[1], x[2] - nd->c[2]};
    double dist = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    if (dist <= nd->r) {
        double m = 0.0;
        for (int k = 0; k < 6; ++k) if (nd->I[k] > m) m = nd->I[k];
        return m / (nd->r * nd->r);   /* r > 0: every emitter has positive area */
    }
    double w[3] = {v[0] / dist, v[1] / dist, v[2] / dist};
    double to_node[3] = {-w[0], -w[1], -w[2]};
    double cs = lb_kappa(lb_angle(n, to_node) - asin(nd->r / dist));
    return nd->I[or_lb_region(w)] * cs / (dist * dist);
}

/* Probability of choosing the left child of internal node `id`. */
double or_lb_p_left(const or_scene *s, int32_t id, const double x[3], const double n[3]) {
    const or_lb_node *nd = &s->lb_nodes[id];
    const or_lb_node *L = &s->lb_nodes[nd->left], *R = &s->lb_nodes[nd->right];
    if (!(L->flux > 0.0)) return 0.0;
    if (!(R->flux > 0.0)) return 1.0;
    double eL = or_lb_estimate(s, nd->left, x, n), eR = or_lb_estimate(s, nd->right, x, n);
    double p = eL + eR > 0.0 ? eL / (eL + eR) : L->flux / (L->flux + R->flux);
    if (p < OR_LB_PMIN) p = OR_LB_PMIN;
    if (p > 1.0 - OR_LB_PMIN) p = 1.0 - OR_LB_PMIN;
    return p;
}

int64_t or_lb_sample(const or_scene *s, const double x[3], const double n[3], double u, double *prob) {
    int32_t id = 0;
    double P = 1.0;
    while (s->lb_nodes[id].count == 0) {
        double p = or_lb_p_left(s, id, x, n);
        if (u < p) {
            u = u / p;
            P *= p;
            id = s->lb_nodes[id].left;
        } else {
            u = (u - p) / (1.0 - p);
            if (u >= 1.0) u = nextafter(1.0, 0.0);
            P *= 1.0 - p;
            id = s->lb_nodes[id].right;
        }
    }
    const or_lb_node *nd = &s->lb_nodes[id];
    double target = u * nd->flux, cum = 0.0;
    int64_t pick = s->lb_perm[nd->first + nd->count - 1];
    for (int64_t i = nd->first; i < nd->first + nd->count; ++i) {
        cum += s->light_flux[s->lb_perm[i]];
        if (target < cum) { pick = s->lb_perm[i]; break; }
    }
    *prob = P * s->light_flux[pick] / nd->flux;
    return pick;
}

double or_lb_prob(const or_scene *s, const double x[3], const double n[3], int64_t e) {
    int32_t id = s->lb_leaf_of[e];
    double P = s->light_flux[e] / s->lb_nodes[id].flux;
    while (s->lb_nodes[id].parent >= 0) {
        int32_t par = s->lb_nodes[id].parent;
        double p = or_lb_p_left(s, par, x, n);
        P *= s->lb_nodes[par].left == id ? p : 1.0 - p;
        id = par;
    }
    return P;
}

int32_t or_lb_num_nodes(const or_scene *s) { return s->lb_n; }

void or_lb_node_info(const or_scene *s, int32_t id, double box[6], double I[6], double *flux, int32_t links[4]) {
    const or_lb_node *nd = &s->lb_nodes[id];
    for (int a = 0; a < 3; ++a) { box[a] = nd->lo[a]; box[3 + a] = nd->hi[a]; }
    for (int k = 0; k < 6; ++k) I[k] = nd->I[k];
    *flux = nd->flux;
    links[0] = nd->left; links[1] = nd->right; links[2] = nd->parent; links[3] = (int32_t)nd->count;
}

int64_t or_lb_light_of_tri(const or_scene *s, int64_t t) { return s->light_of_tri[t]; }
