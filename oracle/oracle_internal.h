/* Oracle-internal scene state. TEST INFRASTRUCTURE ONLY (see oracle.h). */
#ifndef ORACLE_INTERNAL_H
#define ORACLE_INTERNAL_H
#include "oracle.h"

struct or_scene {
    or_scene_desc d;
    int64_t nt;
    double *v64;      /* nt x 9: the three vertices of each triangle */
    double *ng;       /* nt x 3: unit geometric normal */
    double *area;     /* nt */
    /* binary BVH */
    void *nodes;
    int64_t nnodes;
    int64_t *bvh_prims;
    /* emitters: triangles with nonzero emission, sampled by an alias table */
    int64_t nlights;
    int64_t *light_tri;      /* nlights */
    double *light_prob;      /* nlights: flux_i / sum flux */
    double *alias_prob;      /* nlights */
    int64_t *alias_idx;      /* nlights */
    double *tri_light_pdf_area; /* nt: P(select tri) / area, 0 if not an emitter */
    double flux_sum;
    double *light_flux;      /* nlights: luminance x area */
    int64_t *light_of_tri;   /* nt: emitter index of a triangle, -1 if none */
    /* probabilistic light hierarchy (light_bvh scenes): binary tree, node 0
     * the root; lb_perm orders the emitters so that every node covers a
     * contiguous range; lb_leaf_of = leaf of each emitter */
    struct or_lb_node *lb_nodes;
    int32_t lb_n;
    int64_t *lb_perm;
    int32_t *lb_leaf_of;
    /* environment pyramid */
    int32_t env_levels;      /* number of levels, finest first */
    double **env_w;          /* per level: weights (lum x solid angle), finest first */
    int32_t *env_lw, *env_lh;
    double env_wsum;
    double p_env;            /* probability of choosing the environment in NEE */
    /* normal-oriented top levels: levels env_lstar .. top, per normal cell,
     * weights w x kappa (kappa: bound of the clamped cosine between the
     * cell's normals and the region's directions); NULL when plain */
    int32_t env_lstar;
    double *env_nw;          /* 64 cells x env_nstride */
    int64_t env_noff[32];    /* offset of level l inside a cell's block */
    int64_t env_nstride;
    /* photon aiming (photon_aiming.c): clusters of objects (centre and
     * radius of each cluster's sphere), the cluster of every object, and a
     * binary hierarchy over the clusters, node 0 the root */
    int32_t pa_nclusters, pa_nobjects, pa_nnodes;
    double *pa_cc;           /* pa_nclusters x 4: centre, radius */
    int32_t *pa_obj_cluster; /* pa_nobjects */
    struct or_pa_node *pa_nodes;
};

typedef struct or_pa_node {
    double c[3], r;          /* sphere enclosing every cluster sphere below */
    int32_t left, right;     /* children, -1 in a leaf */
    int32_t cluster;         /* leaf: its cluster; -1 otherwise */
} or_pa_node;

/* photon aiming (photon_aiming.c, Sec. 2.1.3); eye = (position, solid
 * angle of the camera's view cone); y, ny = NULL for an environment photon */
void or_build_photon_aiming(or_scene *s);
double or_pa_p_left(const or_scene *s, int32_t node, const double eye[4], const double *y, const double *ny);
int32_t or_pa_sample(const or_scene *s, const double eye[4], const double *y, const double *ny, double u,
                     double *prob);
void or_pa_probs(const or_scene *s, const double eye[4], const double *y, const double *ny, double *P);
double or_pa_env_density(const or_scene *s, const double eye[4], const double x[3], const double w[3]);
double or_pa_dir_density(const or_scene *s, const double eye[4], const double y[3], const double ny[3],
                         const double w[3]);
void or_pa_cone_sample(const or_scene *s, int32_t c, const double y[3], double u1, double u2, double w[3]);
int32_t or_pa_info(const or_scene *s, double *spheres, int32_t *obj_cluster, int32_t *n_objects);
void or_pa_eye(const or_scene *s, const or_camera *c, double out[4]);

#define OR_LB_LEAF 4       /* emitters per leaf of the light hierarchy, at most */
#define OR_LB_PMIN 0.1     /* clamp of a child's probability */

typedef struct or_lb_node {
    double lo[3], hi[3];   /* bounds of the emitters' vertices */
    double c[3], r;        /* box centre and half diagonal */
    double flux;           /* sum of emitter fluxes */
    double I[6];           /* directional values per cube-face region */
    int32_t left, right;   /* children (internal nodes), -1 in a leaf */
    int32_t parent;        /* -1 at the root */
    int64_t first, count;  /* leaf: range of lb_perm; internal: count 0 */
} or_lb_node;

void or_build_light_bvh(or_scene *s);
void or_build_bvh(or_scene *s);
void or_build_lights(or_scene *s);
void or_trace_one(const or_scene *s, const double o[3], const double d[3],
                  double tmin, double tmax, int any_hit, uint32_t *prim,
                  double *t, double *b1, double *b2);
void or_tri_emission(const or_scene *s, uint32_t prim, double b1, double b2,
                     double Le[3]);
/* ray origin moved off the surface along n (render.c) */
void or_offset_origin(const double x[3], const double n[3], double out[3]);

/* two-way path tracing (two_way.c) */
typedef struct {
    double x[3];
    double ng[3];      /* unit geometric normal as stored (not turned) */
    double ns[3];      /* unit interpolated shading normal (ng without normals) */
    uint32_t prim;
} or_tw_vertex;

typedef struct {
    double eye[3], fwd[3], right[3], up[3];
    double th, asp, f;  /* tan(vfov / 2), W / H, focal length in pixels */
    uint32_t W, H;
    double sigma;       /* pixel filter (> 0 Gaussian, else box) */
    double bc[3], br;   /* the scene's bounding sphere (environment photons) */
    int aim;            /* photon aiming (Sec. 2.1.3) instead of uniform emission */
    double aim_eye[4];  /* eye position and the solid angle of the view cone (photon aiming's estimates) */
} or_tw_cam;

/* camera frame and the scene's bounding sphere (centre and half diagonal of
 * the box of its vertices); an environment direction is stored as a vertex
 * with prim OR_MISS and x the unit direction towards the environment */
void or_tw_cam_init(const or_scene *s, const or_camera *c, double sigma, or_tw_cam *tc);
void or_tw_vertex_at(const or_scene *s, uint32_t prim, double b1, double b2, or_tw_vertex *v);
/* area-measure densities of the three techniques for the path x[0] (eye) ..
 * x[k] (emitter) through pixel (px, py); p_lt is zero where the light tracer
 * does not connect to that pixel */
void or_tw_pdfs(const or_scene *s, const or_tw_cam *tc, const or_tw_vertex *x, int k, uint32_t px, uint32_t py,
                double *p_hit, double *p_nee, double *p_lt);
/* heuristic weight of `mine` against two other (count-scaled) densities */
double or_tw_weight(int mode, double mine, double other1, double other2);
#endif
