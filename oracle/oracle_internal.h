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
};

void or_build_bvh(or_scene *s);
void or_build_lights(or_scene *s);
void or_trace_one(const or_scene *s, const double o[3], const double d[3],
                  double tmin, double tmax, int any_hit, uint32_t *prim,
                  double *t, double *b1, double *b2);
void or_tri_emission(const or_scene *s, uint32_t prim, double b1, double b2,
                     double Le[3]);
#endif
