/*
 * Plain FP64 CPU oracle for consistent QMC path tracing with next-event
 * estimation (paper Sec. 2, Sec. 2.1, Sec. 2.2, Appendix A.1-A.3) and for the
 * path-guiding network that sits beside it.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product library may link, call or
 * include anything in this directory; only the tests, the smoke check and the
 * CPU-baseline leg of the benchmark use it. It shares no code with the CUDA
 * path: every routine here is written from the paper (or, where the paper is
 * silent, from the textbook definition named beside it), slowly and plainly,
 * in double precision.
 *
 * Conventions fixed by this oracle (both sides implement them independently):
 *   - directions are unit vectors in a right-handed world frame, +y is "up"
 *     for the equirectangular environment;
 *   - a triangle's geometric normal is normalize(cross(v1-v0, v2-v0)); an
 *     emitter emits only on that side;
 *   - barycentrics (b1, b2) are the weights of v1 and v2;
 *   - a miss is prim == 0xFFFFFFFF with t = +inf.
 */
#ifndef ORACLE_H
#define ORACLE_H

#include <stdint.h>
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define OR_MISS 0xFFFFFFFFu

/* ---------------------------------------------------------------- halton.c */
uint32_t or_prime(int dim);                       /* dim-th prime, dim 0 -> 2 */
uint64_t or_splitmix64(uint64_t *state);          /* Steele, Lea, Flood 2014 */
uint32_t or_scramble_factor(uint64_t seed, uint32_t b);
uint32_t or_radical_inverse_u32(uint32_t b, uint32_t f, uint64_t i);
double   or_u32_to_unit(uint32_t u);              /* (u >> 8) * 2^-24 */
void     or_enum_params(uint32_t W, uint32_t H, uint32_t *k, uint32_t *l,
                        uint64_t *p2, uint64_t *p3);
uint64_t or_pixel_base_index(uint32_t W, uint32_t H, uint32_t x, uint32_t y);
double   or_sample_dim(uint64_t index, int dim, uint32_t k, uint32_t l,
                       const uint32_t *factors);
void     or_sample_dims_batch(const uint64_t *idx, int64_t n, int ndims,
                              uint32_t W, uint32_t H, uint64_t seed,
                              uint32_t *out_u32 /* n x ndims */);

/* -------------------------------------------------------------- geometry.c */
typedef struct or_scene or_scene;

typedef struct {
    /* geometry (world space; instances are flattened by the caller) */
    int64_t nv, nt;
    const float *vertices;   /* nv x 3 */
    const float *normals;    /* nv x 3 or NULL */
    const float *uvs;        /* nv x 2 or NULL */
    const uint32_t *indices; /* nt x 3 */
    const uint32_t *tri_material; /* nt */
    /* materials */
    int32_t nm;
    const float *albedo;     /* nm x 3 */
    const float *roughness;  /* nm */
    const float *ggx_weight; /* nm */
    const float *emission;   /* nm x 3 (scale when a texture is attached) */
    const int32_t *emission_tex; /* nm, -1 = constant */
    /* emission textures: ntex x th x tw x 3 */
    int32_t ntex, tex_w, tex_h;
    const float *textures;
    /* environment: env_h x env_w x 3 equirect, or NULL */
    int32_t env_w, env_h;
    const float *env;
    /* 1: NEE samples the environment from the plain pyramid only (no
     * normal-oriented top levels) */
    int32_t env_plain;
    /* 1: NEE picks triangle emitters through the probabilistic light
     * hierarchy (Sec. 2.1.1) instead of the alias table */
    int32_t light_bvh;
} or_scene_desc;

or_scene *or_scene_create(const or_scene_desc *d);
void      or_scene_destroy(or_scene *s);
int       or_intersect_tri(const double o[3], const double d[3], double tmin,
                           double tmax, const double v0[3], const double v1[3],
                           const double v2[3], double *t, double *b1, double *b2);
void      or_trace(const or_scene *s, const float *rays /* n x 8 */, int64_t n,
                   int any_hit, int use_bvh, uint32_t *prim, double *t,
                   double *b1, double *b2);
int64_t   or_bvh_node_count(const or_scene *s);

/* --------------------------------------------------------------- shading.c */
void   or_onb(const double n[3], double t[3], double b[3]);
void   or_adapt_shading_normal(const double ns[3], const double ng[3],
                               const double wo[3], double out[3]);
double or_ggx_D(double alpha, double cos_h);
double or_ggx_lambda(double alpha, double cos_t);
double or_ggx_G1(double alpha, double cos_t);
double or_schlick(double cos_ih);
void   or_bsdf_eval(const double albedo[3], double rough, double w,
                    const double ns[3], const double wo[3], const double wi[3],
                    double f[3], double *pdf);
int    or_bsdf_sample(const double albedo[3], double rough, double w,
                      const double ns[3], const double wo[3], double u_lobe,
                      double u1, double u2, double wi[3], double f[3],
                      double *pdf);
void   or_ggx_vndf_sample(double alpha, const double wo_local[3], double u1,
                          double u2, double h_local[3]);
double or_luminance(const double c[3]);

/* lights */
void   or_alias_build(const double *w, int64_t n, double *prob, int64_t *alias);
int64_t or_alias_sample(const double *prob, const int64_t *alias, int64_t n,
                        double u);
void   or_env_pyramid_probs(const float *env, int32_t W, int32_t H,
                            double *texel_prob /* H x W */);
void   or_env_sample(const or_scene *s, double u, double v, double wi[3],
                     double *pdf, int32_t *tx, int32_t *ty);
double or_env_pdf(const or_scene *s, const double wi[3]);
/* Normal-oriented top levels of the environment pyramid (Sec. 2.1.2): the
 * geometric normal's cell (64 cells of an 8 x 8 octahedral map); sampling and
 * pdf for a shading point of that normal (equal to or_env_sample /
 * or_env_pdf when the scene has env_plain set). */
/* Probabilistic light hierarchy (Sec. 2.1.1; light_bvh scenes): the emitter
 * drawn with u for a shading point x of geometric normal n and its
 * probability; the probability of emitter e by the deterministic traversal
 * of its path; one node's estimate and left-child probability; node data
 * (box lo/hi, six directional values, flux, links {left, right, parent,
 * emitter count (0: internal)}); the cube-face region of a direction; the
 * emitter index of a triangle (-1 if none). */
int64_t or_lb_sample(const or_scene *s, const double x[3], const double n[3], double u, double *prob);
double  or_lb_prob(const or_scene *s, const double x[3], const double n[3], int64_t e);
double  or_lb_estimate(const or_scene *s, int32_t id, const double x[3], const double n[3]);
double  or_lb_p_left(const or_scene *s, int32_t id, const double x[3], const double n[3]);
int32_t or_lb_num_nodes(const or_scene *s);
void    or_lb_node_info(const or_scene *s, int32_t id, double box[6], double I[6], double *flux, int32_t links[4]);
int     or_lb_region(const double w[3]);
int64_t or_lb_light_of_tri(const or_scene *s, int64_t t);

int    or_env_normal_cell(const double n[3]);
void   or_env_sample_n(const or_scene *s, const double ng[3], double u, double v, double wi[3], double *pdf);
double or_env_pdf_n(const or_scene *s, const double ng[3], const double wi[3]);
/* probability of every finest texel (W x H) for normal cell `cell` */
void   or_env_texel_probs_n(const or_scene *s, int cell, double *texel_prob);
void   or_env_lookup(const or_scene *s, const double wi[3], double L[3]);
double or_scene_light_pdf_area(const or_scene *s, uint32_t prim);
double or_scene_env_select_prob(const or_scene *s);

/* ---------------------------------------------------------------- render.c */
typedef struct {
    double eye[3], look_at[3], up[3];
    double vfov_deg;
    uint32_t width, height;
} or_camera;

typedef struct {
    double filter_sigma;   /* Gaussian filter std-dev in pixels; 0 = box */
    int32_t rr_enable;     /* Russian roulette (off by default) */
    int32_t mis_mode;      /* 0 power heuristic, 1 balance, 2 NEE only, 3 BSDF only */
    uint64_t seed;         /* scramble seed */
    int32_t threads;       /* worker threads, 0 = all cores */
    int32_t lt_aim;        /* two-way: 1 photon aiming (Sec. 2.1.3), 0 uniform over the scene's bound */
} or_render_opts;

void or_camera_ray(const or_camera *c, double sx, double sy, double o[3],
                   double d[3]);
void or_filter_offset(double sigma, double u0, double u1, double *dx,
                      double *dy);
void or_render(const or_scene *s, const or_camera *cam, uint32_t iter0,
               uint32_t spp, uint32_t max_depth, const or_render_opts *opts,
               double *sum /* H*W*3 */, double *sum2 /* H*W*3 */,
               uint32_t *count /* H*W */, uint64_t *rays_traced);
void or_render_pixels(const or_scene *s, const or_camera *cam,
                      const uint32_t *px, const uint32_t *py,
                      const uint32_t *sample_j, int64_t n, uint32_t max_depth,
                      const or_render_opts *opts, double *L /* n x 3 */);
/* Two-way path tracing (render.c, two_way.c; Sec. 2): the camera stage into
 * sum / sum2 / count as or_render, with the light tracer as a third MIS
 * technique, and the light-tracing stage (W x H light paths per iteration)
 * splatted into `splat` (H*W*3, accumulated; per pixel the estimate is
 * (sum + splat) / count). lt_mode 0: MIS of the three techniques; 1: the
 * light tracer alone wherever it can make the path, the camera techniques
 * elsewhere; 2: the camera stage alone with the light tracer's density set
 * to zero (equals or_render; no light stage); 3: the density check of
 * two_way.c (counts, not radiance). mis_mode 0 or 1 only. */
void or_render_two_way(const or_scene *s, const or_camera *cam, uint32_t iter0, uint32_t spp,
                       uint32_t max_depth, const or_render_opts *opts, int32_t lt_mode, double *sum,
                       double *sum2, uint32_t *count, double *splat, uint64_t *rays_traced);
void or_light_trace(const or_scene *s, const or_camera *cam, uint32_t iter0, uint32_t spp, uint32_t D,
                    const or_render_opts *opts, int lt_mode, double *splat, uint64_t *rays_traced);
/* Irradiance probes (see render.c): sums of E = pi L per probe. */
void or_render_probes(const or_scene *s, const double *pos, const double *nrm, uint32_t n,
                      uint32_t iter0, uint32_t spp, uint32_t max_depth,
                      const or_render_opts *opts, double *sum, double *sum2,
                      uint32_t *count, uint64_t *rays_traced);

/* ----------------------------------------------------------------- guide.c */
#define OR_GUIDE_BINS 32
#define OR_GUIDE_IN 224
#define OR_GUIDE_HID 64
#define OR_GUIDE_LOBES 8
#define OR_GUIDE_OUT 40
double or_vmf_pdf(double kappa, const double mu[3], const double w[3]);
void   or_vmf_sample(double kappa, const double mu[3], double u1, double u2,
                     double w[3]);
void   or_oneblob(const double s[7], double *enc /* 224 */);
void   or_guide_features(const double pos01[3], const double wo[3],
                         const double n[3], double s[7]);
void   or_mlp_forward(const double *params, const double *x, int64_t batch,
                      double *out /* batch x 40 */, double *acts /* may be NULL */);
void   or_mixture_from_raw(const double *raw /* 40 */, double mu[8][3],
                           double kappa[8], double weight[8]);
double or_mixture_pdf(const double *raw, const double w[3]);
void   or_mixture_sample(const double *raw, double u_sel, double u1, double u2,
                         double w[3]);
double or_guide_loss_grad(const double *params, const double *x /* B x 224 */,
                          const double *wi /* B x 3 */, const double *weight,
                          int64_t batch, double *grad /* nparams */);
int64_t or_guide_nparams(void);
void   or_adam_step(double *params, const double *grad, double *m, double *v,
                    int64_t n, int64_t t, double lr, double b1, double b2,
                    double eps);

#ifdef __cplusplus
}
#endif
#endif
