/*
 * rt.h - C ABI of the GB300 consistent quasi-Monte Carlo path tracer.
 *
 * The library implements the data-parallel hot path of the light transport
 * simulation described in "The Iray Light Transport Simulation and Rendering
 * System" (Keller et al., arXiv:1705.01263): forward path tracing with next
 * event estimation combined by multiple importance sampling (Sec. 2),
 * importance sampling of triangle emitters and of the environment (Sec. 2.1),
 * a generic layered BSDF (Sec. 2.2), a wavefront state machine with
 * structure-of-arrays sample state, just-in-time queues, regeneration and a
 * megakernel tail (Sec. 3.1), per-pixel FP64 accumulation and sample counts
 * (Sec. 3.2.2, Appendix A.4), filter importance sampling (Appendix A.1),
 * integer-exact scrambled Halton sampling with 64-bit indices (Appendix A.2)
 * and local shading-normal adaptation (Appendix A.3).
 *
 * Conventions for every entry point:
 *   - All functions return rt_status; RT_OK (0) on success. On failure a
 *     message is available from rt_last_error() (thread-local, valid until the
 *     next call on the same thread). No C++ exception crosses this boundary.
 *   - "device" pointers are CUDA global-memory addresses on the current
 *     device; "host" pointers are ordinary CPU memory. The caller owns every
 *     buffer it passes in; the library never frees caller memory.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream). Calls that take a stream are asynchronous on it unless stated.
 *   - Handles (rt_scene, rt_film, rt_guide) own device memory allocated by the
 *     library and are released by their destroy function.
 *   - Kernels never trap: overflow of a fixed-size structure is reported as a
 *     status (RT_STACK_OVERFLOW, RT_QUEUE_OVERFLOW) and device-side waits are
 *     bounded (RT_TIMEOUT).
 */
#ifndef RT_GB300_H
#define RT_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    RT_OK = 0,
    RT_INVALID_ARG = 1,
    RT_OOM = 2,
    RT_CUDA_ERROR = 3,
    RT_TIMEOUT = 4,          /* time budget or abort flag: film is consistent and resumable */
    RT_QUEUE_OVERFLOW = 5,
    RT_STACK_OVERFLOW = 6,
    RT_NOT_SUPPORTED = 7
} rt_status;

typedef struct rt_scene rt_scene;
typedef struct rt_film rt_film;
typedef struct rt_guide rt_guide;

/* Scene description (all HOST pointers, copied by rt_scene_create).
 * Triangles are the only geometry and the only emitters (Sec. 2.1.1). A
 * triangle's geometric normal is normalize(cross(v1 - v0, v2 - v0)); emitters
 * radiate on that side only. Materials are the fixed layered model
 *   f = ggx_weight * f_GGX(roughness) + (1 - ggx_weight) * albedo / pi
 * (Sec. 2.2 names a generic layered BSDF without formulas). Emission of a
 * material is `emission` (RGB), multiplied by the nearest texel of texture
 * `emission_tex` at the interpolated UV when emission_tex >= 0.
 * The environment is an equirectangular RGB map, row 0 looking at +y, W = 2H
 * a power of two (Sec. 2.1.2); env == NULL means no environment.
 * Instancing (optional): when num_instances > 0, triangle range
 * [mesh_tri_offset[m], mesh_tri_offset[m+1]) is mesh m, and instance k places
 * mesh instance_mesh[k] with the row-major 3x4 object-to-world matrix
 * instance_xform[12k .. 12k+11]; hits then report (inst, prim) with prim
 * indexing the triangle list. */
typedef struct {
    int64_t num_vertices;
    int64_t num_triangles;
    const float *vertices;       /* num_vertices x 3 */
    const float *normals;        /* num_vertices x 3, or NULL (flat shading) */
    const float *uvs;            /* num_vertices x 2, or NULL */
    const uint32_t *indices;     /* num_triangles x 3 */
    const uint32_t *tri_material;/* num_triangles */
    int32_t num_materials;
    const float *albedo;         /* num_materials x 3 */
    const float *roughness;      /* num_materials */
    const float *ggx_weight;     /* num_materials */
    const float *emission;       /* num_materials x 3 */
    const int32_t *emission_tex; /* num_materials, -1 = constant emission */
    int32_t num_textures, tex_width, tex_height;
    const float *textures;       /* num_textures x tex_height x tex_width x 3 */
    int32_t env_width, env_height;
    const float *env;            /* env_height x env_width x 3, or NULL */
    int32_t num_meshes;
    const int64_t *mesh_tri_offset;  /* num_meshes + 1 */
    int32_t num_instances;
    const uint32_t *instance_mesh;   /* num_instances */
    const float *instance_xform;     /* num_instances x 12 */
    /* 1: NEE samples the environment from the plain pyramid only; 0: the
     * top pyramid levels are reweighted per geometric-normal cell (Sec.
     * 2.1.2: 64 octahedral cells, finest of the top five levels weighted by a
     * bound of the clamped cosine, coarser ones summed) */
    int32_t env_plain;
    /* 1: NEE picks triangle emitters through the probabilistic light
     * hierarchy (Sec. 2.1.1: a binary BVH over the emitters traversed with
     * branch probabilities from each child's estimated contribution to the
     * shading point, clamped to [0.1, 0.9]; by flux inside a leaf of at most
     * four); 0: the alias table over the emitter fluxes. RT_INVALID_ARG when
     * an instance transform makes one of its mesh's emitters degenerate. */
    int32_t light_bvh;
} rt_scene_desc;

/* Rays and hits for rt_trace: structure-of-arrays of DEVICE pointers, n
 * entries each. A ray is o + t d for t in the open interval (tmin, tmax); d
 * need not be normalised but must be non-zero. A miss is prim == RT_MISS
 * with t = +inf. (u, v) are the barycentric weights of v1 and v2. */
#define RT_MISS 0xFFFFFFFFu
typedef struct {
    const float *ox, *oy, *oz, *dx, *dy, *dz, *tmin, *tmax;
} rt_rays;
typedef struct {
    uint32_t *prim, *inst;
    float *t, *u, *v;
} rt_hits;

/* Pinhole camera; film pixel (x, y) has y growing downwards. */
typedef struct {
    float eye[3], look_at[3], up[3];
    float vfov_deg;
    uint32_t width, height;
} rt_camera;

/* Render statistics (optional output of rt_render). */
typedef struct {
    uint64_t paths;          /* camera paths completed */
    uint64_t extension_rays; /* closest-hit rays traced */
    uint64_t shadow_rays;    /* any-hit rays traced */
    uint32_t waves;          /* iteration sets executed */
    uint32_t wavefront_steps;/* bounce steps run as separate state kernels */
    uint32_t tail_launches;  /* megakernel tail launches */
    uint32_t kernel_launches;/* library kernels launched */
    /* per-kernel device time in ms, filled when rt_render_opts.profile != 0
     * (CUDA events around each launch on the render stream) */
    double trace_ms, shade_ms, shadow_ms, megakernel_ms, other_ms;
    uint32_t trace_launches;
    /* traversal work, filled when rt_render_opts.profile >= 2 (counted by
     * an instrumented variant of the trace kernels) */
    uint64_t ext_nodes, ext_tris, shadow_nodes, shadow_tris;
    uint32_t regen_sets;     /* regeneration scheduler: bounce steps that started new paths */
} rt_stats;

/* Render options. Zero-initialise and set what you need; zero means the
 * documented default for every field. */
typedef struct {
    float filter_sigma;      /* Gaussian filter sigma in pixels (A.1); 0 -> 0.5; <0 -> box */
    int32_t rr_enable;       /* Russian roulette from the 3rd vertex (default off) */
    int32_t mis_mode;        /* 0 power heuristic, 1 balance, 2 NEE only, 3 BSDF only */
    uint64_t seed;           /* scrambling seed for the Halton digits (A.2) */
    double time_budget_ms;   /* stop issuing new paths after this (0 = none); see rt_render */
    uint32_t max_paths_in_flight; /* state-pool capacity; 0 = every requested path at once, at most 2^27 and a
                                   * quarter of free device memory (regeneration refills it beyond); with an abort
                                   * flag or a time budget under scheduler 0, at most 2^24 paths */
    int32_t megakernel_only; /* 1: one megakernel per iteration set (A/B baseline) */
    int32_t sort_by_material;/* 1: material-sorted shading queue */
    uint32_t tail_threshold; /* live paths below which the megakernel finishes a set (0 = auto) */
    uint32_t block_size;     /* threads per block of the state kernels: 0 (= 128) or a multiple of
                              * 32 up to 128, else RT_INVALID_ARG; results do not depend on it */
    const volatile int32_t *abort_flag; /* host memory; nonzero -> stop (A.4); the library's host thread
                              * polls it while it waits for the device and relays it to the kernels */
    rt_guide *guide;         /* online path guiding (NULL = off) */
    rt_stats *stats;         /* optional host output */
    int32_t profile;         /* 1: per-kernel event timing; 2: also count traversal work */
    int32_t trace_kernel;    /* 0: closest hit one ray per thread (warps fetch 32 rays at a time), shadow
                              * rays with lane refill; 1: persistent warps refilling idle lanes, one node or
                              * triangle per step; 2: one ray per thread with the stack top in shared
                              * memory; 3: warps refill idle lanes between node visits (both ray kinds);
                              * 4: one ray per thread for both; 5: as 0 for camera rays, as 3 for later
                              * bounces (the regeneration scheduler runs 5 as 0); 6: as 0 with the
                              * closest-hit triangle tests postponed while few lanes want them; 7: both
                              * kinds one ray per thread with postponed triangle tests; 8: as 0 with one
                              * stack entry per child, the nearest child next and entries beyond the
                              * best hit dropped on pop. Two-level scenes always use 0's closest-hit
                              * kernel for both. */
    int32_t sort_rays;       /* 1: reorder extension rays by direction octant and origin cell (A/B) */
    int32_t scheduler;       /* 0: regeneration (Sec. 3.1.3): a bounded pool whose ended paths are
                              * refilled with the next tasks (a pool of at least 2^21 paths that refills
                              * runs as two half-pools on two streams unless the call can be stopped or
                              * sorts its queues; the film is the same); 1: iteration sets, each held
                              * whole in the pool (A/B). Guided rendering and megakernel_only use
                              * iteration sets. */
    float regen_fraction;    /* scheduler 0: refill once this fraction of the pool has ended (0 = 0.5,
                              * the paper's rule); must be in [0, 1] */
    int32_t lt_emission;     /* rt_render_two_way: 0 photon aiming (Sec. 2.1.3), 1 uniform emission over
                              * the scene's bound and cosine directions (A/B) */
    int32_t state_compression; /* rt_render, scheduler 0 (A/B, Sec. 3.1.1): ray and shadow directions as
                              * 16:16 octahedral codes, throughput and shadow contributions as BF16, the
                              * vertex number in 16 bits (132 instead of 168 bytes of state per path);
                              * RT_NOT_SUPPORTED with iteration sets, guiding or megakernel_only */
} rt_render_opts;

/* ---------------------------------------------------------------- scene */
/* Copies `desc` to device memory, builds the 8-wide compressed BVH (SAH),
 * per-triangle emitter flux + alias table (Sec. 2.1.1) and the environment
 * pyramid (Sec. 2.1.2). Synchronous. `*out` is owned by the caller. */
rt_status rt_scene_create(const rt_scene_desc *desc, rt_scene **out);
rt_status rt_scene_destroy(rt_scene *scene);
/* Node and triangle counts of the BVH and bytes of device memory held. */
rt_status rt_scene_info(const rt_scene *scene, int64_t *nodes, int64_t *leaf_tris,
                        int64_t *device_bytes);

/* ---------------------------------------------------------------- trace */
/* rays -> hits (Sec. 3.1, the ray-casting state kernels). Closest hit when
 * any_hit == 0 (ties in t: lower (inst, prim) wins); otherwise any hit in
 * (tmin, tmax) and prim != RT_MISS iff occluded. The kernel runs on
 * `stream`; its ray-fetch counter and overflow flag belong to that stream (8
 * bytes of device memory and a pinned word per device and stream, allocated
 * on the stream's first call and kept until exit), so calls in flight on
 * different streams or host threads do not interfere. The call
 * waits for its kernel before returning, so that it can report
 * RT_STACK_OVERFLOW: a ray whose traversal needed more than the fixed stack
 * (48 node groups; BVHs built by rt_scene_create stay far below it) has an
 * incomplete hit. n == 0 is a no-op. Errors: RT_INVALID_ARG (null scene,
 * rays or hit pointers, n < 0 or n >= 2^32, host-only scene),
 * RT_STACK_OVERFLOW, RT_CUDA_ERROR. */
rt_status rt_trace(const rt_scene *scene, const rt_rays *rays, int64_t n, const rt_hits *hits,
                   int32_t any_hit, void *stream);

/* ----------------------------------------------------------------- film */
/* Per-pixel FP64 sums of radiance and squared radiance (RGB) and a u32
 * sample count (Appendix A.4), on the device, plus the next iteration index.
 * rt_render accumulates into it; repeated calls add samples (consistency). */
rt_status rt_film_create(uint32_t width, uint32_t height, rt_film **out);
rt_status rt_film_destroy(rt_film *film);
rt_status rt_film_clear(rt_film *film, void *stream);
/* Next iteration (sample index j per pixel) the film will receive. */
rt_status rt_film_next_iteration(const rt_film *film, uint32_t *next);
/* Make the next rt_render start at iteration `next` (the film's sums are
 * kept). Devices that share one image render disjoint iteration sets and
 * their films are summed (Sec. 3.2.2 batch scheduling). */
rt_status rt_film_seek(rt_film *film, uint32_t next);
/* Device pointers to the raw buffers (sum: H*W*3 doubles, sum2 likewise,
 * count: H*W uint32). Valid until rt_film_destroy. */
rt_status rt_film_buffers(const rt_film *film, double **sum, double **sum2, uint32_t **count);
/* mean = sum / count; var = variance of the mean =
 * (sum2 / count - mean^2) / (count - 1). DEVICE float outputs, H*W*3 each;
 * var may be NULL. */
rt_status rt_film_resolve(const rt_film *film, float *mean, float *var, void *stream);

/* --------------------------------------------------------------- render */
/* Accumulate iterations [next, next + spp) of the consistent QMC estimator
 * into `film` (film size must equal the camera's); next =
 * rt_film_next_iteration(film). A film stopped inside an iteration (abort,
 * time budget) first completes that iteration, so rendering
 * total - next more iterations always ends exactly at `total`. max_depth = number of
 * scattering vertices (1 = direct lighting). Blocking with respect to the
 * host; kernels run on `stream`. Each pixel's sums receive its samples in
 * sample order, so results do not depend on the scheduler, the pool size or
 * how a range is split over calls (up to the megakernel tail's FP32 order).
 * Timeout (Appendix A.4): with the regeneration scheduler (the default) the
 * kernels check a host-mapped stop word and the device clock at every bounce
 * step; once the abort flag is seen or the time budget is spent no new path
 * starts, the paths in flight finish (at most max_depth + 1 more steps) and
 * the film receives every task that completed, a contiguous range that may
 * end inside an iteration. With iteration sets (scheduler 1) and guided
 * rendering the check happens between sets. Returns RT_TIMEOUT when stopped
 * early; the next call resumes at the film's next task. */
rt_status rt_render(const rt_scene *scene, const rt_camera *camera, uint32_t spp,
                    uint32_t max_depth, rt_film *film, const rt_render_opts *opts, void *stream);

/* Two-way path tracing (Sec. 2): the path tracer and a light-tracing stage
 * with the same number of paths per iteration (W x H), combined by multiple
 * importance sampling. The light tracer starts on the environment with
 * next-event estimation's probability (a direction from the plain pyramid)
 * or on a triangle emitter in proportion to its flux (a uniform point). With
 * photon aiming (Sec. 2.1.3, the default) it then picks a cluster of objects
 * (connected components of the mesh, or instances, joined when of similar
 * size and touching) through a hierarchy over the clusters, each step in
 * proportion to the solid angle under which the eye sees a child's bounding
 * sphere (at most the view cone's), and aims at it: an environment photon
 * starts on the cluster sphere's disk across its direction, a triangle
 * photon leaves in a direction uniform in the cone the sphere subtends; the
 * MIS densities sum over every cluster the emission passes. Without it
 * (opts->lt_emission = 1) photons start on the disk across the scene's
 * bounding sphere or leave cosine-distributed. The light tracer scatters by
 * the BSDF sampler and connects every
 * vertex to the pinhole camera, adding the connection to each pixel whose
 * Gaussian filter centre lies within 3 sigma of the image point (the box
 * filter: the pixel that holds it). Techniques for a path eye .. emitter or
 * environment with at least one scattering vertex: the camera path's
 * BSDF-sampled hit, next-event estimation, and the light tracer's camera
 * connection (sample counts 1 per pixel against W x H); paths that see an
 * emitter or the environment directly keep the path tracer's weights.
 *   spp, max_depth, film: as rt_render; iterations continue from the film's
 *             next iteration, which must start a pass (RT_INVALID_ARG
 *             otherwise); the film's sums, sums of squares and counts receive
 *             the camera stage (its squares cover that stage only)
 *   opts:     filter_sigma, mis_mode (0 power or 1 balance, else
 *             RT_INVALID_ARG), seed and rr_enable as rt_render; lt_emission
 *             (0 aimed, 1 uniform); the scheduling options are ignored; guide
 *             must be NULL (RT_NOT_SUPPORTED)
 *   lt_mode:  0 MIS of the three techniques; 1 the light tracer alone for
 *             every path it can make, the camera techniques elsewhere
 *   lt_splat: DEVICE double [H][W][3] that the light stage adds into
 *             (caller-owned; the estimate of a pixel is then
 *             (sum + lt_splat) / count), or NULL to add into the film's sums
 *   stats:    optional (paths, extension and shadow rays, kernel launches)
 * The call returns when the work is done (it synchronises `stream`).
 * Errors: RT_INVALID_ARG (null pointers, sizes, depth, modes),
 * RT_NOT_SUPPORTED (a guide), RT_CUDA_ERROR. Instanced scenes work as
 * rt_render's (emitters are (instance, triangle) pairs). With the
 * light hierarchy (Sec. 2.1.1) the camera stage's NEE draws through it and
 * every weight uses its probability; the light stage still emits by flux. */
rt_status rt_render_two_way(const rt_scene *scene, const rt_camera *camera, uint32_t spp, uint32_t max_depth,
                            rt_film *film, const rt_render_opts *opts, int32_t lt_mode, double *lt_splat,
                            rt_stats *stats, void *stream);

/* Irradiance probes (Sec. 4.2, alternate outputs): instead of camera rays,
 * n probe points with normals; each probe's film pixel accumulates estimates
 * of the irradiance E = integral over the hemisphere around its normal of
 * L cos(theta), sampled progressively like a pixel (probe p is the pixel
 * (p, 0) of an n x 1 image for the sample enumeration). A probe path starts
 * at a virtual white Lambertian point (vertex 1: NEE and a cosine-sampled
 * continuation, no emission) and continues as a camera path; max_depth counts
 * the probe as vertex 1, so 1 = direct irradiance.
 *   pos, nrm: DEVICE float arrays [n][3] (normals need not be unit length;
 *             caller-owned, read during the call)
 *   film:     created as rt_film_create(n, 1); iterations continue from its
 *             next iteration like rt_render; resolve gives E per probe
 *   opts:     as rt_render (guide must be NULL: RT_NOT_SUPPORTED)
 * Errors: RT_INVALID_ARG (null pointers, film not n x 1, max_depth out of
 * [1, 64]), RT_TIMEOUT (time budget / abort flag: resumable), as rt_render. */
rt_status rt_render_probes(const rt_scene *scene, const float *pos, const float *nrm, uint32_t n, uint32_t spp,
                           uint32_t max_depth, rt_film *film, const rt_render_opts *opts, void *stream);

/* Rendering that allocates nothing (the paper has no counterpart).
 * For callers that cannot call cudaMalloc or let a library do so - code
 * inside a host framework that owns all device memory through its own
 * arena, services whose device memory is fixed at start-up, threads on
 * which an allocation would synchronise the device. Same estimator and
 * kernels as rt_render, but the path-state pool (at most 65,536 paths in
 * flight), control block and sampling table live in one file-scope device
 * array of RT_STATIC_ARENA_BYTES (9.91 MiB) that every device loading the
 * library holds until the process exits. The caller passes the scene
 * (created earlier with rt_scene_create) and owns the outputs: DEVICE
 * buffers sum and sum2 (H*W*3 doubles) and count (H*W uint32), which are
 * accumulated into, so zero them before the first call. Renders iterations
 * [first_iteration, first_iteration + spp). opts may be NULL;
 * opts->max_paths_in_flight above 65,536 is rejected with RT_INVALID_ARG;
 * guiding and the sorted-queue options are RT_NOT_SUPPORTED.
 * Every call looks up the array's device address in the current context
 * (cudaGetSymbolAddress, which allocates nothing); the first call on a
 * device sets up that lookup, so make it before any stream capture. Every
 * call reuses the same array (the control block is cleared and the sampling
 * table rewritten at the start of each call): calls that overlap on the GPU
 * (other streams, other host threads) race and must not be issued. Blocking
 * with respect to the host, like rt_render. The time budget and abort flag
 * are checked where an iteration is complete only: on RT_TIMEOUT the sums
 * hold iterations [first_iteration, first_iteration + stats.paths / (W H)),
 * and the caller resumes from there. */
#define RT_STATIC_ARENA_BYTES 10388480u
rt_status rt_render_static(const rt_scene *scene, const rt_camera *camera, uint32_t spp, uint32_t max_depth,
                           uint32_t first_iteration, double *sum, double *sum2, uint32_t *count,
                           const rt_render_opts *opts, void *stream);

/* Batched rendering of many independent scenes (not in the paper): one job
 * per (scene, camera, spp, max_depth, film); all jobs share one wavefront
 * path pool (tasks of all jobs are concatenated) and one iteration set is
 * captured as a CUDA graph and replayed until every task is done. Each job
 * accumulates iterations [film next, + spp) into its own film (FP64 atomic
 * additions: equal to rt_render up to FP64 addition order). Blocking;
 * RT_TIMEOUT when the abort flag or time budget stopped it between sets
 * (films hold the completed tasks). A job may carry its own guiding network
 * (`guide`, or NULL; opts->guide must be NULL). A call with guided jobs
 * renders all its jobs in one shared wavefront of iteration sets (2^23 paths
 * unless opts->max_paths_in_flight is set; the jobs' tasks interleaved image
 * by image): before each guided bounce step the queue is sorted by job and
 * each guided job's network runs on its paths; after each set the due jobs
 * take a training step on their own samples (every set during a job's
 * warm-up, then one per 16 x `batch` of its paths rendered, subject to
 * `train_every`). Unguided jobs in such a call give the films they would
 * give alone, bit for bit. */
typedef struct {
    const rt_scene *scene;
    rt_camera camera;
    uint32_t spp;
    uint32_t max_depth;
    rt_film *film;
    rt_guide *guide;       /* this job's guiding network, or NULL */
} rt_render_job;
rt_status rt_render_batch(const rt_render_job *jobs, int32_t njobs, const rt_render_opts *opts, void *stream);

/* Autotuner (not in the paper): renders `sample_spp` of each job with every
 * candidate of path-pool capacity, tail threshold and traversal variant,
 * then with 64, 96 and 128 threads per block at the best of those, and
 * writes the fastest into *opts (max_paths_in_flight, tail_threshold,
 * trace_kernel, block_size). The films receive those samples; callers clear them. Jobs
 * with a guide are rejected (RT_NOT_SUPPORTED). */
rt_status rt_autotune(const rt_render_job *jobs, int32_t njobs, uint32_t sample_spp, rt_render_opts *opts,
                      void *stream);

/* ------------------------------------------------------- QMC sampling */
/* Sequence index of sample j in pixel (x, y) under full-screen enumeration
 * (Appendix A.2): DEVICE arrays px, py, j of n entries -> out (uint64). */
rt_status rt_sample_index(uint32_t width, uint32_t height, const uint32_t *px, const uint32_t *py,
                          const uint32_t *j, int64_t n, uint64_t *out, void *stream);
/* Scrambled Halton sample bits floor(2^32 * phi) of dimensions 0..ndims-1 for
 * DEVICE sequence indices (Appendix A.2); out is n x ndims uint32 (device).
 * Dimensions 0 and 1 are the in-pixel offsets of the (width x height)
 * enumeration; dimension d >= 2 uses the d-th prime with the seed's digit
 * scramble. */
rt_status rt_halton(uint32_t width, uint32_t height, uint64_t seed, const uint64_t *indices, int64_t n,
                    int32_t ndims, uint32_t *out, void *stream);
/* Host check of the strength-reduced division: q[i] = n[i] / d for HOST
 * arrays, computed with the same multiply-high routine the kernels use. */
rt_status rt_divide_u64_host(const uint64_t *n, int64_t count, uint32_t d, uint64_t *q);

/* ------------------------------------------------------------ guiding */
/* Online-trained proposal (not in the paper): one-blob encoded (position,
 * outgoing direction, normal) -> 4 x 64 ReLU MLP with BF16 weights and FP32
 * accumulation on the tensor cores -> 8-lobe von Mises-Fisher mixture,
 * combined with BSDF sampling by one-sample MIS (mixture probability
 * `alpha`). Trained with Adam on up to `batch` radiance samples after each
 * iteration set. For the first `warm_steps` steps (the warm-up) a set
 * renders at most min(`warm_set_batches`, 16) x `batch` paths, records
 * training samples from more of its paths and is followed by up to
 * `warm_set_batches` steps, each on its own `batch` of those samples; until
 * the first step the proposal is BSDF sampling alone. After the warm-up a
 * set renders up to 64 x `batch` paths (rt_render_opts.max_paths_in_flight
 * sets this size) and every `train_every`-th set is followed by one step per
 * 16 x `batch` paths it rendered (at least one, at most four). */
typedef struct {
    uint32_t batch;          /* training samples per pass (0 = 65536) */
    float learning_rate;     /* Adam lr (0 = 1e-2) */
    float alpha;             /* guide-vs-BSDF selection probability (0 = 0.5) */
    uint32_t train_steps;    /* Adam steps per pass (0 = 1) */
    uint64_t seed;           /* weight initialisation seed */
    uint32_t train_every;    /* after the warm-up steps, train after every train_every-th set (0 = 1) */
    uint32_t guide_depth;    /* guide the continuation of vertices 1..guide_depth only, BSDF
                              * sampling beyond (0 = 3; max_depth or more: every vertex);
                              * training records come from those vertices (at most 8) */
    uint32_t warm_steps;     /* training steps taken with small sets before the large ones (0 = 32) */
    uint32_t warm_set_batches; /* training batches (steps) per warm-up set (0 = 32; 1: one step
                                * after each set of `batch` paths) */
} rt_guide_opts;

rt_status rt_guide_create(const rt_scene *scene, const rt_guide_opts *opts, rt_guide **out);
rt_status rt_guide_destroy(rt_guide *guide);
/* Number of FP32 master weights (224*64 + 3*64*64 + 64*40 = 29184), layer by
 * layer, each layer [out][in] row-major. */
int64_t rt_guide_num_params(void);
/* HOST buffers of rt_guide_num_params() floats. set also resets Adam. */
rt_status rt_guide_get_params(const rt_guide *guide, float *params);
rt_status rt_guide_set_params(rt_guide *guide, const float *params);
/* Checkpoint: weights, Adam moments and step counter. */
rt_status rt_guide_state_size(const rt_guide *guide, int64_t *bytes);
rt_status rt_guide_save(const rt_guide *guide, void *host_buffer);
rt_status rt_guide_load(rt_guide *guide, const void *host_buffer);
/* Batched inference: DEVICE features (n x 7 floats in [0,1]: position in the
 * scene box, outgoing direction, normal) -> raw network outputs (n x 40
 * floats, device). Waits for `stream`; RT_TIMEOUT if a tensor-core
 * completion wait inside the kernel ran out (the outputs are then invalid). */
rt_status rt_guide_infer(const rt_guide *guide, const float *features, int64_t n, float *raw,
                         void *stream);
/* As rt_guide_infer, but only enqueued on `stream` (returns at once, no
 * wait): a completion-wait timeout is recorded in the guide and reported by
 * the next rt_guide_check or rt_guide_infer. The buffers must stay valid
 * until the stream reaches the launch. */
rt_status rt_guide_infer_async(const rt_guide *guide, const float *features, int64_t n, float *raw,
                               void *stream);
/* Waits for `stream`; RT_TIMEOUT (and the record cleared) if an earlier
 * asynchronous call on this guide timed out, else RT_OK. */
rt_status rt_guide_check(const rt_guide *guide, void *stream);
/* Loss and gradient on a DEVICE batch (features n x 7, wi n x 3, weight n);
 * grad (device, num_params floats) receives d loss / d weight, *loss (host)
 * the batch loss. Does not update the weights. Synchronous. */
rt_status rt_guide_loss_grad(const rt_guide *guide, const float *features, const float *wi,
                             const float *weight, int64_t n, float *grad, float *loss, void *stream);
/* One fused training step (forward, backward, Adam) on a DEVICE batch. */
rt_status rt_guide_train_step(rt_guide *guide, const float *features, const float *wi,
                              const float *weight, int64_t n, void *stream);

/* BF16 GEMM on the tcgen05 tensor cores with FP32 accumulation (the
 * guiding network's dense-layer primitive; not in the paper):
 * C[M x N] = A[M x K] * B[N x K]^T, or C += ... when accumulate != 0.
 * A, B: DEVICE bf16 row-major with row strides lda, ldb (elements; K, lda,
 * ldb multiples of 8, A and B 16-byte aligned); C: DEVICE float row-major
 * with stride ldc. Synchronous; RT_TIMEOUT if a tensor-core completion wait
 * ran out (the kernel returns without trapping). */
rt_status rt_gemm_bf16(const void *A, const void *B, float *C, int32_t M, int32_t N, int32_t K, int32_t lda,
                       int32_t ldb, int32_t ldc, int32_t accumulate, void *stream);

/* ------------------------------------------------------------ errors */
const char *rt_last_error(void);
const char *rt_status_string(rt_status s);

#ifdef __cplusplus
}
#endif
#endif /* RT_GB300_H */
