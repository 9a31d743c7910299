// C-ABI glue: error reporting, QMC table set-up (Appendix A.2 strength
// reduction: the magic multipliers are computed once on the host), and the
// host-execution test hooks that run the kernels' __host__ __device__ code on
// the CPU for the CPU-only test suite. The hooks are never called by
// rt_trace or rt_render.
#include <cmath>
#include <cstdio>
#include <string>
#include <vector>

#include "internal.h"
#include "shade.cuh"
#include "aiming.cuh"

namespace rtg {

static thread_local std::string g_err;

void set_error(const std::string &msg) { g_err = msg; }

rt_status cuda_status(cudaError_t e, const char *what) {
    g_err = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? RT_OOM : RT_CUDA_ERROR;
}

uint32_t nth_prime(int dim) {
    static std::vector<uint32_t> primes;
    if (primes.empty()) {
        for (uint32_t c = 2; primes.size() < 4096; ++c) {
            bool p = true;
            for (uint32_t q = 2; q * q <= c; ++q)
                if (c % q == 0) { p = false; break; }
            if (p) primes.push_back(c);
        }
    }
    return primes[dim];
}

static uint64_t splitmix64(uint64_t &state) {
    uint64_t z = (state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Linear digit scramble pi(d) = f d mod b with f drawn from SplitMix64
// (state = seed + b, rejection of f = 1); base 2 is left unscrambled.
static uint32_t scramble_multiplier(uint64_t seed, uint32_t b) {
    if (b <= 2) return 1;
    uint64_t st = seed + b;
    for (;;) {
        uint32_t f = 1u + (uint32_t)(splitmix64(st) % (uint64_t)(b - 1));
        if (f != 1u) return f;
    }
}

HaltonDim make_dim(uint32_t base, uint32_t f) {
    HaltonDim h{};
    h.div = make_divisor(base);
    h.f = f;
    uint32_t bits = 0;
    while ((1u << bits) < base) ++bits;
    h.bits = bits;
    // w[0] = floor(2^64 / b) (b > 2 is odd, so 2^64 is not a multiple of it),
    // w[k + 1] = floor(w[k] / b)
    if (base > 2) {
        h.w[0] = ~0ull / base;
        for (int k = 1; k < kMaxDigits; ++k) h.w[k] = h.w[k - 1] / base;
    }
    return h;
}

std::vector<HaltonDim> make_dims(uint64_t seed, int ndims) {
    std::vector<HaltonDim> d((size_t)ndims);
    for (int i = 0; i < ndims; ++i) {
        uint32_t b = nth_prime(i);
        d[i] = make_dim(b, i < 2 ? 1u : scramble_multiplier(seed, b));
    }
    return d;
}

static uint64_t inv_mod(uint64_t a, uint64_t m) {
    // extended Euclid, m > 1, gcd(a, m) = 1
    int64_t t = 0, nt = 1;
    int64_t r = (int64_t)m, nr = (int64_t)(a % m);
    while (nr) {
        int64_t q = r / nr;
        int64_t tmp = t - q * nt; t = nt; nt = tmp;
        tmp = r - q * nr; r = nr; nr = tmp;
    }
    if (t < 0) t += (int64_t)m;
    return (uint64_t)t;
}

Enum make_enum(uint32_t W, uint32_t H) {
    Enum e{};
    e.k = 0; e.p2 = 1;
    while (e.p2 < W) { e.p2 *= 2; ++e.k; }
    e.l = 0; e.p3 = 1;
    while (e.p3 < H) { e.p3 *= 3; ++e.l; }
    e.period = e.p2 * e.p3;
    if (e.p2 == 1 && e.p3 == 1) { e.e2 = 0; e.e3 = 0; }
    else if (e.p2 == 1) { e.e2 = 0; e.e3 = 1; }
    else if (e.p3 == 1) { e.e2 = 1; e.e3 = 0; }
    else {
        e.e2 = (e.p3 * inv_mod(e.p3 % e.p2, e.p2)) % e.period;
        e.e3 = (e.p2 * inv_mod(e.p2 % e.p3, e.p3)) % e.period;
    }
    if (e.l) e.div_p3 = make_divisor((uint32_t)e.p3);
    e.base3 = make_dim(3, 1);
    return e;
}

// Camera basis in double precision, rounded once to float.
CameraView make_camera(const rt_camera &c) {
    double eye[3] = {c.eye[0], c.eye[1], c.eye[2]};
    double f[3] = {c.look_at[0] - eye[0], c.look_at[1] - eye[1], c.look_at[2] - eye[2]};
    double fl = std::sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
    for (double &x : f) x /= fl;
    double up[3] = {c.up[0], c.up[1], c.up[2]};
    double r[3] = {f[1] * up[2] - f[2] * up[1], f[2] * up[0] - f[0] * up[2], f[0] * up[1] - f[1] * up[0]};
    double rl = std::sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    for (double &x : r) x /= rl;
    double u[3] = {r[1] * f[2] - r[2] * f[1], r[2] * f[0] - r[0] * f[2], r[0] * f[1] - r[1] * f[0]};
    CameraView v;
    v.eye = v3((float)eye[0], (float)eye[1], (float)eye[2]);
    v.fwd = v3((float)f[0], (float)f[1], (float)f[2]);
    v.right = v3((float)r[0], (float)r[1], (float)r[2]);
    v.up = v3((float)u[0], (float)u[1], (float)u[2]);
    v.tan_half = (float)std::tan(0.5 * c.vfov_deg * M_PI / 180.0);
    v.aspect = (float)c.width / (float)c.height;
    v.W = c.width;
    v.H = c.height;
    return v;
}

}  // namespace rtg

using namespace rtg;

extern "C" const char *rt_last_error(void) { return g_err.c_str(); }

extern "C" const char *rt_status_string(rt_status s) {
    switch (s) {
        case RT_OK: return "RT_OK";
        case RT_INVALID_ARG: return "RT_INVALID_ARG";
        case RT_OOM: return "RT_OOM";
        case RT_CUDA_ERROR: return "RT_CUDA_ERROR";
        case RT_TIMEOUT: return "RT_TIMEOUT";
        case RT_QUEUE_OVERFLOW: return "RT_QUEUE_OVERFLOW";
        case RT_STACK_OVERFLOW: return "RT_STACK_OVERFLOW";
        case RT_NOT_SUPPORTED: return "RT_NOT_SUPPORTED";
    }
    return "unknown";
}

extern "C" rt_status rt_divide_u64_host(const uint64_t *n, int64_t count, uint32_t d, uint64_t *q) {
    if (d < 2 || count < 0 || (count > 0 && (!n || !q))) { set_error("rt_divide_u64_host: invalid argument"); return RT_INVALID_ARG; }
    Divisor v = make_divisor(d);
    for (int64_t i = 0; i < count; ++i) q[i] = div64(n[i], v);
    return RT_OK;
}

// ----------------------------------------------------------- test hooks
/* Host execution of the kernels' traversal routine on a host-only scene
 * (rt_debug_scene_create_host). rays: n x 8 floats (o, d, tmin, tmax). */
extern "C" rt_status rt_debug_trace_host(const rt_scene *s, const float *rays, int64_t n, int32_t any_hit,
                                         uint32_t *prim, float *t, float *u, float *v, uint32_t *nodes_visited,
                                         uint32_t *inst) {
    if (!s || !s->host_only || n < 0) { set_error("rt_debug_trace_host: needs a host-only scene"); return RT_INVALID_ARG; }
    for (int64_t i = 0; i < n; ++i) {
        const float *r = rays + 8 * i;
        Ray ray{v3(r[0], r[1], r[2]), v3(r[3], r[4], r[5]), r[6], r[7]};
        Hit h;
        h.prim = RT_MISS; h.inst = 0; h.t = INFINITY; h.b1 = h.b2 = 0.f;
        TraceResult tr = any_hit ? trace_scene<true>(s->host, ray, h) : trace_scene<false>(s->host, ray, h);
        if (tr.overflow) { set_error("stack overflow"); return RT_STACK_OVERFLOW; }
        prim[i] = h.prim;
        t[i] = h.prim == RT_MISS ? INFINITY : h.t;
        if (u) u[i] = h.b1;
        if (v) v[i] = h.b2;
        if (nodes_visited) nodes_visited[i] = tr.nodes;
        if (inst) inst[i] = h.inst;
    }
    return RT_OK;
}

/* Host execution of the single-level traversal with a stack of only
 * `stack_entries` (1..48) node groups: the overflow path of the kernels'
 * traversal (a ray that needs more entries ends and the call returns
 * RT_STACK_OVERFLOW) made reachable on small scenes. Otherwise as
 * rt_debug_trace_host. */
extern "C" rt_status rt_debug_trace_host_stack(const rt_scene *s, const float *rays, int64_t n, int32_t any_hit,
                                               int32_t stack_entries, uint32_t *prim, float *t) {
    if (!s || !s->host_only || n < 0 || !prim || !t || (n > 0 && !rays)) {
        set_error("rt_debug_trace_host_stack: needs a host-only scene and outputs");
        return RT_INVALID_ARG;
    }
    if (s->host.two_level) { set_error("rt_debug_trace_host_stack: single-level scenes only"); return RT_INVALID_ARG; }
    if (stack_entries < 1 || stack_entries > kStackSize) {
        set_error("rt_debug_trace_host_stack: stack_entries must be in [1, 48]");
        return RT_INVALID_ARG;
    }
    for (int64_t i = 0; i < n; ++i) {
        const float *r = rays + 8 * i;
        Ray ray{v3(r[0], r[1], r[2]), v3(r[3], r[4], r[5]), r[6], r[7]};
        Hit h;
        h.prim = RT_MISS; h.inst = 0; h.t = INFINITY; h.b1 = h.b2 = 0.f;
        BoundedStack stack;
        stack.cap = stack_entries;
        TraceResult tr = any_hit ? traverse<true, BoundedStack>(s->host.nodes, s->host.tris, 0u, ray, h, 0u, &stack)
                                 : traverse<false, BoundedStack>(s->host.nodes, s->host.tris, 0u, ray, h, 0u, &stack);
        if (tr.overflow) {
            set_error("BVH traversal stack overflow (ray " + std::to_string(i) + ")");
            return RT_STACK_OVERFLOW;
        }
        prim[i] = h.prim;
        t[i] = h.prim == RT_MISS ? INFINITY : h.t;
    }
    return RT_OK;
}

/* Photon aiming's cluster hierarchy of a host-only scene: node spheres
 * (n x 4: centre, radius) and links (n x 2: left, right; a leaf -1,
 * cluster). Pass null outputs to query the counts. */
extern "C" rt_status rt_debug_aim_tree_host(const rt_scene *s, float *spheres, int32_t *links, int32_t *nnodes,
                                            int32_t *nclusters) {
    if (!s || !s->host_only) { set_error("rt_debug_aim_tree_host: needs a host-only scene"); return RT_INVALID_ARG; }
    const DevScene &sc = s->host;
    if (nnodes) *nnodes = sc.pa_nnodes;
    if (nclusters) *nclusters = sc.pa_nclusters;
    for (int32_t i = 0; i < sc.pa_nnodes; ++i) {
        if (spheres) {
            const float4 q = sc.pa_node[i];
            spheres[4 * i] = q.x; spheres[4 * i + 1] = q.y; spheres[4 * i + 2] = q.z; spheres[4 * i + 3] = q.w;
        }
        if (links) { links[2 * i] = sc.pa_link[i].x; links[2 * i + 1] = sc.pa_link[i].y; }
    }
    return RT_OK;
}

/* Host execution of photon aiming's queries (the kernels' code) for n rows
 * of q (9 floats each) with eye = (position, view-cone solid angle):
 *   kind 0: q = (x, w): out[0] = density across w of the environment
 *           photon line through x;
 *   kind 1: q = (y, ny, w): out[0] = solid-angle density of a triangle
 *           photon from y (emitter normal ny) along w;
 *   kind 2: q = (y, ny, u, from_tri): out = sphere of the cluster the
 *           descent picks with u (from_tri = 0: an environment photon);
 *   kind 3: q = (sphere centre, radius, y, u1, u2): out[0..2] = the cone
 *           sample. */
extern "C" rt_status rt_debug_aim_host(const rt_scene *s, const float *eye, int32_t kind, const float *q, int64_t n,
                                       float *out) {
    if (!s || !s->host_only || !eye || n < 0 || (n > 0 && (!q || !out)) || kind < 0 || kind > 3) {
        set_error("rt_debug_aim_host: invalid argument");
        return RT_INVALID_ARG;
    }
    const DevScene &sc = s->host;
    const float4 e = make_float4(eye[0], eye[1], eye[2], eye[3]);
    for (int64_t i = 0; i < n; ++i) {
        const float *r = q + 9 * i;
        float *o = out + 4 * i;
        o[0] = o[1] = o[2] = o[3] = 0.f;
        if (kind == 0) {
            o[0] = aim_env_density(sc, e, v3(r[0], r[1], r[2]), v3(r[3], r[4], r[5]));
        } else if (kind == 1) {
            o[0] = aim_dir_density(sc, e, v3(r[0], r[1], r[2]), v3(r[3], r[4], r[5]), v3(r[6], r[7], r[8]));
        } else if (kind == 2) {
            if (sc.pa_nnodes <= 0) continue;
            const float4 sph = aim_sample(sc, e, r[7] != 0.f, v3(r[0], r[1], r[2]), v3(r[3], r[4], r[5]), r[6]);
            o[0] = sph.x; o[1] = sph.y; o[2] = sph.z; o[3] = sph.w;
        } else {
            const V3 w = aim_cone_sample(make_float4(r[0], r[1], r[2], r[3]), v3(r[4], r[5], r[6]), r[7], r[8]);
            o[0] = w.x; o[1] = w.y; o[2] = w.z;
        }
    }
    return RT_OK;
}

/* Host execution of the environment's NEE sampling (Sec. 2.1.2): for n
 * vertices with geometric normals ng (n x 3) and sample pairs (u, v), the
 * direction drawn for the normal's cell (wi, n x 3), the normal cell, and the
 * solid-angle pdf of that direction for the cell (the environment's share
 * p_env not included). */
extern "C" rt_status rt_debug_env_sample_host(const rt_scene *s, const float *ng, const float *u, const float *v,
                                              int64_t n, float *wi, uint32_t *cell, float *pdf) {
    if (!s || !s->host_only || n < 0) { set_error("rt_debug_env_sample_host: needs a host-only scene"); return RT_INVALID_ARG; }
    const DevScene &sc = s->host;
    if (sc.env_w <= 0) { set_error("rt_debug_env_sample_host: the scene has no environment"); return RT_INVALID_ARG; }
    for (int64_t i = 0; i < n; ++i) {
        const uint32_t c = env_cell(v3(ng[3 * i], ng[3 * i + 1], ng[3 * i + 2]));
        const V3 d = env_sample_cell(sc, c, u[i], v[i]);
        const int tx = env_texel(sc, d);
        wi[3 * i] = d.x; wi[3 * i + 1] = d.y; wi[3 * i + 2] = d.z;
        cell[i] = c;
        pdf[i] = sc.env[tx].w * env_cell_factor(sc, c, tx);
    }
    return RT_OK;
}

/* Host execution of the light hierarchy (Sec. 2.1.1): for n shading points
 * x (n x 3) with geometric normals nrm (n x 3) and numbers u, the emitter
 * drawn (emitter index, the order of the alias table), the probability the
 * descent reports and the probability of that emitter by re-traversal. */
extern "C" rt_status rt_debug_light_bvh_host(const rt_scene *s, const float *x, const float *nrm, const float *u,
                                             int64_t n, uint32_t *emitter, float *p_sample, float *p_retraverse) {
    if (!s || !s->host_only || n < 0) { set_error("rt_debug_light_bvh_host: needs a host-only scene"); return RT_INVALID_ARG; }
    const DevScene &sc = s->host;
    if (!sc.lb_rec) { set_error("rt_debug_light_bvh_host: the scene has no light hierarchy"); return RT_INVALID_ARG; }
    for (int64_t i = 0; i < n; ++i) {
        const V3 p = v3(x[3 * i], x[3 * i + 1], x[3 * i + 2]), nn = v3(nrm[3 * i], nrm[3 * i + 1], nrm[3 * i + 2]);
        float P;
        const uint32_t e = lb_sample(sc, p, nn, u[i], P);
        emitter[i] = e;
        p_sample[i] = P;
        p_retraverse[i] = lb_prob(sc, p, nn, e);
    }
    return RT_OK;
}

/* Host execution of the per-sample path (the megakernel body) for samples
 * (px, py, j): radiance into L (n x 3 floats). */
extern "C" rt_status rt_debug_render_host(const rt_scene *s, const rt_camera *cam, uint32_t max_depth,
                                          const rt_render_opts *opts, const uint32_t *px, const uint32_t *py,
                                          const uint32_t *j, int64_t n, float *L) {
    if (!s || !s->host_only || !cam) { set_error("rt_debug_render_host: needs a host-only scene"); return RT_INVALID_ARG; }
    rt_render_opts o{};
    if (opts) o = *opts;
    std::vector<HaltonDim> dims = make_dims(o.seed, 2 + 7 * (int)(max_depth + 1));
    RenderParams P;
    P.sc = s->host;
    P.cam = make_camera(*cam);
    P.en = make_enum(cam->width, cam->height);
    P.dims = dims.data();
    P.max_depth = max_depth;
    P.sigma = o.filter_sigma == 0.f ? 0.5f : o.filter_sigma;
    P.mis_mode = o.mis_mode;
    P.rr = o.rr_enable;
    const DevScene *sc = &s->host;
    auto closest = [sc](V3 oo, V3 dd, Hit &h) {
        Ray r{oo, dd, 0.f, INFINITY};
        h.prim = RT_MISS; h.inst = 0; h.t = INFINITY; h.b1 = h.b2 = 0.f;
        trace_scene<false>(*sc, r, h);
    };
    auto any = [sc](V3 oo, V3 dd, float tmax) {
        Ray r{oo, dd, 0.f, tmax};
        Hit h;
        h.prim = RT_MISS; h.inst = 0; h.t = INFINITY;
        trace_scene<true>(*sc, r, h);
        return h.prim != RT_MISS;
    };
    for (int64_t i = 0; i < n; ++i) {
        PathState st;
        raygen(P, py[i] * cam->width + px[i], j[i], st);
        uint32_t e = 0, sh = 0;
        finish_path(P, st, closest, any, e, sh);
        L[3 * i] = st.L.x; L[3 * i + 1] = st.L.y; L[3 * i + 2] = st.L.z;
    }
    return RT_OK;
}

/* Host execution of irradiance-probe paths (same code as the kernels):
 * E of sample j[i] of probe p[i] of the n probes pos/nrm (host arrays). */
extern "C" rt_status rt_debug_render_probes_host(const rt_scene *s, const float *pos, const float *nrm, uint32_t n,
                                                 uint32_t max_depth, const rt_render_opts *opts, const uint32_t *p,
                                                 const uint32_t *j, int64_t count, float *E) {
    if (!s || !s->host_only || !pos || !nrm || n == 0) {
        set_error("rt_debug_render_probes_host: needs a host-only scene and probes");
        return RT_INVALID_ARG;
    }
    rt_render_opts o{};
    if (opts) o = *opts;
    std::vector<HaltonDim> dims = make_dims(o.seed, 2 + 7 * (int)(max_depth + 1));
    rt_camera cam{};
    cam.width = n;
    cam.height = 1;
    cam.look_at[2] = 1.f;
    cam.up[1] = 1.f;
    cam.vfov_deg = 45.f;
    RenderParams P;
    P.sc = s->host;
    P.cam = make_camera(cam);
    P.en = make_enum(n, 1);
    P.dims = dims.data();
    P.max_depth = max_depth;
    P.sigma = 0.5f;
    P.mis_mode = o.mis_mode;
    P.rr = o.rr_enable;
    const DevScene *sc = &s->host;
    auto closest = [sc](V3 oo, V3 dd, Hit &h) {
        Ray r{oo, dd, 0.f, INFINITY};
        h.prim = RT_MISS; h.inst = 0; h.t = INFINITY; h.b1 = h.b2 = 0.f;
        trace_scene<false>(*sc, r, h);
    };
    auto any = [sc](V3 oo, V3 dd, float tmax) {
        Ray r{oo, dd, 0.f, tmax};
        Hit h;
        h.prim = RT_MISS; h.inst = 0; h.t = INFINITY;
        trace_scene<true>(*sc, r, h);
        return h.prim != RT_MISS;
    };
    for (int64_t i = 0; i < count; ++i) {
        if (p[i] >= n) { set_error("rt_debug_render_probes_host: probe index out of range"); return RT_INVALID_ARG; }
        PathState st;
        st.index = pixel_base_index(P.en, p[i], 0) + (uint64_t)j[i] * P.en.period;
        st.pixel = p[i];
        st.depth = 1;
        st.beta = v3(kPi, kPi, kPi);
        st.L = v3(0.f, 0.f, 0.f);
        st.prev_pdf = 0.f;
        st.prev_cell = 0;
        st.prev_n = 0;
        st.o = st.d = v3(0.f, 0.f, 0.f);
        const V3 x = v3(pos[3 * (size_t)p[i]], pos[3 * (size_t)p[i] + 1], pos[3 * (size_t)p[i] + 2]);
        const V3 nn = normalize(v3(nrm[3 * (size_t)p[i]], nrm[3 * (size_t)p[i] + 1], nrm[3 * (size_t)p[i] + 2]));
        ShadowRay sh;
        int r = probe_vertex(P, st, x, nn, sh);
        if ((r & 2) && !any(sh.o, sh.d, sh.tmax)) st.L = st.L + sh.contrib;
        uint32_t e = 0, shc = 0;
        if (r & 1) finish_path(P, st, closest, any, e, shc);
        E[3 * i] = st.L.x; E[3 * i + 1] = st.L.y; E[3 * i + 2] = st.L.z;
    }
    return RT_OK;
}

/* Host execution of the Halton routine (same code as the kernels). */
extern "C" rt_status rt_debug_halton_host(uint32_t W, uint32_t H, uint64_t seed, const uint64_t *idx, int64_t n,
                                          int32_t ndims, uint32_t *out) {
    if (W == 0 || H == 0 || n < 0 || ndims < 0) { set_error("rt_debug_halton_host: invalid argument"); return RT_INVALID_ARG; }
    std::vector<HaltonDim> d = make_dims(seed, std::max(ndims, 3));
    Enum en = make_enum(W, H);
    for (int64_t i = 0; i < n; ++i)
        for (int32_t k = 0; k < ndims; ++k)
            out[i * ndims + k] = k == 0 ? dim0_bits(en, idx[i]) : (k == 1 ? dim1_bits(en, idx[i]) : radical_inverse(idx[i], d[k]));
    return RT_OK;
}

extern "C" rt_status rt_debug_sample_index_host(uint32_t W, uint32_t H, uint32_t x, uint32_t y, uint32_t j,
                                                uint64_t *out) {
    Enum en = make_enum(W, H);
    *out = pixel_base_index(en, x, y) + (uint64_t)j * en.period;
    return RT_OK;
}
