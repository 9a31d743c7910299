// Wavefront path tracing on one GPU (paper Sec. 3.1): structure-of-arrays
// sample state, one kernel per state (closest-hit trace, shade, shadow
// trace), queues compacted just in time with warp ballots, a megakernel that
// finishes the tail when few samples remain (Sec. 3.1.3), iteration sets with
// per-pixel FP64 accumulation and sample counts (Sec. 3.2.2, Appendix A.4),
// and the rays -> hits entry point (Sec. 3.1, ray casting state kernels).
//
// Scheduling differs from the paper's single just-in-time queue picked
// greedily by state population: GB300 memory is ample, so every state keeps
// its own queue and each bounce step runs all state kernels in a fixed order
// whose launch grids never depend on host-side counts (kernels read queue
// lengths from device memory). The host only synchronises between
// iteration sets, where it checks the time budget and the abort flag.
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "internal.h"
#include "shade.cuh"
#include "trace_kernel.cuh"
#include "guide_mlp.cuh"

namespace rtg {

struct Ctrl {
    uint32_t n_ext, n_next, n_shadow, cur;
    uint32_t tail, overflow, tail_threshold, pad;
    uint32_t fetch_ext, fetch_shadow, fetch_shade, n_train;
    unsigned long long ext_rays, shadow_rays;
    unsigned long long ext_nodes, ext_tris, shadow_nodes, shadow_tris;
    // regeneration (Sec. 3.1.3): paths that ended this step, emptied slots,
    // tasks of the window issued so far and in total, and the stop state
    uint32_t n_dead, n_free, task_next, n_tasks;
    uint32_t stop, regen_sets;
    // entries of Pool::split written by the closest-hit kernel: hits in the
    // low 32 bits, misses in the high 32 bits (one atomic per warp for both)
    unsigned long long split_counts;
    unsigned long long deadline_ns;   // %globaltimer value after which no task is issued
};

// Structure-of-arrays path state (capacity = pool size).
struct Pool {
    float4 *ray_o;   // pending ray origin
    float4 *ray_d;   // pending ray direction, w = prev_pdf
    float4 *beta;    // throughput, w = vertex number (uint bits)
    float4 *L;       // radiance so far
    uint2 *index;    // 64-bit QMC index
    uint32_t *pixel;
    float4 *hit;     // prim bits, t, b1, b2
    uint32_t *hit_inst; // instance of the hit (two-level scenes only)
    float4 *sh_o;    // shadow origin, w = tmax
    float4 *sh_d;
    float4 *sh_c;    // shadow contribution
    uint32_t *q[2];  // extension-ray queues (current / next)
    uint32_t *qs;    // shadow-ray queue
    Ctrl *ctrl;
    uint32_t capacity;
    uint32_t *nrec;  // guided rendering: training records per path (count | pending flag), else null
    // regeneration only (null otherwise): task of each slot (offset in the
    // window) and the slots whose path ended this step
    uint32_t *task;
    uint32_t *qd;
    // compressed state (Sec. 3.1.1, rt_render_opts.state_compression): when
    // `compact` is set these replace ray_d, beta, sh_d and sh_c (null then):
    // direction as a 16:16 octahedral code + prev_pdf (FP32); throughput as
    // three BF16 + the vertex number (16 bits); shadow direction as an
    // octahedral code; shadow contribution as three BF16
    uint2 *dir_c;
    uint2 *beta_c;
    uint32_t *shd_c;
    uint2 *shc_c;
    int compact;
    // The extension queue as the closest-hit kernel leaves it for shading
    // (null = off): the paths whose ray hit a surface from the front, those
    // whose ray left the scene from the back, so that shading warps run one
    // of the two branches instead of both.
    uint32_t *split;
};

RT_D uint32_t bf16x2_pack(float a, float b) {
    return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(a)) |
           ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(b)) << 16);
}
RT_D float bf16_lo(uint32_t w) { return __bfloat162float(__ushort_as_bfloat16((unsigned short)(w & 0xffffu))); }
RT_D float bf16_hi(uint32_t w) { return __bfloat162float(__ushort_as_bfloat16((unsigned short)(w >> 16))); }

// Accessors of the arrays that have a compressed form: (xyz, w) as in the
// uncompressed float4 layout.
RT_D float4 ld_dir(const Pool &p, uint32_t q) {
    if (!p.compact) return p.ray_d[q];
    const uint2 c = p.dir_c[q];
    const V3 d = oct_decode(c.x);
    return make_float4(d.x, d.y, d.z, __uint_as_float(c.y));
}
RT_D void st_dir(const Pool &p, uint32_t q, V3 d, float prev_pdf) {
    if (!p.compact) p.ray_d[q] = make_float4(d.x, d.y, d.z, prev_pdf);
    else p.dir_c[q] = make_uint2(oct_encode(d), __float_as_uint(prev_pdf));
}
RT_D float4 ld_beta(const Pool &p, uint32_t q) {   // w: vertex number bits
    if (!p.compact) return p.beta[q];
    const uint2 c = p.beta_c[q];
    return make_float4(bf16_lo(c.x), bf16_hi(c.x), bf16_lo(c.y), __uint_as_float(c.y >> 16));
}
RT_D void st_beta(const Pool &p, uint32_t q, V3 b, uint32_t depth) {
    if (!p.compact) p.beta[q] = make_float4(b.x, b.y, b.z, __uint_as_float(depth));
    else p.beta_c[q] = make_uint2(bf16x2_pack(b.x, b.y), (bf16x2_pack(b.z, 0.f) & 0xffffu) | (depth << 16));
}
RT_D float4 ld_shd(const Pool &p, uint32_t q) {
    if (!p.compact) return p.sh_d[q];
    const V3 d = oct_decode(p.shd_c[q]);
    return make_float4(d.x, d.y, d.z, 0.f);
}
RT_D void st_shd(const Pool &p, uint32_t q, V3 d) {
    if (!p.compact) p.sh_d[q] = make_float4(d.x, d.y, d.z, 0.f);
    else p.shd_c[q] = oct_encode(d);
}
RT_D float4 ld_shc(const Pool &p, uint32_t q) {
    if (!p.compact) return p.sh_c[q];
    const uint2 c = p.shc_c[q];
    return make_float4(bf16_lo(c.x), bf16_hi(c.x), bf16_lo(c.y), 0.f);
}
RT_D void st_shc(const Pool &p, uint32_t q, V3 c) {
    if (!p.compact) p.sh_c[q] = make_float4(c.x, c.y, c.z, 0.f);
    else p.shc_c[q] = make_uint2(bf16x2_pack(c.x, c.y), bf16x2_pack(c.z, 0.f));
}

RT_D void store_state(const Pool &p, uint32_t q, const PathState &s) {
    p.ray_o[q] = make_float4(s.o.x, s.o.y, s.o.z, __uint_as_float(s.prev_cell));
    st_dir(p, q, s.d, s.prev_pdf);
    st_beta(p, q, s.beta, s.depth);
    p.L[q] = make_float4(s.L.x, s.L.y, s.L.z, __uint_as_float(s.prev_n));
    p.index[q] = make_uint2((uint32_t)s.index, (uint32_t)(s.index >> 32));
    p.pixel[q] = s.pixel;
}

RT_D PathState load_state(const Pool &p, uint32_t q) {
    PathState s;
    float4 o = p.ray_o[q], d = ld_dir(p, q), b = ld_beta(p, q), L = p.L[q];
    uint2 ix = p.index[q];
    s.o = v3(o.x, o.y, o.z);
    s.prev_cell = __float_as_uint(o.w);
    s.d = v3(d.x, d.y, d.z);
    s.prev_pdf = d.w;
    s.beta = v3(b.x, b.y, b.z);
    s.depth = __float_as_uint(b.w);
    s.L = v3(L.x, L.y, L.z);
    s.prev_n = __float_as_uint(L.w);
    s.index = (uint64_t)ix.x | ((uint64_t)ix.y << 32);
    s.pixel = p.pixel[q];
    return s;
}

// Append `item` to `queue` for every lane with pred set: one atomic per warp
// (ballot + population count), order inside the warp preserved.
RT_D void warp_append(uint32_t *queue, uint32_t *count, bool pred, uint32_t item) {
    const uint32_t full = 0xFFFFFFFFu;
    uint32_t mask = __ballot_sync(full, pred);
    if (!mask) return;
    uint32_t lane = lane_id();
    uint32_t leader = __ffs(mask) - 1;
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(count, (uint32_t)__popc(mask));
    base = __shfl_sync(full, base, leader);
    if (pred) queue[base + __popc(mask & ((1u << lane) - 1u))] = item;
}

// Warp-granular dynamic work distribution: lane 0 reserves the next 32 queue
// entries with one atomic and broadcasts the base; warps that drew short
// work come back for more, so a launch ends when the queue is drained
// rather than when the unluckiest statically assigned thread finishes.
RT_D uint32_t warp_fetch32(uint32_t *counter) {
    uint32_t base = 0;
    if (lane_id() == 0) base = atomicAdd(counter, 32u);
    return __shfl_sync(0xFFFFFFFFu, base, 0);
}

RT_D void count_rays(unsigned long long *ctr, bool pred) {
    uint32_t mask = __ballot_sync(0xFFFFFFFFu, pred);
    if (lane_id() == 0 && mask) atomicAdd(ctr, (unsigned long long)__popc(mask));
}

struct DevTraceClosest {
    const DevScene *sc;
    bool *overflow;
    RT_D void operator()(V3 o, V3 d, Hit &h) const {
        Ray r{o, d, 0.f, INFINITY};
        h.prim = RT_MISS; h.inst = 0; h.t = INFINITY; h.b1 = h.b2 = 0.f;
        TraceResult tr = trace_scene<false>(*sc, r, h);
        if (tr.overflow) *overflow = true;
    }
};
struct DevTraceAny {
    const DevScene *sc;
    bool *overflow;
    RT_D bool operator()(V3 o, V3 d, float tmax) const {
        Ray r{o, d, 0.f, tmax};
        Hit h;
        h.prim = RT_MISS; h.t = INFINITY;
        TraceResult tr = trace_scene<true>(*sc, r, h);
        if (tr.overflow) *overflow = true;
        return h.prim != RT_MISS;
    }
};

// ------------------------------------------------------------------ kernels
__global__ void k_raygen(RenderParams P, Pool pool, uint64_t t0, uint32_t n, uint32_t WH, uint32_t tail_threshold) {
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
        uint64_t t = t0 + q;
        PathState s;
        raygen(P, (uint32_t)(t % WH), (uint32_t)(t / WH), s);
        store_state(pool, q, s);
        pool.q[0][q] = q;
        if (pool.nrec) pool.nrec[q] = 0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        Ctrl *c = pool.ctrl;
        c->n_ext = n;
        c->n_next = 0;
        c->n_shadow = 0;
        c->cur = 0;
        c->fetch_ext = 0;
        c->fetch_shadow = 0;
        c->fetch_shade = 0;
        c->split_counts = 0;
        c->n_train = 0;
        c->tail_threshold = tail_threshold;
        c->tail = n < tail_threshold ? 1u : 0u;
    }
}

// Closest-hit traversal of the current extension queue.
struct ExtJob {
    const float4 *ray_o, *ray_d;
    float4 *hit;
    const uint32_t *queue;
    RT_D Ray load(uint32_t i) const {
        uint32_t q = queue[i];
        float4 o = ray_o[q], d = ray_d[q];
        return Ray{v3(o.x, o.y, o.z), v3(d.x, d.y, d.z), 0.f, INFINITY};
    }
    RT_D void store(uint32_t i, const Hit &h) const {
        hit[queue[i]] = make_float4(__uint_as_float(h.prim), h.t, h.b1, h.b2);
    }
};

template <bool kCount>
__global__ void __launch_bounds__(128) k_trace_ext(DevScene sc, Pool pool) {
    Ctrl *c = pool.ctrl;
    if (c->tail) return;
    const uint32_t n = c->n_ext;
    ExtJob job{pool.ray_o, pool.ray_d, pool.hit, pool.q[c->cur]};
    bool overflow = false;
    WorkCount wc;
    trace_persistent<false, kCount>(sc.nodes, sc.tris, job, n, &c->fetch_ext, overflow, wc);
    if (overflow) atomicOr(&c->overflow, 1u);
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&c->ext_rays, (unsigned long long)n);
    if (kCount) {
        atomicAdd(&c->ext_nodes, (unsigned long long)wc.nodes);
        atomicAdd(&c->ext_tris, (unsigned long long)wc.tris);
    }
}

// Pool::split entry of every lane with `valid` (one atomic per warp): hits
// from the front in queue order, misses from the back.
RT_D void split_append(uint32_t *split, Ctrl *c, uint32_t n, bool valid, bool hit, uint32_t q) {
    const uint32_t full = 0xFFFFFFFFu, lane = lane_id();
    const uint32_t hm = __ballot_sync(full, valid && hit), mm = __ballot_sync(full, valid && !hit);
    unsigned long long b = 0;
    if (lane == 0)
        b = atomicAdd(&c->split_counts, (unsigned long long)__popc(hm) | ((unsigned long long)__popc(mm) << 32));
    b = __shfl_sync(full, b, 0);
    const uint32_t hb = (uint32_t)b, mb = (uint32_t)(b >> 32);
    const uint32_t below = (1u << lane) - 1u;
    if (valid && hit) split[hb + (uint32_t)__popc(hm & below)] = q;
    if (valid && !hit) split[n - 1u - (mb + (uint32_t)__popc(mm & below))] = q;
}

// Capped at 64 registers (8 blocks of 128 per SM): the kernel is latency
// bound, and the extra resident warps outweigh a few spilled registers.
template <bool kLb>
__global__ void __launch_bounds__(128, 8) k_shade(RenderParams P, Pool pool, const uint32_t *sorted) {
    Ctrl *c = pool.ctrl;
    // the closest-hit kernel of this step is done with the split counters
    if (blockIdx.x == 0 && threadIdx.x == 0) c->split_counts = 0;
    if (c->tail) return;
    const uint32_t n = c->n_ext;
    const uint32_t cur = c->cur;
    const uint32_t *queue = sorted ? sorted : pool.q[cur];
    uint32_t *next = pool.q[cur ^ 1u];
    for (;;) {
        uint32_t base = warp_fetch32(&c->fetch_shade);
        if (base >= n) break;
        uint32_t i = base + lane_id();
        bool valid = i < n;
        uint32_t q = 0;
        int r = 0;
        if (valid) {
            q = queue[i];
            PathState s = load_state(pool, q);
            float4 hv = pool.hit[q];
            Hit h;
            h.prim = __float_as_uint(hv.x); h.inst = P.sc.two_level ? pool.hit_inst[q] : 0u;
            h.t = hv.y; h.b1 = hv.z; h.b2 = hv.w;
            ShadowRay sh;
            r = shade<kLb>(P, s, h, sh);
            pool.L[q] = make_float4(s.L.x, s.L.y, s.L.z, __uint_as_float(s.prev_n));
            if (r & 1) {
                pool.ray_o[q] = make_float4(s.o.x, s.o.y, s.o.z, __uint_as_float(s.prev_cell));
                st_dir(pool, q, s.d, s.prev_pdf);
                st_beta(pool, q, s.beta, s.depth);
            }
            if (r & 2) {
                pool.sh_o[q] = make_float4(sh.o.x, sh.o.y, sh.o.z, sh.tmax);
                st_shd(pool, q, sh.d);
                st_shc(pool, q, sh.contrib);
            }
        }
        warp_append(next, &c->n_next, valid && (r & 1), q);
        warp_append(pool.qs, &c->n_shadow, valid && (r & 2), q);
        if (pool.qd) warp_append(pool.qd, &c->n_dead, valid && !(r & 1), q);
    }
}

// One ray per thread, traced to completion (A/B variant of the above).
// kTwoLevel selects the instanced (two-level) traversal at compile time: the
// single-level kernels carry none of its state and need about a third fewer
// registers, which raises the resident warps per SM from 20 to 32 (the launch
// bounds hold them at 64 registers, 8 blocks of 128 per SM).
template <bool kCount, bool kSmemStack, bool kTwoLevel, bool kPostpone = false, bool kNear = false>
__global__ void __launch_bounds__(128, kTwoLevel ? 5 : 8) k_trace_ext_simple(DevScene sc, Pool pool, const uint32_t *sorted) {
    Ctrl *c = pool.ctrl;
    if (c->tail) return;
    const uint32_t n = c->n_ext;
    const uint32_t *queue = sorted ? sorted : pool.q[c->cur];
    extern __shared__ uint2 s_stk[];
    SharedStack sst{s_stk + threadIdx.x, (int)blockDim.x};
    bool overflow = false;
    uint32_t nodes = 0, tris = 0;
    for (;;) {
        uint32_t base = warp_fetch32(&c->fetch_ext);
        if (base >= n) break;
        const uint32_t i = base + lane_id();
        const bool valid = i < n;
        uint32_t q = 0;
        bool hit = false;
        if (valid) {
            q = queue[i];
            float4 o = pool.ray_o[q], d = ld_dir(pool, q);
            Ray r{v3(o.x, o.y, o.z), v3(d.x, d.y, d.z), 0.f, INFINITY};
            Hit h;
            h.prim = RT_MISS; h.inst = 0; h.t = INFINITY; h.b1 = h.b2 = 0.f;
            TraceResult tr = kTwoLevel    ? traverse_two_level<false>(sc, r, h)
                             : kNear      ? traverse_near(sc.nodes, sc.tris, r, h)
                             : kPostpone  ? traverse_pp<false>(sc.nodes, sc.tris, r, h)
                             : kSmemStack ? traverse<false, SharedStack>(sc.nodes, sc.tris, 0u, r, h, 0u, &sst)
                                          : traverse<false>(sc.nodes, sc.tris, 0u, r, h);
            overflow |= tr.overflow;
            if (kCount) { nodes += tr.nodes; tris += tr.tris; }
            pool.hit[q] = make_float4(__uint_as_float(h.prim), h.t, h.b1, h.b2);
            if (kTwoLevel) pool.hit_inst[q] = h.inst;
            hit = h.prim != RT_MISS;
        }
        if (pool.split) split_append(pool.split, c, n, valid, hit, q);
    }
    if (overflow) atomicOr(&c->overflow, 1u);
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&c->ext_rays, (unsigned long long)n);
    if (kCount) {
        atomicAdd(&c->ext_nodes, (unsigned long long)nodes);
        atomicAdd(&c->ext_tris, (unsigned long long)tris);
    }
}

template <bool kCount, bool kSmemStack, bool kTwoLevel, bool kPostpone = false>
__global__ void __launch_bounds__(128, kTwoLevel ? 5 : 8) k_trace_shadow_simple(DevScene sc, Pool pool, const uint32_t *) {
    Ctrl *c = pool.ctrl;
    if (c->tail) return;
    const uint32_t n = c->n_shadow;
    extern __shared__ uint2 s_stk[];
    SharedStack sst{s_stk + threadIdx.x, (int)blockDim.x};
    bool overflow = false;
    uint32_t nodes = 0, tris = 0;
    for (;;) {
        uint32_t base = warp_fetch32(&c->fetch_shadow);
        if (base >= n) break;
        uint32_t i = base + lane_id();
        if (i >= n) continue;
        uint32_t q = pool.qs[i];
        float4 o = pool.sh_o[q], d = ld_shd(pool, q);
        Ray r{v3(o.x, o.y, o.z), v3(d.x, d.y, d.z), 0.f, o.w};
        Hit h;
        h.prim = RT_MISS; h.inst = 0; h.t = INFINITY;
        TraceResult tr = kTwoLevel    ? traverse_two_level<true>(sc, r, h)
                         : kPostpone  ? traverse_pp<true>(sc.nodes, sc.tris, r, h)
                         : kSmemStack ? traverse<true, SharedStack>(sc.nodes, sc.tris, 0u, r, h, 0u, &sst)
                                      : traverse<true>(sc.nodes, sc.tris, 0u, r, h);
        overflow |= tr.overflow;
        if (kCount) { nodes += tr.nodes; tris += tr.tris; }
        if (h.prim == RT_MISS) {
            float4 cc = ld_shc(pool, q), L = pool.L[q];
            pool.L[q] = make_float4(L.x + cc.x, L.y + cc.y, L.z + cc.z, L.w);
        }
    }
    if (overflow) atomicOr(&c->overflow, 1u);
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&c->shadow_rays, (unsigned long long)n);
    if (kCount) {
        atomicAdd(&c->shadow_nodes, (unsigned long long)nodes);
        atomicAdd(&c->shadow_tris, (unsigned long long)tris);
    }
}

// One ray per lane with lane refill (A/B variant, single-level scenes): a
// warp keeps stepping its rays one node visit (with that node's triangles)
// at a time, and whenever at least kRefillLanes of its lanes are idle it
// reserves that many queue entries with one atomic and starts new rays on
// them (dynamic ray fetch, Aila and Laine 2009), so that finished lanes do
// not wait for the longest ray of the warp. Results equal the one-shot
// kernels' (same Traversal steps, same tie rule).
constexpr int kRefillLanes = 8;

template <bool kAnyHit, bool kCount>
__global__ void __launch_bounds__(128, 8) k_trace_refill(DevScene sc, Pool pool, const uint32_t *sorted) {
    Ctrl *c = pool.ctrl;
    if (c->tail) return;
    const uint32_t n = kAnyHit ? c->n_shadow : c->n_ext;
    uint32_t *fetch = kAnyHit ? &c->fetch_shadow : &c->fetch_ext;
    const uint32_t *queue = kAnyHit ? pool.qs : (sorted ? sorted : pool.q[c->cur]);
    const uint32_t FULL = 0xFFFFFFFFu, lane = lane_id();
    LocalStack stack;
    Traversal<kAnyHit> tr;
    Hit h;
    h.prim = RT_MISS; h.inst = 0; h.t = INFINITY; h.b1 = h.b2 = 0.f;
    TraceResult res{false, 0u, 0u};
    bool active = false, exhausted = false, overflow = false;
    uint32_t q = 0, nodes = 0, tris = 0;
    for (;;) {
        const uint32_t idle = __ballot_sync(FULL, !active);
        if (!exhausted && __popc(idle) >= kRefillLanes) {
            const uint32_t cnt = __popc(idle), leader = __ffs(idle) - 1;
            uint32_t base = 0;
            if (lane == leader) base = atomicAdd(fetch, cnt);
            base = __shfl_sync(FULL, base, leader);
            if (base + cnt >= n) exhausted = true;
            if (!active) {
                const uint32_t i = base + __popc(idle & lanemask_lt());
                if (i < n) {
                    q = queue[i];
                    Ray r;
                    if (kAnyHit) {
                        float4 o = pool.sh_o[q], d = ld_shd(pool, q);
                        r = Ray{v3(o.x, o.y, o.z), v3(d.x, d.y, d.z), 0.f, o.w};
                    } else {
                        float4 o = pool.ray_o[q], d = ld_dir(pool, q);
                        r = Ray{v3(o.x, o.y, o.z), v3(d.x, d.y, d.z), 0.f, INFINITY};
                    }
                    h.prim = RT_MISS; h.inst = 0; h.t = INFINITY; h.b1 = h.b2 = 0.f;
                    tr.begin(r, h, 0u, 0u);
                    res = TraceResult{false, 0u, 0u};
                    active = true;
                }
            }
        }
        if (__ballot_sync(FULL, active) == 0u) break;
        if (active && !tr.step(sc.nodes, sc.tris, stack, h, res)) {
            active = false;
            overflow |= res.overflow;
            if (kCount) { nodes += res.nodes; tris += res.tris; }
            if (kAnyHit) {
                if (h.prim == RT_MISS) {
                    float4 cc = ld_shc(pool, q), L = pool.L[q];
                    pool.L[q] = make_float4(L.x + cc.x, L.y + cc.y, L.z + cc.z, L.w);
                }
            } else {
                pool.hit[q] = make_float4(__uint_as_float(h.prim), h.t, h.b1, h.b2);
            }
        }
    }
    if (overflow) atomicOr(&c->overflow, 1u);
    if (blockIdx.x == 0 && threadIdx.x == 0)
        atomicAdd(kAnyHit ? &c->shadow_rays : &c->ext_rays, (unsigned long long)n);
    if (kCount) {
        atomicAdd(kAnyHit ? &c->shadow_nodes : &c->ext_nodes, (unsigned long long)nodes);
        atomicAdd(kAnyHit ? &c->shadow_tris : &c->ext_tris, (unsigned long long)tris);
    }
}

// Counting sorts of the extension queue (A/B options), with one shared
// atomic per distinct key per warp in the histogram and one global atomic
// per distinct key per warp in the scatter:
//  - by material of the hit (misses last), so that lanes shade one material;
//  - by ray direction octant and an 8 x 8 x 8 Morton cell of the origin in
//    the scene box, so that neighbouring lanes traverse similar subtrees.
struct MatKey {
    DevScene sc;
    uint32_t nmat;
    RT_D uint32_t operator()(const Pool &pool, uint32_t q) const {
        uint32_t prim = __float_as_uint(pool.hit[q].x);
        return prim == RT_MISS ? nmat : __ldg(sc.tri_material + prim);
    }
};
RT_D uint32_t spread3(uint32_t x) {   // 3 bits -> every third bit
    return (x & 1u) | ((x & 2u) << 2) | ((x & 4u) << 4);
}
struct RayKey {
    float3 lo, inv_ext;
    RT_D uint32_t operator()(const Pool &pool, uint32_t q) const {
        float4 o = pool.ray_o[q], d = ld_dir(pool, q);
        uint32_t cx = (uint32_t)fminf(7.f, fmaxf(0.f, (o.x - lo.x) * inv_ext.x * 8.f));
        uint32_t cy = (uint32_t)fminf(7.f, fmaxf(0.f, (o.y - lo.y) * inv_ext.y * 8.f));
        uint32_t cz = (uint32_t)fminf(7.f, fmaxf(0.f, (o.z - lo.z) * inv_ext.z * 8.f));
        uint32_t oct = (d.x < 0.f ? 1u : 0u) | (d.y < 0.f ? 2u : 0u) | (d.z < 0.f ? 4u : 0u);
        return (oct << 9) | spread3(cx) | (spread3(cy) << 1) | (spread3(cz) << 2);
    }
};

template <class Key>
__global__ void k_sort_hist(Key key, Pool pool, uint32_t nkeys, uint32_t *hist) {
    extern __shared__ uint32_t sh_hist[];
    Ctrl *c = pool.ctrl;
    if (c->tail) return;
    for (uint32_t k = threadIdx.x; k < nkeys; k += blockDim.x) sh_hist[k] = 0;
    __syncthreads();
    const uint32_t n = c->n_ext;
    const uint32_t *queue = pool.q[c->cur];
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t base = (blockIdx.x * blockDim.x + threadIdx.x) & ~31u; base < n; base += stride) {
        uint32_t i = base + lane_id();
        uint32_t k = i < n ? key(pool, queue[i]) : 0xFFFFFFFFu;
        uint32_t peers = __match_any_sync(0xFFFFFFFFu, k);
        if (i < n && lane_id() == (uint32_t)(__ffs(peers) - 1)) atomicAdd(&sh_hist[k], (uint32_t)__popc(peers));
    }
    __syncthreads();
    for (uint32_t k = threadIdx.x; k < nkeys; k += blockDim.x)
        if (sh_hist[k]) atomicAdd(&hist[k], sh_hist[k]);
}

// Exclusive scan of up to a few thousand counts in one block of 1024 threads.
__global__ void k_sort_scan(Pool pool, uint32_t nkeys, uint32_t *hist) {
    __shared__ uint32_t part[1024];
    if (pool.ctrl->tail) return;
    const uint32_t per = (nkeys + blockDim.x - 1) / blockDim.x;
    const uint32_t b = threadIdx.x * per, e = min(nkeys, b + per);
    uint32_t sum = 0;
    for (uint32_t k = b; k < e; ++k) sum += hist[k];
    part[threadIdx.x] = sum;
    __syncthreads();
    for (uint32_t off = 1; off < blockDim.x; off <<= 1) {
        uint32_t v = threadIdx.x >= off ? part[threadIdx.x - off] : 0u;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    uint32_t acc = part[threadIdx.x] - sum;
    for (uint32_t k = b; k < e; ++k) {
        uint32_t v = hist[k];
        hist[k] = acc;
        acc += v;
    }
}

template <class Key>
__global__ void k_sort_scatter(Key key, Pool pool, uint32_t *offsets, uint32_t *sorted) {
    Ctrl *c = pool.ctrl;
    if (c->tail) return;
    const uint32_t n = c->n_ext;
    const uint32_t *queue = pool.q[c->cur];
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t base = (blockIdx.x * blockDim.x + threadIdx.x) & ~31u; base < n; base += stride) {
        uint32_t i = base + lane_id();
        uint32_t k = 0xFFFFFFFFu, q = 0;
        if (i < n) {
            q = queue[i];
            k = key(pool, q);
        }
        uint32_t peers = __match_any_sync(0xFFFFFFFFu, k);
        uint32_t leader = __ffs(peers) - 1;
        uint32_t pos = 0;
        if (i < n && lane_id() == leader) pos = atomicAdd(&offsets[k], (uint32_t)__popc(peers));
        pos = __shfl_sync(0xFFFFFFFFu, pos, leader);
        if (i < n) sorted[pos + __popc(peers & ((1u << lane_id()) - 1u))] = q;
    }
}

// Any-hit traversal of the shadow queue; unoccluded contributions are added.
struct ShadowJob {
    const float4 *sh_o, *sh_d, *sh_c;
    float4 *L;
    const uint32_t *qs;
    RT_D Ray load(uint32_t i) const {
        uint32_t q = qs[i];
        float4 o = sh_o[q], d = sh_d[q];
        return Ray{v3(o.x, o.y, o.z), v3(d.x, d.y, d.z), 0.f, o.w};
    }
    RT_D void store(uint32_t i, const Hit &h) const {
        if (h.prim != RT_MISS) return;
        uint32_t q = qs[i];
        float4 cc = sh_c[q], l = L[q];
        L[q] = make_float4(l.x + cc.x, l.y + cc.y, l.z + cc.z, l.w);
    }
};

template <bool kCount>
__global__ void __launch_bounds__(128) k_trace_shadow(DevScene sc, Pool pool) {
    Ctrl *c = pool.ctrl;
    if (c->tail) return;
    const uint32_t n = c->n_shadow;
    ShadowJob job{pool.sh_o, pool.sh_d, pool.sh_c, pool.L, pool.qs};
    bool overflow = false;
    WorkCount wc;
    trace_persistent<true, kCount>(sc.nodes, sc.tris, job, n, &c->fetch_shadow, overflow, wc);
    if (overflow) atomicOr(&c->overflow, 1u);
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&c->shadow_rays, (unsigned long long)n);
    if (kCount) {
        atomicAdd(&c->shadow_nodes, (unsigned long long)wc.nodes);
        atomicAdd(&c->shadow_tris, (unsigned long long)wc.tris);
    }
}

__global__ void k_step_end(Pool pool) {
    Ctrl *c = pool.ctrl;
    if (!c->tail) {
        c->n_ext = c->n_next;
        c->n_next = 0;
        c->cur ^= 1u;
        if (c->n_ext < c->tail_threshold) c->tail = 1u;
    }
    c->n_shadow = 0;
    c->fetch_ext = 0;
    c->fetch_shadow = 0;
    c->fetch_shade = 0;
}

// Megakernel: every remaining sample runs to completion in its own thread.
__global__ void __launch_bounds__(128) k_megakernel(RenderParams P, Pool pool) {
    Ctrl *c = pool.ctrl;
    if (!c->tail) return;
    const uint32_t n = c->n_ext;
    const uint32_t *queue = pool.q[c->cur];
    bool overflow = false;
    uint32_t ext = 0, shadow = 0;
    DevTraceClosest closest{&P.sc, &overflow};
    DevTraceAny any{&P.sc, &overflow};
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        uint32_t q = queue[i];
        PathState s = load_state(pool, q);
        finish_path(P, s, closest, any, ext, shadow);
        pool.L[q] = make_float4(s.L.x, s.L.y, s.L.z, __uint_as_float(s.prev_n));
    }
    if (ext) atomicAdd(&c->ext_rays, (unsigned long long)ext);
    if (shadow) atomicAdd(&c->shadow_rays, (unsigned long long)shadow);
    if (overflow) atomicOr(&c->overflow, 1u);
}

// Film accumulation, owner-exclusive per pixel (deterministic order).
// passes > 0: the wave holds `passes` whole passes, slot = pass * WH + pixel.
// passes == 0: the wave holds n <= WH distinct consecutive pixels from t0.
// Irradiance probes (Sec. 4.2). Task t is sample t / n of probe t % n, the
// pixel (p, 0) of an n x 1 image for the sample enumeration. The probe
// vertex (vertex 1) is shaded here with throughput pi (its radiance times pi
// is the irradiance); every path continues into the extension queue, NEE
// shadow rays go to the shadow queue. The counters are set by k_probe_reset.
__global__ void k_probe_reset(Pool pool) {
    Ctrl *c = pool.ctrl;
    c->n_ext = 0;
    c->n_next = 0;
    c->n_shadow = 0;
    c->cur = 0;
    c->fetch_ext = 0;
    c->fetch_shadow = 0;
    c->fetch_shade = 0;
    c->n_train = 0;
    c->tail_threshold = 0;
    c->tail = 0;
}

__global__ void k_probe_start(RenderParams P, Pool pool, const float *pos, const float *nrm, uint64_t t0, uint32_t n,
                              uint32_t WH) {
    Ctrl *c = pool.ctrl;
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t b = blockIdx.x * blockDim.x; b < n; b += stride) {   // uniform per warp (warp_append)
        const uint32_t q = b + threadIdx.x;
        const bool valid = q < n;
        int r = 0;
        if (valid) {
            const uint64_t t = t0 + q;
            const uint32_t p = (uint32_t)(t % WH), j = (uint32_t)(t / WH);
            PathState s;
            s.index = pixel_base_index(P.en, p, 0) + (uint64_t)j * P.en.period;
            s.pixel = p;
            s.depth = 1;
            s.beta = v3(kPi, kPi, kPi);
            s.L = v3(0.f, 0.f, 0.f);
            s.prev_pdf = 0.f;
            s.prev_cell = 0;
            s.prev_n = 0;
            s.o = s.d = v3(0.f, 0.f, 0.f);
            const V3 x = v3(pos[3 * (size_t)p], pos[3 * (size_t)p + 1], pos[3 * (size_t)p + 2]);
            const V3 nn = normalize(v3(nrm[3 * (size_t)p], nrm[3 * (size_t)p + 1], nrm[3 * (size_t)p + 2]));
            ShadowRay sh;
            r = probe_vertex(P, s, x, nn, sh);
            store_state(pool, q, s);
            if (r & 2) {
                pool.sh_o[q] = make_float4(sh.o.x, sh.o.y, sh.o.z, sh.tmax);
                st_shd(pool, q, sh.d);
                st_shc(pool, q, sh.contrib);
            }
        }
        warp_append(pool.q[0], &c->n_ext, valid && (r & 1), q);
        warp_append(pool.qs, &c->n_shadow, valid && (r & 2), q);
    }
}

// After the probe vertex's shadow rays are traced: an empty shadow queue.
__global__ void k_probe_shadow_done(Pool pool) {
    Ctrl *c = pool.ctrl;
    c->n_shadow = 0;
    c->fetch_shadow = 0;
}

__global__ void k_film(Pool pool, double *sum, double *sum2, uint32_t *count, uint64_t t0, uint32_t n, uint32_t WH,
                       uint32_t passes) {
    uint32_t m = passes ? WH : n;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        uint32_t px = passes ? i : (uint32_t)((t0 + i) % WH);
        double s0 = sum[3 * (size_t)px], s1 = sum[3 * (size_t)px + 1], s2 = sum[3 * (size_t)px + 2];
        double q0 = sum2[3 * (size_t)px], q1 = sum2[3 * (size_t)px + 1], q2 = sum2[3 * (size_t)px + 2];
        uint32_t k = passes ? passes : 1u;
        for (uint32_t p = 0; p < k; ++p) {
            uint32_t slot = passes ? p * WH + i : i;
            float4 L = pool.L[slot];
            double a = L.x, b = L.y, cc = L.z;
            s0 += a; s1 += b; s2 += cc;
            q0 += a * a; q1 += b * b; q2 += cc * cc;
        }
        sum[3 * (size_t)px] = s0; sum[3 * (size_t)px + 1] = s1; sum[3 * (size_t)px + 2] = s2;
        sum2[3 * (size_t)px] = q0; sum2[3 * (size_t)px + 1] = q1; sum2[3 * (size_t)px + 2] = q2;
        count[px] += k;
    }
}

__global__ void k_resolve(const double *sum, const double *sum2, const uint32_t *count, uint32_t npix, float *mean,
                          float *var) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < npix; i += gridDim.x * blockDim.x) {
        double n = count[i] > 0 ? (double)count[i] : 1.0;
        for (int c = 0; c < 3; ++c) {
            double m = sum[3 * (size_t)i + c] / n;
            mean[3 * (size_t)i + c] = (float)m;
            if (var) {
                double v = sum2[3 * (size_t)i + c] / n - m * m;
                var[3 * (size_t)i + c] = (float)(fmax(v, 0.0) / fmax(n - 1.0, 1.0));
            }
        }
    }
}

// ------------------------------------------------ regeneration (Sec. 3.1.3)
// A window of n_tasks consecutive tasks (pixel samples, pass-major, from
// absolute task t0) streams through a pool of `capacity` slots. A path that
// ends is retired: its radiance goes to stage[task], indexed by the task's
// offset in the window, and its slot is emptied. Once at least `regen_min`
// slots are empty the next tasks are started in them, so the pool stays
// between half and fully occupied instead of emptying towards the end of a
// set. The film is accumulated from the staging buffer in sample order per
// pixel (k_film_range), so the result does not depend on which slot a task
// ran in or when. A refill also compacts the pool: the paths that continue
// move to slots 0 .. n_next - 1 in queue order and the new tasks take the
// slots after them, so that queue position and slot coincide again and the
// state kernels' loads and stores stay coalesced (paths end at random, so
// refilling the emptied slots in place would scatter every later access).
// Every decision (how many tasks start) is a function of counts read at
// kernel start, made identically by k_regen_gather, k_regen and
// k_regen_step_end, so none needs an atomic or a grid-wide barrier.

RT_D unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__global__ void k_regen_init(RenderParams P, Pool pool, uint64_t t0, uint32_t n_tasks, uint32_t WH,
                             uint32_t tail_threshold, unsigned long long budget_ns,
                             const volatile uint32_t *stop_word) {
    const uint32_t cap = pool.capacity;
    const uint32_t k = min(cap, n_tasks);
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < k; q += gridDim.x * blockDim.x) {
        const uint64_t t = t0 + q;
        PathState s;
        raygen(P, (uint32_t)(t % WH), (uint32_t)(t / WH), s);
        store_state(pool, q, s);
        pool.task[q] = q;
        pool.q[0][q] = q;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        Ctrl *c = pool.ctrl;
        c->n_ext = k;
        c->n_next = c->n_shadow = c->cur = 0;
        c->fetch_ext = c->fetch_shadow = c->fetch_shade = 0;
        c->split_counts = 0;
        c->n_dead = 0;
        c->n_free = cap - k;
        c->task_next = k;
        c->n_tasks = n_tasks;
        c->tail_threshold = tail_threshold;
        c->tail = (k == n_tasks && k < tail_threshold) ? 1u : 0u;
        c->deadline_ns = budget_ns ? globaltimer_ns() + budget_ns : ~0ull;
        c->stop = (stop_word && *stop_word) ? 1u : 0u;   // set before the call: only this first load runs
    }
}

// Tasks started by this step's regeneration (identical in k_regen_gather,
// k_regen and k_regen_step_end: they read the same counts, and `stop`
// changes only after all ran).
RT_HD uint32_t regen_count(const Ctrl *c, uint32_t regen_min) {
    const uint32_t left = c->n_tasks - c->task_next;
    const uint32_t empty = c->n_dead + c->n_free;
    if (c->stop || left == 0 || empty < regen_min) return 0u;
    return left < empty ? left : empty;
}

// What the regeneration kernels of one step do: retire n_dead paths; on a
// refill, move the n_move = n_next continuing paths to slots 0 .. n_move - 1
// and start n_new tasks in slots n_move .. n_move + n_new - 1.
struct RegenPlan {
    uint32_t n_dead, n_move, n_new;
};
RT_HD RegenPlan regen_plan(const Ctrl *c, uint32_t regen_min) {
    const uint32_t n_new = regen_count(c, regen_min);
    return RegenPlan{c->n_dead, n_new ? c->n_next : 0u, n_new};
}

// Counts after a step's regeneration (k_regen_step_end, without the stop
// check and the tail switch).
RT_HD void regen_advance(Ctrl *c, uint32_t regen_min) {
    const uint32_t n_dead = c->n_dead, n_free = c->n_free;
    const uint32_t n_new = regen_count(c, regen_min);
    c->n_free = n_new <= n_dead ? n_free + (n_dead - n_new) : n_free - (n_new - n_dead);
    c->task_next += n_new;
    if (n_new) ++c->regen_sets;
    c->n_ext = c->n_next + n_new;
    c->n_next = 0;
    c->n_dead = 0;
    c->cur ^= 1u;
}

// The persistent state of the paths that continue through a refill, as raw
// words (the compressed arrays keep their encoding: x, y of d and b), in
// queue order.
struct RegenScratch {
    uint4 *o, *d, *b, *L;
    uint2 *index;
    uint32_t *pixel, *task;
};

// After the shadow rays of a step: retire the paths that ended (thread j
// retires dead[j]) and, on a step that refills, copy the state of the path
// at position j of the next extension queue to scratch position j.
__global__ void k_regen_gather(Pool pool, float4 *stage, uint32_t regen_min, RegenScratch g) {
    const Ctrl *c = pool.ctrl;
    if (c->tail) return;
    const RegenPlan pl = regen_plan(c, regen_min);
    const uint32_t n_dead = pl.n_dead, n_move = pl.n_move;
    const uint32_t *next = pool.q[c->cur ^ 1u];
    const uint32_t m = max(n_dead, n_move);
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) {
        if (j < n_dead) {
            const uint32_t slot = pool.qd[j];
            stage[pool.task[slot]] = pool.L[slot];
        }
        if (j < n_move) {
            const uint32_t slot = next[j];
            g.o[j] = ((const uint4 *)pool.ray_o)[slot];
            if (pool.compact) {
                const uint2 d = pool.dir_c[slot], b = pool.beta_c[slot];
                g.d[j] = make_uint4(d.x, d.y, 0u, 0u);
                g.b[j] = make_uint4(b.x, b.y, 0u, 0u);
            } else {
                g.d[j] = ((const uint4 *)pool.ray_d)[slot];
                g.b[j] = ((const uint4 *)pool.beta)[slot];
            }
            g.L[j] = ((const uint4 *)pool.L)[slot];
            g.index[j] = pool.index[slot];
            g.pixel[j] = pool.pixel[slot];
            g.task[j] = pool.task[slot];
        }
    }
}

// On a step that refills (after k_regen_gather): the continuing paths take
// slots 0 .. n_next - 1 in queue order, tasks task_next + j start in slots
// n_next + j, and the next extension queue becomes the identity.
__global__ void k_regen(RenderParams P, Pool pool, uint64_t t0, uint32_t WH, uint32_t regen_min, RegenScratch g) {
    const Ctrl *c = pool.ctrl;
    if (c->tail) return;
    const RegenPlan pl = regen_plan(c, regen_min);
    if (pl.n_new == 0) return;
    const uint32_t n_next = pl.n_move, base = c->task_next;
    uint32_t *next = pool.q[c->cur ^ 1u];
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n_next + pl.n_new; i += gridDim.x * blockDim.x) {
        if (i < n_next) {
            ((uint4 *)pool.ray_o)[i] = g.o[i];
            if (pool.compact) {
                const uint4 d = g.d[i], b = g.b[i];
                pool.dir_c[i] = make_uint2(d.x, d.y);
                pool.beta_c[i] = make_uint2(b.x, b.y);
            } else {
                ((uint4 *)pool.ray_d)[i] = g.d[i];
                ((uint4 *)pool.beta)[i] = g.b[i];
            }
            ((uint4 *)pool.L)[i] = g.L[i];
            pool.index[i] = g.index[i];
            pool.pixel[i] = g.pixel[i];
            pool.task[i] = g.task[i];
        } else {
            const uint32_t off = base + (i - n_next);
            const uint64_t t = t0 + off;
            PathState s;
            raygen(P, (uint32_t)(t % WH), (uint32_t)(t / WH), s);
            store_state(pool, i, s);
            pool.task[i] = off;
        }
        next[i] = i;
    }
}

// End of a bounce step with regeneration: counts for the next step, the stop
// check (a host-mapped word the library's host thread sets on abort or time
// budget, and the device clock against the deadline: one read each, never a
// wait), and the switch to the megakernel tail once no task is left to start.
__global__ void k_regen_step_end(Pool pool, uint32_t regen_min, const volatile uint32_t *stop_word) {
    Ctrl *c = pool.ctrl;
    if (c->tail) return;
    regen_advance(c, regen_min);
    c->n_shadow = 0;
    c->fetch_ext = c->fetch_shadow = c->fetch_shade = 0;
    if (!c->stop && ((stop_word && *stop_word) || globaltimer_ns() >= c->deadline_ns)) c->stop = 1u;
    if ((c->stop || c->task_next == c->n_tasks) && c->n_ext < c->tail_threshold) c->tail = 1u;
}

// After the megakernel finished the tail: retire the paths it finished.
__global__ void k_regen_retire_tail(Pool pool, float4 *stage) {
    const Ctrl *c = pool.ctrl;
    if (!c->tail) return;
    const uint32_t n = c->n_ext;
    const uint32_t *queue = pool.q[c->cur];
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint32_t slot = queue[i];
        stage[pool.task[slot]] = pool.L[slot];
    }
}

// Film accumulation of tasks [t_first, t_first + n) from the staging buffer
// (stage[t - t_first]): one thread per pixel adds its samples in increasing
// sample order, the order in which iteration sets would add them.
__global__ void k_film_range(const float4 *stage, double *sum, double *sum2, uint32_t *count, uint64_t t_first,
                             uint64_t n, uint32_t WH) {
    const uint32_t r0 = (uint32_t)(t_first % WH);
    for (uint32_t px = blockIdx.x * blockDim.x + threadIdx.x; px < WH; px += gridDim.x * blockDim.x) {
        uint64_t off = (uint64_t)((px + WH - r0) % WH);   // first task of this pixel in the range
        if (off >= n) continue;
        double s0 = sum[3 * (size_t)px], s1 = sum[3 * (size_t)px + 1], s2 = sum[3 * (size_t)px + 2];
        double q0 = sum2[3 * (size_t)px], q1 = sum2[3 * (size_t)px + 1], q2 = sum2[3 * (size_t)px + 2];
        uint32_t k = 0;
        for (; off < n; off += WH, ++k) {
            const float4 L = stage[off];
            const double a = L.x, b = L.y, cc = L.z;
            s0 += a; s1 += b; s2 += cc;
            q0 += a * a; q1 += b * b; q2 += cc * cc;
        }
        sum[3 * (size_t)px] = s0; sum[3 * (size_t)px + 1] = s1; sum[3 * (size_t)px + 2] = s2;
        sum2[3 * (size_t)px] = q0; sum2[3 * (size_t)px + 1] = q1; sum2[3 * (size_t)px + 2] = q2;
        count[px] += k;
    }
}

// rays -> hits over caller-owned SoA buffers.
struct UserJob {
    rt_rays rays;
    rt_hits hits;
    RT_D Ray load(uint32_t i) const {
        return Ray{v3(__ldg(rays.ox + i), __ldg(rays.oy + i), __ldg(rays.oz + i)),
                   v3(__ldg(rays.dx + i), __ldg(rays.dy + i), __ldg(rays.dz + i)), __ldg(rays.tmin + i),
                   __ldg(rays.tmax + i)};
    }
    RT_D void store(uint32_t i, const Hit &h) const {
        hits.prim[i] = h.prim;
        if (hits.inst) hits.inst[i] = h.inst;
        hits.t[i] = h.prim == RT_MISS ? INFINITY : h.t;
        if (hits.u) hits.u[i] = h.b1;
        if (hits.v) hits.v[i] = h.b2;
    }
};

template <bool kAny, bool kTwoLevel>
__global__ void __launch_bounds__(128, kTwoLevel ? 5 : 8) k_trace_user(DevScene sc, rt_rays rays, uint32_t n, rt_hits hits,
                                                    uint32_t *scratch /* [0] fetch counter, [1] overflow */) {
    bool overflow = false;
    UserJob job{rays, hits};
    for (;;) {
        uint32_t base = warp_fetch32(&scratch[0]);
        if (base >= n) break;
        uint32_t i = base + lane_id();
        if (i >= n) continue;
        Ray r = job.load(i);
        Hit h;
        h.prim = RT_MISS; h.inst = 0; h.t = INFINITY; h.b1 = h.b2 = 0.f;
        TraceResult tr = kTwoLevel ? traverse_two_level<kAny>(sc, r, h) : traverse<kAny>(sc.nodes, sc.tris, 0u, r, h);
        overflow |= tr.overflow;
        job.store(i, h);
    }
    if (overflow) atomicOr(&scratch[1], 1u);
}

__global__ void k_sample_index(Enum en, const uint32_t *px, const uint32_t *py, const uint32_t *j, int64_t n,
                               uint64_t *out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = pixel_base_index(en, px[i], py[i]) + (uint64_t)j[i] * en.period;
}

__global__ void k_halton(Enum en, const HaltonDim *dims, const uint64_t *idx, int64_t n, int32_t ndims,
                         uint32_t *out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t x = idx[i];
        for (int32_t d = 0; d < ndims; ++d) {
            uint32_t u = d == 0 ? dim0_bits(en, x) : (d == 1 ? dim1_bits(en, x) : radical_inverse(x, dims[d]));
            out[i * ndims + d] = u;
        }
    }
}

// ------------------------------------------------------- guided rendering
constexpr uint32_t kGuideMaxRec = 8;       // vertices per path that feed training
constexpr uint32_t kRecPending = 0x80000000u;

// Network inputs of every vertex in the extension queue (zeros for misses
// and for the last vertex, which only adds emission).
// Network inputs of the paths in the extension queue (hit point, outgoing
// direction and shading normal): the fused inference kernel builds them row
// by row, reading the queue length on the device, so that no host round trip
// sizes the launch.
struct PathFeatures {
    static constexpr bool kContiguous = false;   // output rows are path slots
    RenderParams P;
    Pool pool;
    float3 lo, hi;
    __device__ uint32_t count() const { return pool.ctrl->n_ext; }
    __device__ uint32_t out_row(uint32_t row) const { return row; }
    __device__ void operator()(uint32_t i, float f[7]) const {
        const uint32_t q = pool.q[pool.ctrl->cur][i];
        PathState s = load_state(pool, q);
        float4 hv = pool.hit[q];
        Hit h;
        h.prim = __float_as_uint(hv.x); h.inst = P.sc.two_level ? pool.hit_inst[q] : 0u;
        h.t = hv.y; h.b1 = hv.z; h.b2 = hv.w;
        if (h.prim != RT_MISS && s.depth <= P.max_depth) {
            Vertex vx;
            setup_vertex(P.sc, s, h, vx);
            guide_features(vx.x, vx.wo, vx.ns, lo, hi, f);
        }
    }
};

__global__ void __launch_bounds__(kMiThreads, 1) k_guide_mlp_paths(MlpWeights w, PathFeatures pf, __nv_bfloat16 *raw,
                                                            uint32_t *err) {
    mlp_infer_tiles(w, pf, raw, err);
}

// Shading with the guided mixture. Every rec_stride-th path of the set (at
// most `rec_paths` of them, spread over its pixels and passes) records, at
// its vertices 1..rec_depth (at most kGuideMaxRec),
// (features, wi, throughput) at every continuing vertex and, at the next
// vertex, the radiance gathered so far, so that the radiance returned
// through wi is L_end - L_snapshot; they are the training samples. Record
// slot of path q: q / rec_stride.
__device__ __forceinline__ bool recording_path(uint32_t q, uint32_t rec_stride, uint32_t rec_paths) {
    return q % rec_stride == 0u && q / rec_stride < rec_paths;
}

// Threads per block of the guided shading kernels: each keeps its decoded
// mixture in the block's shared memory (24 KB).
constexpr uint32_t kGuidedShadeThreads = 128;

template <bool kLb>
__global__ void __launch_bounds__(kGuidedShadeThreads, 6) k_shade_guided(RenderParams P, Pool pool, const __nv_bfloat16 *raw, float alpha,
                                                      float4 *rec, uint32_t rec_stride, uint32_t rec_paths,
                                                      uint32_t rec_depth, float3 lo, float3 hi) {
    Ctrl *c = pool.ctrl;
    const uint32_t n = c->n_ext;
    const uint32_t cur = c->cur;
    const uint32_t *queue = pool.q[cur];
    uint32_t *next = pool.q[cur ^ 1u];
    __shared__ float s_mix[kMixFields * kGuideLobes * kGuidedShadeThreads];
    const MixtureStrided mix{s_mix + threadIdx.x, kGuidedShadeThreads};
    for (;;) {
        uint32_t base = warp_fetch32(&c->fetch_shade);
        if (base >= n) break;
        uint32_t i = base + lane_id();
        bool valid = i < n;
        uint32_t q = 0;
        int r = 0;
        if (valid) {
            q = queue[i];
            PathState s = load_state(pool, q);
            const bool recording = recording_path(q, rec_stride, rec_paths);
            const uint32_t slot = q / rec_stride;
            uint32_t nr = recording ? pool.nrec[q] : 0u;
            if (nr & kRecPending) {
                nr &= ~kRecPending;
                float4 *R = rec + ((size_t)slot * kGuideMaxRec + (nr - 1)) * 4;
                R[3] = make_float4(R[3].x, s.L.x, s.L.y, s.L.z);
                pool.nrec[q] = nr;
            }
            float4 hv = pool.hit[q];
            Hit h;
            h.prim = __float_as_uint(hv.x); h.inst = P.sc.two_level ? pool.hit_inst[q] : 0u;
            h.t = hv.y; h.b1 = hv.z; h.b2 = hv.w;
            ShadowRay sh;
            GuideRecord gr;
            const uint32_t v = s.depth;
            const bool want = recording && v <= rec_depth;
            r = shade<kLb, MixtureStrided>(P, s, h, sh, raw ? raw + (size_t)kGuideOut * i : nullptr, alpha,
                                           want ? &gr : nullptr, lo, hi, mix);
            pool.L[q] = make_float4(s.L.x, s.L.y, s.L.z, __uint_as_float(s.prev_n));
            if (r & 1) {
                pool.ray_o[q] = make_float4(s.o.x, s.o.y, s.o.z, __uint_as_float(s.prev_cell));
                st_dir(pool, q, s.d, s.prev_pdf);
                st_beta(pool, q, s.beta, s.depth);
                if (want) {
                    float4 *R = rec + ((size_t)slot * kGuideMaxRec + (v - 1)) * 4;
                    R[0] = make_float4(gr.feat[0], gr.feat[1], gr.feat[2], gr.feat[3]);
                    R[1] = make_float4(gr.feat[4], gr.feat[5], gr.feat[6], gr.wi.x);
                    R[2] = make_float4(gr.wi.y, gr.wi.z, gr.beta.x, gr.beta.y);
                    R[3] = make_float4(gr.beta.z, 0.f, 0.f, 0.f);
                    pool.nrec[q] = v | kRecPending;
                }
            }
            if (r & 2) {
                pool.sh_o[q] = make_float4(sh.o.x, sh.o.y, sh.o.z, sh.tmax);
                st_shd(pool, q, sh.d);
                st_shc(pool, q, sh.contrib);
            }
        }
        warp_append(next, &c->n_next, valid && (r & 1), q);
        warp_append(pool.qs, &c->n_shadow, valid && (r & 2), q);
    }
}

// Training samples of finished paths: weight = luminance of the radiance that
// came back through wi divided by the throughput on arrival, i.e. the
// sampled f cos Li / p of that vertex. The first `keep` samples are kept.
__global__ void k_guide_collect(Pool pool, uint32_t n, const float4 *rec, uint32_t rec_stride, float *tr_feat,
                                float *tr_wi, float *tr_w, uint32_t rec_paths, uint32_t keep) {
    Ctrl *c = pool.ctrl;
    const uint32_t slots = min(rec_paths, (n + rec_stride - 1) / rec_stride);
    for (uint32_t k0 = blockIdx.x * blockDim.x + threadIdx.x; k0 < slots; k0 += gridDim.x * blockDim.x) {
        const uint32_t q = k0 * rec_stride;
        uint32_t nr = pool.nrec[q];
        uint32_t complete = (nr & kRecPending) ? (nr & ~kRecPending) - 1 : nr;
        float4 L = pool.L[q];
        for (uint32_t k = 0; k < complete; ++k) {
            const float4 *R = rec + ((size_t)k0 * kGuideMaxRec + k) * 4;
            float4 r0 = R[0], r1 = R[1], r2 = R[2], r3 = R[3];
            float bx = r2.z, by = r2.w, bz = r3.x;
            float ax = bx > 0.f ? fmaxf(L.x - r3.y, 0.f) / bx : 0.f;
            float ay = by > 0.f ? fmaxf(L.y - r3.z, 0.f) / by : 0.f;
            float az = bz > 0.f ? fmaxf(L.z - r3.w, 0.f) / bz : 0.f;
            float w = lum(v3(ax, ay, az));
            if (!(w > 0.f) || !isfinite(w)) continue;
            uint32_t idx = atomicAdd(&c->n_train, 1u);
            if (idx >= keep) continue;
            float f[7] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z};
            for (int j = 0; j < 7; ++j) tr_feat[7 * (size_t)idx + j] = f[j];
            tr_wi[3 * (size_t)idx] = r1.w;
            tr_wi[3 * (size_t)idx + 1] = r2.x;
            tr_wi[3 * (size_t)idx + 2] = r2.y;
            tr_w[idx] = w;
        }
    }
}

// ---------------------------------------------------------- host helpers
int sm_count() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

// Persistent traversal kernels: one wave of resident blocks.
template <class K>
int grid_persistent(K kernel, int block, size_t smem) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, smem);
    if (per_sm < 1) per_sm = 1;
    return sm_count() * per_sm;
}

inline size_t stack_smem(int block) { return (size_t)kShStack * block * sizeof(uint2); }

// The one-ray-per-thread traversal kernels of one variant (instrumented or
// not, shared-memory stack or not, one level or two) and their persistent
// grids, sized by each kernel's own occupancy.
using TraceFn = void (*)(DevScene, Pool, const uint32_t *);
struct TraceKernels {
    TraceFn ext, shadow;
    int grid_ext, grid_shadow;
    size_t smem;
};

template <bool kCount, bool kSmem, bool kTwo, bool kPostpone = false, bool kNear = false>
TraceKernels trace_kernels_of(int block) {
    TraceKernels k;
    k.ext = k_trace_ext_simple<kCount, kSmem, kTwo, kPostpone, kNear>;
    k.shadow = k_trace_shadow_simple<kCount, kSmem, kTwo, kPostpone>;
    k.smem = kSmem ? (size_t)kSharedEntries * block * sizeof(uint2) : 0;
    k.grid_ext = grid_persistent(k.ext, block, k.smem);
    k.grid_shadow = grid_persistent(k.shadow, block, k.smem);
    return k;
}

template <bool kCount>
TraceKernels refill_kernels(int block) {
    TraceKernels k;
    k.ext = k_trace_refill<false, kCount>;
    k.shadow = k_trace_refill<true, kCount>;
    k.smem = 0;
    k.grid_ext = grid_persistent(k.ext, block, 0);
    k.grid_shadow = grid_persistent(k.shadow, block, 0);
    return k;
}

// variant: 0 (default) closest hit one-shot per ray, shadow rays with lane
// refill (any-hit rays end at very different times, and an occlusion answer
// does not depend on the order of the traversal); 2 both one-shot with the
// stack top in shared memory; 3 both with lane refill; 4 both one-shot;
// 6 closest hit one-shot with postponed triangle tests, shadow rays as 0;
// 7 both one-shot with postponed triangle tests; 8 closest hit one-shot with
// one stack entry per child, nearest child next and far entries dropped on
// pop (traverse_near), shadow rays as 0.
// Two-level scenes always use the one-shot kernels with a thread-local stack.
inline TraceKernels trace_kernels(bool count, int variant, bool two_level, int block) {
    if (two_level) return count ? trace_kernels_of<true, false, true>(block) : trace_kernels_of<false, false, true>(block);
    if (variant == 3) return count ? refill_kernels<true>(block) : refill_kernels<false>(block);
    if (variant == 7)
        return count ? trace_kernels_of<true, false, false, true>(block) : trace_kernels_of<false, false, false, true>(block);
    if (variant == 0 || variant == 6 || variant == 8) {
        TraceKernels k = variant == 6
                             ? (count ? trace_kernels_of<true, false, false, true>(block)
                                      : trace_kernels_of<false, false, false, true>(block))
                         : variant == 8
                             ? (count ? trace_kernels_of<true, false, false, false, true>(block)
                                      : trace_kernels_of<false, false, false, false, true>(block))
                             : (count ? trace_kernels_of<true, false, false>(block) : trace_kernels_of<false, false, false>(block));
        const TraceKernels r = count ? refill_kernels<true>(block) : refill_kernels<false>(block);
        k.shadow = r.shadow;
        k.grid_shadow = r.grid_shadow;
        return k;
    }
    const bool smem_stack = variant == 2;
    if (smem_stack)
        return count ? trace_kernels_of<true, true, false>(block) : trace_kernels_of<false, true, false>(block);
    return count ? trace_kernels_of<true, false, false>(block) : trace_kernels_of<false, false, false>(block);
}

// Whether the closest-hit kernel of `variant` (trace_kernels above) fills
// Pool::split: the one-ray-per-thread single-level kernels do (variants 0,
// 2, 4, 6, 7, 8), the lane-refill and persistent ones do not; two-level
// scenes keep one queue (their kernel runs at 102 registers, and the split
// measured slower on the instanced many-light field: 639.7 against 661.8
// Mpaths/s).
inline bool variant_splits(int variant, bool two_level) {
    return !two_level && !(variant == 1 || variant == 3 || variant == 5);
}

// Threads per block of the state kernels: 0 (128) or a multiple of 32 up to
// the kernels' launch bound of 128.
inline bool valid_block(uint32_t b) { return b == 0 || (b % 32 == 0 && b <= 128); }

template <class K>
int grid_for(K kernel, int block, int64_t work) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, 0);
    if (per_sm < 1) per_sm = 1;
    int64_t full = (int64_t)sm_count() * per_sm;
    int64_t need = (work + block - 1) / block;
    return (int)std::max<int64_t>(1, std::min(full, need));
}

struct PoolAlloc {
    Pool view{};
    // regeneration arrays (task per slot, dead and free slot lists): set in
    // the view only by the scheduler that uses them
    uint32_t *task = nullptr, *qd = nullptr;
    uint32_t *split = nullptr;   // Pool::split storage, set in the view by the renders that use it
    void *block = nullptr;
    uint32_t capacity = 0;
    bool compact = false;   // compressed layout of the direction, throughput and shadow arrays
    ~PoolAlloc() {
        if (block) cudaFree(block);
    }
};

// Device bytes of one path's state in the pool (eight float4 arrays, the
// sequence index, pixel, instance of the hit, four queue entries (the two
// extension queues, the shadow queue, the hit/miss-split shading queue) and
// the regeneration scheduler's task and dead entries), and of the scratch copy
// of a continuing path that a refill moves (regeneration with a pool smaller
// than the request).
constexpr size_t kPoolBytesPerPath = 8 * sizeof(float4) + sizeof(uint2) + 4 + 4 + 4 * 4 + 2 * 4;
constexpr size_t kRegenScratchBytesPerPath = 4 * sizeof(uint4) + sizeof(uint2) + 4 + 4;

// Pool capacity when the caller leaves it to the library: every requested
// path at once when that fits, up to 2^27 paths (about 21 GB of state) and a
// quarter of the free device memory. Large iteration sets pay: the few long
// paths at the end of a set keep the GPU partly idle, once per set.
uint32_t default_capacity(uint64_t paths) {
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) free_b = (size_t)1 << 30;
    const uint64_t by_mem = (uint64_t)(free_b / 4 / kPoolBytesPerPath);
    uint64_t c = std::min<uint64_t>({paths, (uint64_t)1 << 27, by_mem});
    // a pool that is refilled also holds the scratch copy of its continuing paths
    if (c < paths) c = std::min<uint64_t>(c, free_b / 4 / (kPoolBytesPerPath + kRegenScratchBytesPerPath));
    return (uint32_t)std::max<uint64_t>(c, 32u);
}

rt_status ensure_pool(PoolAlloc &pa, uint32_t capacity, bool compact = false) {
    if (pa.block && pa.capacity >= capacity && pa.compact == compact) return RT_OK;
    if (pa.block) { cudaFree(pa.block); pa.block = nullptr; }
    size_t P = capacity;
    size_t f4 = P * sizeof(float4);
    // four float4 arrays always (origin, radiance, hit, shadow origin); four
    // more, or their compressed forms (8 + 8 + 4 + 8 bytes per path)
    size_t bytes = 4 * f4 + (compact ? P * 28 + 4 * 256 : 4 * f4) + P * sizeof(uint2) + P * 4 /*pixel*/ +
                   P * 4 /*hit_inst*/ + 4 * P * 4 /*queues*/ + 2 * P * 4 /*regeneration*/ + 64 * 256;
    cudaError_t e = cudaMalloc(&pa.block, bytes);
    if (e != cudaSuccess) { set_error("path-state pool allocation failed"); return RT_OOM; }
    char *p = (char *)pa.block;
    auto take = [&](size_t b) { char *r = p; p += (b + 255) / 256 * 256; return r; };
    Pool &v = pa.view;
    v = Pool{};
    v.ctrl = (Ctrl *)take(sizeof(Ctrl));
    v.ray_o = (float4 *)take(f4); v.L = (float4 *)take(f4); v.hit = (float4 *)take(f4); v.sh_o = (float4 *)take(f4);
    if (compact) {
        v.dir_c = (uint2 *)take(P * 8); v.beta_c = (uint2 *)take(P * 8);
        v.shd_c = (uint32_t *)take(P * 4); v.shc_c = (uint2 *)take(P * 8);
        v.compact = 1;
    } else {
        v.ray_d = (float4 *)take(f4); v.beta = (float4 *)take(f4); v.sh_d = (float4 *)take(f4); v.sh_c = (float4 *)take(f4);
    }
    pa.compact = compact;
    v.index = (uint2 *)take(P * sizeof(uint2));
    v.pixel = (uint32_t *)take(P * 4);
    v.hit_inst = (uint32_t *)take(P * 4);
    v.q[0] = (uint32_t *)take(P * 4); v.q[1] = (uint32_t *)take(P * 4); v.qs = (uint32_t *)take(P * 4);
    pa.task = (uint32_t *)take(P * 4); pa.qd = (uint32_t *)take(P * 4);
    pa.split = (uint32_t *)take(P * 4);
    v.capacity = capacity;
    pa.capacity = capacity;
    if ((size_t)(p - (char *)pa.block) > bytes) { set_error("pool layout overflow"); return RT_CUDA_ERROR; }
    return RT_OK;
}

}  // namespace rtg

using namespace rtg;

// Per-film render resources (path-state pool, dimension table, pinned ctrl).
struct RenderCache {
    PoolAlloc pool;
    HaltonDim *dims = nullptr;
    uint64_t dims_seed = ~0ull;
    int dims_n = 0;
    Ctrl *host_ctrl = nullptr;
    // sorted queues (A/B options)
    uint32_t *sort_hist = nullptr, *sort_buf[2] = {nullptr, nullptr};
    uint32_t sort_cap = 0, sort_nkeys = 0;
    // regeneration: radiance per task of the window, host-mapped stop word
    float4 *stage = nullptr;
    uint64_t stage_cap = 0;
    void *gscr = nullptr;   // RegenScratch storage for gscr_cap paths
    uint32_t gscr_cap = 0;
    uint32_t *stop_host = nullptr, *stop_dev = nullptr;
    Ctrl *ctrl_ring = nullptr;   // pinned copies of the control block, one per chunk in flight (x2 half-pools)
    cudaEvent_t chunk_ev[4] = {nullptr, nullptr, nullptr, nullptr};
    // regeneration as two half-pools: the second half-pool's control block
    // and stream, and a fork / join event
    Ctrl *ctrl2 = nullptr;
    cudaStream_t st2 = nullptr;
    cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
    // guided rendering
    uint32_t gcap = 0, gbatch = 0, grec_paths = 0;   // guided buffers: network rows, training samples, record paths
    __nv_bfloat16 *gfeat = nullptr;   // network outputs [cap][40] (BF16) of one bounce step
    float *tr_feat = nullptr, *tr_wi = nullptr, *tr_w = nullptr;
    float4 *grec = nullptr;
    uint32_t *gnrec = nullptr;
    ~RenderCache() {
        if (dims) cudaFree(dims);
        if (host_ctrl) cudaFreeHost(host_ctrl);
        if (stage) cudaFree(stage);
        if (gscr) cudaFree(gscr);
        if (stop_host) cudaFreeHost(stop_host);
        if (ctrl_ring) cudaFreeHost(ctrl_ring);
        for (cudaEvent_t e : chunk_ev)
            if (e) cudaEventDestroy(e);
        if (ctrl2) cudaFree(ctrl2);
        if (st2) cudaStreamDestroy(st2);
        if (fork_ev) cudaEventDestroy(fork_ev);
        if (join_ev) cudaEventDestroy(join_ev);
        for (void *p : {(void *)gfeat, (void *)tr_feat, (void *)tr_wi, (void *)tr_w, (void *)grec, (void *)gnrec,
                        (void *)sort_hist, (void *)sort_buf[0], (void *)sort_buf[1]})
            if (p) cudaFree(p);
    }
};

// The set sizes and buffer sizes of a guided render (host arithmetic, also
// run by the host test hook). While the proposal is young (fewer than its
// warm-up training steps) a set holds at most min(wsb, 16) batches of paths
// and up to wsb training steps follow, each on its own batch of the set's
// samples, so that it learns fast (until the first step the proposal is BSDF
// sampling alone). Later a set holds up to 64 batches of paths (a caller's
// max_paths_in_flight sets this size instead) and one step follows per 16
// batches rendered, so that the per-set launches, their drains and the host
// round trip are spread over more paths at the same training rate. Training
// records come from the guided vertices 1..gdepth only (the network is asked
// about no other); a young set records from enough paths for its samples at
// min(4, rec_depth) samples per path, a later one from `batch` paths.
struct GuidedPlan {
    uint32_t cap;          // paths per set after the warm-up
    uint32_t cap_young;    // paths per warm-up set
    uint32_t per_step;     // paths rendered per training step after the warm-up
    uint32_t gdepth;       // last guided vertex
    uint32_t rec_depth;    // last recorded vertex
    uint32_t keep_young;   // samples kept after a warm-up set
    uint32_t rec_young;    // recording paths of a warm-up set
    uint32_t rec_alloc;    // recording paths the record buffer holds
    uint32_t keep_alloc;   // samples the training buffers hold
};
struct GuidedSet {
    uint32_t keep;         // samples kept after this set
    uint32_t rec_paths;    // recording paths (every rec_stride-th path)
    uint32_t rec_stride;
    uint32_t set_steps;    // training steps due after a trained-phase set
};
// batch <= 2^24 (checked by the caller); cap = the pool's paths per set
// before the guided limit; fixed_pool: the caller set max_paths_in_flight.
static GuidedPlan guided_plan(uint32_t batch, uint32_t wsb, uint32_t guide_depth, uint32_t max_depth, uint32_t cap,
                              bool fixed_pool) {
    GuidedPlan g;
    wsb = std::max(1u, wsb);
    g.per_step = 16u * std::max(batch, 32u);
    g.cap = fixed_pool ? cap : (uint32_t)std::min<uint64_t>(cap, 64ull * std::max(batch, 32u));
    g.cap_young = (uint32_t)std::min<uint64_t>({(uint64_t)g.cap, (uint64_t)g.per_step,
                                                (uint64_t)std::max(batch, 32u) * wsb});
    g.gdepth = std::min(guide_depth, max_depth);
    g.rec_depth = std::min(g.gdepth, kGuideMaxRec);
    g.keep_young = (uint32_t)std::min<uint64_t>((uint64_t)batch * wsb, 1ull << 28);
    g.rec_young = std::max(1u, std::min(g.cap_young, g.keep_young / std::max(1u, std::min(4u, g.rec_depth))));
    g.rec_alloc = std::max(batch, g.rec_young);
    g.keep_alloc = std::max(4u * batch, g.keep_young);
    return g;
}
static GuidedSet guided_set(const GuidedPlan &g, uint32_t batch, uint32_t n, bool young) {
    GuidedSet e;
    e.set_steps = std::min(4u, std::max(1u, n / g.per_step));
    e.keep = young ? std::max(batch, g.keep_young) : e.set_steps * batch;
    e.rec_paths = young ? std::max(batch, g.rec_young) : batch;
    e.rec_stride = std::max(1u, n / e.rec_paths);
    return e;
}

// Guided-rendering buffers: network rows for `cap` paths, training records
// of `rec_paths` paths and `samples` training samples.
static rt_status ensure_guided(RenderCache *rc, uint32_t cap, uint32_t rec_paths, uint32_t samples) {
    if (rc->gcap >= cap && rc->grec_paths >= rec_paths && rc->gbatch >= samples) return RT_OK;
    cap = std::max(cap, rc->gcap);
    rec_paths = std::max(rec_paths, rc->grec_paths);
    samples = std::max(samples, rc->gbatch);
    for (void *p : {(void *)rc->gfeat, (void *)rc->tr_feat, (void *)rc->tr_wi, (void *)rc->tr_w, (void *)rc->grec,
                    (void *)rc->gnrec})
        if (p) cudaFree(p);
    rc->gfeat = nullptr;
    rc->tr_feat = rc->tr_wi = rc->tr_w = nullptr;
    rc->grec = nullptr;
    rc->gnrec = nullptr;
    if (cudaMalloc(&rc->gfeat, (size_t)cap * kGuideOut * sizeof(__nv_bfloat16)) != cudaSuccess ||
        cudaMalloc(&rc->grec, (size_t)rec_paths * kGuideMaxRec * 4 * sizeof(float4)) != cudaSuccess ||
        cudaMalloc(&rc->gnrec, (size_t)cap * 4) != cudaSuccess ||
        cudaMalloc(&rc->tr_feat, (size_t)samples * 7 * 4) != cudaSuccess ||
        cudaMalloc(&rc->tr_wi, (size_t)samples * 3 * 4) != cudaSuccess ||
        cudaMalloc(&rc->tr_w, (size_t)samples * 4) != cudaSuccess) {
        set_error("guided rendering: out of device memory");
        return RT_OOM;
    }
    rc->gcap = cap;
    rc->grec_paths = rec_paths;
    rc->gbatch = samples;
    return RT_OK;
}

static RenderCache *cache_of(rt_film *f);

// Per (device, stream) scratch of rt_trace: 8 bytes of device memory and a
// pinned word, allocated on first use and kept until the process exits.
struct TraceScratch {
    uint32_t *dev = nullptr;
    uint32_t *host = nullptr;
};
static rt_status trace_scratch(cudaStream_t st, TraceScratch **out) {
    static std::mutex mu;
    static std::map<std::pair<int, cudaStream_t>, TraceScratch> table;
    int dev = 0;
    RT_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(mu);
    TraceScratch &ts = table[{dev, st}];
    if (!ts.dev) {
        RT_CUDA_TRY(cudaMalloc(&ts.dev, 2 * sizeof(uint32_t)));
        RT_CUDA_TRY(cudaMallocHost(&ts.host, sizeof(uint32_t)));
    }
    *out = &ts;
    return RT_OK;
}

extern "C" rt_status rt_trace(const rt_scene *s, const rt_rays *rays, int64_t n, const rt_hits *hits,
                              int32_t any_hit, void *stream) {
    if (!s || !rays || !hits || n < 0) { set_error("rt_trace: invalid argument"); return RT_INVALID_ARG; }
    if (s->host_only) { set_error("rt_trace: scene has no device copy"); return RT_INVALID_ARG; }
    if (n == 0) return RT_OK;
    if (!hits->prim || !hits->t || !rays->ox || !rays->dx || !rays->tmin || !rays->tmax) {
        set_error("rt_trace: null ray or hit pointer");
        return RT_INVALID_ARG;
    }
    if (n > 0xFFFFFFFFll) { set_error("rt_trace: at most 2^32 - 1 rays per call"); return RT_INVALID_ARG; }
    // Scratch of this stream (ray fetch counter, overflow flag) and a pinned
    // word for the overflow flag: calls on one stream run one after another,
    // so they can share it; calls in flight on different streams (or host
    // threads) never share a counter. The overflow flag comes back to the
    // host, so the call waits for its kernel before it returns.
    cudaStream_t st = (cudaStream_t)stream;
    TraceScratch *ts = nullptr;
    rt_status rs0 = trace_scratch(st, &ts);
    if (rs0 != RT_OK) return rs0;
    RT_CUDA_TRY(cudaMemsetAsync(ts->dev, 0, 2 * sizeof(uint32_t), st));
    const int gb = 128;
    using UserFn = void (*)(DevScene, rt_rays, uint32_t, rt_hits, uint32_t *);
    const UserFn fn = any_hit ? (s->dev.two_level ? (UserFn)k_trace_user<true, true> : (UserFn)k_trace_user<true, false>)
                              : (s->dev.two_level ? (UserFn)k_trace_user<false, true> : (UserFn)k_trace_user<false, false>);
    const int g = grid_persistent(fn, gb, 0);
    fn<<<g, gb, 0, st>>>(s->dev, *rays, (uint32_t)n, *hits, ts->dev);
    RT_CUDA_TRY(cudaGetLastError());
    RT_CUDA_TRY(cudaMemcpyAsync(ts->host, ts->dev + 1, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    RT_CUDA_TRY(cudaStreamSynchronize(st));
    if (*ts->host) {
        set_error("rt_trace: BVH traversal stack overflow (hits of the affected rays are incomplete)");
        return RT_STACK_OVERFLOW;
    }
    return RT_OK;
}

extern "C" rt_status rt_film_create(uint32_t W, uint32_t H, rt_film **out) {
    if (!out || W == 0 || H == 0 || (uint64_t)W * H > (1ull << 31)) {
        set_error("rt_film_create: invalid size");
        return RT_INVALID_ARG;
    }
    rt_film *f = new rt_film();
    f->W = W; f->H = H;
    size_t npix = (size_t)W * H;
    if (cudaMalloc(&f->sum, npix * 3 * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&f->sum2, npix * 3 * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&f->count, npix * sizeof(uint32_t)) != cudaSuccess) {
        rt_film_destroy(f);
        set_error("rt_film_create: out of device memory");
        return RT_OOM;
    }
    cudaMemset(f->sum, 0, npix * 3 * sizeof(double));
    cudaMemset(f->sum2, 0, npix * 3 * sizeof(double));
    cudaMemset(f->count, 0, npix * sizeof(uint32_t));
    RT_CUDA_TRY(cudaDeviceSynchronize());
    *out = f;
    return RT_OK;
}

extern "C" rt_status rt_film_destroy(rt_film *f) {
    if (!f) return RT_OK;
    cudaFree(f->sum); cudaFree(f->sum2); cudaFree(f->count);
    delete (RenderCache *)f->cache;
    delete f;
    return RT_OK;
}

extern "C" rt_status rt_film_clear(rt_film *f, void *stream) {
    if (!f) { set_error("rt_film_clear: null film"); return RT_INVALID_ARG; }
    size_t npix = (size_t)f->W * f->H;
    cudaStream_t st = (cudaStream_t)stream;
    RT_CUDA_TRY(cudaMemsetAsync(f->sum, 0, npix * 3 * sizeof(double), st));
    RT_CUDA_TRY(cudaMemsetAsync(f->sum2, 0, npix * 3 * sizeof(double), st));
    RT_CUDA_TRY(cudaMemsetAsync(f->count, 0, npix * sizeof(uint32_t), st));
    f->next_task = 0;
    return RT_OK;
}

extern "C" rt_status rt_film_next_iteration(const rt_film *f, uint32_t *next) {
    if (!f || !next) { set_error("rt_film_next_iteration: null argument"); return RT_INVALID_ARG; }
    *next = (uint32_t)(f->next_task / ((uint64_t)f->W * f->H));
    return RT_OK;
}

extern "C" rt_status rt_film_seek(rt_film *f, uint32_t next) {
    if (!f) { set_error("rt_film_seek: null film"); return RT_INVALID_ARG; }
    f->next_task = (uint64_t)next * f->W * f->H;
    return RT_OK;
}

extern "C" rt_status rt_film_buffers(const rt_film *f, double **sum, double **sum2, uint32_t **count) {
    if (!f) { set_error("rt_film_buffers: null film"); return RT_INVALID_ARG; }
    if (sum) *sum = f->sum;
    if (sum2) *sum2 = f->sum2;
    if (count) *count = f->count;
    return RT_OK;
}

extern "C" rt_status rt_film_resolve(const rt_film *f, float *mean, float *var, void *stream) {
    if (!f || !mean) { set_error("rt_film_resolve: null argument"); return RT_INVALID_ARG; }
    uint32_t npix = f->W * f->H;
    int g = grid_for(k_resolve, 256, npix);
    k_resolve<<<g, 256, 0, (cudaStream_t)stream>>>(f->sum, f->sum2, f->count, npix, mean, var);
    RT_CUDA_TRY(cudaGetLastError());
    return RT_OK;
}

static RenderCache *cache_of(rt_film *f) {
    if (!f->cache) f->cache = new RenderCache();
    return (RenderCache *)f->cache;
}

// rt_render with regeneration (Sec. 3.1.3): windows of consecutive tasks
// stream through the pool; bounce steps are issued in chunks and the host
// reads the control block of the chunk before the last one (so one chunk is
// always queued behind the running one) to see when the window is done.
// While it waits it relays the caller's abort flag and the time budget to a
// host-mapped word that k_regen_step_end reads; the device also compares its
// own clock with the deadline. Once stopped, no task starts, the paths in
// flight finish, and the film receives the contiguous range of tasks that
// completed (possibly ending inside an iteration; the next call continues
// there).
// Slots [off, off + n) of a pool as a pool of their own, with its own
// control block (every per-slot array offset, the queues included).
static Pool sub_pool(const Pool &p, uint32_t off, uint32_t n, Ctrl *ctrl) {
    Pool v = p;
    auto sh = [&](auto *&a) {
        if (a) a += off;
    };
    sh(v.ray_o); sh(v.ray_d); sh(v.beta); sh(v.L); sh(v.index); sh(v.pixel); sh(v.hit); sh(v.hit_inst);
    sh(v.sh_o); sh(v.sh_d); sh(v.sh_c); sh(v.q[0]); sh(v.q[1]); sh(v.qs); sh(v.nrec); sh(v.task); sh(v.qd);
    sh(v.dir_c); sh(v.beta_c); sh(v.shd_c); sh(v.shc_c); sh(v.split);
    v.ctrl = ctrl;
    v.capacity = n;
    return v;
}
static RegenScratch sub_scratch(const RegenScratch &g, uint32_t off) {
    RegenScratch v = g;
    if (!v.o) return v;
    v.o += off; v.d += off; v.b += off; v.L += off; v.index += off; v.pixel += off; v.task += off;
    return v;
}

static rt_status render_regen(const rt_scene *s, const rt_camera *cam, uint32_t spp, uint32_t max_depth,
                              rt_film *film, const rt_render_opts &o, cudaStream_t st, RenderCache *rc,
                              uint32_t cap) {
    const uint32_t W = cam->width, H = cam->height;
    const uint64_t WH = (uint64_t)W * H;
    RenderParams P;
    P.sc = s->dev;
    P.cam = make_camera(*cam);
    P.en = make_enum(W, H);
    P.dims = rc->dims;
    P.max_depth = max_depth;
    P.sigma = o.filter_sigma == 0.f ? 0.5f : o.filter_sigma;
    P.mis_mode = o.mis_mode;
    P.rr = o.rr_enable;
    const uint32_t tail = o.tail_threshold ? o.tail_threshold : 8192u;
    const float frac = o.regen_fraction > 0.f ? o.regen_fraction : 0.5f;
    const uint32_t regen_min = std::max<uint32_t>(1u, (uint32_t)std::min<double>((double)cap, std::ceil(frac * cap)));
    Pool pool = rc->pool.view;
    pool.task = rc->pool.task;
    pool.qd = rc->pool.qd;
    pool.capacity = cap;   // the allocation may be larger (kept from an earlier call)
    // staging window: the request, at most 2^30 tasks and a quarter of the
    // free device memory (16 bytes per task)
    const uint64_t t_begin = film->next_task, t_end = (film->next_task / WH + (uint64_t)spp) * WH;
    uint64_t win = std::min<uint64_t>(t_end - t_begin, (uint64_t)1 << 30);
    {
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess && rc->stage_cap < win)
            win = std::max<uint64_t>(std::min<uint64_t>(win, free_b / 4 / sizeof(float4)), std::min<uint64_t>(win, cap));
    }
    if (rc->stage_cap < win) {
        if (rc->stage) cudaFree(rc->stage);
        rc->stage = nullptr;
        rc->stage_cap = 0;
        if (cudaMalloc(&rc->stage, win * sizeof(float4)) != cudaSuccess) {
            set_error("rt_render: staging buffer allocation failed");
            return RT_OOM;
        }
        rc->stage_cap = win;
    }
    // scratch of the continuing paths that a refill moves (only a window
    // larger than the pool refills)
    RegenScratch gs{};
    if (win > cap) {
        if (rc->gscr_cap < cap) {
            if (rc->gscr) cudaFree(rc->gscr);
            rc->gscr = nullptr;
            rc->gscr_cap = 0;
            if (cudaMalloc(&rc->gscr, (size_t)cap * kRegenScratchBytesPerPath + 8 * 256) != cudaSuccess) {
                set_error("rt_render: regeneration scratch allocation failed");
                return RT_OOM;
            }
            rc->gscr_cap = cap;
        }
        char *g = (char *)rc->gscr;
        const size_t C = rc->gscr_cap;
        auto take = [&](size_t b) { char *r = g; g += (b + 255) / 256 * 256; return r; };
        gs.o = (uint4 *)take(C * 16); gs.d = (uint4 *)take(C * 16); gs.b = (uint4 *)take(C * 16);
        gs.L = (uint4 *)take(C * 16); gs.index = (uint2 *)take(C * 8);
        gs.pixel = (uint32_t *)take(C * 4); gs.task = (uint32_t *)take(C * 4);
    }
    if (!rc->stop_host) {
        RT_CUDA_TRY(cudaHostAlloc(&rc->stop_host, sizeof(uint32_t), cudaHostAllocMapped));
        RT_CUDA_TRY(cudaHostGetDevicePointer((void **)&rc->stop_dev, rc->stop_host, 0));
    }
    if (!rc->ctrl_ring) RT_CUDA_TRY(cudaMallocHost(&rc->ctrl_ring, 4 * sizeof(Ctrl)));
    for (cudaEvent_t &e : rc->chunk_ev)
        if (!e) RT_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    *(volatile uint32_t *)rc->stop_host = 0u;

    const int gb = o.block_size ? (int)o.block_size : 128;
    const bool prof = o.profile >= 1, count = o.profile >= 2;
    const int variant = (o.trace_kernel == 1 || o.trace_kernel == 5) ? 0 : o.trace_kernel;
    const TraceKernels tk = trace_kernels(count, variant, s->dev.two_level, gb);
    pool.split = variant_splits(variant, s->dev.two_level) ? rc->pool.split : nullptr;
    const int g_shade = grid_persistent(k_shade<true>, gb, 0);
    const int g_regen = grid_for(k_regen, 256, cap);
    const int g_init = grid_for(k_regen_init, 256, cap);
    const int g_mega = grid_for(k_megakernel, gb, cap);
    const uint32_t nmat = s->num_materials;
    const uint32_t nkeys_mat = nmat + 1, nkeys_ray = 8u * 512u;
    const int g_hist = grid_for(k_sort_scatter<RayKey>, 256, cap);
    if ((o.sort_by_material || o.sort_rays) && (rc->sort_cap < cap || rc->sort_nkeys < std::max(nkeys_mat, nkeys_ray))) {
        for (void *p : {(void *)rc->sort_hist, (void *)rc->sort_buf[0], (void *)rc->sort_buf[1]})
            if (p) cudaFree(p);
        rc->sort_hist = rc->sort_buf[0] = rc->sort_buf[1] = nullptr;
        const uint32_t nk = std::max(nkeys_mat, nkeys_ray);
        if (cudaMalloc(&rc->sort_hist, sizeof(uint32_t) * nk) != cudaSuccess ||
            cudaMalloc(&rc->sort_buf[0], sizeof(uint32_t) * (size_t)cap) != cudaSuccess ||
            cudaMalloc(&rc->sort_buf[1], sizeof(uint32_t) * (size_t)cap) != cudaSuccess) {
            set_error("rt_render: sort buffers");
            return RT_OOM;
        }
        rc->sort_cap = cap;
        rc->sort_nkeys = nk;
    }
    RayKey rkey;
    rkey.lo = s->dev.bb_lo;
    rkey.inv_ext = make_float3(1.f / fmaxf(s->dev.bb_hi.x - s->dev.bb_lo.x, 1e-20f),
                               1.f / fmaxf(s->dev.bb_hi.y - s->dev.bb_lo.y, 1e-20f),
                               1.f / fmaxf(s->dev.bb_hi.z - s->dev.bb_lo.z, 1e-20f));
    MatKey mkey{s->dev, nmat};
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> evs;
    auto mark = [&](int kind) -> cudaEvent_t {
        if (!prof) return nullptr;
        cudaEvent_t a, b;
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        cudaEventRecord(a, st);
        evs.push_back({kind, {a, b}});
        return b;
    };
    auto done_ev = [&](cudaEvent_t b) {
        if (b) cudaEventRecord(b, st);
    };
    rt_stats stats{};
    const auto t_start = std::chrono::steady_clock::now();
    auto elapsed_ms = [&]() {
        return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
    };
    bool stop_sent = false;
    auto relay = [&]() {
        if (stop_sent) return;
        if ((o.abort_flag && *o.abort_flag) || (o.time_budget_ms > 0 && elapsed_ms() >= o.time_budget_ms)) {
            *(volatile uint32_t *)rc->stop_host = 1u;
            stop_sent = true;
        }
    };
    // wait for an event, relaying the stop conditions meanwhile
    auto wait = [&](cudaEvent_t e) -> rt_status {
        for (;;) {
            const cudaError_t q = cudaEventQuery(e);
            if (q == cudaSuccess) return RT_OK;
            if (q != cudaErrorNotReady) return cuda_status(q, "rt_render: waiting for a bounce-step chunk");
            relay();
            std::this_thread::yield();
        }
    };
    RT_CUDA_TRY(cudaMemsetAsync(pool.ctrl, 0, sizeof(Ctrl), st));
    // Two half-pools on two streams: a window that refills is split in two
    // halves of its tasks, each run by half of the pool with its own control
    // block, so that the kernels of one half run in the drain at the end of
    // the other's launches. A task's result depends only on its index and
    // the film is accumulated from the staging buffer afterwards, so the film
    // is the same. Not for stoppable calls (a stop must leave a prefix of the
    // tasks done), sorted queues (shared sort buffers) or per-kernel timing.
    const bool stoppable = o.abort_flag || o.time_budget_ms > 0;
    const bool dual = !stoppable && !o.sort_rays && !o.sort_by_material && !prof && cap >= (1u << 21) && win > cap;
    if (dual) {
        if (!rc->ctrl2) RT_CUDA_TRY(cudaMalloc(&rc->ctrl2, sizeof(Ctrl)));
        if (!rc->st2) RT_CUDA_TRY(cudaStreamCreateWithFlags(&rc->st2, cudaStreamNonBlocking));
        if (!rc->fork_ev) RT_CUDA_TRY(cudaEventCreateWithFlags(&rc->fork_ev, cudaEventDisableTiming));
        if (!rc->join_ev) RT_CUDA_TRY(cudaEventCreateWithFlags(&rc->join_ev, cudaEventDisableTiming));
    }
    auto regen_min_of = [&](uint32_t c) {
        return std::max<uint32_t>(1u, (uint32_t)std::min<double>((double)c, std::ceil(frac * c)));
    };
    bool any_single = false;
    unsigned long long dual_counts[7] = {0, 0, 0, 0, 0, 0, 0};   // ext, shadow rays; nodes, tris x2; refills
    constexpr int kChunk = 4;                       // bounce steps per host check
    const uint64_t step_limit = 64ull + 4ull * (max_depth + 2) * ((t_end - t_begin) / std::max<uint64_t>(cap / 2, 1) + 2);
    uint64_t t = t_begin;
    rt_status result = RT_OK;
    bool stopped = false;
    while (t < t_end && !stopped) {
        const uint32_t n_win = (uint32_t)std::min<uint64_t>(t_end - t, win);
        double left_ms = o.time_budget_ms > 0 ? o.time_budget_ms - elapsed_ms() : 0.0;
        const unsigned long long budget_ns =
            o.time_budget_ms > 0 ? (unsigned long long)std::max(1.0, left_ms * 1e6) : 0ull;
        if (dual && n_win > cap) {
            const uint32_t capA = (cap / 2) & ~255u, capB = cap - capA;
            const uint32_t nA = n_win / 2, nB = n_win - nA;
            const Pool sp[2] = {sub_pool(pool, 0u, capA, pool.ctrl), sub_pool(pool, capA, capB, rc->ctrl2)};
            const RegenScratch sg[2] = {gs, sub_scratch(gs, capA)};
            const cudaStream_t ss[2] = {st, rc->st2};
            float4 *const sstage[2] = {rc->stage, rc->stage + nA};
            const uint64_t st0[2] = {t, t + nA};
            const uint32_t sn[2] = {nA, nB}, srm[2] = {regen_min_of(capA), regen_min_of(capB)};
            RT_CUDA_TRY(cudaEventRecord(rc->fork_ev, st));
            RT_CUDA_TRY(cudaStreamWaitEvent(rc->st2, rc->fork_ev, 0));
            for (int i = 0; i < 2; ++i) {
                RT_CUDA_TRY(cudaMemsetAsync(sp[i].ctrl, 0, sizeof(Ctrl), ss[i]));
                k_regen_init<<<g_init, 256, 0, ss[i]>>>(P, sp[i], st0[i], sn[i], (uint32_t)WH, tail, 0ull,
                                                         rc->stop_dev);
            }
            stats.kernel_launches += 2;
            bool fin[2] = {false, false};
            uint64_t steps2 = 0;
            for (int chunk = 0;; ++chunk) {
                for (int i = 0; i < 2; ++i) {
                    if (fin[i]) continue;
                    for (int k = 0; k < kChunk; ++k) {
                        tk.ext<<<tk.grid_ext, gb, tk.smem, ss[i]>>>(s->dev, sp[i], nullptr);
                        (s->dev.lb_rec ? k_shade<true> : k_shade<false>)<<<g_shade, gb, 0, ss[i]>>>(P, sp[i],
                                                                                                  sp[i].split);
                        tk.shadow<<<tk.grid_shadow, gb, tk.smem, ss[i]>>>(s->dev, sp[i], nullptr);
                        k_regen_gather<<<g_regen, 256, 0, ss[i]>>>(sp[i], sstage[i], srm[i], sg[i]);
                        k_regen<<<g_regen, 256, 0, ss[i]>>>(P, sp[i], st0[i], (uint32_t)WH, srm[i], sg[i]);
                        k_regen_step_end<<<1, 1, 0, ss[i]>>>(sp[i], srm[i], rc->stop_dev);
                        stats.kernel_launches += 6;
                        ++stats.trace_launches;
                        ++stats.wavefront_steps;
                    }
                    RT_CUDA_TRY(cudaMemcpyAsync(rc->ctrl_ring + 2 * i + (chunk & 1), sp[i].ctrl, sizeof(Ctrl),
                                                cudaMemcpyDeviceToHost, ss[i]));
                    RT_CUDA_TRY(cudaEventRecord(rc->chunk_ev[2 * i + (chunk & 1)], ss[i]));
                }
                steps2 += kChunk;
                RT_CUDA_TRY(cudaGetLastError());
                if (chunk == 0) continue;
                for (int i = 0; i < 2; ++i) {
                    if (fin[i]) continue;
                    const rt_status ws = wait(rc->chunk_ev[2 * i + ((chunk - 1) & 1)]);
                    if (ws != RT_OK) return ws;
                    const Ctrl &hc = rc->ctrl_ring[2 * i + ((chunk - 1) & 1)];
                    if (hc.tail || (hc.n_ext == 0 && (hc.stop || hc.task_next == hc.n_tasks))) fin[i] = true;
                }
                if (fin[0] && fin[1]) break;
                if (steps2 > step_limit) {
                    set_error("rt_render: the regeneration scheduler did not drain its window");
                    return RT_CUDA_ERROR;
                }
            }
            for (int i = 0; i < 2; ++i) {
                k_megakernel<<<g_mega, gb, 0, ss[i]>>>(P, sp[i]);
                k_regen_retire_tail<<<g_regen, 256, 0, ss[i]>>>(sp[i], sstage[i]);
                RT_CUDA_TRY(cudaMemcpyAsync(rc->ctrl_ring + 2 * i, sp[i].ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost,
                                            ss[i]));
            }
            RT_CUDA_TRY(cudaEventRecord(rc->join_ev, rc->st2));
            RT_CUDA_TRY(cudaStreamWaitEvent(st, rc->join_ev, 0));
            k_film_range<<<grid_for(k_film_range, 256, WH), 256, 0, st>>>(rc->stage, film->sum, film->sum2,
                                                                          film->count, t, n_win, (uint32_t)WH);
            // the first half-pool's control block is the single pool's too
            RT_CUDA_TRY(cudaMemsetAsync(pool.ctrl, 0, sizeof(Ctrl), st));
            stats.kernel_launches += 5;
            stats.tail_launches += 2;
            ++stats.waves;
            RT_CUDA_TRY(cudaGetLastError());
            RT_CUDA_TRY(cudaStreamSynchronize(st));
            bool ovf = false;
            for (int i = 0; i < 2; ++i) {
                const Ctrl &c = rc->ctrl_ring[2 * i];
                if (c.task_next != sn[i] || c.n_tasks != sn[i]) {
                    set_error("rt_render: a half-pool did not finish its tasks");
                    return RT_CUDA_ERROR;
                }
                dual_counts[0] += c.ext_rays;
                dual_counts[1] += c.shadow_rays;
                dual_counts[2] += c.ext_nodes;
                dual_counts[3] += c.ext_tris;
                dual_counts[4] += c.shadow_nodes;
                dual_counts[5] += c.shadow_tris;
                dual_counts[6] += c.regen_sets;
                ovf |= c.overflow != 0;
            }
            t += n_win;
            film->next_task = t;
            stats.paths += n_win;
            if (ovf) { set_error("BVH traversal stack overflow"); result = RT_STACK_OVERFLOW; break; }
            continue;
        }
        any_single = true;
        cudaEvent_t e = mark(4);
        relay();
        k_regen_init<<<g_init, 256, 0, st>>>(P, pool, t, n_win, (uint32_t)WH, tail, budget_ns, rc->stop_dev);
        done_ev(e);
        ++stats.kernel_launches;
        uint64_t steps = 0;
        // a window that fits in the pool starts every task at once: its paths
        // end within max_depth + 1 steps, issued without a host check
        const bool one_load = n_win <= cap;
        const int per_chunk = one_load ? (int)max_depth + 1 : kChunk;
        for (int chunk = 0;; ++chunk) {
            for (int k = 0; k < per_chunk; ++k) {
                const uint32_t *rsorted = nullptr;
                if (o.sort_rays) {
                    e = mark(4);
                    RT_CUDA_TRY(cudaMemsetAsync(rc->sort_hist, 0, sizeof(uint32_t) * nkeys_ray, st));
                    k_sort_hist<RayKey><<<g_hist, 256, nkeys_ray * sizeof(uint32_t), st>>>(rkey, pool, nkeys_ray,
                                                                                          rc->sort_hist);
                    k_sort_scan<<<1, 1024, 0, st>>>(pool, nkeys_ray, rc->sort_hist);
                    k_sort_scatter<RayKey><<<g_hist, 256, 0, st>>>(rkey, pool, rc->sort_hist, rc->sort_buf[0]);
                    done_ev(e);
                    rsorted = rc->sort_buf[0];
                    stats.kernel_launches += 3;
                }
                e = mark(0);
                tk.ext<<<tk.grid_ext, gb, tk.smem, st>>>(s->dev, pool, rsorted);
                done_ev(e);
                const uint32_t *sorted = pool.split ? pool.split : rsorted;
                if (o.sort_by_material) {
                    e = mark(4);
                    RT_CUDA_TRY(cudaMemsetAsync(rc->sort_hist, 0, sizeof(uint32_t) * nkeys_mat, st));
                    k_sort_hist<MatKey><<<g_hist, 256, nkeys_mat * sizeof(uint32_t), st>>>(mkey, pool, nkeys_mat,
                                                                                          rc->sort_hist);
                    k_sort_scan<<<1, 1024, 0, st>>>(pool, nkeys_mat, rc->sort_hist);
                    k_sort_scatter<MatKey><<<g_hist, 256, 0, st>>>(mkey, pool, rc->sort_hist, rc->sort_buf[1]);
                    done_ev(e);
                    sorted = rc->sort_buf[1];
                    stats.kernel_launches += 3;
                }
                e = mark(1);
                (s->dev.lb_rec ? k_shade<true> : k_shade<false>)<<<g_shade, gb, 0, st>>>(P, pool, sorted);
                done_ev(e);
                e = mark(2);
                tk.shadow<<<tk.grid_shadow, gb, tk.smem, st>>>(s->dev, pool, nullptr);
                done_ev(e);
                e = mark(4);
                k_regen_gather<<<g_regen, 256, 0, st>>>(pool, rc->stage, regen_min, gs);
                k_regen<<<g_regen, 256, 0, st>>>(P, pool, t, (uint32_t)WH, regen_min, gs);
                k_regen_step_end<<<1, 1, 0, st>>>(pool, regen_min, rc->stop_dev);
                done_ev(e);
                stats.kernel_launches += 6;
                ++stats.trace_launches;
                ++stats.wavefront_steps;
            }
            steps += per_chunk;
            RT_CUDA_TRY(cudaGetLastError());
            if (one_load) break;
            Ctrl *ring = rc->ctrl_ring;
            RT_CUDA_TRY(cudaMemcpyAsync(ring + (chunk & 1), pool.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
            RT_CUDA_TRY(cudaEventRecord(rc->chunk_ev[chunk & 1], st));
            if (chunk == 0) continue;
            rt_status ws = wait(rc->chunk_ev[(chunk - 1) & 1]);
            if (ws != RT_OK) return ws;
            const Ctrl &hc = ring[(chunk - 1) & 1];
            if (hc.tail || (hc.n_ext == 0 && (hc.stop || hc.task_next == hc.n_tasks))) break;
            if (steps > step_limit) {
                set_error("rt_render: the regeneration scheduler did not drain its window");
                return RT_CUDA_ERROR;
            }
        }
        e = mark(3);
        k_megakernel<<<g_mega, gb, 0, st>>>(P, pool);
        done_ev(e);
        e = mark(4);
        k_regen_retire_tail<<<g_regen, 256, 0, st>>>(pool, rc->stage);
        RT_CUDA_TRY(cudaMemcpyAsync(rc->host_ctrl, pool.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
        rt_status ws = RT_OK;
        RT_CUDA_TRY(cudaEventRecord(rc->chunk_ev[0], st));
        if ((ws = wait(rc->chunk_ev[0])) != RT_OK) return ws;
        const uint32_t done_tasks = rc->host_ctrl->task_next;
        k_film_range<<<grid_for(k_film_range, 256, WH), 256, 0, st>>>(rc->stage, film->sum, film->sum2, film->count,
                                                                      t, done_tasks, (uint32_t)WH);
        done_ev(e);
        stats.kernel_launches += 3;
        ++stats.tail_launches;
        ++stats.waves;
        RT_CUDA_TRY(cudaGetLastError());
        RT_CUDA_TRY(cudaStreamSynchronize(st));
        t += done_tasks;
        film->next_task = t;
        stats.paths += done_tasks;
        if (rc->host_ctrl->overflow) { set_error("BVH traversal stack overflow"); result = RT_STACK_OVERFLOW; break; }
        if (rc->host_ctrl->stop || done_tasks < n_win) stopped = true;
    }
    if (stopped && t < t_end && result == RT_OK) {
        set_error("rt_render: stopped by time budget or abort flag (resumable: the film holds the completed tasks)");
        result = RT_TIMEOUT;
    }
    for (auto &kv : evs) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, kv.second.first, kv.second.second);
        double *dst[5] = {&stats.trace_ms, &stats.shade_ms, &stats.shadow_ms, &stats.megakernel_ms, &stats.other_ms};
        *dst[kv.first] += ms;
        cudaEventDestroy(kv.second.first);
        cudaEventDestroy(kv.second.second);
    }
    const Ctrl zero{};
    const Ctrl &hcs = any_single ? *rc->host_ctrl : zero;
    stats.extension_rays = hcs.ext_rays + dual_counts[0];
    stats.shadow_rays = hcs.shadow_rays + dual_counts[1];
    stats.ext_nodes = hcs.ext_nodes + dual_counts[2];
    stats.ext_tris = hcs.ext_tris + dual_counts[3];
    stats.shadow_nodes = hcs.shadow_nodes + dual_counts[4];
    stats.shadow_tris = hcs.shadow_tris + dual_counts[5];
    stats.regen_sets = hcs.regen_sets + (uint32_t)dual_counts[6];
    if (o.stats) *o.stats = stats;
    return result;
}

extern "C" rt_status rt_render(const rt_scene *s, const rt_camera *cam, uint32_t spp, uint32_t max_depth,
                               rt_film *film, const rt_render_opts *opts_in, void *stream) {
    if (!s || !cam || !film) { set_error("rt_render: null argument"); return RT_INVALID_ARG; }
    if (s->host_only) { set_error("rt_render: scene has no device copy"); return RT_INVALID_ARG; }
    if (cam->width != film->W || cam->height != film->H) { set_error("rt_render: film and camera sizes differ"); return RT_INVALID_ARG; }
    if (max_depth < 1 || max_depth > (uint32_t)kMaxDepth) { set_error("rt_render: max_depth must be in [1, 64]"); return RT_INVALID_ARG; }
    rt_render_opts o{};
    if (opts_in) o = *opts_in;
    if (spp == 0) return RT_OK;
    if (o.trace_kernel < 0 || o.trace_kernel > 8) { set_error("rt_render: trace_kernel must be in [0, 8]"); return RT_INVALID_ARG; }
    if (!valid_block(o.block_size)) { set_error("rt_render: block_size must be 0 or a multiple of 32 up to 128"); return RT_INVALID_ARG; }
    if (s->dev.two_level) o.trace_kernel = 0;   // the persistent variant is single-level only
    cudaStream_t st = (cudaStream_t)stream;
    RenderCache *rc = cache_of(film);
    const uint32_t W = cam->width, H = cam->height;
    const uint64_t WH = (uint64_t)W * H;
    const uint64_t request = (film->next_task / WH + (uint64_t)spp) * WH - film->next_task;
    // the regeneration scheduler streams tasks through a bounded pool; the
    // iteration-set scheduler (A/B) holds a whole set at once
    const bool regen = !o.guide && o.scheduler == 0 && !o.megakernel_only;
    if (o.scheduler < 0 || o.scheduler > 1) { set_error("rt_render: scheduler must be 0 or 1"); return RT_INVALID_ARG; }
    if (!(o.regen_fraction >= 0.f && o.regen_fraction <= 1.f)) {
        set_error("rt_render: regen_fraction must be in [0, 1]");
        return RT_INVALID_ARG;
    }
    // default pool: the whole request at once when it fits (at most 2^27
    // paths and a quarter of free memory): fewer bounce steps, so fewer
    // launch tails, than a smaller pool refilled by regeneration, which then
    // engages only for larger requests. A call that can be stopped (abort
    // flag or time budget) takes 2^24 paths at most instead, so that a stop
    // leaves most of the request unstarted and the paths in flight drain
    // quickly.
    const bool stoppable = o.abort_flag || o.time_budget_ms > 0;
    uint32_t cap = o.max_paths_in_flight ? o.max_paths_in_flight : default_capacity(request);
    if (regen && stoppable && !o.max_paths_in_flight) cap = std::min<uint32_t>(cap, 1u << 24);
    cap = std::max<uint32_t>(cap, 32u);
    if (o.state_compression && !regen) {
        set_error("rt_render: state_compression needs the regeneration scheduler, without guiding or megakernel_only");
        return RT_NOT_SUPPORTED;
    }
    rt_status rs = ensure_pool(rc->pool, cap, o.state_compression != 0);
    if (rs != RT_OK) return rs;
    const int ndims = 2 + 7 * (int)(max_depth + 1);
    if (!rc->dims || rc->dims_seed != o.seed || rc->dims_n < ndims) {
        std::vector<HaltonDim> d = make_dims(o.seed, ndims);
        if (rc->dims) cudaFree(rc->dims);
        RT_CUDA_TRY(cudaMalloc(&rc->dims, d.size() * sizeof(HaltonDim)));
        RT_CUDA_TRY(cudaMemcpy(rc->dims, d.data(), d.size() * sizeof(HaltonDim), cudaMemcpyHostToDevice));
        rc->dims_seed = o.seed;
        rc->dims_n = ndims;
    }
    if (!rc->host_ctrl) RT_CUDA_TRY(cudaMallocHost(&rc->host_ctrl, sizeof(Ctrl)));
    // a request that fits one pool load has nothing to regenerate: unless the
    // call can be stopped (or its state is compressed, which only the
    // regeneration path lays out) it runs as one load of the plain schedule,
    // without staging its radiance per task
    const bool one_load = request <= cap && !stoppable && !o.state_compression;
    if (regen && !one_load) return render_regen(s, cam, spp, max_depth, film, o, st, rc, cap);
    RenderParams P;
    P.sc = s->dev;
    P.cam = make_camera(*cam);
    P.en = make_enum(W, H);
    P.dims = rc->dims;
    P.max_depth = max_depth;
    P.sigma = o.filter_sigma == 0.f ? 0.5f : o.filter_sigma;
    P.mis_mode = o.mis_mode;
    P.rr = o.rr_enable;
    const uint32_t tail = o.megakernel_only ? 0xFFFFFFFFu : (o.tail_threshold ? o.tail_threshold : 8192u);
    Pool pool = rc->pool.view;
    RT_CUDA_TRY(cudaMemsetAsync(pool.ctrl, 0, sizeof(Ctrl), st));
    rt_stats stats{};
    auto t_start = std::chrono::steady_clock::now();
    uint64_t t = film->next_task, t_end = (film->next_task / WH + (uint64_t)spp) * WH;
    rt_status result = RT_OK;
    if (o.guide) {
        // Guided iteration sets: every bounce step reads the queue length,
        // runs the network on the queue's vertices (vertices 1..gdepth),
        // shades with the one-sample MIS mixture and records training
        // samples; training steps follow the set (below). The megakernel
        // tail is off (it has no guided branch).
        rt_guide *gd = o.guide;
        const uint32_t batch = guide_batch(gd);
        // iteration sets, training schedule and buffer sizes: guided_plan
        if (batch > (1u << 24)) { set_error("rt_render: guide batch above 2^24 samples"); return RT_INVALID_ARG; }
        const uint32_t cap_full = cap;
        const GuidedPlan gp = guided_plan(batch, guide_warm_set_batches(gd), guide_depth(gd), max_depth, cap,
                                          o.max_paths_in_flight != 0);
        cap = gp.cap;
        const uint32_t cap_young = gp.cap_young, gdepth = gp.gdepth, rec_depth = gp.rec_depth;
        if ((rs = ensure_guided(rc, cap_full, gp.rec_alloc, gp.keep_alloc)) != RT_OK) return rs;
        rc->pool.view.nrec = rc->gnrec;
        Pool gpool = rc->pool.view;
        gpool.qd = nullptr;      // no regeneration: ended paths are not queued
        gpool.split = nullptr;   // one shading queue
        float3 glo, ghi;
        guide_bounds(gd, glo, ghi);
        const float alpha = guide_alpha(gd);
        const int gbk = (int)kGuidedShadeThreads;
        const int g_ray = grid_for(k_raygen, 256, cap);
        const TraceKernels tk = trace_kernels(false, 0, s->dev.two_level, gbk);
        // both kernels compiled with and without the light hierarchy
        const auto shade_guided = s->dev.lb_rec ? k_shade_guided<true> : k_shade_guided<false>;
        const int g_shade = grid_persistent(shade_guided, gbk, 0);
        const int g_shade_plain = grid_persistent(k_shade<true>, gbk, 0);
        if ((rs = mlp_kernel_attr((const void *)k_guide_mlp_paths, kMlpInferSmem)) != RT_OK) return rs;
        const PathFeatures pf{P, gpool, glo, ghi};
        rt_stats stats{};
        auto t_start = std::chrono::steady_clock::now();
        uint64_t t = film->next_task, t_end = (film->next_task / WH + (uint64_t)spp) * WH;
        rt_status result = RT_OK;
        while (t < t_end) {
            const uint32_t cset = guide_young(gd) ? cap_young : cap;
            uint64_t n64;
            uint32_t passes = 0;
            if (t % WH != 0 || WH > cset) {
                n64 = std::min<uint64_t>({t_end - t, WH - t % WH, (uint64_t)cset});
            } else {
                uint64_t full = std::min<uint64_t>((t_end - t) / WH, cset / WH);
                if (full >= 1) { passes = (uint32_t)full; n64 = full * WH; }
                else n64 = std::min<uint64_t>(t_end - t, cset);
            }
            uint32_t n = (uint32_t)n64;
            const float a = guide_trained(gd) ? alpha : 0.f;
            // recording paths and the samples kept (both within the buffers
            // sized above): every rec_stride-th path records
            const bool young = guide_young(gd);
            const GuidedSet gs = guided_set(gp, batch, n, young);
            const uint32_t set_steps = gs.set_steps, keep = gs.keep, rec_paths = gs.rec_paths,
                           rec_stride = gs.rec_stride;
            k_raygen<<<g_ray, 256, 0, st>>>(P, gpool, t, n, (uint32_t)WH, 0u);
            stats.kernel_launches += 1;
            // every bounce step runs on the device-side queue lengths: no
            // host round trip until the set is done
            for (uint32_t v = 1; v <= max_depth + 1; ++v) {
                tk.ext<<<tk.grid_ext, gbk, 0, st>>>(s->dev, gpool, nullptr);
                // the network runs only where a continuation is guided: not
                // at the last vertex (it only adds emission) nor past gdepth
                const float av = v <= gdepth ? a : 0.f;
                if (av > 0.f) {
                    k_guide_mlp_paths<<<sm_count(), kMiThreads, kMlpInferSmem, st>>>(guide_weights(gd), pf, rc->gfeat,
                                                                            guide_err(gd));
                    stats.kernel_launches += 1;
                }
                if (v <= rec_depth + 1) {
                    // guided, or finishing the records of the vertex before
                    shade_guided<<<g_shade, gbk, 0, st>>>(P, gpool, av > 0.f ? rc->gfeat : nullptr, av, rc->grec,
                                                          rec_stride, rec_paths, rec_depth, glo, ghi);
                } else {
                    (s->dev.lb_rec ? k_shade<true> : k_shade<false>)<<<g_shade_plain, gbk, 0, st>>>(P, gpool, nullptr);
                }
                tk.shadow<<<tk.grid_shadow, gbk, 0, st>>>(s->dev, gpool, nullptr);
                k_step_end<<<1, 1, 0, st>>>(gpool);
                stats.kernel_launches += 4;
                ++stats.wavefront_steps;
            }
            int g_film = grid_for(k_film, 256, passes ? WH : n);
            k_film<<<g_film, 256, 0, st>>>(gpool, film->sum, film->sum2, film->count, t, n, (uint32_t)WH, passes);
            k_guide_collect<<<grid_for(k_guide_collect, 256, std::min(n, rec_paths)), 256, 0, st>>>(
                gpool, n, rc->grec, rec_stride, rc->tr_feat, rc->tr_wi, rc->tr_w, rec_paths, keep);
            stats.kernel_launches += 2;
            RT_CUDA_TRY(cudaGetLastError());
            RT_CUDA_TRY(cudaMemcpyAsync(rc->host_ctrl, gpool.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
            RT_CUDA_TRY(cudaStreamSynchronize(st));
            t += n;
            film->next_task = t;
            stats.paths += n;
            ++stats.waves;
            if (rc->host_ctrl->overflow) { set_error("BVH traversal stack overflow"); result = RT_STACK_OVERFLOW; break; }
            if ((rs = guide_check(gd, st)) != RT_OK) return rs;
            const uint32_t n_train = std::min(rc->host_ctrl->n_train, keep);
            if (n_train >= 256 && guide_should_train(gd)) {
                // one training call per full batch (a young set: at most the
                // warm-up calls still to take; later one per 16 batches of
                // paths rendered), else one on what there is
                const uint32_t steps = std::max(1u, std::min(n_train / batch, young ? guide_warm_left(gd) : set_steps));
                for (uint32_t k = 0; k < steps; ++k) {
                    const size_t off = (size_t)k * batch;
                    const uint32_t m = steps > 1 ? batch : std::min(n_train, batch);
                    if ((rs = guide_train_async(gd, rc->tr_feat + 7 * off, rc->tr_wi + 3 * off, rc->tr_w + off, m, st)) !=
                        RT_OK)
                        return rs;
                    stats.kernel_launches += 40;
                }
            }
            double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
            if (t < t_end && ((o.abort_flag && *o.abort_flag) || (o.time_budget_ms > 0 && ms >= o.time_budget_ms))) {
                set_error("rt_render: stopped by time budget or abort flag (resumable)");
                result = RT_TIMEOUT;
                break;
            }
        }
        RT_CUDA_TRY(cudaStreamSynchronize(st));
        rc->pool.view.nrec = nullptr;
        stats.extension_rays = rc->host_ctrl->ext_rays;
        stats.shadow_rays = rc->host_ctrl->shadow_rays;
        if (o.stats) *o.stats = stats;
        return result;
    }
    const int gb = o.block_size ? (int)o.block_size : 128;
    const int g_ray = grid_for(k_raygen, 256, cap);
    const size_t smem = stack_smem(gb);
    const int g_trace = grid_persistent(k_trace_ext<false>, gb, smem);
    const int g_shade = grid_persistent(k_shade<true>, gb, 0);
    const int g_shadow = grid_persistent(k_trace_shadow<false>, gb, smem);
    const int g_mega = grid_for(k_megakernel, gb, cap);
    const bool prof = o.profile >= 1, count = o.profile >= 2;
    // variant 5: camera rays one per thread (coherent), later bounces with
    // lane refill (incoherent rays that end at very different times)
    const TraceKernels tk = trace_kernels(count, o.trace_kernel == 5 ? 0 : o.trace_kernel, s->dev.two_level, gb);
    const TraceKernels tk_late = o.trace_kernel == 5 && !s->dev.two_level ? trace_kernels(count, 3, false, gb) : tk;
    pool.split = o.trace_kernel != 5 && variant_splits(o.trace_kernel, s->dev.two_level) ? rc->pool.split : nullptr;
    const uint32_t nmat = s->num_materials;
    const uint32_t nkeys_mat = nmat + 1, nkeys_ray = 8u * 512u;
    const int g_hist = grid_for(k_sort_scatter<RayKey>, 256, cap);
    if ((o.sort_by_material || o.sort_rays) && (rc->sort_cap < cap || rc->sort_nkeys < std::max(nkeys_mat, nkeys_ray))) {
        for (void *p : {(void *)rc->sort_hist, (void *)rc->sort_buf[0], (void *)rc->sort_buf[1]})
            if (p) cudaFree(p);
        rc->sort_hist = rc->sort_buf[0] = rc->sort_buf[1] = nullptr;
        const uint32_t nk = std::max(nkeys_mat, nkeys_ray);
        if (cudaMalloc(&rc->sort_hist, sizeof(uint32_t) * nk) != cudaSuccess ||
            cudaMalloc(&rc->sort_buf[0], sizeof(uint32_t) * (size_t)cap) != cudaSuccess ||
            cudaMalloc(&rc->sort_buf[1], sizeof(uint32_t) * (size_t)cap) != cudaSuccess) {
            set_error("rt_render: sort buffers");
            return RT_OOM;
        }
        rc->sort_cap = cap;
        rc->sort_nkeys = nk;
    }
    RayKey rkey;
    rkey.lo = s->dev.bb_lo;
    rkey.inv_ext = make_float3(1.f / fmaxf(s->dev.bb_hi.x - s->dev.bb_lo.x, 1e-20f),
                               1.f / fmaxf(s->dev.bb_hi.y - s->dev.bb_lo.y, 1e-20f),
                               1.f / fmaxf(s->dev.bb_hi.z - s->dev.bb_lo.z, 1e-20f));
    MatKey mkey{s->dev, nmat};
    // event pairs per timed launch: kind 0 trace, 1 shade, 2 shadow, 3 megakernel, 4 other
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> evs;
    auto mark = [&](int kind) -> cudaEvent_t {
        if (!prof) return nullptr;
        cudaEvent_t a, b;
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        cudaEventRecord(a, st);
        evs.push_back({kind, {a, b}});
        return b;
    };
    auto done = [&](cudaEvent_t b) {
        if (b) cudaEventRecord(b, st);
    };
    while (t < t_end) {
        uint64_t n64;
        uint32_t passes = 0;
        if (t % WH != 0 || WH > cap) {
            n64 = std::min<uint64_t>({t_end - t, WH - t % WH, (uint64_t)cap});
        } else {
            uint64_t full = std::min<uint64_t>((t_end - t) / WH, cap / WH);
            if (full >= 1) { passes = (uint32_t)full; n64 = full * WH; }
            else n64 = std::min<uint64_t>(t_end - t, cap);
        }
        uint32_t n = (uint32_t)n64;
        cudaEvent_t e = mark(4);
        k_raygen<<<g_ray, 256, 0, st>>>(P, pool, t, n, (uint32_t)WH, tail);
        done(e);
        ++stats.kernel_launches;
        if (!o.megakernel_only) {
            for (uint32_t v = 1; v <= max_depth + 1; ++v) {
                const uint32_t *rsorted = nullptr;
                if (o.sort_rays && v >= 2) {
                    e = mark(4);
                    RT_CUDA_TRY(cudaMemsetAsync(rc->sort_hist, 0, sizeof(uint32_t) * nkeys_ray, st));
                    k_sort_hist<RayKey><<<g_hist, 256, nkeys_ray * sizeof(uint32_t), st>>>(rkey, pool, nkeys_ray, rc->sort_hist);
                    k_sort_scan<<<1, 1024, 0, st>>>(pool, nkeys_ray, rc->sort_hist);
                    k_sort_scatter<RayKey><<<g_hist, 256, 0, st>>>(rkey, pool, rc->sort_hist, rc->sort_buf[0]);
                    done(e);
                    rsorted = rc->sort_buf[0];
                    stats.kernel_launches += 3;
                }
                e = mark(0);
                if (o.trace_kernel != 1) {
                    const TraceKernels &tv = v >= 2 ? tk_late : tk;
                    tv.ext<<<tv.grid_ext, gb, tv.smem, st>>>(s->dev, pool, rsorted);
                } else if (count) {
                    k_trace_ext<true><<<g_trace, gb, smem, st>>>(s->dev, pool);
                } else {
                    k_trace_ext<false><<<g_trace, gb, smem, st>>>(s->dev, pool);
                }
                done(e);
                const uint32_t *sorted = pool.split ? pool.split : rsorted;
                if (o.sort_by_material) {
                    e = mark(4);
                    RT_CUDA_TRY(cudaMemsetAsync(rc->sort_hist, 0, sizeof(uint32_t) * nkeys_mat, st));
                    k_sort_hist<MatKey><<<g_hist, 256, nkeys_mat * sizeof(uint32_t), st>>>(mkey, pool, nkeys_mat, rc->sort_hist);
                    k_sort_scan<<<1, 1024, 0, st>>>(pool, nkeys_mat, rc->sort_hist);
                    k_sort_scatter<MatKey><<<g_hist, 256, 0, st>>>(mkey, pool, rc->sort_hist, rc->sort_buf[1]);
                    done(e);
                    sorted = rc->sort_buf[1];
                    stats.kernel_launches += 3;
                }
                e = mark(1);
                (s->dev.lb_rec ? k_shade<true> : k_shade<false>)<<<g_shade, gb, 0, st>>>(P, pool, sorted);
                done(e);
                e = mark(2);
                if (o.trace_kernel != 1) {
                    tk.shadow<<<tk.grid_shadow, gb, tk.smem, st>>>(s->dev, pool, nullptr);
                } else if (count) {
                    k_trace_shadow<true><<<g_shadow, gb, smem, st>>>(s->dev, pool);
                } else {
                    k_trace_shadow<false><<<g_shadow, gb, smem, st>>>(s->dev, pool);
                }
                done(e);
                k_step_end<<<1, 1, 0, st>>>(pool);
                stats.kernel_launches += 4;
                ++stats.trace_launches;
                ++stats.wavefront_steps;
            }
        }
        e = mark(3);
        k_megakernel<<<g_mega, gb, 0, st>>>(P, pool);
        done(e);
        ++stats.tail_launches;
        int g_film = grid_for(k_film, 256, passes ? WH : n);
        e = mark(4);
        k_film<<<g_film, 256, 0, st>>>(pool, film->sum, film->sum2, film->count, t, n, (uint32_t)WH, passes);
        done(e);
        stats.kernel_launches += 2;
        RT_CUDA_TRY(cudaGetLastError());
        RT_CUDA_TRY(cudaMemcpyAsync(rc->host_ctrl, pool.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
        RT_CUDA_TRY(cudaStreamSynchronize(st));
        t += n;
        film->next_task = t;
        stats.paths += n;
        ++stats.waves;
        if (rc->host_ctrl->overflow) { set_error("BVH traversal stack overflow"); result = RT_STACK_OVERFLOW; break; }
        double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
        if (t < t_end && ((o.abort_flag && *o.abort_flag) || (o.time_budget_ms > 0 && ms >= o.time_budget_ms))) {
            set_error("rt_render: stopped by time budget or abort flag (resumable)");
            result = RT_TIMEOUT;
            break;
        }
    }
    for (auto &kv : evs) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, kv.second.first, kv.second.second);
        double *dst[5] = {&stats.trace_ms, &stats.shade_ms, &stats.shadow_ms, &stats.megakernel_ms, &stats.other_ms};
        *dst[kv.first] += ms;
        cudaEventDestroy(kv.second.first);
        cudaEventDestroy(kv.second.second);
    }
    stats.extension_rays = rc->host_ctrl->ext_rays;
    stats.shadow_rays = rc->host_ctrl->shadow_rays;
    stats.ext_nodes = rc->host_ctrl->ext_nodes;
    stats.ext_tris = rc->host_ctrl->ext_tris;
    stats.shadow_nodes = rc->host_ctrl->shadow_nodes;
    stats.shadow_tris = rc->host_ctrl->shadow_tris;
    if (o.stats) *o.stats = stats;
    return result;
}

extern "C" rt_status rt_sample_index(uint32_t W, uint32_t H, const uint32_t *px, const uint32_t *py, const uint32_t *j,
                                     int64_t n, uint64_t *out, void *stream) {
    if (W == 0 || H == 0 || n < 0 || (n > 0 && (!px || !py || !j || !out))) {
        set_error("rt_sample_index: invalid argument");
        return RT_INVALID_ARG;
    }
    if (n == 0) return RT_OK;
    Enum en = make_enum(W, H);
    k_sample_index<<<grid_for(k_sample_index, 256, n), 256, 0, (cudaStream_t)stream>>>(en, px, py, j, n, out);
    RT_CUDA_TRY(cudaGetLastError());
    return RT_OK;
}

extern "C" rt_status rt_halton(uint32_t W, uint32_t H, uint64_t seed, const uint64_t *idx, int64_t n, int32_t ndims,
                               uint32_t *out, void *stream) {
    if (W == 0 || H == 0 || n < 0 || ndims < 0 || ndims > 1024 || (n > 0 && (!idx || !out))) {
        set_error("rt_halton: invalid argument");
        return RT_INVALID_ARG;
    }
    if (n == 0 || ndims == 0) return RT_OK;
    std::vector<HaltonDim> d = make_dims(seed, std::max(ndims, 3));
    HaltonDim *dd = nullptr;
    cudaStream_t st = (cudaStream_t)stream;
    RT_CUDA_TRY(cudaMallocAsync(&dd, d.size() * sizeof(HaltonDim), st));
    RT_CUDA_TRY(cudaMemcpyAsync(dd, d.data(), d.size() * sizeof(HaltonDim), cudaMemcpyHostToDevice, st));
    Enum en = make_enum(W, H);
    k_halton<<<grid_for(k_halton, 256, n), 256, 0, st>>>(en, dd, idx, n, ndims, out);
    cudaError_t e = cudaGetLastError();
    cudaFreeAsync(dd, st);
    RT_CUDA_TRY(cudaStreamSynchronize(st));
    RT_CUDA_TRY(e);
    return RT_OK;
}

// ---------------------------------------------------------------------------
// Rendering without device allocations (the paper has no counterpart).
//
// Some callers cannot call cudaMalloc: code embedded in a host framework
// that owns every device allocation through its own arena, services whose
// device memory budget is fixed when they start, or threads on which an
// allocation would synchronise the device and stall unrelated work. For them
// rt_render_static renders with its path-state pool, control block and
// sampling table in one file-scope __device__ array of fixed size instead of
// memory obtained from the allocator. The array exists on every device that
// loads the library, until the process exits.
namespace rtg {

constexpr uint32_t kStaticMaxPaths = 65536;                 // paths in flight
constexpr int kStaticMaxDims = 2 + 7 * (kMaxDepth + 1);     // sampling dimensions
constexpr size_t kAlign = 256;
constexpr size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }
constexpr size_t kStaticCtrl = 0;
constexpr size_t kStaticDims = kStaticCtrl + align_up(sizeof(Ctrl));
constexpr size_t kStaticF4 = kStaticDims + align_up(sizeof(HaltonDim) * kStaticMaxDims);
constexpr size_t kStaticF4Bytes = align_up(sizeof(float4) * kStaticMaxPaths);
constexpr size_t kStaticIndex = kStaticF4 + 8 * kStaticF4Bytes;
constexpr size_t kStaticU32Bytes = align_up(sizeof(uint32_t) * kStaticMaxPaths);
constexpr size_t kStaticPixel = kStaticIndex + align_up(sizeof(uint2) * kStaticMaxPaths);
constexpr size_t kStaticHitInst = kStaticPixel + kStaticU32Bytes;
constexpr size_t kStaticQueues = kStaticHitInst + kStaticU32Bytes;
constexpr size_t kStaticBytes = kStaticQueues + 3 * kStaticU32Bytes;   // 9.91 MiB
static_assert(kStaticBytes == RT_STATIC_ARENA_BYTES, "include/rt.h states the static array's size");

static __device__ __align__(256) unsigned char g_static_arena[kStaticBytes];

// Device address of g_static_arena in the current context. In host code the
// symbol name is only a host-side stand-in, so the address is looked up with
// cudaGetSymbolAddress on every call (after the first call on a device this
// is a host-side table lookup that allocates nothing). It is not cached: a
// cached address would go stale after cudaDeviceReset or belong to another
// context when the caller switches to a non-primary context.
static rt_status static_arena(unsigned char **out) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_arena);
    if (e != cudaSuccess || !p) return cuda_status(e, "cudaGetSymbolAddress(g_static_arena)");
    *out = (unsigned char *)p;
    return RT_OK;
}

}  // namespace rtg

extern "C" rt_status rt_render_probes(const rt_scene *s, const float *pos, const float *nrm, uint32_t n,
                                      uint32_t spp, uint32_t max_depth, rt_film *film, const rt_render_opts *opts_in,
                                      void *stream) {
    if (!s || !film || (n > 0 && (!pos || !nrm))) { set_error("rt_render_probes: null argument"); return RT_INVALID_ARG; }
    if (s->host_only) { set_error("rt_render_probes: scene has no device copy"); return RT_INVALID_ARG; }
    if (n == 0 || film->W != n || film->H != 1) {
        set_error("rt_render_probes: the film must be n x 1 for n > 0 probes");
        return RT_INVALID_ARG;
    }
    if (max_depth < 1 || max_depth > (uint32_t)kMaxDepth) { set_error("rt_render_probes: max_depth must be in [1, 64]"); return RT_INVALID_ARG; }
    rt_render_opts o{};
    if (opts_in) o = *opts_in;
    if (!valid_block(o.block_size)) { set_error("rt_render_probes: block_size must be 0 or a multiple of 32 up to 128"); return RT_INVALID_ARG; }
    if (o.guide) { set_error("rt_render_probes: guiding needs rt_render"); return RT_NOT_SUPPORTED; }
    if (spp == 0) return RT_OK;
    cudaStream_t st = (cudaStream_t)stream;
    RenderCache *rc = cache_of(film);
    const uint64_t WH = n;
    uint32_t cap = o.max_paths_in_flight ? o.max_paths_in_flight
                                         : default_capacity((film->next_task / WH + (uint64_t)spp) * WH - film->next_task);
    cap = std::max<uint32_t>(cap, 32u);
    rt_status rs = ensure_pool(rc->pool, cap);
    if (rs != RT_OK) return rs;
    const int ndims = 2 + 7 * (int)(max_depth + 1);
    if (!rc->dims || rc->dims_seed != o.seed || rc->dims_n < ndims) {
        std::vector<HaltonDim> d = make_dims(o.seed, ndims);
        if (rc->dims) cudaFree(rc->dims);
        RT_CUDA_TRY(cudaMalloc(&rc->dims, d.size() * sizeof(HaltonDim)));
        RT_CUDA_TRY(cudaMemcpy(rc->dims, d.data(), d.size() * sizeof(HaltonDim), cudaMemcpyHostToDevice));
        rc->dims_seed = o.seed;
        rc->dims_n = ndims;
    }
    rt_camera cam{};
    cam.width = n;
    cam.height = 1;
    cam.look_at[2] = 1.f;
    cam.up[1] = 1.f;
    cam.vfov_deg = 45.f;
    RenderParams P;
    P.sc = s->dev;
    P.cam = make_camera(cam);
    P.en = make_enum(n, 1);
    P.dims = rc->dims;
    P.max_depth = max_depth;
    P.sigma = 0.5f;
    P.mis_mode = o.mis_mode;
    P.rr = o.rr_enable;
    Pool pool = rc->pool.view;
    RT_CUDA_TRY(cudaMemsetAsync(pool.ctrl, 0, sizeof(Ctrl), st));
    const int gb = o.block_size ? (int)o.block_size : 128;
    const TraceKernels tk = trace_kernels(false, 0, s->dev.two_level, gb);
    const int g_start = grid_for(k_probe_start, 256, cap);
    const int g_shade = grid_persistent(k_shade<true>, gb, 0);
    rt_stats stats{};
    Ctrl host_ctrl{};
    auto t_start = std::chrono::steady_clock::now();
    uint64_t t = film->next_task, t_end = (film->next_task / WH + (uint64_t)spp) * WH;
    rt_status result = RT_OK;
    while (t < t_end) {
        uint64_t n64;
        uint32_t passes = 0;
        if (t % WH != 0 || WH > cap) {
            n64 = std::min<uint64_t>({t_end - t, WH - t % WH, (uint64_t)cap});
        } else {
            uint64_t full = std::min<uint64_t>((t_end - t) / WH, cap / WH);
            if (full >= 1) { passes = (uint32_t)full; n64 = full * WH; }
            else n64 = std::min<uint64_t>(t_end - t, cap);
        }
        const uint32_t ns = (uint32_t)n64;
        k_probe_reset<<<1, 1, 0, st>>>(pool);
        k_probe_start<<<g_start, 256, 0, st>>>(P, pool, pos, nrm, t, ns, (uint32_t)WH);
        tk.shadow<<<tk.grid_shadow, gb, tk.smem, st>>>(s->dev, pool, nullptr);
        k_probe_shadow_done<<<1, 1, 0, st>>>(pool);
        stats.kernel_launches += 4;
        for (uint32_t v = 2; v <= max_depth + 1; ++v) {
            tk.ext<<<tk.grid_ext, gb, tk.smem, st>>>(s->dev, pool, nullptr);
            (s->dev.lb_rec ? k_shade<true> : k_shade<false>)<<<g_shade, gb, 0, st>>>(P, pool, nullptr);
            tk.shadow<<<tk.grid_shadow, gb, tk.smem, st>>>(s->dev, pool, nullptr);
            k_step_end<<<1, 1, 0, st>>>(pool);
            stats.kernel_launches += 4;
            ++stats.wavefront_steps;
        }
        const int g_film = grid_for(k_film, 256, passes ? WH : ns);
        k_film<<<g_film, 256, 0, st>>>(pool, film->sum, film->sum2, film->count, t, ns, (uint32_t)WH, passes);
        stats.kernel_launches += 1;
        RT_CUDA_TRY(cudaGetLastError());
        RT_CUDA_TRY(cudaMemcpyAsync(&host_ctrl, pool.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
        RT_CUDA_TRY(cudaStreamSynchronize(st));
        t += ns;
        film->next_task = t;
        stats.paths += ns;
        ++stats.waves;
        if (host_ctrl.overflow) { set_error("BVH traversal stack overflow"); result = RT_STACK_OVERFLOW; break; }
        double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
        if (t < t_end && ((o.abort_flag && *o.abort_flag) || (o.time_budget_ms > 0 && ms >= o.time_budget_ms))) {
            set_error("rt_render_probes: stopped by time budget or abort flag (resumable)");
            result = RT_TIMEOUT;
            break;
        }
    }
    stats.extension_rays = host_ctrl.ext_rays;
    stats.shadow_rays = host_ctrl.shadow_rays;
    if (o.stats) *o.stats = stats;
    return result;
}

extern "C" rt_status rt_render_static(const rt_scene *s, const rt_camera *cam, uint32_t spp, uint32_t max_depth,
                                      uint32_t first_iteration, double *sum, double *sum2, uint32_t *count,
                                      const rt_render_opts *opts_in, void *stream) {
    if (!s || !cam || !sum || !sum2 || !count) { set_error("rt_render_static: null argument"); return RT_INVALID_ARG; }
    if (s->host_only) { set_error("rt_render_static: scene has no device copy"); return RT_INVALID_ARG; }
    if (cam->width == 0 || cam->height == 0 || (uint64_t)cam->width * cam->height > (1ull << 31)) {
        set_error("rt_render_static: invalid image size");
        return RT_INVALID_ARG;
    }
    if (max_depth < 1 || max_depth > (uint32_t)kMaxDepth) { set_error("rt_render_static: max_depth must be in [1, 64]"); return RT_INVALID_ARG; }
    rt_render_opts o{};
    if (opts_in) o = *opts_in;
    if (!valid_block(o.block_size)) { set_error("rt_render_static: block_size must be 0 or a multiple of 32 up to 128"); return RT_INVALID_ARG; }
    if (o.guide) { set_error("rt_render_static: guiding needs rt_render"); return RT_NOT_SUPPORTED; }
    if (o.sort_by_material || o.sort_rays || o.state_compression) {
        set_error("rt_render_static: sorted queues and compressed state need buffers of their own (use rt_render)");
        return RT_NOT_SUPPORTED;
    }
    if (o.max_paths_in_flight > kStaticMaxPaths) {
        set_error("rt_render_static: max_paths_in_flight exceeds the static pool of 65536 paths");
        return RT_INVALID_ARG;
    }
    if (spp == 0) return RT_OK;
    if (o.trace_kernel < 0 || o.trace_kernel > 4) { set_error("rt_render_static: trace_kernel must be in [0, 4]"); return RT_INVALID_ARG; }
    if (s->dev.two_level) o.trace_kernel = 0;   // the persistent variant is single-level only
    unsigned char *base = nullptr;
    rt_status rs = static_arena(&base);
    if (rs != RT_OK) return rs;
    const uint32_t cap = o.max_paths_in_flight ? std::max<uint32_t>(o.max_paths_in_flight, 32u) : kStaticMaxPaths;
    Pool pool{};
    pool.ctrl = (Ctrl *)(base + kStaticCtrl);
    float4 *f4[8];
    for (int k = 0; k < 8; ++k) f4[k] = (float4 *)(base + kStaticF4 + k * kStaticF4Bytes);
    pool.ray_o = f4[0]; pool.ray_d = f4[1]; pool.beta = f4[2]; pool.L = f4[3];
    pool.hit = f4[4]; pool.sh_o = f4[5]; pool.sh_d = f4[6]; pool.sh_c = f4[7];
    pool.index = (uint2 *)(base + kStaticIndex);
    pool.pixel = (uint32_t *)(base + kStaticPixel);
    pool.hit_inst = (uint32_t *)(base + kStaticHitInst);
    pool.q[0] = (uint32_t *)(base + kStaticQueues);
    pool.q[1] = (uint32_t *)(base + kStaticQueues + kStaticU32Bytes);
    pool.qs = (uint32_t *)(base + kStaticQueues + 2 * kStaticU32Bytes);
    pool.capacity = cap;
    cudaStream_t st = (cudaStream_t)stream;
    // the arena keeps the previous call's contents: reset the control block
    // and rewrite the sampling table for this seed
    const int ndims = 2 + 7 * (int)(max_depth + 1);
    std::vector<HaltonDim> dims = make_dims(o.seed, ndims);
    HaltonDim *ddims = (HaltonDim *)(base + kStaticDims);
    RT_CUDA_TRY(cudaMemsetAsync(pool.ctrl, 0, sizeof(Ctrl), st));
    RT_CUDA_TRY(cudaMemcpyAsync(ddims, dims.data(), dims.size() * sizeof(HaltonDim), cudaMemcpyHostToDevice, st));
    RenderParams P;
    P.sc = s->dev;
    P.cam = make_camera(*cam);
    P.en = make_enum(cam->width, cam->height);
    P.dims = ddims;
    P.max_depth = max_depth;
    P.sigma = o.filter_sigma == 0.f ? 0.5f : o.filter_sigma;
    P.mis_mode = o.mis_mode;
    P.rr = o.rr_enable;
    const uint32_t tail = o.megakernel_only ? 0xFFFFFFFFu : (o.tail_threshold ? o.tail_threshold : 8192u);
    const uint64_t WH = (uint64_t)cam->width * cam->height;
    const int gb = o.block_size ? (int)o.block_size : 128;
    const size_t smem = stack_smem(gb);
    const int g_ray = grid_for(k_raygen, 256, cap);
    const int g_trace = grid_persistent(k_trace_ext<false>, gb, smem);
    const int g_shade = grid_persistent(k_shade<true>, gb, 0);
    const int g_shadow = grid_persistent(k_trace_shadow<false>, gb, smem);
    const TraceKernels tk = trace_kernels(false, o.trace_kernel == 1 ? 0 : o.trace_kernel, s->dev.two_level, gb);
    const int g_mega = grid_for(k_megakernel, gb, cap);
    auto t_start = std::chrono::steady_clock::now();
    uint64_t t = (uint64_t)first_iteration * WH, t_end = t + (uint64_t)spp * WH;
    rt_stats stats{};
    Ctrl host_ctrl{};
    rt_status result = RT_OK;
    while (t < t_end) {
        uint64_t n64;
        uint32_t passes = 0;
        if (t % WH != 0 || WH > cap) {
            n64 = std::min<uint64_t>({t_end - t, WH - t % WH, (uint64_t)cap});
        } else {
            uint64_t full = std::min<uint64_t>((t_end - t) / WH, cap / WH);
            if (full >= 1) { passes = (uint32_t)full; n64 = full * WH; }
            else n64 = std::min<uint64_t>(t_end - t, cap);
        }
        uint32_t n = (uint32_t)n64;
        k_raygen<<<g_ray, 256, 0, st>>>(P, pool, t, n, (uint32_t)WH, tail);
        if (!o.megakernel_only) {
            for (uint32_t v = 1; v <= max_depth + 1; ++v) {
                if (o.trace_kernel != 1) tk.ext<<<tk.grid_ext, gb, tk.smem, st>>>(s->dev, pool, nullptr);
                else k_trace_ext<false><<<g_trace, gb, smem, st>>>(s->dev, pool);
                (s->dev.lb_rec ? k_shade<true> : k_shade<false>)<<<g_shade, gb, 0, st>>>(P, pool, nullptr);
                if (o.trace_kernel != 1) tk.shadow<<<tk.grid_shadow, gb, tk.smem, st>>>(s->dev, pool, nullptr);
                else k_trace_shadow<false><<<g_shadow, gb, smem, st>>>(s->dev, pool);
                k_step_end<<<1, 1, 0, st>>>(pool);
                stats.kernel_launches += 4;
                ++stats.wavefront_steps;
            }
        }
        k_megakernel<<<g_mega, gb, 0, st>>>(P, pool);
        int g_film = grid_for(k_film, 256, passes ? WH : n);
        k_film<<<g_film, 256, 0, st>>>(pool, sum, sum2, count, t, n, (uint32_t)WH, passes);
        stats.kernel_launches += 3;
        ++stats.tail_launches;
        RT_CUDA_TRY(cudaGetLastError());
        RT_CUDA_TRY(cudaMemcpyAsync(&host_ctrl, pool.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
        RT_CUDA_TRY(cudaStreamSynchronize(st));
        t += n;
        stats.paths += n;
        ++stats.waves;
        if (host_ctrl.overflow) { set_error("BVH traversal stack overflow"); result = RT_STACK_OVERFLOW; break; }
        double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
        // stop only where an iteration is complete: the caller resumes at
        // first_iteration + stats.paths / (W H) without repeating samples
        if (t < t_end && t % WH == 0 &&
            ((o.abort_flag && *o.abort_flag) || (o.time_budget_ms > 0 && ms >= o.time_budget_ms))) {
            set_error("rt_render_static: stopped by time budget or abort flag (resume at first_iteration + "
                      "stats.paths / (width * height))");
            result = RT_TIMEOUT;
            break;
        }
    }
    stats.extension_rays = host_ctrl.ext_rays;
    stats.shadow_rays = host_ctrl.shadow_rays;
    if (o.stats) *o.stats = stats;
    return result;
}

// ---------------------------------------------------------------------------
// Batched rendering: many scenes, cameras and films in one wavefront. Slots
// of one path pool take tasks from a global index space that concatenates
// the jobs ([off_j, off_j + W_j H_j spp_j)); each slot remembers its job,
// and every kernel reads that job's parameters (scene, camera, QMC tables,
// depth) from a device table. One iteration set is captured once as a CUDA
// graph (its start index lives in device memory and is advanced by the graph
// itself) and the graph is replayed until all tasks are done; the host only
// checks the abort flag between replays.
namespace rtg {

struct BatchJob {
    RenderParams P;
    double *sum, *sum2;
    uint32_t *count;
    uint64_t off;        // first global task of the job
    uint64_t ntask;      // W * H * spp
    uint64_t film_task0; // the film's next_task when the batch started
    uint32_t WH;
};

struct BatchCtl {
    uint64_t t0;         // first global task of the current iteration set
    uint64_t total;      // tasks of all jobs
    uint32_t n;          // tasks in the current set
    uint32_t cap;
};

RT_D uint32_t find_job(const BatchJob *jobs, uint32_t njobs, uint64_t t) {
    uint32_t lo = 0, hi = njobs;
    while (hi - lo > 1) {
        uint32_t mid = (lo + hi) >> 1;
        if (jobs[mid].off <= t) lo = mid; else hi = mid;
    }
    return lo;
}

__global__ void k_batch_raygen(const BatchJob *jobs, uint32_t njobs, BatchCtl *bc, Pool pool, uint32_t *job_of) {
    const uint64_t t0 = bc->t0;
    const uint32_t n = (uint32_t)min((uint64_t)bc->cap, bc->total - min(bc->total, t0));
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
        uint64_t t = t0 + q;
        uint32_t j = find_job(jobs, njobs, t);
        const BatchJob &J = jobs[j];
        uint64_t local = t - J.off + J.film_task0;
        PathState s;
        raygen(J.P, (uint32_t)(local % J.WH), (uint32_t)(local / J.WH), s);
        store_state(pool, q, s);
        pool.q[0][q] = q;
        job_of[q] = j;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        Ctrl *c = pool.ctrl;
        bc->n = n;
        c->n_ext = n;
        c->n_next = 0;
        c->n_shadow = 0;
        c->cur = 0;
        c->fetch_ext = c->fetch_shadow = c->fetch_shade = 0;
        c->tail = 0;
    }
}

template <bool kAny>
__global__ void __launch_bounds__(128) k_batch_trace(const BatchJob *jobs, Pool pool, const uint32_t *job_of) {
    Ctrl *c = pool.ctrl;
    const uint32_t n = kAny ? c->n_shadow : c->n_ext;
    const uint32_t *queue = kAny ? pool.qs : pool.q[c->cur];
    uint32_t *fetch = kAny ? &c->fetch_shadow : &c->fetch_ext;
    bool overflow = false;
    for (;;) {
        uint32_t base = warp_fetch32(fetch);
        if (base >= n) break;
        uint32_t i = base + lane_id();
        if (i >= n) continue;
        uint32_t q = queue[i];
        const DevScene &sc = jobs[job_of[q]].P.sc;
        float4 o = kAny ? pool.sh_o[q] : pool.ray_o[q], d = kAny ? ld_shd(pool, q) : ld_dir(pool, q);
        Ray r{v3(o.x, o.y, o.z), v3(d.x, d.y, d.z), 0.f, kAny ? o.w : INFINITY};
        Hit h;
        h.prim = RT_MISS; h.inst = 0; h.t = INFINITY; h.b1 = h.b2 = 0.f;
        TraceResult tr = trace_scene<kAny>(sc, r, h);
        overflow |= tr.overflow;
        if (kAny) {
            if (h.prim == RT_MISS) {
                float4 cc = ld_shc(pool, q), L = pool.L[q];
                pool.L[q] = make_float4(L.x + cc.x, L.y + cc.y, L.z + cc.z, L.w);
            }
        } else {
            pool.hit[q] = make_float4(__uint_as_float(h.prim), h.t, h.b1, h.b2);
            pool.hit_inst[q] = h.inst;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(kAny ? &c->shadow_rays : &c->ext_rays, (unsigned long long)n);
    if (overflow) atomicOr(&c->overflow, 1u);
}

__global__ void __launch_bounds__(128) k_batch_shade(const BatchJob *jobs, Pool pool, const uint32_t *job_of) {
    Ctrl *c = pool.ctrl;
    const uint32_t n = c->n_ext;
    const uint32_t cur = c->cur;
    const uint32_t *queue = pool.q[cur];
    uint32_t *next = pool.q[cur ^ 1u];
    for (;;) {
        uint32_t base = warp_fetch32(&c->fetch_shade);
        if (base >= n) break;
        uint32_t i = base + lane_id();
        bool valid = i < n;
        uint32_t q = 0;
        int r = 0;
        if (valid) {
            q = queue[i];
            const RenderParams &P = jobs[job_of[q]].P;
            PathState s = load_state(pool, q);
            float4 hv = pool.hit[q];
            Hit h;
            h.prim = __float_as_uint(hv.x); h.inst = pool.hit_inst[q]; h.t = hv.y; h.b1 = hv.z; h.b2 = hv.w;
            ShadowRay sh;
            r = shade(P, s, h, sh);
            pool.L[q] = make_float4(s.L.x, s.L.y, s.L.z, __uint_as_float(s.prev_n));
            if (r & 1) {
                pool.ray_o[q] = make_float4(s.o.x, s.o.y, s.o.z, __uint_as_float(s.prev_cell));
                st_dir(pool, q, s.d, s.prev_pdf);
                st_beta(pool, q, s.beta, s.depth);
            }
            if (r & 2) {
                pool.sh_o[q] = make_float4(sh.o.x, sh.o.y, sh.o.z, sh.tmax);
                st_shd(pool, q, sh.d);
                st_shc(pool, q, sh.contrib);
            }
        }
        warp_append(next, &c->n_next, valid && (r & 1), q);
        warp_append(pool.qs, &c->n_shadow, valid && (r & 2), q);
    }
}

__global__ void k_batch_step_end(Pool pool) {
    Ctrl *c = pool.ctrl;
    c->n_ext = c->n_next;
    c->n_next = 0;
    c->cur ^= 1u;
    c->n_shadow = 0;
    c->fetch_ext = c->fetch_shadow = c->fetch_shade = 0;
}

// FP64 atomics into each job's film (several jobs and passes share a set).
__global__ void k_batch_film(const BatchJob *jobs, uint32_t njobs, BatchCtl *bc, Pool pool, const uint32_t *job_of) {
    const uint32_t n = bc->n;
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
        const BatchJob &J = jobs[job_of[q]];
        uint64_t local = bc->t0 + q - J.off + J.film_task0;
        uint32_t px = (uint32_t)(local % J.WH);
        float4 L = pool.L[q];
        double a = L.x, b = L.y, c = L.z;
        atomicAdd(&J.sum[3 * (size_t)px], a);
        atomicAdd(&J.sum[3 * (size_t)px + 1], b);
        atomicAdd(&J.sum[3 * (size_t)px + 2], c);
        atomicAdd(&J.sum2[3 * (size_t)px], a * a);
        atomicAdd(&J.sum2[3 * (size_t)px + 1], b * b);
        atomicAdd(&J.sum2[3 * (size_t)px + 2], c * c);
        atomicAdd(&J.count[px], 1u);
    }
}

// Advance to the next iteration set (after the film kernel has finished).
__global__ void k_batch_advance(BatchCtl *bc) { bc->t0 += bc->n; }

// ---------------------------------------------------------------------------
// Batched rendering with guiding networks inside the shared wavefront. The
// task order interleaves the jobs: block b is chunk c of job j (tasks
// [c WH_j, (c + 1) WH_j) of the job, one image's worth), blocks ordered by
// chunk, then job, so that every iteration set holds tasks of many jobs and
// each guided job collects training samples in every set. Each bounce step
// sorts the extension queue by guided job (counting sort) and runs the fused
// network kernel once per guided job over its range, writing the outputs of
// each path at its slot; shading then takes its job's mixture probability
// (zero until the job's network has trained). Training records come from
// every rec_stride-th slot and are routed to their job's batch after the set.
struct BatchBlock {
    uint64_t off;     // first global task of the block
    uint32_t job;
    uint32_t chunk;   // the block holds the job's local tasks [chunk WH, chunk WH + len)
};

struct BatchGuide {
    float3 lo, hi;        // the guide's feature bounds (its scene box)
    float *tr_feat, *tr_wi, *tr_w;   // the job's training batch
    uint32_t batch;       // its capacity
    uint32_t guided;      // 0: the job has no network
    uint32_t depth;       // the last guided vertex (BSDF sampling beyond it)
};

RT_D uint32_t find_block(const BatchBlock *blocks, uint32_t nblocks, uint64_t t) {
    uint32_t lo = 0, hi = nblocks;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (blocks[mid].off <= t) lo = mid; else hi = mid;
    }
    return lo;
}

// job and job-local task (from the film's first task of the call) of global task t
RT_D uint32_t batch_task(const BatchJob *jobs, const BatchBlock *blocks, uint32_t nblocks, uint64_t t,
                         uint64_t &local) {
    const BatchBlock &B = blocks[find_block(blocks, nblocks, t)];
    local = jobs[B.job].film_task0 + (uint64_t)B.chunk * jobs[B.job].WH + (t - B.off);
    return B.job;
}

__global__ void k_batchg_raygen(const BatchJob *jobs, const BatchBlock *blocks, uint32_t nblocks, BatchCtl *bc,
                                Pool pool, uint32_t *job_of) {
    const uint64_t t0 = bc->t0;
    const uint32_t n = (uint32_t)min((uint64_t)bc->cap, bc->total - min(bc->total, t0));
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
        uint64_t local;
        const uint32_t j = batch_task(jobs, blocks, nblocks, t0 + q, local);
        const BatchJob &J = jobs[j];
        PathState s;
        raygen(J.P, (uint32_t)(local % J.WH), (uint32_t)(local / J.WH), s);
        store_state(pool, q, s);
        pool.q[0][q] = q;
        pool.nrec[q] = 0;
        job_of[q] = j;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        Ctrl *c = pool.ctrl;
        bc->n = n;
        c->n_ext = n;
        c->n_next = 0;
        c->n_shadow = 0;
        c->cur = 0;
        c->fetch_ext = c->fetch_shadow = c->fetch_shade = 0;
        c->tail = 0;
    }
}

// sort key of a queue entry: its job when the job has a network, else njobs
struct GuidedJobKey {
    const uint32_t *job_of;
    const BatchGuide *guides;
    uint32_t njobs;
    RT_D uint32_t operator()(const Pool &, uint32_t q) const {
        const uint32_t j = job_of[q];
        return guides[j].guided ? j : njobs;
    }
};

__global__ void k_copy_u32(const uint32_t *src, uint32_t *dst, uint32_t n) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) dst[i] = src[i];
}

// network inputs of job j's paths: range [starts[j], ends[j]) of the sorted
// queue; no rows while the job's mixture probability is zero
struct JobPathFeatures {
    static constexpr bool kContiguous = false;   // output rows are path slots
    const BatchJob *jobs;
    const BatchGuide *guides;
    Pool pool;
    const uint32_t *sorted, *starts, *ends;
    const float *alpha;
    uint32_t j;
    __device__ uint32_t count() const { return alpha[j] > 0.f ? ends[j] - starts[j] : 0u; }
    __device__ uint32_t out_row(uint32_t row) const { return sorted[starts[j] + row]; }
    __device__ void operator()(uint32_t row, float f[7]) const {
        const uint32_t q = sorted[starts[j] + row];
        const RenderParams &P = jobs[j].P;
        PathState s = load_state(pool, q);
        const float4 hv = pool.hit[q];
        Hit h;
        h.prim = __float_as_uint(hv.x); h.inst = pool.hit_inst[q];
        h.t = hv.y; h.b1 = hv.z; h.b2 = hv.w;
        if (h.prim != RT_MISS && s.depth <= P.max_depth && s.depth <= guides[j].depth) {
            Vertex vx;
            setup_vertex(P.sc, s, h, vx);
            guide_features(vx.x, vx.wo, vx.ns, guides[j].lo, guides[j].hi, f);
        }
    }
};

__global__ void __launch_bounds__(kMiThreads, 1) k_guide_mlp_job(MlpWeights w, JobPathFeatures pf, __nv_bfloat16 *raw,
                                                          uint32_t *err) {
    mlp_infer_tiles(w, pf, raw, err);
}

// shading of the shared queue: a path of a guided job samples the mixture of
// its network's outputs (at its slot) with its job's probability and, on a
// recording slot, keeps the training record of each continuing vertex
__global__ void __launch_bounds__(kGuidedShadeThreads, 6) k_batchg_shade(const BatchJob *jobs, const BatchGuide *guides,
                                                         const float *alpha, Pool pool, const uint32_t *job_of,
                                                         const __nv_bfloat16 *raw, float4 *rec, uint32_t rec_stride,
                                                         uint32_t rec_slots) {
    Ctrl *c = pool.ctrl;
    const uint32_t n = c->n_ext;
    const uint32_t cur = c->cur;
    const uint32_t *queue = pool.q[cur];
    uint32_t *next = pool.q[cur ^ 1u];
    // blocks of up to kGuidedShadeThreads threads (the autotuner's block size)
    __shared__ float s_mix[kMixFields * kGuideLobes * kGuidedShadeThreads];
    const MixtureStrided mix{s_mix + threadIdx.x, blockDim.x};
    for (;;) {
        uint32_t base = warp_fetch32(&c->fetch_shade);
        if (base >= n) break;
        uint32_t i = base + lane_id();
        bool valid = i < n;
        uint32_t q = 0;
        int r = 0;
        if (valid) {
            q = queue[i];
            const uint32_t j = job_of[q];
            const RenderParams &P = jobs[j].P;
            const BatchGuide &G = guides[j];
            PathState s = load_state(pool, q);
            const bool recording = G.guided && recording_path(q, rec_stride, rec_slots);
            const uint32_t slot = q / rec_stride;
            uint32_t nr = recording ? pool.nrec[q] : 0u;
            if (nr & kRecPending) {
                nr &= ~kRecPending;
                float4 *R = rec + ((size_t)slot * kGuideMaxRec + (nr - 1)) * 4;
                R[3] = make_float4(R[3].x, s.L.x, s.L.y, s.L.z);
                pool.nrec[q] = nr;
            }
            float4 hv = pool.hit[q];
            Hit h;
            h.prim = __float_as_uint(hv.x); h.inst = pool.hit_inst[q]; h.t = hv.y; h.b1 = hv.z; h.b2 = hv.w;
            ShadowRay sh;
            GuideRecord gr;
            const uint32_t v = s.depth;
            const bool want = recording && v <= min(kGuideMaxRec, G.depth);
            const float a = G.guided && s.depth <= G.depth ? alpha[j] : 0.f;
            r = shade<true, MixtureStrided>(P, s, h, sh, a > 0.f ? raw + (size_t)kGuideOut * q : nullptr, a,
                                            want ? &gr : nullptr, G.lo, G.hi, mix);
            pool.L[q] = make_float4(s.L.x, s.L.y, s.L.z, __uint_as_float(s.prev_n));
            if (r & 1) {
                pool.ray_o[q] = make_float4(s.o.x, s.o.y, s.o.z, __uint_as_float(s.prev_cell));
                st_dir(pool, q, s.d, s.prev_pdf);
                st_beta(pool, q, s.beta, s.depth);
                if (want) {
                    float4 *R = rec + ((size_t)slot * kGuideMaxRec + (v - 1)) * 4;
                    R[0] = make_float4(gr.feat[0], gr.feat[1], gr.feat[2], gr.feat[3]);
                    R[1] = make_float4(gr.feat[4], gr.feat[5], gr.feat[6], gr.wi.x);
                    R[2] = make_float4(gr.wi.y, gr.wi.z, gr.beta.x, gr.beta.y);
                    R[3] = make_float4(gr.beta.z, 0.f, 0.f, 0.f);
                    pool.nrec[q] = v | kRecPending;
                }
            }
            if (r & 2) {
                pool.sh_o[q] = make_float4(sh.o.x, sh.o.y, sh.o.z, sh.tmax);
                st_shd(pool, q, sh.d);
                st_shc(pool, q, sh.contrib);
            }
        }
        warp_append(next, &c->n_next, valid && (r & 1), q);
        warp_append(pool.qs, &c->n_shadow, valid && (r & 2), q);
    }
}

__global__ void k_batchg_film(const BatchJob *jobs, const BatchBlock *blocks, uint32_t nblocks, BatchCtl *bc, Pool pool,
                              const uint32_t *job_of) {
    const uint32_t n = bc->n;
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
        uint64_t local;
        const uint32_t j = batch_task(jobs, blocks, nblocks, bc->t0 + q, local);
        const BatchJob &J = jobs[j];
        const uint32_t px = (uint32_t)(local % J.WH);
        const float4 L = pool.L[q];
        const double a = L.x, b = L.y, cc = L.z;
        atomicAdd(&J.sum[3 * (size_t)px], a);
        atomicAdd(&J.sum[3 * (size_t)px + 1], b);
        atomicAdd(&J.sum[3 * (size_t)px + 2], cc);
        atomicAdd(&J.sum2[3 * (size_t)px], a * a);
        atomicAdd(&J.sum2[3 * (size_t)px + 1], b * b);
        atomicAdd(&J.sum2[3 * (size_t)px + 2], cc * cc);
        atomicAdd(&J.count[px], 1u);
    }
}

// training samples of the set's recording slots, routed to their job's batch
// (the sampled f cos Li / p of each finished record, as k_guide_collect)
__global__ void k_batchg_collect(const BatchGuide *guides, BatchCtl *bc, Pool pool, const uint32_t *job_of,
                                 const float4 *rec, uint32_t rec_stride, uint32_t rec_slots, uint32_t *ntrain) {
    const uint32_t n = bc->n;
    const uint32_t slots = min(rec_slots, (n + rec_stride - 1) / rec_stride);
    for (uint32_t k0 = blockIdx.x * blockDim.x + threadIdx.x; k0 < slots; k0 += gridDim.x * blockDim.x) {
        const uint32_t q = k0 * rec_stride;
        const uint32_t j = job_of[q];
        const BatchGuide &G = guides[j];
        if (!G.guided) continue;
        const uint32_t nr = pool.nrec[q];
        const uint32_t complete = (nr & kRecPending) ? (nr & ~kRecPending) - 1 : nr;
        const float4 L = pool.L[q];
        for (uint32_t k = 0; k < complete; ++k) {
            const float4 *R = rec + ((size_t)k0 * kGuideMaxRec + k) * 4;
            const float4 r0 = R[0], r1 = R[1], r2 = R[2], r3 = R[3];
            const float bx = r2.z, by = r2.w, bz = r3.x;
            const float ax = bx > 0.f ? fmaxf(L.x - r3.y, 0.f) / bx : 0.f;
            const float ay = by > 0.f ? fmaxf(L.y - r3.z, 0.f) / by : 0.f;
            const float az = bz > 0.f ? fmaxf(L.z - r3.w, 0.f) / bz : 0.f;
            const float w = lum(v3(ax, ay, az));
            if (!(w > 0.f) || !isfinite(w)) continue;
            const uint32_t idx = atomicAdd(&ntrain[j], 1u);
            if (idx >= G.batch) continue;
            const float f[7] = {r0.x, r0.y, r0.z, r0.w, r1.x, r1.y, r1.z};
            for (int e = 0; e < 7; ++e) G.tr_feat[7 * (size_t)idx + e] = f[e];
            G.tr_wi[3 * (size_t)idx] = r1.w;
            G.tr_wi[3 * (size_t)idx + 1] = r2.x;
            G.tr_wi[3 * (size_t)idx + 2] = r2.y;
            G.tr_w[idx] = w;
        }
    }
}

}  // namespace rtg

static rt_status render_batch_shared(const rt_render_job *jobs, int32_t njobs, const rt_render_opts *opts_in,
                                     void *stream);
static rt_status render_batch_guided(const rt_render_job *jobs, int32_t njobs, const rt_render_opts *opts_in,
                                     void *stream);

extern "C" rt_status rt_render_batch(const rt_render_job *jobs, int32_t njobs, const rt_render_opts *opts_in,
                                     void *stream) {
    if (!jobs || njobs <= 0) { set_error("rt_render_batch: no jobs"); return RT_INVALID_ARG; }
    if (opts_in && opts_in->guide) {
        set_error("rt_render_batch: guiding networks go with the jobs (rt_render_job.guide)");
        return RT_NOT_SUPPORTED;
    }
    for (int32_t j = 0; j < njobs; ++j)
        if (jobs[j].guide) return render_batch_guided(jobs, njobs, opts_in, stream);
    return render_batch_shared(jobs, njobs, opts_in, stream);
}

static rt_status render_batch_shared(const rt_render_job *jobs, int32_t njobs, const rt_render_opts *opts_in,
                                     void *stream) {
    rt_render_opts o{};
    if (opts_in) o = *opts_in;
    if (!valid_block(o.block_size)) { set_error("rt_render_batch: block_size must be 0 or a multiple of 32 up to 128"); return RT_INVALID_ARG; }
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<BatchJob> hj((size_t)njobs);
    uint64_t total = 0;
    uint32_t maxd = 1;
    int ndims_max = 0;
    for (int32_t j = 0; j < njobs; ++j) {
        const rt_render_job &J = jobs[j];
        if (!J.scene || !J.film || J.scene->host_only || J.camera.width != J.film->W || J.camera.height != J.film->H ||
            J.max_depth < 1 || J.max_depth > (uint32_t)kMaxDepth) {
            set_error("rt_render_batch: invalid job " + std::to_string(j));
            return RT_INVALID_ARG;
        }
        maxd = std::max(maxd, J.max_depth);
        ndims_max = std::max(ndims_max, 2 + 7 * (int)(J.max_depth + 1));
    }
    // one Halton table (the longest) and one job table for the batch
    struct Scratch {
        std::vector<void *> ptrs;
        ~Scratch() { for (void *p : ptrs) cudaFree(p); }
    } scratch;
    std::vector<HaltonDim> dims = make_dims(o.seed, ndims_max);
    HaltonDim *ddims = nullptr;
    RT_CUDA_TRY(cudaMalloc(&ddims, dims.size() * sizeof(HaltonDim)));
    scratch.ptrs.push_back(ddims);
    RT_CUDA_TRY(cudaMemcpyAsync(ddims, dims.data(), dims.size() * sizeof(HaltonDim), cudaMemcpyHostToDevice, st));
    for (int32_t j = 0; j < njobs; ++j) {
        const rt_render_job &J = jobs[j];
        BatchJob &B = hj[(size_t)j];
        B.P.sc = J.scene->dev;
        B.P.cam = make_camera(J.camera);
        B.P.en = make_enum(J.camera.width, J.camera.height);
        B.P.dims = ddims;
        B.P.max_depth = J.max_depth;
        B.P.sigma = o.filter_sigma == 0.f ? 0.5f : o.filter_sigma;
        B.P.mis_mode = o.mis_mode;
        B.P.rr = o.rr_enable;
        B.sum = J.film->sum;
        B.sum2 = J.film->sum2;
        B.count = J.film->count;
        B.WH = J.camera.width * J.camera.height;
        B.off = total;
        // up to the end of pass (next iteration + spp): a film stopped inside
        // a pass first completes it
        B.ntask = (J.film->next_task / B.WH + (uint64_t)J.spp) * B.WH - J.film->next_task;
        B.film_task0 = J.film->next_task;
        total += B.ntask;
    }
    if (total == 0) return RT_OK;
    const uint32_t cap = std::max<uint32_t>(32u, o.max_paths_in_flight ? o.max_paths_in_flight : default_capacity(total));
    BatchJob *djobs = nullptr;
    BatchCtl *dctl = nullptr;
    uint32_t *job_of = nullptr;
    RT_CUDA_TRY(cudaMalloc(&djobs, hj.size() * sizeof(BatchJob)));
    scratch.ptrs.push_back(djobs);
    RT_CUDA_TRY(cudaMalloc(&dctl, sizeof(BatchCtl)));
    scratch.ptrs.push_back(dctl);
    RT_CUDA_TRY(cudaMalloc(&job_of, sizeof(uint32_t) * cap));
    scratch.ptrs.push_back(job_of);
    RT_CUDA_TRY(cudaMemcpyAsync(djobs, hj.data(), hj.size() * sizeof(BatchJob), cudaMemcpyHostToDevice, st));
    BatchCtl hc{0ull, total, 0u, cap};
    RT_CUDA_TRY(cudaMemcpyAsync(dctl, &hc, sizeof hc, cudaMemcpyHostToDevice, st));
    PoolAlloc pa;
    rt_status rs = ensure_pool(pa, cap);
    if (rs != RT_OK) return rs;
    Pool pool = pa.view;
    RT_CUDA_TRY(cudaMemsetAsync(pool.ctrl, 0, sizeof(Ctrl), st));
    const int gb = o.block_size ? (int)o.block_size : 128;
    const int g_ray = grid_for(k_batch_raygen, 256, cap);
    const int g_trace = grid_persistent(k_batch_trace<false>, gb, 0);
    const int g_shade = grid_persistent(k_batch_shade, gb, 0);
    const int g_film = grid_for(k_batch_film, 256, cap);
    // capture one iteration set
    cudaStream_t cs = nullptr;
    RT_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    RT_CUDA_TRY(cudaStreamSynchronize(st));
    RT_CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    k_batch_raygen<<<g_ray, 256, 0, cs>>>(djobs, (uint32_t)njobs, dctl, pool, job_of);
    for (uint32_t v = 1; v <= maxd + 1; ++v) {
        k_batch_trace<false><<<g_trace, gb, 0, cs>>>(djobs, pool, job_of);
        k_batch_shade<<<g_shade, gb, 0, cs>>>(djobs, pool, job_of);
        k_batch_trace<true><<<g_trace, gb, 0, cs>>>(djobs, pool, job_of);
        k_batch_step_end<<<1, 1, 0, cs>>>(pool);
    }
    k_batch_film<<<g_film, 256, 0, cs>>>(djobs, (uint32_t)njobs, dctl, pool, job_of);
    k_batch_advance<<<1, 1, 0, cs>>>(dctl);
    cudaError_t ce = cudaStreamEndCapture(cs, &graph);
    if (ce != cudaSuccess) { cudaStreamDestroy(cs); return cuda_status(ce, "rt_render_batch: graph capture"); }
    ce = cudaGraphInstantiate(&exec, graph, 0);
    if (ce != cudaSuccess) { cudaGraphDestroy(graph); cudaStreamDestroy(cs); return cuda_status(ce, "rt_render_batch: instantiate"); }
    const uint64_t sets = (total + cap - 1) / cap;
    rt_stats stats{};
    rt_status result = RT_OK;
    uint64_t done_sets = 0;
    auto t_start = std::chrono::steady_clock::now();
    for (; done_sets < sets; ++done_sets) {
        ce = cudaGraphLaunch(exec, st);
        if (ce != cudaSuccess) { result = cuda_status(ce, "rt_render_batch: graph launch"); break; }
        stats.kernel_launches += 3 + 4 * (maxd + 1);
        bool check = (o.abort_flag || o.time_budget_ms > 0) && done_sets + 1 < sets;
        if (check) {
            cudaStreamSynchronize(st);
            double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
            if ((o.abort_flag && *o.abort_flag) || (o.time_budget_ms > 0 && ms >= o.time_budget_ms)) {
                ++done_sets;
                set_error("rt_render_batch: stopped by time budget or abort flag");
                result = RT_TIMEOUT;
                break;
            }
        }
    }
    Ctrl hctl{};
    cudaMemcpyAsync(&hctl, pool.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st);
    cudaError_t se = cudaStreamSynchronize(st);
    cudaGraphExecDestroy(exec);
    cudaGraphDestroy(graph);
    cudaStreamDestroy(cs);
    if (se != cudaSuccess) return cuda_status(se, "rt_render_batch");
    if (hctl.overflow && result == RT_OK) { set_error("BVH traversal stack overflow"); result = RT_STACK_OVERFLOW; }
    // films advance by the tasks of theirs that were completed
    const uint64_t done_tasks = std::min<uint64_t>(total, done_sets * (uint64_t)cap);
    for (int32_t j = 0; j < njobs; ++j) {
        const BatchJob &B = hj[(size_t)j];
        uint64_t dj = done_tasks > B.off ? std::min<uint64_t>(B.ntask, done_tasks - B.off) : 0;
        jobs[j].film->next_task += dj;
    }
    stats.paths = done_tasks;
    stats.waves = (uint32_t)done_sets;
    stats.wavefront_steps = (uint32_t)(done_sets * (maxd + 1));
    stats.extension_rays = hctl.ext_rays;
    stats.shadow_rays = hctl.shadow_rays;
    if (o.stats) *o.stats = stats;
    return result;
}

// All jobs of a batch in which some carry a guiding network: one shared
// wavefront over interleaved tasks (see BatchBlock), the set captured once
// as a CUDA graph with one network launch per guided job and bounce step;
// between replays every guided job whose network is due trains on the
// samples its paths left in the set.
static rt_status render_batch_guided(const rt_render_job *jobs, int32_t njobs, const rt_render_opts *opts_in,
                                     void *stream) {
    rt_render_opts o{};
    if (opts_in) o = *opts_in;
    if (!valid_block(o.block_size)) { set_error("rt_render_batch: block_size must be 0 or a multiple of 32 up to 128"); return RT_INVALID_ARG; }
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<BatchJob> hj((size_t)njobs);
    std::vector<BatchGuide> hg((size_t)njobs);
    uint32_t maxd = 1;
    int ndims_max = 0;
    for (int32_t j = 0; j < njobs; ++j) {
        const rt_render_job &J = jobs[j];
        if (!J.scene || !J.film || J.scene->host_only || J.camera.width != J.film->W || J.camera.height != J.film->H ||
            J.max_depth < 1 || J.max_depth > (uint32_t)kMaxDepth) {
            set_error("rt_render_batch: invalid job " + std::to_string(j));
            return RT_INVALID_ARG;
        }
        maxd = std::max(maxd, J.max_depth);
        ndims_max = std::max(ndims_max, 2 + 7 * (int)(J.max_depth + 1));
    }
    struct Scratch {
        std::vector<void *> ptrs;
        ~Scratch() { for (void *p : ptrs) cudaFree(p); }
    } scratch;
    auto dalloc = [&](void **p, size_t bytes) -> rt_status {
        if (cudaMalloc(p, bytes) != cudaSuccess) { set_error("rt_render_batch: out of device memory"); return RT_OOM; }
        scratch.ptrs.push_back(*p);
        return RT_OK;
    };
    rt_status rs;
    std::vector<HaltonDim> dims = make_dims(o.seed, ndims_max);
    HaltonDim *ddims = nullptr;
    if ((rs = dalloc((void **)&ddims, dims.size() * sizeof(HaltonDim))) != RT_OK) return rs;
    RT_CUDA_TRY(cudaMemcpyAsync(ddims, dims.data(), dims.size() * sizeof(HaltonDim), cudaMemcpyHostToDevice, st));
    // jobs, their chunks, and the interleaved block table
    uint64_t total = 0;
    uint32_t max_chunks = 0;
    std::vector<uint32_t> nchunks((size_t)njobs);
    for (int32_t j = 0; j < njobs; ++j) {
        const rt_render_job &J = jobs[j];
        BatchJob &B = hj[(size_t)j];
        B.P.sc = J.scene->dev;
        B.P.cam = make_camera(J.camera);
        B.P.en = make_enum(J.camera.width, J.camera.height);
        B.P.dims = ddims;
        B.P.max_depth = J.max_depth;
        B.P.sigma = o.filter_sigma == 0.f ? 0.5f : o.filter_sigma;
        B.P.mis_mode = o.mis_mode;
        B.P.rr = o.rr_enable;
        B.sum = J.film->sum;
        B.sum2 = J.film->sum2;
        B.count = J.film->count;
        B.WH = J.camera.width * J.camera.height;
        B.ntask = (J.film->next_task / B.WH + (uint64_t)J.spp) * B.WH - J.film->next_task;
        B.film_task0 = J.film->next_task;
        B.off = 0;
        nchunks[(size_t)j] = (uint32_t)((B.ntask + B.WH - 1) / B.WH);
        max_chunks = std::max(max_chunks, nchunks[(size_t)j]);
        total += B.ntask;
    }
    if (total == 0) return RT_OK;
    std::vector<BatchBlock> blocks;
    for (uint32_t c = 0; c < max_chunks; ++c)
        for (int32_t j = 0; j < njobs; ++j) {
            if (c >= nchunks[(size_t)j]) continue;
            BatchBlock b;
            b.off = blocks.empty() ? 0 : blocks.back().off +
                                          std::min<uint64_t>(hj[blocks.back().job].WH,
                                                             hj[blocks.back().job].ntask -
                                                                 (uint64_t)blocks.back().chunk * hj[blocks.back().job].WH);
            b.job = (uint32_t)j;
            b.chunk = c;
            blocks.push_back(b);
        }
    // set size: the user's pool, else 2^23 paths (the per-set graph replay,
    // host round trip and launch drains spread over more paths; measured for
    // 64 jobs with 8 / 64 guided: 2^21 363 / 253, 2^22 418 / 301, 2^23 462 /
    // 333 Mpaths/s)
    const uint32_t cap = std::max<uint32_t>(
        32u, (uint32_t)std::min<uint64_t>(total, o.max_paths_in_flight ? o.max_paths_in_flight : (1u << 23)));
    // guides: bounds, training batches, mixture probabilities
    uint32_t nguided = 0;
    std::vector<float> alpha_h((size_t)njobs, 0.f);
    for (int32_t j = 0; j < njobs; ++j) {
        BatchGuide &G = hg[(size_t)j];
        G = BatchGuide{};
        rt_guide *gd = jobs[j].guide;
        if (!gd) continue;
        ++nguided;
        G.guided = 1;
        guide_bounds(gd, G.lo, G.hi);
        G.batch = guide_batch(gd);
        G.depth = guide_depth(gd);
        if ((rs = dalloc((void **)&G.tr_feat, (size_t)G.batch * 7 * 4)) != RT_OK ||
            (rs = dalloc((void **)&G.tr_wi, (size_t)G.batch * 3 * 4)) != RT_OK ||
            (rs = dalloc((void **)&G.tr_w, (size_t)G.batch * 4)) != RT_OK)
            return rs;
        alpha_h[(size_t)j] = guide_trained(gd) ? guide_alpha(gd) : 0.f;
    }
    // training records: every rec_stride-th slot of the set, at most 2^18
    const uint32_t rec_slots = std::min<uint32_t>(cap, 1u << 18);
    const uint32_t rec_stride = std::max<uint32_t>(1u, (cap + rec_slots - 1) / rec_slots);
    BatchJob *djobs = nullptr;
    BatchGuide *dguides = nullptr;
    BatchBlock *dblocks = nullptr;
    BatchCtl *dctl = nullptr;
    float *dalpha = nullptr;
    uint32_t *job_of = nullptr, *ntrain = nullptr, *hist = nullptr, *starts = nullptr, *sorted = nullptr;
    float4 *rec = nullptr;
    __nv_bfloat16 *raw = nullptr;
    const uint32_t nkeys = (uint32_t)njobs + 1;
    if ((rs = dalloc((void **)&djobs, hj.size() * sizeof(BatchJob))) != RT_OK ||
        (rs = dalloc((void **)&dguides, hg.size() * sizeof(BatchGuide))) != RT_OK ||
        (rs = dalloc((void **)&dblocks, blocks.size() * sizeof(BatchBlock))) != RT_OK ||
        (rs = dalloc((void **)&dctl, sizeof(BatchCtl))) != RT_OK ||
        (rs = dalloc((void **)&dalpha, sizeof(float) * (size_t)njobs)) != RT_OK ||
        (rs = dalloc((void **)&job_of, sizeof(uint32_t) * (size_t)cap)) != RT_OK ||
        (rs = dalloc((void **)&ntrain, sizeof(uint32_t) * (size_t)njobs)) != RT_OK ||
        (rs = dalloc((void **)&hist, sizeof(uint32_t) * (size_t)nkeys)) != RT_OK ||
        (rs = dalloc((void **)&starts, sizeof(uint32_t) * (size_t)nkeys)) != RT_OK ||
        (rs = dalloc((void **)&sorted, sizeof(uint32_t) * (size_t)cap)) != RT_OK ||
        (rs = dalloc((void **)&rec, sizeof(float4) * 4 * kGuideMaxRec * (size_t)rec_slots)) != RT_OK ||
        (rs = dalloc((void **)&raw, sizeof(__nv_bfloat16) * kGuideOut * (size_t)cap)) != RT_OK)
        return rs;
    uint32_t *nrec = nullptr;
    if ((rs = dalloc((void **)&nrec, sizeof(uint32_t) * (size_t)cap)) != RT_OK) return rs;
    RT_CUDA_TRY(cudaMemcpyAsync(djobs, hj.data(), hj.size() * sizeof(BatchJob), cudaMemcpyHostToDevice, st));
    RT_CUDA_TRY(cudaMemcpyAsync(dguides, hg.data(), hg.size() * sizeof(BatchGuide), cudaMemcpyHostToDevice, st));
    RT_CUDA_TRY(cudaMemcpyAsync(dblocks, blocks.data(), blocks.size() * sizeof(BatchBlock), cudaMemcpyHostToDevice, st));
    RT_CUDA_TRY(cudaMemcpyAsync(dalpha, alpha_h.data(), sizeof(float) * (size_t)njobs, cudaMemcpyHostToDevice, st));
    BatchCtl hc{0ull, total, 0u, cap};
    RT_CUDA_TRY(cudaMemcpyAsync(dctl, &hc, sizeof hc, cudaMemcpyHostToDevice, st));
    PoolAlloc pa;
    if ((rs = ensure_pool(pa, cap)) != RT_OK) return rs;
    Pool pool = pa.view;
    pool.nrec = nrec;
    RT_CUDA_TRY(cudaMemsetAsync(pool.ctrl, 0, sizeof(Ctrl), st));
    if ((rs = mlp_kernel_attr((const void *)k_guide_mlp_job, kMlpInferSmem)) != RT_OK) return rs;
    const int gb = o.block_size ? (int)o.block_size : 128;
    const uint32_t nb = (uint32_t)blocks.size();
    const int g_ray = grid_for(k_batchg_raygen, 256, cap);
    const int g_trace = grid_persistent(k_batch_trace<false>, gb, 0);
    const int g_shade = grid_persistent(k_batchg_shade, gb, 0);
    const int g_film = grid_for(k_batchg_film, 256, cap);
    const int g_hist = grid_for(k_sort_scatter<GuidedJobKey>, 256, cap);
    const int g_coll = grid_for(k_batchg_collect, 256, rec_slots);
    GuidedJobKey key{job_of, dguides, (uint32_t)njobs};
    // capture one iteration set
    cudaStream_t cs = nullptr;
    RT_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    struct StreamGuard {
        cudaStream_t s;
        ~StreamGuard() { if (s) cudaStreamDestroy(s); }
    } guard{cs};
    // side streams: parallel branches of the set graph (the networks of
    // different jobs) and concurrent training steps between replays
    constexpr int kSide = 8;
    struct SideStreams {
        cudaStream_t s[kSide] = {};
        cudaEvent_t fork = nullptr, join[kSide] = {};
        ~SideStreams() {
            for (cudaStream_t x : s) if (x) cudaStreamDestroy(x);
            for (cudaEvent_t e : join) if (e) cudaEventDestroy(e);
            if (fork) cudaEventDestroy(fork);
        }
    } ss;
    for (int b = 0; b < kSide; ++b) {
        RT_CUDA_TRY(cudaStreamCreateWithFlags(&ss.s[b], cudaStreamNonBlocking));
        RT_CUDA_TRY(cudaEventCreateWithFlags(&ss.join[b], cudaEventDisableTiming));
    }
    RT_CUDA_TRY(cudaEventCreateWithFlags(&ss.fork, cudaEventDisableTiming));
    cudaStream_t *side = ss.s;
    cudaEvent_t fork_ev = ss.fork, *join_ev = ss.join;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    RT_CUDA_TRY(cudaStreamSynchronize(st));
    RT_CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    cudaMemsetAsync(ntrain, 0, sizeof(uint32_t) * (size_t)njobs, cs);
    k_batchg_raygen<<<g_ray, 256, 0, cs>>>(djobs, dblocks, nb, dctl, pool, job_of);
    // the guided jobs' networks run at their vertices 1..guide depth (paths
    // of a set advance one vertex per bounce step)
    uint32_t max_gdepth = 0, net_launches = 0;
    for (int32_t j = 0; j < njobs; ++j)
        if (jobs[j].guide) {
            const uint32_t d = std::min(guide_depth(jobs[j].guide), jobs[j].max_depth);
            max_gdepth = std::max(max_gdepth, d);
            net_launches += d;
        }
    for (uint32_t v = 1; v <= maxd + 1; ++v) {
        k_batch_trace<false><<<g_trace, gb, 0, cs>>>(djobs, pool, job_of);
        if (v <= maxd && v <= max_gdepth) {
            // the network of each guided job over its paths (not at the last
            // vertex, which only adds emission, nor past its guide depth)
            cudaMemsetAsync(hist, 0, sizeof(uint32_t) * nkeys, cs);
            k_sort_hist<GuidedJobKey><<<g_hist, 256, nkeys * sizeof(uint32_t), cs>>>(key, pool, nkeys, hist);
            k_sort_scan<<<1, 1024, 0, cs>>>(pool, nkeys, hist);
            k_copy_u32<<<1, 256, 0, cs>>>(hist, starts, nkeys);
            k_sort_scatter<GuidedJobKey><<<g_hist, 256, 0, cs>>>(key, pool, hist, sorted);
            // the jobs' networks in up to kSide parallel branches of the graph
            RT_CUDA_TRY(cudaEventRecord(fork_ev, cs));
            for (int b = 0; b < kSide; ++b) RT_CUDA_TRY(cudaStreamWaitEvent(side[b], fork_ev, 0));
            int k = 0;
            for (int32_t j = 0; j < njobs; ++j) {
                if (!jobs[j].guide || v > std::min(guide_depth(jobs[j].guide), jobs[j].max_depth)) continue;
                const JobPathFeatures pf{djobs, dguides, pool, sorted, starts, hist, dalpha, (uint32_t)j};
                k_guide_mlp_job<<<sm_count(), kMiThreads, kMlpInferSmem, side[k++ % kSide]>>>(
                    guide_weights(jobs[j].guide), pf, raw, guide_err(jobs[j].guide));
            }
            for (int b = 0; b < kSide; ++b) {
                RT_CUDA_TRY(cudaEventRecord(join_ev[b], side[b]));
                RT_CUDA_TRY(cudaStreamWaitEvent(cs, join_ev[b], 0));
            }
        }
        k_batchg_shade<<<g_shade, gb, 0, cs>>>(djobs, dguides, dalpha, pool, job_of, raw, rec, rec_stride, rec_slots);
        k_batch_trace<true><<<g_trace, gb, 0, cs>>>(djobs, pool, job_of);
        k_batch_step_end<<<1, 1, 0, cs>>>(pool);
    }
    k_batchg_film<<<g_film, 256, 0, cs>>>(djobs, dblocks, nb, dctl, pool, job_of);
    k_batchg_collect<<<g_coll, 256, 0, cs>>>(dguides, dctl, pool, job_of, rec, rec_stride, rec_slots, ntrain);
    k_batch_advance<<<1, 1, 0, cs>>>(dctl);
    cudaError_t ce = cudaStreamEndCapture(cs, &graph);
    if (ce != cudaSuccess) return cuda_status(ce, "rt_render_batch: graph capture");
    ce = cudaGraphInstantiate(&exec, graph, 0);
    if (ce != cudaSuccess) { cudaGraphDestroy(graph); return cuda_status(ce, "rt_render_batch: instantiate"); }
    struct GraphGuard {
        cudaGraph_t g;
        cudaGraphExec_t e;
        ~GraphGuard() { if (e) cudaGraphExecDestroy(e); if (g) cudaGraphDestroy(g); }
    } gguard{graph, exec};
    const uint64_t sets = (total + cap - 1) / cap;
    // memset, raygen; per bounce step trace, shade, shadow, step end, and
    // before each shade but the last the job sort (5) and the networks; film,
    // collect, advance
    const uint32_t launches_per_set = 2 + 4 * (maxd + 1) + std::min(maxd, max_gdepth) * 5 + net_launches + 3;
    std::vector<uint32_t> ntrain_h((size_t)njobs);
    // After its warm-up a job's network takes one step per 16 training
    // batches of its own paths rendered (the single-scene schedule), not one
    // per set: its paths in set s are the overlap of its blocks with the
    // set's task range [s cap, (s + 1) cap).
    std::vector<uint64_t> since_step((size_t)njobs, 0);
    std::vector<uint64_t> in_set((size_t)njobs);
    auto block_len = [&](const BatchBlock &b) {
        return std::min<uint64_t>(hj[b.job].WH, hj[b.job].ntask - (uint64_t)b.chunk * hj[b.job].WH);
    };
    rt_stats stats{};
    rt_status result = RT_OK;
    uint64_t done_sets = 0;
    const auto t_start = std::chrono::steady_clock::now();
    for (; done_sets < sets; ++done_sets) {
        {
            std::fill(in_set.begin(), in_set.end(), 0);
            const uint64_t s0 = done_sets * cap, s1 = std::min<uint64_t>(total, s0 + cap);
            for (const BatchBlock &b : blocks) {
                const uint64_t a = std::max(b.off, s0), e = std::min(b.off + block_len(b), s1);
                if (a < e) in_set[b.job] += e - a;
            }
        }
        ce = cudaGraphLaunch(exec, st);
        if (ce != cudaSuccess) { result = cuda_status(ce, "rt_render_batch: graph launch"); break; }
        stats.kernel_launches += launches_per_set;
        RT_CUDA_TRY(cudaMemcpyAsync(ntrain_h.data(), ntrain, sizeof(uint32_t) * (size_t)njobs, cudaMemcpyDeviceToHost, st));
        RT_CUDA_TRY(cudaStreamSynchronize(st));
        // training after the set, each due network on its own samples; the
        // networks are independent, so their steps run on the side streams
        bool alpha_changed = false;
        RT_CUDA_TRY(cudaEventRecord(fork_ev, st));
        for (int b = 0; b < kSide; ++b) RT_CUDA_TRY(cudaStreamWaitEvent(side[b], fork_ev, 0));
        int k = 0;
        for (int32_t j = 0; j < njobs; ++j) {
            rt_guide *gd = jobs[j].guide;
            if (!gd) continue;
            if ((rs = guide_check(gd, st)) != RT_OK) return rs;
            const uint32_t nt = std::min(ntrain_h[(size_t)j], hg[(size_t)j].batch);
            since_step[(size_t)j] += in_set[(size_t)j];
            const uint64_t per_step = 16ull * std::max(guide_batch(gd), 32u);
            const bool due = guide_young(gd) || since_step[(size_t)j] >= per_step;
            if (nt >= 256 && due && guide_should_train(gd)) {
                since_step[(size_t)j] = guide_young(gd) ? 0 : since_step[(size_t)j] - per_step;
                const BatchGuide &G = hg[(size_t)j];
                if ((rs = guide_train_async(gd, G.tr_feat, G.tr_wi, G.tr_w, nt, side[k++ % kSide])) != RT_OK) return rs;
                stats.kernel_launches += 40;
                const float a = guide_alpha(gd);
                if (alpha_h[(size_t)j] != a) { alpha_h[(size_t)j] = a; alpha_changed = true; }
            }
        }
        for (int b = 0; b < kSide; ++b) {
            RT_CUDA_TRY(cudaEventRecord(join_ev[b], side[b]));
            RT_CUDA_TRY(cudaStreamWaitEvent(st, join_ev[b], 0));
        }
        if (alpha_changed)
            RT_CUDA_TRY(cudaMemcpyAsync(dalpha, alpha_h.data(), sizeof(float) * (size_t)njobs, cudaMemcpyHostToDevice, st));
        const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
        if (done_sets + 1 < sets && ((o.abort_flag && *o.abort_flag) || (o.time_budget_ms > 0 && ms >= o.time_budget_ms))) {
            ++done_sets;
            set_error("rt_render_batch: stopped by time budget or abort flag");
            result = RT_TIMEOUT;
            break;
        }
    }
    Ctrl hctl{};
    RT_CUDA_TRY(cudaMemcpyAsync(&hctl, pool.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
    RT_CUDA_TRY(cudaStreamSynchronize(st));
    if (hctl.overflow && result == RT_OK) { set_error("BVH traversal stack overflow"); result = RT_STACK_OVERFLOW; }
    // films advance by the tasks of theirs that were completed: the blocks
    // wholly before the end of the completed sets, and part of the last one
    const uint64_t done_tasks = std::min<uint64_t>(total, done_sets * (uint64_t)cap);
    std::vector<uint64_t> done_j((size_t)njobs, 0);
    for (const BatchBlock &b : blocks) {
        if (b.off >= done_tasks) break;
        const uint64_t len = std::min<uint64_t>(hj[b.job].WH, hj[b.job].ntask - (uint64_t)b.chunk * hj[b.job].WH);
        done_j[b.job] += std::min<uint64_t>(len, done_tasks - b.off);
    }
    for (int32_t j = 0; j < njobs; ++j) jobs[j].film->next_task += done_j[(size_t)j];
    stats.paths = done_tasks;
    stats.waves = (uint32_t)done_sets;
    stats.wavefront_steps = (uint32_t)(done_sets * (maxd + 1));
    stats.extension_rays = hctl.ext_rays;
    stats.shadow_rays = hctl.shadow_rays;
    if (o.stats) *o.stats = stats;
    return result;
}

extern "C" rt_status rt_autotune(const rt_render_job *jobs, int32_t njobs, uint32_t sample_spp, rt_render_opts *opts,
                                 void *stream) {
    if (!jobs || njobs <= 0 || !opts || sample_spp == 0) { set_error("rt_autotune: invalid argument"); return RT_INVALID_ARG; }
    for (int32_t j = 0; j < njobs; ++j)
        if (jobs[j].guide) { set_error("rt_autotune: jobs with a guiding network are not tuned"); return RT_NOT_SUPPORTED; }
    cudaStream_t st = (cudaStream_t)stream;
    struct Cand { uint32_t cap, tail; int32_t tk; };
    std::vector<Cand> cands;
    const uint32_t caps[4] = {1u << 20, 1u << 22, 1u << 24, 1u << 26};
    if (njobs == 1) {
        const uint32_t tails[3] = {1u, 8192u, 65536u};   // 1: the megakernel never takes over
        for (uint32_t c : caps)
            for (uint32_t t : tails)
                for (int32_t k = 0; k < 2; ++k) cands.push_back({c, t, k});
    } else {
        for (uint32_t c : caps) cands.push_back({c, 0u, 0});
    }
    double best = 1e300;
    Cand pick = cands[0];
    for (const Cand &c : cands) {
        rt_render_opts o = *opts;
        o.max_paths_in_flight = c.cap;
        o.tail_threshold = c.tail;
        o.trace_kernel = c.tk;
        o.stats = nullptr;
        o.profile = 0;
        RT_CUDA_TRY(cudaStreamSynchronize(st));
        auto t0 = std::chrono::steady_clock::now();
        rt_status s;
        if (njobs == 1) s = rt_render(jobs[0].scene, &jobs[0].camera, sample_spp, jobs[0].max_depth, jobs[0].film, &o, stream);
        else {
            std::vector<rt_render_job> js(jobs, jobs + njobs);
            for (auto &j : js) j.spp = sample_spp;
            s = rt_render_batch(js.data(), njobs, &o, stream);
        }
        if (s != RT_OK) return s;
        RT_CUDA_TRY(cudaStreamSynchronize(st));
        double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        if (ms < best) { best = ms; pick = c; }
    }
    opts->max_paths_in_flight = pick.cap;
    opts->tail_threshold = pick.tail;
    opts->trace_kernel = pick.tk;
    // then the block shape of the state kernels at those settings
    uint32_t best_block = opts->block_size;
    for (uint32_t b : {64u, 96u, 128u}) {
        rt_render_opts o = *opts;
        o.block_size = b;
        o.stats = nullptr;
        o.profile = 0;
        RT_CUDA_TRY(cudaStreamSynchronize(st));
        auto t0 = std::chrono::steady_clock::now();
        rt_status s;
        if (njobs == 1) s = rt_render(jobs[0].scene, &jobs[0].camera, sample_spp, jobs[0].max_depth, jobs[0].film, &o, stream);
        else {
            std::vector<rt_render_job> js(jobs, jobs + njobs);
            for (auto &j : js) j.spp = sample_spp;
            s = rt_render_batch(js.data(), njobs, &o, stream);
        }
        if (s != RT_OK) return s;
        RT_CUDA_TRY(cudaStreamSynchronize(st));
        double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        if (ms < best) { best = ms; best_block = b; }
    }
    opts->block_size = best_block;
    return RT_OK;
}

// ---------------------------------------------------------------------------
// Host test hook of the regeneration bookkeeping: the decisions of
// k_regen_init, k_regen_gather, k_regen and k_regen_step_end (the same
// counting functions) driven by synthetic path lengths instead of shading.
// n_tasks tasks, `cap` slots, task k lives life[k] >= 1 bounce steps; a stop
// after `stop_step` steps (~0u: none). Writes per task the step at which it
// was retired (~0u: never started) and returns the steps taken and the steps
// that refilled slots. Checks that no task is retired twice and that the
// live paths always occupy distinct slots below `cap`.
extern "C" rt_status rt_debug_regen_host(uint32_t n_tasks, uint32_t cap, uint32_t regen_min, const uint8_t *life,
                                         uint32_t stop_step, uint32_t *retired_at, uint32_t *steps,
                                         uint32_t *regen_steps) {
    if (cap == 0 || regen_min == 0 || !life || !retired_at || !steps || !regen_steps) {
        rtg::set_error("rt_debug_regen_host: invalid argument");
        return RT_INVALID_ARG;
    }
    using namespace rtg;
    std::vector<uint32_t> task(cap, ~0u), q[2] = {std::vector<uint32_t>(cap), std::vector<uint32_t>(cap)};
    std::vector<uint32_t> qd(cap), left(cap, 0), g_task(cap), g_left(cap);
    std::vector<uint8_t> seen(cap);
    for (uint32_t k = 0; k < n_tasks; ++k) retired_at[k] = ~0u;
    Ctrl c{};
    const uint32_t k0 = std::min(cap, n_tasks);
    for (uint32_t s = 0; s < k0; ++s) { task[s] = s; left[s] = life[s]; q[0][s] = s; }
    c.n_ext = k0; c.n_free = cap - k0; c.task_next = k0; c.n_tasks = n_tasks;
    uint32_t step = 0;
    const uint32_t limit = 64u + 4u * 256u * (n_tasks / std::max(1u, cap / 2) + 2u);
    while (c.n_ext > 0 || (!c.stop && c.task_next < c.n_tasks)) {
        if (++step > limit) { set_error("rt_debug_regen_host: no progress"); return RT_CUDA_ERROR; }
        // "shade": every live path takes one step; ended ones go to the dead list
        std::vector<uint32_t> &cur = q[c.cur], &next = q[c.cur ^ 1u];
        for (uint32_t i = 0; i < c.n_ext; ++i) {
            const uint32_t s = cur[i];
            if (--left[s] > 0) next[c.n_next++] = s;
            else qd[c.n_dead++] = s;
        }
        if (c.n_next + c.n_dead != c.n_ext) { set_error("rt_debug_regen_host: lost a path"); return RT_CUDA_ERROR; }
        const RegenPlan pl = regen_plan(&c, regen_min);
        // k_regen_gather
        for (uint32_t j = 0; j < pl.n_dead; ++j) {
            const uint32_t s = qd[j];
            if (retired_at[task[s]] != ~0u) { set_error("rt_debug_regen_host: task retired twice"); return RT_CUDA_ERROR; }
            retired_at[task[s]] = step;
        }
        for (uint32_t j = 0; j < pl.n_move; ++j) { g_task[j] = task[next[j]]; g_left[j] = left[next[j]]; }
        // k_regen
        if (pl.n_new) {
            for (uint32_t i = 0; i < pl.n_move + pl.n_new; ++i) {
                if (i >= cap) { set_error("rt_debug_regen_host: slot out of range"); return RT_CUDA_ERROR; }
                if (i < pl.n_move) {
                    task[i] = g_task[i];
                    left[i] = g_left[i];
                } else {
                    const uint32_t off = c.task_next + (i - pl.n_move);
                    task[i] = off;
                    left[i] = life[off];
                }
                next[i] = i;
            }
        }
        regen_advance(&c, regen_min);
        if (c.n_ext + c.n_free != cap) { set_error("rt_debug_regen_host: slots lost or duplicated"); return RT_CUDA_ERROR; }
        std::fill(seen.begin(), seen.end(), 0);
        for (uint32_t i = 0; i < c.n_ext; ++i) {
            const uint32_t s = q[c.cur][i];
            if (s >= cap || seen[s]) { set_error("rt_debug_regen_host: two live paths in one slot"); return RT_CUDA_ERROR; }
            seen[s] = 1;
        }
        if (step >= stop_step) c.stop = 1u;
    }
    *steps = step;
    *regen_steps = c.regen_sets;
    return RT_OK;
}

// Host test hook: the guided render's set and buffer sizes for a pool of
// `cap` paths per set (fixed_pool: the caller set max_paths_in_flight) and a
// set of n paths, young or not. out[13] = cap, cap_young, per_step, gdepth,
// rec_depth, keep_young, rec_young, rec_alloc, keep_alloc, keep, rec_paths,
// rec_stride, set_steps. Never called by the product entry points.
extern "C" rt_status rt_debug_guided_plan_host(uint32_t batch, uint32_t wsb, uint32_t guide_depth, uint32_t max_depth,
                                               uint32_t cap, int32_t fixed_pool, uint32_t n, int32_t young,
                                               uint32_t *out) {
    if (!out || batch == 0 || batch > (1u << 24) || cap < 32 || n == 0) {
        set_error("rt_debug_guided_plan_host: invalid argument");
        return RT_INVALID_ARG;
    }
    const GuidedPlan g = guided_plan(batch, wsb, guide_depth, max_depth, cap, fixed_pool != 0);
    const GuidedSet e = guided_set(g, batch, n, young != 0);
    const uint32_t v[13] = {g.cap, g.cap_young, g.per_step, g.gdepth, g.rec_depth, g.keep_young, g.rec_young,
                            g.rec_alloc, g.keep_alloc, e.keep, e.rec_paths, e.rec_stride, e.set_steps};
    for (int k = 0; k < 13; ++k) out[k] = v[k];
    return RT_OK;
}
