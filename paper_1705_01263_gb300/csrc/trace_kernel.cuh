// Warp-cooperative BVH8 traversal for the ray-casting state kernels.
//
// Incoherent rays need very different amounts of work (an escaping ray
// touches a few nodes, a ray grazing the displaced ground dozens), so a warp
// that traces 32 rays to completion idles most of its lanes. Here warps are
// persistent and refill idle lanes from the ray queue while others are still
// traversing: a ballot counts the idle lanes, one lane reserves that many
// queue slots with a single atomic and a shuffle hands them out (dynamic ray
// fetching, Aila and Laine 2009). Each loop iteration does one unit of work
// per lane - one triangle test, one child-node visit or one stack pop - and a
// lane postpones its pending triangles onto the stack when fewer than a fifth
// of the active lanes want to test triangles, so that lanes stay on the same
// branch (Ylitie, Karras and Laine 2017). The top of the traversal stack
// lives in shared memory (entry-major, conflict-free), its overflow in local
// memory. Results and tie rules are those of `traverse` in traverse.cuh.
#pragma once

#include "traverse.cuh"

namespace rtg {

constexpr int kShStack = 16;     // stack entries per thread in shared memory
constexpr int kLocStack = 32;    // further entries in local memory
constexpr int kRefill = 8;       // refill a warp when this many lanes are idle

RT_D uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

struct WorkCount {
    uint32_t nodes = 0, tris = 0;
};

// Job: `Ray load(uint32_t i)` and `void store(uint32_t i, const Hit &h)`.
template <bool kAnyHit, bool kCount, class Job>
__device__ __forceinline__ void trace_persistent(const uint4 *__restrict__ nodes, const float4 *__restrict__ tris,
                                                 Job &job, uint32_t n, uint32_t *fetch, bool &overflow,
                                                 WorkCount &wc) {
    extern __shared__ uint2 s_stack[];
    const uint32_t FULL = 0xFFFFFFFFu;
    const uint32_t lane = lane_id();
    const uint32_t tid = threadIdx.x, bd = blockDim.x;
    uint2 l_stack[kLocStack];
    bool active = false, exhausted = false;
    uint32_t item = 0;
    Ray ray;
    RayPre rp;
    Hit h;
    float tbest = 0.f;
    uint2 ng = make_uint2(0u, 0u);
    uint32_t tbase = 0, tmask = 0;
    int sp = 0;
    for (;;) {
        uint32_t idle = __ballot_sync(FULL, !active);
        if (!exhausted && __popc(idle) >= kRefill) {
            uint32_t cnt = __popc(idle);
            uint32_t leader = __ffs(idle) - 1;
            uint32_t base = 0;
            if (lane == leader) base = atomicAdd(fetch, cnt);
            base = __shfl_sync(FULL, base, leader);
            if (base + cnt >= n) exhausted = true;
            if (!active) {
                uint32_t idx = base + __popc(idle & lanemask_lt());
                if (idx < n) {
                    item = idx;
                    ray = job.load(idx);
                    rp = prepare(ray);
                    h.prim = RT_MISS; h.inst = 0; h.t = INFINITY; h.b1 = h.b2 = 0.f;
                    tbest = ray.tmax;
                    ng = make_uint2(0u, (1u << (24 + (0u ^ rp.oct))) | 1u);
                    tmask = 0;
                    sp = 0;
                    active = true;
                }
            }
        }
        uint32_t act = __ballot_sync(FULL, active);
        if (act == 0) break;
        bool want_tri = active && tmask != 0;
        uint32_t tri_lanes = __ballot_sync(FULL, want_tri);
        bool postpone = want_tri && (ng.y & 0xFF000000u) && (__popc(tri_lanes) * 5 < __popc(act));
        if (!active) continue;
        bool finish = false, ray_ovf = false;
        auto push = [&](uint2 e) -> bool {
            if (sp < kShStack) s_stack[sp * bd + tid] = e;
            else if (sp < kShStack + kLocStack) l_stack[sp - kShStack] = e;
            else return false;
            ++sp;
            return true;
        };
        if (postpone) {
            if (push(make_uint2(tbase, tmask))) tmask = 0;
            else ray_ovf = true;
        }
        if (ray_ovf) {
            finish = true;
        } else if (tmask) {
            int k = __ffs(tmask) - 1;
            tmask &= tmask - 1u;
            const float4 *T = tris + 3 * (size_t)(tbase + (uint32_t)k);
            float4 a = __ldg(T), b = __ldg(T + 1), c = __ldg(T + 2);
            if (kCount) ++wc.tris;
            float t, u, v;
            if (intersect_tri(rp, f4xyz(a), f4xyz(b), f4xyz(c), ray.tmin, ray.tmax, tbest, t, u, v)) {
                uint32_t prim = __float_as_uint(a.w);
                if (kAnyHit) {
                    h.prim = prim; h.t = t; h.b1 = u; h.b2 = v;
                    finish = true;
                } else if (t < tbest || h.prim == RT_MISS || prim < h.prim) {
                    h.prim = prim; h.t = t; h.b1 = u; h.b2 = v;
                    tbest = t;
                }
            }
        } else if (ng.y & 0xFF000000u) {
            int bit = 31 - __clz(ng.y);
            uint32_t slot = ((uint32_t)bit - 24u) ^ rp.oct;
            uint32_t rel = __popc((ng.y & 0xFFu) & ((1u << slot) - 1u));
            uint32_t child = ng.x + rel;
            ng.y &= ~(1u << bit);
            if ((ng.y & 0xFF000000u) && !push(ng)) {
                ray_ovf = true;
                finish = true;
            } else {
                const uint4 *N = nodes + 5 * (size_t)child;
                uint4 n0 = __ldg(N), n1 = __ldg(N + 1), n2 = __ldg(N + 2), n3 = __ldg(N + 3), n4 = __ldg(N + 4);
                if (kCount) ++wc.nodes;
                uint32_t tb;
                uint32_t inner = intersect_children(rp, n0, n1, n2, n3, n4, ray.tmin, tbest, tb);
                ng = make_uint2(n1.x, inner | (n0.w >> 24));
                tbase = n1.y;
                tmask = tb;
            }
        } else if (sp > 0) {
            --sp;
            uint2 e = sp < kShStack ? s_stack[sp * bd + tid] : l_stack[sp - kShStack];
            if (e.y & 0xFF000000u) {
                ng = e;
            } else {
                tbase = e.x;
                tmask = e.y;
                ng.y = 0;
            }
        } else {
            finish = true;
        }
        if (finish) {
            if (ray_ovf) {
                overflow = true;
                h.prim = RT_MISS;
            }
            job.store(item, h);
            active = false;
        }
    }
}

}  // namespace rtg
