// Ray casting on the 8-wide compressed BVH: watertight ray/triangle
// intersection (the paper relies on watertight traversal so that no boundary
// crossing is missed, Sec. 2.3) and stack-based traversal of node groups.
//
// Every routine is __host__ __device__: the kernels run them on the GPU, and
// the library's host debug entry point runs the very same code on the CPU so
// that the BVH build and traversal can be checked without a device.
#pragma once

#include "common.cuh"

namespace rtg {

// ----------------------------------------------------------- intrinsics
RT_HD int clz32(uint32_t x) {
#ifdef __CUDA_ARCH__
    return __clz(x);
#else
    return x ? __builtin_clz(x) : 32;
#endif
}
RT_HD int popc32(uint32_t x) {
#ifdef __CUDA_ARCH__
    return __popc(x);
#else
    return __builtin_popcount(x);
#endif
}
RT_HD int ffs32(uint32_t x) {
#ifdef __CUDA_ARCH__
    return __ffs(x);
#else
    return __builtin_ffs(x);
#endif
}
template <class T>
RT_HD T ldg(const T *p) {
#ifdef __CUDA_ARCH__
    return __ldg(p);
#else
    return *p;
#endif
}
// IEEE operations that the compiler may not fuse into FMAs: the watertight
// test needs the mirrored edge functions of two neighbouring triangles to be
// exact negatives of each other.
RT_HD float mul_rn(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fmul_rn(a, b);
#else
    return a * b;
#endif
}
RT_HD float sub_rn(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fsub_rn(a, b);
#else
    return a - b;
#endif
}
RT_HD double dmul_rn(double a, double b) {
#ifdef __CUDA_ARCH__
    return __dmul_rn(a, b);
#else
    return a * b;
#endif
}
RT_HD double dsub_rn(double a, double b) {
#ifdef __CUDA_ARCH__
    return __dsub_rn(a, b);
#else
    return a - b;
#endif
}
RT_HD float fma_rn(float a, float b, float c) {
#ifdef __CUDA_ARCH__
    return __fmaf_rn(a, b, c);
#else
    return fmaf(a, b, c);
#endif
}

struct Ray {
    V3 o, d;
    float tmin, tmax;
};

struct Hit {
    uint32_t prim, inst;
    float t, b1, b2;
};

// Per-ray constants of the watertight test (Woop, Benthin, Wald 2013) and of
// the slab test.
struct RayPre {
    V3 o, d;
    V3 inv;          // 1 / d with zero components replaced by +-1e-20
    uint32_t oct;    // bit a set when d[a] < 0
    int kx, ky, kz;
    float Sx, Sy, Sz;
};

RT_HD float comp(V3 v, int a) { return a == 0 ? v.x : (a == 1 ? v.y : v.z); }

RT_HD RayPre prepare(const Ray &r) {
    RayPre p;
    p.o = r.o;
    p.d = r.d;
    float dx = fabsf(r.d.x) < 1e-20f ? copysignf(1e-20f, r.d.x) : r.d.x;
    float dy = fabsf(r.d.y) < 1e-20f ? copysignf(1e-20f, r.d.y) : r.d.y;
    float dz = fabsf(r.d.z) < 1e-20f ? copysignf(1e-20f, r.d.z) : r.d.z;
    p.inv = v3(1.f / dx, 1.f / dy, 1.f / dz);
    p.oct = (r.d.x < 0.f ? 1u : 0u) | (r.d.y < 0.f ? 2u : 0u) | (r.d.z < 0.f ? 4u : 0u);
    float ax = fabsf(r.d.x), ay = fabsf(r.d.y), az = fabsf(r.d.z);
    int kz = 0;
    if (ay > ax) kz = 1;
    if (az > fmaxf(ax, ay)) kz = 2;
    int kx = kz + 1 == 3 ? 0 : kz + 1;
    int ky = kx + 1 == 3 ? 0 : kx + 1;
    float dkz = comp(r.d, kz);
    if (dkz < 0.f) { int t = kx; kx = ky; ky = t; }
    p.kx = kx; p.ky = ky; p.kz = kz;
    p.Sx = comp(r.d, kx) / dkz;
    p.Sy = comp(r.d, ky) / dkz;
    p.Sz = 1.f / dkz;
    return p;
}

// Watertight intersection; accepts t in (tmin, tmax) and t <= tbest.
RT_HD bool intersect_tri(const RayPre &rp, V3 v0, V3 v1, V3 v2, float tmin, float tmax, float tbest,
                         float &t, float &b1, float &b2) {
    V3 A = v0 - rp.o, B = v1 - rp.o, C = v2 - rp.o;
    float Akx = comp(A, rp.kx), Aky = comp(A, rp.ky), Akz = comp(A, rp.kz);
    float Bkx = comp(B, rp.kx), Bky = comp(B, rp.ky), Bkz = comp(B, rp.kz);
    float Ckx = comp(C, rp.kx), Cky = comp(C, rp.ky), Ckz = comp(C, rp.kz);
    float Ax = fma_rn(-rp.Sx, Akz, Akx), Ay = fma_rn(-rp.Sy, Akz, Aky);
    float Bx = fma_rn(-rp.Sx, Bkz, Bkx), By = fma_rn(-rp.Sy, Bkz, Bky);
    float Cx = fma_rn(-rp.Sx, Ckz, Ckx), Cy = fma_rn(-rp.Sy, Ckz, Cky);
    float U = sub_rn(mul_rn(Cx, By), mul_rn(Cy, Bx));
    float V = sub_rn(mul_rn(Ax, Cy), mul_rn(Ay, Cx));
    float W = sub_rn(mul_rn(Bx, Ay), mul_rn(By, Ax));
    if (U == 0.f || V == 0.f || W == 0.f) {
        // exact products in double decide the sign on an edge
        U = (float)dsub_rn(dmul_rn((double)Cx, (double)By), dmul_rn((double)Cy, (double)Bx));
        V = (float)dsub_rn(dmul_rn((double)Ax, (double)Cy), dmul_rn((double)Ay, (double)Cx));
        W = (float)dsub_rn(dmul_rn((double)Bx, (double)Ay), dmul_rn((double)By, (double)Ax));
    }
    if ((U < 0.f || V < 0.f || W < 0.f) && (U > 0.f || V > 0.f || W > 0.f)) return false;
    float det = U + V + W;
    if (det == 0.f) return false;
    float Az = rp.Sz * Akz, Bz = rp.Sz * Bkz, Cz = rp.Sz * Ckz;
    float T = U * Az + V * Bz + W * Cz;
    float tt = T / det;
    if (!(tt > tmin && tt < tmax && tt <= tbest)) return false;
    float inv = 1.f / det;
    t = tt;
    b1 = V * inv;
    b2 = W * inv;
    return true;
}

RT_HD float exp2i(int e) {
#ifdef __CUDA_ARCH__
    return __int_as_float((e + 127) << 23);
#else
    uint32_t b = (uint32_t)(e + 127) << 23;
    float f;
    memcpy(&f, &b, 4);
    return f;
#endif
}

RT_HD float as_float(uint32_t u) {
#ifdef __CUDA_ARCH__
    return __uint_as_float(u);
#else
    float f;
    memcpy(&f, &u, 4);
    return f;
#endif
}
RT_HD uint32_t as_uint(float f) {
#ifdef __CUDA_ARCH__
    return __float_as_uint(f);
#else
    uint32_t u;
    memcpy(&u, &f, 4);
    return u;
#endif
}

// Exact float value of byte `i` (0..7) of the 8-byte word (lo4, hi4): the
// byte is placed in the mantissa of 2^23 with one byte permute and 2^23 is
// subtracted, which avoids the quarter-rate integer-to-float conversion.
RT_HD float qbyte(uint32_t lo4, uint32_t hi4, int i) {
    uint32_t w = i < 4 ? lo4 : hi4;
#ifdef __CUDA_ARCH__
    uint32_t b = __byte_perm(w, 0x4B000000u, 0x7540u + (uint32_t)(i & 3));
    return __uint_as_float(b) - 8388608.f;
#else
    return (float)((w >> (8 * (i & 3))) & 0xFFu);
#endif
}

// Intersect the 8 child boxes of node (n0..n4); returns the internal-child
// hit bits at 24 + (slot ^ oct) and, through tri_bits, the triangle bits.
RT_HD uint32_t intersect_children_scalar(const RayPre &rp, uint4 n0, uint4 n1, uint4 n2, uint4 n3, uint4 n4,
                                         float tmin, float tmax, uint32_t &tri_bits) {
    V3 p = v3(as_float(n0.x), as_float(n0.y), as_float(n0.z));
    int ex = (int)(int8_t)(n0.w & 0xFF), ey = (int)(int8_t)((n0.w >> 8) & 0xFF),
        ez = (int)(int8_t)((n0.w >> 16) & 0xFF);
    uint32_t imask = n0.w >> 24;
    float ax = exp2i(ex) * rp.inv.x, ay = exp2i(ey) * rp.inv.y, az = exp2i(ez) * rp.inv.z;
    float bx = (p.x - rp.o.x) * rp.inv.x, by = (p.y - rp.o.y) * rp.inv.y, bz = (p.z - rp.o.z) * rp.inv.z;
    // near/far planes per axis follow the direction sign
    const bool sx = rp.inv.x < 0.f, sy = rp.inv.y < 0.f, sz = rp.inv.z < 0.f;
    const uint32_t nxl = sx ? n2.z : n2.x, nxh = sx ? n2.w : n2.y, fxl = sx ? n2.x : n2.z, fxh = sx ? n2.y : n2.w;
    const uint32_t nyl = sy ? n3.z : n3.x, nyh = sy ? n3.w : n3.y, fyl = sy ? n3.x : n3.z, fyh = sy ? n3.y : n3.w;
    const uint32_t nzl = sz ? n4.z : n4.x, nzh = sz ? n4.w : n4.y, fzl = sz ? n4.x : n4.z, fzh = sz ? n4.y : n4.w;
    uint32_t inner = 0, tris = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        float nx = fma_rn(qbyte(nxl, nxh, i), ax, bx), fx = fma_rn(qbyte(fxl, fxh, i), ax, bx);
        float ny = fma_rn(qbyte(nyl, nyh, i), ay, by), fy = fma_rn(qbyte(fyl, fyh, i), ay, by);
        float nz = fma_rn(qbyte(nzl, nzh, i), az, bz), fz = fma_rn(qbyte(fzl, fzh, i), az, bz);
        float t0 = fmaxf(fmaxf(nx, ny), fmaxf(nz, tmin));
        float t1 = fminf(fminf(fx, fy), fminf(fz, tmax));
        bool hit = t0 <= t1 * 1.000001f;
        uint32_t meta = (i < 4 ? n1.z : n1.w) >> (8 * (i & 3)) & 0xFFu;
        uint32_t is_inner = (imask >> i) & 1u;
        uint32_t ib = (hit && meta && is_inner) ? (1u << (24 + (i ^ rp.oct))) : 0u;
        uint32_t tb = (hit && meta && !is_inner) ? ((meta >> 5) << (meta & 31u)) : 0u;
        inner |= ib;
        tris |= tb;
    }
    tri_bits = tris;
    return inner;
}

#ifdef __CUDA_ARCH__
// Blackwell packed FP32 pairs: the near and far plane of one axis go through
// one fma.rn.f32x2 (and the byte decode through one add.rn.f32x2); each lane
// of the pair is the IEEE result of the scalar operation, so the outcome is
// bit-identical to intersect_children_scalar. Three-input min / max fold the
// slab reductions.
__device__ __forceinline__ uint64_t pk2(uint32_t lo, uint32_t hi) {
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "r"(lo), "r"(hi));
    return r;
}
__device__ __forceinline__ void upk2(uint64_t v, float &lo, float &hi) {
    uint32_t a, b;
    asm("mov.b64 {%0, %1}, %2;" : "=r"(a), "=r"(b) : "l"(v));
    lo = __uint_as_float(a);
    hi = __uint_as_float(b);
}
__device__ __forceinline__ uint64_t add2(uint64_t a, uint64_t b) {
    uint64_t r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ uint64_t fma2(uint64_t a, uint64_t b, uint64_t c) {
    uint64_t r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
__device__ __forceinline__ float max3(float a, float b, float c) {
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}
__device__ __forceinline__ float min3(float a, float b, float c) {
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

__device__ __forceinline__ uint32_t intersect_children(const RayPre &rp, uint4 n0, uint4 n1, uint4 n2, uint4 n3,
                                                       uint4 n4, float tmin, float tmax, uint32_t &tri_bits) {
    const float px = __uint_as_float(n0.x), py = __uint_as_float(n0.y), pz = __uint_as_float(n0.z);
    const int ex = (int)(int8_t)(n0.w & 0xFF), ey = (int)(int8_t)((n0.w >> 8) & 0xFF),
              ez = (int)(int8_t)((n0.w >> 16) & 0xFF);
    const uint32_t imask = n0.w >> 24;
    const float ax = exp2i(ex) * rp.inv.x, ay = exp2i(ey) * rp.inv.y, az = exp2i(ez) * rp.inv.z;
    const float bx = (px - rp.o.x) * rp.inv.x, by = (py - rp.o.y) * rp.inv.y, bz = (pz - rp.o.z) * rp.inv.z;
    const uint64_t AX = pk2(__float_as_uint(ax), __float_as_uint(ax)), BX = pk2(__float_as_uint(bx), __float_as_uint(bx));
    const uint64_t AY = pk2(__float_as_uint(ay), __float_as_uint(ay)), BY = pk2(__float_as_uint(by), __float_as_uint(by));
    const uint64_t AZ = pk2(__float_as_uint(az), __float_as_uint(az)), BZ = pk2(__float_as_uint(bz), __float_as_uint(bz));
    const uint64_t MAG = pk2(0xCB000000u, 0xCB000000u);   // (-2^23, -2^23)
    const bool sx = rp.inv.x < 0.f, sy = rp.inv.y < 0.f, sz = rp.inv.z < 0.f;
    const uint32_t nxl = sx ? n2.z : n2.x, nxh = sx ? n2.w : n2.y, fxl = sx ? n2.x : n2.z, fxh = sx ? n2.y : n2.w;
    const uint32_t nyl = sy ? n3.z : n3.x, nyh = sy ? n3.w : n3.y, fyl = sy ? n3.x : n3.z, fyh = sy ? n3.y : n3.w;
    const uint32_t nzl = sz ? n4.z : n4.x, nzh = sz ? n4.w : n4.y, fzl = sz ? n4.x : n4.z, fzh = sz ? n4.y : n4.w;
    // one hit bit per child slot; the bookkeeping that turns hits into the
    // internal-child mask and the triangle mask runs once per node below
    uint32_t hm = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const uint32_t sel = 0x7540u + (uint32_t)(i & 3);
        const uint32_t wnx = i < 4 ? nxl : nxh, wfx = i < 4 ? fxl : fxh;
        const uint32_t wny = i < 4 ? nyl : nyh, wfy = i < 4 ? fyl : fyh;
        const uint32_t wnz = i < 4 ? nzl : nzh, wfz = i < 4 ? fzl : fzh;
        uint64_t qx = add2(pk2(__byte_perm(wnx, 0x4B000000u, sel), __byte_perm(wfx, 0x4B000000u, sel)), MAG);
        uint64_t qy = add2(pk2(__byte_perm(wny, 0x4B000000u, sel), __byte_perm(wfy, 0x4B000000u, sel)), MAG);
        uint64_t qz = add2(pk2(__byte_perm(wnz, 0x4B000000u, sel), __byte_perm(wfz, 0x4B000000u, sel)), MAG);
        float nx, fx, ny, fy, nz, fz;
        upk2(fma2(qx, AX, BX), nx, fx);
        upk2(fma2(qy, AY, BY), ny, fy);
        upk2(fma2(qz, AZ, BZ), nz, fz);
        float t0 = fmaxf(max3(nx, ny, nz), tmin);
        float t1 = fminf(min3(fx, fy, fz), tmax);
        if (t0 <= t1 * 1.000001f) hm |= 1u << i;
    }
    // Empty slots carry neither an imask bit nor triangles (meta 0), so a
    // spurious hit on one adds nothing. Internal children: slot s -> bit
    // 24 + (s ^ oct), i.e. swap bits, bit pairs and nibbles as oct says.
    uint32_t x = hm & imask;
    const uint32_t x1 = ((x & 0x55u) << 1) | ((x >> 1) & 0x55u);
    x = (rp.oct & 1u) ? x1 : x;
    const uint32_t x2 = ((x & 0x33u) << 2) | ((x >> 2) & 0x33u);
    x = (rp.oct & 2u) ? x2 : x;
    const uint32_t x4 = ((x & 0x0Fu) << 4) | ((x >> 4) & 0x0Fu);
    x = (rp.oct & 4u) ? x4 : x;
    // leaf children: meta = (unary triangle count << 5) | first triangle bit
    uint32_t leaves = hm & ~imask, tris = 0;
    while (leaves) {
        const uint32_t i = (uint32_t)(__ffs(leaves) - 1);
        leaves &= leaves - 1u;
        const uint32_t meta = __byte_perm(i < 4u ? n1.z : n1.w, 0u, 0x4440u | (i & 3u));
        tris |= (meta >> 5) << (meta & 31u);
    }
    tri_bits = tris;
    return x << 24;
}
#else
RT_HD uint32_t intersect_children(const RayPre &rp, uint4 n0, uint4 n1, uint4 n2, uint4 n3, uint4 n4, float tmin,
                                  float tmax, uint32_t &tri_bits) {
    return intersect_children_scalar(rp, n0, n1, n2, n3, n4, tmin, tmax, tri_bits);
}
#endif

struct TraceResult {
    bool overflow;
    uint32_t nodes;   // nodes visited
    uint32_t tris;    // triangles tested
};

// Traversal stack in a thread-local array (registers / local memory).
struct LocalStack {
    uint2 e[kStackSize];
    RT_HD uint2 &operator[](int i) { return e[i]; }
    RT_HD static constexpr int capacity() { return kStackSize; }
};
// Thread-local stack with fewer usable entries than kStackSize (host test
// hook: drives the overflow path of the traversal on small scenes).
struct BoundedStack {
    uint2 e[kStackSize];
    int cap;
    RT_HD uint2 &operator[](int i) { return e[i]; }
    RT_HD int capacity() const { return cap; }
};
#ifdef __CUDACC__
// Traversal stack whose top kSharedEntries entries live in shared memory,
// entry-major so that the lanes of a warp touch consecutive words
// (conflict-free); deeper entries spill to a thread-local array. `base`
// points at this thread's first shared entry and `stride` is the block size.
constexpr int kSharedEntries = 16;
struct SharedStack {
    uint2 *base;
    int stride;
    uint2 deep[kStackSize - kSharedEntries];
    __device__ uint2 &operator[](int i) { return i < kSharedEntries ? base[i * stride] : deep[i - kSharedEntries]; }
    __device__ static constexpr int capacity() { return kStackSize; }
};
#endif

// Traversal of one ray against one BVH as a resumable state: begin() sets it
// up, each step() visits one node and tests the triangles of its hit leaf
// children, and returns false once the ray is finished (stack empty, or a hit
// found in any-hit mode). traverse() runs it to completion; kernels that
// refill idle lanes between steps drive it themselves. Closest hit: on equal
// t the lower (instance, primitive) wins.
template <bool kAnyHit>
struct Traversal {
    RayPre rp;
    float tmin, tmax, tbest;
    uint2 ng;   // current node group: child base, hit bits 24..31, imask 0..7
    int sp;
    uint32_t inst;

    RT_HD void begin(const Ray &ray, const Hit &hit, uint32_t root, uint32_t instance) {
        rp = prepare(ray);
        tmin = ray.tmin;
        tmax = ray.tmax;
        tbest = hit.prim == RT_MISS ? ray.tmax : hit.t;
        sp = 0;
        inst = instance;
        // a virtual group holding the root as its only internal child (slot 0)
        ng = make_uint2(root, (1u << (24 + (0u ^ rp.oct))) | 1u);
    }

    template <class Stack>
    RT_HD bool step(const uint4 *nodes, const float4 *tris, Stack &stack, Hit &hit, TraceResult &res) {
        uint32_t tbase = 0, tmask = 0;
        if (ng.y & 0xFF000000u) {
            int bit = 31 - clz32(ng.y);
            uint32_t slot = ((uint32_t)bit - 24u) ^ rp.oct;
            uint32_t rel = popc32((ng.y & 0xFFu) & ((1u << slot) - 1u));
            uint32_t child = ng.x + rel;
            ng.y &= ~(1u << bit);
            if (ng.y & 0xFF000000u) {
                if (sp == stack.capacity()) { res.overflow = true; return false; }
                stack[sp++] = ng;
            }
            const uint4 *N = nodes + 5 * (size_t)child;
            uint4 n0 = ldg(N), n1 = ldg(N + 1), n2 = ldg(N + 2), n3 = ldg(N + 3), n4 = ldg(N + 4);
            ++res.nodes;
            uint32_t tb;
            uint32_t inner = intersect_children(rp, n0, n1, n2, n3, n4, tmin, tbest, tb);
            ng = make_uint2(n1.x, inner | (n0.w >> 24));
            tbase = n1.y;
            tmask = tb;
        } else {
            ng.y = 0u;
        }
        while (tmask) {
            int k = ffs32(tmask) - 1;
            tmask &= tmask - 1u;
            const float4 *T = tris + 3 * (size_t)(tbase + (uint32_t)k);
            float4 a = ldg(T), b = ldg(T + 1), c = ldg(T + 2);
            ++res.tris;
            float t, u, v;
            if (intersect_tri(rp, f4xyz(a), f4xyz(b), f4xyz(c), tmin, tmax, tbest, t, u, v)) {
                uint32_t prim = as_uint(a.w);
                if (kAnyHit) {
                    hit.prim = prim; hit.inst = inst; hit.t = t; hit.b1 = u; hit.b2 = v;
                    return false;
                }
                if (t < tbest || hit.prim == RT_MISS || inst < hit.inst || (inst == hit.inst && prim < hit.prim)) {
                    hit.prim = prim; hit.inst = inst; hit.t = t; hit.b1 = u; hit.b2 = v;
                    tbest = t;
                }
            }
        }
        if (!(ng.y & 0xFF000000u)) {
            if (sp == 0) return false;
            ng = stack[--sp];
        }
        return true;
    }
};

// Closest hit (any_hit = false) or any hit (true) against one BVH.
// On return hit.prim == RT_MISS if nothing was found; hit.t, b1, b2 valid
// otherwise. `hit` may hold a previous best (used for two-level scenes).
// The stack is thread-local unless `ext_stack` is given.
template <bool kAnyHit, class Stack = LocalStack>
RT_HD TraceResult traverse(const uint4 *nodes, const float4 *tris, uint32_t root, const Ray &ray, Hit &hit,
                           uint32_t inst = 0u, Stack *ext_stack = nullptr) {
    TraceResult res{false, 0u, 0u};
    Stack own;
    Stack &stack = ext_stack ? *ext_stack : own;
    Traversal<kAnyHit> tr;
    tr.begin(ray, hit, root, inst);
    while (tr.step(nodes, tris, stack, hit, res)) {
    }
    return res;
}

#ifdef __CUDACC__
// One ray per thread with the triangle tests postponed (Ylitie, Karras and
// Laine 2017). A loop iteration visits one child node, or tests ONE triangle
// of the pending triangle group; when fewer than a fifth of the lanes that
// are still traversing have triangles to test and this lane has nodes left,
// its pending triangles go onto the stack as a group (x = first triangle,
// y = its mask in bits 0..23; node groups always carry hit bits in 24..31)
// and it descends further, so that the lanes of a warp stay on the same
// branch instead of idling through another lane's leaf. Groups are postponed
// only while the stack keeps kPostponeSpare free entries for node groups.
// Same hits and tie rule as `traverse` (the closest hit does not depend on
// the order of the tests).
constexpr int kPostponeSpare = 16;

template <bool kAnyHit, class Stack = LocalStack>
__device__ __forceinline__ TraceResult traverse_pp(const uint4 *nodes, const float4 *tris, const Ray &ray,
                                                   Hit &hit) {
    TraceResult res{false, 0u, 0u};
    Stack stack;
    const RayPre rp = prepare(ray);
    const float tmin = ray.tmin, tmax = ray.tmax;
    float tbest = hit.prim == RT_MISS ? ray.tmax : hit.t;
    int sp = 0;
    uint2 ng = make_uint2(0u, (1u << (24 + (0u ^ rp.oct))) | 1u);
    uint32_t tbase = 0u, tmask = 0u;
    for (;;) {
        const uint32_t act = __activemask();
        if (ng.y & 0xFF000000u) {
            const int bit = 31 - __clz(ng.y);
            const uint32_t slot = ((uint32_t)bit - 24u) ^ rp.oct;
            const uint32_t rel = __popc((ng.y & 0xFFu) & ((1u << slot) - 1u));
            const uint32_t child = ng.x + rel;
            ng.y &= ~(1u << bit);
            if (ng.y & 0xFF000000u) {
                if (sp == stack.capacity()) { res.overflow = true; return res; }
                stack[sp++] = ng;
            }
            const uint4 *N = nodes + 5 * (size_t)child;
            const uint4 n0 = __ldg(N), n1 = __ldg(N + 1), n2 = __ldg(N + 2), n3 = __ldg(N + 3), n4 = __ldg(N + 4);
            ++res.nodes;
            uint32_t tb;
            const uint32_t inner = intersect_children(rp, n0, n1, n2, n3, n4, tmin, tbest, tb);
            ng = make_uint2(n1.x, inner | (n0.w >> 24));
            tbase = n1.y;
            tmask = tb;
        }
        while (tmask) {
            if ((ng.y & 0xFF000000u) && sp + kPostponeSpare < stack.capacity() &&
                __popc(__activemask()) * 5 < __popc(act)) {
                stack[sp++] = make_uint2(tbase, tmask);
                tmask = 0u;
                break;
            }
            const int k = __ffs(tmask) - 1;
            tmask &= tmask - 1u;
            const float4 *T = tris + 3 * (size_t)(tbase + (uint32_t)k);
            const float4 a = __ldg(T), b = __ldg(T + 1), c = __ldg(T + 2);
            ++res.tris;
            float t, u, v;
            if (intersect_tri(rp, f4xyz(a), f4xyz(b), f4xyz(c), tmin, tmax, tbest, t, u, v)) {
                const uint32_t prim = __float_as_uint(a.w);
                if (kAnyHit) {
                    hit.prim = prim; hit.inst = 0u; hit.t = t; hit.b1 = u; hit.b2 = v;
                    return res;
                }
                if (t < tbest || hit.prim == RT_MISS || prim < hit.prim) {
                    hit.prim = prim; hit.inst = 0u; hit.t = t; hit.b1 = u; hit.b2 = v;
                    tbest = t;
                }
            }
        }
        if (!(ng.y & 0xFF000000u)) {
            if (sp == 0) return res;
            const uint2 e = stack[--sp];
            if (e.y & 0xFF000000u) {
                ng = e;
            } else {
                tbase = e.x;
                tmask = e.y;
            }
        }
    }
}
// Closest hit with one stack entry per child: every internal child whose box
// the ray enters is pushed with its entry distance, the nearest of them is
// visited next, and a popped entry farther than the best hit so far is
// dropped without fetching its node (the node-group traversal above culls a
// child only one level later, when its own children are tested). On the
// benchmark step this visits 14% fewer nodes (10.9 against 12.7 per ray)
// and tests 2.5% fewer triangles, but the per-child bookkeeping costs as
// much as it saves (an A/B variant). The drop test keeps the slab test's relative slack, so no node
// that could hold a hit at the best distance (or a tie there) is dropped:
// same hits and tie rule as `traverse`.
__device__ __forceinline__ TraceResult traverse_near(const uint4 *nodes, const float4 *tris, const Ray &ray, Hit &hit) {
#ifndef __CUDA_ARCH__
    return traverse<false>(nodes, tris, 0u, ray, hit);   // the host pass of the CUDA compiler only
#else
    TraceResult res{false, 0u, 0u};
    uint2 stack[kStackSize];   // (node, entry distance bits)
    const RayPre rp = prepare(ray);
    const float tmin = ray.tmin, tmax = ray.tmax;
    float tbest = hit.prim == RT_MISS ? tmax : hit.t;
    int sp = 0;
    uint32_t node = 0u;
    for (;;) {
        const uint4 *N = nodes + 5 * (size_t)node;
        const uint4 n0 = __ldg(N), n1 = __ldg(N + 1), n2 = __ldg(N + 2), n3 = __ldg(N + 3), n4 = __ldg(N + 4);
        ++res.nodes;
        const float px = __uint_as_float(n0.x), py = __uint_as_float(n0.y), pz = __uint_as_float(n0.z);
        const int ex = (int)(int8_t)(n0.w & 0xFF), ey = (int)(int8_t)((n0.w >> 8) & 0xFF),
                  ez = (int)(int8_t)((n0.w >> 16) & 0xFF);
        const uint32_t imask = n0.w >> 24;
        const float ax = exp2i(ex) * rp.inv.x, ay = exp2i(ey) * rp.inv.y, az = exp2i(ez) * rp.inv.z;
        const float bx = (px - rp.o.x) * rp.inv.x, by = (py - rp.o.y) * rp.inv.y, bz = (pz - rp.o.z) * rp.inv.z;
        const uint64_t AX = pk2(__float_as_uint(ax), __float_as_uint(ax)), BX = pk2(__float_as_uint(bx), __float_as_uint(bx));
        const uint64_t AY = pk2(__float_as_uint(ay), __float_as_uint(ay)), BY = pk2(__float_as_uint(by), __float_as_uint(by));
        const uint64_t AZ = pk2(__float_as_uint(az), __float_as_uint(az)), BZ = pk2(__float_as_uint(bz), __float_as_uint(bz));
        const uint64_t MAG = pk2(0xCB000000u, 0xCB000000u);
        const bool sx = rp.inv.x < 0.f, sy = rp.inv.y < 0.f, sz = rp.inv.z < 0.f;
        const uint32_t nxl = sx ? n2.z : n2.x, nxh = sx ? n2.w : n2.y, fxl = sx ? n2.x : n2.z, fxh = sx ? n2.y : n2.w;
        const uint32_t nyl = sy ? n3.z : n3.x, nyh = sy ? n3.w : n3.y, fyl = sy ? n3.x : n3.z, fyh = sy ? n3.y : n3.w;
        const uint32_t nzl = sz ? n4.z : n4.x, nzh = sz ? n4.w : n4.y, fzl = sz ? n4.x : n4.z, fzh = sz ? n4.y : n4.w;
        if (sp + 8 > kStackSize) { res.overflow = true; return res; }
        // every hit internal child is written above the stack top as it
        // comes; the nearest is then visited and the last written one takes
        // its place (keeping the nearest in registers instead and writing
        // only the others measured slower)
        uint32_t hm = 0, cnt = 0, bpos = 0, bchild = 0;
        float bt = INFINITY;
        uint2 last = make_uint2(0u, 0u);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const uint32_t sel = 0x7540u + (uint32_t)(i & 3);
            const uint32_t wnx = i < 4 ? nxl : nxh, wfx = i < 4 ? fxl : fxh;
            const uint32_t wny = i < 4 ? nyl : nyh, wfy = i < 4 ? fyl : fyh;
            const uint32_t wnz = i < 4 ? nzl : nzh, wfz = i < 4 ? fzl : fzh;
            uint64_t qx = add2(pk2(__byte_perm(wnx, 0x4B000000u, sel), __byte_perm(wfx, 0x4B000000u, sel)), MAG);
            uint64_t qy = add2(pk2(__byte_perm(wny, 0x4B000000u, sel), __byte_perm(wfy, 0x4B000000u, sel)), MAG);
            uint64_t qz = add2(pk2(__byte_perm(wnz, 0x4B000000u, sel), __byte_perm(wfz, 0x4B000000u, sel)), MAG);
            float nx, fx, ny, fy, nz, fz;
            upk2(fma2(qx, AX, BX), nx, fx);
            upk2(fma2(qy, AY, BY), ny, fy);
            upk2(fma2(qz, AZ, BZ), nz, fz);
            const float t0 = fmaxf(max3(nx, ny, nz), tmin);
            const float t1 = fminf(min3(fx, fy, fz), tbest);
            const bool h = t0 <= t1 * 1.000001f;
            if (h) hm |= 1u << i;
            if (h && ((imask >> i) & 1u)) {
                // internal child (its index among the node's internal children)
                const uint2 e = make_uint2(n1.x + (uint32_t)__popc(imask & ((1u << i) - 1u)), __float_as_uint(t0));
                stack[sp + (int)cnt] = e;
                if (t0 < bt) { bt = t0; bpos = cnt; bchild = e.x; }
                last = e;
                ++cnt;
            }
        }
        // leaf children: meta = (unary triangle count << 5) | first triangle bit
        uint32_t leaves = hm & ~imask, tmask = 0;
        while (leaves) {
            const uint32_t i = (uint32_t)(__ffs(leaves) - 1);
            leaves &= leaves - 1u;
            const uint32_t meta = __byte_perm(i < 4u ? n1.z : n1.w, 0u, 0x4440u | (i & 3u));
            tmask |= (meta >> 5) << (meta & 31u);
        }
        while (tmask) {
            const int k = __ffs(tmask) - 1;
            tmask &= tmask - 1u;
            const float4 *T = tris + 3 * (size_t)(n1.y + (uint32_t)k);
            const float4 a = __ldg(T), b = __ldg(T + 1), c = __ldg(T + 2);
            ++res.tris;
            float t, u, v;
            if (intersect_tri(rp, f4xyz(a), f4xyz(b), f4xyz(c), tmin, tmax, tbest, t, u, v)) {
                const uint32_t prim = __float_as_uint(a.w);
                if (t < tbest || hit.prim == RT_MISS || prim < hit.prim) {
                    hit.prim = prim; hit.inst = 0u; hit.t = t; hit.b1 = u; hit.b2 = v;
                    tbest = t;
                }
            }
        }
        if (cnt > 0) {
            // descend into the nearest; the last written entry takes its place
            node = bchild;
            stack[sp + (int)bpos] = last;
            sp += (int)cnt - 1;
            continue;
        }
        for (;;) {
            if (sp == 0) return res;
            const uint2 e = stack[--sp];
            if (__uint_as_float(e.y) <= tbest * 1.000001f) { node = e.x; break; }
        }
    }
#endif
}
#endif

// Ray in the object space of instance `inst`: rows 0..2 of inst_xf hold the
// world->object affine map. The direction is not renormalised, so t is the
// same in both spaces.
RT_HD Ray to_object(const float4 *xf, uint32_t inst, const Ray &r) {
    const float4 a = ldg(xf + 6 * (size_t)inst), b = ldg(xf + 6 * (size_t)inst + 1), c = ldg(xf + 6 * (size_t)inst + 2);
    Ray o;
    o.o = v3(a.x * r.o.x + a.y * r.o.y + a.z * r.o.z + a.w, b.x * r.o.x + b.y * r.o.y + b.z * r.o.z + b.w,
             c.x * r.o.x + c.y * r.o.y + c.z * r.o.z + c.w);
    o.d = v3(a.x * r.d.x + a.y * r.d.y + a.z * r.d.z, b.x * r.d.x + b.y * r.d.y + b.z * r.d.z,
             c.x * r.d.x + c.y * r.d.y + c.z * r.d.z);
    o.tmin = r.tmin;
    o.tmax = r.tmax;
    return o;
}

// Two-level traversal: the top-level BVH8 over instance boxes; a leaf slot
// is an instance, whose mesh BVH8 is traversed with the ray mapped to object
// space and the best hit so far.
template <bool kAnyHit>
RT_HD TraceResult traverse_tlas(const DevScene &sc, const Ray &ray, Hit &hit) {
    TraceResult res{false, 0u, 0u};
    RayPre rp = prepare(ray);
    uint2 stack[kStackSize];
    int sp = 0;
    uint2 ng = make_uint2(0u, (1u << (24 + (0u ^ rp.oct))) | 1u);
    for (;;) {
        uint32_t ibase = 0, imask = 0;
        if (ng.y & 0xFF000000u) {
            int bit = 31 - clz32(ng.y);
            uint32_t slot = ((uint32_t)bit - 24u) ^ rp.oct;
            uint32_t rel = popc32((ng.y & 0xFFu) & ((1u << slot) - 1u));
            uint32_t child = ng.x + rel;
            ng.y &= ~(1u << bit);
            if (ng.y & 0xFF000000u) {
                if (sp == kStackSize) { res.overflow = true; break; }
                stack[sp++] = ng;
            }
            const uint4 *N = sc.tlas_nodes + 5 * (size_t)child;
            uint4 n0 = ldg(N), n1 = ldg(N + 1), n2 = ldg(N + 2), n3 = ldg(N + 3), n4 = ldg(N + 4);
            ++res.nodes;
            uint32_t tb;
            float tcur = hit.prim == RT_MISS ? ray.tmax : hit.t;
            uint32_t inner = intersect_children(rp, n0, n1, n2, n3, n4, ray.tmin, tcur, tb);
            ng = make_uint2(n1.x, inner | (n0.w >> 24));
            ibase = n1.y;
            imask = tb;
        } else {
            ng.y = 0u;
        }
        while (imask) {
            int k = ffs32(imask) - 1;
            imask &= imask - 1u;
            uint32_t inst = ldg(sc.tlas_inst + ibase + (uint32_t)k);
            Ray ro = to_object(sc.inst_xf, inst, ray);
            TraceResult r2 = traverse<kAnyHit>(sc.nodes, sc.tris, ldg(sc.inst_root + inst), ro, hit, inst);
            res.nodes += r2.nodes;
            res.tris += r2.tris;
            res.overflow |= r2.overflow;
            if (kAnyHit && hit.prim != RT_MISS) return res;
        }
        if (!(ng.y & 0xFF000000u)) {
            if (sp == 0) break;
            ng = stack[--sp];
        }
    }
    return res;
}

// Closest (or any) hit against the scene, one level or two.
// Two-level traversal in one loop: every iteration visits one node of the
// top-level BVH or of the current instance's BVH, or tests the triangles of
// an instance's leaf, or enters the next instance of a top-level leaf, so
// the lanes of a warp stay in step whichever level they are at (the nested
// form runs a whole instance's traversal while the other lanes wait). One
// stack holds both levels: entering an instance pushes the remaining
// top-level group, the remaining instances of the leaf (x = first |
// kInstGroup, y = mask) and a marker (x = 0xffffffff); popping the marker returns to
// world space (node groups keep their hit bits in y; the flags live in x,
// which for a node group is a node index below 2^31). Same hits and tie
// rules as traverse_tlas.
template <bool kAnyHit>
RT_HD TraceResult traverse_two_level(const DevScene &sc, const Ray &ray, Hit &hit) {
    constexpr uint32_t kInstGroup = 0x80000000u, kMarker = 0xffffffffu;
    TraceResult res{false, 0u, 0u};
    const RayPre rw = prepare(ray);
    RayPre rp = rw;
    uint2 stack[kStackSize];
    int sp = 0;
    uint2 ng = make_uint2(0u, (1u << (24 + (0u ^ rw.oct))) | 1u);   // the top-level root
    const uint4 *nodes = sc.tlas_nodes;
    bool in_inst = false;
    uint32_t inst = 0u;
    uint32_t ibase = 0u, imask = 0u;    // instances of a top-level leaf still to enter
    const float tmin = ray.tmin;
    float tbest = hit.prim == RT_MISS ? ray.tmax : hit.t;
    for (;;) {
        if (imask) {
            // enter the next instance; what is left of this level resumes
            // after it
            const int k = ffs32(imask) - 1;
            imask &= imask - 1u;
            const uint32_t id = ldg(sc.tlas_inst + ibase + (uint32_t)k);
            if (sp + 3 > kStackSize) { res.overflow = true; break; }
            if (ng.y & 0xFF000000u) stack[sp++] = ng;
            if (imask) stack[sp++] = make_uint2(ibase | kInstGroup, imask);
            stack[sp++] = make_uint2(kMarker, 0u);
            imask = 0u;
            inst = id;
            in_inst = true;
            rp = prepare(to_object(sc.inst_xf, id, ray));
            nodes = sc.nodes;
            ng = make_uint2(ldg(sc.inst_root + id), (1u << (24 + (0u ^ rp.oct))) | 1u);
            continue;
        }
        uint32_t tbase = 0u, tmask = 0u;
        if (ng.y & 0xFF000000u) {
            const int bit = 31 - clz32(ng.y);
            const uint32_t slot = ((uint32_t)bit - 24u) ^ rp.oct;
            const uint32_t rel = popc32((ng.y & 0xFFu) & ((1u << slot) - 1u));
            const uint32_t child = ng.x + rel;
            ng.y &= ~(1u << bit);
            if (ng.y & 0xFF000000u) {
                if (sp == kStackSize) { res.overflow = true; break; }
                stack[sp++] = ng;
            }
            const uint4 *N = nodes + 5 * (size_t)child;
            const uint4 n0 = ldg(N), n1 = ldg(N + 1), n2 = ldg(N + 2), n3 = ldg(N + 3), n4 = ldg(N + 4);
            ++res.nodes;
            uint32_t tb;
            const uint32_t inner = intersect_children(rp, n0, n1, n2, n3, n4, tmin, tbest, tb);
            ng = make_uint2(n1.x, inner | (n0.w >> 24));
            if (in_inst) {
                tbase = n1.y;
                tmask = tb;
            } else {
                ibase = n1.y;
                imask = tb;
            }
        } else {
            ng.y = 0u;
        }
        while (tmask) {
            const int k = ffs32(tmask) - 1;
            tmask &= tmask - 1u;
            const float4 *T = sc.tris + 3 * (size_t)(tbase + (uint32_t)k);
            const float4 a = ldg(T), b = ldg(T + 1), c = ldg(T + 2);
            ++res.tris;
            float t, u, v;
            if (intersect_tri(rp, f4xyz(a), f4xyz(b), f4xyz(c), tmin, ray.tmax, tbest, t, u, v)) {
                const uint32_t prim = as_uint(a.w);
                if (kAnyHit) {
                    hit.prim = prim; hit.inst = inst; hit.t = t; hit.b1 = u; hit.b2 = v;
                    return res;
                }
                if (t < tbest || hit.prim == RT_MISS || inst < hit.inst || (inst == hit.inst && prim < hit.prim)) {
                    hit.prim = prim; hit.inst = inst; hit.t = t; hit.b1 = u; hit.b2 = v;
                    tbest = t;
                }
            }
        }
        if (imask || (ng.y & 0xFF000000u)) continue;
        // this group is done: pop (a marker leaves the instance)
        for (;;) {
            if (sp == 0) return res;
            const uint2 e = stack[--sp];
            if (e.x == kMarker) {
                in_inst = false;
                rp = rw;
                nodes = sc.tlas_nodes;
                continue;
            }
            if (e.x & kInstGroup) {
                ibase = e.x & ~kInstGroup;
                imask = e.y;
            } else {
                ng = e;
            }
            break;
        }
    }
    return res;
}

template <bool kAnyHit>
RT_HD TraceResult trace_scene(const DevScene &sc, const Ray &ray, Hit &hit) {
    if (sc.two_level) return traverse_two_level<kAnyHit>(sc, ray, hit);
    return traverse<kAnyHit>(sc.nodes, sc.tris, 0u, ray, hit);
}

}  // namespace rtg
