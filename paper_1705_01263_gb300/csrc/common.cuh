// Shared device/host declarations of the GB300 path tracer: small vector
// math, the device-side scene view and the path-state layout.
#pragma once

#include <cmath>
#include <cstdint>
#include <cstring>
#include <cuda_runtime.h>

#include "../../include/rt.h"

#define RT_HD __host__ __device__ __forceinline__
#define RT_D __device__ __forceinline__

namespace rtg {

constexpr float kPi = 3.14159265358979323846f;
constexpr float kInvPi = 0.318309886183790671538f;
constexpr float kF0 = 0.04f;            // Schlick reflectance at normal incidence
constexpr float kAdaptEps = 1e-3f;       // shading-normal adaptation margin (A.3)
constexpr float kShadowEps = 1e-4f;      // shadow rays to a triangle stop at (1 - eps) * dist
constexpr int kMaxDepth = 64;
constexpr int kStackSize = 48;           // BVH traversal stack entries (node groups)

// ------------------------------------------------------------------ vec3
struct V3 { float x, y, z; };
RT_HD V3 v3(float x, float y, float z) { return V3{x, y, z}; }
RT_HD V3 operator+(V3 a, V3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
RT_HD V3 operator-(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
RT_HD V3 operator-(V3 a) { return {-a.x, -a.y, -a.z}; }
RT_HD V3 operator*(V3 a, float s) { return {a.x * s, a.y * s, a.z * s}; }
RT_HD V3 operator*(float s, V3 a) { return {a.x * s, a.y * s, a.z * s}; }
RT_HD V3 mul(V3 a, V3 b) { return {a.x * b.x, a.y * b.y, a.z * b.z}; }
RT_HD float dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
RT_HD V3 cross(V3 a, V3 b) {
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
RT_HD float length(V3 a) { return sqrtf(dot(a, a)); }
RT_HD V3 normalize(V3 a) {
    float l = sqrtf(dot(a, a));
    return l > 0.f ? a * (1.f / l) : a;
}
RT_HD float maxc(V3 a) { return fmaxf(a.x, fmaxf(a.y, a.z)); }
RT_HD float lum(V3 c) { return 0.2126f * c.x + 0.7152f * c.y + 0.0722f * c.z; }
RT_HD V3 f4xyz(float4 a) { return {a.x, a.y, a.z}; }

// -------------------------------------------------------- device scene view
// BVH node: 80 bytes = 5 x uint4 (see bvh_build.cpp for the encoding).
struct DevScene {
    const uint4 *nodes;        // 5 uint4 per node
    const float4 *tris;        // 3 float4 per leaf triangle (v0.w = prim id bits)
    // two-level scenes: top level over instances, per-mesh bottom levels
    int32_t two_level;
    uint32_t num_instances;
    const uint4 *tlas_nodes;   // top-level nodes; leaf slots index tlas_inst
    const uint32_t *tlas_inst; // top-level leaf slot -> instance id
    const float4 *inst_xf;     // per instance: world->object 3x4 (3 float4) + object->world 3x4 (3 float4)
    const uint32_t *inst_root; // per instance: root node index of its mesh in `nodes`
    // shading data indexed by the original triangle id
    const float *vertices;     // V x 3
    const float *normals;      // V x 3 or null
    const float *uvs;          // V x 2 or null
    const uint32_t *indices;   // T x 3
    const uint32_t *tri_material;
    const float *tri_light_pdf_area; // T: (1 - p_env) P(select) / area, 0 = not an emitter
    const float4 *mat_a;       // albedo rgb, roughness
    const float4 *mat_b;       // emission rgb, ggx weight
    const int32_t *mat_tex;    // emission texture or -1
    int32_t tex_w, tex_h;
    const float *textures;     // K x th x tw x 3
    // emitters
    uint32_t num_lights;
    const float2 *alias;       // x = threshold, y = alias index (bits)
    const uint32_t *light_tri; // emitter -> triangle id
    const uint32_t *light_inst;// emitter -> instance id (two-level scenes)
    const float4 *light_v;     // emitter -> three world-space vertices
    // probabilistic light hierarchy (Sec. 2.1.1; null lb_rec: the alias
    // table picks emitters). One record of 7 float4 per internal node (a
    // tree of at most four emitters gets one record whose second child is
    // empty), holding what a step of the descent needs for both children:
    // per child (box centre, half diagonal), (I0..I3), (I4, I5, flux, link)
    // with I_k the directional value of cube-face region k (+x, -x, +y, -y,
    // +z, -z) and link = the child's record, or for a leaf 0x80000000 |
    // first slot << 3 | count; then (parent record or 0xffffffff, side in the
    // parent, 0, 0).
    const float4 *lb_rec;
    const uint32_t *lb_perm;      // leaf slot -> emitter
    const uint32_t *lb_up;        // emitter -> record of its leaf's parent << 1 | side
    const float *lb_eflux;        // emitter -> flux (luminance x area)
    const uint32_t *lb_tri_rank;  // triangle -> rank among its mesh's emitters
    const uint32_t *lb_inst_base; // instance -> index of its first emitter
    // environment
    int32_t env_w, env_h, env_levels;
    const float4 *env;         // finest level: rgb + pdf (lum / sum w)
    const float *env_pyr;      // all levels of weights, finest first, concatenated
    const int64_t *env_off;    // level offsets into env_pyr (device copy)
    int64_t env_off_h[16];     // same offsets, by value
    float p_env;               // probability of choosing the environment in NEE
    // normal-oriented top levels (null env_nw: plain pyramid only): per cell
    // of the geometric normal, levels env_lstar..top of reweighted weights,
    // level l at env_noff_h[l] inside a cell's block of env_nstride floats;
    // env_nscale[c] = sum of plain weights / sum of cell c's weights (0: the
    // cell uses the plain pyramid); env_nfac[c * env_nregions + R] = the
    // cell's pdf over the plain pdf in region R of level env_lstar (the
    // cosine bound times env_nscale[c]; 1 for a plain cell)
    // the descent reads two levels per load: for a node of level l >= 2 five
    // float4 at env_dq + env_dqoff_h[l] + 5 * node (its children's weights as
    // the quad (x0 y0, x1 y0, x0 y1, x1 y1), then each child's own children
    // quad, in that order); for a node of level 1 one float4 (its children
    // quad) at env_dq + env_dqoff_h[1] + node. env_ndq: the same blocks per
    // normal cell for the levels whose children are reweighted, a cell's
    // blocks env_ndqstride float4 apart, offsets env_ndqoff_h[l] (-1: the
    // level's blocks come from env_dq)
    const float4 *env_dq;
    int64_t env_dqoff_h[16];
    const float4 *env_ndq;
    int64_t env_ndqoff_h[16];
    int64_t env_ndqstride;
    const float *env_nw;
    const float *env_nscale;
    const float *env_nfac;
    int32_t env_nregions;
    int32_t env_lstar;
    int64_t env_nstride;
    int64_t env_noff_h[16];
    float3 bb_lo, bb_hi;       // scene bounds (guiding features)
    // photon aiming (Sec. 2.1.3): binary hierarchy over clusters of objects,
    // node 0 the root; per node its sphere (centre, radius: encloses every
    // cluster sphere below; a leaf's is its cluster's) and its link
    // (left, right) or, for a leaf, (-1, cluster)
    const float4 *pa_node;
    const int2 *pa_link;
    int32_t pa_nnodes, pa_nclusters;
};

// ---------------------------------------------------------- error helpers
RT_D uint32_t lane_id() { return threadIdx.x & 31u; }

}  // namespace rtg
