// Host-side construction of the 8-wide compressed BVH used by the traversal
// kernels: binned-SAH binary build, collapse to 8-wide nodes, quantisation of
// child boxes to 8 bits per plane relative to a per-node origin and
// power-of-two scale (the compressed wide BVH of Ylitie, Karras and Laine,
// HPG 2017). The paper's own ray caster is a library (OptiX Prime, Sec. 3.1)
// and its GPU BVH builder is only cited (Sec. 2.5); this builder is new.
#pragma once

#include <cstdint>
#include <vector>

namespace rtg {

struct Bvh8 {
    std::vector<uint32_t> nodes;   // 20 uint32 (80 bytes) per node
    std::vector<float> tris;       // 12 floats (48 bytes) per leaf triangle
    std::vector<uint32_t> tri_ids; // original triangle index per leaf slot
    int64_t num_nodes() const { return (int64_t)nodes.size() / 20; }
    int64_t num_tris() const { return (int64_t)tris.size() / 12; }
    float lo[3], hi[3];            // root bounds
    int depth = 0;
};

// Build over triangles `tri_ids` (indices into `indices`) of a mesh given by
// `vertices` (V x 3) and `indices` (T x 3). `leaf_tris` is the maximum number
// of triangles per leaf slot (1..3). `threads` = worker threads (0 = auto).
void build_bvh8(const float *vertices, const uint32_t *indices, const uint32_t *tri_ids, int64_t n,
                Bvh8 &out, int threads = 0);

// Build a top-level 8-wide BVH over instance boxes (lo/hi: n x 3 floats);
// leaf slots hold one instance each, whose index is stored in `tri_ids`.
void build_bvh8_boxes(const float *lo, const float *hi, int64_t n, Bvh8 &out);

}  // namespace rtg
