// Host construction of the 8-wide compressed BVH (see bvh_build.h).
//
// Node encoding (80 bytes = 20 x uint32, read by the kernels as 5 x uint4):
//   [0..2]  p: float origin of the quantisation grid (= node box lower corner)
//   [3]     bytes: ex, ey, ez (int8 exponents, box plane = p + q * 2^e), imask
//   [4]     child_base: index of the first internal child node
//   [5]     tri_base: index of the first leaf triangle of this node
//   [6..7]  meta[8]: per child slot; 0 = empty; internal child:
//           0b001 << 5 | (24 + slot); leaf: unary triangle count (1, 3, 7)
//           << 5 | offset of its first triangle from tri_base
//   [8..9]  qlo_x[8], [10..11] qhi_x[8], [12..13] qlo_y, [14..15] qhi_y,
//   [16..17] qlo_z, [18..19] qhi_z (8-bit quantised child boxes)
// Internal children of a node are stored contiguously in slot order; the
// triangles of its leaf children likewise. Slot s holds the child nearest
// for rays whose direction-sign octant is 7 ^ s, so visiting slots in
// decreasing (s ^ octant) order is approximately front to back.
// Leaf triangle record: 3 x float4 (v0.xyz + triangle id bits, v1.xyz, v2.xyz).
#include "bvh_build.h"

#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstring>
#include <deque>
#include <future>

namespace rtg {
namespace {

struct AABB {
    float lo[3] = {FLT_MAX, FLT_MAX, FLT_MAX};
    float hi[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
    void grow(const AABB &b) {
        for (int a = 0; a < 3; ++a) {
            lo[a] = std::min(lo[a], b.lo[a]);
            hi[a] = std::max(hi[a], b.hi[a]);
        }
    }
    void grow(const float *p) {
        for (int a = 0; a < 3; ++a) {
            lo[a] = std::min(lo[a], p[a]);
            hi[a] = std::max(hi[a], p[a]);
        }
    }
    bool valid() const { return lo[0] <= hi[0]; }
    double area() const {
        if (!valid()) return 0.0;
        double dx = (double)hi[0] - lo[0], dy = (double)hi[1] - lo[1], dz = (double)hi[2] - lo[2];
        return 2.0 * (dx * dy + dy * dz + dz * dx);
    }
};

struct Prim {
    AABB b;
    float c[3];
    uint32_t id;
};

struct BNode {
    AABB b;
    int32_t left = -1, right = -1;  // left < 0: leaf
    int32_t first = 0, count = 0;
};

constexpr int kBins = 32;
constexpr double kCostNode = 1.0;
constexpr double kCostTri = 1.0;

struct Builder {
    std::vector<Prim> &prims;
    std::vector<BNode> nodes;
    int leaf_max;
    explicit Builder(std::vector<Prim> &p, int lm) : prims(p), leaf_max(lm) {}

    int32_t build(int32_t first, int32_t count, int depth) {
        int32_t id = (int32_t)nodes.size();
        nodes.emplace_back();
        AABB b, cb;
        for (int32_t i = first; i < first + count; ++i) {
            b.grow(prims[i].b);
            cb.grow(prims[i].c);
        }
        nodes[id].b = b;
        if (count <= 1) { make_leaf(id, first, count); return id; }
        // binned SAH over the three axes
        double best = DBL_MAX;
        int best_axis = -1, best_bin = -1;
        for (int a = 0; a < 3; ++a) {
            double ext = (double)cb.hi[a] - cb.lo[a];
            if (!(ext > 0.0)) continue;
            AABB bb[kBins];
            int cnt[kBins] = {0};
            double scale = kBins / ext;
            for (int32_t i = first; i < first + count; ++i) {
                int k = (int)((prims[i].c[a] - cb.lo[a]) * scale);
                k = std::min(kBins - 1, std::max(0, k));
                bb[k].grow(prims[i].b);
                ++cnt[k];
            }
            double rarea[kBins];
            int rcnt[kBins];
            AABB acc;
            int n = 0;
            for (int k = kBins - 1; k > 0; --k) {
                acc.grow(bb[k]);
                n += cnt[k];
                rarea[k] = acc.area();
                rcnt[k] = n;
            }
            AABB lacc;
            int ln = 0;
            for (int k = 0; k < kBins - 1; ++k) {
                lacc.grow(bb[k]);
                ln += cnt[k];
                if (ln == 0 || rcnt[k + 1] == 0) continue;
                double c = lacc.area() * ln + rarea[k + 1] * rcnt[k + 1];
                if (c < best) { best = c; best_axis = a; best_bin = k; }
            }
        }
        double area = b.area();
        double leaf_cost = kCostTri * count * area;
        double split_cost = kCostNode * area + kCostTri * best;
        if (count <= leaf_max && (best_axis < 0 || leaf_cost <= split_cost)) {
            make_leaf(id, first, count);
            return id;
        }
        int32_t mid;
        if (best_axis >= 0) {
            double ext = (double)cb.hi[best_axis] - cb.lo[best_axis];
            double scale = kBins / ext;
            auto it = std::partition(prims.begin() + first, prims.begin() + first + count, [&](const Prim &p) {
                int k = (int)((p.c[best_axis] - cb.lo[best_axis]) * scale);
                k = std::min(kBins - 1, std::max(0, k));
                return k <= best_bin;
            });
            mid = (int32_t)(it - prims.begin());
        } else {
            mid = first + count / 2;
        }
        if (mid <= first || mid >= first + count) {
            // all centroids coincide: split by index
            mid = first + count / 2;
        }
        int32_t l = build(first, mid - first, depth + 1);
        int32_t r = build(mid, first + count - mid, depth + 1);
        nodes[id].left = l;
        nodes[id].right = r;
        return id;
    }

    void make_leaf(int32_t id, int32_t first, int32_t count) {
        nodes[id].left = -1;
        nodes[id].first = first;
        nodes[id].count = count;
    }
};

int exponent_for(double extent) {
    if (!(extent > 0.0)) return -100;
    int e = (int)std::ceil(std::log2(extent / 255.0));
    while (std::ldexp(255.0, e) < extent) ++e;
    return std::max(-100, std::min(100, e));
}

void collapse(const std::vector<BNode> &bn, const std::vector<Prim> &prims, int32_t root, bool with_tris,
              const float *vertices, const uint32_t *indices, Bvh8 &out) {
    struct Item { int32_t bnode; int64_t wide; int depth; };
    std::deque<Item> queue;
    out.nodes.assign(20, 0u);
    queue.push_back({root, 0, 1});
    int64_t next_node = 1;
    out.depth = 1;
    while (!queue.empty()) {
        Item it = queue.front();
        queue.pop_front();
        out.depth = std::max(out.depth, it.depth);
        const BNode &X = bn[it.bnode];
        std::vector<int32_t> ch;
        if (X.left < 0) {
            ch.push_back(it.bnode);
        } else {
            ch.push_back(X.left);
            ch.push_back(X.right);
            while (ch.size() < 8) {
                int pick = -1;
                double pa = -1.0;
                for (int i = 0; i < (int)ch.size(); ++i) {
                    const BNode &c = bn[ch[i]];
                    if (c.left >= 0 && c.b.area() > pa) { pa = c.b.area(); pick = i; }
                }
                if (pick < 0) break;
                int32_t c = ch[pick];
                ch[pick] = bn[c].left;
                ch.push_back(bn[c].right);
            }
        }
        // slot assignment by octant (greedy on sorted costs)
        int nch = (int)ch.size();
        double cx = 0.5 * ((double)X.b.lo[0] + X.b.hi[0]), cy = 0.5 * ((double)X.b.lo[1] + X.b.hi[1]),
               cz = 0.5 * ((double)X.b.lo[2] + X.b.hi[2]);
        struct Cand { double cost; int child, slot; };
        std::vector<Cand> cand;
        for (int i = 0; i < nch; ++i) {
            const AABB &b = bn[ch[i]].b;
            double dx = 0.5 * ((double)b.lo[0] + b.hi[0]) - cx, dy = 0.5 * ((double)b.lo[1] + b.hi[1]) - cy,
                   dz = 0.5 * ((double)b.lo[2] + b.hi[2]) - cz;
            for (int s = 0; s < 8; ++s) {
                int o = 7 ^ s;
                double c = ((o & 1) ? -dx : dx) + ((o & 2) ? -dy : dy) + ((o & 4) ? -dz : dz);
                cand.push_back({c, i, s});
            }
        }
        std::sort(cand.begin(), cand.end(), [](const Cand &a, const Cand &b) {
            if (a.cost != b.cost) return a.cost < b.cost;
            if (a.child != b.child) return a.child < b.child;
            return a.slot < b.slot;
        });
        int slot_child[8];
        bool used_child[8] = {false};
        for (int s = 0; s < 8; ++s) slot_child[s] = -1;
        for (const Cand &c : cand) {
            if (used_child[c.child] || slot_child[c.slot] >= 0) continue;
            slot_child[c.slot] = c.child;
            used_child[c.child] = true;
        }
        // node header
        uint32_t *N = &out.nodes[(size_t)it.wide * 20];
        float p[3] = {X.b.lo[0], X.b.lo[1], X.b.lo[2]};
        int e[3];
        for (int a = 0; a < 3; ++a) e[a] = exponent_for((double)X.b.hi[a] - p[a]);
        std::memcpy(&N[0], p, 12);
        uint8_t imask = 0;
        uint8_t meta[8] = {0};
        uint8_t qlo[3][8], qhi[3][8];
        for (int a = 0; a < 3; ++a)
            for (int s = 0; s < 8; ++s) { qlo[a][s] = 255; qhi[a][s] = 0; }
        int64_t child_base = next_node;
        int64_t tri_base = with_tris ? out.num_tris() : (int64_t)out.tri_ids.size();
        int tri_off = 0;
        for (int s = 0; s < 8; ++s) {
            int ci = slot_child[s];
            if (ci < 0) continue;
            const BNode &C = bn[ch[ci]];
            for (int a = 0; a < 3; ++a) {
                double sc = std::ldexp(1.0, e[a]);
                double lo = std::floor(((double)C.b.lo[a] - p[a]) / sc) - 1.0;
                double hi = std::ceil(((double)C.b.hi[a] - p[a]) / sc) + 1.0;
                qlo[a][s] = (uint8_t)std::max(0.0, std::min(255.0, lo));
                qhi[a][s] = (uint8_t)std::max(0.0, std::min(255.0, hi));
            }
            if (C.left >= 0) {
                imask |= (uint8_t)(1u << s);
                meta[s] = (uint8_t)((1u << 5) | (24u + s));
                queue.push_back({ch[ci], next_node, it.depth + 1});
                ++next_node;
                out.nodes.resize((size_t)next_node * 20, 0u);
                N = &out.nodes[(size_t)it.wide * 20];
            } else {
                static const uint8_t unary[4] = {0, 1, 3, 7};
                meta[s] = (uint8_t)((unary[C.count] << 5) | tri_off);
                for (int32_t k = 0; k < C.count; ++k) {
                    uint32_t id = prims[C.first + k].id;
                    out.tri_ids.push_back(id);
                    if (with_tris) {
                        float rec[12];
                        for (int v = 0; v < 3; ++v)
                            for (int a = 0; a < 3; ++a)
                                rec[4 * v + a] = vertices[3 * (size_t)indices[3 * (size_t)id + v] + a];
                        std::memcpy(&rec[3], &id, 4);
                        rec[7] = rec[11] = 0.f;
                        out.tris.insert(out.tris.end(), rec, rec + 12);
                    }
                }
                tri_off += C.count;
            }
        }
        N[3] = (uint32_t)(uint8_t)(int8_t)e[0] | ((uint32_t)(uint8_t)(int8_t)e[1] << 8) |
               ((uint32_t)(uint8_t)(int8_t)e[2] << 16) | ((uint32_t)imask << 24);
        N[4] = (uint32_t)child_base;
        N[5] = (uint32_t)tri_base;
        std::memcpy(&N[6], meta, 8);
        for (int a = 0; a < 3; ++a) {
            std::memcpy(&N[8 + 4 * a], qlo[a], 8);
            std::memcpy(&N[10 + 4 * a], qhi[a], 8);
        }
    }
}

}  // namespace

void build_bvh8(const float *vertices, const uint32_t *indices, const uint32_t *tri_ids, int64_t n, Bvh8 &out,
                int threads) {
    (void)threads;
    std::vector<Prim> prims;
    prims.reserve((size_t)n);
    AABB root;
    for (int64_t i = 0; i < n; ++i) {
        Prim p;
        uint32_t id = tri_ids ? tri_ids[i] : (uint32_t)i;
        for (int v = 0; v < 3; ++v) p.b.grow(&vertices[3 * (size_t)indices[3 * (size_t)id + v]]);
        for (int a = 0; a < 3; ++a) p.c[a] = 0.5f * (p.b.lo[a] + p.b.hi[a]);
        p.id = id;
        root.grow(p.b);
        prims.push_back(p);
    }
    out = Bvh8{};
    for (int a = 0; a < 3; ++a) { out.lo[a] = root.lo[a]; out.hi[a] = root.hi[a]; }
    if (n == 0) {
        out.nodes.assign(20, 0u);   // one empty node: every slot empty
        return;
    }
    Builder b(prims, 3);
    b.nodes.reserve((size_t)(2 * n));
    int32_t r = b.build(0, (int32_t)n, 0);
    collapse(b.nodes, prims, r, true, vertices, indices, out);
}

void build_bvh8_boxes(const float *lo, const float *hi, int64_t n, Bvh8 &out) {
    std::vector<Prim> prims;
    prims.reserve((size_t)n);
    AABB root;
    for (int64_t i = 0; i < n; ++i) {
        Prim p;
        for (int a = 0; a < 3; ++a) {
            p.b.lo[a] = lo[3 * i + a];
            p.b.hi[a] = hi[3 * i + a];
            p.c[a] = 0.5f * (p.b.lo[a] + p.b.hi[a]);
        }
        p.id = (uint32_t)i;
        root.grow(p.b);
        prims.push_back(p);
    }
    out = Bvh8{};
    for (int a = 0; a < 3; ++a) { out.lo[a] = root.lo[a]; out.hi[a] = root.hi[a]; }
    if (n == 0) {
        out.nodes.assign(20, 0u);
        return;
    }
    Builder b(prims, 1);
    int32_t r = b.build(0, (int32_t)n, 0);
    collapse(b.nodes, prims, r, false, nullptr, nullptr, out);
}

}  // namespace rtg
