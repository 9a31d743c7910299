// rt_scene_create / rt_scene_destroy / rt_scene_info: host preprocessing of a
// scene and its upload to device memory (paper Sec. 2.1.1: one flux value per
// emitting triangle computed in a preprocess; Sec. 2.1.2: the environment
// hierarchy built in a preprocess; Sec. 5.6: the whole scene resides in the
// memory of each device).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>
#include <vector>

#include "internal.h"
#include "traverse.cuh"

namespace rtg {
namespace {

template <class T>
rt_status upload(rt_scene *s, const T *host, size_t count, const T **dev_out, const T **host_out) {
    *dev_out = nullptr;
    if (host_out) *host_out = nullptr;
    if (count == 0 || host == nullptr) return RT_OK;
    if (host_out && s->host_only) {
        std::vector<uint8_t> keep(count * sizeof(T));
        std::memcpy(keep.data(), host, keep.size());
        s->host_keep.push_back(std::move(keep));
        *host_out = (const T *)s->host_keep.back().data();
    }
    if (s->host_only) return RT_OK;
    void *d = nullptr;
    cudaError_t e = cudaMalloc(&d, count * sizeof(T));
    if (e != cudaSuccess) {
        set_error("cudaMalloc failed for scene data");
        return e == cudaErrorMemoryAllocation ? RT_OOM : RT_CUDA_ERROR;
    }
    s->dev_allocs.push_back(d);
    s->device_bytes += (int64_t)(count * sizeof(T));
    RT_CUDA_TRY(cudaMemcpy(d, host, count * sizeof(T), cudaMemcpyHostToDevice));
    *dev_out = (const T *)d;
    return RT_OK;
}

#define RT_TRY(expr)                       \
    do {                                   \
        rt_status _s = (expr);             \
        if (_s != RT_OK) return _s;        \
    } while (0)

double lum3(const float *c) { return 0.2126 * c[0] + 0.7152 * c[1] + 0.0722 * c[2]; }

// ---- normal-oriented top levels of the environment pyramid (Sec. 2.1.2)
struct Dir3 {
    double x, y, z;
};

Dir3 unit3(double x, double y, double z) {
    double l = std::sqrt(x * x + y * y + z * z);
    return l > 0.0 ? Dir3{x / l, y / l, z / l} : Dir3{x, y, z};
}

double angle3(const Dir3 &a, const Dir3 &b) {
    return std::acos(std::min(1.0, std::max(-1.0, a.x * b.x + a.y * b.y + a.z * b.z)));
}

// Point (px, pz) of the octahedral square [-1, 1]^2 on the unit sphere: the
// upper hemisphere over the inner diamond, the lower one folded outside it.
Dir3 octahedral_dir(double px, double pz) {
    double y = 1.0 - std::fabs(px) - std::fabs(pz);
    if (y < 0.0) {
        double fx = (1.0 - std::fabs(pz)) * (px >= 0.0 ? 1.0 : -1.0);
        double fz = (1.0 - std::fabs(px)) * (pz >= 0.0 ? 1.0 : -1.0);
        px = fx;
        pz = fz;
    }
    return unit3(px, y, pz);
}

// Direction at polar angle theta from +y and azimuth phi from +x towards +z.
Dir3 polar_dir(double theta, double phi) {
    return Dir3{std::sin(theta) * std::cos(phi), std::cos(theta), std::sin(theta) * std::sin(phi)};
}

// Angular radius about `centre` of a patch of the sphere given by its map
// f(s, t), s, t in [0, 1]: the largest angle from the centre to the points of
// a 17 x 17 grid, plus the longest diagonal of a grid square so that the
// points between grid points are covered too.
template <class F>
double patch_radius(const Dir3 &centre, F f) {
    constexpr int G = 16;
    Dir3 g[G + 1][G + 1];
    for (int a = 0; a <= G; ++a)
        for (int b = 0; b <= G; ++b) g[a][b] = f((double)a / G, (double)b / G);
    double far = 0.0, diag = 0.0;
    for (int a = 0; a <= G; ++a)
        for (int b = 0; b <= G; ++b) {
            far = std::max(far, angle3(centre, g[a][b]));
            if (a < G && b < G)
                diag = std::max(diag, std::max(angle3(g[a][b], g[a + 1][b + 1]), angle3(g[a + 1][b], g[a][b + 1])));
        }
    return far + diag;
}

struct EnvNormalTables {
    int lstar = 0, nregions = 0;
    int64_t stride = 0;
    int64_t off[16] = {};
    std::vector<float> nw, scale, fac;
};

// Per normal cell: level lstar = the finest of the top kLevels (five)
// levels holds w(R) x kappa_c(R), kappa the clamped cosine at the smallest
// angle between a normal of the cell's cone and a direction of region R's
// cone (1 where the cones overlap, 0 beyond 90 degrees); coarser levels are
// sums of their children. lv[l] = plain weights of level l (W >> l columns).
void build_env_normal_tables(const std::vector<std::vector<double>> &lv, int32_t W, int32_t H, int levels,
                             double env_sum, EnvNormalTables &t) {
    constexpr int side = 8, cells = side * side, kLevels = 5;
    const double pi = M_PI;
    const int top = levels - 1;
    t.lstar = std::max(0, top - kLevels + 1);
    auto lw = [&](int l) { return W >> l; };
    auto lh = [&](int l) { return std::max(1, H >> l); };
    t.stride = 0;
    for (int l = top; l >= t.lstar; --l) {
        t.off[l] = t.stride;
        t.stride += (int64_t)lw(l) * lh(l);
    }
    const int ls = t.lstar, rw = lw(ls), rh = lh(ls);
    t.nregions = rw * rh;
    std::vector<Dir3> rc(t.nregions);
    std::vector<double> rb(t.nregions);
    for (int y = 0; y < rh; ++y)
        for (int x = 0; x < rw; ++x) {
            const double th0 = pi * y / rh, th1 = pi * (y + 1) / rh;
            const double ph0 = 2.0 * pi * x / rw, ph1 = 2.0 * pi * (x + 1) / rw;
            const int r = y * rw + x;
            rc[r] = polar_dir(0.5 * (th0 + th1), 0.5 * (ph0 + ph1));
            rb[r] = patch_radius(rc[r], [&](double s_, double t_) {
                return polar_dir(th0 + (th1 - th0) * s_, ph0 + (ph1 - ph0) * t_);
            });
        }
    t.nw.assign((size_t)cells * t.stride, 0.f);
    t.scale.assign(cells, 0.f);
    t.fac.assign((size_t)cells * t.nregions, 1.f);
    std::vector<double> blk(t.stride), kap(t.nregions);
    for (int c = 0; c < cells; ++c) {
        const int ci = c % side, cj = c / side;
        auto cell_point = [&](double s_, double t_) {
            return octahedral_dir(2.0 * (ci + s_) / side - 1.0, 2.0 * (cj + t_) / side - 1.0);
        };
        const Dir3 nc = cell_point(0.5, 0.5);
        const double alpha = patch_radius(nc, cell_point);
        std::fill(blk.begin(), blk.end(), 0.0);
        double total = 0.0;
        for (int r = 0; r < t.nregions; ++r) {
            const double gap = angle3(nc, rc[r]) - alpha - rb[r];
            kap[r] = gap <= 0.0 ? 1.0 : (gap >= 0.5 * pi ? 0.0 : std::cos(gap));
            blk[t.off[ls] + r] = lv[ls][r] * kap[r];
            total += blk[t.off[ls] + r];
        }
        for (int l = ls + 1; l <= top; ++l)
            for (int y = 0; y < lh(l - 1); ++y)
                for (int x = 0; x < lw(l - 1); ++x)
                    blk[t.off[l] + (int64_t)(y / 2) * lw(l) + x / 2] += blk[t.off[l - 1] + (int64_t)y * lw(l - 1) + x];
        for (int64_t i = 0; i < t.stride; ++i) t.nw[(size_t)c * t.stride + i] = (float)blk[i];
        if (total > 0.0) {
            t.scale[c] = (float)(env_sum / total);
            for (int r = 0; r < t.nregions; ++r) t.fac[(size_t)c * t.nregions + r] = (float)(kap[r] * env_sum / total);
        }
    }
}

// ---- probabilistic light hierarchy (Sec. 2.1.1)
struct LightBvh {
    std::vector<float4> nodes;   // 4 float4 per node: (centre, r), (I0..I3), (I4, I5, flux, 0), links (below)
    std::vector<uint32_t> perm;  // leaf slot -> emitter
    std::vector<uint32_t> leaf;  // emitter -> leaf node
};
// links of a node, as uint bits: left, right (0xffffffff in a leaf), parent
// (0xffffffff at the root), leaf word (first slot << 3 | count; 0 if internal)

// Descent records (DevScene::lb_rec) from the node tree: one per internal
// node, both children's data and links side by side; per emitter the record
// of its leaf's parent and the side.
void light_bvh_records(const LightBvh &t, std::vector<float4> &rec, std::vector<uint32_t> &up) {
    const size_t nn = t.nodes.size() / 4;
    auto links = [&](size_t i) {
        const float4 d = t.nodes[4 * i + 3];
        return make_uint4(as_uint(d.x), as_uint(d.y), as_uint(d.z), as_uint(d.w));
    };
    std::vector<uint32_t> rmap(nn, 0xffffffffu);
    uint32_t nrec = 0;
    for (size_t i = 0; i < nn; ++i)
        if (links(i).w == 0u) rmap[i] = nrec++;
    rec.clear();
    up.assign(t.leaf.size(), 0u);
    const float4 empty = make_float4(0.f, 0.f, 0.f, 0.f);
    if (nrec == 0) {
        // a single leaf: one record, the leaf on side 0, nothing on side 1
        rec.push_back(t.nodes[0]);
        rec.push_back(t.nodes[1]);
        float4 c = t.nodes[2];
        c.w = as_float(0x80000000u | links(0).w);
        rec.push_back(c);
        rec.push_back(empty);
        rec.push_back(empty);
        rec.push_back(make_float4(0.f, 0.f, 0.f, as_float(0x80000000u)));
        rec.push_back(make_float4(as_float(0xffffffffu), as_float(0u), 0.f, 0.f));
        return;
    }
    rec.resize(7 * (size_t)nrec);
    for (size_t i = 0; i < nn; ++i) {
        const uint4 L = links(i);
        if (L.w != 0u) continue;
        float4 *R = rec.data() + 7 * (size_t)rmap[i];
        for (int side = 0; side < 2; ++side) {
            const uint32_t ch = side ? L.y : L.x;
            const uint4 cl = links(ch);
            float4 c = t.nodes[4 * (size_t)ch + 2];
            c.w = as_float(cl.w != 0u ? (0x80000000u | cl.w) : rmap[ch]);
            R[3 * side] = t.nodes[4 * (size_t)ch];
            R[3 * side + 1] = t.nodes[4 * (size_t)ch + 1];
            R[3 * side + 2] = c;
        }
        const uint32_t par = L.z;
        const uint32_t pside = par == 0xffffffffu ? 0u : (links(par).x == (uint32_t)i ? 0u : 1u);
        R[6] = make_float4(as_float(par == 0xffffffffu ? 0xffffffffu : rmap[par]), as_float(pside), 0.f, 0.f);
    }
    for (size_t e = 0; e < t.leaf.size(); ++e) {
        const uint32_t lf = t.leaf[e], par = links(lf).z;
        up[e] = rmap[par] << 1 | (links(par).x == lf ? 0u : 1u);
    }
}

// Binary tree over the emitters (three world-space vertices each in lv,
// fluxes in flux): leaves of at most kLeaf emitters; a larger set is ordered
// by centroid along the longest axis of its centroid bounds (ties: the lower
// axis, then the lower emitter index) and split at count / 2. Per node: box
// centre and half diagonal, flux, and per cube-face region k the sum over
// its emitters of flux x (the largest clamped cosine between the emitter's
// normal and the directions of a cone around face axis k that holds the
// region).
void build_light_bvh(const std::vector<float4> &lv, const std::vector<double> &flux, LightBvh &out) {
    constexpr int kLeaf = 4;
    const size_t n = flux.size();
    const double face_half_angle = std::acos(1.0 / std::sqrt(3.0));
    std::vector<Dir3> nrm(n);
    std::vector<double> cen(3 * n);
    for (size_t e = 0; e < n; ++e) {
        const float4 a = lv[3 * e], b = lv[3 * e + 1], c = lv[3 * e + 2];
        const double ex = (double)b.x - a.x, ey = (double)b.y - a.y, ez = (double)b.z - a.z;
        const double fx = (double)c.x - a.x, fy = (double)c.y - a.y, fz = (double)c.z - a.z;
        nrm[e] = unit3(ey * fz - ez * fy, ez * fx - ex * fz, ex * fy - ey * fx);
        cen[3 * e] = ((double)a.x + b.x + c.x) / 3.0;
        cen[3 * e + 1] = ((double)a.y + b.y + c.y) / 3.0;
        cen[3 * e + 2] = ((double)a.z + b.z + c.z) / 3.0;
    }
    auto kappa = [](double g) { return g <= 0.0 ? 1.0 : (g >= 0.5 * M_PI ? 0.0 : std::cos(g)); };
    std::vector<double> lobe(6 * n);   // per emitter and region: flux x bound of its cosine lobe
    for (size_t e = 0; e < n; ++e)
        for (int k = 0; k < 6; ++k) {
            Dir3 ax{0.0, 0.0, 0.0};
            (k / 2 == 0 ? ax.x : (k / 2 == 1 ? ax.y : ax.z)) = (k & 1) ? -1.0 : 1.0;
            lobe[6 * e + k] = flux[e] * kappa(angle3(nrm[e], ax) - face_half_angle);
        }
    out.perm.resize(n);
    out.leaf.assign(n, 0u);
    for (size_t e = 0; e < n; ++e) out.perm[e] = (uint32_t)e;
    out.nodes.clear();
    out.nodes.reserve(4 * (2 * n));
    struct Item { size_t first, count; int32_t parent; bool is_left; };
    std::vector<Item> todo{{0, n, -1, false}};
    while (!todo.empty()) {
        Item it = todo.back();
        todo.pop_back();
        const int32_t id = (int32_t)(out.nodes.size() / 4);
        if (it.parent >= 0) {
            float4 &links = out.nodes[4 * (size_t)it.parent + 3];
            (it.is_left ? links.x : links.y) = as_float((uint32_t)id);
        }
        double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
        double clo[3] = {INFINITY, INFINITY, INFINITY}, chi[3] = {-INFINITY, -INFINITY, -INFINITY};
        double F = 0.0, I[6] = {0, 0, 0, 0, 0, 0};
        for (size_t i = it.first; i < it.first + it.count; ++i) {
            const uint32_t e = out.perm[i];
            for (int v = 0; v < 3; ++v) {
                const float4 p = lv[3 * (size_t)e + v];
                const double q[3] = {p.x, p.y, p.z};
                for (int a = 0; a < 3; ++a) { lo[a] = std::min(lo[a], q[a]); hi[a] = std::max(hi[a], q[a]); }
            }
            for (int a = 0; a < 3; ++a) {
                clo[a] = std::min(clo[a], cen[3 * (size_t)e + a]);
                chi[a] = std::max(chi[a], cen[3 * (size_t)e + a]);
            }
            F += flux[e];
            for (int k = 0; k < 6; ++k) I[k] += lobe[6 * (size_t)e + k];
        }
        const double dx = hi[0] - lo[0], dy = hi[1] - lo[1], dz = hi[2] - lo[2];
        out.nodes.push_back(make_float4((float)(0.5 * (lo[0] + hi[0])), (float)(0.5 * (lo[1] + hi[1])),
                                        (float)(0.5 * (lo[2] + hi[2])), (float)(0.5 * std::sqrt(dx * dx + dy * dy + dz * dz))));
        out.nodes.push_back(make_float4((float)I[0], (float)I[1], (float)I[2], (float)I[3]));
        out.nodes.push_back(make_float4((float)I[4], (float)I[5], (float)F, 0.f));
        out.nodes.push_back(make_float4(as_float(0xffffffffu), as_float(0xffffffffu), as_float((uint32_t)it.parent), 0.f));
        if (it.count <= (size_t)kLeaf) {
            out.nodes.back().w = as_float((uint32_t)(it.first << 3) | (uint32_t)it.count);
            for (size_t i = it.first; i < it.first + it.count; ++i) out.leaf[out.perm[i]] = (uint32_t)id;
            continue;
        }
        int axis = 0;
        for (int a = 1; a < 3; ++a)
            if (chi[a] - clo[a] > chi[axis] - clo[axis]) axis = a;
        std::sort(out.perm.begin() + it.first, out.perm.begin() + it.first + it.count, [&](uint32_t a, uint32_t b) {
            const double ca = cen[3 * (size_t)a + axis], cb = cen[3 * (size_t)b + axis];
            return ca < cb || (ca == cb && a < b);
        });
        const size_t half = it.count / 2;
        // right pushed first so that the left subtree is numbered first
        todo.push_back({it.first + half, it.count - half, id, false});
        todo.push_back({it.first, half, id, true});
    }
}

// Mean luminance of a textured emitter over its triangle, by stratified
// supersampling of the UV footprint (16 x 16 strata, nearest texel).
double textured_mean(const rt_scene_desc *d, int64_t t, int32_t tex) {
    const uint32_t *id = d->indices + 3 * t;
    double acc = 0.0;
    const int n = 16;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double u1 = (i + 0.5) / n, u2 = (j + 0.5) / n;
            double su = std::sqrt(u1);
            double b1 = su * (1.0 - u2), b2 = su * u2, b0 = 1.0 - su;
            double u = b0 * d->uvs[2 * id[0]] + b1 * d->uvs[2 * id[1]] + b2 * d->uvs[2 * id[2]];
            double v = b0 * d->uvs[2 * id[0] + 1] + b1 * d->uvs[2 * id[1] + 1] + b2 * d->uvs[2 * id[2] + 1];
            int x = (int)std::floor(std::min(1.0, std::max(0.0, u)) * d->tex_width);
            int y = (int)std::floor(std::min(1.0, std::max(0.0, v)) * d->tex_height);
            x = std::min(x, d->tex_width - 1);
            y = std::min(y, d->tex_height - 1);
            acc += lum3(d->textures + 3 * (((size_t)tex * d->tex_height + y) * d->tex_width + x));
        }
    return acc / (n * n);
}

// Vose's alias method in double precision; thresholds stored as float.
void build_alias(const std::vector<double> &w, std::vector<float2> &out) {
    size_t n = w.size();
    double sum = 0.0;
    for (double x : w) sum += x;
    std::vector<double> p(n);
    std::vector<uint32_t> small, large;
    out.assign(n, make_float2(1.f, 0.f));
    for (size_t i = 0; i < n; ++i) {
        p[i] = w[i] * (double)n / sum;
        uint32_t self = (uint32_t)i;
        float bits;
        std::memcpy(&bits, &self, 4);
        out[i] = make_float2(1.f, bits);
        (p[i] < 1.0 ? small : large).push_back((uint32_t)i);
    }
    while (!small.empty() && !large.empty()) {
        uint32_t s = small.back(); small.pop_back();
        uint32_t g = large.back(); large.pop_back();
        float bits;
        std::memcpy(&bits, &g, 4);
        out[s] = make_float2((float)p[s], bits);
        p[g] = (p[g] + p[s]) - 1.0;
        (p[g] < 1.0 ? small : large).push_back(g);
    }
}

}  // namespace
}  // namespace rtg

using namespace rtg;

namespace rtg {
rt_status scene_create(const rt_scene_desc *d, rt_scene **out, bool host_only);

// Photon aiming (Sec. 2.1.3): clusters of objects and the hierarchy that
// samples them. Objects: the connected components of the mesh (single-level
// scenes) or the instances; two objects belong to one cluster when a chain
// of links joins them, a link being a pair of similar size (neither radius
// above twice the other) whose boxes intersect; a cluster's sphere is the
// centre and half diagonal of its box. The hierarchy splits a set of
// clusters at its median cluster along the longest axis of the centres
// (order: centre, then cluster index); a node's sphere is centred on its
// box and encloses each cluster sphere below it.
struct AimBox {
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    void add(const double *p) {
        for (int a = 0; a < 3; ++a) { lo[a] = std::min(lo[a], p[a]); hi[a] = std::max(hi[a], p[a]); }
    }
    void add(const AimBox &b) { add(b.lo); add(b.hi); }
    void centre(double c[3]) const { for (int a = 0; a < 3; ++a) c[a] = 0.5 * (lo[a] + hi[a]); }
    double radius() const {
        double e2 = 0.0;
        for (int a = 0; a < 3; ++a) e2 += (hi[a] - lo[a]) * (hi[a] - lo[a]);
        return 0.5 * std::sqrt(e2);
    }
};

struct DisjointSets {
    std::vector<int32_t> up;
    explicit DisjointSets(size_t n) : up(n) { for (size_t i = 0; i < n; ++i) up[i] = (int32_t)i; }
    int32_t root(int32_t a) {
        while (up[a] != a) { up[a] = up[up[a]]; a = up[a]; }
        return a;
    }
    void join(int32_t a, int32_t b) {
        a = root(a); b = root(b);
        if (a != b) { if (a < b) up[b] = a; else up[a] = b; }
    }
};

struct AimTree {
    std::vector<float4> node;
    std::vector<int2> link;
    int32_t nclusters = 0;
};

static void aim_tree(const std::vector<AimBox> &objects, AimTree &out) {
    const int32_t n = (int32_t)objects.size();
    if (n == 0) return;
    std::vector<double> oc(3 * (size_t)n), orad(n);
    for (int32_t i = 0; i < n; ++i) { objects[i].centre(&oc[3 * (size_t)i]); orad[i] = objects[i].radius(); }
    DisjointSets ds(n);
    for (int32_t a = 0; a < n; ++a)
        for (int32_t b = a + 1; b < n; ++b) {
            if (!(orad[a] <= 2.0 * orad[b] && orad[b] <= 2.0 * orad[a])) continue;
            bool meet = true;
            for (int k = 0; k < 3; ++k)
                if (objects[a].lo[k] > objects[b].hi[k] || objects[b].lo[k] > objects[a].hi[k]) meet = false;
            if (meet) ds.join(a, b);
        }
    // clusters numbered in the order of their first object
    std::vector<int32_t> cl_of(n, -1), obj_cl(n);
    int32_t ncl = 0;
    for (int32_t i = 0; i < n; ++i) {
        const int32_t r = ds.root(i);
        if (cl_of[r] < 0) cl_of[r] = ncl++;
        obj_cl[i] = cl_of[r];
    }
    std::vector<AimBox> cb(ncl);
    for (int32_t i = 0; i < n; ++i) cb[obj_cl[i]].add(objects[i]);
    std::vector<double> cc(3 * (size_t)ncl), cr(ncl);
    for (int32_t c = 0; c < ncl; ++c) { cb[c].centre(&cc[3 * (size_t)c]); cr[c] = cb[c].radius(); }
    out.nclusters = ncl;
    out.node.clear();
    out.link.clear();
    std::vector<int32_t> idx(ncl);
    for (int32_t c = 0; c < ncl; ++c) idx[c] = c;
    std::function<int32_t(int32_t, int32_t)> build = [&](int32_t first, int32_t count) -> int32_t {
        const int32_t id = (int32_t)out.node.size();
        out.node.push_back(make_float4(0.f, 0.f, 0.f, 0.f));
        out.link.push_back(make_int2(-1, -1));
        AimBox nb;
        for (int32_t i = first; i < first + count; ++i) nb.add(cb[idx[i]]);
        double c[3];
        nb.centre(c);
        double r = 0.0;
        for (int32_t i = first; i < first + count; ++i) {
            const double *q = &cc[3 * (size_t)idx[i]];
            const double dd = std::sqrt((q[0] - c[0]) * (q[0] - c[0]) + (q[1] - c[1]) * (q[1] - c[1]) +
                                        (q[2] - c[2]) * (q[2] - c[2]));
            r = std::max(r, dd + cr[idx[i]]);
        }
        out.node[id] = make_float4((float)c[0], (float)c[1], (float)c[2], (float)r);
        if (count == 1) {
            out.link[id] = make_int2(-1, idx[first]);
            return id;
        }
        double clo[3] = {INFINITY, INFINITY, INFINITY}, chi[3] = {-INFINITY, -INFINITY, -INFINITY};
        for (int32_t i = first; i < first + count; ++i)
            for (int a = 0; a < 3; ++a) {
                clo[a] = std::min(clo[a], cc[3 * (size_t)idx[i] + a]);
                chi[a] = std::max(chi[a], cc[3 * (size_t)idx[i] + a]);
            }
        int axis = 0;
        for (int a = 1; a < 3; ++a)
            if (chi[a] - clo[a] > chi[axis] - clo[axis]) axis = a;
        std::sort(idx.begin() + first, idx.begin() + first + count, [&](int32_t p, int32_t q) {
            const double a = cc[3 * (size_t)p + axis], b = cc[3 * (size_t)q + axis];
            return a < b || (a == b && p < q);
        });
        const int32_t h = count / 2;
        const int32_t l = build(first, h);
        const int32_t rr = build(first + h, count - h);
        out.link[id] = make_int2(l, rr);
        return id;
    };
    build(0, ncl);
}
}

extern "C" rt_status rt_scene_create(const rt_scene_desc *d, rt_scene **out) {
    return scene_create(d, out, false);
}

/* Host-only copy of the scene for the CPU test hooks (no device memory). */
extern "C" rt_status rt_debug_scene_create_host(const rt_scene_desc *d, rt_scene **out) {
    return scene_create(d, out, true);
}

rt_status rtg::scene_create(const rt_scene_desc *d, rt_scene **out, bool host_only) {
    if (!d || !out) { set_error("rt_scene_create: null argument"); return RT_INVALID_ARG; }
    *out = nullptr;
    if (d->num_triangles < 0 || d->num_vertices < 0 || (d->num_triangles > 0 && (!d->vertices || !d->indices ||
                                                                                   !d->tri_material))) {
        set_error("rt_scene_create: missing geometry arrays");
        return RT_INVALID_ARG;
    }
    if (d->num_instances > 0) {
        if (d->num_meshes <= 0 || !d->mesh_tri_offset || !d->instance_mesh || !d->instance_xform) {
            set_error("rt_scene_create: instancing needs meshes, instance_mesh and instance_xform");
            return RT_INVALID_ARG;
        }
        for (int32_t m = 0; m < d->num_meshes; ++m)
            if (d->mesh_tri_offset[m] < 0 || d->mesh_tri_offset[m] > d->mesh_tri_offset[m + 1] ||
                d->mesh_tri_offset[m + 1] > d->num_triangles) {
                set_error("rt_scene_create: mesh_tri_offset must be non-decreasing within [0, num_triangles]");
                return RT_INVALID_ARG;
            }
        for (int32_t k = 0; k < d->num_instances; ++k) {
            if ((int32_t)d->instance_mesh[k] >= d->num_meshes) { set_error("rt_scene_create: instance_mesh out of range"); return RT_INVALID_ARG; }
            const float *X = d->instance_xform + 12 * (size_t)k;
            double det = (double)X[0] * ((double)X[5] * X[10] - (double)X[6] * X[9]) -
                         (double)X[1] * ((double)X[4] * X[10] - (double)X[6] * X[8]) +
                         (double)X[2] * ((double)X[4] * X[9] - (double)X[5] * X[8]);
            if (!std::isfinite(det) || std::fabs(det) < 1e-30) { set_error("rt_scene_create: singular instance transform"); return RT_INVALID_ARG; }
        }
    }
    if (d->num_materials <= 0 || !d->albedo || !d->roughness || !d->ggx_weight || !d->emission) {
        set_error("rt_scene_create: material arrays missing");
        return RT_INVALID_ARG;
    }
    const int64_t T = d->num_triangles, V = d->num_vertices;
    for (int64_t t = 0; t < T; ++t) {
        for (int k = 0; k < 3; ++k)
            if ((int64_t)d->indices[3 * t + k] >= V) { set_error("rt_scene_create: vertex index out of range"); return RT_INVALID_ARG; }
        if ((int32_t)d->tri_material[t] >= d->num_materials) { set_error("rt_scene_create: material index out of range"); return RT_INVALID_ARG; }
    }
    bool any_tex = false;
    if (d->emission_tex)
        for (int32_t m = 0; m < d->num_materials; ++m)
            if (d->emission_tex[m] >= 0) {
                any_tex = true;
                if (d->emission_tex[m] >= d->num_textures || !d->textures || !d->uvs) {
                    set_error("rt_scene_create: emission texture index out of range or uvs missing");
                    return RT_INVALID_ARG;
                }
            }
    if (d->env) {
        int32_t W = d->env_width, H = d->env_height;
        if (W < 2 || H < 1 || W != 2 * H || (W & (W - 1)) != 0) {
            set_error("rt_scene_create: environment must be W x H with W = 2H a power of two");
            return RT_INVALID_ARG;
        }
    }
    rt_scene *s = new rt_scene();
    s->host_only = host_only;
    auto fail = [&](rt_status st) { rt_scene_destroy(s); return st; };
    DevScene &D = s->dev, &Hs = s->host;
    s->num_triangles = T;
    s->num_materials = (uint32_t)d->num_materials;

    // ---- BVH: one level, or per-mesh bottom levels + a top level over instances
    rt_status st;
    std::vector<double> o2w, w2o;   // 12 doubles per instance
    AimTree aim;
    if (d->num_instances > 0) {
        const int32_t M = d->num_meshes, I = d->num_instances;
        std::vector<uint32_t> nodes_all;
        std::vector<float> tris_all;
        std::vector<uint32_t> mesh_root(M);
        std::vector<float> mlo(3 * M), mhi(3 * M);
        int depth = 0;
        for (int32_t m = 0; m < M; ++m) {
            int64_t t0 = d->mesh_tri_offset[m], t1 = d->mesh_tri_offset[m + 1];
            std::vector<uint32_t> ids((size_t)(t1 - t0));
            for (int64_t t = t0; t < t1; ++t) ids[(size_t)(t - t0)] = (uint32_t)t;
            Bvh8 b;
            build_bvh8(d->vertices, d->indices, ids.data(), t1 - t0, b);
            const uint32_t noff = (uint32_t)(nodes_all.size() / 20), toff = (uint32_t)(tris_all.size() / 12);
            for (size_t i = 0; i < b.nodes.size(); i += 20) {
                uint32_t nd[20];
                std::memcpy(nd, &b.nodes[i], sizeof nd);
                nd[4] += noff;
                nd[5] += toff;
                nodes_all.insert(nodes_all.end(), nd, nd + 20);
            }
            tris_all.insert(tris_all.end(), b.tris.begin(), b.tris.end());
            mesh_root[m] = noff;
            for (int a = 0; a < 3; ++a) { mlo[3 * m + a] = b.lo[a]; mhi[3 * m + a] = b.hi[a]; }
            depth = std::max(depth, b.depth);
        }
        o2w.resize(12 * (size_t)I);
        w2o.resize(12 * (size_t)I);
        std::vector<float> ilo(3 * (size_t)I), ihi(3 * (size_t)I);
        std::vector<uint32_t> iroot(I);
        float blo[3] = {INFINITY, INFINITY, INFINITY}, bhi[3] = {-INFINITY, -INFINITY, -INFINITY};
        for (int32_t k = 0; k < I; ++k) {
            const float *X = d->instance_xform + 12 * (size_t)k;
            double *A = &o2w[12 * (size_t)k], *B = &w2o[12 * (size_t)k];
            for (int i = 0; i < 12; ++i) A[i] = X[i];
            // inverse of the affine map [R | t]: [R^-1 | -R^-1 t]
            double r00 = A[0], r01 = A[1], r02 = A[2], r10 = A[4], r11 = A[5], r12 = A[6], r20 = A[8], r21 = A[9], r22 = A[10];
            double det = r00 * (r11 * r22 - r12 * r21) - r01 * (r10 * r22 - r12 * r20) + r02 * (r10 * r21 - r11 * r20);
            double inv[9] = {(r11 * r22 - r12 * r21) / det, (r02 * r21 - r01 * r22) / det, (r01 * r12 - r02 * r11) / det,
                             (r12 * r20 - r10 * r22) / det, (r00 * r22 - r02 * r20) / det, (r02 * r10 - r00 * r12) / det,
                             (r10 * r21 - r11 * r20) / det, (r01 * r20 - r00 * r21) / det, (r00 * r11 - r01 * r10) / det};
            for (int i = 0; i < 3; ++i) {
                for (int j = 0; j < 3; ++j) B[4 * i + j] = inv[3 * i + j];
                B[4 * i + 3] = -(inv[3 * i] * A[3] + inv[3 * i + 1] * A[7] + inv[3 * i + 2] * A[11]);
            }
            uint32_t m = d->instance_mesh[k];
            iroot[k] = mesh_root[m];
            double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
            for (int c = 0; c < 8; ++c) {
                double p[3] = {(c & 1) ? mhi[3 * m] : mlo[3 * m], (c & 2) ? mhi[3 * m + 1] : mlo[3 * m + 1],
                               (c & 4) ? mhi[3 * m + 2] : mlo[3 * m + 2]};
                for (int a = 0; a < 3; ++a) {
                    double w = A[4 * a] * p[0] + A[4 * a + 1] * p[1] + A[4 * a + 2] * p[2] + A[4 * a + 3];
                    lo[a] = std::min(lo[a], w);
                    hi[a] = std::max(hi[a], w);
                }
            }
            for (int a = 0; a < 3; ++a) {
                double pad = 1e-6 * (std::fabs(lo[a]) + std::fabs(hi[a]) + 1e-3);
                ilo[3 * (size_t)k + a] = std::nextafter((float)(lo[a] - pad), -INFINITY);
                ihi[3 * (size_t)k + a] = std::nextafter((float)(hi[a] + pad), INFINITY);
                blo[a] = std::min(blo[a], ilo[3 * (size_t)k + a]);
                bhi[a] = std::max(bhi[a], ihi[3 * (size_t)k + a]);
            }
        }
        Bvh8 tl;
        build_bvh8_boxes(ilo.data(), ihi.data(), I, tl);
        s->num_nodes = (int64_t)nodes_all.size() / 20 + tl.num_nodes();
        s->num_leaf_tris = (int64_t)tris_all.size() / 12;
        s->bvh_depth = depth + tl.depth;
        if ((st = upload(s, (const uint4 *)nodes_all.data(), nodes_all.size() / 4, &D.nodes, &Hs.nodes)) != RT_OK) return fail(st);
        if ((st = upload(s, (const float4 *)tris_all.data(), tris_all.size() / 4, &D.tris, &Hs.tris)) != RT_OK) return fail(st);
        if ((st = upload(s, (const uint4 *)tl.nodes.data(), tl.nodes.size() / 4, &D.tlas_nodes, &Hs.tlas_nodes)) != RT_OK) return fail(st);
        if ((st = upload(s, tl.tri_ids.data(), tl.tri_ids.size(), &D.tlas_inst, &Hs.tlas_inst)) != RT_OK) return fail(st);
        std::vector<float4> xf(6 * (size_t)I);
        for (int32_t k = 0; k < I; ++k)
            for (int r = 0; r < 3; ++r) {
                const double *B = &w2o[12 * (size_t)k + 4 * r], *A = &o2w[12 * (size_t)k + 4 * r];
                xf[6 * (size_t)k + r] = make_float4((float)B[0], (float)B[1], (float)B[2], (float)B[3]);
                xf[6 * (size_t)k + 3 + r] = make_float4((float)A[0], (float)A[1], (float)A[2], (float)A[3]);
            }
        if ((st = upload(s, xf.data(), xf.size(), &D.inst_xf, &Hs.inst_xf)) != RT_OK) return fail(st);
        if ((st = upload(s, iroot.data(), iroot.size(), &D.inst_root, &Hs.inst_root)) != RT_OK) return fail(st);
        D.two_level = Hs.two_level = 1;
        D.num_instances = Hs.num_instances = (uint32_t)I;
        // photon aiming: the instances are the objects
        std::vector<AimBox> objs(I);
        for (int32_t k = 0; k < I; ++k) {
            double lo3[3] = {ilo[3 * (size_t)k], ilo[3 * (size_t)k + 1], ilo[3 * (size_t)k + 2]};
            double hi3[3] = {ihi[3 * (size_t)k], ihi[3 * (size_t)k + 1], ihi[3 * (size_t)k + 2]};
            objs[k].add(lo3);
            objs[k].add(hi3);
        }
        aim_tree(objs, aim);
        D.bb_lo = Hs.bb_lo = make_float3(blo[0], blo[1], blo[2]);
        D.bb_hi = Hs.bb_hi = make_float3(bhi[0], bhi[1], bhi[2]);
    } else {
        Bvh8 bvh;
        build_bvh8(d->vertices, d->indices, nullptr, T, bvh);
        s->num_nodes = bvh.num_nodes();
        s->num_leaf_tris = bvh.num_tris();
        s->bvh_depth = bvh.depth;
        if ((st = upload(s, (const uint4 *)bvh.nodes.data(), bvh.nodes.size() / 4, &D.nodes, &Hs.nodes)) != RT_OK) return fail(st);
        if ((st = upload(s, (const float4 *)bvh.tris.data(), bvh.tris.size() / 4, &D.tris, &Hs.tris)) != RT_OK) return fail(st);
        D.bb_lo = Hs.bb_lo = make_float3(bvh.lo[0], bvh.lo[1], bvh.lo[2]);
        D.bb_hi = Hs.bb_hi = make_float3(bvh.hi[0], bvh.hi[1], bvh.hi[2]);
        // photon aiming: connected components of the mesh (shared vertex
        // indices) are the objects, numbered by their first triangle
        if (T > 0) {
            DisjointSets vs((size_t)V);
            for (int64_t t = 0; t < T; ++t) {
                const uint32_t *id = d->indices + 3 * (size_t)t;
                vs.join((int32_t)id[0], (int32_t)id[1]);
                vs.join((int32_t)id[0], (int32_t)id[2]);
            }
            std::vector<int32_t> obj_of(V, -1);
            std::vector<AimBox> objs;
            for (int64_t t = 0; t < T; ++t) {
                const int32_t r = vs.root((int32_t)d->indices[3 * (size_t)t]);
                if (obj_of[r] < 0) { obj_of[r] = (int32_t)objs.size(); objs.emplace_back(); }
                AimBox &b = objs[obj_of[r]];
                for (int k = 0; k < 3; ++k) {
                    const float *pv = d->vertices + 3 * (size_t)d->indices[3 * (size_t)t + k];
                    const double q[3] = {pv[0], pv[1], pv[2]};
                    b.add(q);
                }
            }
            aim_tree(objs, aim);
        }
    }
    if (!aim.node.empty()) {
        if ((st = upload(s, aim.node.data(), aim.node.size(), &D.pa_node, &Hs.pa_node)) != RT_OK) return fail(st);
        if ((st = upload(s, aim.link.data(), aim.link.size(), &D.pa_link, &Hs.pa_link)) != RT_OK) return fail(st);
        D.pa_nnodes = Hs.pa_nnodes = (int32_t)aim.node.size();
        D.pa_nclusters = Hs.pa_nclusters = aim.nclusters;
    }

    // ---- shading arrays
    if ((st = upload(s, d->vertices, (size_t)V * 3, &D.vertices, &Hs.vertices)) != RT_OK) return fail(st);
    if (d->normals && (st = upload(s, d->normals, (size_t)V * 3, &D.normals, &Hs.normals)) != RT_OK) return fail(st);
    if (d->uvs && (st = upload(s, d->uvs, (size_t)V * 2, &D.uvs, &Hs.uvs)) != RT_OK) return fail(st);
    if ((st = upload(s, d->indices, (size_t)T * 3, &D.indices, &Hs.indices)) != RT_OK) return fail(st);
    if ((st = upload(s, d->tri_material, (size_t)T, &D.tri_material, &Hs.tri_material)) != RT_OK) return fail(st);
    std::vector<float4> ma(d->num_materials), mb(d->num_materials);
    std::vector<int32_t> mt(d->num_materials, -1);
    for (int32_t m = 0; m < d->num_materials; ++m) {
        ma[m] = make_float4(d->albedo[3 * m], d->albedo[3 * m + 1], d->albedo[3 * m + 2], d->roughness[m]);
        mb[m] = make_float4(d->emission[3 * m], d->emission[3 * m + 1], d->emission[3 * m + 2], d->ggx_weight[m]);
        if (d->emission_tex) mt[m] = d->emission_tex[m];
    }
    if ((st = upload(s, ma.data(), ma.size(), &D.mat_a, &Hs.mat_a)) != RT_OK) return fail(st);
    if ((st = upload(s, mb.data(), mb.size(), &D.mat_b, &Hs.mat_b)) != RT_OK) return fail(st);
    if ((st = upload(s, mt.data(), mt.size(), &D.mat_tex, &Hs.mat_tex)) != RT_OK) return fail(st);
    if (any_tex) {
        D.tex_w = Hs.tex_w = d->tex_width;
        D.tex_h = Hs.tex_h = d->tex_height;
        if ((st = upload(s, d->textures, (size_t)d->num_textures * d->tex_width * d->tex_height * 3, &D.textures,
                         &Hs.textures)) != RT_OK)
            return fail(st);
    }

    // ---- environment pyramid: weights = luminance x exact texel solid angle
    double env_sum = 0.0;
    if (d->env) {
        const int32_t W = d->env_width, H = d->env_height;
        int levels = 0;
        for (int32_t w = W; w >= 2; w /= 2) ++levels;
        if (levels > 16) { set_error("environment too large"); return fail(RT_INVALID_ARG); }
        std::vector<std::vector<double>> lv(levels);
        lv[0].resize((size_t)W * H);
        for (int32_t y = 0; y < H; ++y) {
            double om = (2.0 * M_PI / W) * (std::cos(M_PI * y / H) - std::cos(M_PI * (y + 1) / H));
            for (int32_t x = 0; x < W; ++x) {
                double w = lum3(d->env + 3 * ((size_t)y * W + x)) * om;
                lv[0][(size_t)y * W + x] = w;
                env_sum += w;
            }
        }
        for (int l = 1; l < levels; ++l) {
            int32_t pw = W >> (l - 1), ph = std::max(1, H >> (l - 1));
            int32_t lw = W >> l, lh = std::max(1, H >> l);
            lv[l].assign((size_t)lw * lh, 0.0);
            for (int32_t y = 0; y < ph; ++y)
                for (int32_t x = 0; x < pw; ++x) lv[l][(size_t)(y / 2) * lw + x / 2] += lv[l - 1][(size_t)y * pw + x];
        }
        std::vector<float> pyr;
        std::vector<int64_t> off(levels);
        for (int l = 0; l < levels; ++l) {
            off[l] = (int64_t)pyr.size();
            for (double v : lv[l]) pyr.push_back((float)v);
        }
        std::vector<float4> env4((size_t)W * H);
        for (size_t i = 0; i < env4.size(); ++i) {
            const float *c = d->env + 3 * i;
            env4[i] = make_float4(c[0], c[1], c[2], env_sum > 0.0 ? (float)(lum3(c) / env_sum) : 0.f);
        }
        D.env_w = Hs.env_w = W;
        D.env_h = Hs.env_h = H;
        D.env_levels = Hs.env_levels = levels;
        for (int l = 0; l < levels; ++l) D.env_off_h[l] = Hs.env_off_h[l] = off[l];
        if ((st = upload(s, env4.data(), env4.size(), &D.env, &Hs.env)) != RT_OK) return fail(st);
        if ((st = upload(s, pyr.data(), pyr.size(), &D.env_pyr, &Hs.env_pyr)) != RT_OK) return fail(st);
        if ((st = upload(s, off.data(), off.size(), &D.env_off, &Hs.env_off)) != RT_OK) return fail(st);
        // descent blocks: per node of level l >= 1, its children quad and,
        // from level 2 on, its children's quads (weights as stored above)
        auto quad_of = [&](auto &&wt, int l, int32_t x, int32_t y) {
            return make_float4(wt(l, 2 * x, 2 * y), wt(l, 2 * x + 1, 2 * y), wt(l, 2 * x, 2 * y + 1),
                               wt(l, 2 * x + 1, 2 * y + 1));
        };
        auto blocks_of = [&](auto &&wt, int l, std::vector<float4> &out) {
            const int32_t wl = W >> l, hl = std::max(1, H >> l);
            for (int32_t y = 0; y < hl; ++y)
                for (int32_t x = 0; x < wl; ++x) {
                    out.push_back(quad_of(wt, l - 1, x, y));
                    if (l >= 2)
                        for (int k = 0; k < 4; ++k) out.push_back(quad_of(wt, l - 2, 2 * x + (k & 1), 2 * y + (k >> 1)));
                }
        };
        auto plain_w = [&](int l, int32_t x, int32_t y) { return pyr[off[l] + (int64_t)y * (W >> l) + x]; };
        std::vector<float4> dq;
        for (int l = 0; l < 16; ++l) D.env_dqoff_h[l] = Hs.env_dqoff_h[l] = -1;
        for (int l = 1; l < levels; ++l) {
            D.env_dqoff_h[l] = Hs.env_dqoff_h[l] = (int64_t)dq.size();
            blocks_of(plain_w, l, dq);
        }
        for (int l = 0; l < 16; ++l) D.env_ndqoff_h[l] = Hs.env_ndqoff_h[l] = -1;
        if (!dq.empty() && (st = upload(s, dq.data(), dq.size(), &D.env_dq, &Hs.env_dq)) != RT_OK) return fail(st);
        if (!d->env_plain && env_sum > 0.0) {
            EnvNormalTables nt;
            build_env_normal_tables(lv, W, H, levels, env_sum, nt);
            // per cell, the blocks of the levels whose children are reweighted
            std::vector<float4> ndq;
            int64_t stride = 0, noff[16];
            for (int l = 0; l < 16; ++l) noff[l] = -1;
            for (int c = 0; c < 64; ++c) {
                auto cell_w = [&](int l, int32_t x, int32_t y) {
                    return l >= nt.lstar ? nt.nw[(size_t)c * nt.stride + nt.off[l] + (int64_t)y * (W >> l) + x]
                                         : plain_w(l, x, y);
                };
                const size_t start = ndq.size();
                for (int l = levels - 1; l >= 1 && l - 1 >= nt.lstar; --l) {
                    if (c == 0) noff[l] = (int64_t)(ndq.size() - start);
                    blocks_of(cell_w, l, ndq);
                }
                if (c == 0) stride = (int64_t)(ndq.size() - start);
            }
            for (int l = 0; l < 16; ++l) D.env_ndqoff_h[l] = Hs.env_ndqoff_h[l] = noff[l];
            D.env_ndqstride = Hs.env_ndqstride = stride;
            if (!ndq.empty() && (st = upload(s, ndq.data(), ndq.size(), &D.env_ndq, &Hs.env_ndq)) != RT_OK)
                return fail(st);
            D.env_lstar = Hs.env_lstar = nt.lstar;
            D.env_nregions = Hs.env_nregions = nt.nregions;
            D.env_nstride = Hs.env_nstride = nt.stride;
            for (int l = 0; l < 16; ++l) D.env_noff_h[l] = Hs.env_noff_h[l] = nt.off[l];
            if ((st = upload(s, nt.nw.data(), nt.nw.size(), &D.env_nw, &Hs.env_nw)) != RT_OK) return fail(st);
            if ((st = upload(s, nt.scale.data(), nt.scale.size(), &D.env_nscale, &Hs.env_nscale)) != RT_OK) return fail(st);
            if ((st = upload(s, nt.fac.data(), nt.fac.size(), &D.env_nfac, &Hs.env_nfac)) != RT_OK) return fail(st);
        }
    }

    // ---- emitters: mean luminance per triangle; one emitter per emissive
    // (instance, triangle) with its world-space vertices, flux = mean
    // luminance x world area, alias table over the fluxes; the solid-angle
    // pdf of a hit emitter needs only (1 - p_env) * mean luminance / sum(flux)
    std::vector<double> lum_avg((size_t)std::max<int64_t>(T, 1), 0.0);
    for (int64_t t = 0; t < T; ++t) {
        uint32_t m = d->tri_material[t];
        double L = lum3(d->emission + 3 * m);
        if (!(L > 0.0)) continue;
        int32_t tex = d->emission_tex ? d->emission_tex[m] : -1;
        if (tex >= 0) L *= textured_mean(d, t, tex);
        lum_avg[t] = L > 0.0 ? L : 0.0;
    }
    std::vector<double> flux;
    std::vector<uint32_t> light_tri, light_inst;
    std::vector<float4> light_v;
    auto add_light = [&](uint32_t inst, int64_t t, const double *X /* o2w or null */) {
        double p[3][3];
        for (int k = 0; k < 3; ++k) {
            const float *v = d->vertices + 3 * (size_t)d->indices[3 * t + k];
            for (int a = 0; a < 3; ++a)
                p[k][a] = X ? X[4 * a] * v[0] + X[4 * a + 1] * v[1] + X[4 * a + 2] * v[2] + X[4 * a + 3] : (double)v[a];
        }
        float pf[3][3];
        for (int k = 0; k < 3; ++k)
            for (int a = 0; a < 3; ++a) pf[k][a] = (float)p[k][a];
        double e1[3] = {(double)pf[1][0] - pf[0][0], (double)pf[1][1] - pf[0][1], (double)pf[1][2] - pf[0][2]};
        double e2[3] = {(double)pf[2][0] - pf[0][0], (double)pf[2][1] - pf[0][1], (double)pf[2][2] - pf[0][2]};
        double c[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
        double area = 0.5 * std::sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
        if (!(area > 0.0)) return;
        flux.push_back(lum_avg[t] * area);
        light_tri.push_back((uint32_t)t);
        light_inst.push_back(inst);
        for (int k = 0; k < 3; ++k) light_v.push_back(make_float4(pf[k][0], pf[k][1], pf[k][2], 0.f));
    };
    if (d->num_instances > 0) {
        for (int32_t k = 0; k < d->num_instances; ++k) {
            uint32_t m = d->instance_mesh[k];
            for (int64_t t = d->mesh_tri_offset[m]; t < d->mesh_tri_offset[m + 1]; ++t)
                if (lum_avg[t] > 0.0) add_light((uint32_t)k, t, &o2w[12 * (size_t)k]);
        }
    } else {
        for (int64_t t = 0; t < T; ++t)
            if (lum_avg[t] > 0.0) add_light(0u, t, nullptr);
    }
    double flux_sum = 0.0;
    for (double f : flux) flux_sum += f;
    const bool has_env = d->env && env_sum > 0.0;
    const float p_env = has_env ? (flux.empty() ? 1.f : 0.5f) : 0.f;
    D.p_env = Hs.p_env = p_env;
    std::vector<float> lpa((size_t)std::max<int64_t>(T, 1), 0.f);
    if (!flux.empty())
        for (int64_t t = 0; t < T; ++t)
            if (lum_avg[t] > 0.0) lpa[t] = (float)((1.0 - p_env) * lum_avg[t] / flux_sum);
    if ((st = upload(s, lpa.data(), (size_t)T, &D.tri_light_pdf_area, &Hs.tri_light_pdf_area)) != RT_OK) return fail(st);
    if (!flux.empty()) {
        std::vector<float2> alias;
        build_alias(flux, alias);
        D.num_lights = Hs.num_lights = (uint32_t)flux.size();
        if ((st = upload(s, alias.data(), alias.size(), &D.alias, &Hs.alias)) != RT_OK) return fail(st);
        if ((st = upload(s, light_tri.data(), light_tri.size(), &D.light_tri, &Hs.light_tri)) != RT_OK) return fail(st);
        if ((st = upload(s, light_inst.data(), light_inst.size(), &D.light_inst, &Hs.light_inst)) != RT_OK) return fail(st);
        if ((st = upload(s, light_v.data(), light_v.size(), &D.light_v, &Hs.light_v)) != RT_OK) return fail(st);
        if (d->light_bvh) {
            // emitter of a hit (instance, triangle): the instance's first
            // emitter plus the triangle's rank among its mesh's emitters
            const int32_t I = std::max<int32_t>(1, d->num_instances);
            std::vector<uint32_t> base(I, 0u), rank((size_t)std::max<int64_t>(T, 1), 0xffffffffu);
            std::vector<uint8_t> seen(I, 0);
            for (size_t e = 0; e < flux.size(); ++e) {
                const uint32_t k = light_inst[e];
                if (!seen[k]) { seen[k] = 1; base[k] = (uint32_t)e; }
                const uint32_t r = (uint32_t)e - base[k];
                uint32_t &slot = rank[light_tri[e]];
                if (slot != 0xffffffffu && slot != r) {
                    set_error("rt_scene_create: light_bvh needs every instance to keep all of its mesh's emitters "
                              "(an instance transform made one degenerate)");
                    return fail(RT_INVALID_ARG);
                }
                slot = r;
            }
            LightBvh lb;
            build_light_bvh(light_v, flux, lb);
            std::vector<float4> rec;
            std::vector<uint32_t> up;
            light_bvh_records(lb, rec, up);
            if ((st = upload(s, rec.data(), rec.size(), &D.lb_rec, &Hs.lb_rec)) != RT_OK) return fail(st);
            if ((st = upload(s, lb.perm.data(), lb.perm.size(), &D.lb_perm, &Hs.lb_perm)) != RT_OK) return fail(st);
            if ((st = upload(s, up.data(), up.size(), &D.lb_up, &Hs.lb_up)) != RT_OK) return fail(st);
            std::vector<float> ef(flux.begin(), flux.end());
            if ((st = upload(s, ef.data(), ef.size(), &D.lb_eflux, &Hs.lb_eflux)) != RT_OK) return fail(st);
            if ((st = upload(s, rank.data(), rank.size(), &D.lb_tri_rank, &Hs.lb_tri_rank)) != RT_OK) return fail(st);
            if ((st = upload(s, base.data(), base.size(), &D.lb_inst_base, &Hs.lb_inst_base)) != RT_OK) return fail(st);
        }
    }
    *out = s;
    return RT_OK;
}

extern "C" rt_status rt_scene_destroy(rt_scene *s) {
    if (!s) return RT_OK;
    for (void *p : s->dev_allocs) cudaFree(p);
    delete s;
    return RT_OK;
}

extern "C" rt_status rt_scene_info(const rt_scene *s, int64_t *nodes, int64_t *leaf_tris, int64_t *bytes) {
    if (!s) { set_error("rt_scene_info: null scene"); return RT_INVALID_ARG; }
    if (nodes) *nodes = s->num_nodes;
    if (leaf_tris) *leaf_tris = s->num_leaf_tris;
    if (bytes) *bytes = s->device_bytes;
    return RT_OK;
}
