// Static-geometry hierarchy of the hybrid static/dynamic pipeline (Sec. 7):
// a binary bounding-volume hierarchy over the static triangles, built once
// on the host with binned surface-area-heuristic splits (the top levels in
// parallel threads), laid out for the GPU traversal kernel: every node holds
// the boxes of both children.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <future>
#include <limits>
#include <vector>

#include "grca_internal.h"

namespace grca {

namespace {

struct Box {
    float lo[3], hi[3];
    void reset() {
        for (int k = 0; k < 3; ++k) {
            lo[k] = std::numeric_limits<float>::infinity();
            hi[k] = -std::numeric_limits<float>::infinity();
        }
    }
    void grow(const Box& b) {
        for (int k = 0; k < 3; ++k) {
            lo[k] = std::min(lo[k], b.lo[k]);
            hi[k] = std::max(hi[k], b.hi[k]);
        }
    }
    void grow(const float* p) {
        for (int k = 0; k < 3; ++k) {
            lo[k] = std::min(lo[k], p[k]);
            hi[k] = std::max(hi[k], p[k]);
        }
    }
    double area() const {
        double dx = (double)hi[0] - lo[0], dy = (double)hi[1] - lo[1], dz = (double)hi[2] - lo[2];
        if (!(dx >= 0.0) || !(dy >= 0.0) || !(dz >= 0.0)) return 0.0;
        return 2.0 * (dx * dy + dy * dz + dz * dx);
    }
};

constexpr int BINS = 32;
constexpr uint32_t LEAF_TARGET = 2;     // SAH may stop at or below this many triangles
constexpr int MEDIAN_DEPTH = 40;        // beyond this depth, split at the median
constexpr uint32_t PAR_MIN = 1u << 18;  // subtrees at least this large build in their own thread
constexpr int PAR_DEPTH = 4;            // ... down to this depth (up to 16 threads)

struct Shared {
    std::vector<Box> pbox;
    std::vector<float> cen;  // 3 x (sum of the three vertices)
    std::vector<uint32_t> idx;
};

void set_node(BvhNode& nd, const Box& lb, int32_t l, const Box& rb, int32_t r) {
    nd.c0lo_x = lb.lo[0], nd.c0lo_y = lb.lo[1], nd.c0lo_z = lb.lo[2];
    nd.c0hi_x = lb.hi[0], nd.c0hi_y = lb.hi[1], nd.c0hi_z = lb.hi[2];
    nd.c1lo_x = rb.lo[0], nd.c1lo_y = rb.lo[1], nd.c1lo_z = rb.lo[2];
    nd.c1hi_x = rb.hi[0], nd.c1hi_y = rb.hi[1], nd.c1hi_z = rb.hi[2];
    nd.child0 = l;
    nd.child1 = r;
    nd.pad0 = nd.pad1 = 0;
}

// Split decision for idx[b, e): returns the split position m (b < m < e), or
// e when the range becomes a leaf.  bb receives the range's box.
uint32_t split(Shared& S, uint32_t b, uint32_t e, int depth, Box& bb) {
    Box cb;
    bb.reset();
    cb.reset();
    for (uint32_t i = b; i < e; ++i) {
        bb.grow(S.pbox[S.idx[i]]);
        cb.grow(&S.cen[3 * (size_t)S.idx[i]]);
    }
    const uint32_t n = e - b;
    if (n <= LEAF_TARGET) return e;
    int best_axis = -1, best_split = -1;
    double best_cost = std::numeric_limits<double>::infinity();
    if (depth < MEDIAN_DEPTH) {
        for (int ax = 0; ax < 3; ++ax) {
            const float c0 = cb.lo[ax], c1 = cb.hi[ax];
            if (!(c1 > c0)) continue;
            const double scale = BINS / ((double)c1 - c0);
            Box binb[BINS];
            uint32_t binn[BINS] = {};
            for (int k = 0; k < BINS; ++k) binb[k].reset();
            for (uint32_t i = b; i < e; ++i) {
                const uint32_t p = S.idx[i];
                int k = (int)(((double)S.cen[3 * (size_t)p + ax] - c0) * scale);
                k = std::min(std::max(k, 0), BINS - 1);
                binb[k].grow(S.pbox[p]);
                binn[k]++;
            }
            double rarea[BINS];
            uint32_t rcount[BINS];
            Box acc;
            acc.reset();
            uint32_t cnt = 0;
            for (int k = BINS - 1; k > 0; --k) {
                acc.grow(binb[k]);
                cnt += binn[k];
                rarea[k] = acc.area();
                rcount[k] = cnt;
            }
            acc.reset();
            cnt = 0;
            for (int k = 0; k < BINS - 1; ++k) {
                acc.grow(binb[k]);
                cnt += binn[k];
                if (cnt == 0 || rcount[k + 1] == 0) continue;
                const double cost = acc.area() * cnt + rarea[k + 1] * rcount[k + 1];
                if (cost < best_cost) {
                    best_cost = cost;
                    best_axis = ax;
                    best_split = k;
                }
            }
        }
    }
    if (best_axis >= 0) {
        // SAH: a leaf costs n tests; a split about one node visit plus its children
        const double split_cost = 1.0 + best_cost / std::max(bb.area(), 1e-30);
        if (n <= BVH_LEAF_MAX && (double)n <= split_cost) return e;
        const int ax = best_axis;
        const float c0 = cb.lo[ax];
        const double scale = BINS / ((double)cb.hi[ax] - c0);
        auto mid = std::partition(S.idx.begin() + b, S.idx.begin() + e, [&](uint32_t p) {
            int k = (int)(((double)S.cen[3 * (size_t)p + ax] - c0) * scale);
            k = std::min(std::max(k, 0), BINS - 1);
            return k <= best_split;
        });
        uint32_t m = (uint32_t)(mid - S.idx.begin());
        if (m > b && m < e) return m;
    }
    // coincident centroids or deep tree: median split on the widest centroid axis
    int ax = 0;
    float w = -1.f;
    for (int k = 0; k < 3; ++k)
        if (cb.hi[k] - cb.lo[k] > w) {
            w = cb.hi[k] - cb.lo[k];
            ax = k;
        }
    const uint32_t m = b + n / 2;
    std::nth_element(S.idx.begin() + b, S.idx.begin() + m, S.idx.begin() + e,
                     [&](uint32_t p, uint32_t q) { return S.cen[3 * (size_t)p + ax] < S.cen[3 * (size_t)q + ax]; });
    return m;
}

// Builds the subtree over idx[b, e) into `nodes` (inner references relative
// to the start of `nodes`); returns its reference and box.  Ranges that are
// large enough near the top build their left half in another thread.
int32_t build(Shared& S, std::vector<BvhNode>& nodes, uint32_t b, uint32_t e, int depth, Box& out) {
    const uint32_t m = split(S, b, e, depth, out);
    if (m == e) {
        if (e - b <= BVH_LEAF_MAX) return bvh_leaf_ref(b, e - b);
    }
    const size_t me = nodes.size();
    nodes.emplace_back();
    Box lb, rb;
    int32_t l, r;
    if (depth < PAR_DEPTH && e - b >= PAR_MIN) {
        std::vector<BvhNode> left;
        auto fut = std::async(std::launch::async, [&]() { return build(S, left, b, m, depth + 1, lb); });
        std::vector<BvhNode> right;
        r = build(S, right, m, e, depth + 1, rb);
        l = fut.get();
        // splice: left subtree, then right subtree, with relocated inner references
        const int32_t offl = (int32_t)nodes.size();
        for (BvhNode& x : left) {
            if (x.child0 >= 0) x.child0 += offl;
            if (x.child1 >= 0) x.child1 += offl;
        }
        nodes.insert(nodes.end(), left.begin(), left.end());
        const int32_t offr = (int32_t)nodes.size();
        for (BvhNode& x : right) {
            if (x.child0 >= 0) x.child0 += offr;
            if (x.child1 >= 0) x.child1 += offr;
        }
        nodes.insert(nodes.end(), right.begin(), right.end());
        if (l >= 0) l += offl;
        if (r >= 0) r += offr;
    } else {
        l = build(S, nodes, b, m, depth + 1, lb);
        r = build(S, nodes, m, e, depth + 1, rb);
    }
    set_node(nodes[me], lb, l, rb, r);
    return (int32_t)me;
}

inline float down(double x) {
    float f = (float)x;
    return (double)f > x ? std::nextafter(f, -std::numeric_limits<float>::infinity()) : f;
}
inline float up(double x) {
    float f = (float)x;
    return (double)f < x ? std::nextafter(f, std::numeric_limits<float>::infinity()) : f;
}

}  // namespace

bool build_bvh(const float* tris, uint32_t n, BvhHost& out) {
    out = BvhHost();
    if (n == 0) return true;
    if (n >= (1u << 28)) return false;  // leaf references hold 28-bit offsets
    Shared S;
    S.pbox.resize(n);
    S.cen.resize(3 * (size_t)n);
    S.idx.resize(n);
    Box scene;
    scene.reset();
    for (uint32_t i = 0; i < n; ++i) {
        const float* t = tris + 9 * (size_t)i;
        Box b;
        b.reset();
        b.grow(t);
        b.grow(t + 3);
        b.grow(t + 6);
        bool finite = true;
        for (int k = 0; k < 9; ++k) finite = finite && std::isfinite(t[k]);
        if (!finite) b.reset();  // a non-finite triangle never hits: an empty box
        S.pbox[i] = b;
        for (int k = 0; k < 3; ++k) S.cen[3 * (size_t)i + k] = finite ? t[k] + t[3 + k] + t[6 + k] : 0.f;
        S.idx[i] = i;
        if (finite) scene.grow(b);
    }
    std::vector<BvhNode> nodes;
    nodes.reserve(2 * (size_t)n / LEAF_TARGET + 2);
    Box all;
    const int32_t root = build(S, nodes, 0, n, 0, all);
    if (root < 0) {
        // the whole set is one leaf: a root whose two children are that leaf
        // (an inverted "empty" box would pass the slab test, so none is used)
        nodes.assign(1, BvhNode());
        set_node(nodes[0], all, root, all, root);
    }
    out.nodes.swap(nodes);
    out.prim.swap(S.idx);
    // outward inflation of every box by delta (see BvhHost)
    double diag2 = 0.0;
    for (int k = 0; k < 3; ++k) {
        const double ext = std::isfinite(scene.lo[k]) ? (double)scene.hi[k] - scene.lo[k] : 0.0;
        diag2 += ext * ext;
    }
    for (int k = 0; k < 3; ++k) {
        out.scene_lo[k] = scene.lo[k];
        out.scene_hi[k] = scene.hi[k];
    }
    // plus 2^-21 of the largest coordinate: the FP32 slab distances are formed
    // as x / d - o / d, whose rounding is a few ulps of the coordinates
    double cmax = 0.0;
    for (int k = 0; k < 3; ++k)
        if (std::isfinite(scene.lo[k]))
            cmax = std::max(cmax, std::max(std::fabs((double)scene.lo[k]), std::fabs((double)scene.hi[k])));
    out.delta = BVH_ETA * (std::sqrt(diag2) + 1.0) + cmax * 0x1p-21;
    const double d = out.delta;
    for (BvhNode& nd : out.nodes) {
        float* f = reinterpret_cast<float*>(&nd);
        // child 0: lo 0-2, hi 3-5; child 1: lo 6-8, hi 9-11
        for (int c = 0; c < 2; ++c)
            for (int k = 0; k < 3; ++k) {
                float& lo = f[6 * c + k];
                float& hi = f[6 * c + 3 + k];
                if (!(lo <= hi)) continue;  // an empty box stays empty
                lo = down((double)lo - d);
                hi = up((double)hi + d);
            }
    }
    // depth (the traversal keeps at most depth - 1 deferred children)
    int depth = 0;
    std::vector<std::pair<int32_t, int>> st{{0, 1}};
    while (!st.empty()) {
        auto [nd, dp] = st.back();
        st.pop_back();
        depth = std::max(depth, dp);
        const BvhNode& x = out.nodes[nd];
        if (x.child0 >= 0) st.push_back({x.child0, dp + 1});
        if (x.child1 >= 0) st.push_back({x.child1, dp + 1});
    }
    out.depth = depth;
    return depth < BVH_STACK;
}

}  // namespace grca
