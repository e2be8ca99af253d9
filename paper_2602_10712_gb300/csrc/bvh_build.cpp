// bvh_build.cpp -- host construction of the wide BVH used by the tracer.
//
// The paper intersects every ray with every triangle (Sec. 3.2,
// "Estimation") because each of its samples has a new design; for the fixed
// designs traced here with millions of parallel rays per sun direction the
// prior BVH ray-grid approach (Sec. 2.1) applies, and the build cost is
// amortised over all rays and directions of a design.
//
// Build: binary BVH by binned surface-area heuristic (16 bins per axis over
// centroid bounds, split down to one triangle per leaf), then collapsed
// top-down into 4- or 8-wide nodes by repeatedly opening the child of
// largest surface area.  Node bounds are padded outward by a small relative
// epsilon so the
// FP32 slab test in the kernel never rejects a box whose triangle the
// watertight triangle test would hit.
#include <vector_types.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <limits>

#include "srp_internal.h"

namespace srp {
namespace {

struct AABB {
    float lo[3], hi[3];
    void reset() {
        for (int j = 0; j < 3; ++j) { lo[j] = std::numeric_limits<float>::infinity(); hi[j] = -lo[j]; }
    }
    void grow(const AABB& b) {
        for (int j = 0; j < 3; ++j) { lo[j] = std::min(lo[j], b.lo[j]); hi[j] = std::max(hi[j], b.hi[j]); }
    }
    void grow(const float* p) {
        for (int j = 0; j < 3; ++j) { lo[j] = std::min(lo[j], p[j]); hi[j] = std::max(hi[j], p[j]); }
    }
    double area() const {
        double dx = hi[0] - lo[0], dy = hi[1] - lo[1], dz = hi[2] - lo[2];
        if (!(dx >= 0) || !(dy >= 0) || !(dz >= 0)) return 0.0;
        return 2.0 * (dx * dy + dy * dz + dz * dx);
    }
};

struct BNode {       // binary node
    AABB box;
    int left = -1, right = -1;   // children (inner)
    int first = 0, count = 0;    // leaf range in the permutation
};

constexpr int kBins = 16;
// One triangle per leaf: a lane's leaf work is then one triangle test, and
// the wide node tests (four boxes at once) do the sorting.  Measured on the
// 49,776-triangle satellite, 512 suns x 2048^2 rays: leaves of <= 4, 2 and 1
// triangles give 7.40, 8.70 and 8.77 G rays/s at K <= 3 (22.4, 23.9, 24.1 at
// K = 1); the closest hit does not depend on the tree.
constexpr int kMaxLeaf = 1;

struct Builder {
    const std::vector<AABB>& pb;
    const std::vector<float>& cen;  // [T][3]
    std::vector<int32_t>& idx;
    std::vector<BNode> nodes;

    Builder(const std::vector<AABB>& pb_, const std::vector<float>& cen_, std::vector<int32_t>& idx_)
        : pb(pb_), cen(cen_), idx(idx_) {}

    int make_leaf(int b, int e, const AABB& box) {
        BNode n; n.box = box; n.first = b; n.count = e - b;
        nodes.push_back(n);
        return (int)nodes.size() - 1;
    }

    // Iterative build (explicit stack) over idx[b, e).
    int build(int T) {
        struct Job { int b, e, parent, side; };
        std::vector<Job> st;
        st.push_back({0, T, -1, 0});
        int root = -1;
        while (!st.empty()) {
            Job j = st.back(); st.pop_back();
            AABB box, cb; box.reset(); cb.reset();
            for (int i = j.b; i < j.e; ++i) { box.grow(pb[idx[i]]); cb.grow(&cen[3 * idx[i]]); }
            int n = j.e - j.b;
            int me;
            int split = -1;
            if (n > kMaxLeaf) {
                // binned SAH
                double best = std::numeric_limits<double>::infinity();
                int bax = -1, bbin = -1;
                for (int ax = 0; ax < 3; ++ax) {
                    float ext = cb.hi[ax] - cb.lo[ax];
                    if (!(ext > 0.0f)) continue;
                    AABB bb[kBins]; int bc[kBins];
                    for (int k = 0; k < kBins; ++k) { bb[k].reset(); bc[k] = 0; }
                    float sc = kBins / ext;
                    for (int i = j.b; i < j.e; ++i) {
                        int k = (int)((cen[3 * idx[i] + ax] - cb.lo[ax]) * sc);
                        k = std::min(std::max(k, 0), kBins - 1);
                        bb[k].grow(pb[idx[i]]); bc[k]++;
                    }
                    double la[kBins]; int lc[kBins];
                    AABB acc; acc.reset(); int c = 0;
                    for (int k = 0; k < kBins - 1; ++k) {
                        acc.grow(bb[k]); c += bc[k]; la[k] = acc.area(); lc[k] = c;
                    }
                    acc.reset(); c = 0;
                    for (int k = kBins - 1; k > 0; --k) {
                        acc.grow(bb[k]); c += bc[k];
                        double cost = la[k - 1] * lc[k - 1] + acc.area() * c;
                        if (lc[k - 1] > 0 && c > 0 && cost < best) { best = cost; bax = ax; bbin = k; }
                    }
                }
                if (bax >= 0) {
                    float ext = cb.hi[bax] - cb.lo[bax];
                    float sc = kBins / ext;
                    auto mid = std::partition(idx.begin() + j.b, idx.begin() + j.e, [&](int32_t t) {
                        int k = (int)((cen[3 * t + bax] - cb.lo[bax]) * sc);
                        k = std::min(std::max(k, 0), kBins - 1);
                        return k < bbin;
                    });
                    split = (int)(mid - idx.begin());
                }
                if (split <= j.b || split >= j.e) split = j.b + n / 2;  // degenerate: median by index
            }
            if (split < 0) {
                me = make_leaf(j.b, j.e, box);
            } else {
                BNode nd; nd.box = box; nd.count = 0;
                nodes.push_back(nd);
                me = (int)nodes.size() - 1;
                st.push_back({split, j.e, me, 1});
                st.push_back({j.b, split, me, 0});
            }
            if (j.parent < 0) root = me;
            else if (j.side == 0) nodes[j.parent].left = me;
            else nodes[j.parent].right = me;
        }
        return root;
    }
};

}  // namespace

int build_wide_bvh(const float* verts, int V, const int32_t* tris, int T, int width,
                   BuiltBVH* out, std::string* err) {
    if (width != 4 && width != 8) { *err = "width must be 4 or 8"; return SRP_EINVAL; }
    out->width = width;
    std::vector<AABB> pb(std::max(T, 0));
    std::vector<float> cen(3 * (size_t)std::max(T, 0));
    AABB scene; scene.reset();
    for (int t = 0; t < T; ++t) {
        pb[t].reset();
        for (int c = 0; c < 3; ++c) {
            int v = tris[3 * t + c];
            if (v < 0 || v >= V) { *err = "triangle vertex index out of range"; return SRP_EINVAL; }
            const float* p = verts + 3 * (size_t)v;
            for (int j = 0; j < 3; ++j)
                if (!std::isfinite(p[j])) { *err = "non-finite vertex coordinate"; return SRP_EINVAL; }
            pb[t].grow(p);
        }
        for (int j = 0; j < 3; ++j) cen[3 * t + j] = 0.5f * (pb[t].lo[j] + pb[t].hi[j]);
        scene.grow(pb[t]);
    }
    float scale = 0.0f;
    for (int j = 0; j < 3; ++j)
        if (T > 0) scale = std::max(scale, std::max(std::fabs(scene.lo[j]), std::fabs(scene.hi[j])));
    const float pad_abs = 1e-6f * (scale + 1e-3f);

    out->tri_order.resize(std::max(T, 0));
    for (int t = 0; t < T; ++t) out->tri_order[t] = t;

    const int W = width;
    const int node_floats = W == 4 ? 32 : 64;  // 128 B or 256 B
    std::vector<float>& nd = out->node_data;
    nd.clear();
    auto new_node = [&]() {
        size_t base = nd.size();
        nd.resize(base + node_floats, 0.0f);
        float inf = std::numeric_limits<float>::infinity();
        for (int c = 0; c < W; ++c) {
            for (int a = 0; a < 3; ++a) { nd[base + (2 * a) * W + c] = inf; nd[base + (2 * a + 1) * W + c] = -inf; }
        }
        return (int)(base / node_floats);
    };
    auto set_child = [&](int node, int c, const AABB& b, int32_t code) {
        size_t base = (size_t)node * node_floats;
        for (int a = 0; a < 3; ++a) {
            float lo = b.lo[a], hi = b.hi[a];
            nd[base + (2 * a) * W + c] = lo - (std::fabs(lo) * 4e-7f + pad_abs);
            nd[base + (2 * a + 1) * W + c] = hi + (std::fabs(hi) * 4e-7f + pad_abs);
        }
        int32_t* ch = reinterpret_cast<int32_t*>(&nd[base + 6 * W]);
        ch[c] = code;
    };

    out->n_leaves = 0; out->depth = 0;
    out->level_start = {0, 1};
    int root_w = new_node();
    (void)root_w;
    if (T == 0) { out->n_nodes = 1; out->depth = 1; return SRP_OK; }

    Builder b(pb, cen, out->tri_order);
    b.nodes.reserve(2 * (size_t)T / kMaxLeaf + 8);
    int broot = b.build(T);

    auto leaf_code = [&](const BNode& n) -> int32_t {
        return ~((n.first << 3) | (n.count - 1));
    };
    // collapse: work list of (wide node index, binary node index, depth)
    struct Item { int w, bn, depth; };
    std::vector<Item> work;
    if (b.nodes[broot].count > 0) {
        set_child(0, 0, b.nodes[broot].box, leaf_code(b.nodes[broot]));
        out->n_leaves = 1; out->n_nodes = 1; out->depth = 1;
        return SRP_OK;
    }
    work.push_back({0, broot, 1});
    size_t head = 0;
    while (head < work.size()) {
        Item it = work[head++];
        out->depth = std::max(out->depth, it.depth);
        std::vector<int> kids = {b.nodes[it.bn].left, b.nodes[it.bn].right};
        while ((int)kids.size() < W) {
            int best = -1; double ba = -1.0;
            for (int k = 0; k < (int)kids.size(); ++k) {
                const BNode& n = b.nodes[kids[k]];
                if (n.count > 0) continue;
                double a = n.box.area();
                if (a > ba) { ba = a; best = k; }
            }
            if (best < 0) break;
            int open = kids[best];
            kids[best] = b.nodes[open].left;
            kids.push_back(b.nodes[open].right);
        }
        for (int c = 0; c < (int)kids.size(); ++c) {
            const BNode& n = b.nodes[kids[c]];
            if (n.count > 0) {
                set_child(it.w, c, n.box, leaf_code(n));
                out->n_leaves++;
            } else {
                int wn = new_node();
                set_child(it.w, c, n.box, wn);
                work.push_back({wn, kids[c], it.depth + 1});
            }
        }
    }
    out->n_nodes = (int)(nd.size() / node_floats);
    // work[i] describes wide node i (nodes are created in work-list order),
    // and the list is breadth first: depths never decrease along it
    out->level_start.clear();
    for (int i = 0; i < (int)work.size(); ++i)
        if (i == 0 || work[i].depth != work[i - 1].depth) out->level_start.push_back(i);
    out->level_start.push_back(out->n_nodes);
    return SRP_OK;
}

}  // namespace srp
