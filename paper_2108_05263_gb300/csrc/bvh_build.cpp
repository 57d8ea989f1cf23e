// Host BVH construction: a surface-area-heuristic binary BVH with spatial
// splits (triangles marked fixed are never split) collapsed into 4-wide
// nodes whose children boxes are
// stored as SoA float4 rows, with each slot's entry code (bvh.h)
// precomputed, so that one node is six box rows and one entry row of 16
// bytes on the device.
#include <algorithm>
#include <array>
#include <cfloat>
#include <cmath>
#include <cstring>
#include <vector>

#include "bvh.h"

namespace {

struct Box {
    float lo[3] = {FLT_MAX, FLT_MAX, FLT_MAX};
    float hi[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
    void grow(const float* p) {
        for (int a = 0; a < 3; ++a) {
            lo[a] = std::min(lo[a], p[a]);
            hi[a] = std::max(hi[a], p[a]);
        }
    }
    void grow(const Box& b) {
        for (int a = 0; a < 3; ++a) {
            lo[a] = std::min(lo[a], b.lo[a]);
            hi[a] = std::max(hi[a], b.hi[a]);
        }
    }
    float area() const {
        float d[3];
        for (int a = 0; a < 3; ++a) d[a] = std::max(hi[a] - lo[a], 0.f);
        return 2.f * (d[0] * d[1] + d[1] * d[2] + d[2] * d[0]);
    }
    bool valid() const { return lo[0] <= hi[0]; }
};

struct BNode {
    Box box;
    int left = -1, right = -1;   // children (binary), -1 for leaves
    int first = 0, count = 0;    // leaf range in the index array
};

constexpr int kBins = 128;
constexpr int kMaxLeaf = 4;

// Sutherland-Hodgman clip of a convex polygon against one axis-aligned
// half-space (keep side <= c when `below`, else >= c)
int clip_poly(const float (*in)[3], int n, int axis, float c, bool below, float (*out)[3]) {
    int m = 0;
    for (int i = 0; i < n; ++i) {
        const float* p = in[i];
        const float* q = in[(i + 1) % n];
        const float dp = below ? c - p[axis] : p[axis] - c;
        const float dq = below ? c - q[axis] : q[axis] - c;
        if (dp >= 0.f) {
            for (int a = 0; a < 3; ++a) out[m][a] = p[a];
            ++m;
        }
        if ((dp >= 0.f) != (dq >= 0.f)) {
            const float s = dp / (dp - dq);
            for (int a = 0; a < 3; ++a) out[m][a] = p[a] + s * (q[a] - p[a]);
            out[m][axis] = c;
            ++m;
        }
    }
    return m;
}

struct Ref {
    int tri;
    Box box;
};

// the box of the part of triangle `tri` inside `clip` (invalid if none)
Box clip_tri_box(const float* verts, int tri, const Box& clip) {
    float poly[16][3], tmp[16][3];
    const float* v = verts + 9 * (size_t)tri;
    for (int k = 0; k < 3; ++k)
        for (int a = 0; a < 3; ++a) poly[k][a] = v[3 * k + a];
    int n = 3;
    for (int a = 0; a < 3 && n >= 3; ++a)
        for (int side = 0; side < 2 && n >= 3; ++side) {
            n = clip_poly(poly, n, a, side == 0 ? clip.lo[a] : clip.hi[a], side == 1, tmp);
            for (int i = 0; i < n; ++i)
                for (int c = 0; c < 3; ++c) poly[i][c] = tmp[i][c];
        }
    Box b;
    if (n < 3) return b;
    for (int i = 0; i < n; ++i) b.grow(poly[i]);
    for (int a = 0; a < 3; ++a) {   // stay inside the clip box
        b.lo[a] = std::max(b.lo[a], clip.lo[a]);
        b.hi[a] = std::min(b.hi[a], clip.hi[a]);
    }
    return b;
}

float overlap_area(const Box& a, const Box& b) {
    Box o;
    for (int k = 0; k < 3; ++k) {
        o.lo[k] = std::max(a.lo[k], b.lo[k]);
        o.hi[k] = std::min(a.hi[k], b.hi[k]);
        if (o.lo[k] > o.hi[k]) return 0.f;
    }
    return o.area();
}

// Spatial-split SAH build (Stich, Friedrich and Dietrich 2009): at each node
// the binned object split over the references' box centres is compared with
// the best of kSpatialBins spatial splits per axis, for which each reference
// is clipped to every bin it spans (its triangle clipped to the reference's
// box within the bin); spatial splits are tried only where the object
// split's children overlap by more than kSpatialAlpha of the root's surface
// area.  A reference that straddles the chosen plane continues on both
// sides with the boxes of its two parts.  Triangles marked `fixed` are never
// split: they count whole in the bin of their box's centre and go to the
// side of it (their slots' boxes are refitted from whole triangles).  Leaves
// list triangle ids in leaf order (a triangle once per reference).
constexpr float kSpatialAlpha = 1e-3f;
constexpr int kSpatialBins = 32;

int build_spatial(const float* verts, int T, const uint8_t* fixed, std::vector<BNode>& nodes,
                  std::vector<int>& leaf_tri, std::vector<Box>& leaf_box) {
    struct Item {
        std::vector<Ref> refs;
        int parent, side, depth;
    };
    std::vector<Ref> init(T);
    Box rootb;
    for (int t = 0; t < T; ++t) {
        init[t].tri = t;
        for (int k = 0; k < 3; ++k) init[t].box.grow(verts + 9 * (size_t)t + 3 * k);
        rootb.grow(init[t].box);
    }
    const float root_area = rootb.area();
    size_t total = (size_t)T;   // references so far
    std::vector<Item> work;
    work.push_back({std::move(init), -1, 0, 0});
    int root = -1;
    while (!work.empty()) {
        Item it = std::move(work.back());
        work.pop_back();
        const std::vector<Ref>& refs = it.refs;
        const int n = (int)refs.size();
        Box b, cb;
        for (const Ref& r : refs) {
            b.grow(r.box);
            float c[3];
            for (int a = 0; a < 3; ++a) c[a] = 0.5f * (r.box.lo[a] + r.box.hi[a]);
            cb.grow(c);
        }
        // object split: binned SAH over the box centres
        float best_o = FLT_MAX;
        int oa = -1, obin = -1;
        Box oL, oR;
        for (int a = 0; a < 3 && n > 1; ++a) {
            const float ext = cb.hi[a] - cb.lo[a];
            if (!(ext > 0.f)) continue;
            Box bb[kBins];
            int bc[kBins] = {0};
            const float scale = kBins / ext;
            for (const Ref& r : refs) {
                const int bi = std::min(kBins - 1, (int)((0.5f * (r.box.lo[a] + r.box.hi[a]) - cb.lo[a]) * scale));
                bc[bi]++;
                bb[bi].grow(r.box);
            }
            Box lb[kBins], rb[kBins];
            int lc[kBins], rc[kBins];
            Box acc;
            int m = 0;
            for (int i = 0; i < kBins; ++i) {
                acc.grow(bb[i]);
                m += bc[i];
                lb[i] = acc;
                lc[i] = m;
            }
            acc = Box();
            m = 0;
            for (int i = kBins - 1; i >= 0; --i) {
                acc.grow(bb[i]);
                m += bc[i];
                rb[i] = acc;
                rc[i] = m;
            }
            for (int i = 0; i + 1 < kBins; ++i) {
                if (lc[i] == 0 || rc[i + 1] == 0) continue;
                const float c = lb[i].area() * lc[i] + rb[i + 1].area() * rc[i + 1];
                if (c < best_o) {
                    best_o = c;
                    oa = a;
                    obin = i;
                    oL = lb[i];
                    oR = rb[i + 1];
                }
            }
        }
        // spatial split where the object split's children overlap
        float best_s = FLT_MAX, splane = 0.f;
        int sa = -1;
        if (n > 1 && oa >= 0 && it.depth < 64 && total < 4 * (size_t)T &&
            overlap_area(oL, oR) > kSpatialAlpha * root_area) {
            for (int a = 0; a < 3; ++a) {
                const float ext = b.hi[a] - b.lo[a];
                if (!(ext > 0.f)) continue;
                const float w = ext / kSpatialBins;
                Box bb[kSpatialBins];
                int ent[kSpatialBins] = {0}, ex[kSpatialBins] = {0};
                for (const Ref& r : refs) {
                    int b0 = std::min(kSpatialBins - 1, std::max(0, (int)((r.box.lo[a] - b.lo[a]) / w)));
                    int b1 = std::min(kSpatialBins - 1, std::max(0, (int)((r.box.hi[a] - b.lo[a]) / w)));
                    if (fixed && fixed[r.tri])   // whole, in the bin of its centre
                        b0 = b1 = std::min(kSpatialBins - 1,
                                           std::max(0, (int)((0.5f * (r.box.lo[a] + r.box.hi[a]) - b.lo[a]) / w)));
                    ent[b0]++;
                    ex[b1]++;
                    if (b0 == b1) {
                        bb[b0].grow(r.box);
                        continue;
                    }
                    for (int k = b0; k <= b1; ++k) {
                        Box cl = r.box;
                        cl.lo[a] = std::max(cl.lo[a], b.lo[a] + k * w);
                        cl.hi[a] = std::min(cl.hi[a], k == kSpatialBins - 1 ? b.hi[a] : b.lo[a] + (k + 1) * w);
                        const Box pb = clip_tri_box(verts, r.tri, cl);
                        if (pb.valid()) bb[k].grow(pb);
                    }
                }
                Box lb[kSpatialBins], rb[kSpatialBins];
                int lc[kSpatialBins], rc[kSpatialBins];
                Box acc;
                int m = 0;
                for (int i = 0; i < kSpatialBins; ++i) {
                    acc.grow(bb[i]);
                    m += ent[i];
                    lb[i] = acc;
                    lc[i] = m;
                }
                acc = Box();
                m = 0;
                for (int i = kSpatialBins - 1; i >= 0; --i) {
                    acc.grow(bb[i]);
                    m += ex[i];
                    rb[i] = acc;
                    rc[i] = m;
                }
                for (int i = 0; i + 1 < kSpatialBins; ++i) {
                    if (lc[i] == 0 || rc[i + 1] == 0 || lc[i] >= n || rc[i + 1] >= n) continue;
                    const float c = lb[i].area() * lc[i] + rb[i + 1].area() * rc[i + 1];
                    if (c < best_s) {
                        best_s = c;
                        sa = a;
                        splane = b.lo[a] + (i + 1) * w;
                    }
                }
            }
        }
        const float best = std::min(best_o, best_s);
        const float sah = 0.5f * b.area() + best;   // traversal cost of one node
        const bool nosplit = oa < 0 && sa < 0;
        const bool leaf = n <= 2 || (n <= kMaxLeaf && (nosplit || sah >= (float)n * b.area()));
        BNode nd;
        nd.box = b;
        int self;
        if (leaf) {
            nd.first = (int)leaf_tri.size();
            nd.count = n;
            for (const Ref& r : refs) {
                leaf_tri.push_back(r.tri);
                leaf_box.push_back(r.box);
            }
            nodes.push_back(nd);
            self = (int)nodes.size() - 1;
        } else {
            std::vector<Ref> L, R;
            if (sa >= 0 && best_s < best_o) {
                for (const Ref& r : refs) {
                    if (fixed && fixed[r.tri]) {
                        (0.5f * (r.box.lo[sa] + r.box.hi[sa]) < splane ? L : R).push_back(r);
                    } else if (r.box.hi[sa] <= splane) {
                        L.push_back(r);
                    } else if (r.box.lo[sa] >= splane) {
                        R.push_back(r);
                    } else {
                        Box cl = r.box, cr = r.box;
                        cl.hi[sa] = splane;
                        cr.lo[sa] = splane;
                        const Box pl = clip_tri_box(verts, r.tri, cl), pr = clip_tri_box(verts, r.tri, cr);
                        if (pl.valid()) L.push_back({r.tri, pl});
                        if (pr.valid()) R.push_back({r.tri, pr});
                        if (!pl.valid() && !pr.valid()) L.push_back(r);   // never drop a triangle
                    }
                }
                if (L.empty() || R.empty() || (int)L.size() >= n || (int)R.size() >= n) {
                    L.clear();
                    R.clear();
                }
            }
            if (L.empty() && oa >= 0) {
                const float scale = kBins / (cb.hi[oa] - cb.lo[oa]);
                for (const Ref& r : refs) {
                    const int bi =
                        std::min(kBins - 1, (int)((0.5f * (r.box.lo[oa] + r.box.hi[oa]) - cb.lo[oa]) * scale));
                    (bi <= obin ? L : R).push_back(r);
                }
            }
            if (L.empty() || R.empty()) {   // degenerate: split by position
                L.assign(refs.begin(), refs.begin() + n / 2);
                R.assign(refs.begin() + n / 2, refs.end());
            }
            total += L.size() + R.size() - (size_t)n;
            nodes.push_back(nd);
            self = (int)nodes.size() - 1;
            work.push_back({std::move(R), self, 1, it.depth + 1});
            work.push_back({std::move(L), self, 0, it.depth + 1});
        }
        if (it.parent < 0)
            root = self;
        else if (it.side == 0)
            nodes[it.parent].left = self;
        else
            nodes[it.parent].right = self;
    }
    return root;
}

}  // namespace

void build_bvh4(const float* verts, uint32_t num_tris, const uint8_t* fixed, Bvh4* out) {
    const int T = (int)num_tris;
    // the binary tree and its leaves' triangles in leaf order
    std::vector<BNode> nodes;
    std::vector<int> leaf_tri;
    std::vector<Box> leaf_box;
    nodes.reserve(4 * (size_t)T);
    const int root = T > 0 ? build_spatial(verts, T, fixed, nodes, leaf_tri, leaf_box) : -1;
    const int S = (int)leaf_tri.size();
    out->slot_box.resize(6 * (size_t)S);
    for (int k = 0; k < S; ++k)
        for (int a = 0; a < 3; ++a) {
            out->slot_box[6 * (size_t)k + a] = leaf_box[k].lo[a];
            out->slot_box[6 * (size_t)k + 3 + a] = leaf_box[k].hi[a];
        }

    // triangle slots in leaf order: (v0, original index bits), e1, e2
    out->tris.assign(12 * (size_t)S, 0.f);
    for (int k = 0; k < S; ++k) {
        const int t = leaf_tri[k];
        const float* v = verts + 9 * (size_t)t;
        float* o = &out->tris[12 * (size_t)k];
        uint32_t tid = (uint32_t)t;
        o[0] = v[0]; o[1] = v[1]; o[2] = v[2];
        std::memcpy(&o[3], &tid, 4);
        for (int a = 0; a < 3; ++a) {
            o[4 + a] = v[3 + a] - v[a];
            o[8 + a] = v[6 + a] - v[a];
        }
    }

    // collapse to 4-wide nodes, breadth-first
    out->nodes.clear();
    struct Q {
        int bnode;   // binary node whose children become this node's slots
        int depth;
    };
    std::vector<Q> queue;
    std::vector<std::vector<int>> slots;
    if (root < 0) {   // no triangles: a root of four empty slots
        out->nodes.assign(32, 0.f);
        float* n = out->nodes.data();
        for (int c = 0; c < 4; ++c)
            for (int r = 0; r < 6; r += 2) n[4 * r + c] = FLT_MAX, n[4 * r + 4 + c] = -FLT_MAX;
        out->num_nodes = 1;
        out->depth = 1;
        return;
    }
    // SAH-optimal collapse (dynamic programming over the binary tree):
    // cost[n][k] is the least cost of the subtree of binary node n spread
    // over at most k slots of the enclosing 4-wide node; a slot holding an
    // inner node costs its area x kNodeCost plus its own children's best
    // spread over 4 slots, a leaf its area x triangles x kTriCost
    constexpr double kNodeCost = 1.0, kTriCost = 0.4;
    const size_t BN = nodes.size();
    std::vector<std::array<double, 5>> cost(BN);
    std::vector<std::array<signed char, 5>> split(BN);   // k1 of the best spread over exactly k slots, 0: fewer
    {
        std::vector<int> post;
        post.reserve(BN);
        std::vector<int> st{root};
        while (!st.empty()) {   // reverse pre-order (node, right, left) = a post-order
            int n = st.back();
            st.pop_back();
            post.push_back(n);
            if (nodes[n].left >= 0) {
                st.push_back(nodes[n].left);
                st.push_back(nodes[n].right);
            }
        }
        for (auto it = post.rbegin(); it != post.rend(); ++it) {
            const int n = *it;
            const BNode& bn = nodes[n];
            const double A = bn.box.area();
            if (bn.left < 0) {
                for (int k = 1; k <= 4; ++k) {
                    cost[n][k] = A * bn.count * kTriCost;
                    split[n][k] = 0;
                }
                continue;
            }
            const auto& L = cost[bn.left];
            const auto& R = cost[bn.right];
            double open[5] = {0, 0, 0, 0, 0};
            signed char ok1[5] = {0, 0, 0, 0, 0};
            for (int k = 2; k <= 4; ++k) {
                open[k] = 1e300;
                for (int k1 = 1; k1 < k; ++k1) {
                    double c = L[k1] + R[k - k1];
                    if (c < open[k]) {
                        open[k] = c;
                        ok1[k] = (signed char)k1;
                    }
                }
            }
            cost[n][1] = A * kNodeCost + open[4];
            split[n][1] = 0;
            for (int k = 2; k <= 4; ++k) {
                if (open[k] < cost[n][k - 1]) {
                    cost[n][k] = open[k];
                    split[n][k] = ok1[k];
                } else {
                    cost[n][k] = cost[n][k - 1];
                    split[n][k] = 0;
                }
            }
        }
    }
    // the slots of binary node n spread over at most k slots
    auto collect = [&](int n, int k, std::vector<int>& out) {
        std::vector<std::pair<int, int>> st{{n, k}};
        while (!st.empty()) {
            auto [m, km] = st.back();
            st.pop_back();
            while (km > 1 && split[m][km] == 0) --km;
            if (km <= 1 || nodes[m].left < 0) {
                out.push_back(m);
                continue;
            }
            const int k1 = split[m][km];
            st.push_back({nodes[m].right, km - k1});
            st.push_back({nodes[m].left, k1});
        }
    };
    queue.push_back({root, 1});
    uint32_t max_depth = 1;
    for (size_t qi = 0; qi < queue.size(); ++qi) {
        int bn = queue[qi].bnode;
        std::vector<int> ch;
        if (nodes[bn].left < 0) {
            ch.push_back(bn);   // a leaf root: one leaf slot
        } else {
            // the node's children: its two binary children spread over 4 slots
            double bestc = 1e300;
            int bk1 = 1;
            for (int k1 = 1; k1 < 4; ++k1) {
                double c = cost[nodes[bn].left][k1] + cost[nodes[bn].right][4 - k1];
                if (c < bestc) {
                    bestc = c;
                    bk1 = k1;
                }
            }
            collect(nodes[bn].left, bk1, ch);
            collect(nodes[bn].right, 4 - bk1, ch);
        }
        slots.push_back(ch);
        for (int c : ch)
            if (nodes[c].left >= 0) queue.push_back({c, queue[qi].depth + 1});
        max_depth = std::max(max_depth, (uint32_t)queue[qi].depth);
    }
    // queue order is node order; assign indices of inner children
    size_t N = queue.size();
    out->nodes.assign(32 * N, 0.f);
    size_t next = 1;
    for (size_t qi = 0; qi < N; ++qi) {
        float* n = &out->nodes[32 * qi];
        const std::vector<int>& ch = slots[qi];
        for (int c = 0; c < 4; ++c) {
            // an empty slot: inverted box, entry 0
            int32_t entry = 0;
            float lo[3] = {FLT_MAX, FLT_MAX, FLT_MAX}, hi[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
            if (c < (int)ch.size()) {
                const BNode& cn = nodes[ch[c]];
                for (int a = 0; a < 3; ++a) {
                    lo[a] = cn.box.lo[a];
                    hi[a] = cn.box.hi[a];
                }
                entry = cn.left < 0 ? bvh_leaf_entry(cn.first, cn.count) : (int32_t)next++;
            }
            n[0 + c] = lo[0];
            n[4 + c] = hi[0];
            n[8 + c] = lo[1];
            n[12 + c] = hi[1];
            n[16 + c] = lo[2];
            n[20 + c] = hi[2];
            std::memcpy(&n[24 + c], &entry, 4);
            n[28 + c] = 0.f;   // row 7: unused
        }
    }
    out->num_nodes = (uint32_t)N;
    out->depth = max_depth;
}
