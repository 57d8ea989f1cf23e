// Host check of the BVH4 builder (compiled by tests/test_bvh_cpu.py together
// with csrc/bvh_build.cpp; no GPU).  Reads float32 triangles [T][3][3] from
// argv[1], builds with spatial splits for every triangle, for none or for
// every other pair of triangles (argv[2] = 1 / 0 / 2: the others fixed) and
// checks the structure and the geometry:
//   - every inner child index is a node other than the root, reached once;
//     empty slots carry the inverted box, and row 7 is zero;
//   - every triangle is referenced by some leaf (exactly once without split
//     references), and each child box contains its child node's boxes;
//   - without split references, each leaf box contains its triangles; a
//     fixed triangle has exactly one slot, with its whole triangle's box;
//   - closest hits of random rays traced through the tree (fp64 slab and
//     Moller-Trumbore tests, the slab test widened by 1e-9 of the scene size)
//     equal brute force over all triangles: a box that lost part of its
//     triangle would miss.
// Prints one line of counts; exit status 0 when all are clean.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <random>
#include <vector>

#include "../paper_2108_05263_gb300/csrc/bvh.h"

namespace {

struct V3 {
    double x, y, z;
};
V3 sub(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
V3 cross(V3 a, V3 b) { return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }
double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }

// two-sided Moller-Trumbore in fp64; t or +inf
double tri_t(const float* v, V3 o, V3 d) {
    V3 v0 = {v[0], v[1], v[2]}, v1 = {v[3], v[4], v[5]}, v2 = {v[6], v[7], v[8]};
    V3 e1 = sub(v1, v0), e2 = sub(v2, v0);
    V3 p = cross(d, e2);
    double det = dot(e1, p);
    if (det == 0.0) return INFINITY;
    double inv = 1.0 / det;
    V3 tv = sub(o, v0);
    double b1 = dot(tv, p) * inv;
    if (b1 < 0.0 || b1 > 1.0) return INFINITY;
    V3 q = cross(tv, e1);
    double b2 = dot(d, q) * inv;
    if (b2 < 0.0 || b1 + b2 > 1.0) return INFINITY;
    double t = dot(e2, q) * inv;
    return t > 1e-9 ? t : INFINITY;
}

// slot entry: 0 empty, > 0 inner node, < 0 leaf (bvh.h)
int32_t entry_of(const float* nd, int c) {
    int32_t x;
    std::memcpy(&x, &nd[24 + c], 4);
    return x;
}
bool used(const float* nd, int c) { return entry_of(nd, c) != 0; }

}  // namespace

int main(int argc, char** argv) {
    if (argc < 3) return 2;
    FILE* f = std::fopen(argv[1], "rb");
    if (!f) return 2;
    std::vector<float> v;
    float buf[9];
    while (std::fread(buf, 4, 9, f) == 9) v.insert(v.end(), buf, buf + 9);
    std::fclose(f);
    // 0: every triangle fixed (unsplit), 1: none fixed, 2: every other pair fixed
    const int mode = std::atoi(argv[2]);
    const bool split = mode != 0;
    const uint32_t T = (uint32_t)(v.size() / 9);
    Bvh4 b;
    std::vector<uint8_t> fixed(T, 1);
    for (uint32_t t = 0; t < T; ++t) fixed[t] = mode == 0 || (mode == 2 && (t / 2) % 2 == 0);
    build_bvh4(v.data(), T, mode == 1 ? nullptr : fixed.data(), &b);
    // a fixed triangle: exactly one slot, whose reference box is the whole
    // triangle's box (moving triangles' slots are refitted from whole triangles)
    long bad_fixed = 0;
    {
        std::vector<int> refs(T, 0);
        for (uint32_t k = 0; k < (uint32_t)(b.tris.size() / 12); ++k) {
            uint32_t orig;
            std::memcpy(&orig, &b.tris[12 * (size_t)k + 3], 4);
            if (orig >= T || !fixed[orig] || mode == 1) continue;
            refs[orig]++;
            const float* w = &v[9 * (size_t)orig];
            for (int a = 0; a < 3; ++a) {
                const float lo = std::min(w[a], std::min(w[3 + a], w[6 + a]));
                const float hi = std::max(w[a], std::max(w[3 + a], w[6 + a]));
                if (b.slot_box[6 * (size_t)k + a] != lo || b.slot_box[6 * (size_t)k + 3 + a] != hi) bad_fixed++;
            }
        }
        for (uint32_t t = 0; t < T; ++t)
            if (mode != 1 && fixed[t] && refs[t] != 1) bad_fixed++;
    }
    const uint32_t S = (uint32_t)(b.tris.size() / 12);
    long bad_child = 0, bad_box = 0, missing = 0, dup = 0, orphan = 0, bad_tri = 0;
    std::vector<int> seen(T, 0), reached(b.num_nodes, 0);
    for (uint32_t n = 0; n < b.num_nodes; ++n) {
        const float* nd = &b.nodes[32 * (size_t)n];
        for (int c = 0; c < 4; ++c) {
            if (nd[28 + c] != 0.f) bad_child++;   // row 7 is unused
            if (!used(nd, c)) {
                // an empty slot's box is inverted on every axis
                for (int a = 0; a < 3; ++a)
                    if (nd[8 * a + c] != FLT_MAX || nd[8 * a + 4 + c] != -FLT_MAX) bad_box++;
                continue;
            }
            const float lo[3] = {nd[0 + c], nd[8 + c], nd[16 + c]}, hi[3] = {nd[4 + c], nd[12 + c], nd[20 + c]};
            const int32_t ch = entry_of(nd, c);
            if (ch < 0) {
                int32_t first, cnt;
                bvh_leaf_range(ch, &first, &cnt);
                if (first < 0 || first + cnt > (int)S) {
                    bad_child++;
                    continue;
                }
                for (int k = first; k < first + cnt; ++k) {
                    uint32_t orig;
                    std::memcpy(&orig, &b.tris[12 * (size_t)k + 3], 4);
                    if (orig >= T) {
                        bad_tri++;
                        continue;
                    }
                    seen[orig]++;
                    // the slot record is the triangle: v0, e1 = v1 - v0, e2 = v2 - v0
                    const float* t = &b.tris[12 * (size_t)k];
                    const float* w = &v[9 * (size_t)orig];
                    for (int a = 0; a < 3; ++a)
                        if (t[a] != w[a] || t[4 + a] != w[3 + a] - w[a] || t[8 + a] != w[6 + a] - w[a]) bad_tri++;
                    if (split) continue;   // a split reference's box holds part of its triangle
                    for (int p = 0; p < 3; ++p)
                        for (int a = 0; a < 3; ++a) {
                            const float x = w[3 * p + a];
                            if (x < lo[a] || x > hi[a]) bad_box++;
                        }
                }
            } else {
                if ((uint32_t)ch >= b.num_nodes) {
                    bad_child++;
                    continue;
                }
                reached[ch]++;
                const float* cn = &b.nodes[32 * (size_t)ch];
                for (int cc = 0; cc < 4; ++cc) {
                    if (!used(cn, cc)) continue;
                    if (cn[0 + cc] < lo[0] || cn[4 + cc] > hi[0] || cn[8 + cc] < lo[1] || cn[12 + cc] > hi[1] ||
                        cn[16 + cc] < lo[2] || cn[20 + cc] > hi[2])
                        bad_box++;
                }
            }
        }
    }
    for (uint32_t t = 0; t < T; ++t) {
        missing += seen[t] == 0;
        dup += !split && seen[t] > 1;
    }
    for (uint32_t n = 1; n < b.num_nodes; ++n) orphan += reached[n] != 1;

    // random rays: tree traversal against brute force
    double slo[3] = {1e30, 1e30, 1e30}, shi[3] = {-1e30, -1e30, -1e30};
    for (size_t i = 0; i < v.size(); ++i) {
        slo[i % 3] = std::min(slo[i % 3], (double)v[i]);
        shi[i % 3] = std::max(shi[i % 3], (double)v[i]);
    }
    const double diag = std::sqrt((shi[0] - slo[0]) * (shi[0] - slo[0]) + (shi[1] - slo[1]) * (shi[1] - slo[1]) +
                                  (shi[2] - slo[2]) * (shi[2] - slo[2]));
    const double eps = 1e-9 * diag;
    const int rays = argc > 3 ? std::atoi(argv[3]) : 2000;
    std::mt19937 rng(7);
    std::uniform_real_distribution<double> U(0.0, 1.0);
    long ray_mismatch = 0;
    for (int r = 0; r < rays && T > 0; ++r) {
        V3 o = {slo[0] + U(rng) * (shi[0] - slo[0]), slo[1] + U(rng) * (shi[1] - slo[1]),
                slo[2] + U(rng) * (shi[2] - slo[2])};
        double z = 2.0 * U(rng) - 1.0, ph = 6.283185307179586 * U(rng), s = std::sqrt(1.0 - z * z);
        V3 d = {s * std::cos(ph), s * std::sin(ph), z};
        double best_brute = INFINITY;
        for (uint32_t t = 0; t < T; ++t) best_brute = std::min(best_brute, tri_t(&v[9 * (size_t)t], o, d));
        double best = INFINITY;
        std::vector<int> st{0};
        const double inv[3] = {1.0 / d.x, 1.0 / d.y, 1.0 / d.z}, oo[3] = {o.x, o.y, o.z};
        while (!st.empty()) {
            const int n = st.back();
            st.pop_back();
            const float* nd = &b.nodes[32 * (size_t)n];
            for (int c = 0; c < 4; ++c) {
                if (!used(nd, c)) continue;
                double t0 = 0.0, t1 = INFINITY;
                const double lo[3] = {nd[0 + c] - eps, nd[8 + c] - eps, nd[16 + c] - eps};
                const double hi[3] = {nd[4 + c] + eps, nd[12 + c] + eps, nd[20 + c] + eps};
                for (int a = 0; a < 3; ++a) {
                    double ta = (lo[a] - oo[a]) * inv[a], tb = (hi[a] - oo[a]) * inv[a];
                    if (ta > tb) std::swap(ta, tb);
                    t0 = std::max(t0, ta);
                    t1 = std::min(t1, tb);
                }
                if (!(t0 <= t1)) continue;
                const int32_t ch = entry_of(nd, c);
                if (ch > 0) {
                    st.push_back(ch);
                } else {
                    int32_t first, cnt;
                    bvh_leaf_range(ch, &first, &cnt);
                    for (int k = first; k < first + cnt; ++k) {
                        uint32_t orig;
                        std::memcpy(&orig, &b.tris[12 * (size_t)k + 3], 4);
                        if (orig < T) best = std::min(best, tri_t(&v[9 * (size_t)orig], o, d));
                    }
                }
            }
        }
        if (!(best == best_brute || (std::isinf(best) && std::isinf(best_brute)))) ray_mismatch++;
    }
    std::printf("triangles %u slots %u nodes %u depth %u missing %ld dup %ld bad_box %ld bad_child %ld orphan %ld "
                "bad_tri %ld bad_fixed %ld ray_mismatch %ld of %d\n",
                T, S, b.num_nodes, b.depth, missing, dup, bad_box, bad_child, orphan, bad_tri, bad_fixed, ray_mismatch,
                rays);
    return (missing || dup || bad_box || bad_child || orphan || bad_tri || bad_fixed || ray_mismatch) ? 1 : 0;
}
