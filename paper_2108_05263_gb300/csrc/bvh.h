// Host BVH4 build interface (plain C++, no CUDA types).
#pragma once
#include <stdint.h>

#include <vector>

struct Bvh4 {
    std::vector<float> nodes;   // 32 floats per node (layout in trace.cuh)
    std::vector<float> tris;    // 12 floats per triangle slot, leaf order
    std::vector<float> slot_box;  // 6 floats per slot: its reference's box (lo, hi), clipped where split
    uint32_t num_nodes = 0;
    uint32_t depth = 0;
};

// Slot entry codes (row 6 of a node): 0 an empty slot (its box is inverted,
// so no ray enters it), > 0 the index of an inner node (the root, node 0, is
// nobody's child), < 0 a leaf of `count` (1..8) consecutive triangle slots
// from `first`, coded -1 - (first * 8 + count - 1).
inline int32_t bvh_leaf_entry(int32_t first, int32_t count) { return -1 - (first * 8 + count - 1); }
inline void bvh_leaf_range(int32_t entry, int32_t* first, int32_t* count) {
    const int32_t v = -1 - entry;
    *first = v >> 3;
    *count = (v & 7) + 1;
}

// Builds an SAH binary BVH with spatial splits over `num_tris` triangles (9
// floats each) and collapses it to 4-wide nodes: a triangle may be entered as
// several clipped references (it then fills several slots of `tris`), except
// the triangles with fixed[t] != 0, whose slot boxes are refitted from whole
// triangles (moving instances); fixed may be null (every triangle may split).
void build_bvh4(const float* verts, uint32_t num_tris, const uint8_t* fixed, Bvh4* out);
