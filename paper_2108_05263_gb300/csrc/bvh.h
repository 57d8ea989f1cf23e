// Host BVH4 build interface (plain C++, no CUDA types).
#pragma once
#include <stdint.h>

#include <vector>

struct Bvh4 {
    std::vector<float> nodes;   // 32 floats per node (layout in trace.cuh)
    std::vector<float> tris;    // 12 floats per triangle slot, leaf order
    uint32_t num_nodes = 0;
    uint32_t depth = 0;
};

// Builds an SAH binary BVH over `num_tris` triangles (9 floats each) and
// collapses it to 4-wide nodes.  split_large: triangles with large boxes
// enter as several clipped references (a triangle then fills several slots of
// `tris`); off for scenes whose boxes are refitted from whole triangles.
void build_bvh4(const float* verts, uint32_t num_tris, bool split_large, Bvh4* out);
