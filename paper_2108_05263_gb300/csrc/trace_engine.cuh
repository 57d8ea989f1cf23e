// Persistent ray-traversal kernel with per-warp dynamic work refill.
//
// Each lane owns one ray at a time; per loop iteration it descends inner
// nodes until the warp's lanes each hold a leaf (speculative traversal), then
// intersects that leaf; when a lane's ray finishes, the warp hands it the next work item
// from a warp-private pool (refilled 64 items at a time from a global
// counter), so lanes with short rays do not idle behind lanes with long ones.
// A generator functor turns a work index into a ray; the result of work item
// i is written to hits[i] as (t, triangle bits) -- (tmax, 0xFFFFFFFF) on a
// miss or when the generator emits no ray.  Any-hit rays stop at the first
// hit in (tmin, tmax).
//
// BVH entries on the traversal stack: >= 0 inner node index; < 0 a leaf,
// encoded as -1 - (first_triangle * 8 + count - 1).
#pragma once
#include "trace.cuh"

#define ENGINE_THREADS 128
#define ENGINE_GRAB 64u

__device__ __forceinline__ int leaf_entry(int first, int count) { return -1 - (first * 8 + count - 1); }

// traversal stack entry: (BVH entry, entry distance bits), one 8-byte access
// pops the next entry that can still hold a hit closer than `limit`
__device__ __forceinline__ bool pop_entry(const int2* stack, int& sp, float limit, int& node) {
    while (sp > 0) {
        --sp;
        const int2 e = stack[sp];
        if (__int_as_float(e.y) <= limit) {
            node = e.x;
            return true;
        }
    }
    return false;
}

// One step of a ray's traversal: descend inner nodes; the first leaf the
// lane meets is set aside and the lane keeps descending from its stack while
// other lanes of the warp still look for one (Aila & Laine 2009, speculative
// traversal); then the set-aside leaf is intersected.  Returns true when the
// ray is done (best_t / best_tri hold its result).  Shared by the persistent
// engine and the per-thread trace_spec.
// element c (0..3) of a 4-array held in registers, without local memory
template <class T>
__device__ __forceinline__ T sel4(const T (&a)[4], int c) {
    return c == 0 ? a[0] : c == 1 ? a[1] : c == 2 ? a[2] : a[3];
}

template <bool ANY_HIT, bool SORTED>
__device__ __forceinline__ bool trav_step(const SceneView& s, const f3& o, const f3& d, const f3& inv, const f3& oi,
                                          float tmin, float tmax, float& best_t, uint32_t& best_tri, int& node,
                                          int& sp, int& visits, bool& more, int2* stack) {
    const float widen = 1.0000004f;
    bool done = false;
    int leaf = 0;   // set-aside leaf entry (< 0), 0: none
    while (true) {
        if (more && node < 0 && leaf == 0) {
            leaf = node;
            more = pop_entry(stack, sp, best_t * widen, node);
        }
        if (!(more && node >= 0)) break;
        // every lane still descending takes part in the vote
        const bool all_hold = __all_sync(__activemask(), leaf != 0);
        if (leaf != 0 && all_hold) break;
        if (++visits > s.max_visits) {
            atomicOr(s.err, ERRBIT_TRAVERSAL);
            best_tri = DDGI_NONE;
            best_t = tmax;
            done = true;
            break;
        }
        const float4* np = s.nodes + (size_t)node * 8;
        // each axis's near and far rows by the ray's sign: an inverted
        // (empty) box never passes
        const int ox = inv.x < 0.f, oy = inv.y < 0.f, oz = inv.z < 0.f;
        const float4 nx = ldg4(np + ox), fx = ldg4(np + 1 - ox);
        const float4 ny = ldg4(np + 2 + oy), fy = ldg4(np + 3 - oy);
        const float4 nz = ldg4(np + 4 + oz), fz = ldg4(np + 5 - oz);
        const float4 ef = ldg4(np + 6);
        const float nxa[4] = {nx.x, nx.y, nx.z, nx.w}, fxa[4] = {fx.x, fx.y, fx.z, fx.w};
        const float nya[4] = {ny.x, ny.y, ny.z, ny.w}, fya[4] = {fy.x, fy.y, fy.z, fy.w};
        const float nza[4] = {nz.x, nz.y, nz.z, nz.w}, fza[4] = {fz.x, fz.y, fz.z, fz.w};
        const int ent[4] = {__float_as_int(ef.x), __float_as_int(ef.y), __float_as_int(ef.z), __float_as_int(ef.w)};
        float t0[4];
        int key[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            float a = fmaxf(fmaxf(fmaf(nxa[c], inv.x, -oi.x), fmaf(nya[c], inv.y, -oi.y)),
                            fmaxf(fmaf(nza[c], inv.z, -oi.z), tmin));
            float b = fminf(fminf(fmaf(fxa[c], inv.x, -oi.x), fmaf(fya[c], inv.y, -oi.y)),
                            fminf(fmaf(fza[c], inv.z, -oi.z), best_t)) * widen;
            t0[c] = a <= b ? a : INFINITY;
            key[c] = (__float_as_int(t0[c]) & ~3) | c;
        }
        const int nhit = (t0[0] < INFINITY) + (t0[1] < INFINITY) + (t0[2] < INFINITY) + (t0[3] < INFINITY);
        if (sp + nhit > TRAV_STACK) {
            atomicOr(s.err, ERRBIT_STACK);
            best_tri = DDGI_NONE;
            best_t = tmax;
            done = true;
            break;
        }
        if (SORTED) {
            // all hit children by entry distance: push far-to-near, continue
            // with the nearest (sorting network on the keys)
#define KSWAP(i, j)                 \
    {                               \
        const int lo_ = min(key[i], key[j]); \
        key[j] = max(key[i], key[j]);        \
        key[i] = lo_;                        \
    }
            KSWAP(0, 1)
            KSWAP(2, 3)
            KSWAP(0, 2)
            KSWAP(1, 3)
            KSWAP(1, 2)
#undef KSWAP
#pragma unroll
            for (int k = 3; k >= 1; --k)
                if (k < nhit) {
                    const int c = key[k] & 3;
                    stack[sp] = make_int2(sel4(ent, c), __float_as_int(sel4(t0, c)));
                    ++sp;
                }
            if (nhit > 0)
                node = sel4(ent, key[0] & 3);
            else
                more = pop_entry(stack, sp, best_t * widen, node);
        } else {
            // continue with the nearest child; push the others in slot order
            // (far ones are culled when popped)
            const int near = min(min(key[0], key[1]), min(key[2], key[3])) & 3;
#pragma unroll
            for (int c = 3; c >= 0; --c)
                if (c != near && t0[c] < INFINITY) {
                    stack[sp] = make_int2(ent[c], __float_as_int(t0[c]));
                    ++sp;
                }
            if (nhit > 0)
                node = sel4(ent, near);
            else
                more = pop_entry(stack, sp, best_t * widen, node);
        }
    }
    if (!done && leaf != 0) {
        const int v = -1 - leaf;
        const int first = v >> 3, count = (v & 7) + 1;
        for (int k = 0; k < count; ++k) {
            uint32_t orig;
            float t = tri_hit(s.tris + (size_t)(first + k) * 3, o, d, &orig);
            if (t > tmin && t < tmax) {
                if (ANY_HIT) {
                    best_t = t;
                    best_tri = orig;
                    done = true;
                    break;
                }
                if (t < best_t || (t == best_t && orig < best_tri)) {
                    best_t = t;
                    best_tri = orig;
                }
            }
        }
    }
    if (!done && !more) done = true;
    return done;
}

// closest (or any) hit of one ray per thread with the same speculative
// descent, for kernels whose rays are not pooled
template <bool ANY_HIT>
__device__ __forceinline__ Hit trace_spec(const SceneView& s, const Ray& ray) {
    const f3 inv = {safe_inv(ray.d.x), safe_inv(ray.d.y), safe_inv(ray.d.z)};
    const f3 oi = {ray.o.x * inv.x, ray.o.y * inv.y, ray.o.z * inv.z};
    float best_t = ray.tmax;
    uint32_t best_tri = DDGI_NONE;
    int node = 0, sp = 0, visits = 0;
    bool more = true;
    int2 stack[TRAV_STACK];
    while (!trav_step<ANY_HIT, true>(s, ray.o, ray.d, inv, oi, ray.tmin, ray.tmax, best_t, best_tri, node, sp, visits,
                                     more, stack)) {
    }
    Hit h;
    h.t = best_t;
    h.tri = best_tri;
    return h;
}

template <class Gen, bool ANY_HIT>
// 9 CTAs per SM (56 registers: 8 bytes of spill, 36 warps instead of 32
// hide more of the node fetches' latency; 10 CTAs spill 92 bytes)
__global__ void __launch_bounds__(ENGINE_THREADS, 9) k_trace(SceneView s, Gen gen, uint32_t n,
                                                          uint32_t* __restrict__ counter,
                                                          float2* __restrict__ hits) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const unsigned lt_mask = (1u << lane) - 1u;
    // per-lane ray state
    uint32_t idx = DDGI_NONE;
    f3 o = {0.f, 0.f, 0.f}, d = {0.f, 0.f, 1.f}, inv = {0.f, 0.f, 0.f}, oi = {0.f, 0.f, 0.f};
    float tmin = 0.f, tmax = 0.f, best_t = 0.f;
    uint32_t best_tri = DDGI_NONE;
    int node = 0, sp = 0, visits = 0;
    bool more = false;   // node holds an entry still to visit
    int2 stack[TRAV_STACK];
    // warp-uniform work pool
    uint32_t pool = 0, pool_end = 0;
    bool exhausted = false;

    while (true) {
        // ---- refill idle lanes ------------------------------------------------
        while (true) {
            unsigned need = __ballot_sync(FULL, idx == DDGI_NONE);
            if (need == 0u) break;
            if (pool == pool_end) {
                if (exhausted) break;
                uint32_t base = 0;
                if (lane == 0) base = atomicAdd(counter, ENGINE_GRAB);
                base = __shfl_sync(FULL, base, 0);
                if (base >= n) {
                    exhausted = true;
                    break;
                }
                pool = base;
                pool_end = min(base + ENGINE_GRAB, n);
            }
            const uint32_t avail = pool_end - pool;
            const uint32_t rank = __popc(need & lt_mask);
            if (idx == DDGI_NONE && rank < avail) {
                const uint32_t i = pool + rank;
                Ray r;
                if (gen.ray(i, r)) {
                    idx = i;
                    o = r.o;
                    d = r.d;
                    tmin = r.tmin;
                    tmax = r.tmax;
                    inv = {safe_inv(d.x), safe_inv(d.y), safe_inv(d.z)};
                    oi = {o.x * inv.x, o.y * inv.y, o.z * inv.z};
                    best_t = tmax;
                    best_tri = DDGI_NONE;
                    node = 0;
                    more = true;
                    sp = 0;
                    visits = 0;
                } else {
                    hits[i] = make_float2(r.tmax, __uint_as_float(DDGI_NONE));
                }
            }
            pool += min(avail, (uint32_t)__popc(need));
        }
        if (__all_sync(FULL, idx == DDGI_NONE)) break;
        if (idx == DDGI_NONE) continue;

        const bool done = trav_step<ANY_HIT, false>(s, o, d, inv, oi, tmin, tmax, best_t, best_tri, node, sp, visits,
                                                    more, stack);
        if (done) {
            hits[idx] = make_float2(best_t, __uint_as_float(best_tri));
            idx = DDGI_NONE;
        }
    }
}

// Launches the persistent trace over n work items: a few warps per SM, the
// work counter reset on the stream first.
template <class Gen, bool ANY_HIT>
cudaError_t launch_trace(const SceneView& s, const Gen& gen, uint32_t n, uint32_t* counter,
                         float2* hits, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(uint32_t), st);
    if (e != cudaSuccess) return e;
    static int blocks = 0;
    if (blocks == 0) {
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_trace<Gen, ANY_HIT>, ENGINE_THREADS, 0);
        blocks = sms * (per_sm > 0 ? per_sm : 1);
    }
    uint32_t need = (n + ENGINE_THREADS - 1) / ENGINE_THREADS;
    uint32_t grid = need < (uint32_t)blocks ? need : (uint32_t)blocks;
    k_trace<Gen, ANY_HIT><<<grid, ENGINE_THREADS, 0, st>>>(s, gen, n, counter, hits);
    return cudaGetLastError();
}
