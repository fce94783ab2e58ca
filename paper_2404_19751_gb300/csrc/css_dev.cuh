// css_dev.cuh -- device data layout and helpers shared by the library's kernels.
//
// Half-edge convention: face f, corner k, half-edge h = 3f+k runs from corner k to
// corner k+1.  The face layout puts corner 0 at (0,0), corner 1 at (L01,0) and
// corner 2 at (x2, y2 > 0).  The frame of half-edge h has its origin at corner k,
// x along the edge and +y pointing into face f.  A window lives on the half-edge
// of the face it propagates into; its pseudo-source s lies on the other side.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define CSS_FULL 0xffffffffu

namespace css {

// Per half-edge record (64 B): everything one unfolding step needs.
struct __align__(16) HeRec {
    double L;        // edge length
    double cx, cy;   // opposite corner c in this half-edge frame (cy > 0)
    double cl, sl;   // cos/sin of angle(c): rotation into the frame across edge c-u
    double cr, sr;   // cos/sin of angle(v - c): rotation into the frame across edge v-c
    int32_t tl, tr;  // twin of half-edge (f,k+2) [edge c-u] and (f,k+1) [edge v-c], -1: boundary
};

// FP32 copy of HeRec for the FP32 form's arithmetic (32 B)
struct __align__(16) HeRec32 {
    float L, cx, cy, cl, sl, cr, sr;
    int32_t pad;
};

struct DMesh {
    int32_t nv, nf;
    int32_t periodic;
    double per[2];
    const HeRec* he;              // 3 nf
    const int32_t* twin;          // 3 nf
    const int32_t* edge;          // 3 nf, undirected edge id = min(h, twin(h))
    const int32_t* fv;            // 3 nf, vertex at each corner
    const double* lay;            // 3 nf: L01, x2, y2 per face
    const double* frame;          // 9 nf: origin, e1, e2 per face (world)
    const double* theta;          // nv angle sums
    const uint8_t* pseudo;        // nv: boundary, flat or saddle vertex
    const uint8_t* bnd;           // nv: boundary vertex
    const int32_t* ring_start;    // nv + 1
    const int32_t* ring;          // 3 nf corners h with fv[h] == v, grouped by vertex
    const HeRec32* he32;          // 3 nf, FP32 copies of he
    const float* lay32;           // 3 nf, FP32 copies of lay
    const int32_t* frank;         // nf: rank of each face along a Morton curve (bucket order)
    const float2* cang;           // 3 nf: (start, width) of corner h around its vertex, angles
                                  // counted counter-clockwise from one fixed edge; NaN on boundary
                                  // and non-manifold vertices
};

__device__ __forceinline__ double cross2(double ax, double ay, double bx, double by) { return ax * by - ay * bx; }

__device__ __forceinline__ void face_corner(const DMesh& m, int f, int k, double& x, double& y) {
    k = (k >= 3) ? k - 3 : k;
    if (k == 0) { x = 0.0; y = 0.0; }
    else if (k == 1) { x = m.lay[3 * f]; y = 0.0; }
    else { x = m.lay[3 * f + 1]; y = m.lay[3 * f + 2]; }
}

// ------------------------------------------------------------------ generation-tagged hash
// Entry = (gen << 32) | key.  An entry whose gen differs from the current one is
// empty, so tables never need clearing between sources.  Reads bypass L1
// (ld.global.cg) because claims are made with L2 atomics.
__device__ __forceinline__ unsigned long long ld_cg_u64(const unsigned long long* p) { return __ldcg(p); }

__device__ __forceinline__ int ht_insert(unsigned long long* keys, int logcap, uint32_t gen, int32_t key,
                                         bool& claimed) {
    const unsigned long long want = ((unsigned long long)gen << 32) | (uint32_t)key;
    const uint32_t mask = (1u << logcap) - 1u;
    uint32_t slot = ((uint32_t)key * 2654435761u) >> (32 - logcap);
    claimed = false;
    for (uint32_t probe = 0; probe <= mask; ++probe) {
        unsigned long long cur = ld_cg_u64(keys + slot);
        for (;;) {
            if (cur == want) return (int)slot;
            if ((uint32_t)(cur >> 32) == gen) break;          // occupied by another key
            unsigned long long prev = atomicCAS(keys + slot, cur, want);
            if (prev == cur) { claimed = true; return (int)slot; }
            cur = prev;                                        // re-examine what won
        }
        slot = (slot + 1u) & mask;
    }
    return -1;
}

__device__ __forceinline__ int ht_find(const unsigned long long* keys, int logcap, uint32_t gen, int32_t key) {
    const unsigned long long want = ((unsigned long long)gen << 32) | (uint32_t)key;
    const uint32_t mask = (1u << logcap) - 1u;
    uint32_t slot = ((uint32_t)key * 2654435761u) >> (32 - logcap);
    for (uint32_t probe = 0; probe <= mask; ++probe) {
        unsigned long long cur = ld_cg_u64(keys + slot);
        if (cur == want) return (int)slot;
        if ((uint32_t)(cur >> 32) != gen) return -1;
        slot = (slot + 1u) & mask;
    }
    return -1;
}

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

template <class T>
__device__ __forceinline__ T warp_sum(T v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(CSS_FULL, v, o);
    return v;
}

// status bits written to the device status word
enum : int {
    ST_WIN_OVERFLOW = 1,     // window pool full
    ST_HASH_OVERFLOW = 2,    // a hash table full
    ST_PAIR_OVERFLOW = 4,    // per-source pair slab full
    ST_ITER_LIMIT = 8,       // loop cap reached
    ST_PIECES = 16,          // too many interval pieces in one trim
    ST_WALK_LIMIT = 32,      // face walk iteration cap
    ST_BAD_INPUT = 64,
};

}  // namespace css
