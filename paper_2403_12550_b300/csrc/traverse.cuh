// traverse.cuh -- exact search of the Morton bounding-volume hierarchy, one query per thread.
//
// Best-first depth-first walk: at an internal node both children's boxes are
// tested against the query's current bound, the nearer child is entered and
// the farther one pushed (with its distance) if it is also within the bound.
// The walk is written in "while-while" form: a thread first descends through
// internal nodes until it holds a leaf (or is done), then scans leaves until
// its next stack entry is an internal node.  Threads of a warp therefore scan
// their leaves together instead of interleaving leaf scans with node tests,
// which keeps the warp's divergent work close to its busiest lane's.
//
// Exactness: box_d2 is a lower bound, in the same rounded arithmetic
// (common.cuh), on the distance to every point inside the box, and a subtree
// is skipped only when that bound exceeds the query's current bound, which
// only ever shrinks.  Inclusive comparisons keep equal-distance points with
// smaller indices reachable.
#pragma once

#include "common.cuh"

namespace gsicp {

// leaf_fn(leaf) scans one leaf and may lower `bound` (captured by reference).
template <class LeafFn>
__device__ __forceinline__ void traverse(const IndexView& ix, float qx, float qy, float qz, const float& bound,
                                         LeafFn&& leaf_fn)
{
    const int L = ix.L;
    int stk[32];
    float sd[32];
    int sp = 0;
    int node = 1;  // heap index; 0 = done
    while (node != 0) {
        while (node != 0 && node < L) {
            const float4* bx = ix.boxes + 4 * node;  // children 2node, 2node+1
            const float d0 = box_d2(qx, qy, qz, bx[0], bx[1]);
            const float d1 = box_d2(qx, qy, qz, bx[2], bx[3]);
            const bool f0 = d0 <= d1;
            const int cn = f0 ? 2 * node : 2 * node + 1;
            const float dn = f0 ? d0 : d1, df = f0 ? d1 : d0;
            if (dn <= bound) {
                if (df <= bound && sp < 32) {
                    stk[sp] = cn ^ 1;
                    sd[sp] = df;
                    ++sp;
                }
                node = cn;
            } else {
                node = 0;
                while (sp > 0) {
                    --sp;
                    if (sd[sp] <= bound) {
                        node = stk[sp];
                        break;
                    }
                }
            }
        }
        while (node >= L) {
            leaf_fn(node - L);
            node = 0;
            while (sp > 0) {
                --sp;
                if (sd[sp] <= bound) {
                    node = stk[sp];
                    break;
                }
            }
        }
    }
}

// Eight-wide variant of traverse() for latency-bound single searches: a node's descendants three
// levels down are the contiguous heap nodes 8i..8i+7, so one step loads eight boxes (256 bytes) at
// once and a descent to a leaf takes a third of the dependent memory round trips.  The top
// (depth mod 3) levels are entered directly.  Same exactness argument as traverse().
constexpr int TRAVERSE8_STACK = 80;  // >= 7 per step x 10 steps (2^30 leaves) + 3 entry nodes

template <class LeafFn>
__device__ __forceinline__ void traverse8(const IndexView& ix, float qx, float qy, float qz, const float& bound,
                                          LeafFn&& leaf_fn)
{
    const int L = ix.L;
    int stk[TRAVERSE8_STACK];
    float sd[TRAVERSE8_STACK];
    int sp = 0;
    int node;
    const int r = (31 - __clz(L)) % 3;
    if (r == 0) {
        node = 1;
    } else {
        node = 0;
        float best = GSICP_INF;
        for (int c = 1 << r; c < (2 << r); ++c) {
            const float dc = box_d2(qx, qy, qz, ix.boxes[2 * c], ix.boxes[2 * c + 1]);
            if (dc <= bound) {
                if (dc < best) {
                    if (node) { stk[sp] = node; sd[sp] = best; ++sp; }
                    node = c;
                    best = dc;
                } else {
                    stk[sp] = c; sd[sp] = dc; ++sp;
                }
            }
        }
    }
    auto pop = [&]() -> int {
        while (sp > 0) {
            --sp;
            if (sd[sp] <= bound) return stk[sp];
        }
        return 0;
    };
    while (node != 0) {
        while (node != 0 && node < L) {
            const float4* bx = ix.boxes + 16 * node;  // boxes of nodes 8node .. 8node+7
            float dist[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) dist[c] = box_d2(qx, qy, qz, bx[2 * c], bx[2 * c + 1]);
            int nearest = -1;
            float dn = GSICP_INF;
#pragma unroll
            for (int c = 0; c < 8; ++c)
                if (dist[c] <= bound && dist[c] < dn) { dn = dist[c]; nearest = c; }
            if (nearest < 0) {
                node = pop();
                continue;
            }
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                if (c != nearest && dist[c] <= bound && sp < TRAVERSE8_STACK) {
                    stk[sp] = 8 * node + c;
                    sd[sp] = dist[c];
                    ++sp;
                }
            }
            node = 8 * node + nearest;
        }
        while (node >= L) {
            leaf_fn(node - L);
            node = pop();
        }
    }
}

// Visit the points [beg, end) of a sorted point array four at a time, the four loads issued
// before any is used: a latency-bound single search otherwise waits for each load in turn behind
// the data-dependent update.
template <class PointFn>
__device__ __forceinline__ void scan_points4(const float4* __restrict__ pts, int beg, int end, PointFn&& fn)
{
    for (int u0 = beg; u0 < end; u0 += 4) {
        float4 p[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) p[j] = u0 + j < end ? __ldg(pts + u0 + j) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (u0 + j < end) fn(u0 + j, p[j]);
    }
}

// Packet walk: the warp walks the tree once for the queries of all its lanes.  A node is entered
// when at least one searching lane's own bound reaches its box (per-lane box test + ballot); of
// two needed children the one most of those lanes find nearer goes first.  Leaf points are read
// by all lanes at once (same address: one broadcast load) and each lane updates only its own
// result, so the walk costs the union of the lanes' node sets instead of their divergent sum.
// Exactness is the per-lane argument of traverse(): a subtree is skipped only when no lane's
// bound reaches it.  Must be called by all 32 lanes (converged); `active` selects searching lanes.
template <class LeafFn>
__device__ __forceinline__ void packet_traverse(const IndexView& ix, bool active, float qx, float qy, float qz,
                                                const float& bound, LeafFn&& leaf_fn)
{
    constexpr unsigned FULL = 0xffffffffu;
    const int L = ix.L;
    int stk[32];    // same content in every lane (pushes are warp-uniform)
    float sd[32];   // this lane's distance to each stacked node
    int sp = 0;
    int node = __any_sync(FULL, active) ? 1 : 0;
    while (node != 0) {
        if (node >= L) {
            leaf_fn(node - L);
        } else {
            const float4* bx = ix.boxes + 4 * node;  // children 2node, 2node+1
            const float d0 = box_d2(qx, qy, qz, bx[0], bx[1]);
            const float d1 = box_d2(qx, qy, qz, bx[2], bx[3]);
            const bool n0 = active && d0 <= bound, n1 = active && d1 <= bound;
            const unsigned m0 = __ballot_sync(FULL, n0), m1 = __ballot_sync(FULL, n1);
            if (m0 | m1) {
                const unsigned vote0 = __ballot_sync(FULL, (n0 || n1) && d0 <= d1);
                const bool first0 = m0 != 0u && (m1 == 0u || 2 * __popc(vote0) >= __popc(m0 | m1));
                if ((first0 ? m1 : m0) != 0u && sp < 32) {
                    stk[sp] = first0 ? 2 * node + 1 : 2 * node;
                    sd[sp] = first0 ? d1 : d0;
                    ++sp;
                }
                node = first0 ? 2 * node : 2 * node + 1;
                continue;
            }
        }
        node = 0;
        while (sp > 0) {
            --sp;
            if (__any_sync(FULL, active && sd[sp] <= bound)) {
                node = stk[sp];
                break;
            }
        }
    }
}

// Grid fast path.  Looks up the 2x2x2 block of grid cells around q (the octant of q's cell it
// lies in) and returns their point ranges in rng and the radius `cert` within which the block is
// exhaustive: every point outside it is at least cert from q (the distance from q to the block's
// faces, less a margin covering the float cell assignment of points).  Returns -1 without a grid.
__device__ __forceinline__ float grid_block8(const IndexView& ix, float4 qz, float q0, float q1, float q2, int2 rng[8])
{
#pragma unroll
    for (int c = 0; c < 8; ++c) rng[c] = make_int2(0, 0);
    if (!ix.grid_mask || !(qz.w > 0.f)) return -1.f;
    const float cellsz = 1.f / qz.w;
    const int bx = (int)floorf((q0 - qz.x) * qz.w - 0.5f);
    const int by = (int)floorf((q1 - qz.y) * qz.w - 0.5f);
    const int bz = (int)floorf((q2 - qz.z) * qz.w - 0.5f);
    const float lx = qz.x + bx * cellsz, ly = qz.y + by * cellsz, lz = qz.z + bz * cellsz;
    const float cert = fminf(fminf(fminf(q0 - lx, lx + 2.f * cellsz - q0), fminf(q1 - ly, ly + 2.f * cellsz - q1)),
                             fminf(q2 - lz, lz + 2.f * cellsz - q2)) - 1e-5f;
    uint32_t key[8];
    int4 e[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) {  // first probes of all eight cells in flight together
        const int ix_ = bx + (c & 1), iy = by + ((c >> 1) & 1), iz = bz + (c >> 2);
        const bool in = (unsigned)ix_ < 1024u && (unsigned)iy < 1024u && (unsigned)iz < 1024u;
        key[c] = in ? (spread10(ix_) << 2) | (spread10(iy) << 1) | spread10(iz) : GRID_EMPTY;
        e[c] = in ? ix.grid[grid_hash(key[c]) & ix.grid_mask] : make_int4(-1, 0, 0, 0);
    }
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        if (key[c] == GRID_EMPTY || (uint32_t)e[c].x == GRID_EMPTY) continue;
        rng[c] = (uint32_t)e[c].x == key[c] ? make_int2(e[c].y, e[c].z) : grid_find(ix.grid, ix.grid_mask, key[c]);
    }
    return cert;
}

}  // namespace gsicp
