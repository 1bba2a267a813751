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

constexpr int WARP_STACK = 256;  // entries of a warp's shared-memory walk stack

// Packet nearest-point walk: the warp walks the tree once for the nearest point of every lane with
// `active` set (all 32 lanes call it, converged).  The node stack is the warp's (shared memory,
// entries pushed by lane 0): a node is expanded when at least one active lane's bound reaches its
// box; an internal node's eight descendants three levels down are loaded by every lane (the same
// addresses: broadcast loads) and each active lane tests them against its own query and bound; a
// leaf's points are read the same way and each active lane offers them to its own best.  The warp
// pays for the union of its lanes' nodes instead of their divergent sum, which pays when the lanes'
// queries are close together and all search (the first iteration, where most points are ~2 cm off
// the map).  Exactness is the per-lane argument of traverse(): a node is skipped only when no
// active lane's bound reaches its box, and bounds only shrink.  Returns false (lane results
// unchanged since the call's start are still valid bounds, but incomplete) if the stack would
// overflow; the caller then walks each lane alone.  Leaves skip0 (per lane) were scanned by the
// caller.  offer(u, p) updates the calling lane's best with point u.
template <class OfferFn>
__device__ __forceinline__ bool packet_nn8(const IndexView& ix, int nmap, bool active, float qx, float qy, float qz,
                                           const float& bound, int skip0, int2* __restrict__ stk, OfferFn&& offer)
{
    constexpr unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int L = ix.L, B = ix.B;
    int sp = 0;
    if (lane == 0) {  // entry nodes: the 1, 2 or 4 nodes at depth (log2 L) mod 3
        const int first = 1 << ((31 - __clz(L)) % 3);
        for (int c = first; c < 2 * first; ++c) stk[sp++] = make_int2(c, 0);
    }
    sp = __shfl_sync(FULL, sp, 0);
    __syncwarp();
    while (sp > 0) {
        const int node = stk[sp - 1].x;
        --sp;
        const float4* bx = ix.boxes + 2 * node;
        const float dn = box_d2(qx, qy, qz, bx[0], bx[1]);
        if (__ballot_sync(FULL, active && dn <= bound) == 0u) continue;
        if (node >= L) {
            const int lf = node - L, beg = lf * B, end = min(beg + B, nmap);
            const bool mine = active && lf != skip0;
            for (int u0 = beg; u0 < end; u0 += 4) {
                float4 pp[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) pp[j] = u0 + j < end ? ix.pts[u0 + j] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (mine && u0 + j < end) offer(u0 + j, pp[j]);
            }
            continue;
        }
        // eight descendants three levels down: nodes 8 node .. 8 node + 7
        const float4* cb = ix.boxes + 16 * node;
        unsigned need = 0u;
        float dmin = GSICP_INF;
        int cmin = -1;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const float d = box_d2(qx, qy, qz, cb[2 * c], cb[2 * c + 1]);
            const bool ok = active && d <= bound;
            if (__ballot_sync(FULL, ok)) need |= 1u << c;
            if (ok && d < dmin) {
                dmin = d;
                cmin = c;
            }
        }
        if (need == 0u) continue;
        // the child nearest for most active lanes goes on top (visited first), the rest below it
        int top = -1, topn = 0;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int votes = __popc(__ballot_sync(FULL, cmin == c));
            if ((need >> c) & 1u && votes > topn) {
                topn = votes;
                top = c;
            }
        }
        if (top < 0) top = __ffs(need) - 1;
        if (sp + __popc(need) > WARP_STACK) return false;
        __syncwarp();
        if (lane == 0) {
#pragma unroll
            for (int c = 0; c < 8; ++c)
                if (((need >> c) & 1u) && c != top) stk[sp++] = make_int2(8 * node + c, 0);
            stk[sp++] = make_int2(8 * node + top, 0);
        }
        sp = __shfl_sync(FULL, sp, 0);
        __syncwarp();
    }
    return true;
}

// Warp-cooperative exact search for the kk (1 <= kk <= 32) nearest points of ONE query: all 32
// lanes call it, converged, with the same arguments.  The list of the kk smallest (squared
// distance, index) keys below lim_key is kept ascending in lanes 0 .. kk-1 (lane 0 may start with
// a known point at init_pos; the other entries start empty).  Leaves skip0 / skip1 (or -1) are
// scanned first and skipped by the walk.  The walk keeps its stack in shared memory (stk, WARP_STACK
// entries of (node, box distance bits)); each step takes up to four of the top entries whose box
// is still within the bound and gives each eight lanes: an internal node's eight descendants
// three levels down are box-tested and pushed, a leaf's points are read eight at a time and
// offered to the list.  A step thus costs one dependent memory round trip for up to 32 boxes or
// 32 points, where a single-thread walk pays one per node and one per four points.  Exactness is
// the argument of traverse(): a box is dropped only when its lower bound exceeds the current bound,
// which only shrinks.  Returns false, list incomplete, if the stack would overflow; the caller
// then searches this query alone.
__device__ __forceinline__ bool warp_knn(const IndexView& ix, int nmap, float qx, float qy, float qz, int kk,
                                         unsigned long long lim_key, int init_pos, int skip0, int skip1,
                                         int2* __restrict__ stk, unsigned long long& lkey, int& lpos)
{
    constexpr unsigned FULL = 0xffffffffu;
    constexpr unsigned long long NONE = ~0ull;
    const int lane = threadIdx.x & 31, slot = lane >> 3, sub = lane & 7;
    const unsigned below = (1u << lane) - 1u;
    const int L = ix.L, B = ix.B;
    lkey = lim_key;
    lpos = lane == 0 ? init_pos : -1;
    unsigned long long kth = lim_key;  // list entry kk-1 (every lane)
    // offer one candidate key per lane (NONE: none) to the list, one accepted key at a time
    auto offer = [&](unsigned long long ck, int cpos) {
        unsigned m = __ballot_sync(FULL, ck < kth);
        while (m != 0u) {
            const int src = __ffs(m) - 1;
            const unsigned long long k = __shfl_sync(FULL, ck, src);
            const int p = __shfl_sync(FULL, cpos, src);
            const unsigned long long up = __shfl_up_sync(FULL, lkey, 1);
            const int upp = __shfl_up_sync(FULL, lpos, 1);
            if (lane < kk && k < lkey) {
                const bool here = lane == 0 || up < k;
                lkey = here ? k : up;
                lpos = here ? p : upp;
            }
            kth = __shfl_sync(FULL, lkey, kk - 1);
            if (lane == src) ck = NONE;
            m = __ballot_sync(FULL, ck < kth);
        }
    };
    // the points of leaf lf (or none for lf < 0) handled by this lane: sub, sub + 8, ... < B
    auto scan_leaf = [&](int lf) {
        unsigned long long ck[4];
        int cu[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int u = lf * B + sub + 8 * r;
            const bool ok = lf >= 0 && 8 * r < B && u < nmap;
            const float4 p = ok ? __ldg(ix.pts + u) : make_float4(0.f, 0.f, 0.f, 0.f);
            ck[r] = ok ? dkey(point_d2(qx, qy, qz, p), __float_as_int(p.w)) : NONE;
            cu[r] = u;
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) offer(ck[r], cu[r]);
    };
    scan_leaf(slot == 0 ? skip0 : (slot == 1 ? skip1 : -1));
    // entry nodes: the 1, 2 or 4 nodes at depth (log2 L) mod 3, from which 8-way steps reach the leaves
    int sp;
    {
        const int first = 1 << ((31 - __clz(L)) % 3);
        float d = GSICP_INF;
        if (lane < first) d = box_d2(qx, qy, qz, ix.boxes[2 * (first + lane)], ix.boxes[2 * (first + lane) + 1]);
        const bool push = lane < first && d <= key_d2(kth);
        const unsigned pm = __ballot_sync(FULL, push);
        if (push) stk[__popc(pm & below)] = make_int2(first + lane, __float_as_int(d));
        sp = __popc(pm);
        __syncwarp();
    }
    while (sp > 0) {
        const float bound = key_d2(kth);
        // the top eight entries (lane 0 = top); live ones are still within the bound
        const int rd = min(8, sp);
        const int2 e = lane < rd ? stk[sp - 1 - lane] : make_int2(0, __float_as_int(GSICP_INF));
        const unsigned live = __ballot_sync(FULL, lane < rd && __int_as_float(e.y) <= bound);
        // take the first four live entries; entries above the last one taken are consumed
        unsigned rest = live;
#pragma unroll
        for (int i = 0; i < 4; ++i) rest &= rest - 1u;
        const unsigned take = live & ~rest;
        sp -= rest != 0u ? 32 - __clz(take) : rd;
        unsigned mine = take;  // this slot's entry: the slot-th set bit of take
#pragma unroll
        for (int i = 0; i < 3; ++i)
            if (i < slot) mine &= mine - 1u;
        int node = __shfl_sync(FULL, e.x, mine != 0u ? __ffs(mine) - 1 : 0);
        if (mine == 0u) node = 0;
        __syncwarp();  // reads of the popped entries before the pushes below overwrite them
        bool push = false;
        int child = 0;
        float d = GSICP_INF;
        int lf = -1;
        if (node != 0 && node < L) {
            child = 8 * node + sub;
            d = box_d2(qx, qy, qz, __ldg(ix.boxes + 2 * child), __ldg(ix.boxes + 2 * child + 1));
            push = d <= bound;
        } else if (node >= L) {
            lf = node - L;
            if (lf == skip0 || lf == skip1) lf = -1;
        }
        const unsigned pm = __ballot_sync(FULL, push);
        if (sp + __popc(pm) > WARP_STACK) return false;
        if (push) stk[sp + __popc(pm & below)] = make_int2(child, __float_as_int(d));
        sp += __popc(pm);
        if (__any_sync(FULL, lf >= 0)) scan_leaf(lf);
        __syncwarp();  // pushes visible to the next step's reads
    }
    return true;
}

// Grid fast path.  Looks up the 2x2x2 block of grid cells around q (the octant of q's cell it
// lies in) and returns their point ranges in rng and the radius `cert` within which the block is
// exhaustive: every point outside it is at least cert from q (the distance from q to the block's
// faces, less a margin covering the float cell assignment of points).  Returns -1 without a grid.
__device__ __forceinline__ float grid_block8(const IndexView& ix, float4 qz, float q0, float q1, float q2, int2 rng[8])
{
#pragma unroll
    for (int c = 0; c < 8; ++c) rng[c] = make_int2(0, 0);
    if (!ix.grid || !(qz.w > 0.f)) return -1.f;
    const uint32_t mask = *ix.grid_mask;
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
        e[c] = in ? ix.grid[grid_hash(key[c]) & mask] : make_int4(-1, 0, 0, 0);
    }
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        if (key[c] == GRID_EMPTY || (uint32_t)e[c].x == GRID_EMPTY) continue;
        // the home slot holds another cell: go on probing after it
        rng[c] = (uint32_t)e[c].x == key[c] ? make_int2(e[c].y, e[c].z) : grid_find(ix.grid, mask, key[c], 1u);
    }
    return cert;
}

}  // namespace gsicp
