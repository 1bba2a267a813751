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

}  // namespace gsicp
