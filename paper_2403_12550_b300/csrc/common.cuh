// common.cuh -- device-side building blocks shared by the libgsicp kernels.
//
// Spatial index: a bounding-volume hierarchy over points sorted along a
// Morton (Z-order) curve.  Points are cut into fixed-size buckets of B
// consecutive sorted points (the leaves); the tree over the L = 2^levels
// leaves is implicit (1-indexed heap: node i has children 2i, 2i+1, leaves
// are nodes L .. 2L-1).  Every node stores the exact axis-aligned bounding box
// of its points, so a box's squared distance to a query is a lower bound on
// the squared distance of every point inside it, computed with the same
// rounded operations (see sq3) -- pruning never drops an admissible point.
#pragma once

#include <stddef.h>

#include <cuda_runtime.h>
#include <stdint.h>

#define GSICP_INF __int_as_float(0x7f800000)

namespace gsicp {

// Interleave the low 10 bits of v with two zero bits between each.
__device__ __forceinline__ uint32_t spread10(uint32_t v)
{
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

// Sorted point record: x, y, z and the point's original index (int bits in w).
// Node box: two float4 per node, lo.xyz and hi.xyz (w unused).  Empty boxes
// have lo = +inf, hi = -inf, so their distance to any query is +inf.
struct IndexView {
    const float4* pts;    // L*B sorted points (only the first *n are valid)
    const float4* boxes;  // 2 * (2L) float4: node i -> boxes[2i] (lo), boxes[2i+1] (hi)
    const float4* covs;   // optional: 2 float4 per sorted point (xx,xy,xz,yy | yz,zz,-,-)
    const int* n;         // device count of valid points
    const uint32_t* keys; // sorted 30-bit Morton keys of the valid points (map indices only)
    const float4* quant;  // (lo.x, lo.y, lo.z, scale): Morton quantisation of this index
    const int4* grid;     // hash table of occupied grid cells (map indices only; null: no grid), see grid_find
    const uint32_t* grid_mask;  // device word: the table's live capacity - 1 (a power of two, sized on
                                // the device from the number of occupied cells)
    int L;                // leaves (power of two)
    int B;                // points per leaf (8, 16 or 32)
};

// Grid cells.  A map index quantises positions to cells of size 1/scale (the Morton grid), so
// the points of one cell are a contiguous run of the sorted array; the hash table maps a cell's
// 30-bit Morton key to that run: entries (key, start, end, -), empty slots have key 0xffffffff.
// Kernels of a dependent chain (the map-index build, a frame's a1 .. set-up) are launched as
// programmatic dependents of the kernel before them in their stream (launch_dependent,
// internal.h): a launch's set-up overlaps the end of the kernel before it, and its blocks wait
// here, at their first instruction, until that kernel has completed and its writes are visible (a
// no-op in a plain launch).  Nothing is read before the wait, so the work runs in the order of
// plain launches.
__device__ __forceinline__ void wait_prior_grid() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

constexpr uint32_t GRID_EMPTY = 0xffffffffu;

__device__ __forceinline__ uint32_t grid_hash(uint32_t key)
{
    uint32_t h = key * 2654435761u;
    return h ^ (h >> 16);
}

// [start, end) of the cell with this key (empty range if the cell holds no point), skipping the
// first probes_done slots of its probe sequence (a caller that has read the home slot passes 1).
__device__ __forceinline__ int2 grid_find(const int4* __restrict__ table, uint32_t mask, uint32_t key,
                                          uint32_t probes_done = 0)
{
    uint32_t slot = (grid_hash(key) + probes_done) & mask;
    for (uint32_t probe = probes_done; probe <= mask; ++probe) {
        const int4 e = table[slot];
        if ((uint32_t)e.x == key) return make_int2(e.y, e.z);
        if ((uint32_t)e.x == GRID_EMPTY) break;
        slot = (slot + 1) & mask;
    }
    return make_int2(0, 0);
}

// 30-bit Morton key of a point under the index's quantisation (clamped to the cube).
__device__ __forceinline__ uint32_t morton_of(float4 qz, float x, float y, float z)
{
    const uint32_t qx = (uint32_t)min(1023, max(0, (int)((x - qz.x) * qz.w)));
    const uint32_t qy = (uint32_t)min(1023, max(0, (int)((y - qz.y) * qz.w)));
    const uint32_t qq = (uint32_t)min(1023, max(0, (int)((z - qz.z) * qz.w)));
    return (spread10(qx) << 2) | (spread10(qy) << 1) | spread10(qq);
}

// Squared norm with a fixed, monotone evaluation order: used for both point
// and box distances so that box bounds are never above a contained point's
// distance after rounding.
__device__ __forceinline__ float sq3(float dx, float dy, float dz)
{
    return __fmaf_rn(dx, dx, __fmaf_rn(dy, dy, __fmul_rn(dz, dz)));
}

__device__ __forceinline__ float point_d2(float qx, float qy, float qz, float4 p)
{
    return sq3(__fsub_rn(p.x, qx), __fsub_rn(p.y, qy), __fsub_rn(p.z, qz));
}

__device__ __forceinline__ float box_d2(float qx, float qy, float qz, float4 lo, float4 hi)
{
    float dx = fmaxf(fmaxf(__fsub_rn(lo.x, qx), __fsub_rn(qx, hi.x)), 0.f);
    float dy = fmaxf(fmaxf(__fsub_rn(lo.y, qy), __fsub_rn(qy, hi.y)), 0.f);
    float dz = fmaxf(fmaxf(__fsub_rn(lo.z, qz), __fsub_rn(qz, hi.z)), 0.f);
    return sq3(dx, dy, dz);
}

// (d, i) strictly before (e, j) in the order "squared distance, then index".
__device__ __forceinline__ bool before(float d, int i, float e, int j)
{
    return d < e || (d == e && i < j);
}

// (squared distance, index) as one 64-bit key whose unsigned order is the order "distance, then
// index" (non-negative float bits order like unsigned integers).
__device__ __forceinline__ unsigned long long dkey(float d2, int i)
{
    return ((unsigned long long)__float_as_uint(d2) << 32) | (unsigned)i;
}
__device__ __forceinline__ float key_d2(unsigned long long k) { return __uint_as_float((unsigned)(k >> 32)); }
__device__ __forceinline__ int key_idx(unsigned long long k) { return (int)(unsigned)(k & 0xffffffffu); }

// Insert key k into the ascending list L of length K, dropping the last entry (the caller has
// checked k < L[K-1]); an optional companion array P is shifted along.  Each slot is compared
// with k independently and then shifted with selects: a few instructions deep, not K.
template <int K>
__device__ __forceinline__ void key_insert(unsigned long long (&L)[K], unsigned long long k)
{
    bool go[K];
#pragma unroll
    for (int j = 0; j < K; ++j) go[j] = k < L[j];
#pragma unroll
    for (int j = K - 1; j > 0; --j) L[j] = go[j - 1] ? L[j - 1] : (go[j] ? k : L[j]);
    L[0] = go[0] ? k : L[0];
}

template <int K>
__device__ __forceinline__ void key_insert(unsigned long long (&L)[K], int (&P)[K], unsigned long long k, int p)
{
    bool go[K];
#pragma unroll
    for (int j = 0; j < K; ++j) go[j] = k < L[j];
#pragma unroll
    for (int j = K - 1; j > 0; --j) {
        L[j] = go[j - 1] ? L[j - 1] : (go[j] ? k : L[j]);
        P[j] = go[j - 1] ? P[j - 1] : (go[j] ? p : P[j]);
    }
    L[0] = go[0] ? k : L[0];
    P[0] = go[0] ? p : P[0];
}

// Sum of counts[0 .. b), computed by the whole block (all threads get it): a block's offset in
// an order-preserving compaction whose per-block counts another launch wrote, read directly
// instead of through a separate scan (a few hundred words per block, from L2).
__device__ __forceinline__ uint32_t block_prefix(const uint32_t* __restrict__ counts, int b)
{
    __shared__ uint32_t red[32];
    uint32_t v = 0u;
    for (int i = threadIdx.x; i < b; i += blockDim.x) v += __ldcg(counts + i);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int nw = (blockDim.x + 31) >> 5;
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    uint32_t t = 0u;
    for (int w = 0; w < nw; ++w) t += red[w];
    __syncthreads();  // red may be reused by the caller's next call
    return t;
}

// A sorting network for N <= 32 keys: Batcher's merge exchange (Knuth, TAOCP vol. 3, 5.2.2,
// Algorithm M) as a compile-time list of compare-exchange pairs (97 for N = 20, 191 for N = 32).
struct SortNet {
    unsigned char a[256], b[256];
    int n;
};
constexpr SortNet make_sort_net(int N)
{
    SortNet net{};
    net.n = 0;
    int t = 0;
    while ((1 << t) < N) ++t;
    for (int p = t > 0 ? 1 << (t - 1) : 0; p > 0; p >>= 1) {
        int q = 1 << (t - 1), r = 0, d = p;
        for (;;) {
            for (int i = 0; i < N - d; ++i)
                if ((i & p) == r) {
                    net.a[net.n] = (unsigned char)i;
                    net.b[net.n] = (unsigned char)(i + d);
                    ++net.n;
                }
            if (q == p) break;
            d = q - p;
            q >>= 1;
            r = p;
        }
    }
    return net;
}
// Sorts L ascending in registers (every index a compile-time constant).
template <int N>
__device__ __forceinline__ void sort_keys(unsigned long long (&L)[N])
{
    static_assert(N >= 1 && N <= 32, "network sizes up to 32");
    constexpr SortNet net = make_sort_net(N);
#pragma unroll
    for (int c = 0; c < net.n; ++c) {
        const unsigned long long x = L[net.a[c]], y = L[net.b[c]];
        L[net.a[c]] = x < y ? x : y;
        L[net.b[c]] = x < y ? y : x;
    }
}

// Insert (d, i[, p]) into the list (D, I[, P]) of length K sorted by (distance, index), dropping
// the last entry; the caller has checked that the new entry precedes the last one.  Every slot is
// compared with the new entry independently and then shifted with selects, so the dependency
// chain is a few instructions deep instead of K compare-swaps long.
template <int K>
__device__ __forceinline__ void sorted_insert(float (&D)[K], int (&I)[K], float d, int i)
{
    bool go[K];
#pragma unroll
    for (int j = 0; j < K; ++j) go[j] = before(d, i, D[j], I[j]);
#pragma unroll
    for (int j = K - 1; j > 0; --j) {
        D[j] = go[j - 1] ? D[j - 1] : (go[j] ? d : D[j]);
        I[j] = go[j - 1] ? I[j - 1] : (go[j] ? i : I[j]);
    }
    D[0] = go[0] ? d : D[0];
    I[0] = go[0] ? i : I[0];
}

template <int K>
__device__ __forceinline__ void sorted_insert(float (&D)[K], int (&I)[K], int (&P)[K], float d, int i, int p)
{
    bool go[K];
#pragma unroll
    for (int j = 0; j < K; ++j) go[j] = before(d, i, D[j], I[j]);
#pragma unroll
    for (int j = K - 1; j > 0; --j) {
        D[j] = go[j - 1] ? D[j - 1] : (go[j] ? d : D[j]);
        I[j] = go[j - 1] ? I[j - 1] : (go[j] ? i : I[j]);
        P[j] = go[j - 1] ? P[j - 1] : (go[j] ? p : P[j]);
    }
    D[0] = go[0] ? d : D[0];
    I[0] = go[0] ? i : I[0];
    P[0] = go[0] ? p : P[0];
}


// Order-preserving map float -> uint32 (for atomicMin/atomicMax on floats).
__device__ __forceinline__ uint32_t f2ord(float f)
{
    uint32_t u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float ord2f(uint32_t u)
{
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

// ---------------------------------------------------------------------------------------------
// Compensated (double-float) summation: value = hi + lo with |lo| <= ulp(hi)/2.
struct dfloat {
    float hi, lo;
};
__device__ __forceinline__ void df_add(dfloat& a, float x)
{
    float s = __fadd_rn(a.hi, x);
    float bb = __fsub_rn(s, a.hi);
    float err = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(x, bb));
    a.hi = s;
    a.lo = __fadd_rn(a.lo, err);
}

// s + e == a + b exactly (s the rounded sum)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// a += (bhi + blo)
__device__ __forceinline__ void df_merge(dfloat& a, float bhi, float blo)
{
    df_add(a, bhi);
    a.lo = __fadd_rn(a.lo, blo);
}

// ---------------------------------------------------------------------------------------------
// Registration job and state (device memory, written by the host-side set-up
// kernel, read by every Gauss-Newton iteration).

struct Pose16 {
    double v[16];
};

enum { REG_MODE_SOLVE = 0, REG_MODE_LINEARISE = 1 };
enum { REG_ST_RUNNING = 0, REG_ST_CONVERGED = 1, REG_ST_MAXITER = 2, REG_ST_DEGENERATE = 3 };

constexpr int NACC = 30;  // 21 (upper triangle of H) + 6 (b) + cost + count + squared distances

struct RegState {
    double T[16];      // current pose
    double H[36];      // last linearisation
    double b[6];
    double cost;
    long long inliers;
    double sqdist;     // sum of the inliers' squared Euclidean residuals |mu - y|^2 (last linearisation)
    float Rf[9], tf[3];  // float copy of the current pose for the per-point work
    float Rlo[9], tlo[3];  // remainders: Rf + Rlo and tf + tlo carry the pose to ~48 bits
    int iter;          // completed iterations
    int status;        // REG_ST_*
    unsigned int counter;  // blocks finished in the current iteration
    int pad;
    // telemetry, per iteration (first REG_STATS iterations): points whose candidate cache was
    // rebuilt, and nanoseconds spent in the final reduction + solve by the last block
    int refreshes[64];
    int tail_ns[64];
    int solve_ns[64];                      // part of tail_ns spent in the FP64 solve + update
    unsigned long long t_first[64];        // earliest block start (globaltimer, ns)
    unsigned long long t_arrive[64];       // latest block arrival at the reduction
};
constexpr int REG_STATS = 64;
// bytes of RegState before its telemetry: what a registration copies back to the host
constexpr size_t REG_STATE_HEAD = offsetof(RegState, refreshes);

// Map candidates cached per source point.  Gauss-Newton time per 1200x680 frame with 4 / 8: 1.14 /
// 1.16 ms (a shorter list is built and checked faster and read in one 16-byte load; it certifies a
// smaller radius, so a few more caches expire).
constexpr int KC = 4;
static_assert(KC % 4 == 0, "the candidate cache is read and written as int4");

// A source point's cached candidate positions (KC ints at cand + KC s, 16-byte aligned), read
// through L2: in a persistent launch another SM wrote them in the last iteration.
__device__ __forceinline__ void cand_load(const int* cand, long s, int (&cp)[KC])
{
#pragma unroll
    for (int q = 0; q < KC / 4; ++q) {
        const int4 v = __ldcg(reinterpret_cast<const int4*>(cand) + (KC / 4) * s + q);
        cp[4 * q] = v.x;
        cp[4 * q + 1] = v.y;
        cp[4 * q + 2] = v.z;
        cp[4 * q + 3] = v.w;
    }
}
__device__ __forceinline__ void cand_store(int* cand, long s, const int (&P)[KC])
{
#pragma unroll
    for (int q = 0; q < KC / 4; ++q)
        reinterpret_cast<int4*>(cand)[(KC / 4) * s + q] = make_int4(P[4 * q], P[4 * q + 1], P[4 * q + 2], P[4 * q + 3]);
}
// only the first entry: a search without a cache (the rest is not read while the anchor says so,
// except the last entry as a hint of where to start a walk)
__device__ __forceinline__ void cand_store1(int* cand, long s, int p)
{
    reinterpret_cast<int4*>(cand)[(KC / 4) * s] = make_int4(p, -1, -1, -1);
}

// Gauss-Newton block: one source point per thread (a batched registration's work item is one
// block's worth of a pair's points), REG_BLOCKS_PER_SM blocks resident per SM (the kernels' launch
// bounds; 24 warps at 80 registers a thread).  Gauss-Newton time per 1200x680 frame measured for
// 64 / 128 / 256 / 384 threads: 1.73 / 1.61 / 1.53 / 1.51 ms.  384 would save about 1 % there but
// also makes the batched kernel's work items 1.5x larger, which is not measured; 256 is kept.
constexpr int REG_THREADS = 256;
constexpr int REG_BLOCKS_PER_SM = 768 / REG_THREADS;
static_assert(REG_THREADS % 32 == 0 && 768 % REG_THREADS == 0, "GN block: whole warps, 768 threads per SM");

// Gauss-Newton reduction (gicp.cu): block partial rows are summed in groups of GN_GROUP; a
// registration's reduction area holds its nrows rows (32 floats), the group rows (64 floats: hi,
// lo) and the group counters (one word each, zero between iterations).
constexpr int GN_GROUP = 32;
__host__ __device__ constexpr size_t reduction_floats(int nrows)
{
    return 32 * (size_t)nrows + 65 * (size_t)((nrows + GN_GROUP - 1) / GN_GROUP);
}

// Work queue of a batched registration (device memory, zeroed except as set by the host).
struct BatchQueue {
    unsigned int head;     // next slot to claim
    unsigned int tail;     // slots reserved so far
    unsigned int running;  // pairs not yet retired
    unsigned int error;    // a wait exceeded its bound
};

struct RegJob {
    const float4* src;     // source points in Morton order (x, y, z, original index), n
    const float4* covs_s;  // their covariances in the same order, 2 float4 each (xx,xy,xz,yy | yz,zz,-,-)
    const int* n;          // device count
    IndexView map;
    int* cand;             // n x KC: sorted map positions of each point's cached nearest map points (-1 none)
    float4* anchor;        // n: (query position of the last search, radius within which the cached
                           // candidates are complete); radius -1: searched without a cache, -2: never
                           // searched (cand[0] then holds a seed position or -1)
    int* corr_out;         // optional: original map index per source point
    float* partials;       // grid x NACC
    RegState* st;
    float max_d2;
    float slack;           // extra search radius beyond max_corr_dist kept in the cache (m)
    float cache_step;      // a point that moved more than this since its last search searches 1-NN only (m)
    int max_iters;
    double tol_rot, tol_trans;
    int min_inliers;
    int mode;              // REG_MODE_*
    int use_cond;          // 1 when launched inside the conditional-while graph
    int coop_max;          // warps with at most this many tree walks do them together (0: never)
    double* sums_out;      // optional: the NACC FP64 sums of each linearisation (shard registrations)
    int packet_iters;      // iterations (from the first) whose busy warps walk for their nearest points together
    int* sched;            // optional (single registrations): the iteration blocks' start order, kept
                           // from one iteration to the next (gicp.cu, sched_block); sched_ints(grid) ints
};

// Start order of a registration's iteration blocks: each block records which of SCHED_BUCKETS
// duration classes (4.1 us doubling) it fell in, and the next iteration starts its blocks slowest
// class first.  Layout: counts of the classes for even and odd iterations (8 ints each), then the
// lists of block indices per parity and class (grid ints each).
constexpr int SCHED_BUCKETS = 6;
__host__ __device__ constexpr size_t sched_ints(int grid) { return 16 + 2 * (size_t)SCHED_BUCKETS * grid; }

constexpr int COOP_WALKS_DEFAULT = 4;  // default RegJob::coop_max

}  // namespace gsicp
