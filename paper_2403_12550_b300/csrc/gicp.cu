// gicp.cu -- a5-a7: Gauss-Newton G-ICP registration against the map index.
//
// Sec. 3: with correspondences from nearest-neighbour search, the error
// d_i = x^t_i - T x^s_i is Gaussian with covariance C^t_i + T C^s_i T^T (only
// the rotation acts on a covariance), and the pose is the MLE of Eq.
// (MLE_for_T): argmin_T sum_i d_i^T (C^t_i + R C^s_i R^T)^-1 d_i.  It is
// minimised by Gauss-Newton with left perturbations T <- exp(xi^) T,
// xi = (omega, v): J_i = dd_i/dxi = [[y_i]x, -I] with y_i = R x_i + t.
//
// One kernel launch per iteration (chained by programmatic dependent launch, four per pass of a
// conditional-while CUDA graph).  One thread per source point, points in
// the source index's Morton order: transform, exact nearest map mean, then the
// residual, weight, J^T W J (21 unique), J^T W d (6), d^T W d and the inlier
// count -> warp shuffles -> one FP32 partial per block.  The last block to
// finish (threadfence + atomic counter, no waiting) sums the partials with
// compensation; its first warp solves the 6x6 system by FP64 Cholesky, applies
// the FP64 SE(3) exponential (both spread over the warp's lanes) and, inside a
// CUDA graph, sets the conditional-while handle that decides whether the next
// iteration runs.
//
// Nearest-neighbour search with a per-point candidate cache: each point keeps
// its KC nearest map points within max_corr_dist + slack and the radius within
// which that list is complete, measured from where the point was when the list
// was made.  Once the point has moved by delta, no map point outside the list
// can be closer than radius - delta, so when the best cached candidate is
// within that (with float-rounding margins) it is the exact answer and the
// tree is not walked; otherwise the list is rebuilt: from the 2x2x2 block of
// map-grid cells around the point when the block certifies it, else by an
// exact walk of the map's bounding-volume hierarchy (traverse.cuh) bounded by
// what the block found.  The first iteration starts from a Morton-key seed.
#include <algorithm>

#include "internal.h"
#include "traverse.cuh"

namespace gsicp {

constexpr int GN_BODY_ITERS = 4;  // iteration launches per pass of the conditional-while graph

// Exact nearest point of `ix` to q with (d2, original index) lexicographically
// smallest among points with d2 <= the incoming (best_d2, best_oi): an 8-wide walk (a third of the
// dependent round trips of a binary one), leaf points four loads at a time.
__device__ __forceinline__ void nn_search(const IndexView& ix, int n, float qx, float qy, float qz, float& best_d2,
                                          int& best_oi, int& best_pos)
{
    const int B = ix.B;
    traverse8(ix, qx, qy, qz, best_d2, [&](int lf) {
        scan_points4(ix.pts, lf * B, min(lf * B + B, n), [&](int u, const float4& p) {
            const float d2 = point_d2(qx, qy, qz, p);
            const int oi = __float_as_int(p.w);
            if (before(d2, oi, best_d2, best_oi)) {
                best_d2 = d2;
                best_oi = oi;
                best_pos = u;
            }
        });
    });
}

// Index of (r, c), r <= c, in the row-major upper triangle of a 6x6 matrix.
__host__ __device__ constexpr int ut(int r, int c) { return r * 6 - (r * (r - 1)) / 2 + (c - r); }

// ---------------------------------------------------------------------------------------------
// FP64 6x6 solve and SE(3) exponential, spread over the lanes of one warp.  FP64 arithmetic is
// slow on this part and a warp instruction costs as much with one active lane as with 32, so
// each step below is one instruction over every entry it updates.

// Lane p < 27 holds entry (i, j) of the augmented matrix [H ; r^T] (7 rows, 6 columns): the
// lower triangle of H in packed row order (p < 21), then r (p = 21 + j).
__device__ __forceinline__ void chol_lane_coords(int p, int& i, int& j)
{
    if (p >= 21) {
        i = 6;
        j = p - 21;
        return;
    }
    i = 0;
    while ((i + 1) * (i + 2) / 2 <= p) ++i;
    j = p - i * (i + 1) / 2;
}
__device__ __forceinline__ int chol_lane(int i, int j) { return i == 6 ? 21 + j : i * (i + 1) / 2 + j; }

// Solves H x = r by the Cholesky factorisation H = L L^T.  Factorising [H ; r^T] leaves the
// forward substitution L^-1 r in its last row; back substitution follows.  On entry lane p holds
// entry p (see chol_lane_coords); every lane returns the same x.  Returns false on every lane
// when a pivot is not positive (H not positive definite).
__device__ bool warp_chol_solve6(double a, int lane, double x[6])
{
    constexpr unsigned FULL = 0xffffffffu;
    int li = 0, lj = 0;
    const bool holds = lane < 27;
    if (holds) chol_lane_coords(lane, li, lj);
    double inv[6];  // 1 / L(j, j)
#pragma unroll
    for (int j = 0; j < 6; ++j) {
        const double d = __shfl_sync(FULL, a, chol_lane(j, j));
        if (!(d > 0.0) || !isfinite(d)) return false;
        inv[j] = rsqrt(d);
        if (holds && lj == j && li > j) a *= inv[j];  // column j of L
        // trailing update: a(i, k) -= L(i, j) L(k, j) for j < k <= i
        const bool upd = holds && lj > j;
        const double lij = __shfl_sync(FULL, a, upd ? chol_lane(li, j) : lane);
        const double lkj = __shfl_sync(FULL, a, upd ? chol_lane(lj, j) : lane);
        if (upd) a = fma(-lij, lkj, a);
    }
    // L^T x = y, y_j on lane 21 + j
    double y = a;
    const int jj = lane - 21;
#pragma unroll
    for (int i = 5; i >= 0; --i) {
        x[i] = __shfl_sync(FULL, y, 21 + i) * inv[i];
        const bool upd = jj >= 0 && jj < i;
        const double lij = __shfl_sync(FULL, a, upd ? chol_lane(i, jj) : lane);
        if (upd) y = fma(-lij, x[i], y);
    }
    return true;
}

// Taylor coefficients in t^2 of sin(t)/t, (1 - cos t)/t^2 and (t - sin t)/t^3:
// (-1)^m / (2m + o)!, o = 1, 2, 3.  Nine terms leave a remainder below 1e-22 for t < 0.5.
constexpr int EXP_TERMS = 9;
static_assert(EXP_TERMS == 9, "the exponential's series is evaluated as a degree-8 polynomial (Estrin)");
constexpr double inv_factorial(int k)
{
    double f = 1.0;
    for (int q = 2; q <= k; ++q) f *= q;
    return 1.0 / f;
}
#define GSICP_SERIES(o)                                                                                  \
    {inv_factorial(o), -inv_factorial(o + 2), inv_factorial(o + 4), -inv_factorial(o + 6),              \
     inv_factorial(o + 8), -inv_factorial(o + 10), inv_factorial(o + 12), -inv_factorial(o + 14),       \
     inv_factorial(o + 16)}
__constant__ double c_exp_series[3][EXP_TERMS] = {GSICP_SERIES(1), GSICP_SERIES(2), GSICP_SERIES(3)};
#undef GSICP_SERIES

// T <- exp(xi^) T with xi = (omega, v) the same on every lane: the rotation by Rodrigues'
// formula E = I + A K + B K^2 and the translation V v with V = I + B K + C K^2 (K = [omega]x,
// A = sin t / t, B = (1 - cos t) / t^2, C = (t - sin t) / t^3, t = |omega|).  Lane 4r + c < 12
// returns the new T(r, c); Tc holds T(0, c), T(1, c), T(2, c) for the lane's c = lane mod 4 (the
// pose is row-major 4x4 with last row 0 0 0 1).
__device__ double warp_se3_left_update(const double xi[6], const double (&Tc)[3], int lane)
{
    constexpr unsigned FULL = 0xffffffffu;
    const double w0 = xi[0], w1 = xi[1], w2 = xi[2];
    auto wsel = [&](int i) { return i == 0 ? w0 : (i == 1 ? w1 : w2); };
    const double th2 = fma(w0, w0, fma(w1, w1, w2 * w2));
    double A, Bc, Cc;
    if (th2 < 0.25) {
        const int o = min(lane, 2);  // lanes 0, 1, 2 evaluate A, B, C
        // the degree-8 polynomial in t^2 by Estrin's scheme: four dependent steps instead of eight
        const double* c = c_exp_series[o];
        const double x2 = th2 * th2, x4 = x2 * x2, x8 = x4 * x4;
        const double p01 = fma(c[1], th2, c[0]), p23 = fma(c[3], th2, c[2]);
        const double p45 = fma(c[5], th2, c[4]), p67 = fma(c[7], th2, c[6]);
        const double f = fma(c[8], x8, fma(fma(p67, x2, p45), x4, fma(p23, x2, p01)));
        A = __shfl_sync(FULL, f, 0);
        Bc = __shfl_sync(FULL, f, 1);
        Cc = __shfl_sync(FULL, f, 2);
    } else {
        const double th = sqrt(th2), ith2 = 1.0 / th2;
        double sn, cs;
        sincos(th, &sn, &cs);
        A = sn / th;
        Bc = (1.0 - cs) * ith2;
        Cc = (1.0 - A) * ith2;
    }
    // lane 3r + c (< 9): entries (r, c) of E and V, and V(r, c) v_c
    const int r = min(lane / 3, 2), c = lane % 3;
    const double k = c == r ? 0.0 : ((c - r + 3) % 3 == 1 ? -wsel(3 - r - c) : wsel(3 - r - c));
    const double k2 = fma(wsel(r), wsel(c), r == c ? -th2 : 0.0);  // K^2 = w w^T - t^2 I
    const double id = r == c ? 1.0 : 0.0;
    const double E = fma(A, k, fma(Bc, k2, id));
    const double V = fma(Bc, k, fma(Cc, k2, id));
    const double p = V * (c == 0 ? xi[3] : (c == 1 ? xi[4] : xi[5]));
    const double p1 = __shfl_down_sync(FULL, p, 1), p2 = __shfl_down_sync(FULL, p, 2);
    const double Vv = p + p1 + p2;  // lane 3r: (V v)_r
    // lane 4r + c (< 12): new T(r, c) = sum_k E(r, k) T(k, c) (+ (V v)_r for c = 3)
    const int tr = min(lane >> 2, 2), tc = lane & 3;
    const double e0 = __shfl_sync(FULL, E, 3 * tr), e1 = __shfl_sync(FULL, E, 3 * tr + 1),
                 e2 = __shfl_sync(FULL, E, 3 * tr + 2);
    const double tv = __shfl_sync(FULL, Vv, 3 * tr);
    return fma(e0, Tc[0], fma(e1, Tc[1], fma(e2, Tc[2], tc == 3 ? tv : 0.0)));
}

__device__ __forceinline__ void pose_to_float(RegState* st)
{
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c) {
            const double v = st->T[4 * r + c];
            st->Rf[3 * r + c] = (float)v;
            st->Rlo[3 * r + c] = (float)(v - (double)(float)v);
        }
        const double v = st->T[4 * r + 3];
        st->tf[r] = (float)v;
        st->tlo[r] = (float)(v - (double)(float)v);
    }
}

// One coordinate of y = R x + t with R, t given as float pairs (hi + lo): the products of the
// hi parts are split exactly (fmaf), their sum is carried with its rounding errors (two_sum),
// and the lo parts and the errors are added in float.  Returns y as hi + lo, accurate to about
// 1e-13 relative, so that distances and residuals taken as (p - hi) - lo match the FP64 ones.
__device__ __forceinline__ void transform_df(const float* Rh, const float* Rl, float th, float tl, float x0,
                                             float x1, float x2, float& hi, float& lo)
{
    const float p0 = __fmul_rn(Rh[0], x0), p1 = __fmul_rn(Rh[1], x1), p2 = __fmul_rn(Rh[2], x2);
    const float e0 = fmaf(Rh[0], x0, -p0), e1 = fmaf(Rh[1], x1, -p1), e2 = fmaf(Rh[2], x2, -p2);
    float s, c0, c1, c2;
    two_sum(th, p0, s, c0);
    two_sum(s, p1, s, c1);
    two_sum(s, p2, s, c2);
    const float low = fmaf(Rl[0], x0, fmaf(Rl[1], x1, fmaf(Rl[2], x2, tl))) + ((e0 + e1) + (e2 + c0)) + (c1 + c2);
    hi = __fadd_rn(s, low);
    lo = __fsub_rn(low, __fsub_rn(hi, s));
}

// ---------------------------------------------------------------------------------------------

__global__ void reg_setup_kernel(RegJob job, RegJob* __restrict__ job_dst, RegState* __restrict__ st, Pose16 T0)
{
    wait_prior_grid();
    *job_dst = job;
    if (job.sched)  // no history: the first iteration starts its blocks in index order
        for (int i = 0; i < 16; ++i) job.sched[i] = 0;
    for (int i = 0; i < 16; ++i) st->T[i] = T0.v[i];
    for (int i = 0; i < 36; ++i) st->H[i] = 0.0;
    for (int i = 0; i < 6; ++i) st->b[i] = 0.0;
    st->cost = 0.0;
    st->sqdist = 0.0;
    st->inliers = 0;
    st->iter = 0;
    st->status = REG_ST_RUNNING;
    st->counter = 0u;
    for (int i = 0; i < REG_STATS; ++i) {
        st->refreshes[i] = st->tail_ns[i] = st->solve_ns[i] = 0;
        st->t_first[i] = ~0ull;
        st->t_arrive[i] = 0ull;
    }
    pose_to_float(st);
}

// All the Gauss-Newton work for source point s of job J at the float pose (R, t) + (Rl, tl):
// transform, exact nearest map point (cache / grid / tree), residual, weight and J^T W J, J^T W d,
// d^T W d and the inlier count added to acc.  Called by all 32 lanes of a warp, converged (lanes
// with active == false hold no point); wstack is the warp's stack for cooperative walks.
// Returns 1 if the point's nearest-point search ran (its cache was rebuilt).
//
// Tree walks: in a warp where at most J.coop_max points need one, the whole warp walks for each of
// them in turn (warp_knn); in busier warps each point walks alone.  A lone walk of a point far from
// the map is a long chain of dependent loads, and in the late iterations, where a handful of points
// per launch still search, that chain sets the launch's duration.  Both walks are exact, so every
// choice returns the same nearest point and leaves the same cache state.
__device__ __forceinline__ int gn_point(const RegJob& J, const float (&R)[9], const float (&Rl)[9],
                                        const float (&t)[3], const float (&tl)[3], int s, bool active, int nmap,
                                        float (&acc)[NACC], int2* wstack, bool packet)
{
    constexpr unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    int refreshed = 0;
    const float4 qq = *J.map.quant;
    const int B = J.map.B;
    const float max_d = sqrtf(J.max_d2);
    const float Rs = max_d + J.slack, Rs2 = Rs * Rs;
    float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
    float y0 = 0.f, y1 = 0.f, y2 = 0.f, l0 = 0.f, l1 = 0.f, l2 = 0.f;
    float best_d2 = J.max_d2;
    int best_oi = 0x7fffffff, best_pos = -1;
    int walk = 0;     // a tree walk is still needed: 1 nearest point only, 2 the KC nearest within lim
    float lim = 0.f;  // walk 2: squared search radius
    int h0 = -1, h1 = -1;  // leaves of the previous candidates, scanned first by a walk
    auto exact_d2 = [&](const float4& p) {
        return sq3(__fsub_rn(__fsub_rn(p.x, y0), l0), __fsub_rn(__fsub_rn(p.y, y1), l1),
                   __fsub_rn(__fsub_rn(p.z, y2), l2));
    };
    // Nearest-point searches choose by the hi + lo distance but prune boxes with distances from
    // hi: a point whose hi + lo distance is below d is within d + |lo| + rounding of hi, so a walk
    // bounded by the inflated square wb(d^2) drops no point that could still win.  |lo| is at most
    // half an ulp of hi per coordinate (|y| 2^-24 each, sqrt 3 |y| 2^-24 in all); the rest covers
    // the float rounding of the distances (a few ulps, relative).
    float ymag = 0.f;
    auto walk_bound = [&](float d2) {
        const float d = sqrtf(d2) * (1.f + 1e-6f) + ymag * 2.4e-7f + 1e-9f;
        return d * d;
    };
    // the nearest by hi + lo among a sorted KC list (positions P, -1 = none)
    auto pick_exact = [&](const int (&P)[KC]) {
        best_d2 = J.max_d2;
        best_oi = 0x7fffffff;
        best_pos = -1;
#pragma unroll
        for (int j = 0; j < KC; ++j) {
            if (P[j] < 0) continue;
            const float4 p = J.map.pts[P[j]];
            const float ed2 = exact_d2(p);
            const int oi = __float_as_int(p.w);
            if (before(ed2, oi, best_d2, best_oi)) {
                best_d2 = ed2;
                best_oi = oi;
                best_pos = P[j];
            }
        }
    };
    if (active) {
        x = J.src[s];
        // y = R x + t as hi + lo: the searches run on hi; the final choice among the candidates
        // they return, the inlier test and the residual use hi + lo (distance differences at the
        // level of float rounding of y would otherwise flip near-equidistant correspondences)
        transform_df(R, Rl, t[0], tl[0], x.x, x.y, x.z, y0, l0);
        transform_df(R + 3, Rl + 3, t[1], tl[1], x.x, x.y, x.z, y1, l1);
        transform_df(R + 6, Rl + 6, t[2], tl[2], x.x, x.y, x.z, y2, l2);
        ymag = fmaxf(fabsf(y0), fmaxf(fabsf(y1), fabsf(y2)));
        // cache state through L2: in a persistent launch another SM wrote it in the last iteration
        int cp[KC];
        cand_load(J.cand, s, cp);
        const float4 anc = __ldcg(J.anchor + s);
        bool resolved = false;
        if (anc.w > 0.f) {
            // Cached candidates were complete within radius anc.w of the anchor; the query has
            // moved by delta, so every map point outside them is at least anc.w - delta away.
            float e_d2 = J.max_d2;
            int e_oi = 0x7fffffff, e_pos = -1;
#pragma unroll
            for (int j = 0; j < KC; ++j) {
                if (cp[j] < 0) continue;
                const float4 p = J.map.pts[cp[j]];
                const float d2 = point_d2(y0, y1, y2, p);
                const int oi = __float_as_int(p.w);
                if (before(d2, oi, best_d2, best_oi)) {
                    best_d2 = d2;
                    best_oi = oi;
                    best_pos = cp[j];
                }
                const float ed2 = exact_d2(p);
                if (before(ed2, oi, e_d2, e_oi)) {
                    e_d2 = ed2;
                    e_oi = oi;
                    e_pos = cp[j];
                }
            }
            const float delta = sqrtf(sq3(y0 - anc.x, y1 - anc.y, y2 - anc.z)) + 2e-6f + ymag * 4.8e-7f;
            const float bnd = best_pos >= 0 ? sqrtf(best_d2) : max_d;
            // margins (1e-5 relative; 2e-6 m plus twice the largest hi-to-(hi + lo) distance,
            // sqrt 3 |y| 2^-24, on each side) exceed the float rounding of the distances, so the
            // nearest point is among the cached ones by either distance
            resolved = anc.w - delta >= bnd * (1.f + 1e-5f);
            // the nearest by hi + lo among the cached points: the answer if resolved, else where the
            // search below starts (it chooses by hi + lo too)
            best_d2 = e_d2;
            best_oi = e_oi;
            best_pos = e_pos;
        }
        if (!resolved) {
            refreshed = 1;
            // A point that moved more than cache_step since its last search will likely move that
            // much again: search its nearest point only (a cache built now would not survive).
            const bool one_nn = !(anc.w != -2.f &&
                                  sq3(y0 - anc.x, y1 - anc.y, y2 - anc.z) < J.cache_step * J.cache_step);
            // Grid fast path: the 2x2x2 block of map cells around y (the octant of y's cell it lies
            // in).  Every map point outside the block is at least `cert` from y: the distance to the
            // block's faces less a margin for the float cell assignment of the points.
            int2 rng[8];
            const float cert = grid_block8(J.map, qq, y0, y1, y2, rng);
            const float cert2 = cert > 0.f ? cert * cert * (1.f - 2e-5f) : -1.f;
            h0 = cp[0] >= 0 ? cp[0] / B : -1;
            if (one_nn) {
                // the pose is still moving a lot: only the nearest point, no cache
                if (cert2 > 0.f) {
#pragma unroll
                    for (int c = 0; c < 8; ++c)
                        scan_points4(J.map.pts, rng[c].x, rng[c].y, [&](int u, const float4& p) {
                            const float d2 = exact_d2(p);
                            const int oi = __float_as_int(p.w);
                            if (before(d2, oi, best_d2, best_oi)) {
                                best_d2 = d2;
                                best_oi = oi;
                                best_pos = u;
                            }
                        });
                }
                // certified when the best is nearer than the block's faces: cert already holds a
                // margin (1e-5 m) far above |lo|
                if (!(best_pos >= 0 && best_d2 <= cert2)) {
                    walk = 1;
                } else {
                    cand_store1(J.cand, s, best_pos);
                    J.anchor[s] = make_float4(y0, y1, y2, -1.f);  // position of this search, no cache
                }
            } else {
                // exact KC nearest map points, grid block first, else a tree walk within Rs
                unsigned long long Lk[KC];  // ascending (squared distance, index) keys
                int P[KC];                  // their sorted map positions
#pragma unroll
                for (int j = 0; j < KC; ++j) {
                    Lk[j] = dkey(GSICP_INF, 0x7fffffff);
                    P[j] = -1;
                }
                if (cert2 > 0.f) {
#pragma unroll
                    for (int c = 0; c < 8; ++c)
                        scan_points4(J.map.pts, rng[c].x, rng[c].y, [&](int u, const float4& p) {
                            const unsigned long long key = dkey(point_d2(y0, y1, y2, p), __float_as_int(p.w));
                            if (key < Lk[KC - 1]) key_insert(Lk, P, key, u);
                        });
                }
                if (key_idx(Lk[0]) != 0x7fffffff && key_d2(Lk[0]) <= cert2) {
                    // points outside the list: outside the block (>= cert) or beaten by the KC-th
                    const float rc =
                        fminf(cert, key_idx(Lk[KC - 1]) != 0x7fffffff ? sqrtf(key_d2(Lk[KC - 1])) : GSICP_INF) *
                        (1.f - 1e-6f);
                    cand_store(J.cand, s, P);
                    J.anchor[s] = make_float4(y0, y1, y2, rc);
                    pick_exact(P);
                } else {
                    walk = 2;
                    lim = key_idx(Lk[KC - 1]) != 0x7fffffff ? fminf(key_d2(Lk[KC - 1]), Rs2) : Rs2;
                    h1 = (cp[KC - 1] >= 0 && cp[KC - 1] / B != h0) ? cp[KC - 1] / B : -1;
                }
            }
        }
    }
    // Tree walks.  Few in this warp: all lanes walk for each of them in turn.
    unsigned pend = __ballot_sync(FULL, walk != 0);
    if (pend != 0u && __popc(pend) <= J.coop_max) {
        while (pend != 0u) {
            const int o = __ffs(pend) - 1;
            pend &= pend - 1u;
            const int mode = __shfl_sync(FULL, walk, o);
            const float q0 = __shfl_sync(FULL, y0, o), q1 = __shfl_sync(FULL, y1, o),
                        q2 = __shfl_sync(FULL, y2, o);
            // a nearest-point walk collects the KC nearest by hi within the inflated bound of the
            // best so far, and both kinds choose among their list by hi + lo
            const unsigned long long lk = __shfl_sync(FULL, dkey(walk == 1 ? walk_bound(best_d2) : lim, 0x7fffffff), o);
            const int k0 = __shfl_sync(FULL, h0, o), k1 = __shfl_sync(FULL, h1, o);
            const int so = __shfl_sync(FULL, s, o);
            unsigned long long key;
            int pos;
            if (!warp_knn(J.map, nmap, q0, q1, q2, KC, lk, -1, k0, k1, wstack, key, pos))
                continue;  // stack overflow: lane o walks alone below
            // the nearest by hi + lo among the list: lane j < KC tests entry j
            const float m0 = __shfl_sync(FULL, l0, o), m1 = __shfl_sync(FULL, l1, o), m2 = __shfl_sync(FULL, l2, o);
            unsigned long long ek = ~0ull;
            if (lane < KC && pos >= 0) {
                const float4 p = J.map.pts[pos];
                const float ed2 = sq3(__fsub_rn(__fsub_rn(p.x, q0), m0), __fsub_rn(__fsub_rn(p.y, q1), m1),
                                      __fsub_rn(__fsub_rn(p.z, q2), m2));
                const int oi = __float_as_int(p.w);
                if (before(ed2, oi, J.max_d2, 0x7fffffff)) ek = dkey(ed2, oi);
            }
            int ep = pos;
#pragma unroll
            for (int off = 1; off < KC; off <<= 1) {
                const unsigned long long ok = __shfl_xor_sync(FULL, ek, off);
                const int op = __shfl_xor_sync(FULL, ep, off);
                if (ok < ek) {
                    ek = ok;
                    ep = op;
                }
            }
            ek = __shfl_sync(FULL, ek, 0);
            ep = ek != ~0ull ? __shfl_sync(FULL, ep, 0) : -1;
            if (mode == 2) {
                const unsigned long long klast = __shfl_sync(FULL, key, KC - 1);
                const float rc = (key_idx(klast) != 0x7fffffff ? sqrtf(key_d2(klast)) : Rs) * (1.f - 1e-6f);
                if (lane < KC) J.cand[(long)KC * so + lane] = pos;
                if (lane == 0) J.anchor[so] = make_float4(q0, q1, q2, rc);
            } else if (lane == 0) {
                cand_store1(J.cand, so, ep);
                J.anchor[so] = make_float4(q0, q1, q2, -1.f);  // position of this search, no cache
            }
            if (lane == o) {
                walk = 0;
                best_d2 = ek != ~0ull ? key_d2(ek) : J.max_d2;
                best_oi = ek != ~0ull ? key_idx(ek) : 0x7fffffff;
                best_pos = ep;
            }
        }
    }
    // Many in this warp, all after their nearest point, in an iteration that walks in packets: the
    // warp walks once for all of them (each lane first scans its own previous or seed leaf).
    if (packet && __popc(__ballot_sync(FULL, walk != 0)) > J.coop_max && !__any_sync(FULL, walk == 2)) {
        const bool mine = walk == 1;
        float wb = walk_bound(best_d2);
        auto offer = [&](int u, const float4& p) {
            const float d2 = exact_d2(p);
            const int oi = __float_as_int(p.w);
            if (before(d2, oi, best_d2, best_oi)) {
                best_d2 = d2;
                best_oi = oi;
                best_pos = u;
                wb = walk_bound(d2);
            }
        };
        if (mine && h0 >= 0)
            scan_points4(J.map.pts, h0 * B, min(h0 * B + B, nmap), [&](int u, const float4& p) { offer(u, p); });
        if (packet_nn8(J.map, nmap, mine, y0, y1, y2, wb, mine ? h0 : -1, wstack, offer) && mine) {
            cand_store1(J.cand, s, best_pos);
            J.anchor[s] = make_float4(y0, y1, y2, -1.f);  // position of this search, no cache
            walk = 0;
        }
    }
    // Many in this warp (or a cooperative walk ran out of stack): each point walks alone.
    if (walk == 1) {
        float wb = walk_bound(best_d2);
        auto scan1 = [&](int lf) {
            scan_points4(J.map.pts, lf * B, min(lf * B + B, nmap), [&](int u, const float4& p) {
                const float d2 = exact_d2(p);
                const int oi = __float_as_int(p.w);
                if (before(d2, oi, best_d2, best_oi)) {
                    best_d2 = d2;
                    best_oi = oi;
                    best_pos = u;
                    wb = walk_bound(d2);
                }
            });
        };
        if (h0 >= 0) scan1(h0);
        traverse8(J.map, y0, y1, y2, wb, [&](int lf) {
            if (lf != h0) scan1(lf);
        });
        cand_store1(J.cand, s, best_pos);
        J.anchor[s] = make_float4(y0, y1, y2, -1.f);  // position of this search, no cache
    } else if (walk == 2) {
        unsigned long long Lk[KC];
        int P[KC];
#pragma unroll
        for (int j = 0; j < KC; ++j) {
            Lk[j] = dkey(lim, 0x7fffffff);
            P[j] = -1;
        }
        float bound = lim;
        auto scan_leaf = [&](int lf) {
            scan_points4(J.map.pts, lf * B, min(lf * B + B, nmap), [&](int u, const float4& p) {
                const unsigned long long key = dkey(point_d2(y0, y1, y2, p), __float_as_int(p.w));
                if (key < Lk[KC - 1]) key_insert(Lk, P, key, u);
            });
            bound = key_d2(Lk[KC - 1]);
        };
        if (h0 >= 0) scan_leaf(h0);
        if (h1 >= 0) scan_leaf(h1);
        traverse8(J.map, y0, y1, y2, bound, [&](int lf) {
            if (lf != h0 && lf != h1) scan_leaf(lf);
        });
        const float rc = (key_idx(Lk[KC - 1]) != 0x7fffffff ? sqrtf(key_d2(Lk[KC - 1])) : Rs) * (1.f - 1e-6f);
        cand_store(J.cand, s, P);
        J.anchor[s] = make_float4(y0, y1, y2, rc);
        pick_exact(P);
    }
    if (!active) return 0;
    if (J.corr_out) J.corr_out[__float_as_int(x.w)] = best_pos >= 0 ? best_oi : -1;
    if (best_pos < 0) return refreshed;

    acc[28] += 1.f;
    const float4 mu = J.map.pts[best_pos];
    const float4 ca = J.map.covs[2 * best_pos], cb = J.map.covs[2 * best_pos + 1];
    const float4 sa = J.covs_s[2l * s], sb = J.covs_s[2l * s + 1];
    const float S[9] = {sa.x, sa.y, sa.z, sa.y, sa.w, sb.x, sa.z, sb.x, sb.y};
    float RS[9];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c)
            RS[3 * r + c] = fmaf(R[3 * r], S[c], fmaf(R[3 * r + 1], S[3 + c], R[3 * r + 2] * S[6 + c]));
    auto rcr = [&](int r, int c) {
        return fmaf(RS[3 * r], R[3 * c], fmaf(RS[3 * r + 1], R[3 * c + 1], RS[3 * r + 2] * R[3 * c + 2]));
    };
    // Sigma = C^t + R C^s R^T
    const float s00 = ca.x + rcr(0, 0), s01 = ca.y + rcr(0, 1), s02 = ca.z + rcr(0, 2);
    const float s11 = ca.w + rcr(1, 1), s12 = cb.x + rcr(1, 2), s22 = cb.y + rcr(2, 2);
    // W = Sigma^-1 (cofactors / determinant)
    const float c00 = s11 * s22 - s12 * s12, c01 = s02 * s12 - s01 * s22, c02 = s01 * s12 - s02 * s11;
    const float det = s00 * c00 + s01 * c01 + s02 * c02;
    if (!(fabsf(det) > 0.f)) return refreshed;
    const float id = 1.f / det;
    const float W00 = c00 * id, W01 = c01 * id, W02 = c02 * id;
    const float W11 = (s00 * s22 - s02 * s02) * id, W12 = (s01 * s02 - s00 * s12) * id;
    const float W22 = (s00 * s11 - s01 * s01) * id;
    const float W[9] = {W00, W01, W02, W01, W11, W12, W02, W12, W22};
    const float d0 = __fsub_rn(__fsub_rn(mu.x, y0), l0), d1 = __fsub_rn(__fsub_rn(mu.y, y1), l1),
                d2 = __fsub_rn(__fsub_rn(mu.z, y2), l2);
    const float Wd0 = W00 * d0 + W01 * d1 + W02 * d2;
    const float Wd1 = W01 * d0 + W11 * d1 + W12 * d2;
    const float Wd2 = W02 * d0 + W12 * d1 + W22 * d2;
    // A = [y]x ; WA = W A
    const float A[9] = {0.f, -y2, y1, y2, 0.f, -y0, -y1, y0, 0.f};
    float WA[9];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c)
            WA[3 * r + c] = W[3 * r] * A[c] + W[3 * r + 1] * A[3 + c] + W[3 * r + 2] * A[6 + c];
    // A^T W A = -A (W A): column c is -(y x WA[:, c])
    float AWA[9];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float m0 = WA[c], m1 = WA[3 + c], m2 = WA[6 + c];
        AWA[c] = -(y1 * m2 - y2 * m1);
        AWA[3 + c] = -(y2 * m0 - y0 * m2);
        AWA[6 + c] = -(y0 * m1 - y1 * m0);
    }
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = r; c < 3; ++c) acc[ut(r, c)] += AWA[3 * r + c];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) acc[ut(r, 3 + c)] -= WA[3 * c + r];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = r; c < 3; ++c) acc[ut(3 + r, 3 + c)] += W[3 * r + c];
    // b = [A^T W d ; -W d],  A^T u = u x y
    acc[21] += Wd1 * y2 - Wd2 * y1;
    acc[22] += Wd2 * y0 - Wd0 * y2;
    acc[23] += Wd0 * y1 - Wd1 * y0;
    acc[24] -= Wd0;
    acc[25] -= Wd1;
    acc[26] -= Wd2;
    acc[27] += d0 * Wd0 + d1 * Wd1 + d2 * Wd2;
    acc[29] += d0 * d0 + d1 * d1 + d2 * d2;
    return refreshed;
}

// Block-wide sum of acc into row[0 .. NACC) (row[NACC ..32) zeroed; visible device-wide on return
// to thread 0 after its __threadfence); returns the number of threads with refreshed != 0.
static_assert(NACC <= 32, "one partial row of 32 floats, one component per lane");
template <int BS = REG_THREADS>
__device__ __forceinline__ int block_partial(const float (&acc)[NACC], int refreshed, float* row)
{
    __shared__ float red[BS / 32][NACC];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // Transposed butterfly: at each step a lane keeps half of its values and adds the partner's
    // copy of that half, so that lane c ends with component c's warp sum in 31 shuffles (5 per
    // component for a butterfly of each).  Every partial sum is the pairwise sum a butterfly of
    // that component forms (float addition commutes exactly), so the bits are the same.
    float v[32];
#pragma unroll
    for (int a = 0; a < 32; ++a) v[a] = a < NACC ? acc[a] : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int j = 0; j < o; ++j) {
            const float send = up ? v[j] : v[j + o];
            const float keep = up ? v[j + o] : v[j];
            v[j] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
    if (lane < NACC) red[warp][lane] = v[0];
    const int count = __syncthreads_count(refreshed);
    if (threadIdx.x < 32) {
        float v = 0.f;
        if (threadIdx.x < NACC) {
#pragma unroll
            for (int w = 0; w < BS / 32; ++w) v += red[w][threadIdx.x];
        }
        row[threadIdx.x] = v;
        __threadfence();
    }
    __syncthreads();
    return count;
}

// Reduction of the per-block partial rows, in two levels so that the part left to the last block is
// short: blocks are grouped by index in runs of GN_GROUP; the block that completes a group sums its
// group's rows (in row order, compensated float) into a group row of (hi, lo) pairs, and the block
// that completes the last group sums the group rows (in group order) and solves.  The order of every
// sum is fixed by the row indices alone, so a registration's result does not depend on which block
// finished when, and the batched kernel (same rows, same groups) gets the same bits.
// Layout after the nrows block rows (32 floats each) of a reduction area: G group rows (hi[32],
// lo[32]) and G group counters.
__device__ __forceinline__ float* group_rows(float* partials, int nrows) { return partials + 32l * nrows; }
__device__ __forceinline__ unsigned* group_counters(float* partials, int nrows, int ngroups)
{
    return reinterpret_cast<unsigned*>(partials + 32l * nrows + 64l * ngroups);
}

// Warp 0 of the block that completed group g: the compensated sum, in row order, of the group's rows
// below nb into its group row.
__device__ __forceinline__ void group_sum(const float* __restrict__ partials, int g, int nb, float* __restrict__ grow)
{
    const int c = threadIdx.x;  // component (lane of warp 0)
    const int r0 = g * GN_GROUP, r1 = min(r0 + GN_GROUP, nb);
    float v[GN_GROUP];
#pragma unroll
    for (int j = 0; j < GN_GROUP; ++j) v[j] = r0 + j < r1 ? __ldcg(partials + 32l * (r0 + j) + c) : 0.f;
    dfloat a = {0.f, 0.f};
#pragma unroll
    for (int j = 0; j < GN_GROUP; ++j) df_add(a, v[j]);
    grow[64l * g + c] = a.hi;
    grow[64l * g + 32 + c] = a.lo;
}

// One warp (all 32 lanes): records H, b, cost, inliers and the squared residuals of a
// linearisation whose NACC sums are tot[0 .. NACC) into the state.
__device__ __forceinline__ void record_sums(RegState* st, const double* tot, int lane)
{
    const double tot_l = lane < NACC ? tot[lane] : 0.0;  // component `lane`
    if (lane < 21) {
        int r = 0;
        while (ut(r, 5) < lane) ++r;
        const int c = lane - ut(r, r) + r;
        st->H[6 * r + c] = tot_l;
        st->H[6 * c + r] = tot_l;
    } else if (lane < 27) {
        st->b[lane - 21] = tot_l;
    } else if (lane == 27) {
        st->cost = tot_l;
    } else if (lane == 28) {
        st->inliers = (long long)llrint(tot_l);
    } else if (lane == 29) {
        st->sqdist = tot_l;
    }
}

// One warp (all 32 lanes), when solve is set: solves H delta = -b of the sums tot in FP64
// (Cholesky), applies T <- exp(delta^) T and takes the stopping decision: fewer than min_inliers
// correspondences or H not positive definite stop the registration as degenerate.  Returns whether
// another iteration should run (the same value on every lane).
__device__ __forceinline__ bool solve_update(const RegJob& J, RegState* st, const double* tot, int lane, int it_now,
                                             bool solve)
{
    const long long inliers = (long long)llrint(tot[28]);
    bool more = false;
    if (solve) {
        // the pose's column entries this lane combines (lane 4r + c: T(0..2, c)), read before the solve
        const int tcol = lane & 3;
        const double Tc[3] = {st->T[tcol], st->T[4 + tcol], st->T[8 + tcol]};
        // lane p < 27 takes entry (i, j) of [H ; -b^T]
        int ci = 0, cj = 0;
        if (lane < 27) chol_lane_coords(lane, ci, cj);
        double a = lane < 27 ? tot[ci == 6 ? 21 + cj : ut(cj, ci)] : 0.0;
        if (ci == 6) a = -a;
        double delta[6];
        int status = REG_ST_RUNNING;
        if (inliers < J.min_inliers || !warp_chol_solve6(a, lane, delta)) {
            status = REG_ST_DEGENERATE;
        } else {
            const double Tn = warp_se3_left_update(delta, Tc, lane);
            __syncwarp();
            if (lane < 12) {
                st->T[lane] = Tn;
                const float hi = (float)Tn, lo = (float)(Tn - (double)hi);
                if ((lane & 3) == 3) {
                    st->tf[lane >> 2] = hi;
                    st->tlo[lane >> 2] = lo;
                } else {
                    st->Rf[3 * (lane >> 2) + (lane & 3)] = hi;
                    st->Rlo[3 * (lane >> 2) + (lane & 3)] = lo;
                }
            }
            const double dw2 = fma(delta[0], delta[0], fma(delta[1], delta[1], delta[2] * delta[2]));
            const double dv2 = fma(delta[3], delta[3], fma(delta[4], delta[4], delta[5] * delta[5]));
            if (dw2 < J.tol_rot * J.tol_rot && dv2 < J.tol_trans * J.tol_trans) status = REG_ST_CONVERGED;
            else if (it_now + 1 >= J.max_iters || it_now + 1 >= 10000) status = REG_ST_MAXITER;
            else more = true;
        }
        if (lane == 0) {
            st->iter = it_now + 1;
            if (status != REG_ST_RUNNING) st->status = status;
        }
    }
    return more;
}

// The block that completed the last group: the compensated sum of the ng group rows, then in its
// second warp the H, b, cost and inliers of this linearisation and, at the same time in its first
// warp, (solve mode) the FP64 solve, the pose update and the stopping test.  Returns whether another iteration should run (on lane 0 of
// warp 0; false elsewhere).  t_start: globaltimer when the block became the last.
__device__ __forceinline__ bool finalize(const RegJob& J, RegState* st, const float* __restrict__ grow, int ng,
                                         int it_now, unsigned long long t_start)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __shared__ double tot[32];
    if (warp == 0) {
        dfloat a = {0.f, 0.f};
        for (int g0 = 0; g0 < ng; g0 += 8) {
            float hi[8], lo[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const bool in = g0 + j < ng;
                hi[j] = in ? __ldcg(grow + 64l * (g0 + j) + lane) : 0.f;
                lo[j] = in ? __ldcg(grow + 64l * (g0 + j) + 32 + lane) : 0.f;
            }
#pragma unroll
            for (int j = 0; j < 8; ++j) df_merge(a, hi[j], lo[j]);
        }
        tot[lane] = (double)a.hi + (double)a.lo;
    }
    __syncthreads();
    if (warp == 1) {  // H, b, cost and inliers of this linearisation, beside warp 0's solve
        record_sums(st, tot, lane);
        if (J.sums_out && lane < NACC) J.sums_out[lane] = tot[lane];
    }
    if (warp != 0) return false;

    // ---- warp 0: the lane-parallel FP64 solve
    unsigned long long t_solve = 0;
    if (lane == 0) asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t_solve));
    if (lane == 0) st->counter = 0u;
    const bool more = solve_update(J, st, tot, lane, it_now, J.mode == REG_MODE_SOLVE);
    if (lane == 0) {
        unsigned long long t_end;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t_end));
        const int it = J.mode == REG_MODE_SOLVE ? it_now : 0;
        if (it < REG_STATS) {
            st->tail_ns[it] = (int)(t_end - t_start);
            st->solve_ns[it] = (int)(t_end - t_solve);
        }
        __threadfence();
    }
    return more;
}

// Which block of points this launch's block blockIdx.x processes in iteration it: blocks of the
// previous iteration's slowest duration class first, then the next class, and so on; index order
// when there is no complete record (the first iteration).  A block's points, partial row and group
// follow from the block it processes, so the order changes when blocks start, not what they sum.
// In a grid that needs more than one wave of resident blocks, starting the long blocks first keeps
// them from beginning last and setting the iteration's end (the durations of a block's points change
// little from one iteration to the next).
__device__ __forceinline__ int sched_block(const int* __restrict__ sched, int G, int it)
{
    const int p = (it + 1) & 1;  // the record the previous iteration wrote
    const int4 c0 = __ldcg(reinterpret_cast<const int4*>(sched + 8 * p));
    const int2 c1 = __ldcg(reinterpret_cast<const int2*>(sched + 8 * p + 4));
    const int cnt[SCHED_BUCKETS] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y};
    int total = 0;
#pragma unroll
    for (int k = 0; k < SCHED_BUCKETS; ++k) total += cnt[k];
    int b = blockIdx.x;
    if (total != G) return b;
    const int* lists = sched + 16 + (long)p * SCHED_BUCKETS * G;
#pragma unroll
    for (int k = SCHED_BUCKETS - 1; k >= 0; --k) {
        if (b < cnt[k]) return __ldcg(lists + (long)k * G + b);
        b -= cnt[k];
    }
    return blockIdx.x;
}

// Records that block lb of iteration it took dt_ns (its duration class and place in the class's list).
__device__ __forceinline__ void sched_record(int* __restrict__ sched, int G, int it, int lb, unsigned long long dt_ns)
{
    const unsigned q = (unsigned)min(dt_ns >> 12, 0xffffffull);
    const int k = q == 0u ? 0 : min(SCHED_BUCKETS - 1, 32 - __clz(q));
    const int p = it & 1;
    const int pos = atomicAdd(sched + 8 * p + k, 1);
    sched[16 + ((long)p * SCHED_BUCKETS + k) * G + pos] = lb;
}

// One Gauss-Newton iteration, BS source points per block (one per thread): 128, 256 (the batched
// kernel's chunk, which makes the two paths' sums the same bits) or 384.  The launch bounds ask for
// 768 threads per SM at 256 and 384, i.e. 80 registers a thread (per 1200x680 frame, with the
// slowest-first block order: 256 points per block 1.10 ms against 1.15 ms with the 64 registers of
// 1024 threads per SM, whose walks spill; 384: 1.07 ms, 512 at 64 registers 1.11 ms), and 1024 at
// 128 (64 registers).
template <int BS>
__global__ void __launch_bounds__(BS, (BS == 128 ? 1024 : 768) / BS) gicp_iter_kernel(const RegJob* __restrict__ jp,
                                                                 cudaGraphConditionalHandle cond)
{
    // launched as a programmatic dependent of the previous iteration (plain-launch mode): wait for
    // it to complete (a no-op otherwise) before reading the pose and status it wrote
    asm volatile("griddepcontrol.wait;" ::: "memory");
    const RegJob& J = *jp;
    RegState* st = J.st;
    if (st->status != REG_ST_RUNNING) {
        // every block sees the same status here, so only this thread touches the condition
        if (J.use_cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(cond, 0u);
        return;
    }
    const int n = *J.n;
    const int nmap = *J.map.n;
    const int it_now = st->iter;
    __shared__ unsigned long long t_begin;  // thread 0's: kept in shared memory, not a register, over the search
    if (threadIdx.x == 0) {
        unsigned long long t0;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
        t_begin = t0;
        if (it_now < REG_STATS) atomicMin(&st->t_first[it_now], t0);
    }
    const int lb = J.sched ? sched_block(J.sched, gridDim.x, it_now) : blockIdx.x;  // the block of points
    float R[9], t[3], Rl[9], tl[3];
#pragma unroll
    for (int a = 0; a < 9; ++a) {
        R[a] = st->Rf[a];
        Rl[a] = st->Rlo[a];
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        t[a] = st->tf[a];
        tl[a] = st->tlo[a];
    }
    float acc[NACC];
#pragma unroll
    for (int a = 0; a < NACC; ++a) acc[a] = 0.f;
    // One source point per thread (the grid covers the context's capacity; the hardware block
    // scheduler balances the uneven per-point work, and the fixed point -> block mapping keeps
    // the reduction order, hence the result, deterministic).
    __shared__ int2 wstack[BS / 32][WARP_STACK];
    const int s = lb * BS + threadIdx.x;
    const int refreshed = gn_point(J, R, Rl, t, tl, s, s < n, nmap, acc, wstack[threadIdx.x >> 5],
                                   it_now < J.packet_iters);
    const int block_refreshed = block_partial<BS>(acc, refreshed, J.partials + 32l * lb);
    // this block's share is written: the next iteration's launch may begin (its blocks wait in
    // griddepcontrol.wait until this grid, the last block's solve included, has completed)
    asm volatile("griddepcontrol.launch_dependents;");
    const int nrows = gridDim.x, ngroups = (nrows + GN_GROUP - 1) / GN_GROUP, g = lb / GN_GROUP;
    const int nb = (n + BS - 1) / BS;  // rows of blocks that held points (the rest are zero)
    unsigned* gctr = group_counters(J.partials, nrows, ngroups);
    float* grow = group_rows(J.partials, nrows);
    __shared__ bool am_last;
    if (threadIdx.x == 0) {
        if (block_refreshed > 0 && it_now < REG_STATS) atomicAdd(&st->refreshes[it_now], block_refreshed);
        unsigned long long t1;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
        if (it_now < REG_STATS) atomicMax(&st->t_arrive[it_now], t1);
        if (J.sched) sched_record(J.sched, nrows, it_now, lb, t1 - t_begin);
        am_last = atomicAdd(&gctr[g], 1u) == (unsigned)(min(nrows - g * GN_GROUP, GN_GROUP) - 1);
    }
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    if (threadIdx.x < 32) {
        group_sum(J.partials, g, nb, grow);
        __threadfence();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        gctr[g] = 0u;  // every block of the group has counted: ready for the next iteration
        __threadfence();
        am_last = atomicAdd(&st->counter, 1u) == (unsigned)(ngroups - 1);
    }
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    // every block of this iteration has read the previous iteration's record: clear its counts for
    // the next iteration to fill
    if (J.sched && threadIdx.x < 8) J.sched[8 * ((it_now + 1) & 1) + threadIdx.x] = 0;
    unsigned long long t_start = 0;
    if (threadIdx.x == 0) asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t_start));
    // the groups of the blocks that held points: the same rows, groups and order as a batched
    // registration of these points sums
    const bool more = finalize(J, st, grow, (nb + GN_GROUP - 1) / GN_GROUP, it_now, t_start);
    if (threadIdx.x == 0 && J.use_cond) cudaGraphSetConditional(cond, more ? 1u : 0u);
}

static const void* iter_kernel(int bs)
{
    return bs == 128 ? (const void*)gicp_iter_kernel<128>
                     : (bs == 384 ? (const void*)gicp_iter_kernel<384> : (const void*)gicp_iter_kernel<256>);
}

// One plain launch of the iteration kernel of the machine's block size.
static gsicp_status launch_iter(const RegMachine& rm, cudaStream_t s)
{
    const RegJob* jp = rm.job.as<const RegJob>();
    cudaGraphConditionalHandle cond = rm.cond;
    void* args[] = {(void*)&jp, (void*)&cond};
    GSICP_CUDA(cudaLaunchKernel(iter_kernel(rm.bs), dim3(rm.grid), dim3(rm.bs), args, 0, s));
    return GSICP_OK;
}

// ---------------------------------------------------------------------------------------------
// Batched registration: many independent pairs in one persistent launch.
//
// Work items are (pair, REG_THREADS-point chunk) of a pair's current iteration, taken from a device queue
// (an append-only array of 64-bit items, empty slots all ones).  Resident blocks claim slots in
// order (atomic head) and wait, with a bounded spin, for a claimed slot to be filled.  The block
// that finishes a pair's last chunk of an iteration sums that pair's chunk partials in chunk order,
// solves and updates its pose (finalize, as in the single registration) and, if the pair goes on,
// appends the chunks of its next iteration; otherwise it retires the pair.  Pairs thus advance
// independently (a small pair does not wait for a large one), there is no grid-wide barrier, and
// every pair's sums are taken in the same order as gsicp_register's, so each pair's result is
// bit-identical to registering it alone.  Blocks leave when every pair has retired, or when a
// wait exceeds its bound (error flag: the host reports GSICP_ERR_TIMEOUT).
constexpr unsigned long long BATCH_EMPTY = ~0ull;
constexpr unsigned BATCH_SPIN_LIMIT = 1u << 22;  // polls of ~0.25 us each: ~1 s before giving up

__global__ void __launch_bounds__(REG_THREADS, REG_BLOCKS_PER_SM) gicp_batch_kernel(const RegJob* __restrict__ jobs,
                                                                 BatchQueue* __restrict__ q,
                                                                 unsigned long long* __restrict__ items,
                                                                 unsigned capacity)
{
    __shared__ long long s_item;
    __shared__ unsigned s_base;
    __shared__ bool s_last;
    __shared__ int2 wstack[REG_THREADS / 32][WARP_STACK];
    for (;;) {
        if (threadIdx.x == 0) {
            long long got = -1;
            const unsigned idx = atomicAdd(&q->head, 1u);
            if (idx < capacity) {
                for (unsigned spin = 0;; ++spin) {
                    const unsigned long long v = __ldcg(items + idx);
                    if (v != BATCH_EMPTY) {
                        got = (long long)v;
                        break;
                    }
                    if (__ldcg(&q->running) == 0u) break;  // every pair has retired: nothing will come
                    if (spin >= BATCH_SPIN_LIMIT) {
                        atomicExch(&q->error, 1u);
                        break;
                    }
                    __nanosleep(256);
                }
            }
            __threadfence();  // the pair's state was written before its item was published
            s_item = got;
        }
        __syncthreads();
        const long long item = s_item;
        if (item < 0) return;
        const int b = (int)(item >> 32), c = (int)(item & 0xffffffffll);
        const RegJob& J = jobs[b];
        RegState* st = J.st;
        const int n = *J.n, nmap = *J.map.n;
        const int nchunks = (n + REG_THREADS - 1) / REG_THREADS;
        const int it_now = __ldcg(&st->iter);
        float R[9], t[3], Rl[9], tl[3];
#pragma unroll
        for (int a = 0; a < 9; ++a) {
            R[a] = __ldcg(&st->Rf[a]);
            Rl[a] = __ldcg(&st->Rlo[a]);
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            t[a] = __ldcg(&st->tf[a]);
            tl[a] = __ldcg(&st->tlo[a]);
        }
        float acc[NACC];
#pragma unroll
        for (int a = 0; a < NACC; ++a) acc[a] = 0.f;
        const int s = c * REG_THREADS + threadIdx.x;
        const int refreshed = gn_point(J, R, Rl, t, tl, s, s < n, nmap, acc, wstack[threadIdx.x >> 5],
                                       it_now < J.packet_iters);
        block_partial(acc, refreshed, J.partials + 32l * c);
        const int ngroups = (nchunks + GN_GROUP - 1) / GN_GROUP, g = c / GN_GROUP;
        unsigned* gctr = group_counters(J.partials, nchunks, ngroups);
        float* grow = group_rows(J.partials, nchunks);
        if (threadIdx.x == 0)
            s_last = atomicAdd(&gctr[g], 1u) == (unsigned)(min(nchunks - g * GN_GROUP, GN_GROUP) - 1);
        __syncthreads();
        if (s_last) {
            __threadfence();
            if (threadIdx.x < 32) {
                group_sum(J.partials, g, nchunks, grow);
                __threadfence();
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                gctr[g] = 0u;  // reset before the pair's next iteration can be queued
                __threadfence();
                s_last = atomicAdd(&st->counter, 1u) == (unsigned)(ngroups - 1);
            }
            __syncthreads();
        }
        if (s_last) {
            __threadfence();
            const bool more = finalize(J, st, grow, ngroups, it_now, 0ull);
            __threadfence();  // the new pose and status before the next items
            __syncthreads();
            if (threadIdx.x == 0) s_base = more ? atomicAdd(&q->tail, (unsigned)nchunks) : 0xffffffffu;
            __syncthreads();
            if (s_base != 0xffffffffu) {
                for (int j = threadIdx.x; j < nchunks; j += REG_THREADS)
                    if (s_base + (unsigned)j < capacity) items[s_base + j] = ((unsigned long long)b << 32) | (unsigned)j;
            } else if (threadIdx.x == 0) {
                __threadfence();
                atomicSub(&q->running, 1u);
            }
        }
        __syncthreads();  // shared item slots are reused by the next claim
    }
}

// Per pair: initial state (as reg_setup_kernel), and the iteration-0 items of every pair with
// points, written at offsets[b]; block b handles pair b.
__global__ void batch_setup_kernel(const RegJob* __restrict__ jobs, const Pose16* __restrict__ T0, int B,
                                   const unsigned* __restrict__ offsets, unsigned long long* __restrict__ items)
{
    const int b = blockIdx.x;
    if (b >= B) return;
    const RegJob& J = jobs[b];
    RegState* st = J.st;
    const int n = *J.n;
    const int nchunks = (n + REG_THREADS - 1) / REG_THREADS;
    if (threadIdx.x == 0) {
        for (int i = 0; i < 16; ++i) st->T[i] = T0[b].v[i];
        for (int i = 0; i < 36; ++i) st->H[i] = 0.0;
        for (int i = 0; i < 6; ++i) st->b[i] = 0.0;
        st->cost = 0.0;
        st->sqdist = 0.0;
        st->inliers = 0;
        st->iter = 0;
        st->status = n > 0 ? REG_ST_RUNNING : REG_ST_DEGENERATE;
        st->counter = 0u;
        for (int i = 0; i < REG_STATS; ++i) {
            st->refreshes[i] = st->tail_ns[i] = st->solve_ns[i] = 0;
            st->t_first[i] = ~0ull;
            st->t_arrive[i] = 0ull;
        }
        pose_to_float(st);
    }
    for (int j = threadIdx.x; j < nchunks; j += blockDim.x)
        items[offsets[b] + j] = ((unsigned long long)b << 32) | (unsigned)j;
}

// Blocks of the persistent batched kernel: no more than can be resident at once (a claimed queue slot
// is filled by another block, which must be running), as the occupancy calculator gives it.
static int batch_grid()
{
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, gicp_batch_kernel, REG_THREADS, 0) != cudaSuccess)
        occ = REG_BLOCKS_PER_SM;
    return device_sm_count() * std::max(1, std::min(occ, REG_BLOCKS_PER_SM));
}

// The queue wait's bound, exercised: one pair "running" and no item will ever be published, so
// every block's wait runs out, sets the error flag and leaves.  Takes about a second.
gsicp_status batch_wait_selftest(BatchQueue* q_dev, unsigned long long* items, unsigned capacity, cudaStream_t s)
{
    GSICP_CUDA(cudaMemsetAsync(items, 0xff, sizeof(unsigned long long) * (size_t)capacity, s));
    const BatchQueue q0 = {0u, 0u, 1u, 0u};
    GSICP_CUDA(cudaMemcpyAsync(q_dev, &q0, sizeof(q0), cudaMemcpyHostToDevice, s));
    gicp_batch_kernel<<<batch_grid(), REG_THREADS, 0, s>>>(nullptr, q_dev, items, capacity);
    GSICP_CUDA(cudaGetLastError());
    return GSICP_OK;
}

gsicp_status batch_run(const RegJob* jobs_dev, int B, const Pose16* T0_dev, const unsigned* offsets_dev,
                       BatchQueue* q_dev, unsigned long long* items, unsigned capacity, cudaStream_t s)
{
    if (B <= 0) return GSICP_OK;
    GSICP_CUDA(cudaMemsetAsync(items, 0xff, sizeof(unsigned long long) * (size_t)capacity, s));
    batch_setup_kernel<<<B, 256, 0, s>>>(jobs_dev, T0_dev, B, offsets_dev, items);
    gicp_batch_kernel<<<batch_grid(), REG_THREADS, 0, s>>>(jobs_dev, q_dev, items, capacity);
    GSICP_CUDA(cudaGetLastError());
    return GSICP_OK;
}

// ---------------------------------------------------------------------------------------------

gsicp_status RegMachine::init(int capacity)
{
    const int want = std::max(1, (std::max(capacity, 1) + bs - 1) / bs);
    if (exec && want <= grid && built_bs == bs) return GSICP_OK;
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    exec = nullptr;
    graph = nullptr;
    grid = built_bs == bs ? std::max(want, grid) : want;  // grid counts blocks of bs points
    built_bs = bs;
    GSICP_CHECK(partials.ensure(sizeof(float) * reduction_floats(grid)));
    GSICP_CHECK(sched.ensure(sizeof(int) * sched_ints(grid)));
    GSICP_CUDA(cudaMemset(partials.ptr, 0, sizeof(float) * reduction_floats(grid)));  // group counters start at 0
    GSICP_CHECK(job.ensure(sizeof(RegJob)));
    GSICP_CHECK(state.ensure(sizeof(RegState)));
    if (!state_host) GSICP_CUDA(cudaMallocHost((void**)&state_host, sizeof(RegState)));
    GSICP_CUDA(cudaGraphCreate(&graph, 0));
    GSICP_CUDA(cudaGraphConditionalHandleCreate(&cond, graph, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t cnode;
    GSICP_CUDA(cudaGraphAddNode(&cnode, graph, nullptr, nullptr, 0, &cp));
    // The loop body: GN_BODY_ITERS iteration launches in a chain of programmatic edges, so that each
    // launch begins (and its blocks wait in griddepcontrol.wait) while the one before finishes its
    // solve, and the condition is re-evaluated once per GN_BODY_ITERS iterations (launches after
    // convergence exit at once).
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    const RegJob* jptr = job.as<const RegJob>();
    void* args[] = {(void*)&jptr, (void*)&cond};
    cudaKernelNodeParams kp = {};
    kp.func = const_cast<void*>(iter_kernel(bs));
    kp.gridDim = dim3(grid);
    kp.blockDim = dim3(bs);
    kp.sharedMemBytes = 0;
    kp.kernelParams = args;
    cudaGraphNode_t knode[GN_BODY_ITERS];
    for (int k = 0; k < GN_BODY_ITERS; ++k) {
        GSICP_CUDA(cudaGraphAddKernelNode(&knode[k], body, nullptr, 0, &kp));
        if (k > 0) {
            cudaGraphEdgeData ed = {};
            ed.from_port = cudaGraphKernelNodePortProgrammatic;
            ed.to_port = 0;
            ed.type = cudaGraphDependencyTypeProgrammatic;
            GSICP_CUDA(cudaGraphAddDependencies(body, &knode[k - 1], &knode[k], &ed, 1));
        }
    }
    GSICP_CUDA(cudaGraphInstantiate(&exec, graph, 0));
    return GSICP_OK;
}

void BatchMachine::release()
{
    src.release(); covs.release(); cand.release(); anchor.release(); partials.release(); counts.release();
    jobs.release(); states.release(); T0.release(); offsets.release(); queue.release(); items.release();
    ptrs.release(); pofs.release(); quant.release();
    if (host) cudaFreeHost(host);
    host = nullptr;
    host_bytes = 0;
}

void RegMachine::release()
{
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    exec = nullptr;
    graph = nullptr;
    if (state_host) cudaFreeHost(state_host);
    state_host = nullptr;
    partials.release();
    sched.release();
    job.release();
    state.release();
    cand.release();
    anchor.release();
}

// Buffers, first-iteration seeds and initial state of a registration of up to n_cap points; job
// (with the machine's buffers filled in) is copied to rm.job.
static gsicp_status reg_prepare(RegMachine& rm, RegJob& job, const double T0[16], int n_cap, cudaStream_t s)
{
    GSICP_CHECK(rm.init(n_cap));
    GSICP_CHECK(rm.cand.ensure(sizeof(int) * KC * (size_t)std::max(n_cap, 1)));
    GSICP_CHECK(rm.anchor.ensure(sizeof(float4) * (size_t)std::max(n_cap, 1)));
    job.cand = rm.cand.as<int>();
    job.anchor = rm.anchor.as<float4>();
    job.partials = rm.partials.as<float>();
    job.sched = rm.sched.as<int>();
    job.st = rm.state.as<RegState>();
    Pose16 P;
    for (int i = 0; i < 16; ++i) P.v[i] = T0[i];
    GSICP_CHECK(launch_seed(job.map, job.src, job.n, n_cap, T0, job.cand, job.anchor, s));
    GSICP_CUDA(launch_dependent(reg_setup_kernel, 1, 1, s, job, rm.job.as<RegJob>(), rm.state.as<RegState>(), P));
    return GSICP_OK;
}

// The update of a registration whose source points are split across processes: the sums of the
// nparts partial linearisations (NACC doubles each, summed in the order given, so every process
// that passes the same rows gets the same bits) are recorded and solved exactly as the single
// registration's last block does.  One warp.
__global__ void shard_update_kernel(const RegJob* __restrict__ jp, const double* __restrict__ parts, int nparts)
{
    __shared__ double tot[32];
    const int lane = threadIdx.x;
    double v = 0.0;
    if (lane < NACC)
        for (int q = 0; q < nparts; ++q) v += parts[(long)NACC * q + lane];
    tot[lane] = v;
    __syncwarp();
    const RegJob& J = *jp;
    RegState* st = J.st;
    const int it_now = st->iter;
    if (st->status != REG_ST_RUNNING) return;
    record_sums(st, tot, lane);
    solve_update(J, st, tot, lane, it_now, true);
    __threadfence();
}

gsicp_status reg_shard_begin(RegMachine& rm, const RegJob& job_in, const double T0[16], int n_cap, double* sums_out,
                             cudaStream_t s)
{
    RegJob job = job_in;
    job.mode = REG_MODE_LINEARISE;
    job.use_cond = 0;
    job.sums_out = sums_out;
    GSICP_CHECK(reg_prepare(rm, job, T0, n_cap, s));
    rm.shard = true;
    return GSICP_OK;
}

gsicp_status reg_shard_linearise(RegMachine& rm, cudaStream_t s)
{
    return launch_iter(rm, s);
}

gsicp_status reg_shard_update(RegMachine& rm, const double* parts, int nparts, cudaStream_t s)
{
    shard_update_kernel<<<1, 32, 0, s>>>(rm.job.as<const RegJob>(), parts, nparts);
    GSICP_CUDA(cudaGetLastError());
    GSICP_CUDA(cudaMemcpyAsync(rm.state_host, rm.state.ptr, REG_STATE_HEAD, cudaMemcpyDeviceToHost, s));
    return GSICP_OK;
}

gsicp_status reg_run(RegMachine& rm, const RegJob& job_in, const double T0[16], int n_cap, bool solve,
                     cudaStream_t s, cudaEvent_t gn_wait)
{
    RegJob job = job_in;
    job.mode = solve ? REG_MODE_SOLVE : REG_MODE_LINEARISE;
    job.use_cond = solve ? 1 : 0;
    job.sums_out = nullptr;
    rm.shard = false;
    GSICP_CHECK(reg_prepare(rm, job, T0, n_cap, s));
    if (solve && rm.mode == GSICP_GN_PLAIN) {
        // plain-launch mode: one launch per iteration, each a programmatic dependent of the one
        // before (finished launches exit at once)
        job.use_cond = 0;
        Pose16 P;
        for (int i = 0; i < 16; ++i) P.v[i] = T0[i];
        reg_setup_kernel<<<1, 1, 0, s>>>(job, rm.job.as<RegJob>(), rm.state.as<RegState>(), P);
        if (gn_wait) GSICP_CUDA(cudaStreamWaitEvent(s, gn_wait, 0));
        cudaLaunchAttribute attr;
        attr.id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr.val.programmaticStreamSerializationAllowed = 1;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(rm.grid);
        cfg.blockDim = dim3(rm.bs);
        cfg.dynamicSmemBytes = 0;
        cfg.stream = s;
        cfg.attrs = &attr;
        cfg.numAttrs = 1;
        const RegJob* jp = rm.job.as<const RegJob>();
        void* args[] = {(void*)&jp, (void*)&rm.cond};
        for (int i = 0; i < job.max_iters; ++i)
            GSICP_CUDA(cudaLaunchKernelExC(&cfg, iter_kernel(rm.bs), args));
        GSICP_CUDA(cudaGetLastError());
    } else if (solve) {
        if (gn_wait) GSICP_CUDA(cudaStreamWaitEvent(s, gn_wait, 0));
        GSICP_CUDA(cudaGraphLaunch(rm.exec, s));
    } else {
        if (gn_wait) GSICP_CUDA(cudaStreamWaitEvent(s, gn_wait, 0));
        GSICP_CHECK(launch_iter(rm, s));
    }
    GSICP_CUDA(cudaMemcpyAsync(rm.state_host, rm.state.ptr, REG_STATE_HEAD, cudaMemcpyDeviceToHost, s));
    return GSICP_OK;
}

// ---------------------------------------------------------------------------------------------

__global__ void nearest_kernel(IndexView ix, const float* __restrict__ q, int nq, float max_d2,
                               int32_t* __restrict__ idx, float* __restrict__ d2out)
{
    const int nmap = *ix.n;
    const float4 qz = *ix.quant;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nq; i += gridDim.x * blockDim.x) {
        float bd = max_d2;
        int bo = 0x7fffffff, bp = -1;
        const float q0 = q[3l * i], q1 = q[3l * i + 1], q2 = q[3l * i + 2];
        int2 rng[8];
        const float cert = grid_block8(ix, qz, q0, q1, q2, rng);
        if (cert > 0.f) {
#pragma unroll
            for (int c = 0; c < 8; ++c)
                for (int u = rng[c].x; u < rng[c].y; ++u) {
                    const float4 p = ix.pts[u];
                    const float d2 = point_d2(q0, q1, q2, p);
                    const int oi = __float_as_int(p.w);
                    if (before(d2, oi, bd, bo)) {
                        bd = d2;
                        bo = oi;
                        bp = u;
                    }
                }
        }
        if (!(bp >= 0 && bd <= cert * cert * (1.f - 2e-5f))) {  // not certified by the block: full search
            bd = max_d2;
            bo = 0x7fffffff;
            bp = -1;
            nn_search(ix, nmap, q0, q1, q2, bd, bo, bp);
        }
        idx[i] = bp >= 0 ? bo : -1;
        if (d2out) d2out[i] = bp >= 0 ? bd : GSICP_INF;
    }
}

gsicp_status launch_nearest(const IndexView& map, const float* q, int nq, float max_d2, int32_t* idx, float* d2,
                            cudaStream_t s)
{
    if (nq <= 0) return GSICP_OK;
    const int grid = std::max(1, std::min((nq + 255) / 256, device_sm_count() * 8));
    nearest_kernel<<<grid, 256, 0, s>>>(map, q, nq, max_d2, idx, d2);
    GSICP_CUDA(cudaGetLastError());
    return GSICP_OK;
}

__global__ void transform_kernel(Pose16 T, const float* __restrict__ pts, const float* __restrict__ covs, int n,
                                 float* __restrict__ po, float* __restrict__ co)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double x[3] = {pts[3l * i], pts[3l * i + 1], pts[3l * i + 2]};
        for (int r = 0; r < 3; ++r)
            po[3l * i + r] = (float)(T.v[4 * r] * x[0] + T.v[4 * r + 1] * x[1] + T.v[4 * r + 2] * x[2] + T.v[4 * r + 3]);
        if (covs && co) {
            const float* c = covs + 6l * i;
            const double S[9] = {c[0], c[1], c[2], c[1], c[3], c[4], c[2], c[4], c[5]};
            double RS[9];
            for (int r = 0; r < 3; ++r)
                for (int cc = 0; cc < 3; ++cc)
                    RS[3 * r + cc] = T.v[4 * r] * S[cc] + T.v[4 * r + 1] * S[3 + cc] + T.v[4 * r + 2] * S[6 + cc];
            double M[9];
            for (int r = 0; r < 3; ++r)
                for (int cc = 0; cc < 3; ++cc)
                    M[3 * r + cc] = RS[3 * r] * T.v[4 * cc] + RS[3 * r + 1] * T.v[4 * cc + 1] + RS[3 * r + 2] * T.v[4 * cc + 2];
            float* o = co + 6l * i;
            o[0] = (float)M[0]; o[1] = (float)M[1]; o[2] = (float)M[2];
            o[3] = (float)M[4]; o[4] = (float)M[5]; o[5] = (float)M[8];
        }
    }
}

gsicp_status launch_transform(const double T[16], const float* pts, const float* covs, int n, float* pts_out,
                              float* covs_out, cudaStream_t s)
{
    if (n <= 0) return GSICP_OK;
    Pose16 P;
    for (int i = 0; i < 16; ++i) P.v[i] = T[i];
    const int grid = std::max(1, std::min((n + 255) / 256, device_sm_count() * 8));
    transform_kernel<<<grid, 256, 0, s>>>(P, pts, covs, n, pts_out, covs_out);
    GSICP_CUDA(cudaGetLastError());
    return GSICP_OK;
}

// Morton-key seed of one source point (see seed_kernel); R, t: the start pose in float.
__device__ __forceinline__ void seed_point(const IndexView& map, int m, float4 qz, const float (&Rt)[12],
                                           const float4 x, long s, int* __restrict__ cand,
                                           float4* __restrict__ anchor)
{
    int seed = -1;
    if (m > 0 && map.keys) {
        const float y0 = fmaf(Rt[0], x.x, fmaf(Rt[1], x.y, fmaf(Rt[2], x.z, Rt[3])));
        const float y1 = fmaf(Rt[4], x.x, fmaf(Rt[5], x.y, fmaf(Rt[6], x.z, Rt[7])));
        const float y2 = fmaf(Rt[8], x.x, fmaf(Rt[9], x.y, fmaf(Rt[10], x.z, Rt[11])));
        const uint32_t key = morton_of(qz, y0, y1, y2);
        int lo = 0, hi = m;
        while (lo < hi) {  // first sorted position whose key is not below the query's
            const int mid = (lo + hi) >> 1;
            if (map.keys[mid] < key) lo = mid + 1;
            else hi = mid;
        }
        seed = min(lo, m - 1);
    }
    int P[KC];
#pragma unroll
    for (int j = 0; j < KC; ++j) P[j] = j == 0 ? seed : -1;
    cand_store(cand, s, P);
    anchor[s] = make_float4(0.f, 0.f, 0.f, -2.f);  // no previous search
}

__global__ void batch_seed_kernel(const RegJob* __restrict__ jobs, const Pose16* __restrict__ T0,
                                  const int64_t* __restrict__ ofs, int B, long N)
{
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long)gridDim.x * blockDim.x) {
        int lo = 0, hi = B;  // job of point i (as cloud_of)
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (ofs[mid] <= i) lo = mid;
            else hi = mid;
        }
        const RegJob& J = jobs[lo];
        const Pose16& T = T0[lo];
        float Rt[12];
#pragma unroll
        for (int a = 0; a < 12; ++a) Rt[a] = (float)T.v[a];
        const long s = i - ofs[lo];
        seed_point(J.map, *J.map.n, *J.map.quant, Rt, J.src[s], s, J.cand, J.anchor);
    }
}

gsicp_status launch_batch_seed(const RegJob* jobs_dev, const Pose16* T0_dev, const int64_t* ofs_dev, int B, long N,
                               cudaStream_t s)
{
    if (N <= 0) return GSICP_OK;
    const int grid = (int)std::max<long>(1, std::min<long>((N + 255) / 256, device_sm_count() * 8));
    batch_seed_kernel<<<grid, 256, 0, s>>>(jobs_dev, T0_dev, ofs_dev, B, N);
    GSICP_CUDA(cudaGetLastError());
    return GSICP_OK;
}

__global__ void seed_kernel(IndexView map, const float4* __restrict__ src, const int* __restrict__ n_dev, Pose16 T,
                            int* __restrict__ cand, float4* __restrict__ anchor)
{
    wait_prior_grid();
    const int n = *n_dev, m = *map.n;
    const float4 qz = *map.quant;
    float Rt[12];
#pragma unroll
    for (int a = 0; a < 12; ++a) Rt[a] = (float)T.v[a];
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < n; s += gridDim.x * blockDim.x)
        seed_point(map, m, qz, Rt, src[s], s, cand, anchor);
}

gsicp_status launch_seed(const IndexView& map, const float4* src, const int* n_dev, int cap, const double T0[16],
                         int* cand, float4* anchor, cudaStream_t s)
{
    if (cap <= 0) return GSICP_OK;
    Pose16 P;
    for (int i = 0; i < 16; ++i) P.v[i] = T0[i];
    const int grid = std::max(1, std::min((cap + 255) / 256, device_sm_count() * 8));
    GSICP_CUDA(launch_dependent(seed_kernel, grid, 256, s, map, src, n_dev, P, cand, anchor));
    GSICP_CUDA(cudaGetLastError());
    return GSICP_OK;
}

__global__ void permute_covs_kernel(IndexView ix, const float* __restrict__ covs, int cap,
                                    float4* __restrict__ out)
{
    wait_prior_grid();
    const int n = *ix.n;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < min(n, cap); s += gridDim.x * blockDim.x) {
        const long i = __float_as_int(ix.pts[s].w);
        const float* c = covs + 6 * i;
        out[2l * s] = make_float4(c[0], c[1], c[2], c[3]);
        out[2l * s + 1] = make_float4(c[4], c[5], 0.f, 0.f);
    }
}

gsicp_status launch_permute_covs(const IndexView& ix, const float* covs, int cap, float4* out, cudaStream_t s)
{
    if (cap <= 0) return GSICP_OK;
    const int grid = std::max(1, std::min((cap + 255) / 256, device_sm_count() * 8));
    GSICP_CUDA(launch_dependent(permute_covs_kernel, grid, 256, s, ix, covs, cap, out));
    GSICP_CUDA(cudaGetLastError());
    return GSICP_OK;
}

__global__ void set_int_kernel(int* dst, int v) { *dst = v; }

gsicp_status launch_set_int(int* dst, int value, cudaStream_t s)
{
    set_int_kernel<<<1, 1, 0, s>>>(dst, value);
    GSICP_CUDA(cudaGetLastError());
    return GSICP_OK;
}

}  // namespace gsicp
