// covs.cu -- a2+a3: source Gaussians from k nearest neighbours.
//
// Sec. 3: the covariance of a point is the covariance matrix of its k nearest
// neighbours.  Sec. 3.1: C = R Lambda^2 R^T; plane regularisation sets the
// scales to [1, 1, eps] (read as eigenvalues (eps, 1, 1), as in G-ICP);
// ellipse regularisation divides the scale matrix by median(S), i.e. the
// covariance by its middle eigenvalue.  Sec. 3.2: scale aligning divides the
// scales by z^p, i.e. multiplies the covariance by z^(-2p).
//
// One thread per query, a warp's 32 queries being the 32 points of one leaf of
// the source index (Morton order): the warp scans its own leaf and the two next
// to it, then walks the tree once for all 32 queries (packet_traverse in
// traverse.cuh).  Each thread keeps its k best candidates in registers as a
// sorted list, padded at the front with "phantom" entries so that the k-th best
// always sits in the last slot (static register indexing for any k <= KMAX).
#include <algorithm>

#include "internal.h"
#include "traverse.cuh"

namespace gsicp {

constexpr int COV_THREADS = 128;
constexpr float RANK_TOL = 1e-5f;     // middle/largest eigenvalue ratio of a line-like neighbourhood
constexpr float REFINE_GAP = 0.05f;   // (l1 - l0)/l1 below which the plane normal is refined in double

template <int P, int Q>
__device__ __forceinline__ void jacobi_rotate(float A[3][3], float V[3][3])
{
    const float apq = A[P][Q];
    if (apq == 0.f) return;
    const float theta = (A[Q][Q] - A[P][P]) / (2.f * apq);
    float t;
    if (fabsf(theta) > 1e18f) t = 0.5f / theta;
    else t = copysignf(1.f, theta) / (fabsf(theta) + sqrtf(theta * theta + 1.f));
    const float c = 1.f / sqrtf(t * t + 1.f), s = t * c;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        const float arp = A[r][P], arq = A[r][Q];
        A[r][P] = c * arp - s * arq;
        A[r][Q] = s * arp + c * arq;
    }
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        const float apr = A[P][r], aqr = A[Q][r];
        A[P][r] = c * apr - s * aqr;
        A[Q][r] = s * apr + c * aqr;
    }
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        const float vrp = V[r][P], vrq = V[r][Q];
        V[r][P] = c * vrp - s * vrq;
        V[r][Q] = s * vrp + c * vrq;
    }
}

template <int P, int Q>
__device__ __forceinline__ void sort_pair(float w[3], float V[3][3])
{
    if (w[Q] < w[P]) {
        float t = w[P]; w[P] = w[Q]; w[Q] = t;
#pragma unroll
        for (int r = 0; r < 3; ++r) { float x = V[r][P]; V[r][P] = V[r][Q]; V[r][Q] = x; }
    }
}

// Cyclic Jacobi on a symmetric 3x3 (float): eigenvalues ascending in w,
// eigenvectors in the columns of V.
__device__ __forceinline__ void eigh3f(const float C[6], float w[3], float V[3][3])
{
    float A[3][3] = {{C[0], C[1], C[2]}, {C[1], C[3], C[4]}, {C[2], C[4], C[5]}};
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) V[r][c] = r == c ? 1.f : 0.f;
    const float scale = fabsf(C[0]) + fabsf(C[3]) + fabsf(C[5]);
    for (int sweep = 0; sweep < 12; ++sweep) {
        const float off = fabsf(A[0][1]) + fabsf(A[0][2]) + fabsf(A[1][2]);
        if (!(off > 1e-9f * scale)) break;
        jacobi_rotate<0, 1>(A, V);
        jacobi_rotate<0, 2>(A, V);
        jacobi_rotate<1, 2>(A, V);
    }
    w[0] = A[0][0]; w[1] = A[1][1]; w[2] = A[2][2];
    sort_pair<0, 1>(w, V);
    sort_pair<1, 2>(w, V);
    sort_pair<0, 1>(w, V);
}

template <int KMAX>
__global__ void __launch_bounds__(COV_THREADS) knn_cov_kernel(IndexView ix, const float* __restrict__ orig,
                                                              const float* __restrict__ zin, int k, float eps,
                                                              int mode, float p, float* __restrict__ covs,
                                                              int32_t* __restrict__ knn_out,
                                                              float4* __restrict__ covs_sorted)
{
    const int n = *ix.n;
    const int B = ix.B;  // 32: a warp's queries are exactly the points of one leaf
    const int lane = threadIdx.x & 31;
    const int warp0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int base = warp0 * 32; base < n; base += nwarps * 32) {  // warp-uniform loop
        const int s = base + lane;
        const bool active = s < n;
        const float4 q = active ? ix.pts[s] : make_float4(0.f, 0.f, 0.f, 0.f);
        const int qi = __float_as_int(q.w);
        // ascending (squared distance, index) keys; phantom entries (key 0) pad the front so the
        // k-th best is always the last slot, empty slots hold (+inf, INT_MAX)
        unsigned long long Lk[KMAX];
        const unsigned long long empty = dkey(GSICP_INF, 0x7fffffff);
#pragma unroll
        for (int j = 0; j < KMAX; ++j) Lk[j] = j < KMAX - k ? 0ull : empty;
        // ---- exact k-NN (ties -> smaller original index): the warp's own leaf and its two Morton
        // neighbours first (a tight bound for every lane), then one packet walk of the tree for
        // the 32 queries, skipping those three leaves
        float bound = GSICP_INF;
        const int own = base / B;
        auto scan_leaf = [&](int lf) {
            const int beg = lf * B, end = min(beg + B, n);
            for (int t = beg; t < end; ++t) {
                const float4 pp = ix.pts[t];  // same address in every lane: one broadcast load
                if (!active) continue;
        int I[KMAX];
#pragma unroll
        for (int j = 0; j < KMAX; ++j) I[j] = key_idx(Lk[j]);
                const float d2 = point_d2(q.x, q.y, q.z, pp);
                const int oi = __float_as_int(pp.w);
                const unsigned long long key = dkey(d2, oi);
                if (key < Lk[KMAX - 1]) key_insert(Lk, key);
            }
            bound = key_d2(Lk[KMAX - 1]);
        };
        scan_leaf(own);
        if (own > 0) scan_leaf(own - 1);
        if ((own + 1) * B < n) scan_leaf(own + 1);
        packet_traverse(ix, active, q.x, q.y, q.z, bound, [&](int lf) {
            if (lf < own - 1 || lf > own + 1) scan_leaf(lf);
        });
        if (!active) continue;
        int I[KMAX];
#pragma unroll
        for (int j = 0; j < KMAX; ++j) I[j] = key_idx(Lk[j]);
        // ---- covariance of the neighbourhood (two-pass, float), neighbours gathered by original index
        int kk = 0;
        float m0 = 0.f, m1 = 0.f, m2 = 0.f;
#pragma unroll
        for (int j = 0; j < KMAX; ++j) {
            if (j >= KMAX - k && I[j] != 0x7fffffff) {
                const long b = 3l * I[j];
                m0 += __fsub_rn(orig[b], q.x);
                m1 += __fsub_rn(orig[b + 1], q.y);
                m2 += __fsub_rn(orig[b + 2], q.z);
                ++kk;
            }
        }
        const float inv_k = 1.f / (float)max(kk, 1);
        m0 *= inv_k; m1 *= inv_k; m2 *= inv_k;
        float C[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int j = 0; j < KMAX; ++j) {
            if (j >= KMAX - k && I[j] != 0x7fffffff) {
                const long b = 3l * I[j];
                const float e0 = __fsub_rn(orig[b], q.x) - m0;
                const float e1 = __fsub_rn(orig[b + 1], q.y) - m1;
                const float e2 = __fsub_rn(orig[b + 2], q.z) - m2;
                C[0] = fmaf(e0, e0, C[0]); C[1] = fmaf(e0, e1, C[1]); C[2] = fmaf(e0, e2, C[2]);
                C[3] = fmaf(e1, e1, C[3]); C[4] = fmaf(e1, e2, C[4]); C[5] = fmaf(e2, e2, C[5]);
            }
        }
#pragma unroll
        for (int a = 0; a < 6; ++a) C[a] *= inv_k;
        // ---- regularisation (Sec. 3.1)
        float out[6];
        if (mode == GSICP_REG_NONE) {
#pragma unroll
            for (int a = 0; a < 6; ++a) out[a] = C[a];
        } else {
            float w[3], V[3][3];
            eigh3f(C, w, V);
            if (kk < 3 || !(w[2] > 0.f) || w[1] <= RANK_TOL * w[2]) {
                out[0] = 1.f; out[1] = 0.f; out[2] = 0.f; out[3] = 1.f; out[4] = 0.f; out[5] = 1.f;
            } else if (mode == GSICP_REG_PLANE) {
                float n0 = V[0][0], n1 = V[1][0], n2 = V[2][0];
                if (w[1] - w[0] < REFINE_GAP * w[1]) {
                    // near-degenerate normal: one first-order correction of v0 against the
                    // covariance accumulated in double from exact coordinate differences
                    double s1[3] = {0, 0, 0}, s2[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll
                    for (int j = 0; j < KMAX; ++j) {
                        if (j >= KMAX - k && I[j] != 0x7fffffff) {
                            const long b = 3l * I[j];
                            const double e0 = (double)orig[b] - (double)q.x;
                            const double e1 = (double)orig[b + 1] - (double)q.y;
                            const double e2 = (double)orig[b + 2] - (double)q.z;
                            s1[0] += e0; s1[1] += e1; s1[2] += e2;
                            s2[0] += e0 * e0; s2[1] += e0 * e1; s2[2] += e0 * e2;
                            s2[3] += e1 * e1; s2[4] += e1 * e2; s2[5] += e2 * e2;
                        }
                    }
                    const double ik = 1.0 / kk;
                    const double mu0 = s1[0] * ik, mu1 = s1[1] * ik, mu2 = s1[2] * ik;
                    const double Cd[6] = {s2[0] * ik - mu0 * mu0, s2[1] * ik - mu0 * mu1, s2[2] * ik - mu0 * mu2,
                                          s2[3] * ik - mu1 * mu1, s2[4] * ik - mu1 * mu2, s2[5] * ik - mu2 * mu2};
                    double v[3][3];
#pragma unroll
                    for (int r = 0; r < 3; ++r)
#pragma unroll
                        for (int c = 0; c < 3; ++c) v[r][c] = V[r][c];
                    double u[3];  // Cd v0
                    u[0] = Cd[0] * v[0][0] + Cd[1] * v[1][0] + Cd[2] * v[2][0];
                    u[1] = Cd[1] * v[0][0] + Cd[3] * v[1][0] + Cd[4] * v[2][0];
                    u[2] = Cd[2] * v[0][0] + Cd[4] * v[1][0] + Cd[5] * v[2][0];
                    double x0 = v[0][0], x1 = v[1][0], x2 = v[2][0];
                    const double l0 = x0 * u[0] + x1 * u[1] + x2 * u[2];
#pragma unroll
                    for (int c = 1; c < 3; ++c) {
                        const double cc = v[0][c] * u[0] + v[1][c] * u[1] + v[2][c] * u[2];
                        const double lc = (double)w[c];
                        const double gap = l0 - lc;
                        if (fabs(cc) < 0.1 * fabs(gap)) {
                            const double f = cc / gap;
                            x0 += f * v[0][c]; x1 += f * v[1][c]; x2 += f * v[2][c];
                        }
                    }
                    const double nrm = rsqrt(x0 * x0 + x1 * x1 + x2 * x2);
                    n0 = (float)(x0 * nrm); n1 = (float)(x1 * nrm); n2 = (float)(x2 * nrm);
                }
                const float a = 1.f - eps;
                out[0] = 1.f - a * n0 * n0; out[1] = -a * n0 * n1; out[2] = -a * n0 * n2;
                out[3] = 1.f - a * n1 * n1; out[4] = -a * n1 * n2; out[5] = 1.f - a * n2 * n2;
            } else {  // ELLIPSE: C / middle eigenvalue, smallest ratio floored at eps
                const float il = 1.f / w[1];
#pragma unroll
                for (int a = 0; a < 6; ++a) out[a] = C[a] * il;
                const float r0 = w[0] * il;
                if (r0 < eps) {
                    const float f = eps - r0, n0 = V[0][0], n1 = V[1][0], n2 = V[2][0];
                    out[0] += f * n0 * n0; out[1] += f * n0 * n1; out[2] += f * n0 * n2;
                    out[3] += f * n1 * n1; out[4] += f * n1 * n2; out[5] += f * n2 * n2;
                }
            }
        }
        // ---- scale aligning (Sec. 3.2)
        if (p != 0.f) {
            const float sc = powf(zin[qi], -2.f * p);
#pragma unroll
            for (int a = 0; a < 6; ++a) out[a] *= sc;
        }
#pragma unroll
        for (int a = 0; a < 6; ++a) covs[6l * qi + a] = out[a];
        if (covs_sorted) {
            covs_sorted[2l * s] = make_float4(out[0], out[1], out[2], out[3]);
            covs_sorted[2l * s + 1] = make_float4(out[4], out[5], 0.f, 0.f);
        }
        if (knn_out) {
#pragma unroll
            for (int j = 0; j < KMAX; ++j)
                if (j >= KMAX - k) knn_out[(long)qi * k + (j - (KMAX - k))] = I[j] == 0x7fffffff ? -1 : I[j];
        }
    }
}

gsicp_status launch_knn_cov(const IndexView& ix, const float* orig_pts, const float* z, int cap,
                            const gsicp_cov_params& prm, float* covs, int32_t* knn, float4* covs_sorted,
                            cudaStream_t s)
{
    if (cap <= 0) return GSICP_OK;
    if (ix.B != 32) return GSICP_ERR_INVALID_ARG;  // one leaf per warp
    const int grid = std::max(1, std::min((cap + COV_THREADS - 1) / COV_THREADS, device_sm_count() * 16));
    const int k = prm.k;
    if (k <= 8)
        knn_cov_kernel<8><<<grid, COV_THREADS, 0, s>>>(ix, orig_pts, z, k, prm.eps, prm.reg_mode, prm.p, covs, knn,
                                                         covs_sorted);
    else if (k <= 16)
        knn_cov_kernel<16><<<grid, COV_THREADS, 0, s>>>(ix, orig_pts, z, k, prm.eps, prm.reg_mode, prm.p, covs, knn,
                                                         covs_sorted);
    else if (k <= 20)
        knn_cov_kernel<20><<<grid, COV_THREADS, 0, s>>>(ix, orig_pts, z, k, prm.eps, prm.reg_mode, prm.p, covs, knn,
                                                         covs_sorted);
    else
        knn_cov_kernel<32><<<grid, COV_THREADS, 0, s>>>(ix, orig_pts, z, k, prm.eps, prm.reg_mode, prm.p, covs, knn,
                                                         covs_sorted);
    GSICP_CUDA(cudaGetLastError());
    return GSICP_OK;
}

}  // namespace gsicp
