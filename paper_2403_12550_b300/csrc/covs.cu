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

// Neighbour access for finish_cov when keys hold original indices.
struct ByIndex {
    const float* orig;
    __device__ float3 operator()(int i) const { return make_float3(orig[3l * i], orig[3l * i + 1], orig[3l * i + 2]); }
};
struct SameIndex {
    __device__ int operator()(int i) const { return i; }
};

// Covariance of the k neighbours in Lk (ascending keys, phantoms first), its regularisation
// (Sec. 3.1) and scale aligning (Sec. 3.2), written for the query q (q.w: its original index) to
// covs (original order), optionally to covs_sorted at position s and its neighbours to knn_out.
// nb(id) gives the coordinates and oi(id) the original index of the neighbour whose key holds id.
template <int KMAX, class Nb, class Oi>
__device__ __forceinline__ void finish_cov(const unsigned long long (&Lk)[KMAX], int k, float4 q, Nb&& nb, Oi&& oi,
                                           const float* __restrict__ zin, float eps, int mode, float p,
                                           float* __restrict__ covs, int32_t* __restrict__ knn_out,
                                           float4* __restrict__ covs_sorted, long s)
{
    const int qi = __float_as_int(q.w);
    int I[KMAX];
#pragma unroll
    for (int j = 0; j < KMAX; ++j) I[j] = key_idx(Lk[j]);
    // ---- covariance of the neighbourhood (two-pass, float), neighbours gathered by original index
    int kk = 0;
    float m0 = 0.f, m1 = 0.f, m2 = 0.f;
#pragma unroll
    for (int j = 0; j < KMAX; ++j) {
        if (j >= KMAX - k && I[j] != 0x7fffffff) {
            const float3 P = nb(I[j]);
            m0 += __fsub_rn(P.x, q.x);
            m1 += __fsub_rn(P.y, q.y);
            m2 += __fsub_rn(P.z, q.z);
            ++kk;
        }
    }
    const float inv_k = 1.f / (float)max(kk, 1);
    m0 *= inv_k; m1 *= inv_k; m2 *= inv_k;
    float C[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int j = 0; j < KMAX; ++j) {
        if (j >= KMAX - k && I[j] != 0x7fffffff) {
            const float3 P = nb(I[j]);
            const float e0 = __fsub_rn(P.x, q.x) - m0;
            const float e1 = __fsub_rn(P.y, q.y) - m1;
            const float e2 = __fsub_rn(P.z, q.z) - m2;
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
                        const float3 P = nb(I[j]);
                        const double e0 = (double)P.x - (double)q.x;
                        const double e1 = (double)P.y - (double)q.y;
                        const double e2 = (double)P.z - (double)q.z;
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
            if (j >= KMAX - k) knn_out[(long)qi * k + (j - (KMAX - k))] = I[j] == 0x7fffffff ? -1 : oi(I[j]);
    }
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
        finish_cov<KMAX>(Lk, k, q, ByIndex{orig}, SameIndex{}, zin, eps, mode, p, covs, knn_out, covs_sorted, s);
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

// ---------------------------------------------------------------------------------------------
// Image-window k-NN for the points of one depth frame.
//
// The points of a frame come from a pinhole camera: the point of sample (i, j) lies on the ray of
// pixel (u, v) = (s i, s j), x = (u - cx) z / fx, y = (v - cy) z / fy.  Every point of a sample
// column >= i + R + 1 therefore lies in the half-space fx x - (U - cx) z >= 0 with
// U = s (i + R + 1), while the query lies at distance (U - u) z_q / sqrt(fx^2 + (U - cx)^2) on the
// other side of its plane (through the camera centre); likewise for the other three sides of the
// (2R+1) x (2R+1) sample window around the query.  So if the k-th nearest point inside the window
// is closer than the nearest of those four planes (less margins for float rounding of the points
// and distances), no point outside the window can be among the k nearest, and the window's k
// nearest are exactly the k nearest of the whole cloud (same float distances and tie order as the
// tree search).  A 9 x 9 window certifies nearly every point; the rest (grazing surfaces, image
// borders) get a 25 x 25 window, and what that leaves goes to the tree.

// Radius within which the window of half-width R around sample (i, j) holds every point (+inf
// when the window reaches every image border), with the float margins applied.
__device__ __forceinline__ float window_cert(int i, int j, int R, int Ws, int Hs, int stride, float zq, float fx,
                                             float fy, float cx, float cy)
{
    const float u = (float)(stride * i), v = (float)(stride * j);
    const float gap = (float)(stride * (R + 1));
    float cert = GSICP_INF;
    if (i + R + 1 < Ws) cert = fminf(cert, gap * zq * rsqrtf(fx * fx + (u + gap - cx) * (u + gap - cx)));
    if (i - R - 1 >= 0) cert = fminf(cert, gap * zq * rsqrtf(fx * fx + (u - gap - cx) * (u - gap - cx)));
    if (j + R + 1 < Hs) cert = fminf(cert, gap * zq * rsqrtf(fy * fy + (v + gap - cy) * (v + gap - cy)));
    if (j - R - 1 >= 0) cert = fminf(cert, gap * zq * rsqrtf(fy * fy + (v - gap - cy) * (v - gap - cy)));
    // 1e-4 relative (rsqrtf, float products); 1e-5 m (points rounded to float lie up to
    // |p| * 6e-8 off their ray)
    return cert == GSICP_INF ? cert : cert * (1.f - 1e-4f) - 1e-5f;
}

template <int KMAX>
__device__ __forceinline__ bool window_certifies(const unsigned long long (&Lk)[KMAX], float cert)
{
    return key_idx(Lk[KMAX - 1]) != 0x7fffffff && cert > 0.f &&
           (cert == GSICP_INF || key_d2(Lk[KMAX - 1]) <= cert * cert);
}

// One block = 32 x 4 samples; the samples of the block and a halo of R are staged in shared
// memory as float4 (x, y, z, original index), missing samples as (+inf, .., INT_MAX).  The 5 x 5
// samples around the query are taken first, so the list is nearly final before the outer ring
// and few of its points are inserted.  Uncertified queries go to fb_list as (original index,
// sample index).
constexpr int WIN_TX = 32, WIN_TY = 4;

template <int KMAX, int R>
__global__ void __launch_bounds__(WIN_TX * WIN_TY, 6) knn_window_kernel(
    const int* __restrict__ idx_img, int Ws, int Hs, int stride, float fx, float fy, float cx, float cy,
    const float* __restrict__ orig, const float* __restrict__ zin, int k, float eps, int mode, float p,
    float* __restrict__ covs, int32_t* __restrict__ knn_out, int2* __restrict__ fb_list, int* __restrict__ fb_count)
{
    static_assert(R >= 2, "the first pass takes the 5 x 5 centre");
    constexpr int SX = WIN_TX + 2 * R, SY = WIN_TY + 2 * R;
    __shared__ float4 tile[SY][SX];
    const int bx = blockIdx.x * WIN_TX - R, by = blockIdx.y * WIN_TY - R;
    for (int t = threadIdx.x; t < SX * SY; t += WIN_TX * WIN_TY) {
        const int tx = t % SX, ty = t / SX;
        const int sx = bx + tx, sy = by + ty;
        float4 v = make_float4(GSICP_INF, GSICP_INF, GSICP_INF, __int_as_float(0x7fffffff));
        if (sx >= 0 && sx < Ws && sy >= 0 && sy < Hs) {
            const int pi = idx_img[(long)sy * Ws + sx];
            if (pi >= 0) v = make_float4(orig[3l * pi], orig[3l * pi + 1], orig[3l * pi + 2], __int_as_float(pi));
        }
        tile[ty][tx] = v;
    }
    __syncthreads();
    const int lx = threadIdx.x % WIN_TX, ly = threadIdx.x / WIN_TX;
    const int i = blockIdx.x * WIN_TX + lx, j = blockIdx.y * WIN_TY + ly;
    const float4 q = tile[ly + R][lx + R];
    const bool active = i < Ws && j < Hs && __float_as_int(q.w) != 0x7fffffff;
    bool certified = false;
    if (active) {
        unsigned long long Lk[KMAX];
        const unsigned long long empty = dkey(GSICP_INF, 0x7fffffff);
        // keys hold the tile position of the point: tile positions are ordered like the original
        // (row-major) indices, so ties break exactly as by index, and the neighbours are read
        // back from shared memory
        const float4* tl = &tile[0][0];
        auto key_at = [&](int dy, int dx) {
            const int pos = (ly + R + dy) * SX + (lx + R + dx);
            const float4 pp = tl[pos];
            return __float_as_int(pp.w) == 0x7fffffff ? empty : dkey(point_d2(q.x, q.y, q.z, pp), pos);
        };
        // Up to KMAX = 20, the first KMAX samples of the 5 x 5 centre fill the list at once and a
        // sorting network orders them (an insertion each would cost a pass over the list); then
        // only the k smallest stay, in the last k slots, with zero keys in front that nothing
        // displaces: the list that inserting them one by one gives.  (At KMAX = 32 the network's
        // keys no longer fit in registers: the list starts empty.)
        constexpr int NF = KMAX <= 20 ? KMAX : 0;
        if constexpr (NF > 0) {
#pragma unroll
            for (int a = 0; a < KMAX; ++a) Lk[a] = key_at(a / 5 - 2, a % 5 - 2);
            sort_keys(Lk);
            const int sh = KMAX - k;  // shift right by sh, one power of two at a time
#pragma unroll
            for (int b = 1; b < KMAX; b <<= 1)
                if (sh & b) {
#pragma unroll
                    for (int a = KMAX - 1; a >= 0; --a) Lk[a] = a >= b ? Lk[a - b] : 0ull;
                }
        } else {
#pragma unroll
            for (int a = 0; a < KMAX; ++a) Lk[a] = a < KMAX - k ? 0ull : empty;
        }
        auto visit = [&](int dy, int dx) {
            const unsigned long long key = key_at(dy, dx);  // a missing sample: the empty key
            if (key < Lk[KMAX - 1]) key_insert(Lk, key);
        };
        // loops kept rolled: one copy of the insertion code keeps the kernel in the instruction cache
#pragma unroll 1
        for (int c = NF; c < 25; ++c) visit(c / 5 - 2, c % 5 - 2);
#pragma unroll 1
        for (int dy = -R; dy <= R; ++dy) {
            const bool mid = dy >= -2 && dy <= 2;
#pragma unroll 1
            for (int dx = -R; dx <= R; ++dx)
                if (!mid || dx < -2 || dx > 2) visit(dy, dx);
        }
        certified = window_certifies(Lk, window_cert(i, j, R, Ws, Hs, stride, q.z, fx, fy, cx, cy));
        if (certified)
            finish_cov<KMAX>(
                Lk, k, q, [&](int pos) { const float4 v = tl[pos]; return make_float3(v.x, v.y, v.z); },
                [&](int pos) { return __float_as_int(tl[pos].w); }, zin, eps, mode, p, covs, knn_out, nullptr, 0);
    }
    // the rest go to the next pass (one atomic per warp)
    const bool need = active && !certified;
    const unsigned m = __ballot_sync(0xffffffffu, need);
    if (m) {
        const int lane = threadIdx.x & 31;
        int base = 0;
        if (lane == __ffs(m) - 1) base = atomicAdd(fb_count, __popc(m));
        base = __shfl_sync(0xffffffffu, base, __ffs(m) - 1);
        if (need) fb_list[base + __popc(m & ((1u << lane) - 1u))] = make_int2(__float_as_int(q.w), j * Ws + i);
    }
}

// Second pass: one warp per listed query, the (2 R2 + 1)^2 window read straight from memory,
// each lane keeping the k best of its share, then the warp's k best taken one by one (warp
// minimum of the lanes' heads).  Still uncertified queries go to fb2 as (original index, the
// window's k-th squared distance or +inf) for the tree.
template <int KMAX, int R2>
__global__ void __launch_bounds__(COV_THREADS) knn_wide_window_kernel(
    const int2* __restrict__ list, const int* __restrict__ count, const int* __restrict__ idx_img, int Ws, int Hs,
    int stride, float fx, float fy, float cx, float cy, const float* __restrict__ orig, const float* __restrict__ zin,
    int k, float eps, int mode, float p, float* __restrict__ covs, int32_t* __restrict__ knn_out,
    int2* __restrict__ fb2, int* __restrict__ count2)
{
    wait_prior_grid();
    constexpr int D = 2 * R2 + 1, NC = D * D;
    const int lane = threadIdx.x & 31;
    const int m = *count;
    const unsigned long long empty = dkey(GSICP_INF, 0x7fffffff);
    for (int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < m; t += (gridDim.x * blockDim.x) >> 5) {
        const int2 e = list[t];
        const int qi = e.x, i = e.y % Ws, j = e.y / Ws;
        const float4 q = make_float4(orig[3l * qi], orig[3l * qi + 1], orig[3l * qi + 2], __int_as_float(qi));
        unsigned long long L[KMAX];  // this lane's best (no phantoms: ascending, empty at the end)
#pragma unroll
        for (int a = 0; a < KMAX; ++a) L[a] = empty;
        for (int c0 = 0; c0 < NC; c0 += 32 * 4) {
            int pi[4];
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const int c = c0 + 32 * h + lane;
                const int sx = i + c % D - R2, sy = j + c / D - R2;
                pi[h] = c < NC && sx >= 0 && sx < Ws && sy >= 0 && sy < Hs ? idx_img[(long)sy * Ws + sx] : -1;
            }
            float4 pp[4];
#pragma unroll
            for (int h = 0; h < 4; ++h)
                pp[h] = pi[h] >= 0 ? make_float4(orig[3l * pi[h]], orig[3l * pi[h] + 1], orig[3l * pi[h] + 2], 0.f)
                                   : make_float4(GSICP_INF, GSICP_INF, GSICP_INF, 0.f);
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                if (pi[h] < 0) continue;
                const unsigned long long key = dkey(point_d2(q.x, q.y, q.z, pp[h]), pi[h]);
                if (key < L[KMAX - 1]) key_insert(L, key);
            }
        }
        // merge: k rounds of warp minimum over the lanes' heads; the winner drops its head
        unsigned long long Lk[KMAX];
#pragma unroll
        for (int a = 0; a < KMAX; ++a) Lk[a] = a < KMAX - k ? 0ull : empty;
#pragma unroll
        for (int r = 0; r < KMAX; ++r) {
            if (r >= k) break;
            unsigned long long best = L[0];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long other = __shfl_xor_sync(0xffffffffu, best, o);
                best = other < best ? other : best;
            }
            Lk[KMAX - k + r] = best;
            if (L[0] == best && best != empty) {  // keys are unique: exactly one lane holds it
#pragma unroll
                for (int a = 0; a < KMAX - 1; ++a) L[a] = L[a + 1];
                L[KMAX - 1] = empty;
            }
        }
        const bool cert = window_certifies(Lk, window_cert(i, j, R2, Ws, Hs, stride, q.z, fx, fy, cx, cy));
        if (cert) {
            if (lane == 0)
                finish_cov<KMAX>(Lk, k, q, ByIndex{orig}, SameIndex{}, zin, eps, mode, p, covs, knn_out, nullptr, 0);
        } else if (lane == 0) {
            const float wk = key_idx(Lk[KMAX - 1]) != 0x7fffffff ? key_d2(Lk[KMAX - 1]) : GSICP_INF;
            fb2[atomicAdd(count2, 1)] = make_int2(qi, __float_as_int(wk));
        }
    }
}

// Exact k-NN by the tree for the listed queries (list[t] = (original index, an upper bound on its
// k-th squared distance: the window's k-th, or +inf)), one warp per query: the warp's lanes walk the
// tree together (warp_knn: up to 32 boxes or points per dependent step), collecting every point
// within the bound, so the walk starts tight.  These are the few points neither image window
// settled (depth edges, grazing surfaces); one thread each, their walks were long chains of
// dependent loads run by a handful of warps.  Lane 0 then builds the covariance.  If the walk's
// stack would overflow, lane 0 walks alone (same answer: both walks are exact).
template <int KMAX>
__global__ void __launch_bounds__(COV_THREADS) knn_list_kernel(IndexView ix, const int2* __restrict__ list,
                                                               const int* __restrict__ count,
                                                               const float* __restrict__ orig,
                                                               const float* __restrict__ zin, int k, float eps,
                                                               int mode, float p, float* __restrict__ covs,
                                                               int32_t* __restrict__ knn_out)
{
    wait_prior_grid();
    __shared__ int2 wstack[COV_THREADS / 32][WARP_STACK];
    const int n = *ix.n, B = ix.B, m = *count;
    const int lane = threadIdx.x & 31;
    const int w0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int t = w0; t < m; t += nwarps) {
        const int2 e = list[t];
        const int qi = e.x;
        const float4 q = make_float4(orig[3l * qi], orig[3l * qi + 1], orig[3l * qi + 2], __int_as_float(qi));
        const unsigned long long lim = dkey(__int_as_float(e.y), 0x7fffffff);  // accepts every point within the bound
        unsigned long long key;
        int pos;
        const bool ok = warp_knn(ix, n, q.x, q.y, q.z, k, lim, -1, -1, -1, wstack[threadIdx.x >> 5], key, pos);
        unsigned long long Lk[KMAX];  // lane 0: slots KMAX - k .. KMAX - 1 hold the k keys, ascending
#pragma unroll
        for (int a = 0; a < KMAX; ++a) {
            const int src = a - (KMAX - k);
            const unsigned long long v = __shfl_sync(0xffffffffu, key, src >= 0 ? src : 0);
            Lk[a] = src >= 0 ? v : 0ull;
        }
        if (lane == 0) {
            if (!ok) {
                float bound = __int_as_float(e.y);
#pragma unroll
                for (int a = 0; a < KMAX; ++a) Lk[a] = a < KMAX - k ? 0ull : lim;
                traverse(ix, q.x, q.y, q.z, bound, [&](int lf) {
                    const int beg = lf * B, end = min(beg + B, n);
                    for (int u = beg; u < end; ++u) {
                        const float4 pp = ix.pts[u];
                        const unsigned long long kk = dkey(point_d2(q.x, q.y, q.z, pp), __float_as_int(pp.w));
                        if (kk < Lk[KMAX - 1]) key_insert(Lk, kk);
                    }
                    bound = key_d2(Lk[KMAX - 1]);
                });
            }
            finish_cov<KMAX>(Lk, k, q, ByIndex{orig}, SameIndex{}, zin, eps, mode, p, covs, knn_out, nullptr, 0);
        }
        __syncwarp();
    }
}

template <int KMAX>
static gsicp_status launch_frame_knn_t(const IndexView& ix, const int* idx_img, int Ws, int Hs, int stride,
                               const float intr[4], const float* pts, const float* z, int cap,
                               const gsicp_cov_params& prm, float* covs, int32_t* knn, int2* fb_list, int* fb_count,
                               cudaStream_t s)
{
    // fb_list holds the first pass's leftovers from the front and the second's from cap on;
    // fb_count[0], fb_count[1] count them
    const dim3 grid((Ws + WIN_TX - 1) / WIN_TX, (Hs + WIN_TY - 1) / WIN_TY);
    knn_window_kernel<KMAX, 4><<<grid, WIN_TX * WIN_TY, 0, s>>>(idx_img, Ws, Hs, stride, intr[0], intr[1], intr[2],
                                                                 intr[3], pts, z, prm.k, prm.eps, prm.reg_mode,
                                                                 prm.p, covs, knn, fb_list, fb_count);
    const int lgrid = std::max(1, std::min((cap + COV_THREADS - 1) / COV_THREADS, device_sm_count() * 8));
    GSICP_CUDA(launch_dependent(knn_wide_window_kernel<KMAX, 12>, lgrid, COV_THREADS, s, fb_list, fb_count, idx_img, Ws,
                                Hs, stride, intr[0], intr[1], intr[2], intr[3], pts, z, prm.k, prm.eps, prm.reg_mode,
                                prm.p, covs, knn, fb_list + cap, fb_count + 1));
    GSICP_CUDA(launch_dependent(knn_list_kernel<KMAX>, lgrid, COV_THREADS, s, ix, fb_list + cap, fb_count + 1, pts, z,
                                prm.k, prm.eps, prm.reg_mode, prm.p, covs, knn));
    return GSICP_OK;
}

gsicp_status launch_frame_knn_cov(const IndexView& ix, const int* idx_img, int Ws, int Hs, int stride,
                                  const float intr[4], const float* pts, const float* z, int cap,
                                  const gsicp_cov_params& prm, float* covs, int32_t* knn, int* fb_list,
                                  int* fb_count, cudaStream_t s)
{
    if (cap <= 0) return GSICP_OK;
    GSICP_CUDA(cudaMemsetAsync(fb_count, 0, 2 * sizeof(int), s));
    const int k = prm.k;
    int2* fl = reinterpret_cast<int2*>(fb_list);
    if (k <= 8) GSICP_CHECK(launch_frame_knn_t<8>(ix, idx_img, Ws, Hs, stride, intr, pts, z, cap, prm, covs, knn, fl, fb_count, s));
    else if (k <= 16) GSICP_CHECK(launch_frame_knn_t<16>(ix, idx_img, Ws, Hs, stride, intr, pts, z, cap, prm, covs, knn, fl, fb_count, s));
    else if (k <= 20) GSICP_CHECK(launch_frame_knn_t<20>(ix, idx_img, Ws, Hs, stride, intr, pts, z, cap, prm, covs, knn, fl, fb_count, s));
    else GSICP_CHECK(launch_frame_knn_t<32>(ix, idx_img, Ws, Hs, stride, intr, pts, z, cap, prm, covs, knn, fl, fb_count, s));
    GSICP_CUDA(cudaGetLastError());
    return GSICP_OK;
}

}  // namespace gsicp
