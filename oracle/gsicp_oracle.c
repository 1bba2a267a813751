/*
 * gsicp_oracle.c -- FP64 CPU oracle for the G-ICP tracking path of
 * "RGBD GS-ICP SLAM" (arXiv 2403.12550).
 *
 * TEST INFRASTRUCTURE ONLY: the reference the CUDA library is checked
 * against.  Plain serial loops in IEEE double (OpenMP only spreads
 * independent per-point work; every sum is taken in a fixed order, so the
 * result does not depend on the thread count).  Shares nothing with the CUDA
 * sources.
 *
 * Which passage each part follows:
 *   depth -> points ........ Sec. 3 / Fig. 2 (downsample and reproject the depth image)
 *   k-NN covariance ........ Sec. 3 (covariance of the k nearest neighbours of a point)
 *   eigen-decomposition .... Sec. 3.1, Eq. for C = R Lambda^2 R^T
 *   regularisation ......... Sec. 3.1: plane S = [1,1,eps]; ellipse Lambda' = Lambda / median(S)
 *   scale aligning ......... Sec. 3.2: Lambda'' = Lambda' / z^p
 *   error model / MLE ...... Sec. 3, d_i ~ N(0, C^t + T C^s T^T) and Eq. (MLE_for_T)
 *   Gauss-Newton + SE(3) ... the G-ICP optimiser the paper builds on (Segal et al. 2009)
 *
 * Readings of the paper taken here (the paper is silent or garbled):
 *   - the query point is one of its own k neighbours; ties -> smaller index;
 *   - plane regularisation replaces the covariance eigenvalues by (1, 1, eps)
 *     (the garbled scale vector is read as eigenvalues, as in G-ICP);
 *   - ellipse regularisation divides by the middle eigenvalue, flooring the
 *     smallest ratio at eps; a rank-deficient neighbourhood (middle eigenvalue
 *     <= RANK_TOL * largest) gets C' = I;
 *   - scale aligning multiplies the covariance by z^(-2p) (scales are std-devs);
 *   - only the rotation of T acts on a covariance: Sigma = C^t + R C^s R^T;
 *   - the weight W = Sigma^-1 is held fixed while linearising;
 *   - left perturbation T <- exp(xi^) T, xi = (omega, v);
 *   - stop when |d omega| < tol_rot and |d v| < tol_trans.
 *
 * Parity unpinned: the ellipse floor at eps and the line-like threshold RANK_TOL are readings with
 * nothing outside this file to check them against (the tests exercise them, they cannot pin them).
 */
#include "gsicp_oracle.h"

#include <float.h>
#include <math.h>
#include <omp.h>
#include <stdlib.h>
#include <string.h>

#define RANK_TOL 1e-5   /* middle/largest eigenvalue ratio below which a neighbourhood is a line */
#define LEAF_SIZE 8

/* ------------------------------------------------------------------------------------------ */
/* depth -> points                                                                            */
/* ------------------------------------------------------------------------------------------ */

long orc_depth_to_points(const float* depth, int W, int H, const double intr[4], int stride,
                         double z_min, double z_max, double* pts, double* z, long cap)
{
    /* Pinhole back-projection of every stride-th pixel, row-major scan order:
     * pixel (u, v) with depth d -> ((u - cx) d / fx, (v - cy) d / fy, d). */
    if (W <= 0 || H <= 0 || stride <= 0) return -1;
    const double fx = intr[0], fy = intr[1], cx = intr[2], cy = intr[3];
    long n = 0;
    for (int v = 0; v < H; v += stride) {
        for (int u = 0; u < W; u += stride) {
            double d = (double)depth[(long)v * W + u];
            if (!isfinite(d) || d < z_min || d > z_max) continue;
            if (n >= cap) return -1;
            pts[3 * n + 0] = ((double)u - cx) * d / fx;
            pts[3 * n + 1] = ((double)v - cy) * d / fy;
            pts[3 * n + 2] = d;
            if (z) z[n] = d;
            ++n;
        }
    }
    return n;
}

/* ------------------------------------------------------------------------------------------ */
/* k-d tree (exact search; ties broken by smaller point index)                                */
/* ------------------------------------------------------------------------------------------ */

typedef struct {
    int axis;      /* -1 for a leaf */
    double split;
    long lo, hi;   /* range in perm */
    int left, right;
} kd_node;

struct orc_kdtree {
    const double* pts;
    long n;
    int32_t* perm;
    kd_node* nodes;
    int n_nodes, cap_nodes;
};

static double coord(const orc_kdtree* t, long i, int a) { return t->pts[3 * (long)t->perm[i] + a]; }

static void swap_perm(int32_t* p, long i, long j) { int32_t tmp = p[i]; p[i] = p[j]; p[j] = tmp; }

/* Rearrange perm[lo, hi) so that position mid holds the element of rank mid - lo
 * along axis a, everything before it <= and everything after it >= (quickselect). */
static void select_kth(orc_kdtree* t, long lo, long hi, long mid, int a)
{
    while (hi - lo > 1) {
        long m = lo + (hi - lo) / 2;
        double pv = coord(t, m, a);
        swap_perm(t->perm, m, hi - 1);
        long store = lo;
        for (long i = lo; i < hi - 1; ++i)
            if (coord(t, i, a) < pv) swap_perm(t->perm, i, store++);
        /* move equal keys next to the pivot so repeated values cannot stall */
        long eq = store;
        for (long i = store; i < hi - 1; ++i)
            if (coord(t, i, a) == pv) swap_perm(t->perm, i, eq++);
        swap_perm(t->perm, eq, hi - 1);
        if (mid < store) hi = store;
        else if (mid <= eq) return;
        else lo = eq + 1;
    }
}

static int new_node(orc_kdtree* t)
{
    if (t->n_nodes == t->cap_nodes) {
        t->cap_nodes = t->cap_nodes ? 2 * t->cap_nodes : 1024;
        t->nodes = (kd_node*)realloc(t->nodes, sizeof(kd_node) * t->cap_nodes);
    }
    return t->n_nodes++;
}

static int build_rec(orc_kdtree* t, long lo, long hi)
{
    int id = new_node(t);
    t->nodes[id].lo = lo;
    t->nodes[id].hi = hi;
    t->nodes[id].axis = -1;
    if (hi - lo <= LEAF_SIZE) return id;
    double bmin[3] = {DBL_MAX, DBL_MAX, DBL_MAX}, bmax[3] = {-DBL_MAX, -DBL_MAX, -DBL_MAX};
    for (long i = lo; i < hi; ++i)
        for (int a = 0; a < 3; ++a) {
            double c = coord(t, i, a);
            if (c < bmin[a]) bmin[a] = c;
            if (c > bmax[a]) bmax[a] = c;
        }
    int axis = 0;
    for (int a = 1; a < 3; ++a)
        if (bmax[a] - bmin[a] > bmax[axis] - bmin[axis]) axis = a;
    if (bmax[axis] == bmin[axis]) return id; /* all points identical: keep as one leaf */
    long mid = lo + (hi - lo) / 2;
    select_kth(t, lo, hi, mid, axis);
    double split = coord(t, mid, axis);
    int l = build_rec(t, lo, mid);
    int r = build_rec(t, mid, hi);
    t->nodes[id].axis = axis;
    t->nodes[id].split = split;
    t->nodes[id].left = l;
    t->nodes[id].right = r;
    return id;
}

orc_kdtree* orc_kdtree_build(const double* pts, long n)
{
    orc_kdtree* t = (orc_kdtree*)calloc(1, sizeof(orc_kdtree));
    t->pts = pts;
    t->n = n;
    t->perm = (int32_t*)malloc(sizeof(int32_t) * (n > 0 ? n : 1));
    for (long i = 0; i < n; ++i) t->perm[i] = (int32_t)i;
    if (n > 0) build_rec(t, 0, n);
    return t;
}

void orc_kdtree_free(orc_kdtree* t)
{
    if (!t) return;
    free(t->perm);
    free(t->nodes);
    free(t);
}

static double sqdist(const double* a, const double* b)
{
    double dx = a[0] - b[0], dy = a[1] - b[1], dz = a[2] - b[2];
    return dx * dx + dy * dy + dz * dz;
}

/* (d, i) strictly before (e, j) in the order "distance, then index". */
static int before(double d, int32_t i, double e, int32_t j) { return d < e || (d == e && i < j); }

/* Sorted candidate list of capacity k.  Slots beyond the filled count hold
 * (bound, INT32_MAX): a candidate enters only if it precedes the last slot. */
typedef struct {
    int k;
    double* d;
    int32_t* i;
} cand_list;

static void list_offer(cand_list* L, double d, int32_t i)
{
    int k = L->k;
    if (!before(d, i, L->d[k - 1], L->i[k - 1])) return;
    int pos = k - 1;
    while (pos > 0 && before(d, i, L->d[pos - 1], L->i[pos - 1])) {
        L->d[pos] = L->d[pos - 1];
        L->i[pos] = L->i[pos - 1];
        --pos;
    }
    L->d[pos] = d;
    L->i[pos] = i;
}

static void search_rec(const orc_kdtree* t, int id, const double* q, cand_list* L)
{
    const kd_node* nd = &t->nodes[id];
    if (nd->axis < 0) {
        for (long s = nd->lo; s < nd->hi; ++s) {
            int32_t pi = t->perm[s];
            list_offer(L, sqdist(q, t->pts + 3 * (long)pi), pi);
        }
        return;
    }
    double diff = q[nd->axis] - nd->split;
    int near_c = diff < 0 ? nd->left : nd->right;
    int far_c = diff < 0 ? nd->right : nd->left;
    search_rec(t, near_c, q, L);
    /* every point on the far side is at least |diff| away along this axis;
     * "<=" keeps equal-distance points with smaller indices reachable */
    if (diff * diff <= L->d[L->k - 1]) search_rec(t, far_c, q, L);
}

static void finish_row(int k, long n, const cand_list* L, int32_t* idx, double* d2)
{
    for (int j = 0; j < k; ++j) {
        if (j < n && L->i[j] != INT32_MAX) {
            idx[j] = L->i[j];
            d2[j] = L->d[j];
        } else {
            idx[j] = -1;
            d2[j] = INFINITY;
        }
    }
}

int orc_knn(const orc_kdtree* t, const double* queries, long q, int k, int32_t* idx, double* d2)
{
    if (k <= 0) return ORC_ERR_ARG;
#pragma omp parallel
    {
        double* bd = (double*)malloc(sizeof(double) * k);
        int32_t* bi = (int32_t*)malloc(sizeof(int32_t) * k);
#pragma omp for schedule(dynamic, 256)
        for (long s = 0; s < q; ++s) {
            cand_list L = {k, bd, bi};
            for (int j = 0; j < k; ++j) { bd[j] = INFINITY; bi[j] = INT32_MAX; }
            if (t->n > 0) search_rec(t, 0, queries + 3 * s, &L);
            finish_row(k, t->n, &L, idx + s * (long)k, d2 + s * (long)k);
        }
        free(bd);
        free(bi);
    }
    return ORC_OK;
}

int orc_knn_brute(const double* pts, long n, const double* queries, long q, int k, int32_t* idx,
                  double* d2)
{
    if (k <= 0) return ORC_ERR_ARG;
    double* bd = (double*)malloc(sizeof(double) * k);
    int32_t* bi = (int32_t*)malloc(sizeof(int32_t) * k);
    for (long s = 0; s < q; ++s) {
        cand_list L = {k, bd, bi};
        for (int j = 0; j < k; ++j) { bd[j] = INFINITY; bi[j] = INT32_MAX; }
        for (long i = 0; i < n; ++i) list_offer(&L, sqdist(queries + 3 * s, pts + 3 * i), (int32_t)i);
        finish_row(k, n, &L, idx + s * (long)k, d2 + s * (long)k);
    }
    free(bd);
    free(bi);
    return ORC_OK;
}

/* Nearest point within squared radius r2 of one query (idx -1 if none). */
static void nn_one(const orc_kdtree* t, const double* q, double r2, int32_t* idx, double* d2)
{
    double bd = r2;
    int32_t bi = INT32_MAX; /* the bound itself is admissible: d2 <= r2 */
    cand_list L = {1, &bd, &bi};
    if (t->n > 0) search_rec(t, 0, q, &L);
    *idx = bi == INT32_MAX ? -1 : bi;
    *d2 = bi == INT32_MAX ? INFINITY : bd;
}

int orc_nn(const orc_kdtree* t, const double* queries, long q, double r2, int32_t* idx, double* d2)
{
#pragma omp parallel for schedule(dynamic, 256)
    for (long s = 0; s < q; ++s) nn_one(t, queries + 3 * s, r2, idx + s, d2 + s);
    return ORC_OK;
}

int orc_nn_brute(const double* pts, long n, const double* queries, long q, double r2,
                 int32_t* idx, double* d2)
{
    for (long s = 0; s < q; ++s) {
        double bd = r2;
        int32_t bi = INT32_MAX;
        for (long i = 0; i < n; ++i) {
            double d = sqdist(queries + 3 * s, pts + 3 * i);
            if (before(d, (int32_t)i, bd, bi)) { bd = d; bi = (int32_t)i; }
        }
        idx[s] = bi == INT32_MAX ? -1 : bi;
        d2[s] = bi == INT32_MAX ? INFINITY : bd;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------------------------ */
/* 3x3 symmetric eigen-decomposition (cyclic Jacobi)                                          */
/* ------------------------------------------------------------------------------------------ */

void orc_eigh3(const double A6[6], double w[3], double V[9])
{
    double A[3][3] = {{A6[0], A6[1], A6[2]}, {A6[1], A6[3], A6[4]}, {A6[2], A6[4], A6[5]}};
    double Q[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    double scale = fabs(A6[0]) + fabs(A6[3]) + fabs(A6[5]) + fabs(A6[1]) + fabs(A6[2]) + fabs(A6[4]);
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = fabs(A[0][1]) + fabs(A[0][2]) + fabs(A[1][2]);
        if (off <= 1e-300 || off <= 1e-18 * scale) break;
        for (int p = 0; p < 2; ++p) {
            for (int q = p + 1; q < 3; ++q) {
                if (A[p][q] == 0.0) continue;
                /* rotation in the (p, q) plane that zeroes A[p][q] */
                double theta = (A[q][q] - A[p][p]) / (2.0 * A[p][q]);
                double tt = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(tt * tt + 1.0), s = tt * c;
                for (int r = 0; r < 3; ++r) { /* A <- A G */
                    double arp = A[r][p], arq = A[r][q];
                    A[r][p] = c * arp - s * arq;
                    A[r][q] = s * arp + c * arq;
                }
                for (int r = 0; r < 3; ++r) { /* A <- G^T A */
                    double apr = A[p][r], aqr = A[q][r];
                    A[p][r] = c * apr - s * aqr;
                    A[q][r] = s * apr + c * aqr;
                }
                for (int r = 0; r < 3; ++r) { /* Q <- Q G */
                    double qrp = Q[r][p], qrq = Q[r][q];
                    Q[r][p] = c * qrp - s * qrq;
                    Q[r][q] = s * qrp + c * qrq;
                }
            }
        }
    }
    int order[3] = {0, 1, 2};
    double d[3] = {A[0][0], A[1][1], A[2][2]};
    for (int i = 0; i < 3; ++i) /* sort ascending */
        for (int j = i + 1; j < 3; ++j)
            if (d[order[j]] < d[order[i]]) { int tmp = order[i]; order[i] = order[j]; order[j] = tmp; }
    for (int j = 0; j < 3; ++j) {
        w[j] = d[order[j]];
        for (int r = 0; r < 3; ++r) V[3 * r + j] = Q[r][order[j]];
    }
}

/* ------------------------------------------------------------------------------------------ */
/* source Gaussians                                                                           */
/* ------------------------------------------------------------------------------------------ */

static void sym_from_spectrum(const double V[9], const double lam[3], double out[6])
{
    /* out = V diag(lam) V^T */
    double M[3][3];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double s = 0;
            for (int j = 0; j < 3; ++j) s += V[3 * r + j] * lam[j] * V[3 * c + j];
            M[r][c] = s;
        }
    out[0] = M[0][0]; out[1] = M[0][1]; out[2] = M[0][2];
    out[3] = M[1][1]; out[4] = M[1][2]; out[5] = M[2][2];
}

int orc_regularise(const double C[6], int reg_mode, double eps, double out[6], double* gap)
{
    double w[3], V[9];
    orc_eigh3(C, w, V);
    if (gap) *gap = w[1] > 0 ? (w[1] - w[0]) / w[1] : 0.0;
    if (reg_mode == ORC_REG_NONE) {
        memcpy(out, C, sizeof(double) * 6);
        return 0;
    }
    if (!(w[2] > 0) || w[1] <= RANK_TOL * w[2]) { /* collinear or coincident neighbours */
        out[0] = 1; out[1] = 0; out[2] = 0; out[3] = 1; out[4] = 0; out[5] = 1;
        return ORC_FLAG_RANK_DEFICIENT;
    }
    if (reg_mode == ORC_REG_PLANE) {
        /* scales [1, 1, eps] on the principal axes: eigenvalues (eps, 1, 1) */
        double lam[3] = {eps, 1.0, 1.0};
        sym_from_spectrum(V, lam, out);
        return 0;
    }
    /* ellipse: Lambda' = Lambda / median(S)  ->  eigenvalues / middle eigenvalue */
    int flags = 0;
    double r0 = w[0] / w[1];
    if (r0 < eps) { r0 = eps; flags |= ORC_FLAG_FLOORED; }
    double lam[3] = {r0, 1.0, w[2] / w[1]};
    sym_from_spectrum(V, lam, out);
    return flags;
}

int orc_source_covariances(const double* pts, const double* z, long n, int k, double eps,
                           int reg_mode, double p, double* covs, double* raw, double* gap,
                           int32_t* flags)
{
    if (k <= 0 || n < 0 || (p != 0.0 && !z)) return ORC_ERR_ARG;
    if (n == 0) return ORC_OK;
    int kk = k < n ? k : (int)n;
    orc_kdtree* t = orc_kdtree_build(pts, n);
    int32_t* nb = (int32_t*)malloc(sizeof(int32_t) * n * (long)kk);
    double* nd = (double*)malloc(sizeof(double) * n * (long)kk);
    orc_knn(t, pts, n, kk, nb, nd);
#pragma omp parallel for schedule(dynamic, 256)
    for (long i = 0; i < n; ++i) {
        const int32_t* row = nb + i * (long)kk;
        /* two-pass covariance of the neighbourhood (the point itself included) */
        double mu[3] = {0, 0, 0};
        for (int j = 0; j < kk; ++j)
            for (int a = 0; a < 3; ++a) mu[a] += pts[3 * (long)row[j] + a];
        for (int a = 0; a < 3; ++a) mu[a] /= kk;
        double C[6] = {0, 0, 0, 0, 0, 0};
        for (int j = 0; j < kk; ++j) {
            const double* x = pts + 3 * (long)row[j];
            double e0 = x[0] - mu[0], e1 = x[1] - mu[1], e2 = x[2] - mu[2];
            C[0] += e0 * e0; C[1] += e0 * e1; C[2] += e0 * e2;
            C[3] += e1 * e1; C[4] += e1 * e2; C[5] += e2 * e2;
        }
        for (int a = 0; a < 6; ++a) C[a] /= kk;
        if (raw) memcpy(raw + 6 * i, C, sizeof(C));
        double out[6], g = 0.0;
        int f = 0;
        if (kk < 3) {
            f = ORC_FLAG_FEW_POINTS;
            if (reg_mode == ORC_REG_NONE) memcpy(out, C, sizeof(C));
            else { out[0] = 1; out[1] = 0; out[2] = 0; out[3] = 1; out[4] = 0; out[5] = 1; }
        } else {
            f = orc_regularise(C, reg_mode, eps, out, &g);
        }
        /* scale aligning: scales / z^p  ->  covariance * z^(-2p) */
        double s = p != 0.0 ? pow(z[i], -2.0 * p) : 1.0;
        for (int a = 0; a < 6; ++a) covs[6 * i + a] = out[a] * s;
        if (gap) gap[i] = g;
        if (flags) flags[i] = f;
    }
    free(nb);
    free(nd);
    orc_kdtree_free(t);
    return ORC_OK;
}

/* ------------------------------------------------------------------------------------------ */
/* poses                                                                                      */
/* ------------------------------------------------------------------------------------------ */

static void mat3_mul(const double A[9], const double B[9], double C[9])
{
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double s = 0;
            for (int j = 0; j < 3; ++j) s += A[3 * r + j] * B[3 * j + c];
            C[3 * r + c] = s;
        }
}

static void pose_split(const double T[16], double R[9], double t[3])
{
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c) R[3 * r + c] = T[4 * r + c];
        t[r] = T[4 * r + 3];
    }
}

static void rotate_sym(const double R[9], const double S6[6], double out[6])
{
    /* out = R S R^T */
    double S[9] = {S6[0], S6[1], S6[2], S6[1], S6[3], S6[4], S6[2], S6[4], S6[5]};
    double RS[9], M[9];
    mat3_mul(R, S, RS);
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double s = 0;
            for (int j = 0; j < 3; ++j) s += RS[3 * r + j] * R[3 * c + j];
            M[3 * r + c] = s;
        }
    out[0] = M[0]; out[1] = M[1]; out[2] = M[2]; out[3] = M[4]; out[4] = M[5]; out[5] = M[8];
}

void orc_transform_gaussians(const double T[16], const double* pts, const double* covs, long n,
                             double* pts_out, double* covs_out)
{
    double R[9], t[3];
    pose_split(T, R, t);
    for (long i = 0; i < n; ++i) {
        const double* x = pts + 3 * i;
        for (int r = 0; r < 3; ++r)
            pts_out[3 * i + r] = R[3 * r] * x[0] + R[3 * r + 1] * x[1] + R[3 * r + 2] * x[2] + t[r];
        if (covs && covs_out) rotate_sym(R, covs + 6 * i, covs_out + 6 * i);
    }
}

void orc_se3_exp(const double xi[6], double T[16])
{
    /* exp of the twist (omega, v): R = I + A K + B K^2, t = (I + B K + Cc K^2) v
     * with K = [omega]x, theta = |omega|, A = sin/theta, B = (1 - cos)/theta^2,
     * Cc = (theta - sin)/theta^3 (series below 1e-3 rad). */
    const double* w = xi;
    const double* v = xi + 3;
    double th2 = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
    double th = sqrt(th2);
    double A, B, Cc;
    if (th < 1e-3) {
        A = 1.0 - th2 / 6.0 + th2 * th2 / 120.0;
        B = 0.5 - th2 / 24.0 + th2 * th2 / 720.0;
        Cc = 1.0 / 6.0 - th2 / 120.0 + th2 * th2 / 5040.0;
    } else {
        double s = sin(th), h = sin(0.5 * th);
        A = s / th;
        B = 2.0 * h * h / th2;
        Cc = (th - s) / (th2 * th);
    }
    double K[9] = {0, -w[2], w[1], w[2], 0, -w[0], -w[1], w[0], 0};
    double K2[9];
    mat3_mul(K, K, K2);
    double R[9], Vm[9];
    for (int i = 0; i < 9; ++i) {
        double id = (i % 4 == 0) ? 1.0 : 0.0;
        R[i] = id + A * K[i] + B * K2[i];
        Vm[i] = id + B * K[i] + Cc * K2[i];
    }
    memset(T, 0, sizeof(double) * 16);
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c) T[4 * r + c] = R[3 * r + c];
        T[4 * r + 3] = Vm[3 * r] * v[0] + Vm[3 * r + 1] * v[1] + Vm[3 * r + 2] * v[2];
    }
    T[15] = 1.0;
}

static void pose_mul(const double A[16], const double B[16], double C[16])
{
    double M[16];
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) {
            double s = 0;
            for (int j = 0; j < 4; ++j) s += A[4 * r + j] * B[4 * j + c];
            M[4 * r + c] = s;
        }
    memcpy(C, M, sizeof(M));
}

/* ------------------------------------------------------------------------------------------ */
/* Gauss-Newton on Eq. (MLE_for_T)                                                            */
/* ------------------------------------------------------------------------------------------ */

void orc_residual_jacobian(const double T[16], const double x[3], const double mu[3], double d[3],
                           double J[18])
{
    double R[9], t[3], y[3];
    pose_split(T, R, t);
    for (int r = 0; r < 3; ++r) y[r] = R[3 * r] * x[0] + R[3 * r + 1] * x[1] + R[3 * r + 2] * x[2] + t[r];
    for (int r = 0; r < 3; ++r) d[r] = mu[r] - y[r];
    /* exp(xi) y ~ y + omega x y + v, so dd/domega = [y]x and dd/dv = -I */
    double Y[9] = {0, -y[2], y[1], y[2], 0, -y[0], -y[1], y[0], 0};
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c) {
            J[6 * r + c] = Y[3 * r + c];
            J[6 * r + 3 + c] = (r == c) ? -1.0 : 0.0;
        }
    }
}

static int inv_sym3(const double S[6], double W[6])
{
    double a = S[0], b = S[1], c = S[2], d = S[3], e = S[4], f = S[5];
    double c00 = d * f - e * e, c01 = c * e - b * f, c02 = b * e - c * d;
    double det = a * c00 + b * c01 + c * c02;
    if (!(fabs(det) > 0) || !isfinite(det)) return -1;
    W[0] = c00 / det;
    W[1] = c01 / det;
    W[2] = c02 / det;
    W[3] = (a * f - c * c) / det;
    W[4] = (b * c - a * e) / det;
    W[5] = (a * d - b * b) / det;
    return 0;
}

/* Add J^T W J, J^T W d and d^T W d of one correspondence to (H, b, cost). */
static void accumulate(const double T[16], const double x[3], const double mu[3], const double R[9],
                       const double Cs[6], const double Ct[6], double H[36], double b[6], double* cost)
{
    double d[3], J[18], RCs[6], Sig[6], W6[6];
    orc_residual_jacobian(T, x, mu, d, J);
    rotate_sym(R, Cs, RCs);
    for (int a = 0; a < 6; ++a) Sig[a] = Ct[a] + RCs[a];
    if (inv_sym3(Sig, W6) != 0) return;
    double W[9] = {W6[0], W6[1], W6[2], W6[1], W6[3], W6[4], W6[2], W6[4], W6[5]};
    double WJ[18], Wd[3];
    for (int r = 0; r < 3; ++r) {
        Wd[r] = W[3 * r] * d[0] + W[3 * r + 1] * d[1] + W[3 * r + 2] * d[2];
        for (int c = 0; c < 6; ++c)
            WJ[6 * r + c] = W[3 * r] * J[c] + W[3 * r + 1] * J[6 + c] + W[3 * r + 2] * J[12 + c];
    }
    for (int r = 0; r < 6; ++r) {
        for (int c = 0; c < 6; ++c)
            H[6 * r + c] += J[r] * WJ[c] + J[6 + r] * WJ[6 + c] + J[12 + r] * WJ[12 + c];
        b[r] += J[r] * Wd[0] + J[6 + r] * Wd[1] + J[12 + r] * Wd[2];
    }
    *cost += d[0] * Wd[0] + d[1] * Wd[1] + d[2] * Wd[2];
}

#define CHUNK 1024

int orc_linearise(const double* src, const double* covs_s, long n, const orc_kdtree* map_tree,
                  const double* map, const double* covs_t, const double T[16], double max_dist,
                  double H[36], double b[6], double* cost, long* inliers, int32_t* corr)
{
    double R[9], t[3];
    pose_split(T, R, t);
    long nchunks = (n + CHUNK - 1) / CHUNK;
    double* part = (double*)calloc((size_t)(nchunks > 0 ? nchunks : 1) * 44, sizeof(double));
    double r2 = max_dist * max_dist;
    /* per fixed-size chunk partial sums, then a serial sum over chunks: the
     * result is independent of how threads are scheduled */
#pragma omp parallel for schedule(dynamic, 1)
    for (long ch = 0; ch < nchunks; ++ch) {
        double* P = part + 44 * ch; /* H[36], b[6], cost, count */
        long end = (ch + 1) * CHUNK < n ? (ch + 1) * CHUNK : n;
        for (long i = ch * CHUNK; i < end; ++i) {
            const double* x = src + 3 * i;
            double y[3];
            for (int r = 0; r < 3; ++r) y[r] = R[3 * r] * x[0] + R[3 * r + 1] * x[1] + R[3 * r + 2] * x[2] + t[r];
            int32_t j;
            double dd;
            nn_one(map_tree, y, r2, &j, &dd);
            if (corr) corr[i] = j;
            if (j < 0) continue;
            accumulate(T, x, map + 3 * (long)j, R, covs_s + 6 * i, covs_t + 6 * (long)j, P, P + 36, P + 42);
            P[43] += 1.0;
        }
    }
    memset(H, 0, sizeof(double) * 36);
    memset(b, 0, sizeof(double) * 6);
    double c = 0, cnt = 0;
    for (long ch = 0; ch < nchunks; ++ch) {
        const double* P = part + 44 * ch;
        for (int a = 0; a < 36; ++a) H[a] += P[a];
        for (int a = 0; a < 6; ++a) b[a] += P[36 + a];
        c += P[42];
        cnt += P[43];
    }
    free(part);
    *cost = c;
    *inliers = (long)cnt;
    return ORC_OK;
}

static int cholesky_solve6(const double H[36], const double b[6], double x[6])
{
    double L[36] = {0};
    for (int i = 0; i < 6; ++i) {
        for (int j = 0; j <= i; ++j) {
            double s = H[6 * i + j];
            for (int k = 0; k < j; ++k) s -= L[6 * i + k] * L[6 * j + k];
            if (i == j) {
                if (!(s > 0) || !isfinite(s)) return -1;
                L[6 * i + i] = sqrt(s);
            } else {
                L[6 * i + j] = s / L[6 * j + j];
            }
        }
    }
    double y[6];
    for (int i = 0; i < 6; ++i) {
        double s = b[i];
        for (int k = 0; k < i; ++k) s -= L[6 * i + k] * y[k];
        y[i] = s / L[6 * i + i];
    }
    for (int i = 5; i >= 0; --i) {
        double s = y[i];
        for (int k = i + 1; k < 6; ++k) s -= L[6 * k + i] * x[k];
        x[i] = s / L[6 * i + i];
    }
    return 0;
}

/* One GN update from (H, b): delta = -H^-1 b, T <- exp(delta) T.  Returns 1 if
 * converged, 0 if not, -1 if H is not positive definite. */
static int gn_update(const double H[36], const double b[6], double T[16], const orc_reg_params* prm)
{
    double nb[6], delta[6], E[16];
    for (int a = 0; a < 6; ++a) nb[a] = -b[a];
    if (cholesky_solve6(H, nb, delta) != 0) return -1;
    orc_se3_exp(delta, E);
    pose_mul(E, T, T);
    double dw = sqrt(delta[0] * delta[0] + delta[1] * delta[1] + delta[2] * delta[2]);
    double dv = sqrt(delta[3] * delta[3] + delta[4] * delta[4] + delta[5] * delta[5]);
    return (dw < prm->tol_rot && dv < prm->tol_trans) ? 1 : 0;
}

int orc_gn_update(const double H[36], const double b[6], double T[16], const orc_reg_params* prm)
{
    return gn_update(H, b, T, prm);
}

int orc_register(const double* src, const double* covs_s, long n, const orc_kdtree* map_tree,
                 const double* map, const double* covs_t, const double T0[16],
                 const orc_reg_params* prm, double T_out[16], double H_out[36], double b_out[6],
                 int* iters, double* cost, long* inliers)
{
    double T[16], H[36], b[6], c = 0;
    long cnt = 0;
    memcpy(T, T0, sizeof(T));
    memset(H, 0, sizeof(H));
    memset(b, 0, sizeof(b));
    int status = ORC_OK, it = 0;
    while (it < prm->max_iters) {
        orc_linearise(src, covs_s, n, map_tree, map, covs_t, T, prm->max_corr_dist, H, b, &c, &cnt, NULL);
        ++it;
        if (cnt < prm->min_inliers) { status = ORC_ERR_DEGENERATE; break; }
        int r = gn_update(H, b, T, prm);
        if (r < 0) { status = ORC_ERR_DEGENERATE; break; }
        if (r == 1) break;
    }
    memcpy(T_out, T, sizeof(T));
    if (H_out) memcpy(H_out, H, sizeof(H));
    if (b_out) memcpy(b_out, b, sizeof(b));
    if (iters) *iters = it;
    if (cost) *cost = c;
    if (inliers) *inliers = cnt;
    return status;
}

int orc_register_fixed(const double* src, const double* covs_s, long n, const double* map,
                       const double* covs_t, const double T0[16], const orc_reg_params* prm,
                       double T_out[16], int* iters, double* cost)
{
    double T[16], R[9], t[3];
    memcpy(T, T0, sizeof(T));
    int status = ORC_OK, it = 0;
    double c = 0;
    while (it < prm->max_iters) {
        double H[36] = {0}, b[6] = {0};
        c = 0;
        pose_split(T, R, t);
        for (long i = 0; i < n; ++i) accumulate(T, src + 3 * i, map + 3 * i, R, covs_s + 6 * i, covs_t + 6 * i, H, b, &c);
        ++it;
        int r = gn_update(H, b, T, prm);
        if (r < 0) { status = ORC_ERR_DEGENERATE; break; }
        if (r == 1) break;
    }
    memcpy(T_out, T, sizeof(T));
    if (iters) *iters = it;
    if (cost) *cost = c;
    return status;
}

/* ------------------------------------------------------------------------------------------ */
/* threads                                                                                    */
/* ------------------------------------------------------------------------------------------ */

void orc_set_threads(int n) { omp_set_num_threads(n > 0 ? n : omp_get_num_procs()); }

int orc_threads(void) { return omp_get_max_threads(); }
