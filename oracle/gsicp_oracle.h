/*
 * gsicp_oracle.h -- FP64 CPU oracle for the G-ICP tracking path of
 * "RGBD GS-ICP SLAM" (Ha, Yeon, Yu; arXiv 2403.12550).
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the plain, slow, obviously
 * correct reference that the CUDA path is checked against.  Only the test
 * suite, the smoke check and the benchmark's CPU-baseline leg may load it.
 * It shares no code, header, table or helper with the CUDA library.
 *
 * All arithmetic is IEEE double.  Inputs are double arrays; callers that
 * hold float32 data widen it exactly before the call.
 *
 * Layouts: points n x 3 row-major (x, y, z); symmetric 3x3 matrices as 6
 * doubles (xx, xy, xz, yy, yz, zz); poses 4x4 row-major, T maps source
 * (camera) coordinates into map (world) coordinates.
 */
#ifndef GSICP_ORACLE_H
#define GSICP_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_OK = 0, ORC_ERR_ARG = 1, ORC_ERR_DEGENERATE = 4 };
enum { ORC_REG_PLANE = 0, ORC_REG_ELLIPSE = 1, ORC_REG_NONE = 2 };

/* Per-point flags written by orc_source_covariances. */
enum { ORC_FLAG_FEW_POINTS = 1, ORC_FLAG_RANK_DEFICIENT = 2, ORC_FLAG_FLOORED = 4 };

typedef struct orc_kdtree orc_kdtree;

/* Depth image -> point cloud (Sec. 3, Fig. 2: downsample + reproject). */
long orc_depth_to_points(const float* depth, int W, int H, const double intr[4], int stride,
                         double z_min, double z_max, double* pts, double* z, long cap);

/* k-d tree over n points (the array must outlive the tree). */
orc_kdtree* orc_kdtree_build(const double* pts, long n);
void orc_kdtree_free(orc_kdtree* t);

/* Exact k nearest neighbours of each query (ties -> smaller index).  Rows of
 * idx/d2 hold min(k, n) entries followed by -1 / +inf padding. */
int orc_knn(const orc_kdtree* t, const double* queries, long q, int k, int32_t* idx, double* d2);
int orc_knn_brute(const double* pts, long n, const double* queries, long q, int k, int32_t* idx,
                  double* d2);
/* Nearest neighbour with squared distance <= r2 (else idx -1, d2 +inf). */
int orc_nn(const orc_kdtree* t, const double* queries, long q, double r2, int32_t* idx, double* d2);
int orc_nn_brute(const double* pts, long n, const double* queries, long q, double r2,
                 int32_t* idx, double* d2);

/* Symmetric 3x3 eigen-decomposition by cyclic Jacobi: w ascending, V row-major
 * with column j the unit eigenvector of w[j]. */
void orc_eigh3(const double A[6], double w[3], double V[9]);

/* Source Gaussians (Sec. 3 covariance from k-NN; Sec. 3.1 scale
 * regularisation; Sec. 3.2 scale aligning).  z may be NULL when p == 0.
 * raw (n x 6), gap (n) and flags (n) may be NULL. */
int orc_source_covariances(const double* pts, const double* z, long n, int k, double eps,
                           int reg_mode, double p, double* covs, double* raw, double* gap,
                           int32_t* flags);
/* Regularise one covariance (Sec. 3.1); returns flags. */
int orc_regularise(const double C[6], int reg_mode, double eps, double out[6], double* gap);

/* y = R x + t, C' = R C R^T for n Gaussians (map insertion of a keyframe). */
void orc_transform_gaussians(const double T[16], const double* pts, const double* covs, long n,
                             double* pts_out, double* covs_out);

/* SE(3) exponential of xi = (omega, v), 4x4 row-major. */
void orc_se3_exp(const double xi[6], double T[16]);

/* One Gauss-Newton linearisation of Eq. (MLE_for_T) at pose T.  Outputs the
 * full 6x6 H (row-major), b (6), cost and inlier count; corr (n, nullable)
 * receives the map index matched to each source point (-1 if none). */
int orc_linearise(const double* src, const double* covs_s, long n, const orc_kdtree* map_tree,
                  const double* map, const double* covs_t, const double T[16], double max_dist,
                  double H[36], double b[6], double* cost, long* inliers, int32_t* corr);

/* Residual and analytic Jacobian of one correspondence at pose T:
 * d = mu - (R x + t), J = dd/dxi (3x6 row-major) for T <- exp(xi) T. */
void orc_residual_jacobian(const double T[16], const double x[3], const double mu[3], double d[3],
                           double J[18]);

typedef struct {
    double max_corr_dist;
    int max_iters;
    double tol_rot, tol_trans;
    int min_inliers;
} orc_reg_params;

/* One Gauss-Newton update of the registration loop (Sec. 3, Eq. (MLE_for_T); G-ICP's optimiser):
 * delta = -H^-1 b by Cholesky, T <- exp(delta^) T.  Returns 1 when |delta_omega| < tol_rot and
 * |delta_v| < tol_trans, 0 otherwise, -1 (T unchanged) when H is not positive definite. */
int orc_gn_update(const double H[36], const double b[6], double T[16], const orc_reg_params* prm);

/* Full registration (Gauss-Newton on Eq. MLE_for_T).  Returns ORC_OK or
 * ORC_ERR_DEGENERATE; T_out always holds the last valid pose. */
int orc_register(const double* src, const double* covs_s, long n, const orc_kdtree* map_tree,
                 const double* map, const double* covs_t, const double T0[16],
                 const orc_reg_params* prm, double T_out[16], double H_out[36], double b_out[6],
                 int* iters, double* cost, long* inliers);

/* Same Gauss-Newton, but source point i corresponds to map point i (no
 * search); used to pin the solver against closed forms. */
int orc_register_fixed(const double* src, const double* covs_s, long n, const double* map,
                       const double* covs_t, const double T0[16], const orc_reg_params* prm,
                       double T_out[16], int* iters, double* cost);

/* OpenMP threads used by the per-point loops from now on (n <= 0: all processors), and how many
 * that is.  Results do not depend on it. */
void orc_set_threads(int n);
int orc_threads(void);

#ifdef __cplusplus
}
#endif
#endif
