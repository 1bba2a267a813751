/*
 * gsicp.h -- C ABI of libgsicp.so: the G-ICP tracking hot path of
 * "RGBD GS-ICP SLAM" (Ha, Yeon, Yu; arXiv 2403.12550) on one B300 (sm_103a).
 *
 * Per frame the path is: depth image -> point cloud (Sec. 3, Fig. 2) ->
 * per-point k-NN covariances with scale regularisation (Sec. 3.1) and scale
 * aligning (Sec. 3.2) -> Gauss-Newton minimisation of Eq. (MLE_for_T) against
 * the target Gaussians of the map, with nearest-neighbour correspondences
 * re-searched at every iteration (Sec. 3).
 *
 * General conventions
 *   - Device pointers ("_dev") are CUDA global-memory addresses on the
 *     context's device, owned by the caller; the library never frees them.
 *     Host pointers ("_host" or plain arrays) are ordinary CPU memory.
 *   - Points are n x 3 float32 row-major (x, y, z).  Symmetric 3x3 matrices
 *     are 6 float32 (xx, xy, xz, yy, yz, zz).  Poses are 4x4 float64
 *     row-major; a pose T maps source (camera) coordinates into map (world)
 *     coordinates: p_w = R p_c + t.
 *   - Twists are ordered xi = (omega, v) and act on the left, T <- exp(xi^) T;
 *     the 6x6 H returned uses that order.
 *   - Every call is ordered on the caller's CUDA stream (`stream` is a
 *     cudaStream_t; NULL = legacy default stream).  Calls that return host
 *     values synchronise that stream once before returning.
 *   - A context owns reusable device scratch and the CUDA graphs of the
 *     Gauss-Newton loop; use one context from one host thread and one
 *     stream at a time.  Scratch grows on demand and is never shrunk; in the
 *     steady state no call allocates.
 *   - Errors are returned as gsicp_status; no function aborts or traps.  On
 *     GSICP_ERR_CUDA the CUDA error text is available from
 *     gsicp_last_error().
 */
#ifndef GSICP_H
#define GSICP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GSICP_OK = 0,
    GSICP_ERR_INVALID_ARG = 1,    /* null pointer, negative size, bad parameter */
    GSICP_ERR_CUDA = 2,           /* a CUDA runtime call failed (see gsicp_last_error) */
    GSICP_ERR_OOM = 3,            /* device allocation failed */
    GSICP_ERR_DEGENERATE = 4,     /* fewer than min_inliers correspondences, or H not positive definite */
    GSICP_ERR_TIMEOUT = 5,        /* a bounded device-side wait gave up */
    GSICP_ERR_NOT_IMPLEMENTED = 6,
    GSICP_ERR_CAPACITY = 7        /* an output buffer is too small for the result */
} gsicp_status;

typedef enum {
    GSICP_REG_PLANE = 0,   /* Sec. 3.1: scales [1, 1, eps] -> eigenvalues (eps, 1, 1) */
    GSICP_REG_ELLIPSE = 1, /* Sec. 3.1: Lambda' = Lambda / median(S) -> C / middle eigenvalue */
    GSICP_REG_NONE = 2     /* raw k-NN covariance (the unregularised row of Table 5) */
} gsicp_reg_mode;

/* Source-covariance parameters (Sec. 3, 3.1, 3.2). */
typedef struct {
    int k;          /* neighbours per point, the point itself included; 1 <= k <= 32 (paper: not stated; 20) */
    float eps;      /* plane/ellipse regularisation constant (1e-3) */
    int reg_mode;   /* gsicp_reg_mode */
    float p;        /* scale-aligning exponent: covariance *= z^(-2p); 0 disables (paper's best: 1.5, Table 6) */
} gsicp_cov_params;

/* Registration parameters (Sec. 3, Eq. MLE_for_T). */
typedef struct {
    float max_corr_dist; /* a source point has a correspondence iff its nearest map mean is within this distance (m) */
    int max_iters;       /* Gauss-Newton iteration cap (>= 1) */
    double tol_rot;      /* converged when |d omega| < tol_rot (rad) ... */
    double tol_trans;    /* ... and |d v| < tol_trans (m) */
    int min_inliers;     /* fewer correspondences than this -> GSICP_ERR_DEGENERATE */
} gsicp_reg_params;

/* Spatial-index parameters: a bounding-volume hierarchy over the Gaussians in Morton order, plus a
 * hash grid of the Morton cells for the common short-range searches. */
typedef struct {
    int bucket;          /* points per leaf: 8, 16 or 32 (0 = default 16) */
    float cell;          /* grid cell size in metres (0 = default 0.012); coarsened automatically
                            when 1024 cells per axis do not cover the map's bounding cube */
} gsicp_index_params;

typedef struct gsicp_ctx_s* gsicp_ctx;
typedef struct gsicp_map_s* gsicp_map;

/* ---------------------------------------------------------------------------------------------
 * Context and status
 * ------------------------------------------------------------------------------------------- */

/* Create a context on the current CUDA device.  *out receives the handle. */
gsicp_status gsicp_ctx_create(gsicp_ctx* out);
/* Free a context and all its scratch (synchronises the device first). NULL is ignored. */
void gsicp_ctx_destroy(gsicp_ctx ctx);
const char* gsicp_status_string(gsicp_status s);
/* Text of the last CUDA error seen by this library in the calling thread ("" if none). */
const char* gsicp_last_error(void);
/* Library version, e.g. "0.1.0". */
const char* gsicp_version(void);

/* Profiling: when enabled, gsicp_track_frame / gsicp_track_frame_host record CUDA events between
 * their phases, and gsicp_ctx_phase_times returns the device time (ms) of the last such frame:
 * out[0] a1 depth->points, out[1] source index build, out[2] k-NN covariances (with their
 * reordering; they run on a second stream of the context, beside the registration's seeds and
 * set-up on the call's stream), out[3] Gauss-Newton loop (from the covariances' end to the
 * registration's end), out[4] whole frame; out[5] = Gauss-Newton iterations.  Disabled by default
 * (no events are recorded). */
gsicp_status gsicp_ctx_set_timing(gsicp_ctx ctx, int enable);
/* The last registration's (or linearisation's) final linearisation: *sqdist_out = the sum over its
 * inlier correspondences of |mu - T x|^2 (squared Euclidean residuals, m^2), *inliers_out
 * (nullable) their count.  The tracker's fallback test uses sqrt(sqdist / inliers).  Valid after
 * the call that registered has returned; GSICP_ERR_INVALID_ARG before any registration. */
gsicp_status gsicp_ctx_last_residual(gsicp_ctx ctx, double* sqdist_out, int64_t* inliers_out);
/* Search tuning of this context's registrations (gsicp_register, gsicp_linearise,
 * gsicp_register_batch, gsicp_track_frame*): in each warp of 32 source points, when at most
 * max_per_warp of them need a walk of the map's tree in an iteration, the warp's 32 lanes walk for
 * each of them in turn (one query at a time, 32 boxes or points per step); otherwise each point
 * walks alone.  0 = always alone, 32 = always together.  Results do not depend on it (both walks
 * are exact); only time does.  Default 4.  GSICP_ERR_INVALID_ARG outside 0..32 or for a null ctx. */
gsicp_status gsicp_ctx_set_coop_walks(gsicp_ctx ctx, int max_per_warp);
/* Search tuning: in the first `iters` Gauss-Newton iterations of this context's registrations, a
 * warp in which more than the cooperative-walk threshold of points need a tree walk for their
 * nearest map point walks the tree once for all of them (a packet walk: a node is visited when any
 * of those points' bound reaches it; each point keeps its own nearest), instead of each point
 * walking alone.  It pays where the warp's points are close together and nearly all search, as in
 * the first iteration.  Results do not depend on it (every walk is exact).  Default 1; 0 = never.
 * GSICP_ERR_INVALID_ARG outside 0 .. 10000 or for a null ctx. */
gsicp_status gsicp_ctx_set_packet_iters(gsicp_ctx ctx, int iters);
/* Search tuning: a source point whose query moved more than `meters` since its last search
 * (Gauss-Newton iterations where the pose still moves a lot) searches for its nearest map point
 * alone; one that moved less builds a cache of its nearest map points and the radius within which
 * that list is complete, which later iterations check in place of a search while the point stays
 * within it (Sec. 3: correspondences are searched again each iteration).  Results do not depend
 * on it: every search and every cache check returns the nearest point by the same distance;
 * 0 = never build caches.  Default 0.0005 (0.5 mm).  GSICP_ERR_INVALID_ARG for a negative or
 * non-finite value or a null ctx. */
gsicp_status gsicp_ctx_set_cache_step(gsicp_ctx ctx, float meters);
/* How this context launches the Gauss-Newton iterations of gsicp_register and gsicp_track_frame*:
 * GSICP_GN_GRAPH (default) runs them as one CUDA graph whose conditional WHILE node repeats until
 * the last iteration's solve reports convergence (no host round trip per iteration);
 * GSICP_GN_PLAIN launches max_iters kernels on the stream, each a programmatic dependent of the
 * one before, and the launches after convergence exit at once.  The two give identical results;
 * PLAIN makes every iteration an ordinary kernel launch that launch-listing profilers see.
 * GSICP_ERR_INVALID_ARG for another value or a null ctx. */
typedef enum { GSICP_GN_GRAPH = 0, GSICP_GN_PLAIN = 1 } gsicp_gn_launch_mode;
gsicp_status gsicp_ctx_set_gn_launch_mode(gsicp_ctx ctx, int mode);
/* Source points per thread block of this context's Gauss-Newton iterations (gsicp_register,
 * gsicp_linearise, gsicp_track_frame*, the shard calls): 128, 256 (default) or 384, one point per
 * thread.  A block's points form one row of the reduction, so the block size
 * fixes the order of the sums: poses agree to rounding across sizes, and at 256 they equal
 * gsicp_register_batch's (whose work items are 256 points) bit for bit.  Takes effect at the next
 * registration.  GSICP_ERR_INVALID_ARG for another value or a null ctx. */
gsicp_status gsicp_ctx_set_gn_block(gsicp_ctx ctx, int points_per_block);
gsicp_status gsicp_ctx_phase_times(gsicp_ctx ctx, double out[6]);

/* Telemetry of the last frame whose covariances this context computed (gsicp_frame_covariances,
 * gsicp_track_frame*): out[0] the number of points the 9 x 9 window did not certify (searched in
 * the 25 x 25 window), out[1] those that window did not certify either (searched in the tree).
 * Synchronises the device. */
gsicp_status gsicp_ctx_frame_stats(gsicp_ctx ctx, int64_t out[2]);

/* Telemetry of the last registration on this context (gsicp_register, gsicp_track_frame*): for
 * each of the first min(n, 64) Gauss-Newton iterations, the number of source points whose cached
 * map candidates had to be searched again (refreshes_out), the device time in ns from the first
 * block's start to the last block's arrival at the reduction (main_ns_out), of the final
 * reduction and solve by the last block (tail_ns_out) and of the FP64 solve and pose update alone
 * (solve_ns_out).  Any output may be NULL. */
gsicp_status gsicp_ctx_reg_stats(gsicp_ctx ctx, int n, int32_t* refreshes_out, int32_t* tail_ns_out,
                                 int32_t* solve_ns_out, int32_t* main_ns_out);

/* ---------------------------------------------------------------------------------------------
 * a1  Depth image -> point cloud   (Sec. 3, Fig. 2: "downsampling and reprojecting the depth image")
 *
 * Every stride-th pixel (u, v) = (stride*i, stride*j) of the W x H float32 depth image
 * (metres, row-major) is kept iff its depth d is finite and z_min <= d <= z_max, and
 * back-projected to ((u - cx) d / fx, (v - cy) d / fy, d), intr = {fx, fy, cx, cy}.
 * Kept points are written in row-major pixel order to pts_dev (cap x 3) and their depth to
 * z_dev (cap, may be NULL).  The count goes to n_dev (device int32, may be NULL) and, if
 * n_host is non-NULL, to *n_host after a stream synchronisation.  If more than cap points
 * survive, GSICP_ERR_CAPACITY is returned (only detectable when n_host is given) and at most
 * cap points are written.
 * ------------------------------------------------------------------------------------------- */
gsicp_status gsicp_depth_to_points(gsicp_ctx ctx, const float* depth_dev, int W, int H,
                                   const float intr[4], int stride, float z_min, float z_max,
                                   float* pts_dev, float* z_dev, int64_t cap, int32_t* n_dev,
                                   int64_t* n_host, void* stream);

/* Allocation-free variant of gsicp_depth_to_points (the paper has no counterpart: this is a
 * deployment aid).  For callers that must not allocate device memory when they need the result:
 * a tracking loop with a hard per-frame deadline (cudaMalloc / cudaFree may synchronise the
 * device and take an unbounded time), an application whose own memory pool owns the device, or
 * code that may not allocate after initialisation.  No context is needed and nothing is
 * allocated: the step's scratch (128 KB) is a fixed array inside the library, present on every
 * GPU that loads it until the process exits.  Same arguments and results as
 * gsicp_depth_to_points, except that the count goes to n_dev (device int32, required) and the
 * count before clamping to cap to total_dev (device int32, nullable); nothing is synchronised.
 * The sampled grid ceil(W/stride) * ceil(H/stride) may hold at most 4194304 pixels; larger
 * images are rejected with GSICP_ERR_INVALID_ARG, as are NULL required pointers, non-positive
 * sizes and a zero focal length (each with a message in gsicp_last_error()).  The first call in
 * a device's context looks up the array's device address (cached per device with the context's
 * id; a new context, e.g. after cudaDeviceReset, is looked up again on its first call, and a
 * failed lookup is not cached); make that first call before any stream capture.  All calls on a
 * device share the array and it keeps the last call's contents (every entry a call reads is
 * written by that call first): calls that may overlap on the GPU (e.g. on unordered streams)
 * race on it and must be serialised by the caller. */
gsicp_status gsicp_depth_to_points_noalloc(const float* depth_dev, int W, int H, const float intr[4],
                                           int stride, float z_min, float z_max, float* pts_dev,
                                           float* z_dev, int64_t cap, int32_t* n_dev,
                                           int32_t* total_dev, void* stream);

/* ---------------------------------------------------------------------------------------------
 * a2+a3  Source Gaussians   (Sec. 3: covariance of the k nearest neighbours; Sec. 3.1 scale
 * regularisation; Sec. 3.2 scale aligning)
 *
 * For each of the n points (pts_dev, n x 3): its k nearest neighbours among the n points by
 * squared Euclidean distance, the point itself included, ties broken by smaller index; the
 * covariance C = (1/k) sum (x_j - mu)(x_j - mu)^T of those neighbours; C' by the
 * regularisation of params->reg_mode; C'' = C' * z^(-2p) with z = z_dev[i] (z_dev may be NULL
 * when p == 0).  Fewer than 3 points, or a line-like neighbourhood (middle eigenvalue <= 1e-5
 * x largest) under PLANE/ELLIPSE, give C' = I.  ELLIPSE floors the smallest eigenvalue ratio at
 * eps.  Writes covs_dev (n x 6).  If knn_dev is non-NULL it receives the neighbour indices
 * (n x k int32, nearest first; -1 padding when n < k).
 * ------------------------------------------------------------------------------------------- */
gsicp_status gsicp_source_covariances(gsicp_ctx ctx, const float* pts_dev, const float* z_dev,
                                      int64_t n, const gsicp_cov_params* params, float* covs_dev,
                                      int32_t* knn_dev, void* stream);

/* a1 + a2 + a3 of one depth frame in one call (Sec. 3, Fig. 2; Sec. 3.1; Sec. 3.2): the frame's
 * points exactly as gsicp_depth_to_points writes them (row-major, pts_dev cap x 3, z_dev cap,
 * nullable) and their Gaussians exactly as gsicp_source_covariances of those points would give
 * them (covs_dev cap x 6, same order, same neighbour sets and ties).  The k-NN search uses the
 * image: for the point of sample (i, j) it takes the k nearest among the 9 x 9 samples around it,
 * and that answer is exact when the k-th is nearer than the four planes through the camera
 * centre that bound the samples outside the window; the other points are searched in a tree.
 * *n_out (host) receives the number of points after a stream synchronisation; more than cap
 * points give GSICP_ERR_CAPACITY with the first cap written (points, depths and covariances of
 * the whole frame are computed, the covariances use all of them). */
gsicp_status gsicp_frame_covariances(gsicp_ctx ctx, const float* depth_dev, int W, int H,
                                     const float intr[4], int stride, float z_min, float z_max,
                                     const gsicp_cov_params* params, float* pts_dev, float* z_dev,
                                     float* covs_dev, int64_t cap, int64_t* n_out, void* stream);

/* ---------------------------------------------------------------------------------------------
 * a4  Map index   (target Gaussians G^t = {X^t, C^t}, Sec. 3)
 *
 * Builds the spatial index over m map Gaussians (means_dev m x 3, covs_dev m x 6) and keeps a
 * packed, index-ordered copy of both, so the caller's buffers may be reused after the call.
 * *out receives a handle owned by the caller (free with gsicp_map_destroy).  params may be NULL.
 * ------------------------------------------------------------------------------------------- */
gsicp_status gsicp_build_map_index(gsicp_ctx ctx, const float* means_dev, const float* covs_dev,
                                   int64_t m, const gsicp_index_params* params, void* stream,
                                   gsicp_map* out);
/* Append m_add Gaussians to a map and rebuild its index (keyframe insertion, Fig. 2). */
gsicp_status gsicp_map_append(gsicp_ctx ctx, gsicp_map map, const float* means_dev,
                              const float* covs_dev, int64_t m_add, void* stream);
/* Rebuild a map's index over the Gaussians it already holds (the a4 step alone; no allocation
 * once the map exists).  Stream-ordered, no synchronisation. */
gsicp_status gsicp_map_rebuild(gsicp_ctx ctx, gsicp_map map, void* stream);
/* Introspection of a map's index (tests and tools).  pts_dev (nullable) receives the index-ordered
 * means as 4 float32 per Gaussian (x, y, z, original index as int32 bits); boxes_dev (nullable)
 * receives the axis-aligned boxes of the 2L heap nodes (node i: lo.xyz, 0, hi.xyz, 0; node 1 is
 * the root, nodes L..2L-1 the leaves, node 0 unused); *n_leaves_out = L, *bucket_out = points per
 * leaf.  Stream-ordered, no synchronisation. */
gsicp_status gsicp_map_inspect(gsicp_map map, float* pts_dev, float* boxes_dev, int64_t* n_leaves_out,
                               int* bucket_out, void* stream);
/* Number of Gaussians in a map. */
int64_t gsicp_map_size(gsicp_map map);
void gsicp_map_destroy(gsicp_map map);

/* Helper for map insertion: y = R x + t and C' = R C R^T for n Gaussians (covs may be NULL). */
gsicp_status gsicp_transform_gaussians(const double T[16], const float* pts_dev,
                                       const float* covs_dev, int64_t n, float* pts_out_dev,
                                       float* covs_out_dev, void* stream);

/* ---------------------------------------------------------------------------------------------
 * a5-a7  Registration   (Sec. 3: d_i = x^t_i - T x^s_i ~ N(0, C^t_i + T C^s_i T^T);
 * Eq. MLE_for_T minimised by Gauss-Newton)
 *
 * Starting from T0, each iteration: y_i = R x_i + t; j* = nearest map mean (ties -> smaller map
 * index) with |mu_j* - y_i| <= max_corr_dist, else no correspondence; d_i = mu_j* - y_i;
 * W_i = (C^t_j* + R C^s_i R^T)^-1; J_i = [[y_i]x, -I]; H = sum J^T W J, b = sum J^T W d,
 * cost = sum d^T W d.  Then delta = -H^-1 b (FP64 Cholesky) and T <- exp(delta^) T (FP64).
 * Stops when |d omega| < tol_rot and |d v| < tol_trans, or after max_iters iterations (not an
 * error: *iters_out == max_iters).
 *
 * Outputs (host): T_out[16] final pose; H_out[36] (nullable) and b_out[6] (nullable) of the last
 * linearisation; iters_out, cost_out (cost at the last linearisation), inliers_out (its
 * correspondence count); all nullable except T_out.  GSICP_ERR_DEGENERATE leaves T_out at the
 * last valid pose.  Synchronises the stream.
 * ------------------------------------------------------------------------------------------- */
gsicp_status gsicp_register(gsicp_ctx ctx, const float* src_pts_dev, const float* src_covs_dev,
                            int64_t n, gsicp_map map, const double T0[16],
                            const gsicp_reg_params* params, double T_out[16], double H_out[36],
                            double b_out[6], int* iters_out, double* cost_out,
                            int64_t* inliers_out, void* stream);

/* ---------------------------------------------------------------------------------------------
 * One registration split across processes (Sec. 3, Eq. (MLE_for_T): the cost and its Gauss-Newton
 * system are sums over the correspondences, so each process can take a share of the source
 * points and the shares' sums add up to the whole registration's).
 *
 * Every process holds the whole map (its own gsicp_map) and a share of the source points:
 *   gsicp_shard_begin      sets up this context's registration of its share from T0 (Morton order,
 *                          first-iteration seeds, candidate cache), stream-ordered;
 *   gsicp_shard_linearise  linearises at the current pose and writes the share's GSICP_SHARD_SUMS
 *                          FP64 sums to partial_dev (device), stream-ordered: entries 0..20 the
 *                          upper triangle of H row by row ((0,0), (0,1), .., (0,5), (1,1), ..),
 *                          21..26 b, 27 the cost, 28 the correspondence count, 29 the sum of the
 *                          correspondences' squared distances;
 *   (the caller gathers every process's partial, e.g. an all-gather of GSICP_SHARD_SUMS doubles)
 *   gsicp_shard_update     sums the nparts rows of sums_dev (nparts x GSICP_SHARD_SUMS, device) in
 *                          row order, solves H delta = -b in FP64 and updates the pose as
 *                          gsicp_register does, synchronises the stream and reports *status_out:
 *                          GSICP_SHARD_RUNNING (linearise again), _CONVERGED, _MAXITER or
 *                          _DEGENERATE (fewer than min_inliers correspondences in all, or H not
 *                          positive definite; the call then returns GSICP_ERR_DEGENERATE).
 * Processes that pass the same rows in the same order compute the same bits, so every process
 * holds the same pose after every update.  T_out, H_out, iters_out, cost_out and inliers_out are
 * nullable host outputs as in gsicp_register (H, cost and inliers of the whole, last
 * linearisation).  Any other registration on the same context (gsicp_register, gsicp_linearise,
 * gsicp_track_frame*) ends the shard registration; linearise / update without a begun one return
 * GSICP_ERR_INVALID_ARG.
 * ------------------------------------------------------------------------------------------- */
#define GSICP_SHARD_SUMS 30
typedef enum { GSICP_SHARD_RUNNING = 0, GSICP_SHARD_CONVERGED = 1, GSICP_SHARD_MAXITER = 2,
               GSICP_SHARD_DEGENERATE = 3 } gsicp_shard_status;
gsicp_status gsicp_shard_begin(gsicp_ctx ctx, const float* src_pts_dev, const float* src_covs_dev,
                               int64_t n, gsicp_map map, const double T0[16],
                               const gsicp_reg_params* params, void* stream);
gsicp_status gsicp_shard_linearise(gsicp_ctx ctx, double* partial_dev, void* stream);
gsicp_status gsicp_shard_update(gsicp_ctx ctx, const double* sums_dev, int nparts, int* status_out,
                                double T_out[16], double H_out[36], int* iters_out, double* cost_out,
                                int64_t* inliers_out, void* stream);

/* Batched registration (NEXT row of the hot path: many independent registrations at once; the
 * paper registers one frame at a time).  B pairs, each exactly as gsicp_register would register
 * it: source b (src_pts_dev[b], n[b] x 3, with covariances src_covs_dev[b], n[b] x 6) against map
 * maps[b] from pose T0[16 b .. 16 b + 15], all with the same params.  The host arrays hold B
 * device pointers / counts / handles.  All pairs run in one persistent launch that takes
 * (pair, 256-point chunk) work items from a device queue: each pair advances through its own
 * iterations, the pair's solve enqueueing its next iteration, and each pair's sums are taken in
 * the same order as gsicp_register's, so each T_out equals what gsicp_register returns for that
 * pair alone.  Outputs (host, B entries each, all but T_out nullable): T_out (B x 16), iters_out,
 * cost_out, inliers_out, status_out (GSICP_OK, or GSICP_ERR_DEGENERATE for that pair: fewer than
 * min_inliers correspondences, H not positive definite, or no points).  Returns GSICP_OK, an
 * argument / CUDA error, or GSICP_ERR_TIMEOUT if a bounded wait of the work queue ran out.
 * Synchronises the stream. */
gsicp_status gsicp_register_batch(gsicp_ctx ctx, int B, const float* const* src_pts_dev,
                                  const float* const* src_covs_dev, const int64_t* n,
                                  const gsicp_map* maps, const double* T0,
                                  const gsicp_reg_params* params, double* T_out, int* iters_out,
                                  double* cost_out, int64_t* inliers_out, int* status_out,
                                  void* stream);

/* Self-test of the batch queue's bounded wait (no counterpart in the paper): runs the batch
 * kernel on a queue that claims one pair is running but never receives an item, so every
 * block's wait runs out after about a second.  Returns GSICP_ERR_TIMEOUT when the bound works
 * (the context stays usable), GSICP_OK if the waits somehow ended without it. */
gsicp_status gsicp_selftest_batch_timeout(gsicp_ctx ctx, void* stream);

/* One linearisation at pose T (no update): H (6x6), b, cost and inlier count as in
 * gsicp_register's first iteration.  corr_dev (n int32, nullable) receives each source point's
 * map index (-1 if none).  Synchronises the stream. */
gsicp_status gsicp_linearise(gsicp_ctx ctx, const float* src_pts_dev, const float* src_covs_dev,
                             int64_t n, gsicp_map map, const double T[16], float max_corr_dist,
                             double H_out[36], double b_out[6], double* cost_out,
                             int64_t* inliers_out, int32_t* corr_dev, void* stream);

/* Nearest map mean of each of q query points (queries_dev q x 3, map frame) within max_dist:
 * idx_dev (q int32, -1 if none, ties -> smaller index) and d2_dev (q float32 squared
 * distances, +inf if none; nullable).  Stream-ordered, no synchronisation. */
gsicp_status gsicp_map_nearest(gsicp_ctx ctx, gsicp_map map, const float* queries_dev, int64_t q,
                               float max_dist, int32_t* idx_dev, float* d2_dev, void* stream);

/* ---------------------------------------------------------------------------------------------
 * One whole tracking frame: a1 -> a2+a3 -> a5-a7 with every intermediate kept on the device
 * (one stream synchronisation at the end).  Same semantics as calling gsicp_depth_to_points,
 * gsicp_source_covariances (z = the points' depth) and gsicp_register in sequence.
 * depth_dev is a device image; gsicp_track_frame_host takes a host image (pinned memory for an
 * asynchronous copy), of which only the rows a1 samples (every stride-th, ceil(H / stride) x W
 * floats) are uploaded inside the call, on a stream of the context's own so that the copy overlaps
 * work the caller queued on `stream` before the call (a map-index rebuild, say); `stream` waits for
 * the upload before the frame's first kernel.  n_points_out (nullable) receives the frame's point
 * count.
 * ------------------------------------------------------------------------------------------- */
gsicp_status gsicp_track_frame(gsicp_ctx ctx, const float* depth_dev, int W, int H,
                               const float intr[4], int stride, float z_min, float z_max,
                               const gsicp_cov_params* cov_params, gsicp_map map,
                               const double T0[16], const gsicp_reg_params* reg_params,
                               double T_out[16], double H_out[36], int* iters_out,
                               double* cost_out, int64_t* inliers_out, int64_t* n_points_out,
                               void* stream);
gsicp_status gsicp_track_frame_host(gsicp_ctx ctx, const float* depth_host, int W, int H,
                                    const float intr[4], int stride, float z_min, float z_max,
                                    const gsicp_cov_params* cov_params, gsicp_map map,
                                    const double T0[16], const gsicp_reg_params* reg_params,
                                    double T_out[16], double H_out[36], int* iters_out,
                                    double* cost_out, int64_t* inliers_out,
                                    int64_t* n_points_out, void* stream);

/* ---------------------------------------------------------------------------------------------
 * Tracking loop with the paper's keyframe policy (NEXT row around the hot path).
 *
 * Sec. 3 Keyframe Selection: a frame whose proportion of correspondences with the map (inliers /
 * points) falls below min_inlier_ratio becomes a keyframe; of its Gaussians only those that do not
 * overlap the map (no map mean within overlap_radius) are added.  Sec. 3 Additional Keyframe
 * Selection for Mapping: the force_every-th frame after a keyframe becomes one if none was
 * selected before (30 in the paper), and every mapping_every-th frame after a keyframe (10) is a
 * mapping-only keyframe: its new Gaussians go to the mapping map only.  Tracking registers against
 * the tracking map (keyframes only); the mapping map holds keyframes and mapping-only keyframes.
 * The paper gives no threshold values for the ratio or the overlap: min_inlier_ratio = 0.85 and
 * overlap_radius = 0.01 m are this library's readings.
 * ------------------------------------------------------------------------------------------- */
typedef struct {
    float min_inlier_ratio;  /* keyframe when inliers / points < this */
    int force_every;         /* keyframe at this many frames after the last one at the latest */
    int mapping_every;       /* mapping-only keyframe every this many frames after a keyframe (0: none) */
    float overlap_radius;    /* m: a Gaussian with a map mean this close is not added */
} gsicp_keyframe_params;

typedef enum { GSICP_FRAME = 0, GSICP_KEYFRAME = 1, GSICP_MAPPING_KEYFRAME = 2 } gsicp_frame_kind;

typedef struct {
    int kind;               /* gsicp_frame_kind */
    int status;             /* the frame's registration status (GSICP_OK or GSICP_ERR_DEGENERATE) */
    int iters;              /* Gauss-Newton iterations (0 for the first frame) */
    int64_t n_points;       /* points of the frame */
    int64_t inliers;        /* correspondences of the last linearisation */
    double inlier_ratio;    /* inliers / n_points */
    int64_t added_tracking; /* Gaussians added to the tracking map */
    int64_t added_mapping;  /* Gaussians added to the mapping map */
    int cov_source;         /* covariances of the accepted registration: 0 k-NN, 1 the surrogate's */
    int fell_back;          /* 1: the surrogate's registration was rejected, the frame re-tracked with k-NN */
    double residual;        /* RMS distance (m) of the accepted registration's inlier correspondences */
} gsicp_frame_info;

typedef struct gsicp_tracker_s* gsicp_tracker;
typedef struct gsicp_surrogate_s* gsicp_surrogate;  /* see "Learned covariance surrogate" below */

/* A tracker on ctx (the ctx must outlive it); frames are taken with the given stride and depth
 * range, covariances and registrations with cov / reg. */
gsicp_status gsicp_tracker_create(gsicp_ctx ctx, int stride, float z_min, float z_max,
                                  const gsicp_cov_params* cov, const gsicp_reg_params* reg,
                                  const gsicp_keyframe_params* kf, gsicp_tracker* out);
void gsicp_tracker_destroy(gsicp_tracker t);
/* Tracks one depth frame (device, W x H float32 metres).  The first frame needs T_start (its
 * pose) and becomes a keyframe; later frames start from T_start if given, else from the
 * constant-velocity prediction T_{f-1} (T_{f-2}^-1 T_{f-1}) (T_{f-1} for the second frame).
 * T_out (host) receives the frame's pose, *info (nullable) what happened.  Returns the
 * registration's status (GSICP_ERR_DEGENERATE: the frame is not used and T_out holds the last
 * valid pose of its registration).  Synchronises the stream. */
gsicp_status gsicp_tracker_frame(gsicp_tracker t, const float* depth_dev, int W, int H,
                                 const float intr[4], const double* T_start, double T_out[16],
                                 gsicp_frame_info* info, void* stream);
/* Track with a learned surrogate's covariances (sg null: k-NN covariances only, the default).
 * The first tracked frame and then every calib_every-th (>= 1) are calibration frames, tracked
 * with k-NN covariances; their residual (RMS distance of the inlier correspondences at the final
 * pose, a measure that does not depend on the covariances) is the reference.  Every other frame is
 * tracked with the surrogate's covariances, and when that registration fails or its residual
 * exceeds fallback_ratio times the reference, the frame is tracked again from the same start with
 * k-NN covariances (and becomes the new reference).  A keyframe adds to the maps the covariances of
 * its accepted registration (keyframe_knn = 0) or, when that was the surrogate's, its k-NN
 * covariances computed then (keyframe_knn = 1: the maps hold k-NN covariances only).  sg must
 * outlive its use by the tracker. */
gsicp_status gsicp_tracker_set_surrogate(gsicp_tracker t, gsicp_surrogate sg, float fallback_ratio,
                                         int calib_every, int keyframe_knn);
/* The tracker's maps (owned by the tracker; NULL before the first frame). */
gsicp_status gsicp_tracker_maps(gsicp_tracker t, gsicp_map* tracking_map, gsicp_map* mapping_map);

/* ---------------------------------------------------------------------------------------------
 * Learned covariance surrogate.  A small convolutional network over the stride-sampled point map
 * of a depth frame predicts each point's surface normal n; the point's Gaussian is then the
 * plane-regularised, scale-aligned covariance of Sec. 3 built on it, (I - (1 - eps) n n^T)
 * z^(-2p), in place of the k-NN covariance (a2 + a3).  Network: layer 1 maps the centred
 * differences M(u+d) (P(u+d) - P(u)) of the 5 x 5 samples around u (P the back-projected sample,
 * M its validity) to 32 channels, layer 2 is a 5 x 5 convolution 32 -> 32, layer 3 a 5 x 5
 * convolution 32 -> 3 giving v, n = v / |v| (|v| = 0: isotropic z^(-2p) I); no biases; ReLU and
 * bfloat16 rounding after layers 1 and 2, zero at invalid samples; taps read (i + dy - 2,
 * j + dx - 2), zero outside the image.  Weights are bfloat16 (the float weights rounded to
 * nearest even); every sum is float.  Weight vector layout (GSICP_SURROGATE_WEIGHTS floats):
 * W1[32][3][5][5], W2[32][32][5][5], W3[3][32][5][5] ([out][in][dy][dx]).
 * ------------------------------------------------------------------------------------------- */
#define GSICP_SURROGATE_WEIGHTS 30400

/* A surrogate with the given weights (host, GSICP_SURROGATE_WEIGHTS floats) on the current
 * device; Adam state zero.  Synchronises the device's default stream. */
gsicp_status gsicp_surrogate_create(const float* weights, gsicp_surrogate* out);
void gsicp_surrogate_destroy(gsicp_surrogate sg);
/* Profiling: with timing enabled, every forward of the network records CUDA events on its stream
 * between its layers; gsicp_surrogate_layer_times returns the device time (ms) of the last one
 * (after a synchronisation): out[0] grid + layer 1, out[1] layer 2, out[2] layer 3 + covariances.
 * GSICP_ERR_INVALID_ARG before timing was ever enabled. */
gsicp_status gsicp_surrogate_set_timing(gsicp_surrogate sg, int enable);
gsicp_status gsicp_surrogate_layer_times(gsicp_surrogate sg, double out[3]);
/* Copy the current float weights out (host) / replace them (host; resets the Adam state). */
gsicp_status gsicp_surrogate_get_weights(gsicp_surrogate sg, float* weights);
gsicp_status gsicp_surrogate_set_weights(gsicp_surrogate sg, const float* weights);

/* a1 + the surrogate's covariances of one depth frame: points as gsicp_depth_to_points writes
 * them (pts_dev cap x 3, z_dev nullable) and their covariances (covs_dev cap x 6, same order)
 * from params->eps and params->p (k and reg_mode unused).  v_dev (nullable, device,
 * ceil(H/stride) x ceil(W/stride) x 3 floats): the network's raw output per sample, zero at
 * invalid samples.  *n_out as gsicp_frame_covariances (synchronises; GSICP_ERR_CAPACITY when the
 * frame has more than cap points). */
gsicp_status gsicp_surrogate_covariances(gsicp_ctx ctx, gsicp_surrogate sg, const float* depth_dev, int W, int H,
                                         const float intr[4], int stride, float z_min, float z_max,
                                         const gsicp_cov_params* params, float* pts_dev, float* z_dev,
                                         float* covs_dev, float* v_dev, int64_t cap, int64_t* n_out, void* stream);

/* One training step on one depth frame.  Targets: target_covs_dev (device, the frame's points'
 * plane-regularised covariances in a1 order, cap x 6) or, when null, the frame's own k-NN
 * covariances from params (reg_mode must then be GSICP_REG_PLANE).  Loss: the mean over points
 * whose target is a plane covariance (T = (I - C z^(2p)) / (1 - eps) with trace within 0.01 of
 * 1) of 1 - n^T T n.  Gradients by back-propagation, the bfloat16 roundings taken as the
 * identity.  apply = 1: one Adam step (b1 0.9, b2 0.999, eps 1e-8, learning rate lr) on the
 * float weights; apply = 0: weights and Adam state untouched.  loss_out, count_out (targets used)
 * and grad_out (host, GSICP_SURROGATE_WEIGHTS floats: the gradient of the mean) are nullable.
 * Synchronises the stream. */
gsicp_status gsicp_surrogate_train_step(gsicp_ctx ctx, gsicp_surrogate sg, const float* depth_dev, int W, int H,
                                        const float intr[4], int stride, float z_min, float z_max,
                                        const gsicp_cov_params* params, const float* target_covs_dev, float lr,
                                        int apply, double* loss_out, int64_t* count_out, float* grad_out,
                                        void* stream);

/* gsicp_track_frame with the surrogate's covariances in place of the k-NN ones (cov_params
 * supplies eps and p). */
gsicp_status gsicp_track_frame_surrogate(gsicp_ctx ctx, gsicp_surrogate sg, const float* depth_dev, int W, int H,
                                         const float intr[4], int stride, float z_min, float z_max,
                                         const gsicp_cov_params* cov_params, gsicp_map map, const double T0[16],
                                         const gsicp_reg_params* reg_params, double T_out[16], double H_out[36],
                                         int* iters_out, double* cost_out, int64_t* inliers_out,
                                         int64_t* n_points_out, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* GSICP_H */
