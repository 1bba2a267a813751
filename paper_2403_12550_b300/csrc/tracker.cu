// tracker.cu -- the tracking loop around the hot path: keyframe selection and map growth.
//
// Sec. 3 (Keyframe Selection): a frame whose proportion of correspondences with the map falls
// below a threshold becomes a keyframe, and only those of its Gaussians that do not overlap the
// existing map are added to it.  Sec. 3 (Additional Keyframe Selection for Mapping): if no
// keyframe was selected up to the 30th frame after the last one, that frame becomes a keyframe,
// and every 10th frame after a keyframe is a mapping-only keyframe, whose Gaussians go to the map
// used for mapping but not to the one tracking registers against.  Tracking keyframes add to
// both.  The next frame starts from the constant-velocity prediction of the last two poses.
//
// Optionally the frames are tracked with a learned surrogate's covariances, with a per-frame
// fallback to the k-NN ones (gsicp_tracker_set_surrogate).
//
// Per frame on the device: gsicp_track_frame's kernels (a1..a7), then, for a keyframe, the
// frame's Gaussians moved into the world frame, the exact nearest map mean of each (a
// non-overlap test: none within the overlap radius), an order-preserving compaction of the new
// ones, and an append (index rebuild) of each map they go to.
#include <math.h>
#include <string.h>

#include <new>

#include "internal.h"

using namespace gsicp;

namespace gsicp {

gsicp_status set_error(gsicp_status st, const char* msg);

constexpr int KEEP_THREADS = 256;

// idx[i] == -1: Gaussian i overlaps no map mean and is kept
__global__ void keep_count_kernel(const int32_t* __restrict__ idx, int n, uint32_t* __restrict__ counts)
{
    const int i = blockIdx.x * KEEP_THREADS + threadIdx.x;
    const int c = __syncthreads_count(i < n && idx[i] < 0);
    if (threadIdx.x == 0) counts[blockIdx.x] = (uint32_t)c;
}

__global__ void keep_write_kernel(const int32_t* __restrict__ idx, int n, const float* __restrict__ pts,
                                  const float* __restrict__ covs, const uint32_t* __restrict__ offs,
                                  const uint32_t* __restrict__ counts, int nblocks, float* __restrict__ out_pts,
                                  float* __restrict__ out_covs, int* __restrict__ n_out)
{
    __shared__ uint32_t wsum[KEEP_THREADS / 32];
    const int i = blockIdx.x * KEEP_THREADS + threadIdx.x;
    const bool keep = i < n && idx[i] < 0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t bal = __ballot_sync(0xffffffffu, keep);
    if (lane == 0) wsum[warp] = __popc(bal);
    __syncthreads();
    uint32_t before = 0;
    for (int w = 0; w < warp; ++w) before += wsum[w];
    const uint32_t pos = offs[blockIdx.x] + before + __popc(bal & ((1u << lane) - 1u));
    if (keep) {
        for (int a = 0; a < 3; ++a) out_pts[3l * pos + a] = pts[3l * i + a];
        for (int a = 0; a < 6; ++a) out_covs[6l * pos + a] = covs[6l * i + a];
    }
    if (blockIdx.x == nblocks - 1 && threadIdx.x == 0) *n_out = (int)(offs[nblocks - 1] + counts[nblocks - 1]);
}

}  // namespace gsicp

struct gsicp_tracker_s {
    gsicp_ctx ctx = nullptr;
    gsicp_cov_params cov{};
    gsicp_reg_params reg{};
    gsicp_keyframe_params kf{};
    int stride = 2;
    float z_min = 0.f, z_max = 0.f;
    gsicp_map track_map = nullptr, mapping_map = nullptr;
    int64_t frames = 0;
    int since_kf = 0;
    double T1[16], T2[16];  // the last two poses (T1 the latest)
    DevBuf wpts, wcovs, idx, kpts, kcovs, counts, sums, nk;
    // learned covariances (gsicp_tracker_set_surrogate)
    gsicp_surrogate sg = nullptr;
    float fallback_ratio = 1.1f;
    int calib_every = 30;
    double ref_residual = 0.0;  // residual of the last frame tracked with k-NN covariances
    int since_calib = 0;        // frames tracked with the surrogate since then
    int keyframe_knn = 1;       // keyframes tracked with the surrogate add k-NN covariances to the maps
};

static void mat_mul(const double* A, const double* B, double* C)
{
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) {
            double v = 0.0;
            for (int k = 0; k < 4; ++k) v += A[4 * r + k] * B[4 * k + c];
            C[4 * r + c] = v;
        }
}

// Constant velocity: T1 (T2^-1 T1), the rotation replaced by its nearest rotation (polar
// factor by Newton iteration R <- (R + R^-T) / 2), as products of estimated poses drift off.
static void predict(const double* T1, const double* T2, double* T)
{
    double inv2[16] = {0}, rel[16];
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c) inv2[4 * r + c] = T2[4 * c + r];
        inv2[4 * r + 3] = -(T2[r] * T2[3] + T2[4 + r] * T2[7] + T2[8 + r] * T2[11]);
    }
    inv2[15] = 1.0;
    mat_mul(inv2, T1, rel);
    mat_mul(T1, rel, T);
    double R[9];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) R[3 * r + c] = T[4 * r + c];
    for (int it = 0; it < 4; ++it) {
        const double det = R[0] * (R[4] * R[8] - R[5] * R[7]) - R[1] * (R[3] * R[8] - R[5] * R[6]) +
                           R[2] * (R[3] * R[7] - R[4] * R[6]);
        double cof[9] = {R[4] * R[8] - R[5] * R[7], R[5] * R[6] - R[3] * R[8], R[3] * R[7] - R[4] * R[6],
                         R[2] * R[7] - R[1] * R[8], R[0] * R[8] - R[2] * R[6], R[1] * R[6] - R[0] * R[7],
                         R[1] * R[5] - R[2] * R[4], R[2] * R[3] - R[0] * R[5], R[0] * R[4] - R[1] * R[3]};
        for (int a = 0; a < 9; ++a) R[a] = 0.5 * (R[a] + cof[a] / det);  // R^-T = cof / det
    }
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) T[4 * r + c] = R[3 * r + c];
    T[12] = T[13] = T[14] = 0.0;
    T[15] = 1.0;
}

// RMS Euclidean distance of the last registration's inlier correspondences: a residual that does
// not depend on the covariances used, so registrations with different ones compare on one scale.
static double rms_residual(gsicp_ctx ctx, int64_t inliers)
{
    const RegState* st = ctx->reg.state_host;
    return inliers > 0 && st ? sqrt(st->sqdist / (double)inliers) : 0.0;
}

// Gaussians (world frame, n) not within the overlap radius of any mean of `map` (all of them if
// the map is null), appended to it (or a new map built from them).  *added = how many.
static gsicp_status add_new(gsicp_tracker trk, gsicp_map* map, const float* wpts, const float* wcovs, int n,
                            int64_t* added, cudaStream_t s)
{
    gsicp_ctx ctx = trk->ctx;
    *added = 0;
    if (n <= 0) return GSICP_OK;
    const float* kp = wpts;
    const float* kc = wcovs;
    int nk = n;
    if (*map) {
        GSICP_CHECK(trk->idx.ensure(sizeof(int32_t) * n));
        GSICP_CHECK(trk->kpts.ensure(sizeof(float) * 3 * n));
        GSICP_CHECK(trk->kcovs.ensure(sizeof(float) * 6 * n));
        const int nb = (n + KEEP_THREADS - 1) / KEEP_THREADS;
        GSICP_CHECK(trk->counts.ensure(sizeof(uint32_t) * 2 * nb));
        GSICP_CHECK(trk->nk.ensure(sizeof(int)));
        const float r = trk->kf.overlap_radius;
        GSICP_CHECK(launch_nearest((*map)->index.view(), wpts, n, r * r, trk->idx.as<int32_t>(), nullptr, s));
        uint32_t* cnt = trk->counts.as<uint32_t>();
        keep_count_kernel<<<nb, KEEP_THREADS, 0, s>>>(trk->idx.as<int32_t>(), n, cnt);
        GSICP_CHECK(exclusive_scan_u32(cnt, cnt + nb, nb, trk->sums, s));
        keep_write_kernel<<<nb, KEEP_THREADS, 0, s>>>(trk->idx.as<int32_t>(), n, wpts, wcovs, cnt + nb, cnt, nb,
                                                      trk->kpts.as<float>(), trk->kcovs.as<float>(),
                                                      trk->nk.as<int>());
        GSICP_CUDA(cudaGetLastError());
        int h = 0;
        GSICP_CUDA(cudaMemcpyAsync(&h, trk->nk.ptr, sizeof(int), cudaMemcpyDeviceToHost, s));
        GSICP_CUDA(cudaStreamSynchronize(s));
        nk = h;
        kp = trk->kpts.as<float>();
        kc = trk->kcovs.as<float>();
    }
    if (nk == 0) return GSICP_OK;
    if (*map) {
        GSICP_CHECK(gsicp_map_append(ctx, *map, kp, kc, nk, s));
    } else {
        GSICP_CHECK(gsicp_build_map_index(ctx, kp, kc, nk, nullptr, s, map));
    }
    *added = nk;
    return GSICP_OK;
}

extern "C" gsicp_status gsicp_tracker_create(gsicp_ctx ctx, int stride, float z_min, float z_max,
                                             const gsicp_cov_params* cov, const gsicp_reg_params* reg,
                                             const gsicp_keyframe_params* kf, gsicp_tracker* out)
{
    if (!ctx || !cov || !reg || !kf || !out || stride <= 0 || !(z_max > z_min) || kf->force_every < 1 ||
        kf->mapping_every < 0 || !(kf->overlap_radius > 0.f) || !(kf->min_inlier_ratio >= 0.f) ||
        cov->k < 1 || reg->max_iters < 1 || !(reg->max_corr_dist > 0.f))
        return GSICP_ERR_INVALID_ARG;
    gsicp_tracker t = new (std::nothrow) gsicp_tracker_s;
    if (!t) return GSICP_ERR_OOM;
    t->ctx = ctx;
    t->cov = *cov;
    t->reg = *reg;
    t->kf = *kf;
    t->stride = stride;
    t->z_min = z_min;
    t->z_max = z_max;
    *out = t;
    return GSICP_OK;
}

extern "C" void gsicp_tracker_destroy(gsicp_tracker t)
{
    if (!t) return;
    if (t->track_map) gsicp_map_destroy(t->track_map);
    if (t->mapping_map) gsicp_map_destroy(t->mapping_map);
    t->wpts.release(); t->wcovs.release(); t->idx.release(); t->kpts.release(); t->kcovs.release();
    t->counts.release(); t->sums.release(); t->nk.release();
    delete t;
}

extern "C" gsicp_status gsicp_tracker_frame(gsicp_tracker t, const float* depth_dev, int W, int H, const float intr[4],
                                            const double* T_start, double T_out[16], gsicp_frame_info* info,
                                            void* stream)
{
    if (!t || !depth_dev || !intr || W <= 0 || H <= 0 || !T_out || !(intr[0] != 0.f) || !(intr[1] != 0.f))
        return GSICP_ERR_INVALID_ARG;
    if (t->frames == 0 && !T_start) return set_error(GSICP_ERR_INVALID_ARG, "the first frame needs T_start");
    const int64_t cap64 = (int64_t)((W + t->stride - 1) / t->stride) * ((H + t->stride - 1) / t->stride);
    if (cap64 > (1 << 30)) return GSICP_ERR_INVALID_ARG;
    const int cap = (int)cap64;
    cudaStream_t s = (cudaStream_t)stream;
    gsicp_ctx ctx = t->ctx;
    gsicp_frame_info fi;
    memset(&fi, 0, sizeof(fi));
    double T[16];
    gsicp_status st = GSICP_OK;
    int64_t n = 0;
    if (t->frames == 0) {
        memcpy(T, T_start, sizeof(T));
        GSICP_CHECK(frame_covariances(ctx, depth_dev, W, H, intr, t->stride, t->z_min, t->z_max, &t->cov, cap, s,
                                      nullptr));
        int h = 0;
        GSICP_CUDA(cudaMemcpyAsync(&h, ctx->n_dev.ptr, sizeof(int), cudaMemcpyDeviceToHost, s));
        GSICP_CUDA(cudaStreamSynchronize(s));
        n = h;
        fi.kind = GSICP_KEYFRAME;
    } else {
        double T0[16];
        if (T_start) memcpy(T0, T_start, sizeof(T0));
        else if (t->frames >= 2) predict(t->T1, t->T2, T0);
        else memcpy(T0, t->T1, sizeof(T0));
        int iters = 0;
        int64_t inl = 0;
        double cost = 0.0;
        // Learned covariances: a frame is tracked with the surrogate's covariances unless it is a
        // calibration frame (the first tracked one, then every calib_every-th); the result stands
        // if its residual (RMS correspondence distance) is within fallback_ratio of the last
        // k-NN-tracked frame's, else the frame is tracked again, from the same start, with k-NN
        // covariances.
        const bool use_sg = t->sg && t->ref_residual > 0.0 && t->since_calib < t->calib_every - 1;
        if (use_sg) {
            st = track_frame_impl(ctx, depth_dev, W, H, intr, t->stride, t->z_min, t->z_max, &t->cov, t->track_map,
                                  T0, &t->reg, T, nullptr, &iters, &cost, &inl, &n, s, t->sg);
            if (st != GSICP_OK && st != GSICP_ERR_DEGENERATE) return st;
            GSICP_CHECK(surrogate_status(t->sg));
            fi.residual = rms_residual(ctx, inl);
            fi.cov_source = 1;
            if (st == GSICP_OK && inl > 0 && fi.residual <= (double)t->fallback_ratio * t->ref_residual) {
                t->since_calib += 1;
            } else {
                fi.fell_back = 1;
            }
        }
        if (!use_sg || fi.fell_back) {
            st = track_frame_impl(ctx, depth_dev, W, H, intr, t->stride, t->z_min, t->z_max, &t->cov, t->track_map,
                                  T0, &t->reg, T, nullptr, &iters, &cost, &inl, &n, s, nullptr);
            if (st != GSICP_OK && st != GSICP_ERR_DEGENERATE) return st;
            fi.residual = rms_residual(ctx, inl);
            fi.cov_source = 0;
            if (t->sg && st == GSICP_OK && inl > 0) {
                t->ref_residual = fi.residual;
                t->since_calib = 0;
            }
        }
        fi.iters = iters;
        fi.inliers = inl;
        fi.inlier_ratio = n > 0 ? (double)inl / (double)n : 0.0;
        t->since_kf += 1;
        if (st == GSICP_OK && (fi.inlier_ratio < t->kf.min_inlier_ratio || t->since_kf >= t->kf.force_every))
            fi.kind = GSICP_KEYFRAME;
        else if (st == GSICP_OK && t->kf.mapping_every > 0 && t->since_kf % t->kf.mapping_every == 0)
            fi.kind = GSICP_MAPPING_KEYFRAME;
        else
            fi.kind = GSICP_FRAME;
    }
    fi.n_points = n;
    fi.status = st;
    if (fi.kind != GSICP_FRAME && n > 0 && fi.cov_source == 1 && t->keyframe_knn) {
        // the maps keep k-NN covariances: recompute them for this keyframe (same points)
        GSICP_CHECK(frame_covariances(ctx, depth_dev, W, H, intr, t->stride, t->z_min, t->z_max, &t->cov, cap, s,
                                      nullptr));
    }
    if (fi.kind != GSICP_FRAME && n > 0) {
        // the frame's Gaussians (row-major, as a1 wrote them) moved into the world frame
        GSICP_CHECK(t->wpts.ensure(sizeof(float) * 3 * n));
        GSICP_CHECK(t->wcovs.ensure(sizeof(float) * 6 * n));
        GSICP_CHECK(launch_transform(T, ctx->frame_pts.as<float>(), ctx->frame_covs.as<float>(), (int)n,
                                     t->wpts.as<float>(), t->wcovs.as<float>(), s));
        if (fi.kind == GSICP_KEYFRAME)
            GSICP_CHECK(add_new(t, &t->track_map, t->wpts.as<float>(), t->wcovs.as<float>(), (int)n,
                                &fi.added_tracking, s));
        GSICP_CHECK(add_new(t, &t->mapping_map, t->wpts.as<float>(), t->wcovs.as<float>(), (int)n,
                            &fi.added_mapping, s));
    }
    if (fi.kind == GSICP_KEYFRAME) t->since_kf = 0;
    memcpy(t->T2, t->T1, sizeof(T));
    memcpy(t->T1, T, sizeof(T));
    t->frames += 1;
    memcpy(T_out, T, sizeof(T));
    if (info) *info = fi;
    return st;
}

extern "C" gsicp_status gsicp_tracker_set_surrogate(gsicp_tracker t, gsicp_surrogate sg, float fallback_ratio,
                                                    int calib_every, int keyframe_knn)
{
    if (!t || (sg && (!(fallback_ratio >= 0.f) || calib_every < 1 || (keyframe_knn != 0 && keyframe_knn != 1))))
        return GSICP_ERR_INVALID_ARG;
    t->keyframe_knn = keyframe_knn;
    t->sg = sg;
    t->fallback_ratio = fallback_ratio;
    t->calib_every = calib_every;
    t->ref_residual = 0.0;
    t->since_calib = 0;
    return GSICP_OK;
}

extern "C" gsicp_status gsicp_tracker_maps(gsicp_tracker t, gsicp_map* tracking_map, gsicp_map* mapping_map)
{
    if (!t) return GSICP_ERR_INVALID_ARG;
    if (tracking_map) *tracking_map = t->track_map;
    if (mapping_map) *mapping_map = t->mapping_map;
    return GSICP_OK;
}
