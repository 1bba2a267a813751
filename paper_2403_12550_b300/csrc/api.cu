// api.cu -- the C ABI of libgsicp.so (declared in include/gsicp.h): argument
// checks, context / map lifetime, and the sequencing of the kernels of each
// entry point on the caller's stream.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>

#include <vector>

#include "internal.h"

namespace gsicp {

static thread_local std::string g_last_error;

gsicp_status cuda_status(cudaError_t e, const char* where)
{
    g_last_error = std::string(cudaGetErrorName(e)) + ": " + cudaGetErrorString(e) + " (" + where + ")";
    cudaGetLastError();  // clear a non-sticky error
    return e == cudaErrorMemoryAllocation ? GSICP_ERR_OOM : GSICP_ERR_CUDA;
}

gsicp_status set_error(gsicp_status st, const char* msg)
{
    g_last_error = msg;
    return st;
}

gsicp_status DevBuf::ensure(size_t want)
{
    if (want <= bytes && ptr) return GSICP_OK;
    release();
    size_t b = std::max<size_t>(want, 256);
    cudaError_t e = cudaMalloc(&ptr, b);
    if (e != cudaSuccess) {
        ptr = nullptr;
        return cuda_status(e, "cudaMalloc");
    }
    bytes = b;
    return GSICP_OK;
}

void DevBuf::release()
{
    if (ptr) cudaFree(ptr);
    ptr = nullptr;
    bytes = 0;
}

int device_sm_count()
{
    static int cache[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return 148;
    if (dev < 64 && cache[dev]) return cache[dev];
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 148;
    if (dev < 64) cache[dev] = sms;
    return sms;
}

static bool valid_pose(const double T[16])
{
    for (int i = 0; i < 16; ++i)
        if (!isfinite(T[i])) return false;
    return T[12] == 0.0 && T[13] == 0.0 && T[14] == 0.0 && T[15] == 1.0;
}

static bool valid_cov_params(const gsicp_cov_params* p)
{
    return p && p->k >= 1 && p->k <= 32 && p->eps > 0.f && p->eps < 1.f && isfinite(p->p) &&
           (p->reg_mode == GSICP_REG_PLANE || p->reg_mode == GSICP_REG_ELLIPSE || p->reg_mode == GSICP_REG_NONE);
}

static bool valid_reg_params(const gsicp_reg_params* p)
{
    return p && p->max_corr_dist > 0.f && isfinite(p->max_corr_dist) && p->max_iters >= 1 && p->tol_rot >= 0.0 &&
           p->tol_trans >= 0.0 && p->min_inliers >= 0;
}

static gsicp_status finish_registration(gsicp_ctx ctx, cudaStream_t s, double T_out[16], double H_out[36],
                                        double b_out[6], int* iters_out, double* cost_out, int64_t* inliers_out)
{
    GSICP_CUDA(cudaStreamSynchronize(s));
    const RegState& st = *ctx->reg.state_host;
    if (T_out) memcpy(T_out, st.T, sizeof(double) * 16);
    if (H_out) memcpy(H_out, st.H, sizeof(double) * 36);
    if (b_out) memcpy(b_out, st.b, sizeof(double) * 6);
    if (iters_out) *iters_out = st.iter;
    if (cost_out) *cost_out = st.cost;
    if (inliers_out) *inliers_out = st.inliers;
    if (st.status == REG_ST_DEGENERATE) return GSICP_ERR_DEGENERATE;
    return GSICP_OK;
}

constexpr float CACHE_SLACK = 0.01f;  // m beyond max_corr_dist kept in the candidate cache (gicp.cu)
// m: default map grid cell.  With the benchmark frame's map (2.04M Gaussians from ten 1200x680 views,
// ~3.6 per occupied 8 mm cell) 12 mm cells cut the Gauss-Newton loop from ~1.6 to ~1.25 ms against
// 8 mm: their 2x2x2 block certifies more nearest-point searches and more complete candidate lists, so
// fewer points walk the tree; larger cells cost more in the scans of the block (see autotune.py for
// a per-map choice).
constexpr float MAP_CELL = 0.012f;

static RegJob make_job(gsicp_ctx ctx, const float4* src, const float4* covs_s, const int* n_dev, gsicp_map map,
                       const gsicp_reg_params* prm)
{
    RegJob job;
    memset(&job, 0, sizeof(job));
    job.coop_max = ctx->coop_walks;
    job.packet_iters = ctx->packet_iters;
    job.src = src;
    job.covs_s = covs_s;
    job.slack = CACHE_SLACK;
    job.cache_step = ctx->cache_step;
    job.n = n_dev;
    job.map = map->index.view();
    job.corr_out = nullptr;
    const float d = prm ? prm->max_corr_dist : 0.f;
    job.max_d2 = d * d;
    job.max_iters = prm ? prm->max_iters : 1;
    job.tol_rot = prm ? prm->tol_rot : 0.0;
    job.tol_trans = prm ? prm->tol_trans : 0.0;
    job.min_inliers = prm ? prm->min_inliers : 0;
    return job;
}

// Morton-ordered copy of a caller's source cloud and its covariances (for gsicp_register/linearise).
static gsicp_status prepare_source(gsicp_ctx ctx, const float* pts, const float* covs, int n, cudaStream_t s)
{
    GSICP_CHECK(launch_set_int(ctx->n_dev.as<int>(), n, s));
    GSICP_CHECK(build_index(pts, nullptr, n, ctx->n_dev.as<int>(), 32, ctx->src_index, ctx->build, s));
    GSICP_CHECK(ctx->covs_sorted.ensure(sizeof(float4) * 2 * (size_t)std::max(n, 1)));
    return launch_permute_covs(ctx->src_index.view(), covs, n, ctx->covs_sorted.as<float4>(), s);
}

static gsicp_status map_build(gsicp_ctx ctx, gsicp_map map, int bucket, cudaStream_t s)
{
    GSICP_CHECK(launch_set_int(map->count.as<int>(), (int)map->m, s));
    return build_index(map->means.as<float>(), map->covs.as<float>(), (int)map->m, map->count.as<int>(), bucket,
                       map->index, ctx->build, s, true, map->cell, true);
}

}  // namespace gsicp

using namespace gsicp;

extern "C" {

const char* gsicp_version(void) { return "0.1.0"; }

const char* gsicp_last_error(void) { return g_last_error.c_str(); }

const char* gsicp_status_string(gsicp_status s)
{
    switch (s) {
        case GSICP_OK: return "ok";
        case GSICP_ERR_INVALID_ARG: return "invalid argument";
        case GSICP_ERR_CUDA: return "CUDA error";
        case GSICP_ERR_OOM: return "out of device memory";
        case GSICP_ERR_DEGENERATE: return "degenerate registration (too few correspondences or H not positive definite)";
        case GSICP_ERR_TIMEOUT: return "bounded device wait expired";
        case GSICP_ERR_NOT_IMPLEMENTED: return "not implemented";
        case GSICP_ERR_CAPACITY: return "output capacity too small";
    }
    return "unknown status";
}

gsicp_status gsicp_ctx_create(gsicp_ctx* out)
{
    if (!out) return GSICP_ERR_INVALID_ARG;
    *out = nullptr;
    gsicp_ctx c = new (std::nothrow) gsicp_ctx_s();
    if (!c) return GSICP_ERR_OOM;
    cudaError_t e = cudaGetDevice(&c->device);
    if (e != cudaSuccess) {
        delete c;
        return cuda_status(e, "cudaGetDevice");
    }
    gsicp_status st = c->n_dev.ensure(sizeof(int) * 4);
    if (st == GSICP_OK) st = c->total_dev.ensure(sizeof(int) * 4);
    if (st == GSICP_OK) {
        e = cudaMallocHost((void**)&c->host_pinned, sizeof(int64_t) * 8);
        if (e != cudaSuccess) st = cuda_status(e, "cudaMallocHost");
    }
    if (st == GSICP_OK) st = c->reg.init(1 << 18);
    if (st != GSICP_OK) {
        gsicp_ctx_destroy(c);
        return st;
    }
    *out = c;
    return GSICP_OK;
}

void gsicp_ctx_destroy(gsicp_ctx ctx)
{
    if (!ctx) return;
    cudaDeviceSynchronize();
    ctx->reg.release();
    ctx->batch.release();
    BuildScratch& b = ctx->build;
    b.k0.release(); b.k1.release(); b.v0.release(); b.v1.release(); b.hist.release(); b.sums.release();
    b.bbox.release();
    ctx->src_index.pts.release(); ctx->src_index.boxes.release(); ctx->src_index.covs.release();
    ctx->src_index.quant.release();
    ctx->a1_counts.release(); ctx->a1_sums.release(); ctx->n_dev.release(); ctx->total_dev.release();
    ctx->frame_pts.release(); ctx->frame_z.release(); ctx->frame_covs.release(); ctx->frame_depth.release();
    ctx->frame_idx.release(); ctx->fb_list.release(); ctx->fb_count.release();
    ctx->covs_sorted.release();
    ctx->shard_sums.release();
    ctx->morton_samples.release();
    if (ctx->host_pinned) cudaFreeHost(ctx->host_pinned);
    for (cudaEvent_t& e : ctx->ev)
        if (e) cudaEventDestroy(e);
    if (ctx->copy_done) cudaEventDestroy(ctx->copy_done);
    if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
    if (ctx->cov_fork) cudaEventDestroy(ctx->cov_fork);
    if (ctx->cov_join) cudaEventDestroy(ctx->cov_join);
    if (ctx->cov_stream) cudaStreamDestroy(ctx->cov_stream);
    delete ctx;
}

gsicp_status gsicp_ctx_set_timing(gsicp_ctx ctx, int enable)
{
    if (!ctx) return GSICP_ERR_INVALID_ARG;
    if (enable && !ctx->ev[0])
        for (cudaEvent_t& e : ctx->ev) GSICP_CUDA(cudaEventCreate(&e));
    ctx->timing = enable != 0;
    return GSICP_OK;
}

gsicp_status gsicp_ctx_set_coop_walks(gsicp_ctx ctx, int max_per_warp)
{
    if (!ctx || max_per_warp < 0 || max_per_warp > 32) return GSICP_ERR_INVALID_ARG;
    ctx->coop_walks = max_per_warp;
    return GSICP_OK;
}

gsicp_status gsicp_ctx_set_gn_launch_mode(gsicp_ctx ctx, int mode)
{
    if (!ctx || (mode != GSICP_GN_GRAPH && mode != GSICP_GN_PLAIN)) return GSICP_ERR_INVALID_ARG;
    ctx->reg.mode = mode;
    return GSICP_OK;
}

gsicp_status gsicp_ctx_set_packet_iters(gsicp_ctx ctx, int iters)
{
    if (!ctx || iters < 0 || iters > 10000)
        return set_error(GSICP_ERR_INVALID_ARG, "gsicp_ctx_set_packet_iters: 0 .. 10000 iterations");
    ctx->packet_iters = iters;
    return GSICP_OK;
}

gsicp_status gsicp_ctx_set_cache_step(gsicp_ctx ctx, float meters)
{
    if (!ctx || !(meters >= 0.f) || !isfinite(meters))
        return set_error(GSICP_ERR_INVALID_ARG, "gsicp_ctx_set_cache_step: a finite distance >= 0 (m)");
    ctx->cache_step = meters;
    return GSICP_OK;
}

gsicp_status gsicp_ctx_set_gn_block(gsicp_ctx ctx, int points_per_block)
{
    if (!ctx || (points_per_block != 128 && points_per_block != 256 && points_per_block != 384))
        return set_error(GSICP_ERR_INVALID_ARG, "gsicp_ctx_set_gn_block: 128, 256 or 384 points per block");
    ctx->reg.bs = points_per_block;
    return GSICP_OK;
}

gsicp_status gsicp_ctx_phase_times(gsicp_ctx ctx, double out[6])
{
    if (!ctx || !out) return GSICP_ERR_INVALID_ARG;
    for (int i = 0; i < 6; ++i) out[i] = ctx->phase_ms[i];
    return GSICP_OK;
}

gsicp_status gsicp_ctx_frame_stats(gsicp_ctx ctx, int64_t out[2])
{
    if (!ctx || !out) return GSICP_ERR_INVALID_ARG;
    int v[2] = {0, 0};
    if (ctx->fb_count.ptr) GSICP_CUDA(cudaMemcpy(v, ctx->fb_count.ptr, sizeof(v), cudaMemcpyDeviceToHost));
    out[0] = v[0];
    out[1] = v[1];
    return GSICP_OK;
}

gsicp_status gsicp_ctx_last_residual(gsicp_ctx ctx, double* sqdist_out, int64_t* inliers_out)
{
    if (!ctx || !sqdist_out || !ctx->reg.state_host) return GSICP_ERR_INVALID_ARG;
    *sqdist_out = ctx->reg.state_host->sqdist;
    if (inliers_out) *inliers_out = ctx->reg.state_host->inliers;
    return GSICP_OK;
}

gsicp_status gsicp_ctx_reg_stats(gsicp_ctx ctx, int n, int32_t* refreshes_out, int32_t* tail_ns_out,
                                 int32_t* solve_ns_out, int32_t* main_ns_out)
{
    if (!ctx || n < 0 || !ctx->reg.state_host) return GSICP_ERR_INVALID_ARG;
    // a registration copies back only the state's head; the telemetry is read here, on demand
    GSICP_CUDA(cudaDeviceSynchronize());
    GSICP_CUDA(cudaMemcpy(reinterpret_cast<char*>(ctx->reg.state_host) + REG_STATE_HEAD,
                          ctx->reg.state.as<char>() + REG_STATE_HEAD, sizeof(RegState) - REG_STATE_HEAD,
                          cudaMemcpyDeviceToHost));
    const RegState& st = *ctx->reg.state_host;
    for (int i = 0; i < n; ++i) {
        const bool in = i < REG_STATS;
        if (refreshes_out) refreshes_out[i] = in ? st.refreshes[i] : 0;
        if (tail_ns_out) tail_ns_out[i] = in ? st.tail_ns[i] : 0;
        if (solve_ns_out) solve_ns_out[i] = in ? st.solve_ns[i] : 0;
        if (main_ns_out)
            main_ns_out[i] = in && st.t_arrive[i] >= st.t_first[i] ? (int32_t)(st.t_arrive[i] - st.t_first[i]) : 0;
    }
    return GSICP_OK;
}

gsicp_status gsicp_depth_to_points(gsicp_ctx ctx, const float* depth_dev, int W, int H, const float intr[4],
                                   int stride, float z_min, float z_max, float* pts_dev, float* z_dev, int64_t cap,
                                   int32_t* n_dev, int64_t* n_host, void* stream)
{
    if (!ctx || !depth_dev || !intr || !pts_dev || W <= 0 || H <= 0 || stride <= 0 || cap < 0 || cap > INT32_MAX)
        return GSICP_ERR_INVALID_ARG;
    if (!(intr[0] != 0.f) || !(intr[1] != 0.f)) return GSICP_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int* nd = n_dev ? (int*)n_dev : ctx->n_dev.as<int>();
    GSICP_CHECK(launch_depth_to_points(depth_dev, W, H, intr, stride, z_min, z_max, pts_dev, z_dev, (int)cap, nd,
                                       ctx->total_dev.as<int>(), ctx->a1_counts, ctx->a1_sums, s));
    if (n_host) {
        int* h = (int*)ctx->host_pinned;
        GSICP_CUDA(cudaMemcpyAsync(h, ctx->total_dev.ptr, sizeof(int), cudaMemcpyDeviceToHost, s));
        GSICP_CUDA(cudaStreamSynchronize(s));
        const int total = h[0];
        *n_host = std::min<int64_t>(total, cap);
        if (total > cap) return GSICP_ERR_CAPACITY;
    }
    return GSICP_OK;
}

gsicp_status gsicp_source_covariances(gsicp_ctx ctx, const float* pts_dev, const float* z_dev, int64_t n,
                                      const gsicp_cov_params* params, float* covs_dev, int32_t* knn_dev, void* stream)
{
    if (!ctx || !valid_cov_params(params) || n < 0 || n > (1 << 30)) return GSICP_ERR_INVALID_ARG;
    if (n == 0) return GSICP_OK;
    if (!pts_dev || !covs_dev || (params->p != 0.f && !z_dev)) return GSICP_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    GSICP_CHECK(launch_set_int(ctx->n_dev.as<int>(), (int)n, s));
    GSICP_CHECK(build_index(pts_dev, nullptr, (int)n, ctx->n_dev.as<int>(), 32, ctx->src_index, ctx->build, s));
    return launch_knn_cov(ctx->src_index.view(), pts_dev, z_dev, (int)n, *params, covs_dev, knn_dev, nullptr, s);
}

gsicp_status gsicp_build_map_index(gsicp_ctx ctx, const float* means_dev, const float* covs_dev, int64_t m,
                                   const gsicp_index_params* params, void* stream, gsicp_map* out)
{
    if (!out) return GSICP_ERR_INVALID_ARG;
    *out = nullptr;
    if (!ctx || m < 0 || m > (1 << 30) || (m > 0 && (!means_dev || !covs_dev))) return GSICP_ERR_INVALID_ARG;
    int bucket = params && params->bucket ? params->bucket : 16;
    if (bucket != 8 && bucket != 16 && bucket != 32) return GSICP_ERR_INVALID_ARG;
    const float cell = params && params->cell > 0.f ? params->cell : MAP_CELL;
    if (!isfinite(cell)) return GSICP_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    gsicp_map map = new (std::nothrow) gsicp_map_s();
    if (!map) return GSICP_ERR_OOM;
    map->device = ctx->device;
    map->m = m;
    map->cell = cell;
    gsicp_status st = map->count.ensure(sizeof(int) * 4);
    if (st == GSICP_OK) st = map->means.ensure(sizeof(float) * 3 * (size_t)std::max<int64_t>(m, 1));
    if (st == GSICP_OK) st = map->covs.ensure(sizeof(float) * 6 * (size_t)std::max<int64_t>(m, 1));
    if (st == GSICP_OK && m > 0) {
        cudaError_t e = cudaMemcpyAsync(map->means.ptr, means_dev, sizeof(float) * 3 * m, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(map->covs.ptr, covs_dev, sizeof(float) * 6 * m, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) st = cuda_status(e, "cudaMemcpyAsync");
    }
    if (st == GSICP_OK) st = map_build(ctx, map, bucket, s);
    if (st != GSICP_OK) {
        gsicp_map_destroy(map);
        return st;
    }
    *out = map;
    return GSICP_OK;
}

gsicp_status gsicp_map_append(gsicp_ctx ctx, gsicp_map map, const float* means_dev, const float* covs_dev,
                              int64_t m_add, void* stream)
{
    if (!ctx || !map || m_add < 0 || map->m + m_add > (1 << 30) || (m_add > 0 && (!means_dev || !covs_dev)))
        return GSICP_ERR_INVALID_ARG;
    if (m_add == 0) return GSICP_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t m = map->m + m_add;
    DevBuf nm, nc;
    GSICP_CHECK(nm.ensure(sizeof(float) * 3 * (size_t)m));
    gsicp_status st = nc.ensure(sizeof(float) * 6 * (size_t)m);
    if (st != GSICP_OK) {
        nm.release();
        return st;
    }
    cudaError_t e = cudaSuccess;
    if (map->m > 0) {
        e = cudaMemcpyAsync(nm.ptr, map->means.ptr, sizeof(float) * 3 * map->m, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(nc.ptr, map->covs.ptr, sizeof(float) * 6 * map->m, cudaMemcpyDeviceToDevice, s);
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(nm.as<float>() + 3 * map->m, means_dev, sizeof(float) * 3 * m_add,
                            cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(nc.as<float>() + 6 * map->m, covs_dev, sizeof(float) * 6 * m_add,
                            cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // old buffers are read by the copies above
    if (e != cudaSuccess) {
        nm.release();
        nc.release();
        return cuda_status(e, "gsicp_map_append copy");
    }
    map->means.release();
    map->covs.release();
    map->means = nm;
    map->covs = nc;
    map->m = m;
    return map_build(ctx, map, map->index.B, s);
}

gsicp_status gsicp_map_rebuild(gsicp_ctx ctx, gsicp_map map, void* stream)
{
    if (!ctx || !map) return GSICP_ERR_INVALID_ARG;
    return map_build(ctx, map, map->index.B, (cudaStream_t)stream);
}

gsicp_status gsicp_map_inspect(gsicp_map map, float* pts_dev, float* boxes_dev, int64_t* n_leaves_out,
                               int* bucket_out, void* stream)
{
    if (!map) return GSICP_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (pts_dev && map->m > 0)
        GSICP_CUDA(cudaMemcpyAsync(pts_dev, map->index.pts.ptr, sizeof(float4) * (size_t)map->m,
                                   cudaMemcpyDeviceToDevice, s));
    if (boxes_dev)
        GSICP_CUDA(cudaMemcpyAsync(boxes_dev, map->index.boxes.ptr, sizeof(float4) * 4 * (size_t)map->index.L,
                                   cudaMemcpyDeviceToDevice, s));
    if (n_leaves_out) *n_leaves_out = map->index.L;
    if (bucket_out) *bucket_out = map->index.B;
    return GSICP_OK;
}

int64_t gsicp_map_size(gsicp_map map) { return map ? map->m : 0; }

void gsicp_map_destroy(gsicp_map map)
{
    if (!map) return;
    cudaDeviceSynchronize();
    map->index.pts.release();
    map->index.boxes.release();
    map->index.covs.release();
    map->index.keys.release();
    map->index.grid_meta.release();
    map->index.quant.release();
    map->index.grid.release();
    map->means.release();
    map->covs.release();
    map->count.release();
    delete map;
}

gsicp_status gsicp_transform_gaussians(const double T[16], const float* pts_dev, const float* covs_dev, int64_t n,
                                       float* pts_out_dev, float* covs_out_dev, void* stream)
{
    if (!T || n < 0 || n > INT32_MAX || (n > 0 && (!pts_dev || !pts_out_dev)) || !valid_pose(T))
        return GSICP_ERR_INVALID_ARG;
    return launch_transform(T, pts_dev, covs_dev, (int)n, pts_out_dev, covs_out_dev, (cudaStream_t)stream);
}

gsicp_status gsicp_register(gsicp_ctx ctx, const float* src_pts_dev, const float* src_covs_dev, int64_t n,
                            gsicp_map map, const double T0[16], const gsicp_reg_params* params, double T_out[16],
                            double H_out[36], double b_out[6], int* iters_out, double* cost_out,
                            int64_t* inliers_out, void* stream)
{
    if (!ctx || !map || !T0 || !T_out || !valid_reg_params(params) || n < 0 || n > (1 << 30) || !valid_pose(T0))
        return GSICP_ERR_INVALID_ARG;
    if (n > 0 && (!src_pts_dev || !src_covs_dev)) return GSICP_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    GSICP_CHECK(prepare_source(ctx, src_pts_dev, src_covs_dev, (int)n, s));
    RegJob job = make_job(ctx, ctx->src_index.pts.as<float4>(), ctx->covs_sorted.as<float4>(), ctx->n_dev.as<int>(),
                          map, params);
    GSICP_CHECK(reg_run(ctx->reg, job, T0, (int)n, true, s));
    return finish_registration(ctx, s, T_out, H_out, b_out, iters_out, cost_out, inliers_out);
}

static_assert(NACC == GSICP_SHARD_SUMS, "shard sums are the Gauss-Newton kernel's accumulators");
static_assert((int)GSICP_SHARD_RUNNING == (int)REG_ST_RUNNING && (int)GSICP_SHARD_CONVERGED == (int)REG_ST_CONVERGED &&
                  (int)GSICP_SHARD_MAXITER == (int)REG_ST_MAXITER &&
                  (int)GSICP_SHARD_DEGENERATE == (int)REG_ST_DEGENERATE,
              "shard status values are the registration state's");

gsicp_status gsicp_shard_begin(gsicp_ctx ctx, const float* src_pts_dev, const float* src_covs_dev, int64_t n,
                               gsicp_map map, const double T0[16], const gsicp_reg_params* params, void* stream)
{
    if (!ctx || !map || !T0 || !valid_reg_params(params) || n < 0 || n > (1 << 30) || !valid_pose(T0))
        return set_error(GSICP_ERR_INVALID_ARG, "gsicp_shard_begin: invalid argument");
    if (n > 0 && (!src_pts_dev || !src_covs_dev))
        return set_error(GSICP_ERR_INVALID_ARG, "gsicp_shard_begin: NULL source points or covariances");
    cudaStream_t s = (cudaStream_t)stream;
    GSICP_CHECK(ctx->shard_sums.ensure(sizeof(double) * NACC));
    GSICP_CHECK(prepare_source(ctx, src_pts_dev, src_covs_dev, (int)n, s));
    RegJob job = make_job(ctx, ctx->src_index.pts.as<float4>(), ctx->covs_sorted.as<float4>(), ctx->n_dev.as<int>(),
                          map, params);
    return reg_shard_begin(ctx->reg, job, T0, (int)n, ctx->shard_sums.as<double>(), s);
}

gsicp_status gsicp_shard_linearise(gsicp_ctx ctx, double* partial_dev, void* stream)
{
    if (!ctx || !partial_dev) return set_error(GSICP_ERR_INVALID_ARG, "gsicp_shard_linearise: NULL argument");
    if (!ctx->reg.shard)
        return set_error(GSICP_ERR_INVALID_ARG, "gsicp_shard_linearise: no shard registration begun on this context");
    cudaStream_t s = (cudaStream_t)stream;
    GSICP_CHECK(reg_shard_linearise(ctx->reg, s));
    GSICP_CUDA(cudaMemcpyAsync(partial_dev, ctx->shard_sums.ptr, sizeof(double) * NACC, cudaMemcpyDeviceToDevice, s));
    return GSICP_OK;
}

gsicp_status gsicp_shard_update(gsicp_ctx ctx, const double* sums_dev, int nparts, int* status_out, double T_out[16],
                                double H_out[36], int* iters_out, double* cost_out, int64_t* inliers_out,
                                void* stream)
{
    if (!ctx || !sums_dev || nparts < 1 || !status_out)
        return set_error(GSICP_ERR_INVALID_ARG, "gsicp_shard_update: NULL argument or nparts < 1");
    if (!ctx->reg.shard)
        return set_error(GSICP_ERR_INVALID_ARG, "gsicp_shard_update: no shard registration begun on this context");
    cudaStream_t s = (cudaStream_t)stream;
    GSICP_CHECK(reg_shard_update(ctx->reg, sums_dev, nparts, s));
    const gsicp_status st = finish_registration(ctx, s, T_out, H_out, nullptr, iters_out, cost_out, inliers_out);
    *status_out = ctx->reg.state_host->status;
    return st;
}

gsicp_status gsicp_register_batch(gsicp_ctx ctx, int B, const float* const* src_pts_dev,
                                  const float* const* src_covs_dev, const int64_t* n, const gsicp_map* maps,
                                  const double* T0, const gsicp_reg_params* params, double* T_out, int* iters_out,
                                  double* cost_out, int64_t* inliers_out, int* status_out, void* stream)
{
    if (!ctx || B < 0 || B > 65535 || !valid_reg_params(params)) return GSICP_ERR_INVALID_ARG;
    if (B == 0) return GSICP_OK;
    if (!src_pts_dev || !src_covs_dev || !n || !maps || !T0 || !T_out) return GSICP_ERR_INVALID_ARG;
    int64_t total = 0, chunks = 0;
    for (int b = 0; b < B; ++b) {
        if (n[b] < 0 || n[b] > (1 << 30) || !maps[b] || !valid_pose(T0 + 16l * b)) return GSICP_ERR_INVALID_ARG;
        if (n[b] > 0 && (!src_pts_dev[b] || !src_covs_dev[b])) return GSICP_ERR_INVALID_ARG;
        total += n[b];
        chunks += (n[b] + REG_THREADS - 1) / REG_THREADS;
    }
    const int64_t capacity = chunks * params->max_iters;
    if (total > (1 << 30) || capacity > (int64_t)UINT32_MAX - 1) return GSICP_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    BatchMachine& bm = ctx->batch;
    const size_t N = (size_t)std::max<int64_t>(total, 1), C = (size_t)std::max<int64_t>(chunks, 1);
    GSICP_CHECK(bm.src.ensure(sizeof(float4) * N));
    GSICP_CHECK(bm.covs.ensure(sizeof(float4) * 2 * N));
    GSICP_CHECK(bm.cand.ensure(sizeof(int) * KC * N));
    GSICP_CHECK(bm.anchor.ensure(sizeof(float4) * N));
    size_t red_floats = 0;
    for (int b = 0; b < B; ++b) red_floats += reduction_floats((int)((n[b] + REG_THREADS - 1) / REG_THREADS));
    GSICP_CHECK(bm.partials.ensure(sizeof(float) * std::max<size_t>(red_floats, 1)));
    GSICP_CHECK(bm.counts.ensure(sizeof(int) * B));
    GSICP_CHECK(bm.jobs.ensure(sizeof(RegJob) * B));
    GSICP_CHECK(bm.states.ensure(sizeof(RegState) * B));
    GSICP_CHECK(bm.T0.ensure(sizeof(Pose16) * B));
    GSICP_CHECK(bm.offsets.ensure(sizeof(unsigned) * B));
    GSICP_CHECK(bm.queue.ensure(sizeof(BatchQueue)));
    GSICP_CHECK(bm.items.ensure(sizeof(unsigned long long) * (size_t)std::max<int64_t>(capacity, 1)));
    GSICP_CHECK(bm.ptrs.ensure(sizeof(float*) * 2 * B));
    GSICP_CHECK(bm.pofs.ensure(sizeof(int64_t) * (B + 1)));
    // pinned staging, laid out: jobs | states | poses | counts | offsets | queue | pointers | point offsets
    const size_t off_states = sizeof(RegJob) * B, off_T0 = off_states + sizeof(RegState) * B,
                 off_counts = off_T0 + sizeof(Pose16) * B, off_offsets = off_counts + sizeof(int) * B,
                 off_queue = (off_offsets + sizeof(unsigned) * B + 15) / 16 * 16,
                 off_ptrs = off_queue + 16 * ((sizeof(BatchQueue) + 15) / 16),
                 off_pofs = off_ptrs + sizeof(float*) * 2 * B,
                 host_need = off_pofs + sizeof(int64_t) * (B + 1);
    if (bm.host_bytes < host_need) {
        if (bm.host) GSICP_CUDA(cudaFreeHost(bm.host));
        bm.host = nullptr;
        bm.host_bytes = 0;
        GSICP_CUDA(cudaMallocHost(&bm.host, host_need));
        bm.host_bytes = host_need;
    }
    GSICP_CUDA(cudaStreamSynchronize(s));  // the staging area may still feed an earlier batch's copies
    char* hb = static_cast<char*>(bm.host);
    RegJob* jobs_h = reinterpret_cast<RegJob*>(hb);
    RegState* states_h = reinterpret_cast<RegState*>(hb + off_states);
    Pose16* T0_h = reinterpret_cast<Pose16*>(hb + off_T0);
    int* counts_h = reinterpret_cast<int*>(hb + off_counts);
    unsigned* offsets_h = reinterpret_cast<unsigned*>(hb + off_offsets);
    BatchQueue* queue_h = reinterpret_cast<BatchQueue*>(hb + off_queue);
    int running = 0;
    {
        int64_t po = 0, co = 0;
        size_t red_off = 0;
        for (int b = 0; b < B; ++b) {
            counts_h[b] = (int)n[b];
            offsets_h[b] = (unsigned)co;
            for (int i = 0; i < 16; ++i) T0_h[b].v[i] = T0[16l * b + i];
            RegJob j = make_job(ctx, bm.src.as<float4>() + po, bm.covs.as<float4>() + 2 * po, bm.counts.as<int>() + b,
                                maps[b], params);
            j.cand = bm.cand.as<int>() + KC * po;
            j.anchor = bm.anchor.as<float4>() + po;
            j.partials = bm.partials.as<float>() + red_off;
            j.st = bm.states.as<RegState>() + b;
            j.mode = REG_MODE_SOLVE;
            j.use_cond = 0;
            jobs_h[b] = j;
            running += n[b] > 0;
            po += n[b];
            co += (n[b] + REG_THREADS - 1) / REG_THREADS;
            red_off += reduction_floats((int)((n[b] + REG_THREADS - 1) / REG_THREADS));
        }
        *queue_h = BatchQueue{0u, (unsigned)chunks, (unsigned)running, 0u};
    }
    // Morton-ordered copy of every source and its covariances (all clouds in one sort), then the
    // first-iteration seeds of every pair
    const float** ptr_h = reinterpret_cast<const float**>(hb + off_ptrs);
    int64_t* pofs_h = reinterpret_cast<int64_t*>(hb + off_pofs);
    {
        int64_t po = 0;
        for (int b = 0; b < B; ++b) {
            ptr_h[b] = n[b] > 0 ? src_pts_dev[b] : nullptr;
            ptr_h[B + b] = n[b] > 0 ? src_covs_dev[b] : nullptr;
            pofs_h[b] = po;
            po += n[b];
        }
        pofs_h[B] = po;
    }
    GSICP_CUDA(cudaMemsetAsync(bm.partials.ptr, 0, sizeof(float) * std::max<size_t>(red_floats, 1), s));
    GSICP_CUDA(cudaMemcpyAsync(bm.counts.ptr, counts_h, sizeof(int) * B, cudaMemcpyHostToDevice, s));
    GSICP_CUDA(cudaMemcpyAsync(bm.ptrs.ptr, ptr_h, sizeof(float*) * 2 * B, cudaMemcpyHostToDevice, s));
    GSICP_CUDA(cudaMemcpyAsync(bm.pofs.ptr, pofs_h, sizeof(int64_t) * (B + 1), cudaMemcpyHostToDevice, s));
    GSICP_CUDA(cudaMemcpyAsync(bm.jobs.ptr, jobs_h, sizeof(RegJob) * B, cudaMemcpyHostToDevice, s));
    GSICP_CUDA(cudaMemcpyAsync(bm.T0.ptr, T0_h, sizeof(Pose16) * B, cudaMemcpyHostToDevice, s));
    GSICP_CUDA(cudaMemcpyAsync(bm.offsets.ptr, offsets_h, sizeof(unsigned) * B, cudaMemcpyHostToDevice, s));
    GSICP_CUDA(cudaMemcpyAsync(bm.queue.ptr, queue_h, sizeof(BatchQueue), cudaMemcpyHostToDevice, s));
    const float* const* ptrs_dev = bm.ptrs.as<const float* const>();
    GSICP_CHECK(batch_morton_order(ptrs_dev, ptrs_dev + B, bm.pofs.as<const int64_t>(), B, (long)total,
                                   bm.src.as<float4>(), bm.covs.as<float4>(), ctx->build, bm.quant, s));
    GSICP_CHECK(launch_batch_seed(bm.jobs.as<const RegJob>(), bm.T0.as<const Pose16>(), bm.pofs.as<const int64_t>(),
                                  B, (long)total, s));
    GSICP_CHECK(batch_run(bm.jobs.as<const RegJob>(), B, bm.T0.as<const Pose16>(), bm.offsets.as<const unsigned>(),
                          bm.queue.as<BatchQueue>(), bm.items.as<unsigned long long>(), (unsigned)capacity, s));
    GSICP_CUDA(cudaMemcpyAsync(states_h, bm.states.ptr, sizeof(RegState) * B, cudaMemcpyDeviceToHost, s));
    GSICP_CUDA(cudaMemcpyAsync(queue_h, bm.queue.ptr, sizeof(BatchQueue), cudaMemcpyDeviceToHost, s));
    GSICP_CUDA(cudaStreamSynchronize(s));
    for (int b = 0; b < B; ++b) {
        const RegState& st = states_h[b];
        memcpy(T_out + 16l * b, st.T, sizeof(double) * 16);
        if (iters_out) iters_out[b] = st.iter;
        if (cost_out) cost_out[b] = st.cost;
        if (inliers_out) inliers_out[b] = st.inliers;
        if (status_out) status_out[b] = st.status == REG_ST_DEGENERATE ? GSICP_ERR_DEGENERATE : GSICP_OK;
    }
    if (queue_h->error) return set_error(GSICP_ERR_TIMEOUT, "gsicp_register_batch: a work-queue wait ran out");
    return GSICP_OK;
}

gsicp_status gsicp_selftest_batch_timeout(gsicp_ctx ctx, void* stream)
{
    if (!ctx) return GSICP_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    BatchMachine& bm = ctx->batch;
    const unsigned capacity = 4096;
    GSICP_CHECK(bm.queue.ensure(sizeof(BatchQueue)));
    GSICP_CHECK(bm.items.ensure(sizeof(unsigned long long) * capacity));
    GSICP_CHECK(batch_wait_selftest(bm.queue.as<BatchQueue>(), bm.items.as<unsigned long long>(), capacity, s));
    BatchQueue q;
    GSICP_CUDA(cudaMemcpyAsync(&q, bm.queue.ptr, sizeof(q), cudaMemcpyDeviceToHost, s));
    GSICP_CUDA(cudaStreamSynchronize(s));
    if (q.error) return set_error(GSICP_ERR_TIMEOUT, "gsicp_selftest_batch_timeout: the queue waits ran out");
    return GSICP_OK;
}

gsicp_status gsicp_linearise(gsicp_ctx ctx, const float* src_pts_dev, const float* src_covs_dev, int64_t n,
                             gsicp_map map, const double T[16], float max_corr_dist, double H_out[36],
                             double b_out[6], double* cost_out, int64_t* inliers_out, int32_t* corr_dev, void* stream)
{
    if (!ctx || !map || !T || n < 0 || n > (1 << 30) || !(max_corr_dist > 0.f) || !valid_pose(T))
        return GSICP_ERR_INVALID_ARG;
    if (n > 0 && (!src_pts_dev || !src_covs_dev)) return GSICP_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    gsicp_reg_params prm = {max_corr_dist, 1, 0.0, 0.0, 0};
    GSICP_CHECK(prepare_source(ctx, src_pts_dev, src_covs_dev, (int)n, s));
    RegJob job = make_job(ctx, ctx->src_index.pts.as<float4>(), ctx->covs_sorted.as<float4>(), ctx->n_dev.as<int>(),
                          map, &prm);
    job.corr_out = corr_dev;
    GSICP_CHECK(reg_run(ctx->reg, job, T, (int)n, false, s));
    gsicp_status st = finish_registration(ctx, s, nullptr, H_out, b_out, nullptr, cost_out, inliers_out);
    return st == GSICP_ERR_DEGENERATE ? GSICP_OK : st;
}

gsicp_status gsicp_map_nearest(gsicp_ctx ctx, gsicp_map map, const float* queries_dev, int64_t q, float max_dist,
                               int32_t* idx_dev, float* d2_dev, void* stream)
{
    if (!ctx || !map || q < 0 || q > INT32_MAX || !(max_dist > 0.f) || (q > 0 && (!queries_dev || !idx_dev)))
        return GSICP_ERR_INVALID_ARG;
    return launch_nearest(map->index.view(), queries_dev, (int)q, max_dist * max_dist, idx_dev, d2_dev,
                          (cudaStream_t)stream);
}

// a1 -> source index -> a2+a3 for one depth frame, into the context's frame buffers (points in
// row-major order, their covariances in the same order and in the source index's order).
// The sample indices of a Ws x Hs grid (Ws, Hs <= 1024) in 2D Morton order of (column, row), kept by the
// context for the grid it was last built for (made on the host, uploaded once per grid size).
static gsicp_status sample_morton_order(gsicp_ctx ctx, int Ws, int Hs)
{
    if (ctx->morton_w == Ws && ctx->morton_h == Hs && ctx->morton_samples.ptr) return GSICP_OK;
    auto spread = [](uint32_t v) {
        v &= 0x3ffu;
        v = (v | (v << 8)) & 0x00ff00ffu;
        v = (v | (v << 4)) & 0x0f0f0f0fu;
        v = (v | (v << 2)) & 0x33333333u;
        v = (v | (v << 1)) & 0x55555555u;
        return v;
    };
    const size_t n = (size_t)Ws * Hs;
    std::vector<std::pair<uint32_t, int>> code(n);
    for (int j = 0; j < Hs; ++j)
        for (int i = 0; i < Ws; ++i) code[(size_t)j * Ws + i] = {spread((uint32_t)i) | (spread((uint32_t)j) << 1), j * Ws + i};
    std::sort(code.begin(), code.end());
    std::vector<int> order(n);
    for (size_t k = 0; k < n; ++k) order[k] = code[k].second;
    GSICP_CHECK(ctx->morton_samples.ensure(sizeof(int) * std::max<size_t>(n, 1)));
    GSICP_CUDA(cudaMemcpy(ctx->morton_samples.ptr, order.data(), sizeof(int) * n, cudaMemcpyHostToDevice));
    ctx->morton_w = Ws;
    ctx->morton_h = Hs;
    return GSICP_OK;
}

gsicp_status frame_covariances(gsicp_ctx ctx, const float* depth_dev, int W, int H, const float intr[4],
                                      int stride, float z_min, float z_max, const gsicp_cov_params* cov_params,
                                      int cap, cudaStream_t s, gsicp_surrogate sg, int row_step, bool fork)
{
    const int Ws = (W + stride - 1) / stride, Hs = (H + stride - 1) / stride;
    GSICP_CHECK(ctx->frame_pts.ensure(sizeof(float) * 3 * (size_t)cap));
    GSICP_CHECK(ctx->frame_z.ensure(sizeof(float) * (size_t)cap));
    GSICP_CHECK(ctx->frame_covs.ensure(sizeof(float) * 6 * (size_t)cap));
    GSICP_CHECK(ctx->frame_idx.ensure(sizeof(int) * (size_t)cap));
    GSICP_CHECK(ctx->fb_list.ensure(sizeof(int) * 4 * (size_t)cap));
    GSICP_CHECK(ctx->fb_count.ensure(sizeof(int) * 2));
    GSICP_CHECK(ctx->covs_sorted.ensure(sizeof(float4) * 2 * (size_t)cap));
    int* nd = ctx->n_dev.as<int>();
    const bool tm = ctx->timing;
    if (tm) GSICP_CUDA(cudaEventRecord(ctx->ev[0], s));
    GSICP_CHECK(launch_depth_to_points(depth_dev, W, H, intr, stride, z_min, z_max, ctx->frame_pts.as<float>(),
                                       ctx->frame_z.as<float>(), cap, nd, ctx->total_dev.as<int>(), ctx->a1_counts,
                                       ctx->a1_sums, s, ctx->frame_idx.as<int>(), row_step));
    if (tm) GSICP_CUDA(cudaEventRecord(ctx->ev[1], s));
    if (Ws <= 1024 && Hs <= 1024) {
        // the frame's points are near one another exactly where their samples are: index them in
        // the 2D Morton order of the samples (a compaction, no sort)
        GSICP_CHECK(sample_morton_order(ctx, Ws, Hs));
        GSICP_CHECK(build_index_pixel_order(ctx->frame_pts.as<float>(), ctx->frame_idx.as<int>(),
                                            ctx->morton_samples.as<int>(), Ws * Hs, cap, nd, 32, ctx->src_index,
                                            ctx->build, s));
    } else {
        GSICP_CHECK(build_index(ctx->frame_pts.as<float>(), nullptr, cap, nd, 32, ctx->src_index, ctx->build, s));
    }
    if (tm) GSICP_CUDA(cudaEventRecord(ctx->ev[2], s));
    cudaStream_t cs = s;  // the stream of the covariances
    if (fork) {
        if (!ctx->cov_stream) {
            GSICP_CUDA(cudaStreamCreateWithFlags(&ctx->cov_stream, cudaStreamNonBlocking));
            GSICP_CUDA(cudaEventCreateWithFlags(&ctx->cov_fork, cudaEventDisableTiming));
            GSICP_CUDA(cudaEventCreateWithFlags(&ctx->cov_join, cudaEventDisableTiming));
        }
        GSICP_CUDA(cudaEventRecord(ctx->cov_fork, s));
        GSICP_CUDA(cudaStreamWaitEvent(ctx->cov_stream, ctx->cov_fork, 0));
        cs = ctx->cov_stream;
    }
    if (sg)
        GSICP_CHECK(surrogate_forward(sg, ctx->frame_pts.as<float>(), ctx->frame_idx.as<int>(), Ws, Hs,
                                      cov_params->eps, cov_params->p, ctx->frame_covs.as<float>(), nullptr, cs));
    else
        GSICP_CHECK(launch_frame_knn_cov(ctx->src_index.view(), ctx->frame_idx.as<int>(), Ws, Hs, stride, intr,
                                         ctx->frame_pts.as<float>(), ctx->frame_z.as<float>(), cap, *cov_params,
                                         ctx->frame_covs.as<float>(), nullptr, ctx->fb_list.as<int>(),
                                         ctx->fb_count.as<int>(), cs));
    GSICP_CHECK(launch_permute_covs(ctx->src_index.view(), ctx->frame_covs.as<float>(), cap,
                                    ctx->covs_sorted.as<float4>(), cs));
    if (tm) GSICP_CUDA(cudaEventRecord(ctx->ev[3], cs));
    if (fork) GSICP_CUDA(cudaEventRecord(ctx->cov_join, cs));
    return GSICP_OK;
}

gsicp_status gsicp_frame_covariances(gsicp_ctx ctx, const float* depth_dev, int W, int H, const float intr[4],
                                     int stride, float z_min, float z_max, const gsicp_cov_params* params,
                                     float* pts_dev, float* z_dev, float* covs_dev, int64_t cap, int64_t* n_out,
                                     void* stream)
{
    if (!ctx || !depth_dev || !intr || !pts_dev || !covs_dev || !n_out || W <= 0 || H <= 0 || stride <= 0 ||
        cap < 0 || cap > INT32_MAX || !valid_cov_params(params))
        return GSICP_ERR_INVALID_ARG;
    if (!(intr[0] != 0.f) || !(intr[1] != 0.f)) return GSICP_ERR_INVALID_ARG;
    const int64_t frame_cap = (int64_t)((W + stride - 1) / stride) * ((H + stride - 1) / stride);
    if (frame_cap > (1 << 30)) return GSICP_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    GSICP_CHECK(frame_covariances(ctx, depth_dev, W, H, intr, stride, z_min, z_max, params, (int)frame_cap, s, nullptr));
    int* h = (int*)ctx->host_pinned;
    GSICP_CUDA(cudaMemcpyAsync(h, ctx->n_dev.ptr, sizeof(int), cudaMemcpyDeviceToHost, s));
    GSICP_CUDA(cudaStreamSynchronize(s));
    const int64_t n = h[0];
    const int64_t m = std::min(n, cap);
    if (m > 0) {
        GSICP_CUDA(cudaMemcpyAsync(pts_dev, ctx->frame_pts.ptr, sizeof(float) * 3 * m, cudaMemcpyDeviceToDevice, s));
        GSICP_CUDA(cudaMemcpyAsync(covs_dev, ctx->frame_covs.ptr, sizeof(float) * 6 * m, cudaMemcpyDeviceToDevice, s));
        if (z_dev) GSICP_CUDA(cudaMemcpyAsync(z_dev, ctx->frame_z.ptr, sizeof(float) * m, cudaMemcpyDeviceToDevice, s));
    }
    *n_out = m;
    return n > cap ? GSICP_ERR_CAPACITY : GSICP_OK;
}

gsicp_status track_frame_impl(gsicp_ctx ctx, const float* depth_dev, int W, int H, const float intr[4],
                                     int stride, float z_min, float z_max, const gsicp_cov_params* cov_params,
                                     gsicp_map map, const double T0[16], const gsicp_reg_params* reg_params,
                                     double T_out[16], double H_out[36], int* iters_out, double* cost_out,
                                     int64_t* inliers_out, int64_t* n_points_out, cudaStream_t s,
                                     gsicp_surrogate sg, int row_step)
{
    const int64_t cap64 = (int64_t)((W + stride - 1) / stride) * ((H + stride - 1) / stride);
    if (cap64 > (1 << 30)) return GSICP_ERR_INVALID_ARG;
    const int cap = (int)cap64;
    int* nd = ctx->n_dev.as<int>();
    const bool tm = ctx->timing;
    // the covariances on the context's second stream, beside the registration's seeds and set-up
    GSICP_CHECK(frame_covariances(ctx, depth_dev, W, H, intr, stride, z_min, z_max, cov_params, cap, s, sg, row_step,
                                  true));
    RegJob job = make_job(ctx, ctx->src_index.pts.as<float4>(), ctx->covs_sorted.as<float4>(), nd, map, reg_params);
    GSICP_CHECK(reg_run(ctx->reg, job, T0, cap, true, s, ctx->cov_join));
    if (tm) GSICP_CUDA(cudaEventRecord(ctx->ev[4], s));
    if (n_points_out) GSICP_CUDA(cudaMemcpyAsync(ctx->host_pinned, nd, sizeof(int), cudaMemcpyDeviceToHost, s));
    gsicp_status st = finish_registration(ctx, s, T_out, H_out, nullptr, iters_out, cost_out, inliers_out);
    if (n_points_out) *n_points_out = ((int*)ctx->host_pinned)[0];
    if (tm) {
        float ms = 0.f;
        for (int i = 0; i < 4; ++i) {
            GSICP_CUDA(cudaEventElapsedTime(&ms, ctx->ev[i], ctx->ev[i + 1]));
            ctx->phase_ms[i] = ms;
        }
        GSICP_CUDA(cudaEventElapsedTime(&ms, ctx->ev[0], ctx->ev[4]));
        ctx->phase_ms[4] = ms;
        ctx->phase_ms[5] = ctx->reg.state_host->iter;
    }
    return st;
}

static bool valid_frame_args(gsicp_ctx ctx, const float* depth, int W, int H, const float intr[4], int stride,
                             const gsicp_cov_params* cp, gsicp_map map, const double T0[16],
                             const gsicp_reg_params* rp, const double* T_out)
{
    return ctx && depth && W > 0 && H > 0 && intr && intr[0] != 0.f && intr[1] != 0.f && stride > 0 &&
           valid_cov_params(cp) && map && T0 && valid_pose(T0) && valid_reg_params(rp) && T_out;
}

gsicp_status gsicp_track_frame(gsicp_ctx ctx, const float* depth_dev, int W, int H, const float intr[4], int stride,
                               float z_min, float z_max, const gsicp_cov_params* cov_params, gsicp_map map,
                               const double T0[16], const gsicp_reg_params* reg_params, double T_out[16],
                               double H_out[36], int* iters_out, double* cost_out, int64_t* inliers_out,
                               int64_t* n_points_out, void* stream)
{
    if (!valid_frame_args(ctx, depth_dev, W, H, intr, stride, cov_params, map, T0, reg_params, T_out))
        return GSICP_ERR_INVALID_ARG;
    return track_frame_impl(ctx, depth_dev, W, H, intr, stride, z_min, z_max, cov_params, map, T0, reg_params, T_out,
                            H_out, iters_out, cost_out, inliers_out, n_points_out, (cudaStream_t)stream, nullptr);
}

gsicp_status gsicp_track_frame_surrogate(gsicp_ctx ctx, gsicp_surrogate sg, const float* depth_dev, int W, int H,
                                         const float intr[4], int stride, float z_min, float z_max,
                                         const gsicp_cov_params* cov_params, gsicp_map map, const double T0[16],
                                         const gsicp_reg_params* reg_params, double T_out[16], double H_out[36],
                                         int* iters_out, double* cost_out, int64_t* inliers_out,
                                         int64_t* n_points_out, void* stream)
{
    if (!sg || !valid_frame_args(ctx, depth_dev, W, H, intr, stride, cov_params, map, T0, reg_params, T_out))
        return GSICP_ERR_INVALID_ARG;
    const gsicp_status st = track_frame_impl(ctx, depth_dev, W, H, intr, stride, z_min, z_max, cov_params, map, T0,
                                             reg_params, T_out, H_out, iters_out, cost_out, inliers_out, n_points_out,
                                             (cudaStream_t)stream, sg);
    GSICP_CHECK(surrogate_status(sg));  // the stream is synchronised by now
    return st;
}

gsicp_status gsicp_track_frame_host(gsicp_ctx ctx, const float* depth_host, int W, int H, const float intr[4],
                                    int stride, float z_min, float z_max, const gsicp_cov_params* cov_params,
                                    gsicp_map map, const double T0[16], const gsicp_reg_params* reg_params,
                                    double T_out[16], double H_out[36], int* iters_out, double* cost_out,
                                    int64_t* inliers_out, int64_t* n_points_out, void* stream)
{
    if (!valid_frame_args(ctx, depth_host, W, H, intr, stride, cov_params, map, T0, reg_params, T_out))
        return GSICP_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    // Only the rows a1 samples (every stride-th) go up: ceil(H / stride) rows of W floats.
    const int Hs = (H + stride - 1) / stride;
    const size_t row = sizeof(float) * (size_t)W;
    GSICP_CHECK(ctx->frame_depth.ensure(row * (size_t)Hs));
    // The depth rows go up on the context's own copy stream, so that they overlap whatever the
    // caller queued on `stream` before this call (e.g. a map-index rebuild); `stream` waits for them
    // before a1.  The buffer is free: the previous call on this context synchronised its stream.
    if (!ctx->copy_stream) {
        GSICP_CUDA(cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking));
        GSICP_CUDA(cudaEventCreateWithFlags(&ctx->copy_done, cudaEventDisableTiming));
    }
    if (stride == 1)
        GSICP_CUDA(cudaMemcpyAsync(ctx->frame_depth.ptr, depth_host, row * (size_t)H, cudaMemcpyHostToDevice,
                                   ctx->copy_stream));
    else
        GSICP_CUDA(cudaMemcpy2DAsync(ctx->frame_depth.ptr, row, depth_host, row * (size_t)stride, row, (size_t)Hs,
                                     cudaMemcpyHostToDevice, ctx->copy_stream));
    GSICP_CUDA(cudaEventRecord(ctx->copy_done, ctx->copy_stream));
    GSICP_CUDA(cudaStreamWaitEvent(s, ctx->copy_done, 0));
    return track_frame_impl(ctx, ctx->frame_depth.as<float>(), W, H, intr, stride, z_min, z_max, cov_params, map, T0,
                            reg_params, T_out, H_out, iters_out, cost_out, inliers_out, n_points_out, s, nullptr, 1);
}

}  // extern "C"
