// depth.cu -- a1: depth image -> point cloud (Sec. 3, Fig. 2: "a point cloud by
// downsampling and reprojecting the current depth image").
//
// Every stride-th pixel (u, v) whose depth d is finite and within
// [z_min, z_max] becomes ((u - cx) d / fx, (v - cy) d / fy, d), in row-major
// pixel order.  The two products/quotients are evaluated in double and
// rounded once to float, so each coordinate is the correctly rounded value of
// the formula.  Order-preserving compaction: per-block counts, then the write, each block summing
// the counts of the blocks before it.
#include "internal.h"

namespace gsicp {

// D2P_THREADS: internal.h

// Sample idx (row j, column i of the Ws-wide sample grid) is pixel (u, v) = (i, j) * stride; its
// depth is row j * row_step of the image in memory (row_step = stride for a whole image, 1 when only
// the sampled rows are in memory, W floats each).
__device__ __forceinline__ bool pixel_valid(const float* depth, int W, int stride, int row_step, int Ws, long idx,
                                            float z_min, float z_max, int& u, int& v, float& d)
{
    const int j = (int)(idx / Ws), i = (int)(idx % Ws);
    u = i * stride;
    v = j * stride;
    d = depth[(long)j * row_step * W + u];
    return isfinite(d) && d >= z_min && d <= z_max;
}

__global__ void d2p_count_kernel(const float* __restrict__ depth, int W, int stride, int row_step, int Ws, long total,
                                 float z_min, float z_max, uint32_t* __restrict__ counts)
{
    const long idx = (long)blockIdx.x * D2P_THREADS + threadIdx.x;
    int u, v;
    float d;
    bool ok = idx < total && pixel_valid(depth, W, stride, row_step, Ws, idx, z_min, z_max, u, v, d);
    int c = __syncthreads_count(ok);
    if (threadIdx.x == 0) counts[blockIdx.x] = (uint32_t)c;
}

// The block's valid pixels written from offset off (all_total: every block's valid pixels, used
// by the last block for the counts).
__device__ __forceinline__ void d2p_write_block(const float* __restrict__ depth, int W, int stride, int row_step, int Ws, long total,
                                                float z_min, float z_max, double fx, double fy, double cx, double cy,
                                                uint32_t off, bool last, uint32_t all_total, float* __restrict__ pts,
                                                float* __restrict__ z, int cap, int* n_dev, int* total_dev,
                                                int* __restrict__ idx_img)
{
    __shared__ uint32_t wsum[D2P_THREADS / 32];
    const long idx = (long)blockIdx.x * D2P_THREADS + threadIdx.x;
    int u = 0, v = 0;
    float d = 0.f;
    const bool ok = idx < total && pixel_valid(depth, W, stride, row_step, Ws, idx, z_min, z_max, u, v, d);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t bal = __ballot_sync(0xffffffffu, ok);
    if (lane == 0) wsum[warp] = __popc(bal);
    __syncthreads();
    uint32_t before = 0;
    for (int w = 0; w < warp; ++w) before += wsum[w];
    const uint32_t pos = off + before + __popc(bal & ((1u << lane) - 1u));
    if (ok && pos < (uint32_t)cap) {
        const double dd = (double)d;
        pts[3l * pos + 0] = (float)(((double)u - cx) * dd / fx);
        pts[3l * pos + 1] = (float)(((double)v - cy) * dd / fy);
        pts[3l * pos + 2] = d;
        if (z) z[pos] = d;
    }
    // sample -> point index (-1: no point), for searches over the image grid
    if (idx_img && idx < total) idx_img[idx] = ok && pos < (uint32_t)cap ? (int)pos : -1;
    if (last && threadIdx.x == 0) {
        if (n_dev) *n_dev = (int)min(all_total, (uint32_t)cap);
        if (total_dev) *total_dev = (int)all_total;
    }
}

// Writes with the blocks' exclusive offsets from a scan (offs).
__global__ void d2p_write_kernel(const float* __restrict__ depth, int W, int stride, int row_step, int Ws, long total,
                                 float z_min, float z_max, double fx, double fy, double cx, double cy,
                                 const uint32_t* __restrict__ offs, const uint32_t* __restrict__ counts, int nblocks,
                                 float* __restrict__ pts, float* __restrict__ z, int cap, int* n_dev, int* total_dev,
                                 int* __restrict__ idx_img)
{
    const bool last = blockIdx.x == nblocks - 1;
    const uint32_t off = offs[blockIdx.x];
    d2p_write_block(depth, W, stride, row_step, Ws, total, z_min, z_max, fx, fy, cx, cy, off, last,
                    last ? off + counts[blockIdx.x] : 0u, pts, z, cap, n_dev, total_dev, idx_img);
}

// Writes with each block's offset summed from the counts of the blocks before it (no scan launches).
__global__ void d2p_write_prefix_kernel(const float* __restrict__ depth, int W, int stride, int row_step, int Ws, long total,
                                        float z_min, float z_max, double fx, double fy, double cx, double cy,
                                        const uint32_t* __restrict__ counts, int nblocks, float* __restrict__ pts,
                                        float* __restrict__ z, int cap, int* n_dev, int* total_dev,
                                        int* __restrict__ idx_img)
{
    wait_prior_grid();
    const bool last = blockIdx.x == nblocks - 1;
    const uint32_t off = block_prefix(counts, blockIdx.x);
    d2p_write_block(depth, W, stride, row_step, Ws, total, z_min, z_max, fx, fy, cx, cy, off, last,
                    last ? off + __ldcg(counts + blockIdx.x) : 0u, pts, z, cap, n_dev, total_dev, idx_img);
}

gsicp_status launch_depth_to_points(const float* depth, int W, int H, const float intr[4], int stride,
                                    float z_min, float z_max, float* pts, float* z, int cap, int* n_dev,
                                    int* total_dev, DevBuf& counts, DevBuf& sums, cudaStream_t s, int* idx_img,
                                    int row_step)
{
    if (row_step <= 0) row_step = stride;
    const int Ws = (W + stride - 1) / stride, Hs = (H + stride - 1) / stride;
    const long total = (long)Ws * Hs;
    const int nb = (int)((total + D2P_THREADS - 1) / D2P_THREADS);
    (void)sums;
    GSICP_CHECK(counts.ensure(sizeof(uint32_t) * (size_t)nb));
    uint32_t* cnt = counts.as<uint32_t>();
    d2p_count_kernel<<<nb, D2P_THREADS, 0, s>>>(depth, W, stride, row_step, Ws, total, z_min, z_max, cnt);
    GSICP_CUDA(launch_dependent(d2p_write_prefix_kernel, nb, D2P_THREADS, s, depth, W, stride, row_step, Ws, total,
                                z_min, z_max, (double)intr[0], (double)intr[1], (double)intr[2], (double)intr[3],
                                (const uint32_t*)cnt, nb, pts, z, cap, n_dev, total_dev, idx_img));
    GSICP_CUDA(cudaGetLastError());
    return GSICP_OK;
}

}  // namespace gsicp
