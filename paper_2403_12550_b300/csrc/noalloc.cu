// noalloc.cu -- gsicp_depth_to_points_noalloc: the depth -> points step without any allocation.
//
// Some callers cannot allocate device memory at the time they need the result: a tracking loop
// with a hard per-frame deadline (cudaMalloc / cudaFree may synchronise the device and take an
// unbounded time), an application that has handed the whole device to its own memory pool, or
// code that is not allowed to allocate once initialisation is over.  This entry point runs the
// same kernels as gsicp_depth_to_points, but their scratch (per-block pixel counts, their
// prefix sums and the scan's block totals) lives in one fixed array in this file, reserved when
// the library is loaded: every GPU that loads the library holds these bytes until the process
// exits.  The caller still provides the depth image, the outputs and the count.
//
// The array is shared by every call on a device and keeps the last call's contents; the kernels
// overwrite every entry they read, so nothing needs clearing between calls, but two calls whose
// work overlaps on the GPU (different streams, no ordering) race on it.
#include <mutex>

#include "internal.h"

namespace gsicp {

// d2p_* (depth.cu) and scan_* (index.cu) kernels, launched here with the fixed scratch.
__global__ void d2p_count_kernel(const float* __restrict__ depth, int W, int stride, int Ws, long total,
                                 float z_min, float z_max, uint32_t* __restrict__ counts);
__global__ void d2p_write_kernel(const float* __restrict__ depth, int W, int stride, int Ws, long total,
                                 float z_min, float z_max, double fx, double fy, double cx, double cy,
                                 const uint32_t* __restrict__ offs, const uint32_t* __restrict__ counts, int nblocks,
                                 float* __restrict__ pts, float* __restrict__ z, int cap, int* n_dev, int* total_dev,
                                 int* __restrict__ idx_img);
__global__ void scan_reduce_kernel(const uint32_t* __restrict__ in, int n, uint32_t* __restrict__ sums);
__global__ void scan_sums_kernel(uint32_t* sums, int nb);
__global__ void scan_apply_kernel(const uint32_t* __restrict__ in, uint32_t* __restrict__ out, int n,
                                  const uint32_t* __restrict__ sums);

gsicp_status set_error(gsicp_status st, const char* msg);

namespace {

constexpr long NOALLOC_MAX_SAMPLES = 1l << 22;            // sampled pixels ceil(W/s) * ceil(H/s)
constexpr int NOALLOC_BLOCKS = (int)(NOALLOC_MAX_SAMPLES / 256);  // 256 pixels per counting block
constexpr int NOALLOC_SUMS = NOALLOC_BLOCKS / 2048 + 1;   // block totals of the scan (2048 per tile)
// layout (uint32): counts[NOALLOC_BLOCKS] | offsets[NOALLOC_BLOCKS] | scan totals[NOALLOC_SUMS]
constexpr int NOALLOC_WORDS = 2 * NOALLOC_BLOCKS + NOALLOC_SUMS;

__device__ __align__(256) uint32_t g_d2p_scratch[NOALLOC_WORDS];

constexpr int MAX_DEVICES = 64;
uint32_t* g_scratch_addr[MAX_DEVICES];
cudaError_t g_lookup_status[MAX_DEVICES];
std::once_flag g_lookup_once[MAX_DEVICES];

// Device address of the scratch array on the current device (looked up once per device).
gsicp_status scratch_address(uint32_t** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_status(e, "cudaGetDevice");
    if (dev < 0 || dev >= MAX_DEVICES) return set_error(GSICP_ERR_INVALID_ARG, "device ordinal too large");
    std::call_once(g_lookup_once[dev], [dev]() {
        void* p = nullptr;
        g_lookup_status[dev] = cudaGetSymbolAddress(&p, g_d2p_scratch);
        g_scratch_addr[dev] = static_cast<uint32_t*>(p);
    });
    if (g_lookup_status[dev] != cudaSuccess) return cuda_status(g_lookup_status[dev], "cudaGetSymbolAddress");
    *out = g_scratch_addr[dev];
    return GSICP_OK;
}

}  // namespace
}  // namespace gsicp

using namespace gsicp;

extern "C" gsicp_status gsicp_depth_to_points_noalloc(const float* depth_dev, int W, int H, const float intr[4],
                                                      int stride, float z_min, float z_max, float* pts_dev,
                                                      float* z_dev, int64_t cap, int32_t* n_dev, int32_t* total_dev,
                                                      void* stream)
{
    if (!depth_dev || !intr || !pts_dev || !n_dev || W <= 0 || H <= 0 || stride <= 0 || cap < 0 || cap > INT32_MAX)
        return GSICP_ERR_INVALID_ARG;
    if (!(intr[0] != 0.f) || !(intr[1] != 0.f)) return GSICP_ERR_INVALID_ARG;
    const int Ws = (W + stride - 1) / stride, Hs = (H + stride - 1) / stride;
    const long total = (long)Ws * Hs;
    if (total > NOALLOC_MAX_SAMPLES)
        return set_error(GSICP_ERR_INVALID_ARG,
                         "gsicp_depth_to_points_noalloc: more than 4194304 sampled pixels "
                         "(ceil(W/stride) * ceil(H/stride)); use gsicp_depth_to_points");
    uint32_t* scratch = nullptr;
    GSICP_CHECK(scratch_address(&scratch));
    cudaStream_t s = (cudaStream_t)stream;
    const int nb = (int)((total + 255) / 256);
    uint32_t* counts = scratch;
    uint32_t* offs = scratch + NOALLOC_BLOCKS;
    uint32_t* sums = scratch + 2 * NOALLOC_BLOCKS;
    d2p_count_kernel<<<nb, 256, 0, s>>>(depth_dev, W, stride, Ws, total, z_min, z_max, counts);
    const int ns = (nb + 2047) / 2048;  // scan tiles of 2048 block counts (<= NOALLOC_SUMS)
    scan_reduce_kernel<<<ns, 256, 0, s>>>(counts, nb, sums);
    scan_sums_kernel<<<1, 1024, 0, s>>>(sums, ns);
    scan_apply_kernel<<<ns, 256, 0, s>>>(counts, offs, nb, sums);
    d2p_write_kernel<<<nb, 256, 0, s>>>(depth_dev, W, stride, Ws, total, z_min, z_max, (double)intr[0],
                                        (double)intr[1], (double)intr[2], (double)intr[3], offs, counts, nb, pts_dev,
                                        z_dev, (int)cap, (int*)n_dev, (int*)total_dev, nullptr);
    GSICP_CUDA(cudaGetLastError());
    return GSICP_OK;
}
