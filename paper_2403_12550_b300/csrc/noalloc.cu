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
#include <cuda.h>  // driver API types only: the two calls used are fetched through the runtime

#include <mutex>

#include "internal.h"

namespace gsicp {

// d2p_* (depth.cu) and scan_* (index.cu) kernels, launched here with the fixed scratch.
__global__ void d2p_count_kernel(const float* __restrict__ depth, int W, int stride, int row_step, int Ws, long total,
                                 float z_min, float z_max, uint32_t* __restrict__ counts);
__global__ void d2p_write_kernel(const float* __restrict__ depth, int W, int stride, int row_step, int Ws, long total,
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

constexpr long NOALLOC_MAX_SAMPLES = 1l << 22;  // sampled pixels ceil(W/s) * ceil(H/s)
// one count per a1 block of D2P_THREADS pixels, one scan partial per SCAN_TILE counts
constexpr int NOALLOC_BLOCKS = (int)((NOALLOC_MAX_SAMPLES + D2P_THREADS - 1) / D2P_THREADS);
constexpr int NOALLOC_SUMS = (NOALLOC_BLOCKS + SCAN_TILE - 1) / SCAN_TILE;
// layout (uint32): counts[NOALLOC_BLOCKS] | offsets[NOALLOC_BLOCKS] | scan totals[NOALLOC_SUMS]
constexpr int NOALLOC_WORDS = 2 * NOALLOC_BLOCKS + NOALLOC_SUMS;
static_assert((long)NOALLOC_BLOCKS * D2P_THREADS >= NOALLOC_MAX_SAMPLES, "a count per block of the largest image");
static_assert((long)NOALLOC_SUMS * SCAN_TILE >= NOALLOC_BLOCKS, "a scan partial per tile of the largest image");

__device__ __align__(256) uint32_t g_d2p_scratch[NOALLOC_WORDS];

// The array's device address belongs to the context that loaded the library's module: a device
// reset (or any teardown of the primary context) makes a new context in which the module, and
// the array with it, may sit elsewhere.  So the address is cached per device together with the
// process-unique id of the context it was looked up in, and looked up again when the current
// context's id differs.  A failed lookup is never cached.  cuCtxGetCurrent / cuCtxGetId are
// fetched through the runtime, so the library does not link the driver library itself.
typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);

struct DriverFns {
    CtxGetCurrentFn get_current = nullptr;
    CtxGetIdFn get_id = nullptr;
};

const DriverFns& driver_fns()
{
    static const DriverFns fns = [] {
        DriverFns f;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            f.get_current = reinterpret_cast<CtxGetCurrentFn>(p);
        p = nullptr;
        q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            f.get_id = reinterpret_cast<CtxGetIdFn>(p);
        cudaGetLastError();
        return f;
    }();
    return fns;
}

// Id of the calling thread's current context; 0 when none is current or it cannot be read
// (then nothing is cached and every call looks the address up).
unsigned long long current_context_id()
{
    const DriverFns& f = driver_fns();
    if (!f.get_current || !f.get_id) return 0;
    CUcontext c = nullptr;
    if (f.get_current(&c) != CUDA_SUCCESS || !c) return 0;
    unsigned long long id = 0;
    return f.get_id(c, &id) == CUDA_SUCCESS ? id : 0;
}

constexpr int MAX_DEVICES = 64;
struct CachedAddress {
    unsigned long long context_id = 0;
    uint32_t* addr = nullptr;
};
CachedAddress g_cached[MAX_DEVICES];
std::mutex g_cached_mutex;

// Device address of the scratch array in the current device's current context.
gsicp_status scratch_address(uint32_t** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_status(e, "cudaGetDevice");
    if (dev < 0 || dev >= MAX_DEVICES)
        return set_error(GSICP_ERR_INVALID_ARG, "gsicp_depth_to_points_noalloc: device ordinal above 63");
    unsigned long long id = current_context_id();
    if (id != 0) {
        std::lock_guard<std::mutex> lock(g_cached_mutex);
        if (g_cached[dev].context_id == id) {
            *out = g_cached[dev].addr;
            return GSICP_OK;
        }
    }
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_d2p_scratch);
    if (e != cudaSuccess) return cuda_status(e, "cudaGetSymbolAddress");
    id = current_context_id();  // the lookup makes the device's primary context current if none was
    if (id != 0) {
        std::lock_guard<std::mutex> lock(g_cached_mutex);
        g_cached[dev].context_id = id;
        g_cached[dev].addr = static_cast<uint32_t*>(p);
    }
    *out = static_cast<uint32_t*>(p);
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
    if (!depth_dev || !intr || !pts_dev || !n_dev)
        return set_error(GSICP_ERR_INVALID_ARG,
                         "gsicp_depth_to_points_noalloc: depth_dev, intr, pts_dev and n_dev must not be NULL");
    if (W <= 0 || H <= 0 || stride <= 0)
        return set_error(GSICP_ERR_INVALID_ARG, "gsicp_depth_to_points_noalloc: W, H and stride must be positive");
    if (cap < 0 || cap > INT32_MAX)
        return set_error(GSICP_ERR_INVALID_ARG, "gsicp_depth_to_points_noalloc: cap outside [0, 2^31 - 1]");
    if (!(intr[0] != 0.f) || !(intr[1] != 0.f))
        return set_error(GSICP_ERR_INVALID_ARG, "gsicp_depth_to_points_noalloc: the focal lengths fx and fy must be non-zero");
    const int Ws = (W + stride - 1) / stride, Hs = (H + stride - 1) / stride;
    const long total = (long)Ws * Hs;
    if (total > NOALLOC_MAX_SAMPLES)
        return set_error(GSICP_ERR_INVALID_ARG,
                         "gsicp_depth_to_points_noalloc: more than 4194304 sampled pixels "
                         "(ceil(W/stride) * ceil(H/stride)); use gsicp_depth_to_points");
    uint32_t* scratch = nullptr;
    GSICP_CHECK(scratch_address(&scratch));
    cudaStream_t s = (cudaStream_t)stream;
    const int nb = (int)((total + D2P_THREADS - 1) / D2P_THREADS);  // <= NOALLOC_BLOCKS
    const int ns = (nb + SCAN_TILE - 1) / SCAN_TILE;                     // <= NOALLOC_SUMS
    uint32_t* counts = scratch;
    uint32_t* offs = scratch + NOALLOC_BLOCKS;
    uint32_t* sums = scratch + 2 * NOALLOC_BLOCKS;
    d2p_count_kernel<<<nb, D2P_THREADS, 0, s>>>(depth_dev, W, stride, stride, Ws, total, z_min, z_max, counts);
    scan_reduce_kernel<<<ns, SCAN_THREADS, 0, s>>>(counts, nb, sums);
    scan_sums_kernel<<<1, 1024, 0, s>>>(sums, ns);
    scan_apply_kernel<<<ns, SCAN_THREADS, 0, s>>>(counts, offs, nb, sums);
    d2p_write_kernel<<<nb, D2P_THREADS, 0, s>>>(depth_dev, W, stride, stride, Ws, total, z_min, z_max, (double)intr[0],
                                        (double)intr[1], (double)intr[2], (double)intr[3], offs, counts, nb, pts_dev,
                                        z_dev, (int)cap, (int*)n_dev, (int*)total_dev, nullptr);
    GSICP_CUDA(cudaGetLastError());
    return GSICP_OK;
}
