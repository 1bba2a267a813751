// internal.h -- host-side declarations shared by the libgsicp translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <utility>

#include "../../include/gsicp.h"
#include "common.cuh"

namespace gsicp {

// A launch as a programmatic dependent of the kernel before it in stream s
// (cudaLaunchAttributeProgrammaticStreamSerialization); the kernel must begin with
// wait_prior_grid() (common.cuh).
template <typename... KArgs, typename... Args>
static inline cudaError_t launch_dependent(void (*kernel)(KArgs...), int grid, int block, cudaStream_t s,
                                           Args&&... args)
{
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr.val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// Launch shapes shared by translation units that launch the same kernels with their own scratch
// (depth.cu and noalloc.cu launch the a1 kernels; index.cu and noalloc.cu the scan kernels).
constexpr int D2P_THREADS = 256;                    // sampled pixels per a1 counting / writing block
constexpr int SCAN_THREADS = 256;                   // threads of a scan tile
constexpr int SCAN_ITEMS = 8;                       // values per scan thread
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;  // values per scan tile (one partial sum each)

// Record a CUDA error for gsicp_last_error() and map it to a status.
gsicp_status cuda_status(cudaError_t e, const char* where);

#define GSICP_CUDA(call)                                                \
    do {                                                                \
        cudaError_t e_ = (call);                                        \
        if (e_ != cudaSuccess) return ::gsicp::cuda_status(e_, #call); \
    } while (0)

#define GSICP_CHECK(st)                          \
    do {                                         \
        gsicp_status s_ = (st);                  \
        if (s_ != GSICP_OK) return s_;           \
    } while (0)

// Grow-only device buffer.
struct DevBuf {
    void* ptr = nullptr;
    size_t bytes = 0;
    gsicp_status ensure(size_t want);
    void release();
    template <class T>
    T* as() const { return static_cast<T*>(ptr); }
};

// Buffers of one spatial index (either owned by a map or scratch of a context).
struct IndexBufs {
    DevBuf pts, boxes, covs;
    DevBuf keys, quant;          // sorted Morton keys (built when with_seed is set), quantisation
    DevBuf grid;                 // cell hash table (built when with_grid is set)
    DevBuf grid_meta;            // device words: [0] live capacity - 1, [1] occupied cells
    bool has_grid = false;
    const int* n_ptr = nullptr;  // device count of valid points (set by build_index)
    int L = 0, B = 16, cap = 0;
    IndexView view() const;
};

// Scratch for building an index: sort keys/values (double-buffered), histogram, scan sums, bbox.
struct BuildScratch {
    DevBuf k0, k1, v0, v1, hist, sums, bbox;
    bool bbox_ready = false;     // bbox holds the empty box and a zero block counter (reset by each use)
};

// Build an index over the first *n_dev of `cap` points (pts n x 3, covs n x 6 optional).
// cell > 0 quantises the Morton grid to cells of that size (coarsened if the bounding cube needs
// more than 1024 cells per axis); with_grid then also builds the cell hash table.
gsicp_status build_index(const float* pts, const float* covs, int cap, const int* n_dev, int bucket,
                         IndexBufs& out, BuildScratch& scr, cudaStream_t s, bool with_seed = false,
                         float cell = 0.f, bool with_grid = false);

// Index of a depth frame's points (pts: a1 output, idx_img: sample -> point index or -1) with the
// points in the 2D Morton order of their samples: msamp lists the nsamp sample indices of the grid
// in that order (sample_morton_order).  No sort: a compaction of the valid samples in that order.
gsicp_status build_index_pixel_order(const float* pts, const int* idx_img, const int* msamp, int nsamp, int cap,
                                     const int* n_dev, int bucket, IndexBufs& out, BuildScratch& scr, cudaStream_t s);

// First-iteration search seeds: for each Morton-ordered source point x_s, the map position found by
// a Morton-key lookup of T0 x_s (cand[s][0], -1 if none); every cache entry is marked "search".
gsicp_status launch_seed(const IndexView& map, const float4* src, const int* n_dev, int cap, const double T0[16],
                         int* cand, float4* anchor, cudaStream_t s);

// Device-wide exclusive scan of uint32 values; in may equal out.  `sums` is scratch.
gsicp_status exclusive_scan_u32(const uint32_t* in, uint32_t* out, int n, DevBuf& sums, cudaStream_t s);

// a1: depth -> points (row-major compaction).  Writes *n_dev (clamped to cap) and *total_dev (unclamped).
// row_step: rows of `depth` (W floats each) between sample rows; 0 = stride (the whole image), 1 when
// only every stride-th row is in memory.
gsicp_status launch_depth_to_points(const float* depth, int W, int H, const float intr[4], int stride,
                                    float z_min, float z_max, float* pts, float* z, int cap, int* n_dev,
                                    int* total_dev, DevBuf& counts, DevBuf& sums, cudaStream_t s,
                                    int* idx_img = nullptr,  // optional: sample -> point index (-1 none)
                                    int row_step = 0);

// a2+a3: k-NN covariances of the points of `ix` (its pts hold the n points; orig gives the
// unsorted xyz for neighbour gathering).
gsicp_status launch_knn_cov(const IndexView& ix, const float* orig_pts, const float* z, int cap,
                            const gsicp_cov_params& prm, float* covs, int32_t* knn, float4* covs_sorted,
                            cudaStream_t s);

// a2+a3 for the points of one depth frame (a1's output in row-major order, idx_img its
// sample -> point map): image-window k-NN certified by the camera geometry, the uncertified
// queries by the tree of `ix` (built over the same points).  fb_list (4 x cap ints) and fb_count
// (2 ints) are scratch.  covs in original order.
gsicp_status launch_frame_knn_cov(const IndexView& ix, const int* idx_img, int Ws, int Hs, int stride,
                                  const float intr[4], const float* pts, const float* z, int cap,
                                  const gsicp_cov_params& prm, float* covs, int32_t* knn, int* fb_list,
                                  int* fb_count, cudaStream_t s);

// Copy covariances (n x 6, original order) into the index's Morton order (2 float4 per point).
gsicp_status launch_permute_covs(const IndexView& ix, const float* covs, int cap, float4* out, cudaStream_t s);

// Registration machinery.
struct RegMachine {
    int grid = 0;
    DevBuf partials, sched, job, state, cand, anchor;
    RegState* state_host = nullptr;  // pinned
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphConditionalHandle cond{};
    int mode = 0;           // gsicp_gn_launch_mode: the conditional graph or plain launches
    int bs = 256;           // source points per block of the iteration kernel (128, 256 or 384)
    int built_bs = 0;       // block size the graph and the reduction rows were built for
    bool shard = false;     // the state belongs to a shard registration (reg_shard_begin, not reg_run since)
    gsicp_status init(int capacity);  // (re)builds the graph when the point capacity grows
    void release();
};

// A registration on stream s: seeds and set-up, then the Gauss-Newton launches, which first wait
// for gn_wait when it is given (work of another stream that the iterations read, e.g. the source
// covariances, may run beside the seeds).
gsicp_status reg_run(RegMachine& rm, const RegJob& job, const double T0[16], int n_cap, bool solve,
                     cudaStream_t s, cudaEvent_t gn_wait = nullptr);

// A registration whose source points are split across processes (one shard here): set-up with the
// linearisation sums going to sums_out (NACC doubles, device), one linearisation at the current
// pose (the candidate cache carried over), and the update from the rows of every shard's sums
// (state copied to rm.state_host, stream-ordered).
gsicp_status reg_shard_begin(RegMachine& rm, const RegJob& job, const double T0[16], int n_cap, double* sums_out,
                             cudaStream_t s);
gsicp_status reg_shard_linearise(RegMachine& rm, cudaStream_t s);
gsicp_status reg_shard_update(RegMachine& rm, const double* parts, int nparts, cudaStream_t s);

// Morton order of B clouds at once (pts_dev / covs_dev: device arrays of B pointers; ofs_dev: B + 1
// offsets of each cloud in the concatenated order, N = ofs[B]): src_out (N float4: x, y, z, index
// within the cloud) and covs_out (2N float4) hold each cloud, in build_index's order for it alone,
// at its offset.  quant: scratch.
gsicp_status batch_morton_order(const float* const* pts_dev, const float* const* covs_dev, const int64_t* ofs_dev,
                                int B, long N, float4* src_out, float4* covs_out, BuildScratch& scr, DevBuf& quant,
                                cudaStream_t s);

// First-iteration seeds of the B jobs' points at once (as launch_seed for each; ofs_dev as above).
gsicp_status launch_batch_seed(const RegJob* jobs_dev, const Pose16* T0_dev, const int64_t* ofs_dev, int B, long N,
                               cudaStream_t s);

// Batched registration (one persistent launch over B jobs; see gicp.cu).  items: capacity slots;
// offsets_dev[b]: first slot of pair b's iteration-0 items; q_dev: head = 0, tail = total
// iteration-0 items, running = pairs with points, error = 0.
gsicp_status batch_run(const RegJob* jobs_dev, int B, const Pose16* T0_dev, const unsigned* offsets_dev,
                       BatchQueue* q_dev, unsigned long long* items, unsigned capacity, cudaStream_t s);

// Runs the batch kernel on a queue whose one running pair never gets an item (its waits run out).
gsicp_status batch_wait_selftest(BatchQueue* q_dev, unsigned long long* items, unsigned capacity, cudaStream_t s);

// Buffers of batched registrations (grown on demand, kept by the context).
struct BatchMachine {
    DevBuf src, covs, cand, anchor, partials, counts, jobs, states, T0, offsets, queue, items;
    DevBuf ptrs, pofs, quant;  // cloud pointer tables, point offsets, per-cloud quantisation
    void* host = nullptr;  // pinned staging: jobs, poses, counts, offsets, queue, states
    size_t host_bytes = 0;
    void release();
};

gsicp_status launch_nearest(const IndexView& map, const float* q, int nq, float max_d2, int32_t* idx,
                            float* d2, cudaStream_t s);

gsicp_status launch_transform(const double T[16], const float* pts, const float* covs, int n, float* pts_out,
                              float* covs_out, cudaStream_t s);

gsicp_status launch_set_int(int* dst, int value, cudaStream_t s);

int device_sm_count();

// The surrogate's layers 1-3 over a frame's a1 output (pts in a1 order, idx_img the sample ->
// point map of the ws x hs sample grid): covariances (a1 order, nullable) and v per sample
// (nullable).  Defined in surrogate.cu.
gsicp_status surrogate_forward(gsicp_surrogate_s* sg, const float* pts, const int* idx_img, int ws, int hs, float eps,
                               float p, float* covs, float* v_out, cudaStream_t s);
// GSICP_ERR_TIMEOUT (and the flag cleared) if a bounded wait of the surrogate's kernels ran out
// since the last call; read after the stream has been synchronised.
gsicp_status surrogate_status(gsicp_surrogate_s* sg);

}  // namespace gsicp

struct gsicp_ctx_s {
    int device = 0;
    gsicp::BuildScratch build;
    gsicp::IndexBufs src_index;       // per-frame source index
    gsicp::DevBuf a1_counts, a1_sums, n_dev, total_dev;
    gsicp::DevBuf frame_pts, frame_z, frame_covs, frame_depth;
    gsicp::DevBuf frame_idx, fb_list, fb_count;  // sample -> point map; tree-search list of the window k-NN
    gsicp::DevBuf covs_sorted;         // source covariances in the source index's order
    gsicp::DevBuf morton_samples;      // sample indices of the frame grid in 2D Morton order
    int morton_w = 0, morton_h = 0;    // the grid they are for
    gsicp::DevBuf shard_sums;          // NACC doubles: the last shard linearisation's sums
    gsicp::RegMachine reg;
    gsicp::BatchMachine batch;
    int64_t* host_pinned = nullptr;   // small pinned scratch for counts
    bool timing = false;
    int coop_walks = gsicp::COOP_WALKS_DEFAULT;  // RegJob::coop_max of this context's registrations
    int packet_iters = 1;              // RegJob::packet_iters of this context's registrations
    float cache_step = 0.0005f;        // RegJob::cache_step (m) of this context's registrations
    cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    cudaStream_t copy_stream = nullptr;  // host-buffer entry points' uploads (overlap the caller's queue)
    cudaEvent_t copy_done = nullptr;
    // a frame's k-NN covariances run on cov_stream beside the registration's seeds and set-up on the
    // caller's stream: cov_fork (source index built) -> cov_stream, cov_join (covariances reordered)
    // -> the Gauss-Newton launches
    cudaStream_t cov_stream = nullptr;
    cudaEvent_t cov_fork = nullptr, cov_join = nullptr;
    double phase_ms[6] = {0, 0, 0, 0, 0, 0};
};

struct gsicp_map_s {
    int device = 0;
    int64_t m = 0;
    float cell = 0.f;                 // requested grid cell size (m)
    gsicp::IndexBufs index;
    gsicp::DevBuf means, covs;        // unsorted copies (for appends)
    gsicp::DevBuf count;              // device int: number of Gaussians
};

// Frame helpers of api.cu used by the tracker (tracker.cu); defined in api.cu's C-linkage section.
extern "C" {
// a1 -> source index -> a2+a3 of one depth frame into the context's frame buffers; with a
// surrogate (non-null sg) the covariances are its predictions instead of the k-NN ones.
// fork: the covariances and their reordering go on ctx->cov_stream after the source index, ending
// with ctx->cov_join recorded there (the caller makes its stream wait for it).
gsicp_status frame_covariances(gsicp_ctx ctx, const float* depth_dev, int W, int H, const float intr[4], int stride,
                               float z_min, float z_max, const gsicp_cov_params* cov_params, int cap,
                               cudaStream_t s, gsicp_surrogate sg,
                               int row_step = 0,  // launch_depth_to_points' row_step
                               bool fork = false);
// The whole a1..a7 step of gsicp_track_frame (arguments already checked), covariances as above.
gsicp_status track_frame_impl(gsicp_ctx ctx, const float* depth_dev, int W, int H, const float intr[4], int stride,
                              float z_min, float z_max, const gsicp_cov_params* cov_params, gsicp_map map,
                              const double T0[16], const gsicp_reg_params* reg_params, double T_out[16],
                              double H_out[36], int* iters_out, double* cost_out, int64_t* inliers_out,
                              int64_t* n_points_out, cudaStream_t s, gsicp_surrogate sg, int row_step = 0);
}  // extern "C"
