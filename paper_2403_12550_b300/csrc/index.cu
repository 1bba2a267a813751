// index.cu -- device-built spatial index over a point set (map Gaussians or
// the current frame's points): Morton codes -> stable LSD radix sort ->
// bucketed leaves -> bottom-up bounding boxes.  Used for the nearest-neighbour
// correspondence search of the registration (Sec. 3: correspondences "determined
// by nearest neighbor search") and for the k-nearest-neighbour covariances
// (Sec. 3: covariance "of k-nearest neighbors").
#include <algorithm>

#include "internal.h"

namespace gsicp {

// ------------------------------------------------------------------------------------------
// device-wide exclusive scan (uint32)

// SCAN_THREADS, SCAN_ITEMS, SCAN_TILE: internal.h

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* warp_sums, uint32_t& total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < (int)(blockDim.x >> 5) ? warp_sums[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        warp_sums[lane] = w;  // inclusive prefix of warp totals
    }
    __syncthreads();
    uint32_t warp_prefix = warp > 0 ? warp_sums[warp - 1] : 0u;
    total = warp_sums[(blockDim.x >> 5) - 1];
    __syncthreads();
    return warp_prefix + x - v;
}

__global__ void scan_reduce_kernel(const uint32_t* __restrict__ in, int n, uint32_t* __restrict__ sums)
{
    __shared__ uint32_t ws[32];
    const long base = (long)blockIdx.x * SCAN_TILE + (long)threadIdx.x * SCAN_ITEMS;
    uint32_t s = 0;
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; ++j)
        if (base + j < n) s += in[base + j];
    uint32_t total;
    block_exclusive_scan(s, ws, total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void scan_sums_kernel(uint32_t* sums, int nb)
{
    __shared__ uint32_t ws[32];
    uint32_t carry = 0;
    for (int base = 0; base < nb; base += blockDim.x) {
        int i = base + threadIdx.x;
        uint32_t v = i < nb ? sums[i] : 0u;
        uint32_t total;
        uint32_t ex = block_exclusive_scan(v, ws, total);
        if (i < nb) sums[i] = carry + ex;
        carry += total;
    }
}

__global__ void scan_apply_kernel(const uint32_t* __restrict__ in, uint32_t* __restrict__ out, int n,
                                  const uint32_t* __restrict__ sums)
{
    __shared__ uint32_t ws[32];
    const long base = (long)blockIdx.x * SCAN_TILE + (long)threadIdx.x * SCAN_ITEMS;
    uint32_t v[SCAN_ITEMS];
    uint32_t s = 0;
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; ++j) {
        v[j] = base + j < n ? in[base + j] : 0u;
        s += v[j];
    }
    uint32_t total;
    uint32_t run = block_exclusive_scan(s, ws, total) + sums[blockIdx.x];
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; ++j) {
        if (base + j < n) out[base + j] = run;
        run += v[j];
    }
}

gsicp_status exclusive_scan_u32(const uint32_t* in, uint32_t* out, int n, DevBuf& sums, cudaStream_t s)
{
    if (n <= 0) return GSICP_OK;
    int nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    GSICP_CHECK(sums.ensure(sizeof(uint32_t) * nb));
    scan_reduce_kernel<<<nb, SCAN_THREADS, 0, s>>>(in, n, sums.as<uint32_t>());
    scan_sums_kernel<<<1, 1024, 0, s>>>(sums.as<uint32_t>(), nb);
    scan_apply_kernel<<<nb, SCAN_THREADS, 0, s>>>(in, out, n, sums.as<uint32_t>());
    GSICP_CUDA(cudaGetLastError());
    return GSICP_OK;
}

// ------------------------------------------------------------------------------------------
// stable LSD radix sort of (uint32 key, uint32 value), 8 bits per pass

constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
// 32-key rounds per warp: 16 (4096 keys per tile) halves the tiles of 8, with them the look-back
// chains and the per-tile counter work (map rebuild of 2.04M Gaussians 0.243 -> 0.230 ms; 12:
// 0.234, 24: 0.242 at 128 registers, 32: 0.228 ms at 127)
constexpr int RS_ROUNDS = 16;
constexpr int RS_TILE = RS_THREADS * RS_ROUNDS;   // 4096 keys per block

// One kernel per 8-bit pass (digit counts of all passes first): each block takes the next tile
// of RS_TILE keys (tile numbers handed out in the order blocks start), counts its digits, publishes
// them, and finds its tile's offset per digit by looking back over the earlier tiles' published
// counts until one whose offset is already complete (decoupled look-back); then it scatters its
// keys (each warp ranks a contiguous run of 32 x RS_ROUNDS keys in order, 32 at a time, peers found with
// match.any, so equal digits keep their input order: stable).  A tile only waits on tiles claimed before it, by blocks that
// are running or done and never wait on it, so every wait ends; the spin is bounded all the same
// (err set if a bound ever ran out).
constexpr uint32_t OS_FLAG_AGG = 1u << 30;   // the tile's own counts are published
constexpr uint32_t OS_FLAG_INC = 2u << 30;   // the tile's counts including all earlier tiles
constexpr uint32_t OS_VALUE = (1u << 30) - 1u;
constexpr unsigned OS_SPIN_LIMIT = 1u << 21;

// Digit counts of every pass (hist[p][256]), then in the last block their exclusive scans
// (offs[p][256]); hist and *done must be zero on entry.
__global__ void os_hist_kernel(const uint32_t* __restrict__ keys, int n, int passes, uint32_t* __restrict__ hist,
                               uint32_t* __restrict__ offs, uint32_t* __restrict__ done)
{
    __shared__ uint32_t h[4][256];
    __shared__ uint32_t ws[32];
    __shared__ bool last;
    for (int j = threadIdx.x; j < 4 * 256; j += RS_THREADS) (&h[0][0])[j] = 0u;
    __syncthreads();
    for (long i = (long)blockIdx.x * RS_THREADS + threadIdx.x; i < n; i += (long)gridDim.x * RS_THREADS) {
        const uint32_t k = keys[i];
        for (int p = 0; p < passes; ++p) atomicAdd(&h[p][(k >> (8 * p)) & 255u], 1u);
    }
    __syncthreads();
    for (int j = threadIdx.x; j < passes * 256; j += RS_THREADS) {
        const uint32_t v = (&h[0][0])[j];
        if (v) atomicAdd(&hist[j], v);
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    for (int p = 0; p < passes; ++p) {
        uint32_t total;
        const uint32_t ex = block_exclusive_scan(__ldcg(&hist[p * 256 + threadIdx.x]), ws, total);
        offs[p * 256 + threadIdx.x] = ex;
    }
}

__global__ void __launch_bounds__(RS_THREADS) os_pass_kernel(const uint32_t* __restrict__ kin,
                                                             const uint32_t* __restrict__ vin,
                                                             uint32_t* __restrict__ kout, uint32_t* __restrict__ vout,
                                                             int n, int shift, const uint32_t* __restrict__ offs,
                                                             uint32_t* __restrict__ status,
                                                             uint32_t* __restrict__ tile_ctr,
                                                             uint32_t* __restrict__ err)
{
    wait_prior_grid();
    __shared__ uint32_t wc[RS_WARPS][256];
    __shared__ uint32_t base[256];
    __shared__ int s_tile;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_tile = (int)atomicAdd(tile_ctr, 1u);
    for (int j = threadIdx.x; j < RS_WARPS * 256; j += RS_THREADS) (&wc[0][0])[j] = 0u;
    __syncthreads();
    const int tile = s_tile;
    const long sub = (long)tile * RS_TILE + (long)warp * (32 * RS_ROUNDS);
    const uint32_t lt_mask = (1u << lane) - 1u;
    uint32_t key[RS_ROUNDS], dig[RS_ROUNDS];
#pragma unroll
    for (int r = 0; r < RS_ROUNDS; ++r) {
        const long i = sub + r * 32 + lane;
        key[r] = i < n ? kin[i] : 0u;
        dig[r] = i < n ? ((key[r] >> shift) & 255u) : 256u;
        const uint32_t peers = __match_any_sync(0xffffffffu, dig[r]);
        if (dig[r] < 256u && lane == __ffs(peers) - 1) wc[warp][dig[r]] += __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    {   // per digit: the tile's count, prefix over its warps, then the offset over earlier tiles
        const int d = threadIdx.x;
        uint32_t cnt = 0u;
#pragma unroll
        for (int w = 0; w < RS_WARPS; ++w) {
            const uint32_t c = wc[w][d];
            wc[w][d] = cnt;
            cnt += c;
        }
        uint32_t* my = status + (long)tile * 256 + d;
        uint32_t excl = 0u;
        if (tile > 0) {
            atomicExch(my, OS_FLAG_AGG | cnt);
            // eight predecessors per step, read together (the walk is a chain of dependent loads)
            unsigned spins = 0;
            for (int t = tile - 1; t >= 0;) {
                uint32_t v[8];
#pragma unroll
                for (int j = 0; j < 8; ++j)
                    v[j] = t - j >= 0 ? *reinterpret_cast<volatile uint32_t*>(status + (long)(t - j) * 256 + d)
                                      : (2u << 30);  // before tile 0: nothing (complete, 0)
                int used = 0;
                bool stop = false;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    if (stop || used < j) continue;  // a gap: that tile had not published yet
                    const uint32_t f = v[j] & ~OS_VALUE;
                    if (f == 0u) continue;
                    excl += v[j] & OS_VALUE;
                    ++used;
                    if (f == OS_FLAG_INC) stop = true;
                }
                if (stop) break;
                t -= used;
                if (used == 0 && ++spins > OS_SPIN_LIMIT) {
                    atomicExch(err, 1u);
                    break;
                }
            }
        }
        atomicExch(my, OS_FLAG_INC | (excl + cnt));
        base[d] = offs[d] + excl;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < RS_ROUNDS; ++r) {
        const long i = sub + r * 32 + lane;
        const uint32_t peers = __match_any_sync(0xffffffffu, dig[r]);
        if (dig[r] < 256u) {
            const uint32_t pos = base[dig[r]] + wc[warp][dig[r]] + __popc(peers & lt_mask);
            kout[pos] = key[r];
            vout[pos] = vin[i];
        }
        __syncwarp();
        if (dig[r] < 256u && lane == __ffs(peers) - 1) wc[warp][dig[r]] += __popc(peers);
        __syncwarp();
    }
}

// Scratch layout of a sort (uint32 words): digit counts [4][256] | their exclusive scans [4][256] |
// finished-block counter | error flag | tile counter per pass [4] | look-back status per pass
// [4][tiles][256].  One memset clears everything a sort needs before its first kernel.
struct RadixScratch {
    uint32_t *H, *O, *done, *err, *tile_ctr, *status;
    int n, tiles, passes, real;
};
constexpr size_t RS_HEADER = 2 * 4 * 256 + 2 + 4;

static gsicp_status radix_prepare(DevBuf& hist, int n, int bits, cudaStream_t s, RadixScratch& r)
{
    if (n > (int)OS_VALUE) return GSICP_ERR_INVALID_ARG;
    r.n = n;
    r.tiles = std::max(1, (n + RS_TILE - 1) / RS_TILE);
    r.passes = (bits + 7) / 8;
    if (r.passes & 1) ++r.passes;  // even count: the result lands back in (k0, v0)
    r.real = std::min(r.passes, 4);
    const size_t words = RS_HEADER + 4 * 256 * (size_t)r.tiles;
    GSICP_CHECK(hist.ensure(sizeof(uint32_t) * words));
    r.H = hist.as<uint32_t>();
    r.O = r.H + 4 * 256;
    r.done = r.H + 2 * 4 * 256;
    r.err = r.done + 1;
    r.tile_ctr = r.err + 1;
    r.status = r.H + RS_HEADER;
    GSICP_CUDA(cudaMemsetAsync(r.H, 0, sizeof(uint32_t) * (RS_HEADER + 256 * (size_t)r.tiles * r.real), s));
    return GSICP_OK;
}

// The one-sweep passes of a prepared sort whose digit counts and offsets are in place.
static gsicp_status radix_passes(const RadixScratch& r, uint32_t* k0, uint32_t* v0, uint32_t* k1, uint32_t* v1,
                                 cudaStream_t s)
{
    const int n = r.n;
    for (int p = 0; p < r.passes; ++p) {
        const int shift = 8 * p;
        uint32_t* ki = (p & 1) ? k1 : k0;
        uint32_t* vi = (p & 1) ? v1 : v0;
        uint32_t* ko = (p & 1) ? k0 : k1;
        uint32_t* vo = (p & 1) ? v0 : v1;
        if (shift >= 32) {  // no bits left: plain copy keeps the ping-pong parity
            GSICP_CUDA(cudaMemcpyAsync(ko, ki, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, s));
            GSICP_CUDA(cudaMemcpyAsync(vo, vi, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, s));
            continue;
        }
        GSICP_CUDA(launch_dependent(os_pass_kernel, r.tiles, RS_THREADS, s, (const uint32_t*)ki, (const uint32_t*)vi, ko,
                                    vo, n, shift, (const uint32_t*)(r.O + 256 * p),
                                    r.status + 256 * (size_t)r.tiles * p, r.tile_ctr + p, r.err));
    }
    GSICP_CUDA(cudaGetLastError());
    return GSICP_OK;
}

// Sorts (k0, v0) into (k0, v0) using (k1, v1) as the ping-pong buffer; `bits` <= 32.
static gsicp_status radix_sort_pairs(uint32_t* k0, uint32_t* v0, uint32_t* k1, uint32_t* v1, int n, int bits,
                                     DevBuf& hist, DevBuf& sums, cudaStream_t s)
{
    (void)sums;
    if (n <= 1) return GSICP_OK;
    RadixScratch r;
    GSICP_CHECK(radix_prepare(hist, n, bits, s, r));
    const int hgrid = std::max(1, std::min(r.tiles, device_sm_count() * 4));
    os_hist_kernel<<<hgrid, RS_THREADS, 0, s>>>(k0, n, r.real, r.H, r.O, r.done);
    return radix_passes(r, k0, v0, k1, v1, s);
}

// ------------------------------------------------------------------------------------------
// index build kernels

// bb: min[3] | max[3] (order-preserving encodings) | finished-block counter.  Set to the empty box
// and zero once when the scratch is allocated; every bbox_quant_kernel leaves it so again.
__global__ void bbox_init_kernel(uint32_t* bb)
{
    if (threadIdx.x < 3) bb[threadIdx.x] = 0xffffffffu;      // min (ordered encoding)
    else if (threadIdx.x < 7) bb[threadIdx.x] = 0u;          // max, counter
}

// Bounding box of the valid points, then (last block to finish) the Morton quantisation: cells of
// size `cell` when 1024 of them cover the bounding cube, else 1024 cells across the cube; the
// box words and the counter are reset for the next build.
__global__ void bbox_quant_kernel(const float* __restrict__ pts, const int* __restrict__ n_dev, uint32_t* bb,
                                  float cell, float4* __restrict__ quant)
{
    wait_prior_grid();
    const int n = *n_dev;
    float lo[3] = {GSICP_INF, GSICP_INF, GSICP_INF}, hi[3] = {-GSICP_INF, -GSICP_INF, -GSICP_INF};
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            float c = pts[3 * i + a];
            lo[a] = fminf(lo[a], c);
            hi[a] = fmaxf(hi[a], c);
        }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lo[a] = fminf(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], o));
            hi[a] = fmaxf(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], o));
        }
    }
    // one atomic per block and coordinate: same-address atomics from every warp serialise in L2
    __shared__ float slo[3][32], shi[3][32];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    if (lane == 0) {
#pragma unroll
        for (int a = 0; a < 3; ++a) { slo[a][warp] = lo[a]; shi[a][warp] = hi[a]; }
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            lo[a] = lane < nw ? slo[a][lane] : GSICP_INF;
            hi[a] = lane < nw ? shi[a][lane] : -GSICP_INF;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                lo[a] = fminf(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], o));
                hi[a] = fmaxf(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], o));
            }
        }
        if (lane == 0) {
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                atomicMin(&bb[a], f2ord(lo[a]));
                atomicMax(&bb[3 + a], f2ord(hi[a]));
            }
            __threadfence();
            last = atomicAdd(&bb[6], 1u) == gridDim.x - 1;
        }
    }
    __syncthreads();
    if (!last || threadIdx.x != 0) return;
    __threadfence();
    uint32_t w[6];
#pragma unroll
    for (int a = 0; a < 6; ++a) w[a] = __ldcg(&bb[a]);
    const float lx = ord2f(w[0]), ly = ord2f(w[1]), lz = ord2f(w[2]);
    const float ext = fmaxf(fmaxf(ord2f(w[3]) - lx, ord2f(w[4]) - ly), ord2f(w[5]) - lz);
    float scale = ext > 0.f ? 1024.f / ext : 0.f;
    if (cell > 0.f && !(ext > 1024.f * cell)) scale = 1.f / cell;
    *quant = make_float4(lx, ly, lz, scale);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        bb[a] = 0xffffffffu;
        bb[3 + a] = 0u;
    }
    bb[6] = 0u;
}

// 30-bit Morton key of each valid point over the bounding cube (padding slots get 0xffffffff, so
// they sort after every valid point), with the digit counts of the sort's four 8-bit passes taken
// on the way (as os_hist_kernel does for keys already in memory): per-block counts in shared
// memory, added to H, and the last block to finish writes their exclusive scans to O.
__global__ void __launch_bounds__(RS_THREADS) morton_hist_kernel(const float* __restrict__ pts,
                                                                 const int* __restrict__ n_dev, int cap,
                                                                 const float4* __restrict__ quant,
                                                                 uint32_t* __restrict__ keys, uint32_t* __restrict__ vals,
                                                                 uint32_t* __restrict__ H, uint32_t* __restrict__ O,
                                                                 uint32_t* __restrict__ done)
{
    wait_prior_grid();
    __shared__ uint32_t h[4][256];
    __shared__ uint32_t ws[32];
    __shared__ bool last;
    for (int j = threadIdx.x; j < 4 * 256; j += RS_THREADS) (&h[0][0])[j] = 0u;
    __syncthreads();
    const int n = *n_dev;
    const float4 qz = *quant;
    for (long i = (long)blockIdx.x * RS_THREADS + threadIdx.x; i < cap; i += (long)gridDim.x * RS_THREADS) {
        const uint32_t k = i < n ? morton_of(qz, pts[3 * i + 0], pts[3 * i + 1], pts[3 * i + 2]) : 0xffffffffu;
        keys[i] = k;
        vals[i] = (uint32_t)i;
#pragma unroll
        for (int p = 0; p < 4; ++p) atomicAdd(&h[p][(k >> (8 * p)) & 255u], 1u);
    }
    __syncthreads();
    for (int j = threadIdx.x; j < 4 * 256; j += RS_THREADS) {
        const uint32_t v = (&h[0][0])[j];
        if (v) atomicAdd(&H[j], v);
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    for (int p = 0; p < 4; ++p) {
        uint32_t total;
        const uint32_t ex = block_exclusive_scan(__ldcg(&H[p * 256 + threadIdx.x]), ws, total);
        O[p * 256 + threadIdx.x] = ex;
    }
}

// The live size of the cell hash table: a power of two at least four times the number of occupied
// cells (load factor <= 1/4: searches of empty cells, half of a query's 2x2x2 block on a surface,
// end at the first or second slot; per 1200x680 bench frame GN 1.012 -> 0.999 ms and the map
// rebuild 0.244 -> 0.240 ms against load factor <= 1/2), at least 1024, at most the allocated
// capacity.  meta: [0] live
// capacity - 1, [1] occupied cells (counted by gather_leaf_kernel; reset here for the next build).
__global__ void grid_size_kernel(uint32_t* __restrict__ meta, uint32_t max_capacity)
{
    wait_prior_grid();
    const uint32_t cells = meta[1];
    uint32_t cap = 1024;
    while (cap < 4u * cells && cap < max_capacity) cap <<= 1;
    meta[0] = min(cap, max_capacity) - 1u;
    meta[1] = 0u;
}

__global__ void grid_clear_kernel(int4* __restrict__ table, const uint32_t* __restrict__ meta, uint32_t max_capacity)
{
    wait_prior_grid();
    const uint32_t live = meta[0] + 1u;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < min(live, max_capacity); i += gridDim.x * blockDim.x)
        table[i] = make_int4((int)GRID_EMPTY, 0, 0, 0);
}

// One entry per occupied cell (key, start, end).  A warp takes 32 consecutive sorted positions:
// the cells that start among them end at the next start among them, and the one that starts last
// (or, with no start among them, none) may run on past them; its end is found by the whole warp
// reading 32 keys at a time until the key changes.  Each start lane then inserts its cell.
__global__ void grid_fill_kernel(const uint32_t* __restrict__ keys, const int* __restrict__ n_dev,
                                 int4* __restrict__ table, const uint32_t* __restrict__ meta)
{
    wait_prior_grid();
    const int n = *n_dev;
    const uint32_t mask = meta[0];
    const int lane = threadIdx.x & 31;
    const long nwarps = ((long)gridDim.x * blockDim.x) >> 5;
    for (long base = (((long)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32; base < n; base += nwarps * 32) {
        const long s = base + lane;
        const uint32_t key = s < n ? keys[s] : 0u;
        const bool start = s < n && (s == 0 || keys[s - 1] != key);
        const unsigned starts = __ballot_sync(0xffffffffu, start);
        if (starts == 0u) continue;
        const int last = 31 - __clz(starts);
        // the end of the last cell starting here: the first position past this run whose key differs
        long tail_end = base + 32;
        const uint32_t last_key = __shfl_sync(0xffffffffu, key, last);
        if (tail_end < n) {
            for (long c = tail_end;; c += 32) {
                const long q = c + lane;
                const bool stop = q >= n || keys[q] != last_key;
                const unsigned st = __ballot_sync(0xffffffffu, stop);
                if (st != 0u) {
                    tail_end = c + __ffs(st) - 1;
                    break;
                }
            }
        }
        tail_end = min(tail_end, (long)n);
        if (!start) continue;
        const unsigned later = starts & ~((2u << lane) - 1u);  // starts after this lane (lane < 31)
        const long end = lane == last ? tail_end : base + __ffs(later) - 1;
        uint32_t slot = grid_hash(key) & mask;
        for (uint32_t probe = 0; probe <= mask; ++probe) {
            const uint32_t prev = atomicCAS(reinterpret_cast<unsigned int*>(&table[slot].x), GRID_EMPTY, key);
            if (prev == GRID_EMPTY) {  // each key is inserted by one thread only
                table[slot].y = (int)s;
                table[slot].z = (int)end;
                break;
            }
            slot = (slot + 1) & mask;
        }
    }
}

// The sorted copy (one slot per thread, block b = slots [256 b, 256 b + 256)): points (x, y, z,
// original index) and covariances gathered in sorted order, padding slots beyond n set to +inf;
// the sorted keys copied out (keys_out, nullable); the occupied cells counted into
// grid_meta[1] (nullable); and the leaf boxes, each leaf's B slots being B consecutive lanes of
// one warp (B divides 32).
__global__ void __launch_bounds__(256) gather_leaf_kernel(const float* __restrict__ pts, const float* __restrict__ covs,
                                                          const uint32_t* __restrict__ order,
                                                          const uint32_t* __restrict__ skeys,
                                                          const int* __restrict__ n_dev, int total, int L, int B,
                                                          float4* __restrict__ spts, float4* __restrict__ scovs,
                                                          float4* __restrict__ boxes, uint32_t* __restrict__ keys_out,
                                                          int keys_n, uint32_t* __restrict__ grid_meta)
{
    wait_prior_grid();
    const int n = *n_dev;
    const long s = (long)blockIdx.x * 256 + threadIdx.x;
    float4 p = make_float4(GSICP_INF, GSICP_INF, GSICP_INF, __int_as_float(-1));
    bool starts = false;
    if (s < total) {
        if (s < n) {
            const uint32_t i = order[s];
            p = make_float4(pts[3l * i], pts[3l * i + 1], pts[3l * i + 2], __int_as_float((int)i));
            if (scovs) {
                const float* c = covs + 6l * i;
                scovs[2 * s] = make_float4(c[0], c[1], c[2], c[3]);
                scovs[2 * s + 1] = make_float4(c[4], c[5], 0.f, 0.f);
            }
            starts = grid_meta && (s == 0 || skeys[s - 1] != skeys[s]);
        } else if (scovs) {
            scovs[2 * s] = make_float4(0.f, 0.f, 0.f, 0.f);
            scovs[2 * s + 1] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        spts[s] = p;
        if (keys_out && s < keys_n) keys_out[s] = skeys[s];
    }
    if (grid_meta) {
        const int c = __syncthreads_count(starts);
        if (threadIdx.x == 0 && c) atomicAdd(&grid_meta[1], (uint32_t)c);
    }
    // leaf box over the leaf's valid points (padding slots hold +inf and contribute nothing)
    const bool valid = s < n;
    float lo[3] = {valid ? p.x : GSICP_INF, valid ? p.y : GSICP_INF, valid ? p.z : GSICP_INF};
    float hi[3] = {valid ? p.x : -GSICP_INF, valid ? p.y : -GSICP_INF, valid ? p.z : -GSICP_INF};
    for (int o = B >> 1; o > 0; o >>= 1) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            lo[a] = fminf(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], o));
            hi[a] = fmaxf(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], o));
        }
    }
    if (s < total && (threadIdx.x & (B - 1)) == 0) {
        const long leaf = s / B;
        boxes[2l * (L + leaf)] = make_float4(lo[0], lo[1], lo[2], 0.f);
        boxes[2l * (L + leaf) + 1] = make_float4(hi[0], hi[1], hi[2], 0.f);
    }
}

// Reduce up to 8 levels of the implicit tree: level `count` (heap nodes
// [count, 2count)) is read, each block merges a group of g = min(256, count)
// consecutive nodes into their ancestors down to one node per group.
__global__ void level_reduce_kernel(float4* __restrict__ boxes, int count)
{
    wait_prior_grid();
    __shared__ float4 slo[256], shi[256];
    const int g = min(256, count);
    const int t = threadIdx.x;
    const long first = (long)count + (long)blockIdx.x * g;
    if (t < g) {
        slo[t] = boxes[2 * (first + t)];
        shi[t] = boxes[2 * (first + t) + 1];
    }
    __syncthreads();
    int level = count, width = g;
    long lfirst = first;
    while (width > 1) {
        const int half = width >> 1;
        float4 lo, hi;
        if (t < half) {
            float4 a = slo[2 * t], b = slo[2 * t + 1], c = shi[2 * t], d = shi[2 * t + 1];
            lo = make_float4(fminf(a.x, b.x), fminf(a.y, b.y), fminf(a.z, b.z), 0.f);
            hi = make_float4(fmaxf(c.x, d.x), fmaxf(c.y, d.y), fmaxf(c.z, d.z), 0.f);
        }
        __syncthreads();
        level >>= 1;
        lfirst >>= 1;
        if (t < half) {
            slo[t] = lo;
            shi[t] = hi;
            boxes[2 * (lfirst + t)] = lo;
            boxes[2 * (lfirst + t) + 1] = hi;
        }
        __syncthreads();
        width = half;
    }
}

static int ceil_pow2(long x)
{
    int p = 1;
    while (p < x) p <<= 1;
    return p;
}

gsicp_status build_index(const float* pts, const float* covs, int cap, const int* n_dev, int bucket,
                         IndexBufs& out, BuildScratch& scr, cudaStream_t s, bool with_seed, float cell,
                         bool with_grid)
{
    if (bucket != 8 && bucket != 16 && bucket != 32) return GSICP_ERR_INVALID_ARG;
    const int B = bucket;
    const int L = std::max(1, ceil_pow2(((long)cap + B - 1) / B));
    const int total = L * B;  // sorted slots incl. padding
    GSICP_CHECK(out.pts.ensure(sizeof(float4) * (size_t)total));
    GSICP_CHECK(out.boxes.ensure(sizeof(float4) * 4 * (size_t)L));
    if (covs) GSICP_CHECK(out.covs.ensure(sizeof(float4) * 2 * (size_t)total));
    out.L = L;
    out.B = B;
    out.cap = cap;
    out.n_ptr = n_dev;
    const int sort_n = std::max(cap, 1);
    GSICP_CHECK(scr.k0.ensure(sizeof(uint32_t) * sort_n));
    GSICP_CHECK(scr.k1.ensure(sizeof(uint32_t) * sort_n));
    GSICP_CHECK(scr.v0.ensure(sizeof(uint32_t) * sort_n));
    GSICP_CHECK(scr.v1.ensure(sizeof(uint32_t) * sort_n));
    const int sms = device_sm_count();
    const int grid = std::max(1, std::min((cap + 255) / 256, sms * 8));
    GSICP_CHECK(out.quant.ensure(sizeof(float4)));
    const void* bb_before = scr.bbox.ptr;
    GSICP_CHECK(scr.bbox.ensure(sizeof(uint32_t) * 8));
    if (!scr.bbox_ready || scr.bbox.ptr != bb_before) {
        bbox_init_kernel<<<1, 32, 0, s>>>(scr.bbox.as<uint32_t>());
        scr.bbox_ready = true;
    }
    GSICP_CUDA(launch_dependent(bbox_quant_kernel, std::max(1, std::min((cap + 255) / 256, sms * 2)), 256, s, pts,
                                n_dev, scr.bbox.as<uint32_t>(), cell, out.quant.as<float4>()));
    // keys and the sort's digit counts in one pass; 30-bit keys take four 8-bit passes
    RadixScratch rs;
    GSICP_CHECK(radix_prepare(scr.hist, std::max(cap, 1), 30, s, rs));
    GSICP_CUDA(launch_dependent(morton_hist_kernel, grid, RS_THREADS, s, pts, n_dev, cap,
                                (const float4*)out.quant.as<float4>(), scr.k0.as<uint32_t>(), scr.v0.as<uint32_t>(),
                                rs.H, rs.O, rs.done));
    GSICP_CUDA(cudaGetLastError());
    if (cap > 1)
        GSICP_CHECK(radix_passes(rs, scr.k0.as<uint32_t>(), scr.v0.as<uint32_t>(), scr.k1.as<uint32_t>(),
                                 scr.v1.as<uint32_t>(), s));
    uint32_t grid_capacity = 0;
    if (with_grid) {
        grid_capacity = 1024;
        while (grid_capacity < 2u * (uint32_t)sort_n) grid_capacity <<= 1;
        GSICP_CHECK(out.grid.ensure(sizeof(int4) * (size_t)grid_capacity));
        const void* meta_before = out.grid_meta.ptr;
        GSICP_CHECK(out.grid_meta.ensure(sizeof(uint32_t) * 4));
        if (!out.has_grid || out.grid_meta.ptr != meta_before)
            GSICP_CUDA(cudaMemsetAsync(out.grid_meta.ptr, 0, sizeof(uint32_t) * 4, s));
    }
    out.has_grid = with_grid;
    if (with_seed) GSICP_CHECK(out.keys.ensure(sizeof(uint32_t) * (size_t)sort_n));
    GSICP_CUDA(launch_dependent(gather_leaf_kernel, (total + 255) / 256, 256, s, pts, covs,
                                (const uint32_t*)scr.v0.as<uint32_t>(), (const uint32_t*)scr.k0.as<uint32_t>(), n_dev,
                                total, L, B, out.pts.as<float4>(), covs ? out.covs.as<float4>() : nullptr,
                                out.boxes.as<float4>(), with_seed ? out.keys.as<uint32_t>() : nullptr, sort_n,
                                with_grid ? out.grid_meta.as<uint32_t>() : nullptr));
    for (int count = L; count > 1; count = count / std::min(256, count)) {
        const int blocks = count / std::min(256, count);
        GSICP_CUDA(launch_dependent(level_reduce_kernel, blocks, 256, s, out.boxes.as<float4>(), count));
    }
    if (with_grid) {
        const int ggrid = std::max(1, std::min((cap + 255) / 256, sms * 8));
        GSICP_CUDA(launch_dependent(grid_size_kernel, 1, 1, s, out.grid_meta.as<uint32_t>(), grid_capacity));
        GSICP_CUDA(launch_dependent(grid_clear_kernel, std::max(1, std::min((int)(grid_capacity / 256), sms * 8)), 256,
                                    s, out.grid.as<int4>(), (const uint32_t*)out.grid_meta.as<uint32_t>(),
                                    grid_capacity));
        GSICP_CUDA(launch_dependent(grid_fill_kernel, ggrid, 256, s, (const uint32_t*)scr.k0.as<uint32_t>(), n_dev,
                                    out.grid.as<int4>(), (const uint32_t*)out.grid_meta.as<uint32_t>()));
    }
    GSICP_CUDA(cudaGetLastError());
    return GSICP_OK;
}

// ------------------------------------------------------------------------------------------
// Index of a depth frame's points in the 2D Morton order of their samples

// Valid samples (idx_img[sample] >= 0) among the 256 Morton-ordered samples of each block.
__global__ void pix_count_kernel(const int* __restrict__ idx_img, const int* __restrict__ msamp, int nsamp,
                                 uint32_t* __restrict__ counts)
{
    wait_prior_grid();
    const int k = blockIdx.x * 256 + threadIdx.x;
    const bool ok = k < nsamp && idx_img[msamp[k]] >= 0;
    const int c = __syncthreads_count(ok);
    if (threadIdx.x == 0) counts[blockIdx.x] = (uint32_t)c;
}

// The point index of every valid sample, in the samples' Morton order (stable compaction); each
// block's offset is the sum of the counts of the blocks before it.
__global__ void pix_write_kernel(const int* __restrict__ idx_img, const int* __restrict__ msamp, int nsamp,
                                 const uint32_t* __restrict__ counts, uint32_t* __restrict__ order)
{
    wait_prior_grid();
    __shared__ uint32_t ws[32];
    const int k = blockIdx.x * 256 + threadIdx.x;
    const int pi = k < nsamp ? idx_img[msamp[k]] : -1;
    const uint32_t off = block_prefix(counts, blockIdx.x);
    uint32_t total;
    const uint32_t rank = block_exclusive_scan(pi >= 0 ? 1u : 0u, ws, total);
    if (pi >= 0) order[off + rank] = (uint32_t)pi;
}

gsicp_status build_index_pixel_order(const float* pts, const int* idx_img, const int* msamp, int nsamp, int cap,
                                     const int* n_dev, int bucket, IndexBufs& out, BuildScratch& scr, cudaStream_t s)
{
    if (bucket != 8 && bucket != 16 && bucket != 32) return GSICP_ERR_INVALID_ARG;
    const int B = bucket;
    const int L = std::max(1, ceil_pow2(((long)cap + B - 1) / B));
    const int total = L * B;
    GSICP_CHECK(out.pts.ensure(sizeof(float4) * (size_t)total));
    GSICP_CHECK(out.boxes.ensure(sizeof(float4) * 4 * (size_t)L));
    out.L = L;
    out.B = B;
    out.cap = cap;
    out.n_ptr = n_dev;
    out.has_grid = false;
    GSICP_CHECK(out.quant.ensure(sizeof(float4)));
    const int nb = std::max(1, (nsamp + 255) / 256);
    GSICP_CHECK(scr.k1.ensure(sizeof(uint32_t) * (size_t)nb));
    GSICP_CHECK(scr.v0.ensure(sizeof(uint32_t) * (size_t)std::max(cap, 1)));
    uint32_t* counts = scr.k1.as<uint32_t>();
    GSICP_CUDA(launch_dependent(pix_count_kernel, nb, 256, s, idx_img, msamp, nsamp, counts));
    GSICP_CUDA(launch_dependent(pix_write_kernel, nb, 256, s, idx_img, msamp, nsamp, (const uint32_t*)counts,
                                scr.v0.as<uint32_t>()));
    GSICP_CUDA(launch_dependent(gather_leaf_kernel, (total + 255) / 256, 256, s, pts, (const float*)nullptr,
                                (const uint32_t*)scr.v0.as<uint32_t>(), (const uint32_t*)nullptr, n_dev, total, L, B,
                                out.pts.as<float4>(), (float4*)nullptr, out.boxes.as<float4>(), (uint32_t*)nullptr, 0,
                                (uint32_t*)nullptr));
    for (int count = L; count > 1; count = count / std::min(256, count)) {
        const int blocks = count / std::min(256, count);
        GSICP_CUDA(launch_dependent(level_reduce_kernel, blocks, 256, s, out.boxes.as<float4>(), count));
    }
    GSICP_CUDA(cudaGetLastError());
    return GSICP_OK;
}

// ---------------------------------------------------------------------------------------------
// Batched Morton order of B clouds (batched registration).  Each cloud gets exactly the order
// build_index gives it alone -- 30-bit Morton keys over its own bounding cube, stable sort, ties
// in original order -- by sorting all clouds' keys together and then, stably, by cloud.

// Cloud of global point i: the last b with ofs[b] <= i (empty clouds have equal offsets).
__device__ __forceinline__ int cloud_of(const int64_t* __restrict__ ofs, int B, long i)
{
    int lo = 0, hi = B;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (ofs[mid] <= i) lo = mid;
        else hi = mid;
    }
    return lo;
}

__global__ void seg_bbox_init_kernel(uint32_t* __restrict__ bb, int B)
{
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < 6 * B; t += gridDim.x * blockDim.x)
        bb[t] = (t % 6) < 3 ? 0xffffffffu : 0u;
}

__global__ void seg_bbox_kernel(const float* const* __restrict__ ptrs, const int64_t* __restrict__ ofs, int B,
                                long N, uint32_t* __restrict__ bb)
{
    for (long i0 = (long)blockIdx.x * blockDim.x; i0 < N; i0 += (long)gridDim.x * blockDim.x) {
        const long i = i0 + threadIdx.x;
        const bool in = i < N;
        const int b = in ? cloud_of(ofs, B, i) : -1;
        float v[3] = {0.f, 0.f, 0.f};
        if (in) {
            const float* p = ptrs[b] + 3l * (i - ofs[b]);
            v[0] = p[0]; v[1] = p[1]; v[2] = p[2];
        }
        // lanes of the same cloud combine first (order-preserving integer encoding), then one
        // atomic per cloud and warp
        const unsigned peers = __match_any_sync(0xffffffffu, b);
        const int leader = __ffs(peers) - 1, lane = threadIdx.x & 31;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const uint32_t lo = __reduce_min_sync(peers, f2ord(v[a]));
            const uint32_t hi = __reduce_max_sync(peers, f2ord(v[a]));
            if (in && lane == leader) {
                atomicMin(&bb[6 * b + a], lo);
                atomicMax(&bb[6 * b + 3 + a], hi);
            }
        }
    }
}

__global__ void seg_quant_kernel(const uint32_t* __restrict__ bb, int B, float4* __restrict__ quant)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const uint32_t* q = bb + 6 * b;
    const float lx = ord2f(q[0]), ly = ord2f(q[1]), lz = ord2f(q[2]);
    const float ext = fmaxf(fmaxf(ord2f(q[3]) - lx, ord2f(q[4]) - ly), ord2f(q[5]) - lz);
    quant[b] = make_float4(lx, ly, lz, ext > 0.f ? 1024.f / ext : 0.f);  // as bbox_quant_kernel with no cell
}

__global__ void seg_morton_kernel(const float* const* __restrict__ ptrs, const int64_t* __restrict__ ofs, int B,
                                  long N, const float4* __restrict__ quant, uint32_t* __restrict__ keys,
                                  uint32_t* __restrict__ vals)
{
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long)gridDim.x * blockDim.x) {
        const int b = cloud_of(ofs, B, i);
        const float* p = ptrs[b] + 3l * (i - ofs[b]);
        keys[i] = morton_of(quant[b], p[0], p[1], p[2]);
        vals[i] = (uint32_t)i;
    }
}

__global__ void seg_cloud_keys_kernel(const uint32_t* __restrict__ vals, const int64_t* __restrict__ ofs, int B,
                                      long N, uint32_t* __restrict__ keys)
{
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long)gridDim.x * blockDim.x)
        keys[i] = (uint32_t)cloud_of(ofs, B, vals[i]);
}

__global__ void seg_gather_kernel(const float* const* __restrict__ pts, const float* const* __restrict__ covs,
                                  const int64_t* __restrict__ ofs, int B, long N, const uint32_t* __restrict__ vals,
                                  float4* __restrict__ src_out, float4* __restrict__ covs_out)
{
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (long)gridDim.x * blockDim.x) {
        const long gi = vals[i];
        const int b = cloud_of(ofs, B, gi);
        const long li = gi - ofs[b];
        const float* p = pts[b] + 3 * li;
        src_out[i] = make_float4(p[0], p[1], p[2], __int_as_float((int)li));
        const float* c = covs[b] + 6 * li;
        covs_out[2 * i] = make_float4(c[0], c[1], c[2], c[3]);
        covs_out[2 * i + 1] = make_float4(c[4], c[5], 0.f, 0.f);
    }
}

gsicp_status batch_morton_order(const float* const* pts_dev, const float* const* covs_dev, const int64_t* ofs_dev,
                                int B, long N, float4* src_out, float4* covs_out, BuildScratch& scr, DevBuf& quant,
                                cudaStream_t s)
{
    if (N <= 0) return GSICP_OK;
    if (N > INT32_MAX) return GSICP_ERR_INVALID_ARG;
    GSICP_CHECK(scr.k0.ensure(sizeof(uint32_t) * N));
    GSICP_CHECK(scr.k1.ensure(sizeof(uint32_t) * N));
    GSICP_CHECK(scr.v0.ensure(sizeof(uint32_t) * N));
    GSICP_CHECK(scr.v1.ensure(sizeof(uint32_t) * N));
    GSICP_CHECK(scr.bbox.ensure(sizeof(uint32_t) * 6 * (size_t)B));
    GSICP_CHECK(quant.ensure(sizeof(float4) * (size_t)B));
    const int sms = device_sm_count();
    const int grid = (int)std::max<long>(1, std::min<long>((N + 255) / 256, sms * 8));
    scr.bbox_ready = false;  // the segmented boxes below leave the words in another state
    seg_bbox_init_kernel<<<(6 * B + 255) / 256, 256, 0, s>>>(scr.bbox.as<uint32_t>(), B);
    seg_bbox_kernel<<<grid, 256, 0, s>>>(pts_dev, ofs_dev, B, N, scr.bbox.as<uint32_t>());
    seg_quant_kernel<<<(B + 255) / 256, 256, 0, s>>>(scr.bbox.as<uint32_t>(), B, quant.as<float4>());
    seg_morton_kernel<<<grid, 256, 0, s>>>(pts_dev, ofs_dev, B, N, quant.as<float4>(), scr.k0.as<uint32_t>(),
                                           scr.v0.as<uint32_t>());
    GSICP_CUDA(cudaGetLastError());
    GSICP_CHECK(radix_sort_pairs(scr.k0.as<uint32_t>(), scr.v0.as<uint32_t>(), scr.k1.as<uint32_t>(),
                                 scr.v1.as<uint32_t>(), (int)N, 30, scr.hist, scr.sums, s));
    seg_cloud_keys_kernel<<<grid, 256, 0, s>>>(scr.v0.as<uint32_t>(), ofs_dev, B, N, scr.k0.as<uint32_t>());
    GSICP_CHECK(radix_sort_pairs(scr.k0.as<uint32_t>(), scr.v0.as<uint32_t>(), scr.k1.as<uint32_t>(),
                                 scr.v1.as<uint32_t>(), (int)N, B <= 256 ? 8 : 16, scr.hist, scr.sums, s));
    seg_gather_kernel<<<grid, 256, 0, s>>>(pts_dev, covs_dev, ofs_dev, B, N, scr.v0.as<uint32_t>(), src_out,
                                           covs_out);
    GSICP_CUDA(cudaGetLastError());
    return GSICP_OK;
}

IndexView IndexBufs::view() const
{
    IndexView v;
    v.pts = pts.as<const float4>();
    v.boxes = boxes.as<const float4>();
    v.covs = covs.ptr ? covs.as<const float4>() : nullptr;
    v.n = n_ptr;
    v.keys = keys.ptr ? keys.as<const uint32_t>() : nullptr;
    v.quant = quant.as<const float4>();
    v.grid = has_grid ? grid.as<const int4>() : nullptr;
    v.grid_mask = has_grid ? grid_meta.as<const uint32_t>() : nullptr;
    v.L = L;
    v.B = B;
    return v;
}

}  // namespace gsicp
