// surrogate.cu -- the learned covariance surrogate: a 3-layer 5x5 convolutional network over the
// point map of a depth frame that predicts each point's surface normal, from which the point's
// plane-regularised, scale-aligned covariance (Sec. 3) is built in place of the k-NN step.
//
// Network (bias-free, ReLU; weights bfloat16, activations bfloat16 between layers, every sum in
// float):
//   a1(u)[o] = sum_{d, c} W1[o][c][d] M(u+d) (P_c(u+d) - P_c(u))      3 -> 32 channels
//   h1 = bf16(relu(a1)) M,   a2 = W2 * h1,   h2 = bf16(relu(a2)) M       32 -> 32
//   v = W3 * h2,   n = v / |v|,   C = (I - (1 - eps) n n^T) z^(-2p)      32 -> 3
// over the stride-sampled grid (P the back-projected samples, M their validity), 5 x 5 taps read
// (i + dy - 2, j + dx - 2), zero outside the image.  Centred differences make layer 1 blind to
// the patch's position; without biases every layer is positively homogeneous, so n does not
// depend on the distance to the surface.
//
// Training minimises the mean over points with a k-NN target of 1 - n^T T n, T = (I - C_knn
// z^(2p)) / (1 - eps) the projector on the k-NN normal (points whose k-NN covariance is not a plane
// one, trace(T) off 1, are skipped); back-propagation treats the bfloat16 roundings as the
// identity; Adam (Kingma & Ba) updates float master weights.
//
// Layout: per-pixel tensors channels-last over the sample grid (h1, h2: 32 bfloat16 = 64 B per
// pixel; gradients float).  Forward: layer 1 on CUDA cores (float: the centred differences need
// it), layers 2 and 3 as tcgen05 implicit GEMMs fed by TMA (sg_conv_tc_kernel).  Training kernels
// (CUDA cores, float) work on 16 x 16 output tiles with a 2-pixel halo staged in shared memory,
// channel-major ([c][20 * 20 + 1]) so that lanes that differ in pixel or in channel hit distinct
// banks, weights staged in shared memory and read as broadcasts.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <new>

#include "internal.h"

namespace gsicp {

gsicp_status set_error(gsicp_status st, const char* msg);

constexpr int SG_T = 16;               // output tile side
constexpr int SG_HS = SG_T + 4;        // halo tile side
constexpr int SG_HP = SG_HS * SG_HS;   // halo positions (400)
constexpr int SG_HPAD = SG_HP + 1;     // channel stride in shared memory
constexpr int SG_C = 32;               // hidden channels
constexpr int SG_TAPS = 25;
constexpr int SG_NW1 = SG_C * 3 * SG_TAPS, SG_NW2 = SG_C * SG_C * SG_TAPS, SG_NW3 = 3 * SG_C * SG_TAPS;
constexpr int SG_NW = SG_NW1 + SG_NW2 + SG_NW3;
static_assert(SG_NW == GSICP_SURROGATE_WEIGHTS, "weight count");

// CUDA-core layouts of the bfloat16-rounded weights (float values), in one buffer (layers 2 and 3
// run forward on the tensor cores from their own bfloat16 layouts):
constexpr int WK_W1 = 0;                           // float4 [25 t][32 o]: (W1[o][0..2][t], 0)
constexpr int WK_W2T = WK_W1 + 4 * SG_TAPS * SG_C; // float  [32 o][25 t][32 c]: W2[o][c][24 - t] (backward)
constexpr int WK_W3T = WK_W2T + SG_NW2;            // float4 [25 t][32 c]: (W3[0..2][c][24 - t], 0) (backward)
constexpr int WK_TOTAL = WK_W3T + 4 * SG_TAPS * SG_C;

}  // namespace gsicp

struct gsicp_surrogate_s {
    int device = 0;
    gsicp::DevBuf w, m, s, g;      // float [SG_NW]: master weights, Adam moments, gradient sums
    gsicp::DevBuf wk;              // kernel layouts (WK_TOTAL floats)
    gsicp::DevBuf wmma;            // layers 2 and 3 as tensor-core B operands (bfloat16, see sg_conv_tc_kernel)
    unsigned* err = nullptr;       // pinned, device-visible: a bounded wait of a kernel ran out
    bool timing = false;           // record events around the layers of every forward
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    gsicp::DevBuf grid, h1, h2, v, dv, da2, da1;  // per-pixel buffers
    gsicp::DevBuf scal;            // double loss sum | unsigned long long target count
    int64_t pix_cap = 0;
    int steps = 0;                 // Adam steps taken
};

namespace gsicp {

namespace {

__device__ __forceinline__ int halo_of(int t, int tx, int ty) { return (ty + t / 5) * SG_HS + tx + t % 5; }

// ---------------------------------------------------------------------------------------------
// grid and weight preparation

__global__ void sg_grid_kernel(const float* __restrict__ pts, const int* __restrict__ idx_img, int npix,
                               float4* __restrict__ grid)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npix) return;
    const int id = idx_img[i];
    grid[i] = id >= 0 ? make_float4(pts[3l * id], pts[3l * id + 1], pts[3l * id + 2], 1.f)
                      : make_float4(0.f, 0.f, 0.f, 0.f);
}

__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

__global__ void sg_layout_kernel(const float* __restrict__ w, float* __restrict__ wk, __nv_bfloat16* __restrict__ w2mma)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < SG_NW1) {  // W1[o][c][t]
        const int o = i / 75, c = (i / 25) % 3, t = i % 25;
        wk[WK_W1 + 4 * (t * SG_C + o) + c] = bf16r(w[i]);
        if (c == 0) wk[WK_W1 + 4 * (t * SG_C + o) + 3] = 0.f;
    } else if (i < SG_NW1 + SG_NW2) {  // W2[o][c][t]
        const int j = i - SG_NW1, o = j / 800, c = (j / 25) % 32, t = j % 25;
        const float v = bf16r(w[i]);
        wk[WK_W2T + (o * SG_TAPS + (24 - t)) * SG_C + c] = v;
        // tensor-core B operand: [tap t][channel group c / 8][output o][c % 8]
        w2mma[((t * 4 + c / 8) * SG_C + o) * 8 + c % 8] = __float2bfloat16_rn(v);
    } else if (i < SG_NW) {  // W3[o][c][t]
        const int j = i - SG_NW1 - SG_NW2, o = j / 800, c = (j / 25) % 32, t = j % 25;
        const float v = bf16r(w[i]);
        wk[WK_W3T + 4 * ((24 - t) * SG_C + c) + o] = v;
        if (o == 0) wk[WK_W3T + 4 * ((24 - t) * SG_C + c) + 3] = 0.f;
        // tensor-core B operand of layer 3 (after layer 2's): [tap][group][16 outputs, 3 used][8]
        w2mma[SG_NW2 + ((t * 4 + c / 8) * 16 + o) * 8 + c % 8] = __float2bfloat16_rn(v);
    }
}

// Stage a channels-last 32-channel tensor's halo tile into shared memory as float [c][SG_HPAD].
template <bool kBf16>
__device__ __forceinline__ void stage32(const void* __restrict__ in, int w, int h, int x0, int y0, float* tile)
{
    for (int q = threadIdx.x; q < SG_HP * 4; q += blockDim.x) {
        const int pos = q >> 2, part = q & 3;
        const int yy = y0 + pos / SG_HS - 2, xx = x0 + pos % SG_HS - 2;
        float v[8];
        if (yy >= 0 && yy < h && xx >= 0 && xx < w) {
            const long pix = (long)yy * w + xx;
            if (kBf16) {
                const uint4 raw = reinterpret_cast<const uint4*>(in)[pix * 4 + part];
                const __nv_bfloat162* b = reinterpret_cast<const __nv_bfloat162*>(&raw);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const float2 f = __bfloat1622float2(b[k]);
                    v[2 * k] = f.x;
                    v[2 * k + 1] = f.y;
                }
            } else {
                const float4 a = reinterpret_cast<const float4*>(in)[pix * 8 + 2 * part];
                const float4 b = reinterpret_cast<const float4*>(in)[pix * 8 + 2 * part + 1];
                v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
                v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
            }
        } else {
#pragma unroll
            for (int k = 0; k < 8; ++k) v[k] = 0.f;
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) tile[(part * 8 + k) * SG_HPAD + pos] = v[k];
    }
}

__device__ __forceinline__ void store_bf16x16(__nv_bfloat16* dst, const float* v)
{
    uint4 out[2];
    __nv_bfloat162* b = reinterpret_cast<__nv_bfloat162*>(out);
#pragma unroll
    for (int k = 0; k < 8; ++k) b[k] = __floats2bfloat162_rn(v[2 * k], v[2 * k + 1]);
    reinterpret_cast<uint4*>(dst)[0] = out[0];
    reinterpret_cast<uint4*>(dst)[1] = out[1];
}

// ---------------------------------------------------------------------------------------------
// forward

// Layer 1 (centred differences, 3 -> 32) + ReLU + bfloat16, zero at invalid pixels.  The 16 x 16
// tile's 20 x 20 halo of points and the weights sit in shared memory; each thread computes two
// vertically adjacent pixels, so every weight read (a broadcast) feeds both; an invalid neighbour
// contributes its difference times 0.  The tap loop stays rolled: unrolled, the 4800 multiply-adds
// overflow the instruction cache.
constexpr int SG_L1_THREADS = SG_T * SG_T / 2;

__global__ void __launch_bounds__(SG_L1_THREADS) sg_l1_kernel(const float4* __restrict__ grid, int w, int h,
                                                              const float4* __restrict__ w1k,
                                                              __nv_bfloat16* __restrict__ h1)
{
    __shared__ float4 tile[SG_HP];
    __shared__ float4 ws[SG_TAPS * SG_C];
    const int x0 = blockIdx.x * SG_T, y0 = blockIdx.y * SG_T;
    for (int i = threadIdx.x; i < SG_TAPS * SG_C; i += blockDim.x) ws[i] = w1k[i];
    for (int q = threadIdx.x; q < SG_HP; q += blockDim.x) {
        const int yy = y0 + q / SG_HS - 2, xx = x0 + q % SG_HS - 2;
        tile[q] = (yy >= 0 && yy < h && xx >= 0 && xx < w) ? grid[(long)yy * w + xx] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncthreads();
    const int tx = threadIdx.x % SG_T, ty = 2 * (threadIdx.x / SG_T);  // pixels (tx, ty) and (tx, ty + 1)
    const int x = x0 + tx, y = y0 + ty;
    if (x >= w || y >= h) return;
    const float4 c0 = tile[(ty + 2) * SG_HS + tx + 2], c1 = tile[(ty + 3) * SG_HS + tx + 2];
    float a0[SG_C], a1[SG_C];
#pragma unroll
    for (int o = 0; o < SG_C; ++o) a0[o] = a1[o] = 0.f;
#pragma unroll 1
    for (int t = 0; t < SG_TAPS; ++t) {
        const float4 n0 = tile[halo_of(t, tx, ty)], n1 = tile[halo_of(t, tx, ty + 1)];
        const float dx0 = (n0.x - c0.x) * n0.w, dy0 = (n0.y - c0.y) * n0.w, dz0 = (n0.z - c0.z) * n0.w;
        const float dx1 = (n1.x - c1.x) * n1.w, dy1 = (n1.y - c1.y) * n1.w, dz1 = (n1.z - c1.z) * n1.w;
        const float4* wt = ws + t * SG_C;
#pragma unroll
        for (int o = 0; o < SG_C; ++o) {
            const float4 wv = wt[o];
            a0[o] = fmaf(wv.x, dx0, fmaf(wv.y, dy0, fmaf(wv.z, dz0, a0[o])));
            a1[o] = fmaf(wv.x, dx1, fmaf(wv.y, dy1, fmaf(wv.z, dz1, a1[o])));
        }
    }
#pragma unroll
    for (int o = 0; o < SG_C; ++o) {
        a0[o] = c0.w != 0.f ? fmaxf(a0[o], 0.f) : 0.f;
        a1[o] = c1.w != 0.f ? fmaxf(a1[o], 0.f) : 0.f;
    }
    __nv_bfloat16* dst = h1 + ((long)y * w + x) * SG_C;
    store_bf16x16(dst, a0);
    store_bf16x16(dst + 16, a0 + 16);
    if (y + 1 < h) {
        dst += (long)w * SG_C;
        store_bf16x16(dst, a1);
        store_bf16x16(dst + 16, a1 + 16);
    }
}

// Back-propagation through layer 2: da1 = [h1 > 0] (W2 transposed * da2), a 32 -> 32 channel 5 x 5
// convolution of the float da2 with the flipped, channel-swapped weights wk ([32 in][25 t][32 out]),
// output channels [16 half, 16 half + 16), gated by h1 > 0.  Float on CUDA cores (training only).
// Dynamic shared memory: SG_C * SG_HPAD + 32 * 25 * 16 floats.
__global__ void __launch_bounds__(256) sg_dl2_kernel(const float* __restrict__ da2, int w, int h,
                                                     const float* __restrict__ wk,
                                                     const __nv_bfloat16* __restrict__ h1, float* __restrict__ da1)
{
    extern __shared__ float sm[];
    float* tile = sm;                       // [32][SG_HPAD]
    float* ws = sm + SG_C * SG_HPAD;        // [32 c][25 t][16 o]
    const int half = blockIdx.z;
    const int x0 = blockIdx.x * SG_T, y0 = blockIdx.y * SG_T;
    for (int i = threadIdx.x; i < SG_C * SG_TAPS * 16; i += blockDim.x) {
        const int ct = i >> 4, o = i & 15;
        ws[i] = wk[ct * SG_C + 16 * half + o];
    }
    stage32<false>(da2, w, h, x0, y0, tile);
    __syncthreads();
    const int tx = threadIdx.x % SG_T, ty = threadIdx.x / SG_T;
    const int x = x0 + tx, y = y0 + ty;
    if (x >= w || y >= h) return;
    float acc[16];
#pragma unroll
    for (int o = 0; o < 16; ++o) acc[o] = 0.f;
    for (int c = 0; c < SG_C; ++c) {
        const float* tc = tile + c * SG_HPAD;
        const float4* wc = reinterpret_cast<const float4*>(ws + c * SG_TAPS * 16);
#pragma unroll 5
        for (int t = 0; t < SG_TAPS; ++t) {
            const float xv = tc[halo_of(t, tx, ty)];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float4 wv = wc[t * 4 + q];
                acc[4 * q + 0] = fmaf(wv.x, xv, acc[4 * q + 0]);
                acc[4 * q + 1] = fmaf(wv.y, xv, acc[4 * q + 1]);
                acc[4 * q + 2] = fmaf(wv.z, xv, acc[4 * q + 2]);
                acc[4 * q + 3] = fmaf(wv.w, xv, acc[4 * q + 3]);
            }
        }
    }
    const long pix = (long)y * w + x;
    const __nv_bfloat16* gp = h1 + pix * SG_C + 16 * half;
    float4* dst = reinterpret_cast<float4*>(da1 + pix * SG_C + 16 * half);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        float r[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) r[k] = __bfloat162float(gp[4 * q + k]) > 0.f ? acc[4 * q + k] : 0.f;
        dst[q] = make_float4(r[0], r[1], r[2], r[3]);
    }
}

// The plane covariance on n = v / |v| with the scale aligning factor z^(-2p): (I - (1 - eps) n n^T)
// z^(-2p) as (xx, xy, xz, yy, yz, zz); |v| = 0 gives the isotropic z^(-2p) I.
__device__ __forceinline__ void plane_cov_from_v(float v0, float v1, float v2, float z, float eps, float p, float* C)
{
    const float s = powf(z, -2.f * p);
    const float nn = sqrtf(fmaf(v0, v0, fmaf(v1, v1, v2 * v2)));
    if (!(nn > 0.f)) {
        C[0] = s; C[1] = 0.f; C[2] = 0.f; C[3] = s; C[4] = 0.f; C[5] = s;
        return;
    }
    const float n0 = v0 / nn, n1 = v1 / nn, n2 = v2 / nn, k = 1.f - eps;
    C[0] = (1.f - k * n0 * n0) * s;
    C[1] = (-k * n0 * n1) * s;
    C[2] = (-k * n0 * n2) * s;
    C[3] = (1.f - k * n1 * n1) * s;
    C[4] = (-k * n1 * n2) * s;
    C[5] = (1.f - k * n2 * n2) * s;
}

// Layers 2 and 3 on the tensor cores (tcgen05, an implicit GEMM).  A CTA of 4 warps takes output
// tiles of 8 x 16 pixels = the 128 rows of one MMA (M = 128, K = 16 per instruction, bfloat16
// operands, float accumulator in tensor memory; N = 32 output channels for layer 2, 16 for layer
// 3, whose 3 outputs are padded with zero weights).  The 32-channel input's halo of the tile (12 x
// 20 pixels) is brought into shared memory by the tensor-memory-access unit as four 8-channel
// boxes (one 3-D tiled copy each: 8 channels x 12 columns x 20 rows, zero outside the image) that
// land as [group][halo row][halo column][16 B]: the canonical K-major layout without swizzle, in
// which a core matrix (8 rows x 16 B) is one output row's 8 pixels shifted by the tap, so the A
// operand of every tap is the same staged tile seen through a descriptor with its own start address
// (row stride SBO = one halo row, K stride LBO = one channel plane).  The weights (B,
// [tap][group][output][8 channels]) arrive once per CTA by one bulk copy.  Two tile buffers and two
// accumulators in tensor memory: the next tile's 50 MMAs (25 taps x 2 channel halves) are issued
// into the other accumulator before the current tile's epilogue and run under it; a buffer is
// refilled with the tile after next as soon as its tile's MMAs complete.  One thread issues copies
// and MMAs; each accumulator's MMAs are committed to its own mbarrier; the epilogue reads the
// accumulator (warp w: rows 32w..32w+31) with tcgen05.ld.  Layer 2's epilogue applies ReLU, the validity mask and bfloat16
// rounding and writes h2; layer 3's writes v and the point's plane covariance.  Every wait is
// bounded: when one runs out the CTA records it in err, waits (bounded) for its copies in flight,
// frees its tensor memory and returns.
constexpr int TC_TW = 8, TC_TH = 16;                  // output tile (128 pixels)
constexpr int TC_HW = TC_TW + 4, TC_HH = TC_TH + 4;   // halo tile 12 x 20
constexpr int TC_PLANE = TC_HW * TC_HH * 16;          // one 8-channel plane of the halo: 3840 B (30 x 128)
constexpr int TC_A_BYTES = 4 * TC_PLANE;              // 15360 B per tile buffer
template <int kN>
constexpr int tc_b_bytes() { return SG_TAPS * 4 * kN * 16; }
// slack after B, so that every descriptor's reach, read with LBO and SBO either way round, stays
// inside the allocation (at most 23872 + 15 x 3840 + 319 = 81791 bytes from the base)
template <int kN>
constexpr int tc_pad() { return kN == 16 ? 28672 : 4096; }
template <int kN>
constexpr size_t tc_smem() { return 2 * TC_A_BYTES + tc_b_bytes<kN>() + tc_pad<kN>(); }
static_assert(2 * TC_A_BYTES + 25600 + 28672 > 81791 && 2 * TC_A_BYTES + 51200 + 4096 > 81791, "descriptor slack");
constexpr unsigned TC_SPIN_LIMIT = 1u << 22;
// instruction descriptor, kind::f16: D float (bit 4), A and B bfloat16 (bits 7, 10), both K-major,
// N / 8 at bit 17, M / 16 at bit 24
template <int kN>
constexpr uint32_t tc_idesc() { return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kN >> 3) << 17) | ((128u >> 4) << 24); }

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor, canonical layout without swizzle: start address, the byte
// distance between core matrices along K (lbo) and along M or N (sbo), all in 16-byte units;
// descriptor version 1 (bit 46).  Shared-memory addresses are below 2^18, so start addresses fit
// the 14-bit field and adding a 16-byte-unit offset to a descriptor moves only its start address.
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr >> 4) & 0x3fffu) | ((uint64_t)((lbo >> 4) & 0x3fffu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3fffu) << 32) | (1ull << 46);
}

// Bounded wait for the completion of the mbarrier phase with this parity; true if it completed.
__device__ __forceinline__ bool tc_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok = 0;
    for (unsigned it = 0; it < TC_SPIN_LIMIT && !ok; ++it)
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     "selp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
    return ok != 0;
}

__device__ __forceinline__ void tc_expect(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// The four 8-channel boxes of the halo of the tile at (x0, y0) into tile buffer dst.
__device__ __forceinline__ void tc_load_tile(const CUtensorMap* tmap, uint32_t dst, int x0, int y0, uint32_t bar)
{
    tc_expect(bar, TC_A_BYTES);
#pragma unroll
    for (int g = 0; g < 4; ++g)
        asm volatile("cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
                     "[%0], [%1, {%2, %3, %4}], [%5];"
                     ::"r"(dst + g * TC_PLANE), "l"(reinterpret_cast<uint64_t>(tmap)), "r"(8 * g), "r"(x0 - 2),
                       "r"(y0 - 2), "r"(bar)
                     : "memory");
}

template <int kN>
__global__ void __launch_bounds__(128) sg_conv_tc_kernel(const __grid_constant__ CUtensorMap tmap, int w, int h,
                                                         const uint4* __restrict__ wb,
                                                         const float4* __restrict__ grid,
                                                         __nv_bfloat16* __restrict__ h2, const int* __restrict__ idx_img,
                                                         float eps, float p, float* __restrict__ covs,
                                                         float* __restrict__ v_out, unsigned* __restrict__ err)
{
    static_assert(kN == 32 || kN == 16, "layer 2 (N = 32) or layer 3 (N = 16)");
    constexpr uint32_t kCols = 2 * kN < 32 ? 32u : 2u * kN;  // two accumulators (an allocation is >= 32 columns)
    extern __shared__ __align__(1024) uint8_t tc_smem_[];
    uint8_t* sB = tc_smem_ + 2 * TC_A_BYTES;
    __shared__ __align__(8) uint64_t bars[5];  // B copy, tile buffers 0 and 1, MMAs done into accumulators 0 and 1
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tiles_x = (w + TC_TW - 1) / TC_TW, tiles_y = (h + TC_TH - 1) / TC_TH;
    const int ntiles = tiles_x * tiles_y;
    const uint32_t a0 = smem_u32(tc_smem_), b0 = smem_u32(sB);
    const uint32_t bar_b = smem_u32(&bars[0]);
    auto bar_a = [&](int buf) { return smem_u32(&bars[1 + buf]); };
    auto bar_m = [&](int acc) { return smem_u32(&bars[3 + acc]); };
    auto tile_x0 = [&](int tile) { return (tile % tiles_x) * TC_TW; };
    auto tile_y0 = [&](int tile) { return (tile / tiles_x) * TC_TH; };
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(kCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    const int t0 = blockIdx.x, t1 = blockIdx.x + gridDim.x;
    if (tid == 0) {
        for (int i = 0; i < 5; ++i) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bars[i])));
        asm volatile("fence.mbarrier_init.release.cluster;");
        // the weights: one bulk copy; the first two tiles: four box copies each
        tc_expect(bar_b, tc_b_bytes<kN>());
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                     ::"r"(b0), "l"(reinterpret_cast<uint64_t>(wb)), "r"(tc_b_bytes<kN>()), "r"(bar_b)
                     : "memory");
        if (t0 < ntiles) tc_load_tile(&tmap, a0, tile_x0(t0), tile_y0(t0), bar_a(0));
        if (t1 < ntiles) tc_load_tile(&tmap, a0 + TC_A_BYTES, tile_x0(t1), tile_y0(t1), bar_a(1));
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = tmem_base;
    // thread 0: tile buffer buf's 50 MMAs (25 taps x 2 channel halves) into accumulator acc, committed
    // to bar_m(acc); the 50 descriptors differ only in their start address (the low 14 bits, in
    // 16-byte units, which no offset here carries out of): base + constant
    auto issue = [&](int buf, int acc) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint64_t da0 = tc_desc(a0 + buf * TC_A_BYTES, TC_PLANE, TC_HW * 16), db0 = tc_desc(b0, kN * 16, 128);
        const uint32_t d = tmem + (uint32_t)(acc * kN);
#pragma unroll
        for (int t = 0; t < SG_TAPS; ++t) {
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const uint64_t da = da0 + (uint64_t)((2 * j * TC_PLANE + ((t / 5) * TC_HW + t % 5) * 16) >> 4);
                const uint64_t db = db0 + (uint64_t)(((t * 4 + 2 * j) * (kN * 16)) >> 4);
                asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                             "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                             ::"r"(d), "l"(da), "l"(db), "r"(tc_idesc<kN>()), "r"((t | j) != 0 ? 1u : 0u));
            }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                     ::"r"(bar_m(acc)) : "memory");
    };
    // copies and MMAs this CTA started and has not yet seen complete (thread 0's bookkeeping): on a
    // wait that runs out they are waited for again before the CTA leaves
    bool failed = false, b_pending = true;
    bool a_pend[2] = {t0 < ntiles, t1 < ntiles}, m_pend[2] = {false, false};
    uint32_t a_par[2] = {0u, 0u}, m_par[2] = {0u, 0u};
    if (tid == 0) {
        failed = !tc_wait(bar_b, 0);
        b_pending = failed;
        if (!failed && t0 < ntiles) {
            failed = !tc_wait(bar_a(0), 0);
            if (!failed) {
                a_pend[0] = false;
                issue(0, 0);
                m_pend[0] = true;
            }
        }
    }
    int k = 0;
    if (!__syncthreads_or(failed)) {
        // Tile k: its MMAs were issued one step earlier (into accumulator k mod 2); tile k + 1's are
        // issued now, into the other accumulator, so that they run under tile k's epilogue.
        for (int tile = t0; tile < ntiles; tile += gridDim.x, ++k) {
            const int buf = k & 1, acc = k & 1;
            const int next = tile + gridDim.x;
            bool bad = false;
            if (tid == 0 && next < ntiles) {
                bad = !tc_wait(bar_a(buf ^ 1), ((k + 1) >> 1) & 1);
                if (!bad) {
                    a_pend[buf ^ 1] = false;
                    issue(buf ^ 1, acc ^ 1);
                    m_pend[acc ^ 1] = true;
                    m_par[acc ^ 1] = ((k + 1) >> 1) & 1;
                }
            }
            // the epilogue's inputs, which do not depend on the MMAs, are read while they run
            const int x0 = tile_x0(tile), y0 = tile_y0(tile);
            const int pr = warp * 32 + lane, x = x0 + (pr & 7), y = y0 + (pr >> 3);
            const bool inside = x < w && y < h;
            const long pix = (long)y * w + x;
            const float4 g = inside ? grid[pix] : make_float4(0.f, 0.f, 0.f, 0.f);
            const bool valid = inside && g.w != 0.f;
            const int id = kN == 16 && valid && covs ? idx_img[pix] : -1;
            if (__syncthreads_or(bad)) {
                failed = true;
                break;
            }
            if (__syncthreads_or(!tc_wait(bar_m(acc), (k >> 1) & 1))) {
                failed = true;
                break;
            }
            if (tid == 0) {
                m_pend[acc] = false;
                // tile k's MMAs are done, so its buffer is free: tile k + 2's copy goes into it
                const int after = tile + 2 * gridDim.x;
                if (after < ntiles) {
                    tc_load_tile(&tmap, a0 + buf * TC_A_BYTES, tile_x0(after), tile_y0(after), bar_a(buf));
                    a_pend[buf] = true;
                    a_par[buf] = ((k + 2) >> 1) & 1;
                }
            }
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(acc * kN);
            if (kN == 32) {
                uint32_t r[32];
                asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                             "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
                             "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
                             : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                               "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
                               "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
                               "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
                               "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
                               "=r"(r[31])
                             : "r"(taddr));
                asm volatile("tcgen05.wait::ld.sync.aligned;");
                if (inside) {
                    float v[32];
#pragma unroll
                    for (int q = 0; q < 32; ++q) v[q] = valid ? fmaxf(__uint_as_float(r[q]), 0.f) : 0.f;
                    store_bf16x16(h2 + pix * SG_C, v);
                    store_bf16x16(h2 + pix * SG_C + 16, v + 16);
                }
            } else {
                uint32_t r[4];
                asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
                             : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(taddr));
                asm volatile("tcgen05.wait::ld.sync.aligned;");
                if (inside) {
                    const float v0 = valid ? __uint_as_float(r[0]) : 0.f, v1 = valid ? __uint_as_float(r[1]) : 0.f,
                                v2 = valid ? __uint_as_float(r[2]) : 0.f;
                    if (v_out) {
                        v_out[3 * pix] = v0;
                        v_out[3 * pix + 1] = v1;
                        v_out[3 * pix + 2] = v2;
                    }
                    if (id >= 0) plane_cov_from_v(v0, v1, v2, g.z, eps, p, covs + 6l * id);
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncthreads();  // accumulator acc read before tile k + 2's MMAs overwrite it
        }
    }
    if (failed && tid == 0) {
        *reinterpret_cast<volatile unsigned*>(err) = 1u;  // pinned host word
        // no copy may land and no MMA may read after the CTA is gone (each wait bounded again)
        if (b_pending) tc_wait(bar_b, 0);
        for (int b = 0; b < 2; ++b)
            if (a_pend[b]) tc_wait(bar_a(b), a_par[b]);
        for (int a = 0; a < 2; ++a)
            if (m_pend[a]) tc_wait(bar_m(a), m_par[a]);
    }
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols));
    }
}

// ---------------------------------------------------------------------------------------------
// training

// Loss and dL/dv (without the 1/N of the mean: the gradient sums are scaled when applied).
__global__ void sg_loss_kernel(const float* __restrict__ v, const float4* __restrict__ grid,
                               const int* __restrict__ idx_img, const float* __restrict__ covs_knn, int npix,
                               float eps, float p, float* __restrict__ dv, double* __restrict__ loss_sum,
                               unsigned long long* __restrict__ count)
{
    __shared__ double sl[8];
    __shared__ unsigned sc[8];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    double l = 0.0;
    unsigned cnt = 0u;
    float g0 = 0.f, g1 = 0.f, g2 = 0.f;
    if (i < npix && grid[i].w != 0.f && idx_img[i] >= 0) {
        const float* C = covs_knn + 6l * idx_img[i];
        const float s = powf(grid[i].z, 2.f * p), inv = 1.f / (1.f - eps);
        const float T00 = (1.f - C[0] * s) * inv, T01 = (-C[1] * s) * inv, T02 = (-C[2] * s) * inv;
        const float T11 = (1.f - C[3] * s) * inv, T12 = (-C[4] * s) * inv, T22 = (1.f - C[5] * s) * inv;
        if (fabsf(T00 + T11 + T22 - 1.f) < 0.01f) {
            cnt = 1u;
            const float a = v[3l * i], b = v[3l * i + 1], c = v[3l * i + 2];
            const float nn = sqrtf(fmaf(a, a, fmaf(b, b, c * c)));
            if (nn > 0.f) {
                const float n0 = a / nn, n1 = b / nn, n2 = c / nn;
                const float t0 = T00 * n0 + T01 * n1 + T02 * n2;
                const float t1 = T01 * n0 + T11 * n1 + T12 * n2;
                const float t2 = T02 * n0 + T12 * n1 + T22 * n2;
                const float q = n0 * t0 + n1 * t1 + n2 * t2;
                l = 1.0 - (double)q;
                // dL/dn = -2 T n; dL/dv = (I - n n^T) dL/dn / |v|
                const float e0 = -2.f * t0, e1 = -2.f * t1, e2 = -2.f * t2;
                const float ne = n0 * e0 + n1 * e1 + n2 * e2;
                g0 = (e0 - n0 * ne) / nn;
                g1 = (e1 - n1 * ne) / nn;
                g2 = (e2 - n2 * ne) / nn;
            } else {
                l = 1.0;
            }
        }
    }
    if (i < npix) {
        dv[3l * i] = g0;
        dv[3l * i + 1] = g1;
        dv[3l * i + 2] = g2;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        l += __shfl_xor_sync(0xffffffffu, l, o);
        cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    }
    if (lane == 0) {
        sl[warp] = l;
        sc[warp] = cnt;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double L = 0.0;
        unsigned long long N = 0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
            L += sl[k];
            N += sc[k];
        }
        if (N) {
            atomicAdd(loss_sum, L);
            atomicAdd(count, N);
        }
    }
}

// dW3[o][c][t] += sum over the tile's pixels of dv[o](u) h2[c](u + d_t).
__global__ void __launch_bounds__(256) sg_gw3_kernel(const float* __restrict__ dv, const __nv_bfloat16* __restrict__ h2,
                                                     int w, int h, float* __restrict__ gw3)
{
    extern __shared__ float sm[];
    float* tile = sm;                         // h2 halo [32][SG_HPAD]
    float* dt = sm + SG_C * SG_HPAD;          // dv [3][256]
    const int x0 = blockIdx.x * SG_T, y0 = blockIdx.y * SG_T;
    stage32<true>(h2, w, h, x0, y0, tile);
    {
        const int tx = threadIdx.x % SG_T, ty = threadIdx.x / SG_T, x = x0 + tx, y = y0 + ty;
        const bool in = x < w && y < h;
        const long pix = (long)y * w + x;
#pragma unroll
        for (int o = 0; o < 3; ++o) dt[o * 256 + threadIdx.x] = in ? dv[3 * pix + o] : 0.f;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < SG_NW3; j += blockDim.x) {
        const int o = j / 800, c = (j / 25) % 32, t = j % 25;
        const float* tc = tile + c * SG_HPAD;
        const float* d = dt + o * 256;
        float acc = 0.f;
        for (int q = 0; q < 256; ++q) acc = fmaf(d[q], tc[halo_of(t, q % SG_T, q / SG_T)], acc);
        if (acc != 0.f) atomicAdd(gw3 + j, acc);
    }
}

// da2[c](u) = [h2[c](u) > 0] sum_{t, o} W3[o][c][24 - t] dv[o](u + d_t)  (layer 3 transposed).
__global__ void __launch_bounds__(256) sg_dl3_kernel(const float* __restrict__ dv, int w, int h,
                                                     const float4* __restrict__ w3t,
                                                     const __nv_bfloat16* __restrict__ h2, float* __restrict__ da2)
{
    __shared__ float4 tile[SG_HP];
    __shared__ float4 ws[SG_TAPS * SG_C];
    const int x0 = blockIdx.x * SG_T, y0 = blockIdx.y * SG_T;
    for (int i = threadIdx.x; i < SG_TAPS * SG_C; i += blockDim.x) ws[i] = w3t[i];
    for (int q = threadIdx.x; q < SG_HP; q += blockDim.x) {
        const int yy = y0 + q / SG_HS - 2, xx = x0 + q % SG_HS - 2;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (yy >= 0 && yy < h && xx >= 0 && xx < w) {
            const long pix = (long)yy * w + xx;
            v = make_float4(dv[3 * pix], dv[3 * pix + 1], dv[3 * pix + 2], 0.f);
        }
        tile[q] = v;
    }
    __syncthreads();
    const int tx = threadIdx.x % SG_T, ty = threadIdx.x / SG_T;
    const int x = x0 + tx, y = y0 + ty;
    if (x >= w || y >= h) return;
    float acc[SG_C];
#pragma unroll
    for (int c = 0; c < SG_C; ++c) acc[c] = 0.f;
    for (int t = 0; t < SG_TAPS; ++t) {
        const float4 d = tile[halo_of(t, tx, ty)];
        if (d.x == 0.f && d.y == 0.f && d.z == 0.f) continue;
#pragma unroll
        for (int c = 0; c < SG_C; ++c) {
            const float4 wv = ws[t * SG_C + c];
            acc[c] = fmaf(wv.x, d.x, fmaf(wv.y, d.y, fmaf(wv.z, d.z, acc[c])));
        }
    }
    const long pix = (long)y * w + x;
    const __nv_bfloat16* gp = h2 + pix * SG_C;
    float4* dst = reinterpret_cast<float4*>(da2 + pix * SG_C);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        float r[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) r[k] = __bfloat162float(gp[4 * q + k]) > 0.f ? acc[4 * q + k] : 0.f;
        dst[q] = make_float4(r[0], r[1], r[2], r[3]);
    }
}

// dW2[o][c][t] += sum over the tile's pixels of da2[o](u) h1[c](u + d_t).  Thread (c = lane,
// o-group = warp) holds 4 outputs x 5 taps of one tap row at a time.
__global__ void __launch_bounds__(256) sg_gw2_kernel(const float* __restrict__ da2, const __nv_bfloat16* __restrict__ h1,
                                                     int w, int h, float* __restrict__ gw2)
{
    extern __shared__ float sm[];
    float* tile = sm;                      // h1 halo [32][SG_HPAD]
    float* dt = sm + SG_C * SG_HPAD;       // da2 [32 o][256]
    const int x0 = blockIdx.x * SG_T, y0 = blockIdx.y * SG_T;
    stage32<true>(h1, w, h, x0, y0, tile);
    {
        const int tx = threadIdx.x % SG_T, ty = threadIdx.x / SG_T, x = x0 + tx, y = y0 + ty;
        const bool in = x < w && y < h;
        const long pix = (long)y * w + x;
        for (int o = 0; o < SG_C; ++o) dt[o * 256 + threadIdx.x] = in ? da2[pix * SG_C + o] : 0.f;
    }
    __syncthreads();
    const int c = threadIdx.x & 31, og = threadIdx.x >> 5;
    const float* tc = tile + c * SG_HPAD;
    for (int dy = 0; dy < 5; ++dy) {
        float acc[4][5];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 5; ++b) acc[a][b] = 0.f;
        for (int q = 0; q < 256; ++q) {
            const int qx = q % SG_T, qy = q / SG_T;
            float d[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) d[a] = dt[(4 * og + a) * 256 + q];
            const float* row = tc + (qy + dy) * SG_HS + qx;
#pragma unroll
            for (int b = 0; b < 5; ++b) {
                const float xv = row[b];
#pragma unroll
                for (int a = 0; a < 4; ++a) acc[a][b] = fmaf(d[a], xv, acc[a][b]);
            }
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 5; ++b)
                if (acc[a][b] != 0.f) atomicAdd(gw2 + (4 * og + a) * 800 + c * 25 + dy * 5 + b, acc[a][b]);
    }
}

// dW1[o][c][t] += sum over the tile's pixels of da1[o](u) M(u + d_t) (P_c(u + d_t) - P_c(u)).
__global__ void __launch_bounds__(256) sg_gw1_kernel(const float* __restrict__ da1, const float4* __restrict__ grid,
                                                     int w, int h, float* __restrict__ gw1)
{
    extern __shared__ float sm[];
    float4* tile = reinterpret_cast<float4*>(sm);   // grid halo [SG_HP]
    float* dt = sm + 4 * SG_HP;                      // da1 [32 o][256]
    const int x0 = blockIdx.x * SG_T, y0 = blockIdx.y * SG_T;
    for (int q = threadIdx.x; q < SG_HP; q += blockDim.x) {
        const int yy = y0 + q / SG_HS - 2, xx = x0 + q % SG_HS - 2;
        tile[q] = (yy >= 0 && yy < h && xx >= 0 && xx < w) ? grid[(long)yy * w + xx] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    {
        const int tx = threadIdx.x % SG_T, ty = threadIdx.x / SG_T, x = x0 + tx, y = y0 + ty;
        const bool in = x < w && y < h;
        const long pix = (long)y * w + x;
        for (int o = 0; o < SG_C; ++o) dt[o * 256 + threadIdx.x] = in ? da1[pix * SG_C + o] : 0.f;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < SG_NW1; j += blockDim.x) {
        const int o = j / 75, c = (j / 25) % 3, t = j % 25;
        const float* d = dt + o * 256;
        float acc = 0.f;
        for (int q = 0; q < 256; ++q) {
            const float dq = d[q];
            if (dq == 0.f) continue;
            const int qx = q % SG_T, qy = q / SG_T;
            const float4 nb = tile[halo_of(t, qx, qy)];
            if (nb.w == 0.f) continue;
            const float4 ce = tile[(qy + 2) * SG_HS + qx + 2];
            const float diff = c == 0 ? nb.x - ce.x : (c == 1 ? nb.y - ce.y : nb.z - ce.z);
            acc = fmaf(dq, diff, acc);
        }
        if (acc != 0.f) atomicAdd(gw1 + j, acc);
    }
}

// Adam on the float master weights with the gradient sums scaled by inv_n; bc1, bc2 = 1 - b^t.
__global__ void sg_adam_kernel(float* __restrict__ w, float* __restrict__ m, float* __restrict__ s,
                               const float* __restrict__ g, float inv_n, float lr, float b1, float b2, float eps,
                               float bc1, float bc2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= SG_NW) return;
    const float gi = g[i] * inv_n;
    const float mi = fmaf(b1, m[i], (1.f - b1) * gi);
    const float si = fmaf(b2, s[i], (1.f - b2) * gi * gi);
    m[i] = mi;
    s[i] = si;
    w[i] -= lr * (mi / bc1) / (sqrtf(si / bc2) + eps);
}

constexpr size_t SMEM_CONV = sizeof(float) * (SG_C * SG_HPAD + SG_C * SG_TAPS * 16);
constexpr size_t SMEM_GW3 = sizeof(float) * (SG_C * SG_HPAD + 3 * 256);
constexpr size_t SMEM_GW2 = sizeof(float) * (SG_C * SG_HPAD + SG_C * 256);
constexpr size_t SMEM_GW1 = sizeof(float) * (4 * SG_HP + SG_C * 256);

gsicp_status sg_set_smem()
{
    static bool done = false;
    if (done) return GSICP_OK;
    GSICP_CUDA(cudaFuncSetAttribute(sg_dl2_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_CONV));
    GSICP_CUDA(cudaFuncSetAttribute(sg_conv_tc_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)tc_smem<32>()));
    GSICP_CUDA(cudaFuncSetAttribute(sg_conv_tc_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)tc_smem<16>()));
    GSICP_CUDA(cudaFuncSetAttribute(sg_gw3_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_GW3));
    GSICP_CUDA(cudaFuncSetAttribute(sg_gw2_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_GW2));
    GSICP_CUDA(cudaFuncSetAttribute(sg_gw1_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_GW1));
    done = true;
    return GSICP_OK;
}

gsicp_status sg_ensure(gsicp_surrogate_s* sg, int64_t npix)
{
    if (npix <= sg->pix_cap) return GSICP_OK;
    const size_t n = (size_t)npix;
    GSICP_CHECK(sg->grid.ensure(sizeof(float4) * n));
    GSICP_CHECK(sg->h1.ensure(sizeof(__nv_bfloat16) * SG_C * n));
    GSICP_CHECK(sg->h2.ensure(sizeof(__nv_bfloat16) * SG_C * n));
    GSICP_CHECK(sg->v.ensure(sizeof(float) * 3 * n));
    GSICP_CHECK(sg->dv.ensure(sizeof(float) * 3 * n));
    GSICP_CHECK(sg->da2.ensure(sizeof(float) * SG_C * n));
    GSICP_CHECK(sg->da1.ensure(sizeof(float) * SG_C * n));
    sg->pix_cap = npix;
    return GSICP_OK;
}

// Tensor map of a channels-last 32-channel bfloat16 activation (w x h pixels): boxes of 8 channels
// x 12 columns x 20 rows (a tile's halo, one channel group), no swizzle, zero fill outside.
gsicp_status act_tensor_map(CUtensorMap* m, void* base, int w, int h)
{
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        cudaDriverEntryPointQueryResult q;
        void* fn = nullptr;
        GSICP_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q));
        if (q != cudaDriverEntryPointSuccess || !fn) return set_error(GSICP_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
        encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    const cuuint64_t dims[3] = {(cuuint64_t)SG_C, (cuuint64_t)w, (cuuint64_t)h};
    const cuuint64_t strides[2] = {(cuuint64_t)SG_C * 2, (cuuint64_t)SG_C * 2 * (cuuint64_t)w};
    const cuuint32_t box[3] = {8, (cuuint32_t)TC_HW, (cuuint32_t)TC_HH};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, base, dims, strides, box, estr,
                              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_error(GSICP_ERR_CUDA, "cuTensorMapEncodeTiled failed");
    return GSICP_OK;
}

}  // namespace

// Grid + layers 1-3 over the frame's a1 output (pts in a1 order, idx_img the sample -> point map).
gsicp_status surrogate_status(gsicp_surrogate_s* sg)
{
    if (sg && sg->err && *reinterpret_cast<volatile unsigned*>(sg->err)) {
        *sg->err = 0u;
        return set_error(GSICP_ERR_TIMEOUT, "surrogate: a tensor-core wait ran out");
    }
    return GSICP_OK;
}

gsicp_status surrogate_forward(gsicp_surrogate_s* sg, const float* pts, const int* idx_img, int ws, int hs, float eps,
                        float p, float* covs, float* v_out, cudaStream_t s)
{
    const int64_t npix = (int64_t)ws * hs;
    if (npix <= 0) return GSICP_OK;
    GSICP_CHECK(sg_set_smem());
    GSICP_CHECK(sg_ensure(sg, npix));
    const float* wk = sg->wk.as<float>();
    float4* grid = sg->grid.as<float4>();
    if (sg->timing) GSICP_CUDA(cudaEventRecord(sg->ev[0], s));
    sg_grid_kernel<<<(int)((npix + 255) / 256), 256, 0, s>>>(pts, idx_img, (int)npix, grid);
    const dim3 tiles((ws + SG_T - 1) / SG_T, (hs + SG_T - 1) / SG_T);
    sg_l1_kernel<<<tiles, SG_L1_THREADS, 0, s>>>(grid, ws, hs, reinterpret_cast<const float4*>(wk + WK_W1),
                                                 sg->h1.as<__nv_bfloat16>());
    if (sg->timing) GSICP_CUDA(cudaEventRecord(sg->ev[1], s));
    const int ntc = ((ws + TC_TW - 1) / TC_TW) * ((hs + TC_TH - 1) / TC_TH);
    const int gtc = std::max(1, std::min(ntc, 2 * device_sm_count()));
    CUtensorMap m1, m2;
    GSICP_CHECK(act_tensor_map(&m1, sg->h1.ptr, ws, hs));
    GSICP_CHECK(act_tensor_map(&m2, sg->h2.ptr, ws, hs));
    sg_conv_tc_kernel<32><<<gtc, 128, tc_smem<32>(), s>>>(m1, ws, hs, sg->wmma.as<const uint4>(), grid,
                                                          sg->h2.as<__nv_bfloat16>(), nullptr, 0.f, 0.f, nullptr,
                                                          nullptr, sg->err);
    if (sg->timing) GSICP_CUDA(cudaEventRecord(sg->ev[2], s));
    sg_conv_tc_kernel<16><<<gtc, 128, tc_smem<16>(), s>>>(m2, ws, hs, sg->wmma.as<const uint4>() + tc_b_bytes<32>() / 16,
                                                          grid, nullptr, idx_img, eps, p, covs, v_out, sg->err);
    if (sg->timing) GSICP_CUDA(cudaEventRecord(sg->ev[3], s));
    GSICP_CUDA(cudaGetLastError());
    return GSICP_OK;
}

namespace {

// Back-propagation of the loss against covs_knn (a1 order) into sg->g (sums, not means).
gsicp_status sg_backward(gsicp_surrogate_s* sg, const int* idx_img, const float* covs_knn, int ws, int hs,
                         float eps, float p, cudaStream_t s)
{
    const int64_t npix = (int64_t)ws * hs;
    const float* wk = sg->wk.as<float>();
    const float4* grid = sg->grid.as<const float4>();
    double* loss_sum = sg->scal.as<double>();
    unsigned long long* count = reinterpret_cast<unsigned long long*>(loss_sum + 1);
    GSICP_CUDA(cudaMemsetAsync(sg->g.ptr, 0, sizeof(float) * SG_NW, s));
    GSICP_CUDA(cudaMemsetAsync(sg->scal.ptr, 0, 16, s));
    if (npix <= 0) return GSICP_OK;
    const dim3 tiles((ws + SG_T - 1) / SG_T, (hs + SG_T - 1) / SG_T);
    float* g = sg->g.as<float>();
    sg_loss_kernel<<<(int)((npix + 255) / 256), 256, 0, s>>>(sg->v.as<float>(), grid, idx_img, covs_knn, (int)npix,
                                                             eps, p, sg->dv.as<float>(), loss_sum, count);
    sg_gw3_kernel<<<tiles, 256, SMEM_GW3, s>>>(sg->dv.as<float>(), sg->h2.as<__nv_bfloat16>(), ws, hs,
                                               g + SG_NW1 + SG_NW2);
    float* da2 = sg->da2.as<float>();
    float* da1 = sg->da1.as<float>();
    sg_dl3_kernel<<<tiles, 256, 0, s>>>(sg->dv.as<float>(), ws, hs, reinterpret_cast<const float4*>(wk + WK_W3T),
                                        sg->h2.as<__nv_bfloat16>(), da2);
    sg_gw2_kernel<<<tiles, 256, SMEM_GW2, s>>>(da2, sg->h1.as<__nv_bfloat16>(), ws, hs, g + SG_NW1);
    // da1 = [h1 > 0] (layer 2 transposed: W2 with flipped taps, channels swapped) * da2
    sg_dl2_kernel<<<dim3(tiles.x, tiles.y, 2), 256, SMEM_CONV, s>>>(da2, ws, hs, wk + WK_W2T,
                                                                    sg->h1.as<__nv_bfloat16>(), da1);
    sg_gw1_kernel<<<tiles, 256, SMEM_GW1, s>>>(da1, grid, ws, hs, g);
    GSICP_CUDA(cudaGetLastError());
    return GSICP_OK;
}

gsicp_status sg_upload(gsicp_surrogate_s* sg, const float* w_host, cudaStream_t s)
{
    GSICP_CUDA(cudaMemcpyAsync(sg->w.ptr, w_host, sizeof(float) * SG_NW, cudaMemcpyHostToDevice, s));
    GSICP_CUDA(cudaMemsetAsync(sg->m.ptr, 0, sizeof(float) * SG_NW, s));
    GSICP_CUDA(cudaMemsetAsync(sg->s.ptr, 0, sizeof(float) * SG_NW, s));
    sg_layout_kernel<<<(SG_NW + 255) / 256, 256, 0, s>>>(sg->w.as<float>(), sg->wk.as<float>(),
                                                         sg->wmma.as<__nv_bfloat16>());
    GSICP_CUDA(cudaGetLastError());
    sg->steps = 0;
    return GSICP_OK;
}

}  // namespace
}  // namespace gsicp

// ---------------------------------------------------------------------------------------------
// C ABI

using namespace gsicp;

extern "C" {

gsicp_status gsicp_surrogate_create(const float* weights, gsicp_surrogate* out)
{
    if (!weights || !out) return GSICP_ERR_INVALID_ARG;
    *out = nullptr;
    gsicp_surrogate_s* sg = new (std::nothrow) gsicp_surrogate_s;
    if (!sg) return GSICP_ERR_OOM;
    cudaGetDevice(&sg->device);
    gsicp_status st = GSICP_OK;
    if ((st = sg->w.ensure(sizeof(float) * SG_NW)) != GSICP_OK || (st = sg->m.ensure(sizeof(float) * SG_NW)) != GSICP_OK ||
        (st = sg->s.ensure(sizeof(float) * SG_NW)) != GSICP_OK || (st = sg->g.ensure(sizeof(float) * SG_NW)) != GSICP_OK ||
        (st = sg->wk.ensure(sizeof(float) * WK_TOTAL)) != GSICP_OK || (st = sg->scal.ensure(16)) != GSICP_OK ||
        (st = sg->wmma.ensure(sizeof(__nv_bfloat16) * (SG_NW2 + SG_TAPS * SG_C * 16))) != GSICP_OK ||
        (st = (cudaMemset(sg->wmma.ptr, 0, sizeof(__nv_bfloat16) * (SG_NW2 + SG_TAPS * SG_C * 16)) == cudaSuccess
                   ? GSICP_OK : GSICP_ERR_CUDA)) != GSICP_OK ||
        (st = (cudaMallocHost((void**)&sg->err, sizeof(unsigned)) == cudaSuccess ? GSICP_OK : GSICP_ERR_OOM)) != GSICP_OK ||
        (st = sg_upload(sg, weights, nullptr)) != GSICP_OK) {
        gsicp_surrogate_destroy(sg);
        return st;
    }
    *sg->err = 0u;
    cudaError_t e = cudaStreamSynchronize(nullptr);
    if (e != cudaSuccess) {
        gsicp_surrogate_destroy(sg);
        return cuda_status(e, "gsicp_surrogate_create");
    }
    *out = sg;
    return GSICP_OK;
}

void gsicp_surrogate_destroy(gsicp_surrogate sg)
{
    if (!sg) return;
    for (DevBuf* b : {&sg->w, &sg->m, &sg->s, &sg->g, &sg->wk, &sg->wmma, &sg->grid, &sg->h1, &sg->h2, &sg->v, &sg->dv,
                      &sg->da2, &sg->da1, &sg->scal})
        b->release();
    if (sg->err) cudaFreeHost(sg->err);
    for (cudaEvent_t& e : sg->ev)
        if (e) cudaEventDestroy(e);
    delete sg;
}

gsicp_status gsicp_surrogate_set_timing(gsicp_surrogate sg, int enable)
{
    if (!sg) return GSICP_ERR_INVALID_ARG;
    if (enable && !sg->ev[0])
        for (cudaEvent_t& e : sg->ev) GSICP_CUDA(cudaEventCreate(&e));
    sg->timing = enable != 0;
    return GSICP_OK;
}

gsicp_status gsicp_surrogate_layer_times(gsicp_surrogate sg, double out[3])
{
    if (!sg || !out || !sg->ev[0]) return GSICP_ERR_INVALID_ARG;
    float ms[3];
    for (int i = 0; i < 3; ++i) GSICP_CUDA(cudaEventElapsedTime(&ms[i], sg->ev[i], sg->ev[i + 1]));
    for (int i = 0; i < 3; ++i) out[i] = ms[i];
    return GSICP_OK;
}

gsicp_status gsicp_surrogate_get_weights(gsicp_surrogate sg, float* weights)
{
    if (!sg || !weights) return GSICP_ERR_INVALID_ARG;
    GSICP_CUDA(cudaMemcpy(weights, sg->w.ptr, sizeof(float) * SG_NW, cudaMemcpyDeviceToHost));
    return GSICP_OK;
}

gsicp_status gsicp_surrogate_set_weights(gsicp_surrogate sg, const float* weights)
{
    if (!sg || !weights) return GSICP_ERR_INVALID_ARG;
    GSICP_CHECK(sg_upload(sg, weights, nullptr));
    GSICP_CUDA(cudaStreamSynchronize(nullptr));
    return GSICP_OK;
}

static bool valid_sg_frame(gsicp_ctx ctx, gsicp_surrogate sg, const void* depth, int W, int H, const float intr[4],
                           int stride, const gsicp_cov_params* params)
{
    return ctx && sg && depth && intr && W > 0 && H > 0 && stride > 0 && params && params->eps > 0.f &&
           params->eps < 1.f && params->p >= 0.f && intr[0] != 0.f && intr[1] != 0.f &&
           (int64_t)((W + stride - 1) / stride) * ((H + stride - 1) / stride) <= (1 << 30);
}

gsicp_status gsicp_surrogate_covariances(gsicp_ctx ctx, gsicp_surrogate sg, const float* depth_dev, int W, int H,
                                         const float intr[4], int stride, float z_min, float z_max,
                                         const gsicp_cov_params* params, float* pts_dev, float* z_dev,
                                         float* covs_dev, float* v_dev, int64_t cap, int64_t* n_out, void* stream)
{
    if (!valid_sg_frame(ctx, sg, depth_dev, W, H, intr, stride, params) || !pts_dev || !covs_dev || !n_out || cap < 0 ||
        cap > INT32_MAX)
        return GSICP_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int ws = (W + stride - 1) / stride, hs = (H + stride - 1) / stride;
    const int fcap = ws * hs;
    GSICP_CHECK(ctx->frame_pts.ensure(sizeof(float) * 3 * (size_t)fcap));
    GSICP_CHECK(ctx->frame_z.ensure(sizeof(float) * (size_t)fcap));
    GSICP_CHECK(ctx->frame_covs.ensure(sizeof(float) * 6 * (size_t)fcap));
    GSICP_CHECK(ctx->frame_idx.ensure(sizeof(int) * (size_t)fcap));
    GSICP_CHECK(launch_depth_to_points(depth_dev, W, H, intr, stride, z_min, z_max, ctx->frame_pts.as<float>(),
                                       ctx->frame_z.as<float>(), fcap, ctx->n_dev.as<int>(), ctx->total_dev.as<int>(),
                                       ctx->a1_counts, ctx->a1_sums, s, ctx->frame_idx.as<int>()));
    GSICP_CHECK(surrogate_forward(sg, ctx->frame_pts.as<float>(), ctx->frame_idx.as<int>(), ws, hs, params->eps,
                                  params->p, ctx->frame_covs.as<float>(), v_dev, s));
    int* h = (int*)ctx->host_pinned;
    GSICP_CUDA(cudaMemcpyAsync(h, ctx->n_dev.ptr, sizeof(int), cudaMemcpyDeviceToHost, s));
    GSICP_CUDA(cudaStreamSynchronize(s));
    GSICP_CHECK(surrogate_status(sg));
    const int64_t n = h[0], m = std::min<int64_t>(n, cap);
    if (m > 0) {
        GSICP_CUDA(cudaMemcpyAsync(pts_dev, ctx->frame_pts.ptr, sizeof(float) * 3 * m, cudaMemcpyDeviceToDevice, s));
        GSICP_CUDA(cudaMemcpyAsync(covs_dev, ctx->frame_covs.ptr, sizeof(float) * 6 * m, cudaMemcpyDeviceToDevice, s));
        if (z_dev) GSICP_CUDA(cudaMemcpyAsync(z_dev, ctx->frame_z.ptr, sizeof(float) * m, cudaMemcpyDeviceToDevice, s));
    }
    *n_out = m;
    return n > cap ? GSICP_ERR_CAPACITY : GSICP_OK;
}

gsicp_status gsicp_surrogate_train_step(gsicp_ctx ctx, gsicp_surrogate sg, const float* depth_dev, int W, int H,
                                        const float intr[4], int stride, float z_min, float z_max,
                                        const gsicp_cov_params* params, const float* target_covs_dev, float lr,
                                        int apply, double* loss_out, int64_t* count_out, float* grad_out,
                                        void* stream)
{
    if (!valid_sg_frame(ctx, sg, depth_dev, W, H, intr, stride, params) || !(lr >= 0.f) || (apply != 0 && apply != 1))
        return GSICP_ERR_INVALID_ARG;
    if (!target_covs_dev && params->reg_mode != GSICP_REG_PLANE) return GSICP_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int ws = (W + stride - 1) / stride, hs = (H + stride - 1) / stride;
    const int fcap = ws * hs;
    if (target_covs_dev) {  // a1 only; the caller's targets are in a1 order
        GSICP_CHECK(ctx->frame_pts.ensure(sizeof(float) * 3 * (size_t)fcap));
        GSICP_CHECK(ctx->frame_z.ensure(sizeof(float) * (size_t)fcap));
        GSICP_CHECK(ctx->frame_idx.ensure(sizeof(int) * (size_t)fcap));
        GSICP_CHECK(launch_depth_to_points(depth_dev, W, H, intr, stride, z_min, z_max, ctx->frame_pts.as<float>(),
                                           ctx->frame_z.as<float>(), fcap, ctx->n_dev.as<int>(),
                                           ctx->total_dev.as<int>(), ctx->a1_counts, ctx->a1_sums, s,
                                           ctx->frame_idx.as<int>()));
    } else {  // the plain k-NN covariances of the frame are the targets
        GSICP_CHECK(frame_covariances(ctx, depth_dev, W, H, intr, stride, z_min, z_max, params, fcap, s, nullptr));
    }
    const float* targets = target_covs_dev ? target_covs_dev : ctx->frame_covs.as<float>();
    GSICP_CHECK(sg_ensure(sg, (int64_t)fcap));  // sg->v must exist before its address is taken
    GSICP_CHECK(surrogate_forward(sg, ctx->frame_pts.as<float>(), ctx->frame_idx.as<int>(), ws, hs, params->eps,
                                  params->p, nullptr, sg->v.as<float>(), s));
    GSICP_CHECK(sg_backward(sg, ctx->frame_idx.as<int>(), targets, ws, hs, params->eps, params->p, s));
    double* hs_ = reinterpret_cast<double*>(ctx->host_pinned);
    GSICP_CUDA(cudaMemcpyAsync(hs_, sg->scal.ptr, 16, cudaMemcpyDeviceToHost, s));
    GSICP_CUDA(cudaStreamSynchronize(s));
    GSICP_CHECK(surrogate_status(sg));
    const double loss_sum = hs_[0];
    const unsigned long long cnt = reinterpret_cast<unsigned long long*>(hs_)[1];
    if (loss_out) *loss_out = cnt ? loss_sum / (double)cnt : 0.0;
    if (count_out) *count_out = (int64_t)cnt;
    if (grad_out) {
        GSICP_CUDA(cudaMemcpy(grad_out, sg->g.ptr, sizeof(float) * SG_NW, cudaMemcpyDeviceToHost));
        if (cnt)
            for (int i = 0; i < SG_NW; ++i) grad_out[i] = (float)((double)grad_out[i] / (double)cnt);
    }
    if (apply && cnt) {
        const int t = sg->steps + 1;
        const double b1 = 0.9, b2 = 0.999;
        sg_adam_kernel<<<(SG_NW + 255) / 256, 256, 0, s>>>(sg->w.as<float>(), sg->m.as<float>(), sg->s.as<float>(),
                                                            sg->g.as<float>(), (float)(1.0 / (double)cnt), lr,
                                                            (float)b1, (float)b2, 1e-8f, (float)(1.0 - pow(b1, t)),
                                                            (float)(1.0 - pow(b2, t)));
        sg_layout_kernel<<<(SG_NW + 255) / 256, 256, 0, s>>>(sg->w.as<float>(), sg->wk.as<float>(),
                                                             sg->wmma.as<__nv_bfloat16>());
        GSICP_CUDA(cudaGetLastError());
        sg->steps = t;
    }
    return GSICP_OK;
}

}  // extern "C"
