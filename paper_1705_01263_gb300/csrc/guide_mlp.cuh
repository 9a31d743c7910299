// Fused forward pass of the guiding network on the tensor cores. The
// training forward (mlp_tiles<true>) works as follows; the inference kernel
// (mlp_infer_tiles, below) keeps six tiles in flight instead of one. One
// persistent CTA of 512 threads per SM keeps all five BF16 weight matrices
// (58 KB, copied in by one bulk copy of a prepared image) in shared memory and walks tiles of 128 rows, four threads per row (part p =
// warp / 4 of row 32 (warp % 4) + lane), so that each SM sub-partition has
// four warps to switch between. The CTA gathers the 7 features of four
// tiles at once (one row per thread, so that the dependent loads behind a
// feature overlap across 512 rows), then runs the tiles. For a tile, every
// thread builds a quarter of the
// row's one-blob encoding (56 of 224 BF16 values); one elected thread issues
// the tcgen05.mma of layer 1 (128 x 64 x 224, FP32 accumulator in tensor
// memory); each warp reads 16 accumulator columns of its 32 rows back with
// tcgen05.ld (a warp reaches the tensor-memory lanes 32 (warp % 4) + 0..31),
// applies ReLU, rounds to BF16 and writes them into the next layer's A
// operand in shared memory; layers 2-4 (64 -> 64) and 5 (64 -> 48, 40 used)
// follow the same way, and the outputs go straight from tensor memory to
// global memory. Nothing but the features and the outputs touches global
// memory, and the whole network is one launch.
//
// Operands use the canonical no-swizzle K-major layout of umma.cuh. Every
// wait on the tensor core is bounded; on a timeout the kernel sets *err and
// stops. Results equal the layer-by-layer GEMM path (same BF16 inputs, same
// K order of the accumulation).
#pragma once

#include <cuda_bf16.h>

#include <type_traits>

#include "guide.cuh"
#include "umma.cuh"

namespace rtg {

struct MlpWeights {
    const __nv_bfloat16 *W[5];   // [out_pad][in] row-major BF16 (layer 5 padded to 48 rows)
    // the five matrices as the kernels hold them in shared memory (offsets
    // kMlpW1 .. kMlpW5, canonical K-major layout): kMlpX bytes, 16-byte aligned
    const void *image;
};

// Training forward pass: besides the network outputs, the kernel keeps what
// the backward pass needs (rows n..n_pad-1 zero): the one-blob input
// transposed, XT [224][n_pad]; the hidden activations H_l [n_pad][64] and
// their transposes HT_l [64][n_pad]; and, from the outputs, the gradient of
// the loss sum_r weight_r * inv_n * -log q(wi_r) with respect to them,
// dY [n_pad][48] and dYT [48][n_pad] (BF16), the loss summed into *loss.
struct MlpTrain {
    const float *wi, *weight;
    float inv_n;
    uint32_t n_pad;
    __nv_bfloat16 *XT, *H[4], *HT[4], *dY, *dYT;
    float *loss;
};

constexpr uint32_t kMlpTile = 128;      // rows per tile (the MMA's M)
constexpr uint32_t kMlpThreads = 512;   // four threads per row
constexpr uint32_t kMlpW1 = 0;                                            // 64 x 224
constexpr uint32_t kMlpW2 = kMlpW1 + kGuideHid * kGuideIn * 2;           // 64 x 64
constexpr uint32_t kMlpW3 = kMlpW2 + kGuideHid * kGuideHid * 2;
constexpr uint32_t kMlpW4 = kMlpW3 + kGuideHid * kGuideHid * 2;
constexpr uint32_t kMlpW5 = kMlpW4 + kGuideHid * kGuideHid * 2;          // 48 x 64
constexpr uint32_t kMlpX = kMlpW5 + kGuideOutPad * kGuideHid * 2;        // 128 x 224
constexpr uint32_t kMlpH = kMlpX + kMlpTile * kGuideIn * 2;              // 128 x 64
constexpr uint32_t kMlpGroup = 4;                                        // tiles whose features are gathered together
constexpr uint32_t kMlpF = kMlpH + kMlpTile * kGuideHid * 2;             // 512 x 8 FP32 features
constexpr uint32_t kMlpBar = kMlpF + kMlpGroup * kMlpTile * 8 * 4;       // mbarrier, TMEM address
constexpr uint32_t kMlpSmem = kMlpBar + 64;                              // 149,568 bytes
constexpr uint32_t kMlpOut = kMlpSmem;                                   // training: 128 x 48 FP32 outputs
constexpr uint32_t kMlpSmemTrain = kMlpOut + kMlpTile * kGuideOutPad * 4; // 174,144 bytes

// Byte offset in the shared-memory weight image of element (o, k) of layer
// l (row o of the [out_pad][in] matrix).
__host__ __device__ constexpr uint32_t mlp_image_base(int l) {
    return l == 0 ? kMlpW1 : (l == 1 ? kMlpW2 : (l == 2 ? kMlpW3 : (l == 3 ? kMlpW4 : kMlpW5)));
}

// The weight image into shared memory at offset 0 with one bulk copy (one
// thread issues it; every thread then waits on `bar`, bounded). Returns
// false, in every thread of the block, on a timeout. The barrier completes
// its phase 0 here.
__device__ __forceinline__ bool mlp_load_image(unsigned char *smem, const void *image, uint64_t *bar) {
    if (threadIdx.x == 0) {
        umma::mbar_init(bar, 1);
        const uint32_t b = umma::smem_addr(bar);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(kMlpX) : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                umma::smem_addr(smem)),
            "l"(image), "r"(kMlpX), "r"(b)
            : "memory");
    }
    __syncthreads();
    return __syncthreads_and(umma::mbar_wait(bar, 0u) ? 1 : 0) != 0;
}

// Issue one layer: D[128 x n] = A[128 x k] * B[n x k]^T, K in steps of 16.
__device__ __forceinline__ void mlp_issue(uint32_t taddr, uint32_t a0, uint32_t b0, uint32_t k, uint32_t n,
                                          uint64_t *bar) {
    const uint32_t idesc = umma::make_idesc_bf16(kMlpTile, n);
    const uint32_t sbo = k / 8 * 128;
    umma::fence_after_sync();
    for (uint32_t kk = 0; kk < k / 16; ++kk) {
        const uint64_t ad = umma::make_desc(a0 + kk * 256, 128, sbo);
        const uint64_t bd = umma::make_desc(b0 + kk * 256, 128, sbo);
        umma::mma_bf16(taddr, ad, bd, idesc, kk > 0 ? 1u : 0u);
    }
    umma::mma_commit(bar);
}

// Features: `void operator()(uint32_t row, float f[7]) const` (device),
// `uint32_t count() const` (rows to infer, read once per launch) and, for
// the inference kernel, `uint32_t out_row(uint32_t row) const` (the output
// row of that input row) and `static constexpr bool kContiguous` (out_row is
// the identity).
template <bool kTrain, class Features>
__device__ void mlp_tiles(const MlpWeights &w, const Features &feat, float *raw, uint32_t *err, const MlpTrain &tr) {
    extern __shared__ __align__(1024) unsigned char smem[];
    uint64_t *bar = (uint64_t *)(smem + kMlpBar);
    uint32_t *s_taddr = (uint32_t *)(smem + kMlpBar + 16);
    float *s_feat = (float *)(smem + kMlpF);
    const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31u;
    const uint32_t quarter = warp & 3u, part = warp >> 2;      // rows 32 quarter + lane, part 0..3
    const uint32_t r = 32u * quarter + lane;                    // this thread's row in the tile
    const uint32_t n = feat.count();
    const uint32_t tiles = (n + kMlpTile - 1) / kMlpTile;
    const uint32_t groups = (tiles + kMlpGroup - 1) / kMlpGroup;
    if (blockIdx.x >= groups) return;
    const bool image_ok = mlp_load_image(smem, w.image, (uint64_t *)(smem + kMlpBar + 32));
    if (warp == 0) umma::tmem_alloc(s_taddr, 64);
    if (tid == 0) umma::mbar_init(bar, 1);
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    const uint32_t taddr = *s_taddr;
    const uint32_t lane_addr = taddr + ((32u * quarter) << 16);
    const uint32_t sbase = umma::smem_addr(smem);
    uint32_t phase = 0;
    bool ok = image_ok;
    // Bounded wait for the layer just issued; the outcome is made uniform
    // over the block, so that all threads leave (or stay) together.
    auto wait_layer = [&]() -> bool {
        const bool done = umma::mbar_wait(bar, phase);
        phase ^= 1u;
        return __syncthreads_and(done ? 1 : 0) != 0;
    };
    for (uint32_t gi = blockIdx.x; gi < groups && ok; gi += gridDim.x) {
      {
        // features of the group's 512 rows, one per thread
        const uint32_t grow = gi * kMlpGroup * kMlpTile + tid;
        float f[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (grow < n) feat(grow, f);
        __syncthreads();   // the previous group's last tile is done with s_feat
#pragma unroll
        for (int k = 0; k < 7; ++k) s_feat[8 * tid + k] = f[k];
        __syncthreads();
      }
      for (uint32_t sub = 0; sub < kMlpGroup; ++sub) {
        const uint32_t t = gi * kMlpGroup + sub;
        if (t >= tiles) break;
        const uint32_t row = t * kMlpTile + r;
        const float *frow = s_feat + 8 * (sub * kMlpTile + r);
        // one-blob encoding: this part writes columns 56 part .. 56 part + 55
        // (feature c / 32, bin c % 32), 8 at a time
#pragma unroll 1
        for (uint32_t j = 0; j < 7; ++j) {
            const uint32_t col = 56u * part + 8u * j;
            const float fv = frow[col / kGuideBins];
            __align__(16) __nv_bfloat16 b[8];
            float g8[8];
            oneblob_chunk(fv, (int)(col % kGuideBins), g8);
#pragma unroll
            for (int e = 0; e < 8; ++e) b[e] = __float2bfloat16(g8[e]);
            *(uint4 *)(smem + kMlpX + umma::kmajor_offset(r, col, kGuideIn)) = *(const uint4 *)b;
            if (kTrain) {
                const __nv_bfloat16 z = __float2bfloat16(0.f);
#pragma unroll
                for (int e = 0; e < 8; ++e) tr.XT[(size_t)(col + e) * tr.n_pad + row] = row < n ? b[e] : z;
            }
        }
        umma::fence_proxy_async();
        umma::fence_before_sync();
        __syncthreads();
        // layers 1..4: MMA, then ReLU -> BF16 -> the next layer's A operand
#pragma unroll 1
        for (int l = 0; l < 4; ++l) {
            if (tid == 0) {
                const uint32_t a0 = sbase + (l == 0 ? kMlpX : kMlpH);
                const uint32_t b0 = sbase + (l == 0 ? kMlpW1 : (l == 1 ? kMlpW2 : (l == 2 ? kMlpW3 : kMlpW4)));
                mlp_issue(taddr, a0, b0, l == 0 ? kGuideIn : kGuideHid, kGuideHid, bar);
            }
            if (!(ok = wait_layer())) break;
            umma::fence_after_sync();
            {
                const uint32_t c0 = 16u * part;   // this warp's 16 columns
                float v[16];
                umma::tmem_ld16(lane_addr + c0, v);
                __align__(16) __nv_bfloat16 b[16];
#pragma unroll
                for (int e = 0; e < 16; ++e) b[e] = __float2bfloat16(row < n || !kTrain ? fmaxf(v[e], 0.f) : 0.f);
                *(uint4 *)(smem + kMlpH + umma::kmajor_offset(r, c0, kGuideHid)) = *(const uint4 *)b;
                *(uint4 *)(smem + kMlpH + umma::kmajor_offset(r, c0 + 8, kGuideHid)) = *(const uint4 *)(b + 8);
                if (kTrain) {
                    uint4 *hr = (uint4 *)(tr.H[l] + (size_t)row * kGuideHid + c0);
                    hr[0] = *(const uint4 *)b;
                    hr[1] = *(const uint4 *)(b + 8);
#pragma unroll
                    for (int e = 0; e < 16; ++e) tr.HT[l][(size_t)(c0 + e) * tr.n_pad + row] = b[e];
                }
            }
            umma::fence_proxy_async();
            umma::fence_before_sync();
            __syncthreads();
        }
        if (!ok) break;
        // layer 5: 48 outputs (40 used); parts 0..2 store 16 columns each
        if (tid == 0) mlp_issue(taddr, sbase + kMlpH, sbase + kMlpW5, kGuideHid, kGuideOutPad, bar);
        if (!(ok = wait_layer())) break;
        umma::fence_after_sync();
        if (part < 3) {
            const uint32_t c0 = 16u * part;
            float v[16];
            umma::tmem_ld16(lane_addr + c0, v);
            if (kTrain) {
                float *so = (float *)(smem + kMlpOut) + r * kGuideOutPad + c0;
#pragma unroll
                for (int e = 0; e < 16; ++e) so[e] = v[e];
            } else if (row < n) {
                float4 *dst = (float4 *)(raw + (size_t)row * kGuideOutPad + c0);
#pragma unroll
                for (int e = 0; e < 4; ++e) dst[e] = make_float4(v[4 * e], v[4 * e + 1], v[4 * e + 2], v[4 * e + 3]);
            }
        }
        if (kTrain) {
            // loss and its gradient per row, from the row's 40 outputs
            __syncthreads();
            if (part == 0) {
                float g[kGuideOutPad];
#pragma unroll
                for (int k = 0; k < kGuideOutPad; ++k) g[k] = 0.f;
                float lw = 0.f;
                if (row < n) {
                    const float *so = (const float *)(smem + kMlpOut) + r * kGuideOutPad;
                    const float w3[3] = {tr.wi[3 * (size_t)row], tr.wi[3 * (size_t)row + 1], tr.wi[3 * (size_t)row + 2]};
                    lw = mixture_loss_grad(so, w3, tr.weight[row] * tr.inv_n, g);
                }
                __align__(16) __nv_bfloat16 b[kGuideOutPad];
#pragma unroll
                for (int k = 0; k < kGuideOutPad; ++k) b[k] = __float2bfloat16(g[k]);
                uint4 *dr = (uint4 *)(tr.dY + (size_t)row * kGuideOutPad);
#pragma unroll
                for (int k = 0; k < kGuideOutPad / 8; ++k) dr[k] = ((const uint4 *)b)[k];
#pragma unroll
                for (int k = 0; k < kGuideOutPad; ++k) tr.dYT[(size_t)k * tr.n_pad + row] = b[k];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) lw += __shfl_xor_sync(0xFFFFFFFFu, lw, o);
                if (lane == 0) atomicAdd(tr.loss, lw);
            }
        }
        // the accumulator, X and H are reused by the next tile
        umma::fence_before_sync();
        __syncthreads();
      }
      if (!ok) break;
    }
    if (!ok) {
        // the layer in flight may still complete: wait for it once more
        // (bounded) before the tensor memory is released
        if (tid == 0) {
            umma::mbar_wait(bar, phase ^ 1u);
            atomicExch(err, 1u);
        }
    }
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    if (warp == 0) umma::tmem_dealloc(taddr, 64);
}

// ---------------------------------------------------------------- inference
// kMiGroups tiles in flight: the threads form independent groups of 128
// (four warps), one thread per row (warp w of a group reaches tensor-memory
// lanes 32 (w % 4) + 0..31, its rows), each group with its own 64
// tensor-memory columns, mbarrier and named barrier (ids 1..kMiGroups),
// sharing the weights. A group loads the next tile's features before it
// works on the current one, so that their latency overlaps the products.
// A group's shared buffer is 128 x 80 BF16: layer 1 runs in three K chunks,
// the one-blob columns 0..79, 80..159 and 160..223 encoded in turn into the
// same buffer (each after the previous product has completed, the products
// accumulating in tensor memory); the hidden activations (128 x 64) and at
// the end the tile's output rows then overlay it. Six tiles are in flight per
// SM (the weights and six buffers fill 182 KB of shared memory and the six
// accumulators 384 tensor-memory columns): each product takes ~1,300 cycles
// from issue to the completion seen by the group, most of it latency, so the
// throughput comes from how many groups wait at once. While one group waits
// on its tensor-core product the others encode, read back or store.
constexpr uint32_t kMiChunkK = 80;                                         // layer-1 K per product
static_assert((kGuideIn + kMiChunkK - 1) / kMiChunkK == 3, "layer 1 runs as three chunk products");
constexpr uint32_t kMiBuf = kMlpTile * kMiChunkK * 2;                      // 20,480 bytes
constexpr uint32_t kMiGroup0 = kMlpX;                                      // after the weights (59,392)
constexpr uint32_t kMiGroups = 6;
constexpr uint32_t kMiOutRow = kGuideOut * 4;                              // an output row, bytes (FP32)
static_assert(kMlpTile * kMiOutRow <= kMiBuf, "output staging fits the group buffer");
constexpr uint32_t kMiThreads = 128 * kMiGroups;
constexpr uint32_t kMiTmemCols = 64 * kMiGroups <= 256 ? 256 : 512;       // a power of two
// weight-image mbarrier, one mbarrier per group, TMEM address
constexpr uint32_t kMiBar = kMiGroup0 + kMiGroups * kMiBuf;
constexpr uint32_t kMiBarBytes = 16 + 8 * kMiGroups + 16;
constexpr uint32_t kMlpInferSmem = kMiBar + kMiBarBytes;                   // 182,352 bytes
static_assert(kMlpInferSmem <= 227 * 1024, "inference kernel shared memory");

__device__ __forceinline__ void group_sync(uint32_t id) {
    asm volatile("bar.sync %0, 128;" ::"r"(id) : "memory");
}
// Barrier of the group that also returns whether pred held in all its threads.
__device__ __forceinline__ bool group_all(uint32_t id, bool pred) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\t"
        "bar.red.and.pred q, %2, 128, p;\n\tselp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"(pred ? 1u : 0u), "r"(id)
        : "memory");
    return r != 0;
}

// Two floats to a packed BF16 pair (round to nearest even), the first in the
// low half; with kRelu, negative values become zero (one instruction).
template <bool kRelu>
__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
    uint32_t d;
    if (kRelu) asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    else asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
    return d;
}

// Width of layer-1 K chunk c (80, 80, 64).
__host__ __device__ constexpr uint32_t mlp_chunk_k(uint32_t c) {
    return (c + 1) * kMiChunkK <= (uint32_t)kGuideIn ? kMiChunkK : (uint32_t)kGuideIn - c * kMiChunkK;
}

// Layer-1 product over K chunk c: D (+)= A[128 x kc] * W1[:, 80 c .. 80 c + kc - 1]^T,
// A in the chunk buffer (rows of kMiChunkK elements).
__device__ __forceinline__ void mlp_issue_chunk(uint32_t taddr, uint32_t a0, uint32_t w1, uint32_t c, uint64_t *bar) {
    const uint32_t idesc = umma::make_idesc_bf16(kMlpTile, kGuideHid);
    const uint32_t sbo_a = kMiChunkK / 8 * 128, sbo_b = kGuideIn / 8 * 128;
    const uint32_t b0 = w1 + c * (kMiChunkK / 8) * 128;
    const uint32_t kc = mlp_chunk_k(c);
    umma::fence_after_sync();
    for (uint32_t kk = 0; kk < kc / 16; ++kk) {
        const uint64_t ad = umma::make_desc(a0 + kk * 256, 128, sbo_a);
        const uint64_t bd = umma::make_desc(b0 + kk * 256, 128, sbo_b);
        umma::mma_bf16(taddr, ad, bd, idesc, (c > 0 || kk > 0) ? 1u : 0u);
    }
    umma::mma_commit(bar);
}

// Out: float (the API's n x 40 rows) or __nv_bfloat16 (the guided render's
// rows, 80 bytes each).
template <class Out, class Features>
__device__ void mlp_infer_tiles(const MlpWeights &w, const Features &feat, Out *out, uint32_t *err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    const uint32_t tid = threadIdx.x, warp = tid >> 5, lane = tid & 31u;
    const uint32_t g = warp >> 2, quarter = warp & 3u, gtid = tid & 127u;
    const uint32_t r = 32u * quarter + lane;                     // this thread's row in the tile
    const uint32_t bar_id = 1u + g;
    uint64_t *bar = (uint64_t *)(smem + kMiBar + 16) + g;
    uint32_t *s_taddr = (uint32_t *)(smem + kMiBar + 16 + 8 * kMiGroups);
    unsigned char *buf = smem + kMiGroup0 + g * kMiBuf;
    const uint32_t n = feat.count();
    const uint32_t tiles = (n + kMlpTile - 1) / kMlpTile;
    if (kMiGroups * blockIdx.x >= tiles) return;
    // the first tile's features load while the weights arrive
    float f[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    {
        const uint32_t row0 = (kMiGroups * blockIdx.x + g) * kMlpTile + r;
        if (row0 < n) feat(row0, f);
    }
    const bool image_ok = mlp_load_image(smem, w.image, (uint64_t *)(smem + kMiBar));
    if (warp == 0) umma::tmem_alloc(s_taddr, kMiTmemCols);
    if (tid < kMiGroups) umma::mbar_init((uint64_t *)(smem + kMiBar + 16) + tid, 1);
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    const uint32_t taddr = *s_taddr + 64u * g;                   // this group's 64 columns
    const uint32_t lane_addr = taddr + ((32u * quarter) << 16);
    const uint32_t sbase = umma::smem_addr(smem), bbase = umma::smem_addr(buf);
    uint32_t phase = 0;
    bool ok = image_ok;
    auto wait_layer = [&]() -> bool {
        const bool done = umma::mbar_wait(bar, phase);
        phase ^= 1u;
        return group_all(bar_id, done);
    };
    // this row's 16-byte piece j of a layer-1 chunk sits at row_chunk + 128 j
    unsigned char *const row_chunk = buf + umma::kmajor_offset(r, 0u, kMiChunkK);
    unsigned char *const row_hid = buf + umma::kmajor_offset(r, 0u, kGuideHid);
    // one-blob columns [80 c, 80 c + kc) of this row into the buffer; the
    // 8-column pieces are unrolled so that each one's feature and bins are
    // constants
    auto encode_chunk = [&](const float *f, auto chunk) {
        constexpr uint32_t c0 = decltype(chunk)::value * kMiChunkK;
        constexpr uint32_t kc = mlp_chunk_k(decltype(chunk)::value);
#pragma unroll
        for (uint32_t j = 0; j < kc / 8; ++j) {
            const uint32_t col = c0 + 8u * j;
            float g8[8];
            oneblob_chunk(f[col / kGuideBins], (int)(col % kGuideBins), g8);
            *(uint4 *)(row_chunk + 128u * j) =
                make_uint4(pack_bf16x2<false>(g8[0], g8[1]), pack_bf16x2<false>(g8[2], g8[3]),
                           pack_bf16x2<false>(g8[4], g8[5]), pack_bf16x2<false>(g8[6], g8[7]));
        }
        umma::fence_proxy_async();
        umma::fence_before_sync();
        group_sync(bar_id);
    };
    const uint32_t stride = kMiGroups * gridDim.x;
    for (uint32_t t = kMiGroups * blockIdx.x + g; t < tiles && ok; t += stride) {
        const uint32_t row = t * kMlpTile + r;
        float fn[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};   // the next tile's
        {
            const uint32_t nrow = (t + stride) * kMlpTile + r;
            if (t + stride < tiles && nrow < n) feat(nrow, fn);
        }
        if (t != kMiGroups * blockIdx.x + g) {
            // the previous tile's output copies have read the buffer
            umma::bulk_wait_read();
            group_sync(bar_id);
        }
        encode_chunk(f, std::integral_constant<uint32_t, 0>{});
        if (gtid == 0) mlp_issue_chunk(taddr, bbase, sbase + kMlpW1, 0u, bar);
        if (!(ok = wait_layer())) break;
        encode_chunk(f, std::integral_constant<uint32_t, 1>{});
        if (gtid == 0) mlp_issue_chunk(taddr, bbase, sbase + kMlpW1, 1u, bar);
        if (!(ok = wait_layer())) break;
        encode_chunk(f, std::integral_constant<uint32_t, 2>{});
        if (gtid == 0) mlp_issue_chunk(taddr, bbase, sbase + kMlpW1, 2u, bar);
        if (!(ok = wait_layer())) break;
        // layers 2..5: read back, ReLU -> BF16 -> the activation buffer
        // (overlaying the one-blob buffer), next product
#pragma unroll 1
        for (int l = 1; l < 5; ++l) {
            umma::fence_after_sync();
            // 32 columns per wait: two 16-column loads in flight
#pragma unroll
            for (uint32_t c0 = 0; c0 < (uint32_t)kGuideHid; c0 += 32) {
                uint32_t a[16], b[16];
                umma::tmem_ld16_async(lane_addr + c0, a);
                umma::tmem_ld16_async(lane_addr + c0 + 16, b);
                umma::tmem_wait_ld32(a, b);
                const float *v = (const float *)a, *w = (const float *)b;
                *(uint4 *)(row_hid + 16u * c0) =
                    make_uint4(pack_bf16x2<true>(v[0], v[1]), pack_bf16x2<true>(v[2], v[3]),
                               pack_bf16x2<true>(v[4], v[5]), pack_bf16x2<true>(v[6], v[7]));
                *(uint4 *)(row_hid + 16u * c0 + 128u) =
                    make_uint4(pack_bf16x2<true>(v[8], v[9]), pack_bf16x2<true>(v[10], v[11]),
                               pack_bf16x2<true>(v[12], v[13]), pack_bf16x2<true>(v[14], v[15]));
                *(uint4 *)(row_hid + 16u * c0 + 256u) =
                    make_uint4(pack_bf16x2<true>(w[0], w[1]), pack_bf16x2<true>(w[2], w[3]),
                               pack_bf16x2<true>(w[4], w[5]), pack_bf16x2<true>(w[6], w[7]));
                *(uint4 *)(row_hid + 16u * c0 + 384u) =
                    make_uint4(pack_bf16x2<true>(w[8], w[9]), pack_bf16x2<true>(w[10], w[11]),
                               pack_bf16x2<true>(w[12], w[13]), pack_bf16x2<true>(w[14], w[15]));
            }
            umma::fence_proxy_async();
            umma::fence_before_sync();
            group_sync(bar_id);
            if (gtid == 0) {
                const uint32_t b0 = sbase + (l == 1 ? kMlpW2 : (l == 2 ? kMlpW3 : (l == 3 ? kMlpW4 : kMlpW5)));
                mlp_issue(taddr, bbase, b0, kGuideHid, l == 4 ? kGuideOutPad : kGuideHid, bar);
            }
            if (!(ok = wait_layer())) break;
        }
        if (!ok) break;
        umma::fence_after_sync();
        // outputs 0..39 of this row. Rows that are consecutive in the output
        // (Features::kContiguous) go through the now free buffer, row-major,
        // and leave with one bulk copy per tile that runs while the group goes
        // on (the buffer is rewritten only after the copy has read it); rows
        // that go to path slots are stored from registers, 16 bytes at a time.
        {
            uint32_t a[16], b[16], c[16];
            umma::tmem_ld16_async(lane_addr, a);
            umma::tmem_ld16_async(lane_addr + 16, b);
            umma::tmem_wait_ld32(a, b);
            umma::tmem_ld16_async(lane_addr + 32, c);
            umma::tmem_wait_ld16(c);
            uint4 o[kMiOutRow / 16];   // the row as stored (FP32: 10 x 16 bytes, BF16: 5)
            if constexpr (sizeof(Out) == 4) {
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    o[e] = make_uint4(a[4 * e], a[4 * e + 1], a[4 * e + 2], a[4 * e + 3]);
                    o[4 + e] = make_uint4(b[4 * e], b[4 * e + 1], b[4 * e + 2], b[4 * e + 3]);
                }
                o[8] = make_uint4(c[0], c[1], c[2], c[3]);
                o[9] = make_uint4(c[4], c[5], c[6], c[7]);
            } else {
                const float *v = (const float *)a, *v2 = (const float *)b, *v3 = (const float *)c;
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    o[e] = make_uint4(pack_bf16x2<false>(v[8 * e], v[8 * e + 1]), pack_bf16x2<false>(v[8 * e + 2], v[8 * e + 3]),
                                      pack_bf16x2<false>(v[8 * e + 4], v[8 * e + 5]), pack_bf16x2<false>(v[8 * e + 6], v[8 * e + 7]));
                    o[2 + e] = make_uint4(
                        pack_bf16x2<false>(v2[8 * e], v2[8 * e + 1]), pack_bf16x2<false>(v2[8 * e + 2], v2[8 * e + 3]),
                        pack_bf16x2<false>(v2[8 * e + 4], v2[8 * e + 5]), pack_bf16x2<false>(v2[8 * e + 6], v2[8 * e + 7]));
                }
                o[4] = make_uint4(pack_bf16x2<false>(v3[0], v3[1]), pack_bf16x2<false>(v3[2], v3[3]),
                                  pack_bf16x2<false>(v3[4], v3[5]), pack_bf16x2<false>(v3[6], v3[7]));
            }
            constexpr int kParts = kGuideOut * (int)sizeof(Out) / 16;
            if constexpr (Features::kContiguous) {
                uint4 *srow = (uint4 *)(buf + r * kGuideOut * (uint32_t)sizeof(Out));
#pragma unroll
                for (int e = 0; e < kParts; ++e) srow[e] = o[e];
                umma::fence_proxy_async();
            } else if (row < n) {
                uint4 *dst = (uint4 *)(out + (size_t)feat.out_row(row) * kGuideOut);
#pragma unroll
                for (int e = 0; e < kParts; ++e) dst[e] = o[e];
            }
        }
        // the accumulator and the buffer are reused by the next tile
        umma::fence_before_sync();
        group_sync(bar_id);
        if constexpr (Features::kContiguous) {
            if (gtid == 0) {
                const uint32_t rows = min(kMlpTile, n - t * kMlpTile);
                umma::bulk_store(out + (size_t)feat.out_row(t * kMlpTile) * kGuideOut, bbase,
                                 rows * kGuideOut * (uint32_t)sizeof(Out));
                umma::bulk_commit();
            }
        }
#pragma unroll
        for (int k = 0; k < 7; ++k) f[k] = fn[k];
    }
    if (!ok && gtid == 0) {
        // the product in flight may still complete: wait for it once more
        // (bounded) before the tensor memory is released
        umma::mbar_wait(bar, phase ^ 1u);
        atomicExch(err, 1u);
    }
    umma::bulk_wait_all();   // this thread's output copies are done
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    if (warp == 0) umma::tmem_dealloc(*s_taddr, kMiTmemCols);
}

}  // namespace rtg
