// BF16 GEMM on the tcgen05 tensor cores with FP32 accumulation in tensor
// memory: C[M x N] = A[M x K] * B[N x K]^T (or C += ...). It is the dense
// layer primitive of the guiding network (forward, input gradients and weight
// gradients are all expressed as this product with suitably stored operands).
//
// One CTA of 128 threads computes a 128 x NT tile (NT <= 256, a multiple of
// 16) over one split of K (several CTAs share an SM, as many as its tensor
// memory holds): K is walked in chunks of 64; each chunk of A and B
// is copied from global memory into the canonical no-swizzle K-major shared
// layout with 16-byte loads, then one thread issues four 128 x NT x 16 MMAs
// and commits them to an mbarrier that every thread waits on (bounded) before
// the buffers are refilled. The epilogue reads the accumulator with
// tcgen05.ld (warp w owns rows 32w..32w+31) and stores, or atomically adds
// when K is split across CTAs.
#include <algorithm>
#include <cuda_bf16.h>

#include "internal.h"
#include "umma.cuh"

namespace rtg {

struct GemmArgs {
    const __nv_bfloat16 *A, *B;
    float *C;
    int M, N, K, lda, ldb, ldc;
    int k_split;        // K elements per split (multiple of 64)
    int nt;             // N columns per CTA (multiple of 16, <= 256)
    int mode;           // 0 store, 1 atomic add, 2 ReLU backward (below), 3 partial of split blockIdx.z
    float *part;        // mode 3: partial sums, split z at part + z * M * N (row-major, ld N)
    uint32_t *err;      // set to 1 if a tensor-core wait timed out
    // mode 2: instead of C, dY = bf16(C * (H > 0)) row-major [M][N] (ld N)
    // and its transpose dYT [N][ldt], H BF16 row-major [M][N]
    const __nv_bfloat16 *H;
    __nv_bfloat16 *dY, *dYT;
    int64_t ldt;
};

constexpr int kGemmKChunk = 64;
constexpr int kGemmSmemMax = 116 * 1024;   // attribute limit of the launch below

// Dynamic shared memory of a launch with `nt` columns per CTA: the A and B
// chunks and the barrier, raised so that the CTAs that fit on one SM (228 KB
// of shared memory, 1 KB reserved per CTA) never ask for more than the 512
// tensor-memory columns an SM has: an allocation then never waits.
inline int gemm_smem(int nt, uint32_t ncols) {
    const int need = 16384 + nt * 128 + 64;
    const int max_ctas = (int)(512u / ncols);
    const int floor_bytes = 233472 / (max_ctas + 1) - 1024 + 16;
    return std::min(kGemmSmemMax, std::max(need, floor_bytes));
}

__global__ void __launch_bounds__(128, 1) k_gemm_bf16(GemmArgs g) {
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *sA = smem;                    // 128 x 64 bf16 = 16 KB
    unsigned char *sB = smem + 16384;            // nt x 64 bf16 <= 32 KB
    uint64_t *mbar = (uint64_t *)(smem + 16384 + g.nt * 128);
    uint32_t *s_taddr = (uint32_t *)(smem + 16384 + g.nt * 128 + 16);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * 128, n0 = blockIdx.y * g.nt;
    const int k_begin = blockIdx.z * g.k_split;
    const int k_end = min(g.K, k_begin + g.k_split);
    const uint32_t ncols = g.nt <= 32 ? 32u : (g.nt <= 64 ? 64u : (g.nt <= 128 ? 128u : 256u));
    if (warp == 0) umma::tmem_alloc(s_taddr, ncols);
    if (tid == 0) umma::mbar_init(mbar, 1);
    umma::fence_before_sync();
    __syncthreads();
    umma::fence_after_sync();
    const uint32_t taddr = *s_taddr;
    const uint32_t idesc = umma::make_idesc_bf16(128, (uint32_t)g.nt);
    uint32_t phase = 0;
    bool ok = true, any = false;
    for (int k0 = k_begin; k0 < k_end; k0 += kGemmKChunk) {
        // stage A (128 rows) and B (nt rows) chunks; rows or k beyond the
        // matrix are zero
        for (int c = tid; c < 128 * 8; c += 128) {
            int r = c >> 3, g8 = c & 7;
            int gr = m0 + r, gk = k0 + 8 * g8;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (gr < g.M && gk < k_end) v = *(const uint4 *)(g.A + (size_t)gr * g.lda + gk);
            *(uint4 *)(sA + umma::kmajor_offset(r, 8 * g8, kGemmKChunk)) = v;
        }
        for (int c = tid; c < g.nt * 8; c += 128) {
            int r = c >> 3, g8 = c & 7;
            int gr = n0 + r, gk = k0 + 8 * g8;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (gr < g.N && gk < k_end) v = *(const uint4 *)(g.B + (size_t)gr * g.ldb + gk);
            *(uint4 *)(sB + umma::kmajor_offset(r, 8 * g8, kGemmKChunk)) = v;
        }
        umma::fence_proxy_async();
        __syncthreads();
        if (tid == 0) {
            umma::fence_after_sync();
            const uint32_t a0 = umma::smem_addr(sA), b0 = umma::smem_addr(sB);
#pragma unroll
            for (int kk = 0; kk < kGemmKChunk / 16; ++kk) {
                uint64_t ad = umma::make_desc(a0 + kk * 256, 128, (kGemmKChunk / 8) * 128);
                uint64_t bd = umma::make_desc(b0 + kk * 256, 128, (kGemmKChunk / 8) * 128);
                umma::mma_bf16(taddr, ad, bd, idesc, (any || kk > 0) ? 1u : 0u);
            }
            umma::mma_commit(mbar);
        }
        any = true;
        if (!umma::mbar_wait(mbar, phase)) ok = false;
        phase ^= 1u;
        umma::fence_after_sync();
        __syncthreads();
        if (!ok) break;
    }
    if (!ok && tid == 0) atomicExch(g.err, 1u);
    if (ok && any) {
        const int row = m0 + warp * 32 + lane;
        for (int c0 = 0; c0 < g.nt; c0 += 16) {
            float v[16];
            umma::tmem_ld16(taddr + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
            if (row < g.M && g.mode == 2 && (g.N % 16) == 0 && n0 + c0 + 16 <= g.N) {
                // whole 16-column chunk: the row's 32 bytes of H and dY in
                // two 16-byte accesses, dYT column by column (coalesced over
                // the warp's consecutive rows)
                const size_t i0 = (size_t)row * g.N + n0 + c0;
                const uint4 h0 = *(const uint4 *)(g.H + i0), h1 = *(const uint4 *)(g.H + i0 + 8);
                __align__(16) __nv_bfloat16 hb[16], b[16];
                *(uint4 *)hb = h0;
                *(uint4 *)(hb + 8) = h1;
#pragma unroll
                for (int j = 0; j < 16; ++j) b[j] = __float2bfloat16(__bfloat162float(hb[j]) > 0.f ? v[j] : 0.f);
                *(uint4 *)(g.dY + i0) = *(const uint4 *)b;
                *(uint4 *)(g.dY + i0 + 8) = *(const uint4 *)(b + 8);
#pragma unroll
                for (int j = 0; j < 16; ++j) g.dYT[(size_t)(n0 + c0 + j) * g.ldt + row] = b[j];
            } else if (row < g.M && g.mode == 2) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int col = n0 + c0 + j;
                    if (col < g.N) {
                        const size_t i = (size_t)row * g.N + col;
                        const __nv_bfloat16 b = __float2bfloat16(__bfloat162float(g.H[i]) > 0.f ? v[j] : 0.f);
                        g.dY[i] = b;
                        g.dYT[(size_t)col * g.ldt + row] = b;
                    }
                }
            } else if (row < g.M && g.mode == 3) {
                float *dst = g.part + (size_t)blockIdx.z * g.M * g.N + (size_t)row * g.N;
                if ((g.N % 4) == 0 && n0 + c0 + 16 <= g.N) {
                    float4 *d4 = (float4 *)(dst + n0 + c0);
#pragma unroll
                    for (int e = 0; e < 4; ++e) d4[e] = make_float4(v[4 * e], v[4 * e + 1], v[4 * e + 2], v[4 * e + 3]);
                } else {
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const int col = n0 + c0 + j;
                        if (col < g.N) dst[col] = v[j];
                    }
                }
            } else if (row < g.M) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    int col = n0 + c0 + j;
                    if (col < g.N) {
                        float *dst = g.C + (size_t)row * g.ldc + col;
                        if (g.mode == 1) atomicAdd(dst, v[j]);
                        else *dst = v[j];
                    }
                }
            }
        }
    }
    umma::fence_before_sync();
    __syncthreads();
    if (warp == 0) umma::tmem_dealloc(taddr, ncols);
}

// C (+)= the sum of the splits' partial products. A block takes 32
// consecutive elements; its eight warps sum the splits z = g, g + 8, ... of
// them (warp g; loads coalesced over the elements), and the eight partial
// sums are added in warp order: a fixed order, so the result is the same on
// every run.
constexpr int kSumGroups = 8;
__global__ void __launch_bounds__(32 * kSumGroups) k_sum_splits(const float *part, int splits, int M, int N, float *C,
                                                                int ldc, int accumulate) {
    __shared__ float s_part[kSumGroups][32];
    const int64_t n = (int64_t)M * N;
    const int e = threadIdx.x & 31, g = threadIdx.x >> 5;
    for (int64_t i0 = (int64_t)blockIdx.x * 32; i0 < n; i0 += (int64_t)gridDim.x * 32) {
        const int64_t i = i0 + e;
        float acc = 0.f;
        if (i < n)
            for (int z = g; z < splits; z += kSumGroups) acc += part[(size_t)z * n + i];
        s_part[g][e] = acc;
        __syncthreads();
        if (g == 0 && i < n) {
            float sum = s_part[0][e];
            for (int k = 1; k < kSumGroups; ++k) sum += s_part[k][e];
            float *dst = C + (i / N) * ldc + (i % N);
            *dst = accumulate ? *dst + sum : sum;
        }
        __syncthreads();
    }
}

// Partial-sum workspace of the split-K products, one per device, grown on
// demand and kept for the life of the process (like a GEMM library's
// workspace).
static float *split_workspace(size_t floats, rt_status &st) {
    static float *buf[64] = {nullptr};
    static size_t cap[64] = {0};
    int dev = 0;
    st = RT_OK;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) { st = RT_CUDA_ERROR; return nullptr; }
    if (cap[dev] < floats) {
        if (buf[dev]) cudaFree(buf[dev]);
        buf[dev] = nullptr;
        cap[dev] = 0;
        if (cudaMalloc(&buf[dev], floats * sizeof(float)) != cudaSuccess) {
            set_error("gemm_bf16: split-K workspace allocation failed");
            st = RT_OOM;
            return nullptr;
        }
        cap[dev] = floats;
    }
    return buf[dev];
}

static rt_status gemm_launch(GemmArgs g, int accumulate, bool relu_bwd, cudaStream_t st) {
    const int M = g.M, N = g.N, K = g.K;
    if (M <= 0 || N <= 0 || K <= 0) return RT_OK;
    if ((K % 8) || (g.lda % 8) || (g.ldb % 8) || ((uintptr_t)g.A % 16) || ((uintptr_t)g.B % 16)) {
        set_error("gemm_bf16: K, lda, ldb must be multiples of 8 and A, B 16-byte aligned");
        return RT_INVALID_ARG;
    }
    static bool attr_set[64] = {false};
    int dev = 0;
    RT_CUDA_TRY(cudaGetDevice(&dev));
    if (dev >= 0 && dev < 64 && !attr_set[dev]) {
        RT_CUDA_TRY(cudaFuncSetAttribute(k_gemm_bf16, cudaFuncAttributeMaxDynamicSharedMemorySize, kGemmSmemMax));
        attr_set[dev] = true;
    }
    g.nt = std::min(256, (N + 15) / 16 * 16);
    const int mt = (M + 127) / 128, ntiles = (N + g.nt - 1) / g.nt;
    // split K when the output grid alone cannot fill the machine (not for
    // the ReLU-backward epilogue, which needs whole sums)
    int splits = 1;
    const int ctas = mt * ntiles;
    if (!relu_bwd && ctas < 152 && K > 4 * kGemmKChunk)
        splits = std::min((K + kGemmKChunk - 1) / kGemmKChunk, (2 * 152 + ctas - 1) / ctas);
    g.k_split = ((K + splits - 1) / splits + kGemmKChunk - 1) / kGemmKChunk * kGemmKChunk;
    splits = (K + g.k_split - 1) / g.k_split;
    // split K: each split stores its partial product and one pass sums them
    // (no atomics on the same addresses from every split)
    g.mode = relu_bwd ? 2 : (splits > 1 ? 3 : (accumulate ? 1 : 0));
    if (g.mode == 3) {
        rt_status ws;
        g.part = split_workspace((size_t)splits * M * N, ws);
        if (ws != RT_OK) return ws;
    }
    dim3 grid(mt, ntiles, splits);
    const uint32_t ncols = g.nt <= 32 ? 32u : (g.nt <= 64 ? 64u : (g.nt <= 128 ? 128u : 256u));
    k_gemm_bf16<<<grid, 128, gemm_smem(g.nt, ncols), st>>>(g);
    RT_CUDA_TRY(cudaGetLastError());
    if (g.mode == 3) {
        const int64_t n = (int64_t)M * N;
        const int blocks = (int)std::min<int64_t>((n + 31) / 32, 4096);
        k_sum_splits<<<blocks, 32 * kSumGroups, 0, st>>>(g.part, splits, M, N, g.C, g.ldc, accumulate);
        RT_CUDA_TRY(cudaGetLastError());
    }
    return RT_OK;
}

rt_status gemm_bf16(const __nv_bfloat16 *A, const __nv_bfloat16 *B, float *C, int M, int N, int K, int lda, int ldb,
                    int ldc, int accumulate, uint32_t *err, cudaStream_t st) {
    GemmArgs g{A, B, C, M, N, K, lda, ldb, ldc, 0, 0, 0, nullptr, err, nullptr, nullptr, nullptr, 0};
    return gemm_launch(g, accumulate, false, st);
}

// dY = bf16((A B^T) * (H > 0)) [M][N] and dYT [N][ldt]: the backward step of
// a ReLU layer fused into the product's epilogue.
rt_status gemm_bf16_relu_bwd(const __nv_bfloat16 *A, const __nv_bfloat16 *B, int M, int N, int K, int lda, int ldb,
                             const __nv_bfloat16 *H, __nv_bfloat16 *dY, __nv_bfloat16 *dYT, int64_t ldt, uint32_t *err,
                             cudaStream_t st) {
    GemmArgs g{A, B, nullptr, M, N, K, lda, ldb, N, 0, 0, 0, nullptr, err, H, dY, dYT, ldt};
    return gemm_launch(g, 0, true, st);
}

}  // namespace rtg

using namespace rtg;

extern "C" rt_status rt_gemm_bf16(const void *A, const void *B, float *C, int32_t M, int32_t N, int32_t K, int32_t lda,
                                  int32_t ldb, int32_t ldc, int32_t accumulate, void *stream) {
    if (!A || !B || !C || M < 0 || N < 0 || K < 0 || lda < K || ldb < K || ldc < N) {
        set_error("rt_gemm_bf16: invalid argument");
        return RT_INVALID_ARG;
    }
    static uint32_t *err[64] = {nullptr};
    int dev = 0;
    RT_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) { set_error("rt_gemm_bf16: device index out of range"); return RT_INVALID_ARG; }
    if (!err[dev]) {
        RT_CUDA_TRY(cudaMalloc(&err[dev], sizeof(uint32_t)));
        RT_CUDA_TRY(cudaMemset(err[dev], 0, sizeof(uint32_t)));
    }
    cudaStream_t st = (cudaStream_t)stream;
    rt_status s = gemm_bf16((const __nv_bfloat16 *)A, (const __nv_bfloat16 *)B, C, M, N, K, lda, ldb, ldc, accumulate,
                            err[dev], st);
    if (s != RT_OK) return s;
    uint32_t h = 0;
    RT_CUDA_TRY(cudaMemcpyAsync(&h, err[dev], sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    RT_CUDA_TRY(cudaStreamSynchronize(st));
    if (h) {
        cudaMemsetAsync(err[dev], 0, sizeof(uint32_t), st);
        set_error("rt_gemm_bf16: tensor-core completion wait timed out");
        return RT_TIMEOUT;
    }
    return RT_OK;
}
