// BF16 GEMM on the tcgen05 tensor cores with FP32 accumulation in tensor
// memory: C[M x N] = A[M x K] * B[N x K]^T (or C += ...). It is the dense
// layer primitive of the guiding network (forward, input gradients and weight
// gradients are all expressed as this product with suitably stored operands).
//
// One CTA of 128 threads computes a 128 x NT tile (NT <= 256, a multiple of
// 16) over one split of K: K is walked in chunks of 64; each chunk of A and B
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
    int mode;           // 0 store, 1 atomic add
    uint32_t *err;      // set to 1 if a tensor-core wait timed out
};

constexpr int kGemmKChunk = 64;
constexpr int kGemmSmem = 116 * 1024;   // one CTA per SM: its 256 TMEM columns always fit

__global__ void __launch_bounds__(128, 1) k_gemm_bf16(GemmArgs g) {
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *sA = smem;                    // 128 x 64 bf16 = 16 KB
    unsigned char *sB = smem + 16384;            // nt x 64 bf16 <= 32 KB
    uint64_t *mbar = (uint64_t *)(smem + 16384 + 32768);
    uint32_t *s_taddr = (uint32_t *)(smem + 16384 + 32768 + 16);
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
            if (row < g.M) {
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

rt_status gemm_bf16(const __nv_bfloat16 *A, const __nv_bfloat16 *B, float *C, int M, int N, int K, int lda, int ldb,
                    int ldc, int accumulate, uint32_t *err, cudaStream_t st) {
    if (M <= 0 || N <= 0 || K <= 0) return RT_OK;
    if ((K % 8) || (lda % 8) || (ldb % 8) || ((uintptr_t)A % 16) || ((uintptr_t)B % 16)) {
        set_error("gemm_bf16: K, lda, ldb must be multiples of 8 and A, B 16-byte aligned");
        return RT_INVALID_ARG;
    }
    static bool attr_set[64] = {false};
    int dev = 0;
    RT_CUDA_TRY(cudaGetDevice(&dev));
    if (dev >= 0 && dev < 64 && !attr_set[dev]) {
        RT_CUDA_TRY(cudaFuncSetAttribute(k_gemm_bf16, cudaFuncAttributeMaxDynamicSharedMemorySize, kGemmSmem));
        attr_set[dev] = true;
    }
    GemmArgs g{A, B, C, M, N, K, lda, ldb, ldc, 0, 0, 0, err};
    g.nt = std::min(256, (N + 15) / 16 * 16);
    const int mt = (M + 127) / 128, ntiles = (N + g.nt - 1) / g.nt;
    // split K when the output grid alone cannot fill the machine
    int splits = 1;
    const int ctas = mt * ntiles;
    if (ctas < 152 && K > 4 * kGemmKChunk) splits = std::min((K + kGemmKChunk - 1) / kGemmKChunk, (2 * 152 + ctas - 1) / ctas);
    g.k_split = ((K + splits - 1) / splits + kGemmKChunk - 1) / kGemmKChunk * kGemmKChunk;
    splits = (K + g.k_split - 1) / g.k_split;
    g.mode = (splits > 1 || accumulate) ? 1 : 0;
    if (g.mode == 1 && !accumulate) RT_CUDA_TRY(cudaMemsetAsync(C, 0, sizeof(float) * ((size_t)(M - 1) * ldc + N), st));
    dim3 grid(mt, ntiles, splits);
    k_gemm_bf16<<<grid, 128, kGemmSmem, st>>>(g);
    RT_CUDA_TRY(cudaGetLastError());
    return RT_OK;
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
