// Online-trained path-guiding proposal (not part of the paper): a one-blob
// encoded (position, outgoing direction, normal) -> 224 -> 64 -> 64 -> 64 ->
// 64 -> 40 ReLU MLP whose 40 outputs parameterise an 8-lobe von Mises-Fisher
// mixture over directions. It is mixed with BSDF sampling by one-sample MIS
// in the shading kernel, so the estimator stays consistent whatever the
// network predicts. Weights are kept as FP32 masters with Adam moments on the
// device and as BF16 copies for the tensor cores; every dense product (the
// forward layers, the input gradients and the weight gradients) runs on
// tcgen05 through gemm_bf16, with FP32 accumulation.
//
// Layouts (row-major): weights W_l [out][in] (layer 5 padded to 48 output
// rows); activations H_l [n][64] BF16 plus their transposes [64][n] for the
// weight gradients; network outputs [n][48] FP32 (first 40 used, lobe k at
// 5k: mu xyz, kappa (softplus), logit).
//
// Kernels: inference is one fused launch (guide_mlp.cuh); a training step is
// the fused forward pass with the loss gradient (same file, training mode),
// then per layer a tcgen05 GEMM for dY_l = (dY_{l+1} W_{l+1}) * relu'(H_l)
// with the ReLU mask and the transposed copy in its epilogue, one for the
// weight gradient dW_l = dY_l^T X_{l-1}, and one Adam launch plus the BF16
// repacking of the weights. gemm_bf16's layer-by-layer forward pass remains
// as a cross-check of the fused kernel.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <cuda_bf16.h>
#include <vector>

#include "guide.cuh"
#include "guide_mlp.cuh"
#include "internal.h"

namespace rtg {

rt_status gemm_bf16(const __nv_bfloat16 *A, const __nv_bfloat16 *B, float *C, int M, int N, int K, int lda, int ldb,
                    int ldc, int accumulate, uint32_t *err, cudaStream_t st);
rt_status gemm_bf16_relu_bwd(const __nv_bfloat16 *A, const __nv_bfloat16 *B, int M, int N, int K, int lda, int ldb,
                             const __nv_bfloat16 *H, __nv_bfloat16 *dY, __nv_bfloat16 *dYT, int64_t ldt, uint32_t *err,
                             cudaStream_t st);

static const int kIn[5] = {kGuideIn, kGuideHid, kGuideHid, kGuideHid, kGuideHid};
static const int kOut[5] = {kGuideHid, kGuideHid, kGuideHid, kGuideHid, kGuideOut};
static const int kOutPad[5] = {kGuideHid, kGuideHid, kGuideHid, kGuideHid, kGuideOutPad};

static int64_t param_offset(int l) {
    int64_t o = 0;
    for (int i = 0; i < l; ++i) o += (int64_t)kIn[i] * kOut[i];
    return o;
}

// ------------------------------------------------------------ kernels
// The activations of the training forward pass and the backward signals are
// stored twice, row-major [n_pad][C] for the next layer's product and
// transposed [C][n_pad] for the weight gradients. A block builds a tile of
// 64 rows in shared memory (row stride C + 2, so that the transposed reads
// fall in different banks) and writes both copies with coalesced stores.
constexpr int kTileRows = 64;

template <int C, class F>
__device__ __forceinline__ void store_tile_and_transpose(int64_t r0, int64_t n_pad, const F &val, __nv_bfloat16 *M,
                                                         __nv_bfloat16 *MT) {
    __shared__ __nv_bfloat16 tile[kTileRows * (C + 2)];
    for (int i = threadIdx.x; i < kTileRows * C; i += blockDim.x) {
        const int rr = i / C, c = i % C;
        const __nv_bfloat16 b = __float2bfloat16(val(r0 + rr, c));
        tile[rr * (C + 2) + c] = b;
        M[(r0 + rr) * C + c] = b;
    }
    if (!MT) return;
    __syncthreads();
    for (int i = threadIdx.x; i < kTileRows * C; i += blockDim.x) {
        const int c = i / kTileRows, rr = i % kTileRows;
        MT[(int64_t)c * n_pad + r0 + rr] = tile[rr * (C + 2) + c];
    }
}

// X = one-blob(features) [n_pad][224] (zero rows past n) and X^T.
__global__ void k_oneblob(const float *feat, int64_t n, int64_t n_pad, __nv_bfloat16 *X, __nv_bfloat16 *XT) {
    const int64_t r0 = (int64_t)blockIdx.x * kTileRows;
    auto val = [&](int64_t r, int c) { return r < n ? oneblob_bin(feat[r * 7 + c / kGuideBins], c % kGuideBins) : 0.f; };
    store_tile_and_transpose<kGuideIn>(r0, n_pad, val, X, XT);
}

// H = bf16(relu(Z)) [n_pad][64] (zero rows past n); optional transpose HT.
__global__ void k_relu_pack(const float *Z, int64_t n, int64_t n_pad, __nv_bfloat16 *H, __nv_bfloat16 *HT) {
    const int64_t r0 = (int64_t)blockIdx.x * kTileRows;
    auto val = [&](int64_t r, int c) { return r < n ? fmaxf(Z[r * kGuideHid + c], 0.f) : 0.f; };
    store_tile_and_transpose<kGuideHid>(r0, n_pad, val, H, HT);
}

// Adam (Kingma and Ba 2015); omb1 = 1 - beta1 and omb2 = 1 - beta2 come from
// the host in double precision (1 - 0.999f in FP32 is 1.3e-5 off 0.001).
__global__ void k_adam(float *p, const float *g, float *m, float *v, int64_t n, float lr, float b1, float b2,
                       float omb1, float omb2, float eps, float c1, float c2) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float gi = g[i];
        float mi = b1 * m[i] + omb1 * gi;
        float vi = b2 * v[i] + omb2 * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// BF16 copies of layer l: W [out_pad][in], W^T [in][out_pad] and the layer's
// part of the fused kernels' shared-memory image (canonical K-major layout
// at byte offset mlp_image_base(l)).
__global__ void k_pack_layer(const float *W32, int in, int out, int out_pad, __nv_bfloat16 *W, __nv_bfloat16 *WT,
                             unsigned char *image, uint32_t image_base) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < out_pad * in; i += gridDim.x * blockDim.x) {
        int o = i / in, k = i % in;
        float v = o < out ? W32[(int64_t)o * in + k] : 0.f;
        __nv_bfloat16 b = __float2bfloat16(v);
        W[i] = b;
        if (WT) WT[(int64_t)k * out_pad + o] = b;
        *(__nv_bfloat16 *)(image + image_base + umma::kmajor_offset((uint32_t)o, (uint32_t)k, (uint32_t)in)) = b;
    }
}

// Gradient of the padded layer-5 output (48 rows) into the 40-row layout.
__global__ void k_copy_rows(const float *src, int rows, int cols, float *dst) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < rows * cols; i += gridDim.x * blockDim.x) dst[i] = src[i];
}

// Fused inference (guide_mlp.cuh) over rows of given features [n][7].
struct ArrayFeatures {
    static constexpr bool kContiguous = true;   // output row of row r is r
    const float *feat;
    uint32_t n;
    __device__ uint32_t count() const { return n; }
    __device__ uint32_t out_row(uint32_t row) const { return row; }
    __device__ void operator()(uint32_t row, float f[7]) const {
#pragma unroll
        for (int k = 0; k < 7; ++k) f[k] = feat[7 * (size_t)row + k];
    }
};

__global__ void __launch_bounds__(kMiThreads, 1) k_guide_mlp(MlpWeights w, ArrayFeatures feat, float *raw, uint32_t *err) {
    mlp_infer_tiles(w, feat, raw, err);
}

// Training forward pass with the loss gradient (guide_mlp.cuh, MlpTrain).
__global__ void __launch_bounds__(512, 1) k_guide_mlp_train(MlpWeights w, ArrayFeatures feat, MlpTrain tr,
                                                            uint32_t *err) {
    mlp_tiles<true>(w, feat, nullptr, err, tr);
}

static int grid1d(int64_t n, int block = 256) {
    int64_t g = (n + block - 1) / block;
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, 152 * 16));
}

}  // namespace rtg

using namespace rtg;

struct rt_guide {
    rt_guide_opts opts{};
    int64_t nparams = 0;
    float *W32 = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr;
    __nv_bfloat16 *Wb[5] = {nullptr}, *WTb[5] = {nullptr};
    unsigned char *image = nullptr;   // the five layers in the fused kernels' shared-memory layout
    int64_t step = 0;
    uint64_t sets = 0;   // iteration sets rendered with this guide
    // scratch for a batch of up to cap rows
    int64_t cap = 0;
    __nv_bfloat16 *X0 = nullptr, *X0T = nullptr, *H[4] = {nullptr}, *HT[4] = {nullptr}, *dY = nullptr, *dYT = nullptr;
    __nv_bfloat16 *dYh[2] = {nullptr, nullptr}, *dYhT[2] = {nullptr, nullptr};   // hidden-layer gradients
    float *Z = nullptr, *raw = nullptr, *dW5 = nullptr, *loss = nullptr;
    uint32_t *err = nullptr;
    std::vector<void *> allocs;
    float3 bb_lo, bb_hi;
};

namespace {

template <class T>
rt_status galloc(rt_guide *g, T **p, size_t count) {
    cudaError_t e = cudaMalloc((void **)p, count * sizeof(T));
    if (e != cudaSuccess) { set_error("guide: device allocation failed"); return RT_OOM; }
    g->allocs.push_back(*p);
    return RT_OK;
}

rt_status repack(rt_guide *g, cudaStream_t st) {
    for (int l = 0; l < 5; ++l) {
        k_pack_layer<<<grid1d((int64_t)kOutPad[l] * kIn[l]), 256, 0, st>>>(g->W32 + param_offset(l), kIn[l], kOut[l],
                                                                            kOutPad[l], g->Wb[l], g->WTb[l], g->image,
                                                                            mlp_image_base(l));
    }
    RT_CUDA_TRY(cudaGetLastError());
    return RT_OK;
}

rt_status ensure_scratch(rt_guide *g, int64_t n) {
    int64_t need = (n + 127) / 128 * 128;
    if (need <= g->cap) return RT_OK;
    // grow: drop the old scratch (weights stay)
    cudaDeviceSynchronize();
    for (void *p : {(void *)g->X0, (void *)g->X0T, (void *)g->H[0], (void *)g->H[1], (void *)g->H[2], (void *)g->H[3],
                    (void *)g->HT[0], (void *)g->HT[1], (void *)g->HT[2], (void *)g->HT[3], (void *)g->dY, (void *)g->dYT,
                    (void *)g->dYh[0], (void *)g->dYh[1], (void *)g->dYhT[0], (void *)g->dYhT[1],
                    (void *)g->Z, (void *)g->raw}) {
        if (!p) continue;
        cudaFree(p);
        g->allocs.erase(std::remove(g->allocs.begin(), g->allocs.end(), p), g->allocs.end());
    }
    rt_status s;
    if ((s = galloc(g, &g->X0, need * kGuideIn)) || (s = galloc(g, &g->X0T, need * kGuideIn)) ||
        (s = galloc(g, &g->dY, need * kGuideOutPad)) || (s = galloc(g, &g->dYT, need * kGuideOutPad)) ||
        (s = galloc(g, &g->dYh[0], need * kGuideHid)) || (s = galloc(g, &g->dYhT[0], need * kGuideHid)) ||
        (s = galloc(g, &g->dYh[1], need * kGuideHid)) || (s = galloc(g, &g->dYhT[1], need * kGuideHid)) ||
        (s = galloc(g, &g->Z, need * kGuideHid)) || (s = galloc(g, &g->raw, need * kGuideOutPad)))
        return s;
    for (int l = 0; l < 4; ++l)
        if ((s = galloc(g, &g->H[l], need * kGuideHid)) || (s = galloc(g, &g->HT[l], need * kGuideHid))) return s;
    g->cap = need;
    return RT_OK;
}

// Forward pass over n rows of features; raw outputs in g->raw [n_pad][48].
rt_status forward(rt_guide *g, const float *feat, int64_t n, bool keep_transposes, cudaStream_t st) {
    const int64_t n_pad = (n + 127) / 128 * 128;
    const int tiles = (int)(n_pad / kTileRows);
    k_oneblob<<<tiles, 256, 0, st>>>(feat, n, n_pad, g->X0, keep_transposes ? g->X0T : nullptr);
    const __nv_bfloat16 *x = g->X0;
    for (int l = 0; l < 4; ++l) {
        rt_status s = gemm_bf16(x, g->Wb[l], g->Z, (int)n_pad, kGuideHid, kIn[l], kIn[l], kIn[l], kGuideHid, 0, g->err, st);
        if (s != RT_OK) return s;
        k_relu_pack<<<tiles, 256, 0, st>>>(g->Z, n, n_pad, g->H[l], keep_transposes ? g->HT[l] : nullptr);
        x = g->H[l];
    }
    rt_status s = gemm_bf16(x, g->Wb[4], g->raw, (int)n_pad, kGuideOutPad, kGuideHid, kGuideHid, kGuideHid,
                            kGuideOutPad, 0, g->err, st);
    if (s != RT_OK) return s;
    RT_CUDA_TRY(cudaGetLastError());
    return RT_OK;
}

// Fused training forward pass: activations, their transposes and the loss
// gradient dY / dYT for n rows (one launch), loss summed into g->loss.
rt_status train_forward(rt_guide *g, const float *feat, const float *wi, const float *weight, int64_t n,
                        cudaStream_t st) {
    const int64_t n_pad = (n + 127) / 128 * 128;
    rt_status s = mlp_kernel_attr((const void *)k_guide_mlp_train, kMlpSmemTrain);
    if (s != RT_OK) return s;
    RT_CUDA_TRY(cudaMemsetAsync(g->loss, 0, sizeof(float), st));
    MlpTrain tr{};
    tr.wi = wi;
    tr.weight = weight;
    tr.inv_n = 1.f / (float)n;
    tr.n_pad = (uint32_t)n_pad;
    tr.XT = g->X0T;
    for (int l = 0; l < 4; ++l) { tr.H[l] = g->H[l]; tr.HT[l] = g->HT[l]; }
    tr.dY = g->dY;
    tr.dYT = g->dYT;
    tr.loss = g->loss;
    const int grid = (int)std::min<int64_t>((n_pad + kMlpGroup * kMlpTile - 1) / (kMlpGroup * kMlpTile),
                                            (int64_t)sm_count());
    k_guide_mlp_train<<<grid, kMlpThreads, kMlpSmemTrain, st>>>(guide_weights(g), ArrayFeatures{feat, (uint32_t)n},
                                                                 tr, g->err);
    RT_CUDA_TRY(cudaGetLastError());
    return RT_OK;
}

// Gradient of the mean loss into g->grad (FP32, layer-major [out][in]),
// from dY / dYT of the training forward pass.
rt_status backward(rt_guide *g, int64_t n, cudaStream_t st) {
    const int64_t n_pad = (n + 127) / 128 * 128;
    rt_status s;
    // layer 5: dW5 [48][64] = dY5^T H4 ; dY4 = (dY5 W5) * relu'(H4)
    if ((s = gemm_bf16(g->dYT, g->HT[3], g->dW5, kGuideOutPad, kGuideHid, (int)n_pad, (int)n_pad, (int)n_pad,
                       kGuideHid, 0, g->err, st)))
        return s;
    k_copy_rows<<<grid1d(kGuideOut * kGuideHid), 256, 0, st>>>(g->dW5, kGuideOut, kGuideHid, g->grad + param_offset(4));
    // the layer-5 gradient lives in the [n_pad][48] dY buffer; the hidden
    // layers' go to dYh ([n_pad][64], ping-pong with dYh2)
    const __nv_bfloat16 *dy = g->dY, *dyT = g->dYT;
    int kdy = kGuideOutPad;
    __nv_bfloat16 *bufs[2][2] = {{g->dYh[0], g->dYhT[0]}, {g->dYh[1], g->dYhT[1]}};
    for (int l = 3; l >= 0; --l) {
        __nv_bfloat16 *ndy = bufs[l & 1][0], *ndyT = bufs[l & 1][1];
        // dY_l = (dY_{l+1} W_{l+1}) * relu'(H_l), and its transpose
        if ((s = gemm_bf16_relu_bwd(dy, g->WTb[l + 1], (int)n_pad, kGuideHid, kdy, kdy, kdy, g->H[l], ndy, ndyT, n_pad,
                                    g->err, st)))
            return s;
        // dW_l [64][in] = dY_l^T X_{l-1}
        const __nv_bfloat16 *xT = l == 0 ? g->X0T : g->HT[l - 1];
        if ((s = gemm_bf16(ndyT, xT, g->grad + param_offset(l), kGuideHid, kIn[l], (int)n_pad, (int)n_pad, (int)n_pad,
                           kIn[l], 0, g->err, st)))
            return s;
        dy = ndy;
        dyT = ndyT;
        kdy = kGuideHid;
    }
    (void)dyT;
    RT_CUDA_TRY(cudaGetLastError());
    return RT_OK;
}

rt_status check_err(rt_guide *g, cudaStream_t st) {
    uint32_t h = 0;
    RT_CUDA_TRY(cudaMemcpyAsync(&h, g->err, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    RT_CUDA_TRY(cudaStreamSynchronize(st));
    if (h) {
        cudaMemsetAsync(g->err, 0, sizeof(uint32_t), st);
        set_error("guide: tensor-core completion wait timed out");
        return RT_TIMEOUT;
    }
    return RT_OK;
}

}  // namespace

namespace rtg {
rt_status guide_check(rt_guide *g, cudaStream_t st) { return check_err(g, st); }

MlpWeights guide_weights(const rt_guide *g) {
    MlpWeights w;
    for (int l = 0; l < 5; ++l) w.W[l] = g->Wb[l];
    w.image = g->image;
    return w;
}
uint32_t *guide_err(const rt_guide *g) { return g->err; }

// Shared-memory opt-in of a fused network kernel, once per device.
rt_status mlp_kernel_attr(const void *kernel, uint32_t bytes) {
    int dev = 0;
    RT_CUDA_TRY(cudaGetDevice(&dev));
    static std::vector<std::pair<const void *, int>> done;
    for (auto &p : done)
        if (p.first == kernel && p.second == dev) return RT_OK;
    RT_CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    done.push_back({kernel, dev});
    return RT_OK;
}

// Raw outputs [n_pad][48] for n feature rows (device), no sync: the fused
// tensor-core kernel, one launch.
rt_status guide_infer_async(rt_guide *g, const float *feat, int64_t n, float *out, cudaStream_t st) {
    rt_status s;
    if ((s = mlp_kernel_attr((const void *)k_guide_mlp, kMlpInferSmem)) != RT_OK) return s;
    const int64_t per_cta = kMiGroups * kMlpTile;   // one tile per group
    const int grid = (int)std::min<int64_t>((n + per_cta - 1) / per_cta, (int64_t)sm_count());
    k_guide_mlp<<<grid, kMiThreads, kMlpInferSmem, st>>>(guide_weights(g), ArrayFeatures{feat, (uint32_t)n}, out,
                                                           g->err);
    RT_CUDA_TRY(cudaGetLastError());
    return RT_OK;
}

// The same outputs layer by layer through gemm_bf16 (the training forward).
rt_status guide_infer_layers_async(rt_guide *g, const float *feat, int64_t n, const float **raw_out, cudaStream_t st) {
    rt_status s = ensure_scratch(g, n);
    if (s != RT_OK) return s;
    s = forward(g, feat, n, false, st);
    *raw_out = g->raw;
    return s;
}
rt_status guide_train_async(rt_guide *g, const float *feat, const float *wi, const float *weight, int64_t n,
                            cudaStream_t st) {
    if (n <= 0) return RT_OK;
    rt_status s = ensure_scratch(g, n);
    if (s != RT_OK) return s;
    for (uint32_t it = 0; it < std::max(1u, g->opts.train_steps); ++it) {
        if ((s = train_forward(g, feat, wi, weight, n, st)) || (s = backward(g, n, st))) return s;
        ++g->step;
        float b1 = 0.9f, b2 = 0.999f;
        // bias corrections in double: 1.f - (float)0.999^t loses 1.3e-5 to cancellation
        float c1 = (float)(1.0 - std::pow(0.9, (double)g->step)), c2 = (float)(1.0 - std::pow(0.999, (double)g->step));
        k_adam<<<grid1d(g->nparams), 256, 0, st>>>(g->W32, g->grad, g->m, g->v, g->nparams, g->opts.learning_rate, b1,
                                                   b2, (float)(1.0 - 0.9), (float)(1.0 - 0.999), 1e-8f, c1, c2);
        if ((s = repack(g, st))) return s;
    }
    return RT_OK;
}
float guide_alpha(const rt_guide *g) { return g->opts.alpha; }
void guide_bounds(const rt_guide *g, float3 &lo, float3 &hi) { lo = g->bb_lo; hi = g->bb_hi; }
uint32_t guide_batch(const rt_guide *g) { return g->opts.batch; }
bool guide_trained(const rt_guide *g) { return g->step > 0; }
uint32_t guide_depth(const rt_guide *g) { return g->opts.guide_depth; }
// Training cadence: after every set for the first warm_steps steps, then
// after every train_every-th set.
bool guide_young(const rt_guide *g) { return g->step < (int64_t)g->opts.warm_steps; }
uint32_t guide_warm_left(const rt_guide *g) {
    if (!guide_young(g)) return 0u;
    const int64_t per = std::max(1u, g->opts.train_steps);
    return (uint32_t)(((int64_t)g->opts.warm_steps - g->step + per - 1) / per);
}
uint32_t guide_warm_set_batches(const rt_guide *g) { return g->opts.warm_set_batches; }
bool guide_should_train(rt_guide *g) {
    const uint64_t k = g->sets++;
    const uint32_t every = std::max(1u, g->opts.train_every);
    return guide_young(g) || k % every == 0;
}
}  // namespace rtg

extern "C" int64_t rt_guide_num_params(void) { return kGuideParams; }

extern "C" rt_status rt_guide_create(const rt_scene *scene, const rt_guide_opts *opts, rt_guide **out) {
    if (!out) { set_error("rt_guide_create: null output"); return RT_INVALID_ARG; }
    *out = nullptr;
    rt_guide *g = new rt_guide();
    if (opts) g->opts = *opts;
    if (!g->opts.batch) g->opts.batch = 65536;
    if (!(g->opts.learning_rate > 0.f)) g->opts.learning_rate = 1e-2f;
    if (!(g->opts.alpha > 0.f)) g->opts.alpha = 0.5f;
    if (g->opts.alpha > 1.f) { delete g; set_error("rt_guide_create: alpha must be in (0, 1]"); return RT_INVALID_ARG; }
    if (!g->opts.train_steps) g->opts.train_steps = 1;
    if (!g->opts.warm_steps) g->opts.warm_steps = 32;
    if (!g->opts.warm_set_batches) g->opts.warm_set_batches = 32;
    if (!g->opts.guide_depth) g->opts.guide_depth = 3;
    g->nparams = kGuideParams;
    if (scene) { g->bb_lo = scene->dev.bb_lo; g->bb_hi = scene->dev.bb_hi; }
    else { g->bb_lo = make_float3(0.f, 0.f, 0.f); g->bb_hi = make_float3(1.f, 1.f, 1.f); }
    auto fail = [&](rt_status s) { rt_guide_destroy(g); return s; };
    rt_status s;
    if ((s = galloc(g, &g->W32, g->nparams)) || (s = galloc(g, &g->m, g->nparams)) || (s = galloc(g, &g->v, g->nparams)) ||
        (s = galloc(g, &g->grad, g->nparams)) || (s = galloc(g, &g->dW5, (size_t)kGuideOutPad * kGuideHid)) ||
        (s = galloc(g, &g->loss, 1)) || (s = galloc(g, &g->err, 1)))
        return fail(s);
    for (int l = 0; l < 5; ++l)
        if ((s = galloc(g, &g->Wb[l], (size_t)kOutPad[l] * kIn[l])) || (s = galloc(g, &g->WTb[l], (size_t)kOutPad[l] * kIn[l])))
            return fail(s);
    if ((s = galloc(g, &g->image, (size_t)kMlpX))) return fail(s);
    // He-style initialisation from SplitMix64 (seeded), uniform in +-sqrt(6 / fan_in)
    std::vector<float> w(g->nparams);
    uint64_t st = g->opts.seed ^ 0x6A09E667F3BCC908ull;
    for (int l = 0; l < 5; ++l) {
        double a = std::sqrt(6.0 / kIn[l]) * (l == 4 ? 0.1 : 1.0);
        for (int64_t i = 0; i < (int64_t)kIn[l] * kOut[l]; ++i) {
            uint64_t z = (st += 0x9E3779B97F4A7C15ull);
            z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
            z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
            z ^= z >> 31;
            double u = (double)(z >> 11) * (1.0 / 9007199254740992.0);
            w[param_offset(l) + i] = (float)((2.0 * u - 1.0) * a);
        }
    }
    if (cudaMemcpy(g->W32, w.data(), w.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(g->m, 0, g->nparams * 4) != cudaSuccess || cudaMemset(g->v, 0, g->nparams * 4) != cudaSuccess ||
        cudaMemset(g->err, 0, 4) != cudaSuccess) {
        set_error("rt_guide_create: upload failed");
        return fail(RT_CUDA_ERROR);
    }
    if ((s = repack(g, 0)) != RT_OK) return fail(s);
    if (cudaDeviceSynchronize() != cudaSuccess) { set_error("rt_guide_create: init failed"); return fail(RT_CUDA_ERROR); }
    *out = g;
    return RT_OK;
}

extern "C" rt_status rt_guide_destroy(rt_guide *g) {
    if (!g) return RT_OK;
    for (void *p : g->allocs) cudaFree(p);
    delete g;
    return RT_OK;
}

extern "C" rt_status rt_guide_get_params(const rt_guide *g, float *params) {
    if (!g || !params) { set_error("rt_guide_get_params: null argument"); return RT_INVALID_ARG; }
    RT_CUDA_TRY(cudaMemcpy(params, g->W32, g->nparams * 4, cudaMemcpyDeviceToHost));
    return RT_OK;
}

extern "C" rt_status rt_guide_set_params(rt_guide *g, const float *params) {
    if (!g || !params) { set_error("rt_guide_set_params: null argument"); return RT_INVALID_ARG; }
    RT_CUDA_TRY(cudaMemcpy(g->W32, params, g->nparams * 4, cudaMemcpyHostToDevice));
    RT_CUDA_TRY(cudaMemset(g->m, 0, g->nparams * 4));
    RT_CUDA_TRY(cudaMemset(g->v, 0, g->nparams * 4));
    g->step = 0;
    rt_status s = repack(g, 0);
    if (s != RT_OK) return s;
    RT_CUDA_TRY(cudaDeviceSynchronize());
    return RT_OK;
}

extern "C" rt_status rt_guide_state_size(const rt_guide *g, int64_t *bytes) {
    if (!g || !bytes) { set_error("rt_guide_state_size: null argument"); return RT_INVALID_ARG; }
    *bytes = 3 * g->nparams * 4 + 8;
    return RT_OK;
}

extern "C" rt_status rt_guide_save(const rt_guide *g, void *buf) {
    if (!g || !buf) { set_error("rt_guide_save: null argument"); return RT_INVALID_ARG; }
    char *b = (char *)buf;
    RT_CUDA_TRY(cudaMemcpy(b, g->W32, g->nparams * 4, cudaMemcpyDeviceToHost));
    RT_CUDA_TRY(cudaMemcpy(b + g->nparams * 4, g->m, g->nparams * 4, cudaMemcpyDeviceToHost));
    RT_CUDA_TRY(cudaMemcpy(b + 2 * g->nparams * 4, g->v, g->nparams * 4, cudaMemcpyDeviceToHost));
    std::memcpy(b + 3 * g->nparams * 4, &g->step, 8);
    return RT_OK;
}

extern "C" rt_status rt_guide_load(rt_guide *g, const void *buf) {
    if (!g || !buf) { set_error("rt_guide_load: null argument"); return RT_INVALID_ARG; }
    const char *b = (const char *)buf;
    RT_CUDA_TRY(cudaMemcpy(g->W32, b, g->nparams * 4, cudaMemcpyHostToDevice));
    RT_CUDA_TRY(cudaMemcpy(g->m, b + g->nparams * 4, g->nparams * 4, cudaMemcpyHostToDevice));
    RT_CUDA_TRY(cudaMemcpy(g->v, b + 2 * g->nparams * 4, g->nparams * 4, cudaMemcpyHostToDevice));
    std::memcpy(&g->step, b + 3 * g->nparams * 4, 8);
    rt_status s = repack(g, 0);
    if (s != RT_OK) return s;
    RT_CUDA_TRY(cudaDeviceSynchronize());
    return RT_OK;
}

extern "C" rt_status rt_guide_infer(const rt_guide *gc, const float *features, int64_t n, float *raw, void *stream) {
    rt_guide *g = const_cast<rt_guide *>(gc);
    if (!g || (n > 0 && (!features || !raw)) || n < 0) { set_error("rt_guide_infer: invalid argument"); return RT_INVALID_ARG; }
    if (n == 0) return RT_OK;
    cudaStream_t st = (cudaStream_t)stream;
    rt_status s = guide_infer_async(g, features, n, raw, st);
    if (s != RT_OK) return s;
    return check_err(g, st);
}

extern "C" rt_status rt_guide_infer_async(const rt_guide *gc, const float *features, int64_t n, float *raw,
                                          void *stream) {
    rt_guide *g = const_cast<rt_guide *>(gc);
    if (!g || (n > 0 && (!features || !raw)) || n < 0) { set_error("rt_guide_infer_async: invalid argument"); return RT_INVALID_ARG; }
    if (n == 0) return RT_OK;
    return guide_infer_async(g, features, n, raw, (cudaStream_t)stream);
}

extern "C" rt_status rt_guide_check(const rt_guide *gc, void *stream) {
    rt_guide *g = const_cast<rt_guide *>(gc);
    if (!g) { set_error("rt_guide_check: invalid argument"); return RT_INVALID_ARG; }
    return check_err(g, (cudaStream_t)stream);
}

extern "C" rt_status rt_debug_guide_infer_layers(const rt_guide *gc, const float *features, int64_t n, float *raw,
                                                 void *stream) {
    rt_guide *g = const_cast<rt_guide *>(gc);
    if (!g || (n > 0 && (!features || !raw)) || n < 0) { set_error("rt_debug_guide_infer_layers: invalid argument"); return RT_INVALID_ARG; }
    if (n == 0) return RT_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const float *r = nullptr;
    rt_status s = guide_infer_layers_async(g, features, n, &r, st);
    if (s != RT_OK) return s;
    RT_CUDA_TRY(cudaMemcpy2DAsync(raw, kGuideOut * 4, r, kGuideOutPad * 4, kGuideOut * 4, n, cudaMemcpyDeviceToDevice, st));
    return check_err(g, st);
}

namespace rtg {
// The device mixture code of guided shading on given raw outputs: the
// density at wi, a direction drawn with (u_sel, u1, u2), and the density at
// that direction.
__global__ void k_debug_mixture(const float *raw, const float *wi, const float *u, int64_t n, float *pdf_wi,
                                float *ws, float *pdf_ws) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        Mixture m;
        decode_mixture(raw + kGuideOut * i, m);
        pdf_wi[i] = mixture_pdf(m, v3(wi[3 * i], wi[3 * i + 1], wi[3 * i + 2]));
        const V3 w = mixture_sample(m, u[3 * i], u[3 * i + 1], u[3 * i + 2]);
        ws[3 * i] = w.x; ws[3 * i + 1] = w.y; ws[3 * i + 2] = w.z;
        pdf_ws[i] = mixture_pdf(m, w);
    }
}
}  // namespace rtg

/* Test hook: the device-side von Mises-Fisher mixture of guided shading
 * (decode, density, sampling) on DEVICE arrays raw [n][40], wi [n][3],
 * u [n][3] (lobe select, u1, u2) -> pdf_wi [n], ws [n][3], pdf_ws [n]. */
extern "C" rt_status rt_debug_guide_mixture(const float *raw, const float *wi, const float *u, int64_t n,
                                            float *pdf_wi, float *ws, float *pdf_ws, void *stream) {
    if (n < 0 || (n > 0 && (!raw || !wi || !u || !pdf_wi || !ws || !pdf_ws))) {
        set_error("rt_debug_guide_mixture: invalid argument");
        return RT_INVALID_ARG;
    }
    if (n == 0) return RT_OK;
    k_debug_mixture<<<grid1d(n), 256, 0, (cudaStream_t)stream>>>(raw, wi, u, n, pdf_wi, ws, pdf_ws);
    RT_CUDA_TRY(cudaGetLastError());
    return RT_OK;
}

extern "C" rt_status rt_guide_loss_grad(const rt_guide *gc, const float *features, const float *wi, const float *weight,
                                        int64_t n, float *grad, float *loss, void *stream) {
    rt_guide *g = const_cast<rt_guide *>(gc);
    if (!g || n <= 0 || !features || !wi || !weight || !grad) { set_error("rt_guide_loss_grad: invalid argument"); return RT_INVALID_ARG; }
    cudaStream_t st = (cudaStream_t)stream;
    rt_status s = ensure_scratch(g, n);
    if (s != RT_OK) return s;
    if ((s = train_forward(g, features, wi, weight, n, st)) || (s = backward(g, n, st))) return s;
    RT_CUDA_TRY(cudaMemcpyAsync(grad, g->grad, g->nparams * 4, cudaMemcpyDeviceToDevice, st));
    if (loss) RT_CUDA_TRY(cudaMemcpyAsync(loss, g->loss, 4, cudaMemcpyDeviceToHost, st));
    return check_err(g, st);
}

extern "C" rt_status rt_guide_train_step(rt_guide *g, const float *features, const float *wi, const float *weight,
                                         int64_t n, void *stream) {
    if (!g || n <= 0 || !features || !wi || !weight) { set_error("rt_guide_train_step: invalid argument"); return RT_INVALID_ARG; }
    cudaStream_t st = (cudaStream_t)stream;
    rt_status s = guide_train_async(g, features, wi, weight, n, st);
    if (s != RT_OK) return s;
    return check_err(g, st);
}
