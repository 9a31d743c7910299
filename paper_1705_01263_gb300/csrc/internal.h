// Library-internal declarations shared by the translation units.
#pragma once

#include <string>
#include <vector>

#include "bvh_build.h"
#include "common.cuh"
#include "halton.cuh"

struct rt_scene {
    rtg::DevScene dev{};       // device pointers
    rtg::DevScene host{};      // the same arrays in host memory (debug entry points)
    std::vector<void *> dev_allocs;
    std::vector<std::vector<uint8_t>> host_keep;
    int64_t num_nodes = 0, num_leaf_tris = 0, device_bytes = 0;
    int64_t num_triangles = 0;
    uint32_t num_materials = 0;
    int bvh_depth = 0;
    bool host_only = false;
};

struct rt_film {
    uint32_t W = 0, H = 0;
    double *sum = nullptr, *sum2 = nullptr;
    uint32_t *count = nullptr;
    uint64_t next_task = 0;    // tasks (pixel samples) accumulated so far, pass-major
    void *cache = nullptr;     // render resources reused across calls
};

namespace rtg {

void set_error(const std::string &msg);
rt_status cuda_status(cudaError_t e, const char *what);
#define RT_CUDA_TRY(expr)                                                  \
    do {                                                                   \
        cudaError_t _e = (expr);                                           \
        if (_e != cudaSuccess) return ::rtg::cuda_status(_e, #expr);       \
    } while (0)

std::vector<HaltonDim> make_dims(uint64_t seed, int ndims);

// guiding network (guide.cu)
rt_status guide_infer_async(rt_guide *g, const float *feat, int64_t n, float *out, cudaStream_t st);   // out: n x 40
rt_status guide_train_async(rt_guide *g, const float *feat, const float *wi, const float *weight, int64_t n,
                            cudaStream_t st);
float guide_alpha(const rt_guide *g);
void guide_bounds(const rt_guide *g, float3 &lo, float3 &hi);
uint32_t guide_batch(const rt_guide *g);
bool guide_trained(const rt_guide *g);
uint32_t guide_depth(const rt_guide *g);   // last guided vertex (0 = all)
bool guide_should_train(rt_guide *g);   // advances the set counter
bool guide_young(const rt_guide *g);    // fewer than its warm-up training steps taken
uint32_t guide_warm_left(const rt_guide *g);          // warm-up training calls (of train_steps steps) still to take
uint32_t guide_warm_set_batches(const rt_guide *g);   // training batches per warm-up set
struct MlpWeights;
MlpWeights guide_weights(const rt_guide *g);   // BF16 layers for the fused inference kernel
uint32_t *guide_err(const rt_guide *g);        // set by a tensor-core wait that timed out
rt_status guide_check(rt_guide *g, cudaStream_t st);   // RT_TIMEOUT (and clears) if it was set
rt_status mlp_kernel_attr(const void *kernel, uint32_t bytes);  // shared-memory opt-in of a fused network kernel
int sm_count();
uint32_t nth_prime(int dim);

}  // namespace rtg
