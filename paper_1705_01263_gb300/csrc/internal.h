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
uint32_t nth_prime(int dim);

}  // namespace rtg
