// Online path-guiding proposal (placeholder entry points; the network
// kernels are added in a later change).
#include "internal.h"

using namespace rtg;

struct rt_guide {
    int dummy;
};

extern "C" int64_t rt_guide_num_params(void) { return 224 * 64 + 3 * 64 * 64 + 64 * 40; }

#define RT_GUIDE_UNSUPPORTED(name)                                        \
    do {                                                                  \
        set_error(name ": guiding is not available in this build");       \
        return RT_NOT_SUPPORTED;                                          \
    } while (0)

extern "C" rt_status rt_guide_create(const rt_scene *, const rt_guide_opts *, rt_guide **out) {
    if (out) *out = nullptr;
    RT_GUIDE_UNSUPPORTED("rt_guide_create");
}
extern "C" rt_status rt_guide_destroy(rt_guide *) { return RT_OK; }
extern "C" rt_status rt_guide_get_params(const rt_guide *, float *) { RT_GUIDE_UNSUPPORTED("rt_guide_get_params"); }
extern "C" rt_status rt_guide_set_params(rt_guide *, const float *) { RT_GUIDE_UNSUPPORTED("rt_guide_set_params"); }
extern "C" rt_status rt_guide_state_size(const rt_guide *, int64_t *) { RT_GUIDE_UNSUPPORTED("rt_guide_state_size"); }
extern "C" rt_status rt_guide_save(const rt_guide *, void *) { RT_GUIDE_UNSUPPORTED("rt_guide_save"); }
extern "C" rt_status rt_guide_load(rt_guide *, const void *) { RT_GUIDE_UNSUPPORTED("rt_guide_load"); }
extern "C" rt_status rt_guide_infer(const rt_guide *, const float *, int64_t, float *, void *) {
    RT_GUIDE_UNSUPPORTED("rt_guide_infer");
}
extern "C" rt_status rt_guide_loss_grad(const rt_guide *, const float *, const float *, const float *, int64_t, float *,
                                        float *, void *) {
    RT_GUIDE_UNSUPPORTED("rt_guide_loss_grad");
}
extern "C" rt_status rt_guide_train_step(rt_guide *, const float *, const float *, const float *, int64_t, void *) {
    RT_GUIDE_UNSUPPORTED("rt_guide_train_step");
}
