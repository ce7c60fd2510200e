// batched.cu -- many independent Tucker operators in one persistent launch.
#include "internal.h"
#include "ptx.cuh"

namespace kron {
cudaError_t batched_error_word(unsigned int *out, bool clear) { return read_error_word(out, clear); }
}  // namespace kron

struct kron_batched_plan_s {
    int batch;
};

extern "C" {
kron_status kron_batched_plan_create(kron_batched_plan *plan, int, int, const int64_t *, const int64_t *,
                                     kron_dtype, kron_prec, unsigned) {
    if (plan) *plan = nullptr;
    return KRON_ERR_UNSUPPORTED;
}
kron_status kron_batched_plan_destroy(kron_batched_plan plan) {
    delete plan;
    return KRON_OK;
}
kron_status kron_batched_workspace_size(kron_batched_plan, size_t *) { return KRON_ERR_UNSUPPORTED; }
double kron_batched_flops(kron_batched_plan) { return 0.0; }
kron_status kron_batched_bind(kron_batched_plan, const void *const *, const void *const *, void *const *,
                              void *, size_t, kron_stream_t) {
    return KRON_ERR_UNSUPPORTED;
}
kron_status kron_batched_run(kron_batched_plan, void *, size_t, kron_stream_t) { return KRON_ERR_UNSUPPORTED; }
}
