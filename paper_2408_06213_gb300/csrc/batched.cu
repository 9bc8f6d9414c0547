// batched.cu -- many independent shuffles and samples (placeholder).
#include "brr_common.cuh"
#include "internal.h"

namespace brr {

brr_status launch_shuffle_batched(brr_ctx *, void *, const uint64_t *, uint32_t, uint32_t,
                                  const uint64_t *, uint64_t, const brr_schedule *, cudaStream_t) {
    return BRR_EINVAL;
}

brr_status launch_sample_batched(brr_ctx *, const uint64_t *, const uint32_t *, const uint64_t *,
                                 const uint64_t *, uint32_t, uint32_t, const brr_schedule *,
                                 uint32_t *, cudaStream_t, const uint64_t *, uint32_t, uint64_t) {
    return BRR_EINVAL;
}

}  // namespace brr
