// kl_tc.cu -- tcgen05 BF16x3 KL contraction (placeholder until the kernel lands).
#include "common.cuh"
#include "kl_tc.cuh"

namespace msg {
size_t kl_tc_prepared_bytes(int64_t, int32_t) { return 0; }
int32_t kl_tc_prepare(const double*, const double*, int64_t, int32_t, void*, cudaStream_t)
{
    set_error("BF16X3 mode not built");
    return MSG_ERR_UNSUPPORTED;
}
int32_t kl_tc_sample(const void*, int64_t, int32_t, const double*, int64_t, void*, int32_t, cudaStream_t)
{
    set_error("BF16X3 mode not built");
    return MSG_ERR_UNSUPPORTED;
}
}  // namespace msg
