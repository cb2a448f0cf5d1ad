// kl_tc.cuh -- tensor-core (tcgen05) KL contraction, internal interface.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace msg {
// mode: MSG_GEMM_BF16X3 or MSG_GEMM_TF32
size_t kl_tc_prepared_bytes(int64_t npts, int32_t M, int32_t mode);
int32_t kl_tc_prepare(const double* Phi, const double* sqrt_lambda, int64_t npts, int32_t M, int32_t mode,
                      void* prepared, cudaStream_t st);
int32_t kl_tc_sample(const void* prepared, int64_t npts, int32_t M, int32_t mode, const double* xi, int64_t S, void* Z,
                     int32_t z_fp32, cudaStream_t st);
}  // namespace msg
