// common.cuh -- internal helpers of the MSG-MIMC CUDA library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/msg_mimc.h"

namespace msg {

// thread-local last error, set by every failing entry point
void set_error(const std::string& what);
void clear_error();

#define MSG_CUDA_TRY(expr)                                                                        \
    do {                                                                                          \
        cudaError_t _e = (expr);                                                                  \
        if (_e != cudaSuccess) {                                                                  \
            ::msg::set_error(std::string(#expr) + ": " + cudaGetErrorString(_e));                 \
            return MSG_ERR_CUDA;                                                                  \
        }                                                                                         \
    } while (0)

#define MSG_CHECK_LAUNCH()                                                                        \
    do {                                                                                          \
        cudaError_t _e = cudaGetLastError();                                                      \
        if (_e != cudaSuccess) {                                                                  \
            ::msg::set_error(std::string("kernel launch: ") + cudaGetErrorString(_e));            \
            return MSG_ERR_CUDA;                                                                  \
        }                                                                                         \
    } while (0)

// Pinned host staging for the host-side tables an entry point uploads, so that
// the upload is a true asynchronous copy and the call returns without waiting
// for the stream.  staging_acquire hands out a slot of at least `bytes`;
// staging_release records an event on `st` after the copies from the slot were
// enqueued, and the slot is handed out again only once that event has completed.
int staging_acquire(size_t bytes, void** ptr, int* token);
int staging_release(int token, cudaStream_t st);

// ---------------------------------------------------------------------------
// Hierarchy layout.
//
// Grid (p,q) of the semi-coarsened hierarchy (Eq. (2.1)) has nx = 2^p,
// ny = 2^q cells and (nx+1)(ny+1) nodes including the boundary, stored row by
// row (x fastest).  All grids (p',q') with p' <= P, q' <= Q of one rectangle
// are stored back to back in (p' major, q' minor) order, so with
//   T(n) = sum_{k=1..n} (2^k + 1) = 2^(n+1) - 2 + n
// grid (p',q') starts at node T(p'-1) T(Q) + (2^p' + 1) T(q'-1) and the whole
// rectangle holds T(P) T(Q) nodes.
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ int64_t tsum(int n) { return (int64_t(2) << n) - 2 + n; }
__host__ __device__ __forceinline__ int64_t grid_offset(int p, int q, int Qtop)
{
    return tsum(p - 1) * tsum(Qtop) + (int64_t)((1 << p) + 1) * tsum(q - 1);
}
__host__ __device__ __forceinline__ int64_t rect_nodes(int P, int Q) { return tsum(P) * tsum(Q); }
__host__ __device__ __forceinline__ int64_t field_nodes(int P, int Q)
{
    return (int64_t)((1 << (P + 1)) + 1) * ((1 << (Q + 1)) + 1);
}

}  // namespace msg
