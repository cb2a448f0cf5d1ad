// prof.cuh -- launch counting and optional per-kernel-class event timing.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace msg {

enum KernelClass {
    K_PRE = 0,   // PRE half of a visit above the cut (zero, nu1 sweeps, restriction)
    K_POST,      // POST half of a visit above the cut (prolongation, nu2 sweeps)
    K_LOW,       // whole recursion at and below the cut, one warp per item (k_low)
    K_RESIDUAL,  // FP64 residual + convergence decision
    K_UPDATE,    // FP64 update u += e
    K_INTERP,    // FMSG cubic interpolation
    K_QOI,       // quantity of interest
    K_COEFFS,    // a = exp(Z) on every grid
    K_NORMALS,   // Philox + Box-Muller
    K_KL,        // KL contraction
    K_MIMC,      // multi-index differences
    K_CE,        // circulant-embedding sampler (covariance, spectrum scaling, extraction)
    K_NCLASS
};

// Every kernel launch of the library goes through these two calls:
//   prof_begin(cls, st) before the launch, prof_end(cls, st, bytes, flops, level) after.
// They count launches always and, while profiling is on, record CUDA events on
// `st` for a random 1/n of each class's launches.  `level` tags multigrid
// launches with their diagonal (-1: none).
void prof_begin(int cls, cudaStream_t st);
void prof_end(int cls, cudaStream_t st, double bytes, double flops, int level = -1);

}  // namespace msg
