// field.cu -- xi generation (Philox4x64-10 + Box-Muller) and the truncated KL
// contraction Z = Phi diag(sqrt(lambda)) xi (field law of Sec. 1, Eq. (1.2),
// sampled by a truncated Karhunen-Loeve sum instead of the paper's circulant
// embedding).
#include <cmath>

#include "common.cuh"
#include "kl_tc.cuh"
#include "philox.cuh"
#include "prof.cuh"

namespace msg {

__global__ void k_normals(uint64_t seed, uint64_t s0, int64_t S, int M, double* xi)
{
    const int nb = (M + 3) / 4;
    const int64_t total = S * nb;
    const double two_pi = 6.283185307179586476925286766559;
    const double inv53 = 1.0 / 9007199254740992.0;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = t / nb;
        int j = (int)(t % nb);
        uint64_t x0 = (uint64_t)j, x1 = s0 + (uint64_t)i, x2 = 0, x3 = 0;
        philox4x64_10(x0, x1, x2, x3, seed, 0);
        uint64_t w[4] = {x0, x1, x2, x3};
        double z[4];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            double ua = (double)(w[2 * h] >> 11) * inv53;
            double ub = (double)(w[2 * h + 1] >> 11) * inv53;
            double rad = sqrt(-2.0 * log(1.0 - ua));
            double sn, cs;
            sincos(two_pi * ub, &sn, &cs);
            z[2 * h] = rad * cs;
            z[2 * h + 1] = rad * sn;
        }
        double* out = xi + i * M + 4 * j;
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (4 * j + k < M) out[k] = z[k];
    }
}

// ---------------------------------------------------------------- SIMT GEMM --
// Z[s][x] = sum_m Phi[x][m] * (sqrt_lambda[m] * xi[s][m]); 64x64 tile per CTA,
// 16-deep K slices staged in shared memory, 4x4 outputs per thread.
template <class TP, class TA, class TZ>
__global__ void __launch_bounds__(256) k_kl_simt(const TP* __restrict__ Phi, const double* __restrict__ sl,
                                                 const double* __restrict__ xi, int64_t npts, int M, int64_t S,
                                                 TZ* __restrict__ Z)
{
    __shared__ TA sA[16][64 + 1];  // [k][s]
    __shared__ TA sB[16][64 + 1];  // [k][x]
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int64_t s0 = (int64_t)blockIdx.y * 64, x0 = (int64_t)blockIdx.x * 64;
    TA acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = TA(0);
    for (int k0 = 0; k0 < M; k0 += 16) {
        for (int e = threadIdx.x; e < 64 * 16; e += 256) {
            int r = e / 16, k = e % 16;
            int64_t s = s0 + r, x = x0 + r;
            int m = k0 + k;
            sA[k][r] = (s < S && m < M) ? (TA)(sl[m] * xi[s * M + m]) : TA(0);
            sB[k][r] = (x < npts && m < M) ? (TA)Phi[x * M + m] : TA(0);
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            TA av[4], bv[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) av[a] = sA[k][ty * 4 + a];
#pragma unroll
            for (int b = 0; b < 4; ++b) bv[b] = sB[k][tx * 4 + b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] += av[a] * bv[b];
        }
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        int64_t s = s0 + ty * 4 + a;
        if (s >= S) continue;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            int64_t x = x0 + tx * 4 + b;
            if (x < npts) Z[s * npts + x] = (TZ)acc[a][b];
        }
    }
}

__global__ void k_to_float(const double* in, float* out, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (float)in[i];
}

}  // namespace msg

using namespace msg;

extern "C" int32_t msg_normals(uint64_t seed, uint64_t s0, int64_t S, int32_t M, double* xi, void* stream)
{
    clear_error();
    if (S < 0 || M < 1) { set_error("msg_normals: need S >= 0 and M >= 1"); return MSG_ERR_INVALID; }
    if (S == 0) return MSG_OK;
    if (!xi) { set_error("msg_normals: xi is NULL"); return MSG_ERR_INVALID; }
    int64_t total = S * ((M + 3) / 4);
    int blocks = (int)std::min<int64_t>((total + 255) / 256, 152 * 16);
    prof_begin(K_NORMALS, (cudaStream_t)stream);
    k_normals<<<blocks, 256, 0, (cudaStream_t)stream>>>(seed, s0, S, M, xi);
    prof_end(K_NORMALS, (cudaStream_t)stream, 8.0 * S * M, 0.0);
    MSG_CHECK_LAUNCH();
    return MSG_OK;
}

namespace {
size_t align256(size_t x) { return (x + 255) / 256 * 256; }
}

extern "C" size_t kl_prepared_bytes(int64_t npts, int32_t M, int32_t mode)
{
    clear_error();
    if (npts < 1 || M < 1) return 0;
    switch (mode) {
    case MSG_GEMM_FP64: return align256(sizeof(double) * npts * M) + align256(sizeof(double) * M);
    case MSG_GEMM_FP32: return align256(sizeof(float) * npts * M) + align256(sizeof(double) * M);
    case MSG_GEMM_BF16X3:
    case MSG_GEMM_TF32: return kl_tc_prepared_bytes(npts, M, mode);
    default: return 0;
    }
}

extern "C" int32_t kl_prepare(const double* Phi, const double* sqrt_lambda, int64_t npts, int32_t M, int32_t mode,
                              void* prepared, size_t prepared_bytes, void* stream)
{
    clear_error();
    if (npts < 1 || M < 1 || !Phi || !sqrt_lambda || !prepared) {
        set_error("kl_prepare: invalid arguments");
        return MSG_ERR_INVALID;
    }
    size_t need = kl_prepared_bytes(npts, M, mode);
    if (need == 0) { set_error("kl_prepare: unknown mode"); return MSG_ERR_INVALID; }
    if (prepared_bytes < need) { set_error("kl_prepare: buffer too small"); return MSG_ERR_WORKSPACE; }
    cudaStream_t st = (cudaStream_t)stream;
    char* base = (char*)prepared;
    if (mode == MSG_GEMM_BF16X3 || mode == MSG_GEMM_TF32) {
        if ((uintptr_t)prepared % 256) { set_error("kl_prepare: prepared buffer must be 256-byte aligned"); return MSG_ERR_INVALID; }
        return kl_tc_prepare(Phi, sqrt_lambda, npts, M, mode, prepared, st);
    }
    if (mode == MSG_GEMM_FP64) {
        MSG_CUDA_TRY(cudaMemcpyAsync(base, Phi, sizeof(double) * npts * M, cudaMemcpyDeviceToDevice, st));
        MSG_CUDA_TRY(cudaMemcpyAsync(base + align256(sizeof(double) * npts * M), sqrt_lambda, sizeof(double) * M,
                                     cudaMemcpyDeviceToDevice, st));
    } else {
        prof_begin(K_KL, st);
        k_to_float<<<152 * 8, 256, 0, st>>>(Phi, (float*)base, npts * M);
        prof_end(K_KL, st, 12.0 * npts * M, 0.0);
        MSG_CHECK_LAUNCH();
        MSG_CUDA_TRY(cudaMemcpyAsync(base + align256(sizeof(float) * npts * M), sqrt_lambda, sizeof(double) * M,
                                     cudaMemcpyDeviceToDevice, st));
    }
    return MSG_OK;
}

extern "C" int32_t sample_field(const void* prepared, int64_t npts, int32_t M, int32_t mode, const double* xi,
                                int64_t S, void* Z, int32_t z_fp32, void* stream)
{
    clear_error();
    if (npts < 1 || M < 1 || S < 0) { set_error("sample_field: invalid sizes"); return MSG_ERR_INVALID; }
    if (S == 0) return MSG_OK;
    if (!prepared || !xi || !Z) { set_error("sample_field: NULL pointer"); return MSG_ERR_INVALID; }
    cudaStream_t st = (cudaStream_t)stream;
    if (mode == MSG_GEMM_BF16X3 || mode == MSG_GEMM_TF32) {
        if ((uintptr_t)prepared % 256) { set_error("sample_field: prepared buffer must be 256-byte aligned"); return MSG_ERR_INVALID; }
        return kl_tc_sample(prepared, npts, M, mode, xi, S, Z, z_fp32, st);
    }
    if (S > 65535LL * 64) { set_error("sample_field: too many samples for one call"); return MSG_ERR_INVALID; }
    dim3 grid((unsigned)((npts + 63) / 64), (unsigned)((S + 63) / 64));
    const char* base = (const char*)prepared;
    const double pe = mode == MSG_GEMM_FP64 ? 8.0 : 4.0, ze = z_fp32 ? 4.0 : 8.0;
    prof_begin(K_KL, st);
    if (mode == MSG_GEMM_FP64) {
        const double* Phi = (const double*)base;
        const double* sl = (const double*)(base + align256(sizeof(double) * npts * M));
        if (z_fp32) k_kl_simt<double, double, float><<<grid, 256, 0, st>>>(Phi, sl, xi, npts, M, S, (float*)Z);
        else k_kl_simt<double, double, double><<<grid, 256, 0, st>>>(Phi, sl, xi, npts, M, S, (double*)Z);
    } else if (mode == MSG_GEMM_FP32) {
        const float* Phi = (const float*)base;
        const double* sl = (const double*)(base + align256(sizeof(float) * npts * M));
        if (z_fp32) k_kl_simt<float, float, float><<<grid, 256, 0, st>>>(Phi, sl, xi, npts, M, S, (float*)Z);
        else k_kl_simt<float, float, double><<<grid, 256, 0, st>>>(Phi, sl, xi, npts, M, S, (double*)Z);
    } else {
        set_error("sample_field: unknown mode");
        return MSG_ERR_INVALID;
    }
    prof_end(K_KL, st, pe * npts * M + 8.0 * S * M + ze * S * npts, 2.0 * npts * M * S);
    MSG_CHECK_LAUNCH();
    return MSG_OK;
}
