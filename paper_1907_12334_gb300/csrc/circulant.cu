// circulant.cu -- circulant-embedding sampler of the paper's own field law
// (Sec. 4, numerical experiments): Matern covariance (Eq. (1.2)) with the
// scaling/rotation map T of Sec. 1, per-sample anisotropic ratio eta and
// rotation theta (hyper-parameters), hence per-sample eigenvalues.
//
// Per batch of B samples, in one stream:
//   k_ce_hyper    eta, theta of each sample (one Philox block each);
//   k_ce_cov      generating array c on the periodic M1 x M2 grid, FP64;
//   cuFFT D2Z     eigenvalues Lambda = DFT2(c) (half spectrum), FP64;
//   k_ce_scale    sqrt(max(Lambda, 0) / M) (xi1 + i xi2) as complex FP32, with
//                 xi drawn in place from the sample's Philox stream;
//   cuFFT C2C     forward transform in place, FP32;
//   k_ce_extract  real part on the field nodes -> Z (FP64, solver layout).
// The eigenvalues need FP64: in FP32 the smallest ones (the high frequencies,
// ~1e-3 of the largest at 256 x 256 and L = 7) would carry absolute errors
// near 1e-4, which is ~1e-3 of error in the field.  The sample transform in
// FP32 leaves ~1e-6.
#include <cufft.h>

#include <cmath>
#include <map>
#include <mutex>
#include <tuple>

#include "common.cuh"
#include "philox.cuh"
#include "prof.cuh"

namespace msg {
namespace {

struct CeLawDev {
    double nu, lam, eta_lo, eta_hi, th_lo, th_hi;  // rotation range in degrees
    int scale;                                     // 0: S as Sec. 1 prints it; 1: lambda as a length
};

// Eq. (1.2) for half-integer smoothness, x = 2 sqrt(nu) r:
// nu = 1/2: exp(-x); 3/2: (1 + x) exp(-x); 5/2: (1 + x + x^2/3) exp(-x).
__device__ __forceinline__ double ce_matern(double r, double nu)
{
    const double x = 2.0 * sqrt(nu) * r, e = exp(-x);
    if (nu == 0.5) return e;
    if (nu == 1.5) return (1.0 + x) * e;
    return (1.0 + x + x * x / 3.0) * e;
}

// Covariance at offset (dx, dy): r = ||S R (dx, dy)||, S = diag(1/sqrt(eta
// lambda), 1/sqrt(lambda)), R the rotation by theta (Sec. 1).
__device__ __forceinline__ double ce_cov(double dx, double dy, double ct, double st, double ieta_lam, double ilam,
                                         double nu)
{
    const double rx = ct * dx - st * dy, ry = st * dx + ct * dy;
    return ce_matern(sqrt(rx * rx * ieta_lam + ry * ry * ilam), nu);
}

// eta and theta (radians) of global samples s0 .. s0 + n - 1.
__global__ void k_ce_hyper(uint64_t seed, uint64_t s0, int n, CeLawDev law, double* et)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint64_t x0 = 0, x1 = s0 + (uint64_t)i, x2 = 1, x3 = 0;
    philox4x64_10(x0, x1, x2, x3, seed, 0);
    const double inv53 = 1.0 / 9007199254740992.0;
    const double u0 = (double)(x0 >> 11) * inv53, u1 = (double)(x1 >> 11) * inv53;
    et[2 * i] = law.eta_lo + (law.eta_hi - law.eta_lo) * u0;
    const double deg = law.th_lo + (law.th_hi - law.th_lo) * u1;
    et[2 * i + 1] = deg * (3.14159265358979323846 / 180.0);
}

// Generating array of sample blockIdx.y: c[k2][k1] = C(d1 hx, d2 hy) with d
// the signed periodic offset (k, or k - M above M/2); at k = M/2 both signs
// are averaged so that the embedding stays symmetric under the rotation.
// C(-d) = C(d) bit for bit (the rotated offset only changes sign), so half of
// the points are evaluated and each value is also stored at its mirror
// (-k1, -k2) mod (M1, M2): the rows 1..M2/2-1 whole, and the first half of
// the two rows that are their own mirror (k2 = 0 and k2 = M2/2).
__device__ __forceinline__ double ce_cov_at(int k1, int k2, int M1, int M2, double hx, double hy, double ct,
                                            double st, double ieta_lam, double ilam, double nu)
{
    const int d1 = k1 <= M1 / 2 ? k1 : k1 - M1, d2 = k2 <= M2 / 2 ? k2 : k2 - M2;
    const double dx = d1 * hx, dy = d2 * hy;
    if (2 * k1 != M1 && 2 * k2 != M2) return ce_cov(dx, dy, ct, st, ieta_lam, ilam, nu);
    const double dx2 = (2 * k1 == M1) ? -dx : dx, dy2 = (2 * k2 == M2) ? -dy : dy;
    return (ce_cov(dx, dy, ct, st, ieta_lam, ilam, nu) + ce_cov(dx, dy2, ct, st, ieta_lam, ilam, nu) +
            ce_cov(dx2, dy, ct, st, ieta_lam, ilam, nu) + ce_cov(dx2, dy2, ct, st, ieta_lam, ilam, nu)) /
           4.0;
}

__global__ void k_ce_cov(int M1, int M2, double hx, double hy, CeLawDev law, const double* et, double* c)
{
    const int64_t N = (int64_t)M1 * M2;
    const int b = blockIdx.y;
    const double eta = et[2 * b], th = et[2 * b + 1];
    const double ct = cos(th), st = sin(th);
    // r^2 = rx^2 ieta_lam + ry^2 ilam: S = diag(1/sqrt(eta lam), 1/sqrt(lam)) or diag(1/(eta lam), 1/lam)
    const double ieta_lam = law.scale ? 1.0 / ((eta * law.lam) * (eta * law.lam)) : 1.0 / (eta * law.lam);
    const double ilam = law.scale ? 1.0 / (law.lam * law.lam) : 1.0 / law.lam;
    double* cb = c + (int64_t)b * N;
    const int64_t full = (int64_t)(M2 / 2 - 1) * M1, self = 2 * (int64_t)(M1 / 2 + 1);
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < full + self;
         t += (int64_t)gridDim.x * blockDim.x) {
        int k1, k2;
        if (t < full) {
            k2 = 1 + (int)(t / M1);
            k1 = (int)(t - (int64_t)(k2 - 1) * M1);
        } else {
            const int64_t u = t - full;
            k2 = u < M1 / 2 + 1 ? 0 : M2 / 2;
            k1 = (int)(u < M1 / 2 + 1 ? u : u - (M1 / 2 + 1));
        }
        const double v = ce_cov_at(k1, k2, M1, M2, hx, hy, ct, st, ieta_lam, ilam, law.nu);
        const int m1 = (M1 - k1) % M1, m2 = (M2 - k2) % M2;
        cb[(int64_t)k2 * M1 + k1] = v;
        cb[(int64_t)m2 * M1 + m1] = v;
    }
}

// Lambda at point (k1, k2) from the half spectrum (M2 rows of M1/2 + 1) that
// D2Z leaves: the spectrum of a real array is Hermitian, Lambda(k) = conj
// Lambda(-k), and the real part is the eigenvalue.
__device__ __forceinline__ double ce_lambda(const double2* sp, int M1, int M2, int k1, int k2)
{
    const int H = M1 / 2 + 1;
    if (k1 < H) return sp[(int64_t)k2 * H + k1].x;
    return sp[(int64_t)((M2 - k2) % M2) * H + (M1 - k1)].x;
}

// buf[k] = sqrt(max(Lambda_k, 0) / M) (xi1_k + i xi2_k) for sample blockIdx.y
// (global sample s0 + blockIdx.y).  Points 2j and 2j+1 share Philox block
// (j, s, 0, 0) under key (seed, 0): normals 4j..4j+3 of the sample's stream,
// numbered as msg_normals numbers them; Box-Muller on the same 53-bit uniforms
// with log (log1p below 1/2) and sin/cos in single precision.
__global__ void k_ce_scale(int M1, int M2, uint64_t seed, uint64_t s0, const double2* spec, float2* buf,
                           int32_t* status)
{
    const int64_t N = (int64_t)M1 * M2, pairs = N / 2;
    const int b = blockIdx.y;
    const double2* sp = spec + (int64_t)b * M2 * (M1 / 2 + 1);
    float2* out = buf + (int64_t)b * N;
    const double l0 = sp[0].x;  // sum of c > 0: the largest eigenvalue
    const double inv_n = 1.0 / (double)N, inv53 = 1.0 / 9007199254740992.0;
    bool neg = false;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < pairs; j += (int64_t)gridDim.x * blockDim.x) {
        uint64_t x0 = (uint64_t)j, x1 = s0 + (uint64_t)b, x2 = 0, x3 = 0;
        philox4x64_10(x0, x1, x2, x3, seed, 0);
        const uint64_t w[4] = {x0, x1, x2, x3};
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int64_t k = 2 * j + h;
            const int k2 = (int)(k / M1), k1 = (int)(k - (int64_t)k2 * M1);
            const double lam = ce_lambda(sp, M1, M2, k1, k2);
            neg |= lam < -1e-10 * l0;
            const float a = sqrtf((float)(fmax(lam, 0.0) * inv_n));  // single precision suffices: a is a float
            const double ua = (double)(w[2 * h] >> 11) * inv53, ub = (double)(w[2 * h + 1] >> 11) * inv53;
            const float lg = ua < 0.5 ? log1pf(-(float)ua) : logf((float)(1.0 - ua));
            const float rad = a * sqrtf(-2.0f * lg);
            float sn, cs;
            sincospif(2.0f * (float)ub, &sn, &cs);
            out[k] = make_float2(rad * cs, rad * sn);
        }
    }
    if (neg && status) atomicOr(&status[b], MSG_CE_NEGATIVE_EIGENVALUE);
}

// Z[b][j nfx + i] = Re buf[b][j M1 + i] on the field's nodes.
__global__ void k_ce_extract(int M1, int nfx, int nfy, int64_t N, const float2* buf, double* Z)
{
    const int b = blockIdx.y;
    const int64_t n = (int64_t)nfx * nfy;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(k / nfx), i = (int)(k - (int64_t)j * nfx);
        Z[(int64_t)b * n + k] = (double)buf[(int64_t)b * N + (int64_t)j * M1 + i].x;
    }
}

size_t al256(size_t x) { return (x + 255) / 256 * 256; }

struct CeSizes {
    int M1, M2, nfx, nfy;
    int64_t N, H;  // points of the periodic grid; complex values of its half spectrum
    size_t et, buf, spec, total;
};

CeSizes ce_sizes(int P, int Q, const msg_ce_law& law)
{
    CeSizes z;
    z.M1 = law.L << (P + 1);
    z.M2 = law.L << (Q + 1);
    z.nfx = (1 << (P + 1)) + 1;
    z.nfy = (1 << (Q + 1)) + 1;
    z.N = (int64_t)z.M1 * z.M2;
    z.H = (int64_t)z.M2 * (z.M1 / 2 + 1);
    const size_t B = (size_t)law.batch;
    z.et = al256(16 * B);
    z.buf = al256(8 * B * (size_t)z.N);  // c (double), then the sample spectrum (float2)
    z.spec = al256(16 * B * (size_t)z.H);
    z.total = z.et + z.buf + z.spec;
    return z;
}

// cuFFT plans, created on first use for a (device, stream, M1, M2, batch,
// kind) and kept for the life of the library.  A plan owns its work area, so
// plans are not shared between streams: transforms on two streams never run
// in one work area at once, and on one stream they are ordered by the stream.
// The map and cufftSetStream + exec are guarded by one lock.
std::mutex g_plan_mu;
std::map<std::tuple<int, uintptr_t, int, int, int, int>, cufftHandle> g_plans;

int ce_plan(cudaStream_t st, int M1, int M2, int batch, bool d2z, cufftHandle* out)
{
    int dev = 0;
    cudaGetDevice(&dev);
    const auto key = std::make_tuple(dev, (uintptr_t)st, M1, M2, batch, d2z ? 1 : 0);
    auto it = g_plans.find(key);
    if (it != g_plans.end()) {
        *out = it->second;
        return MSG_OK;
    }
    cufftHandle h;
    if (cufftCreate(&h) != CUFFT_SUCCESS) {
        set_error("cufftCreate failed");
        return MSG_ERR_CUDA;
    }
    long long n[2] = {M2, M1};
    size_t work = 0;
    if (cufftMakePlanMany64(h, 2, n, nullptr, 1, 0, nullptr, 1, 0, d2z ? CUFFT_D2Z : CUFFT_C2C, batch, &work) !=
        CUFFT_SUCCESS) {
        cufftDestroy(h);
        set_error("cuFFT plan creation failed (" + std::to_string(M1) + " x " + std::to_string(M2) + ", batch " +
                  std::to_string(batch) + ")");
        return MSG_ERR_CUDA;
    }
    g_plans[key] = h;
    *out = h;
    return MSG_OK;
}

int ce_validate(int P, int Q, const msg_ce_law* law)
{
    if (!law) { set_error("law is NULL"); return MSG_ERR_INVALID; }
    if (P < 1 || Q < 1 || P > 10 || Q > 10) { set_error("P, Q must be in [1, 10]"); return MSG_ERR_INVALID; }
    if (law->nu != 0.5 && law->nu != 1.5 && law->nu != 2.5) {
        set_error("nu must be 0.5, 1.5 or 2.5");
        return MSG_ERR_INVALID;
    }
    if (!(law->lambda > 0) || !(law->eta_lo > 0) || !(law->eta_hi >= law->eta_lo) ||
        !(law->theta_hi >= law->theta_lo) || !std::isfinite(law->theta_lo) || !std::isfinite(law->theta_hi) ||
        !std::isfinite(law->eta_hi) || !std::isfinite(law->lambda)) {
        set_error("law: need lambda > 0, 0 < eta_lo <= eta_hi, theta_lo <= theta_hi, all finite");
        return MSG_ERR_INVALID;
    }
    // L >= 2: the periodic grid must hold every field node (2^(P+1) + 1 of them a row)
    if (law->scale != 0 && law->scale != 1) { set_error("law: scale must be 0 or 1"); return MSG_ERR_INVALID; }
    if (law->L < 2 || law->L > 64 || law->batch < 1) { set_error("law: need 2 <= L <= 64, batch >= 1"); return MSG_ERR_INVALID; }
    return MSG_OK;
}

}  // namespace
}  // namespace msg

using namespace msg;

extern "C" int32_t ce_padding(double nu, int32_t p0, int32_t q0)
{
    clear_error();
    if (!(nu > 0) || !std::isfinite(nu) || p0 < 0 || q0 < 0 || p0 > 30 || q0 > 30) {
        set_error("ce_padding: need nu > 0 and 0 <= p0, q0 <= 30");
        return 0;
    }
    // log2(max(2^p0, 2^q0)) = max(p0, q0)
    return 1 + 2 * (int32_t)std::ceil(std::sqrt(nu) * (double)std::max(p0, q0));
}

extern "C" size_t ce_workspace_bytes(int32_t P, int32_t Q, const msg_ce_law* law)
{
    clear_error();
    if (ce_validate(P, Q, law) != MSG_OK) return 0;
    return ce_sizes(P, Q, *law).total;
}

extern "C" int32_t ce_sample_field(int32_t P, int32_t Q, int64_t S, const msg_ce_law* law, uint64_t seed,
                                   uint64_t s0, double* Z, double* eta_theta, int32_t* status, void* workspace,
                                   size_t ws_bytes, void* stream)
{
    clear_error();
    int rc = ce_validate(P, Q, law);
    if (rc != MSG_OK) return rc;
    if (S < 0) { set_error("S < 0"); return MSG_ERR_INVALID; }
    if (S == 0) return MSG_OK;
    if (!Z || !workspace) { set_error("Z or workspace is NULL"); return MSG_ERR_INVALID; }
    if ((uintptr_t)workspace % 256) { set_error("workspace must be 256-byte aligned"); return MSG_ERR_INVALID; }
    const CeSizes z = ce_sizes(P, Q, *law);
    if (ws_bytes < z.total) {
        set_error("workspace too small: need " + std::to_string(z.total) + " bytes");
        return MSG_ERR_WORKSPACE;
    }
    cudaStream_t st = (cudaStream_t)stream;
    char* ws = (char*)workspace;
    double* et_ws = (double*)ws;
    double* c = (double*)(ws + z.et);                // generating arrays (FP64) ...
    float2* smp = (float2*)(ws + z.et);              // ... then, in the same bytes, the sample spectra
    double2* spec = (double2*)(ws + z.et + z.buf);   // eigenvalues (half spectra)
    const CeLawDev ld{law->nu, law->lambda, law->eta_lo, law->eta_hi, law->theta_lo, law->theta_hi, law->scale};
    const double hx = std::ldexp(1.0, -(P + 1)), hy = std::ldexp(1.0, -(Q + 1));
    const int64_t nf = (int64_t)z.nfx * z.nfy;
    if (status) MSG_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(int32_t) * S, st));
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms < 1) sms = 1;
    for (int64_t b0 = 0; b0 < S; b0 += law->batch) {
        const int nb = (int)std::min<int64_t>(law->batch, S - b0);
        double* et = eta_theta ? eta_theta + 2 * b0 : et_ws;
        // blocks per sample: enough to fill the GPU about four times over per batch
        const unsigned gx = (unsigned)std::max<int64_t>(1, std::min<int64_t>((z.N + 255) / 256, 4LL * sms * 8 / nb + 1));
        prof_begin(K_CE, st);
        k_ce_hyper<<<(nb + 127) / 128, 128, 0, st>>>(seed, s0 + (uint64_t)b0, nb, ld, et);
        prof_end(K_CE, st, 16.0 * nb, 0.0);
        MSG_CHECK_LAUNCH();
        prof_begin(K_CE, st);
        k_ce_cov<<<dim3(gx, nb), 256, 0, st>>>(z.M1, z.M2, hx, hy, ld, et, c);
        prof_end(K_CE, st, 8.0 * z.N * nb, 20.0 * z.N * nb);
        MSG_CHECK_LAUNCH();
        {
            std::lock_guard<std::mutex> lk(g_plan_mu);
            cufftHandle pd, pc;
            if ((rc = ce_plan(st, z.M1, z.M2, nb, true, &pd)) != MSG_OK) return rc;
            if ((rc = ce_plan(st, z.M1, z.M2, nb, false, &pc)) != MSG_OK) return rc;
            if (cufftSetStream(pd, st) != CUFFT_SUCCESS ||
                cufftExecD2Z(pd, (cufftDoubleReal*)c, (cufftDoubleComplex*)spec) != CUFFT_SUCCESS) {
                set_error("cuFFT D2Z failed");
                return MSG_ERR_CUDA;
            }
            prof_begin(K_CE, st);
            k_ce_scale<<<dim3(gx, nb), 256, 0, st>>>(z.M1, z.M2, seed, s0 + (uint64_t)b0, spec, smp,
                                                     status ? status + b0 : nullptr);
            prof_end(K_CE, st, (16.0 * z.H + 8.0 * z.N) * nb, 30.0 * z.N * nb);
            MSG_CHECK_LAUNCH();
            if (cufftSetStream(pc, st) != CUFFT_SUCCESS ||
                cufftExecC2C(pc, (cufftComplex*)smp, (cufftComplex*)smp, CUFFT_FORWARD) !=
                    CUFFT_SUCCESS) {
                set_error("cuFFT C2C failed");
                return MSG_ERR_CUDA;
            }
        }
        prof_begin(K_CE, st);
        const unsigned gxe = (unsigned)std::max<int64_t>(1, std::min<int64_t>((nf + 255) / 256, 4LL * sms * 8 / nb + 1));
        k_ce_extract<<<dim3(gxe, nb), 256, 0, st>>>(z.M1, z.nfx, z.nfy, z.N, smp, Z + b0 * nf);
        prof_end(K_CE, st, 16.0 * nf * nb, 0.0);
        MSG_CHECK_LAUNCH();
    }
    return MSG_OK;
}
