// mimc.cu -- multi-index differences (Sec. 3, Eq. (3.2)) and the per-sample
// estimator term Y (Eq. (3.6)).  Index arithmetic is integer; the differences
// are formed in the order D_1 then D_2 of the worked example of Sec. 3.
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "prof.cuh"

namespace msg {

struct MimcSample {
    int L1, L2;
    int64_t q_off;   // start of the sample's QoIs (finest grid (p0+L1, q0+L2))
    int64_t d_off;   // start of the sample's (L1+1)(L2+1) differences
};

__global__ void k_mimc(const MimcSample* smp, int64_t S, int p0, int q0, const double* Q, const double* ptau, int ld2,
                       double* dQ, double* Y)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < S; i += (int64_t)gridDim.x * blockDim.x) {
        const MimcSample m = smp[i];
        const int Qn = q0 + m.L2;  // columns of the sample's QoI block
        const double* Qs = Q + m.q_off;
        double y = 0.0;
        for (int t1 = 0; t1 <= m.L1; ++t1)
            for (int t2 = 0; t2 <= m.L2; ++t2) {
                double d1 = Qs[(p0 + t1 - 1) * Qn + (q0 + t2 - 1)];
                if (t1 > 0) d1 -= Qs[(p0 + t1 - 2) * Qn + (q0 + t2 - 1)];
                double d = d1;
                if (t2 > 0) {
                    double d1m = Qs[(p0 + t1 - 1) * Qn + (q0 + t2 - 2)];
                    if (t1 > 0) d1m -= Qs[(p0 + t1 - 2) * Qn + (q0 + t2 - 2)];
                    d = d1 - d1m;
                }
                dQ[m.d_off + t1 * (m.L2 + 1) + t2] = d;
                if (ptau) y += d / ptau[t1 * ld2 + t2];
            }
        if (Y) Y[i] = ptau ? y : 0.0;
    }
}

}  // namespace msg

using namespace msg;

extern "C" int32_t mimc_differences(const int32_t* L, int64_t S, int32_t p0, int32_t q0, const double* Q,
                                    const double* ptau, int32_t ld1, int32_t ld2, double* dQ, double* Y, void* stream)
{
    clear_error();
    if (S < 0 || p0 < 1 || q0 < 1) { set_error("mimc_differences: need S >= 0, p0 >= 1, q0 >= 1"); return MSG_ERR_INVALID; }
    if (S == 0) return MSG_OK;
    if (!L || !Q || !dQ) { set_error("mimc_differences: NULL pointer"); return MSG_ERR_INVALID; }
    int maxL1 = 0, maxL2 = 0;
    for (int64_t i = 0; i < S; ++i) {
        int l1 = L[2 * i], l2 = L[2 * i + 1];
        if (l1 < 0 || l2 < 0 || p0 + l1 > 12 || q0 + l2 > 12) {
            set_error("mimc_differences: multi-index out of range");
            return MSG_ERR_INVALID;
        }
        maxL1 = l1 > maxL1 ? l1 : maxL1;
        maxL2 = l2 > maxL2 ? l2 : maxL2;
    }
    if (ptau && (ld1 <= maxL1 || ld2 <= maxL2)) {
        set_error("mimc_differences: ptau table smaller than the largest multi-index");
        return MSG_ERR_INVALID;
    }
    cudaStream_t st = (cudaStream_t)stream;
    // the tables are built in pinned staging (released by an event once copied) and
    // uploaded into a stream-ordered temporary: the call does not wait for the stream
    const size_t tb = sizeof(MimcSample) * S, tb_al = (tb + 255) / 256 * 256;
    const size_t pb = ptau ? sizeof(double) * ld1 * ld2 : 0;
    void* hp = nullptr;
    int token = -1;
    int rc = staging_acquire(tb_al + pb, &hp, &token);
    if (rc != MSG_OK) return rc;
    MimcSample* h = (MimcSample*)hp;
    int64_t qo = 0, dof = 0;
    for (int64_t i = 0; i < S; ++i) {
        const int l1 = L[2 * i], l2 = L[2 * i + 1];
        h[i] = MimcSample{l1, l2, qo, dof};
        qo += (int64_t)(p0 + l1) * (q0 + l2);
        dof += (int64_t)(l1 + 1) * (l2 + 1);
    }
    if (ptau) memcpy((char*)hp + tb_al, ptau, pb);
    char* dbuf = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&dbuf, tb_al + pb + 256, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dbuf, hp, tb_al + pb, cudaMemcpyHostToDevice, st);
    const int rel = staging_release(token, st);
    if (e != cudaSuccess) {
        set_error(std::string("mimc_differences: ") + cudaGetErrorString(e));
        return MSG_ERR_CUDA;
    }
    if (rel != MSG_OK) return rel;
    const double* dp = ptau ? (const double*)(dbuf + tb_al) : nullptr;
    int blocks = (int)std::min<int64_t>((S + 255) / 256, 152 * 8);
    prof_begin(K_MIMC, st);
    k_mimc<<<blocks, 256, 0, st>>>((const MimcSample*)dbuf, S, p0, q0, Q, dp, ld2, dQ, Y);
    prof_end(K_MIMC, st, 8.0 * (qo + 2.0 * dof) + tb, 0.0);
    MSG_CHECK_LAUNCH();
    MSG_CUDA_TRY(cudaFreeAsync(dbuf, st));
    return MSG_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free variant of mimc_differences.
//
// For callers that may not allocate device memory once they are running (a
// program whose device memory is all reserved by its own pool, or a loop that
// cannot afford an allocator call), the per-sample offset table and the p_tau
// table go to a fixed array in the library's own device memory instead of a
// temporary from cudaMallocAsync.  The array is a file-scope __device__
// symbol: every GPU that loads the library holds it until the process exits.
// In host code its name is only a host-side stand-in, so the device address
// is looked up with cudaGetSymbolAddress once per device (on the first call
// made with that device current) and cached.  The cache is not invalidated by
// cudaDeviceReset: after a reset of a device in this process the entry point
// must not be called on that device again.
// ---------------------------------------------------------------------------
namespace msg {
namespace {

constexpr size_t kNoAllocBytes = size_t(16) << 20;  // 16 MiB per device
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// host staging of the same size: filled and copied under the lock, so the
// entry point needs no host or device allocation either
alignas(256) unsigned char g_noalloc_host[kNoAllocBytes];
std::mutex g_noalloc_mu;
constexpr int kMaxDevices = 64;
void* g_noalloc_dev[kMaxDevices] = {};

int noalloc_scratch(void** out)
{
    int dev = -1;
    MSG_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("mimc_differences_noalloc: device ordinal out of range");
        return MSG_ERR_UNSUPPORTED;
    }
    if (!g_noalloc_dev[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            set_error(std::string("mimc_differences_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
            return MSG_ERR_CUDA;
        }
        g_noalloc_dev[dev] = p;
    }
    *out = g_noalloc_dev[dev];
    return MSG_OK;
}

}  // namespace
}  // namespace msg

extern "C" int32_t mimc_differences_noalloc(const int32_t* L, int64_t S, int32_t p0, int32_t q0, const double* Q,
                                            const double* ptau, int32_t ld1, int32_t ld2, double* dQ, double* Y,
                                            void* stream)
{
    clear_error();
    if (S < 0 || p0 < 1 || q0 < 1) {
        set_error("mimc_differences_noalloc: need S >= 0, p0 >= 1, q0 >= 1");
        return MSG_ERR_INVALID;
    }
    if (S == 0) return MSG_OK;
    if (!L || !Q || !dQ) { set_error("mimc_differences_noalloc: NULL pointer"); return MSG_ERR_INVALID; }
    const size_t tb = sizeof(MimcSample) * (size_t)S;
    const size_t tb_al = (tb + 255) / 256 * 256;
    const size_t pb = ptau ? sizeof(double) * (size_t)std::max(ld1, 0) * (size_t)std::max(ld2, 0) : 0;
    if (pb >= kNoAllocBytes) {
        set_error("mimc_differences_noalloc: the ptau table alone (" + std::to_string(pb) +
                  " bytes) does not fit the fixed " + std::to_string(kNoAllocBytes) + "-byte scratch");
        return MSG_ERR_INVALID;
    }
    if (tb_al + pb > kNoAllocBytes) {
        set_error("mimc_differences_noalloc: batch needs " + std::to_string(tb_al + pb) +
                  " bytes of scratch, more than the fixed " + std::to_string(kNoAllocBytes) +
                  " (with this ptau table at most " +
                  std::to_string((kNoAllocBytes - pb) / 256 * 256 / sizeof(MimcSample)) + " samples per call)");
        return MSG_ERR_INVALID;
    }
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    MimcSample* h = (MimcSample*)g_noalloc_host;
    int64_t qo = 0, dof = 0;
    int maxL1 = 0, maxL2 = 0;
    for (int64_t i = 0; i < S; ++i) {
        int l1 = L[2 * i], l2 = L[2 * i + 1];
        if (l1 < 0 || l2 < 0 || p0 + l1 > 12 || q0 + l2 > 12) {
            set_error("mimc_differences_noalloc: multi-index out of range");
            return MSG_ERR_INVALID;
        }
        h[i] = MimcSample{l1, l2, qo, dof};
        qo += (int64_t)(p0 + l1) * (q0 + l2);
        dof += (int64_t)(l1 + 1) * (l2 + 1);
        maxL1 = l1 > maxL1 ? l1 : maxL1;
        maxL2 = l2 > maxL2 ? l2 : maxL2;
    }
    if (ptau && (ld1 <= maxL1 || ld2 <= maxL2)) {
        set_error("mimc_differences_noalloc: ptau table smaller than the largest multi-index");
        return MSG_ERR_INVALID;
    }
    if (ptau) memcpy(g_noalloc_host + tb_al, ptau, pb);
    void* dbase = nullptr;
    int rc = noalloc_scratch(&dbase);
    if (rc != MSG_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    char* d = (char*)dbase;
    MSG_CUDA_TRY(cudaMemcpyAsync(d, g_noalloc_host, tb_al + pb, cudaMemcpyHostToDevice, st));
    const double* dp = ptau ? (const double*)(d + tb_al) : nullptr;
    int blocks = (int)std::min<int64_t>((S + 255) / 256, 152 * 8);
    prof_begin(K_MIMC, st);
    k_mimc<<<blocks, 256, 0, st>>>((const MimcSample*)d, S, p0, q0, Q, dp, ld2, dQ, Y);
    prof_end(K_MIMC, st, 8.0 * (qo + 2.0 * dof) + tb, 0.0);
    MSG_CHECK_LAUNCH();
    // the host staging and the device array are reused by the next call
    MSG_CUDA_TRY(cudaStreamSynchronize(st));
    return MSG_OK;
}
