// kl_tc.cu -- KL contraction Z = Phi diag(sqrt(lambda)) xi on the 5th-generation
// tensor cores (tcgen05) with FP32 accumulation, in two operand modes:
//   BF16X3  each operand v is split into bf16 parts v = hi + lo + O(2^-16 |v|) and
//           the product uses hi*hi + hi*lo + lo*hi (kind::f16), about 1e-5 of
//           sum_m |A B| -- the lo*lo term and the remainders are below the FP32
//           accumulation of a 400-term sum of unit-scale products;
//   TF32    both operands rounded to TF32 (10-bit mantissa, round to nearest) and
//           one product per term (kind::tf32), about 1e-3 of sum_m |A B|.
// Neither is the FP64 path; the sampler's error is stated per result in the tests
// and the bench.
//
// Z[s][x] = sum_m A[s][m] B[x][m] with A = sqrt(lambda) * xi (samples x terms)
// and B = Phi (points x terms).  One CTA computes a 128 (samples) x 256 (points)
// tile of Z: accumulators in 256 TMEM columns, K in 128-byte chunks (64 bf16 or
// 32 TF32 terms) staged through shared memory in the 128-byte-swizzled K-major
// layout the UMMA descriptors expect.  A is converted from FP64
// xi and sqrt(lambda) once per call into a stream-ordered temporary; B is
// converted once per basis by kl_tc_prepare; both are zero-padded [rows][Kp] part
// arrays whose tiles arrive by 16-byte asynchronous copies (cp.async) through a
// ring of stages (2 for BF16X3, 4 for TF32) filled ahead of the MMAs that read
// them.  One elected thread issues the
// MMAs and commits them to an mbarrier per stage; every wait is bounded and a
// timeout sets a device flag (read by msg_device_status) instead of hanging.  The
// epilogue moves each warp's 32 x 32 accumulator blocks through shared memory so
// that every global store of a warp writes 32 consecutive points of one sample.
#include <cuda_bf16.h>

#include "common.cuh"
#include "kl_tc.cuh"
#include "prof.cuh"

namespace msg {

namespace {

constexpr int kTM = 128;  // samples per tile (UMMA M)
constexpr int kTN = 256;  // points per tile (UMMA N)
constexpr int kThreadsTC = 256;
constexpr int kRowBytes = 128;                        // one swizzled K row
constexpr int kAbytes = kTM * kRowBytes;              // 16 KB per A part and stage
constexpr int kBbytes = kTN * kRowBytes;              // 32 KB per B part and stage
constexpr long long kSpinLimit = 1ll << 22;           // bounded mbarrier waits (seconds)

// Operand modes of the tensor-core kernel.
enum { TC_BF16X3 = 0, TC_TF32 = 1 };
template <int MODE> struct TcCfg;
template <> struct TcCfg<TC_BF16X3> {
    typedef __nv_bfloat16 E;
    static constexpr int parts = 2;   // hi, lo
    static constexpr int TK = 64;     // terms per 128-byte row
    static constexpr int stages = 2;  // 96 KB each
};
template <> struct TcCfg<TC_TF32> {
    typedef float E;
    static constexpr int parts = 1;
    static constexpr int TK = 32;
    static constexpr int stages = 4;  // 48 KB each
};
template <int MODE> constexpr int stage_bytes() { return TcCfg<MODE>::parts * (kAbytes + kBbytes); }
template <int MODE> constexpr int smem_bytes() { return TcCfg<MODE>::stages * stage_bytes<MODE>() + 1024; }  // + alignment slack

__host__ __device__ inline int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

__device__ int g_tc_error;  // set by a kernel whose mbarrier wait ran out (sticky until msg_device_status)

// Byte offset of 16-byte chunk `chunk` (0..7) of row r in a K-major tile with the
// 128-byte swizzle: 8-row atoms of 1024 bytes, chunk c of row rr stored at
// chunk position c ^ rr.
__device__ __forceinline__ uint32_t sw128(int r, int chunk) { return (r >> 3) * 1024 + (r & 7) * 128 + ((chunk ^ (r & 7)) << 4); }

// tcgen05 shared-memory matrix descriptor: start address >> 4 in bits 0-13,
// leading byte offset >> 4 in 16-29 (unused by swizzled K-major tiles),
// stride byte offset >> 4 in 32-45 (1024: next 8-row atom), descriptor
// version 1 in bits 46-47, swizzle mode 2 (128-byte) in bits 61-63.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr)
{
    return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)(16 >> 4) << 16) | ((uint64_t)(1024 >> 4) << 32) |
           (1ull << 46) | (2ull << 61);
}

// Instruction descriptor: D = F32 (bits 4-5 = 1); A and B formats in bits 7-9
// and 10-12 (kind::f16: 1 = BF16; kind::tf32: 2 = TF32), both K-major;
// N >> 3 in bits 17-22, M >> 4 in bits 24-28.
template <int MODE>
__host__ __device__ constexpr uint32_t instr_desc()
{
    return (1u << 4) | ((MODE == TC_TF32 ? 2u : 1u) << 7) | ((MODE == TC_TF32 ? 2u : 1u) << 10) |
           ((uint32_t)(kTN >> 3) << 17) | ((uint32_t)(kTM >> 4) << 24);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Wait until the mbarrier phase with the given parity has completed; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity)
{
    const uint32_t a = smem_u32(bar);
    for (long long it = 0; it < kSpinLimit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

template <int MODE>
__device__ __forceinline__ void mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t acc)
{
    if constexpr (MODE == TC_TF32)
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
            ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(instr_desc<MODE>()), "r"(acc)
            : "memory");
    else
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
            ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(instr_desc<MODE>()), "r"(acc)
            : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// 32 consecutive FP32 accumulator columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v)
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int k = 0; k < 32; ++k) v[k] = __uint_as_float(r[k]);
}

// Split of FP64 values into bf16 hi/lo.
__device__ __forceinline__ void split2(double v, __nv_bfloat16& hi, __nv_bfloat16& lo)
{
    hi = __double2bfloat16(v);
    lo = __double2bfloat16(v - (double)__bfloat162float(hi));
}

// FP64 -> TF32 (round to nearest, ties away), kept in an FP32 container.
__device__ __forceinline__ float to_tf32(double v)
{
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"((float)v));
    return __uint_as_float(r);
}

// Operand conversion of 8 consecutive terms into the parts of one 16-byte chunk
// (BF16X3: 8 terms -> 16 bytes per part; TF32: 4 terms -> 16 bytes).
__global__ void k_split_phi(const double* Phi, int64_t npts, int M, int64_t Kp, int64_t Np, __nv_bfloat16* Bhi,
                            __nv_bfloat16* Blo)
{
    const int64_t n = Np * Kp;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t x = e / Kp, m = e % Kp;
        double v = (x < npts && m < M) ? Phi[x * M + m] : 0.0;
        __nv_bfloat16 h, l;
        split2(v, h, l);
        Bhi[e] = h;
        Blo[e] = l;
    }
}

__global__ void k_tf32_phi(const double* Phi, int64_t npts, int M, int64_t Kp, int64_t Np, float* B)
{
    const int64_t n = Np * Kp;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t x = e / Kp, m = e % Kp;
        B[e] = (x < npts && m < M) ? to_tf32(Phi[x * M + m]) : 0.f;
    }
}

// A = sqrt(lambda) * xi converted once per call into zero-padded [Sp][Kp] part
// arrays in the operand format (the main loop then only copies).
template <int MODE>
__global__ void k_prep_a(const double* sl, const double* xi, int64_t S, int M, int64_t Kp, int64_t Sp,
                         typename TcCfg<MODE>::E* A0, typename TcCfg<MODE>::E* A1)
{
    const int64_t n = Sp * Kp;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = e / Kp, m = e % Kp;
        const double v = (s < S && m < M) ? sl[m] * xi[s * M + m] : 0.0;
        if constexpr (MODE == TC_TF32) {
            A0[e] = to_tf32(v);
        } else {
            __nv_bfloat16 h, l;
            split2(v, h, l);
            A0[e] = h;
            A1[e] = l;
        }
    }
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}

template <int MODE, class TZ>
__global__ void __launch_bounds__(kThreadsTC, 1)
    k_kl_tc(const typename TcCfg<MODE>::E* __restrict__ A0, const typename TcCfg<MODE>::E* __restrict__ A1,
            const typename TcCfg<MODE>::E* __restrict__ B0, const typename TcCfg<MODE>::E* __restrict__ B1,
            int64_t npts, int64_t Kp, int64_t S, TZ* __restrict__ Z)
{
    typedef typename TcCfg<MODE>::E E;
    constexpr int parts = TcCfg<MODE>::parts, TK = TcCfg<MODE>::TK, NST = TcCfg<MODE>::stages;
    constexpr int EPC = 16 / (int)sizeof(E);  // terms per 16-byte chunk
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t bars[NST];
    __shared__ uint32_t tmem_base_slot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // 1024-aligned stage buffers (swizzle atoms must start on 1024 bytes)
    const uint32_t raw = smem_u32(smem_raw);
    unsigned char* base = smem_raw + (((raw + 1023) & ~1023u) - raw);
    // blockIdx.x runs over the sample tiles: the CTAs that read one Phi tile are
    // launched next to each other and find it in L2 (A is small and stays there)
    const int64_t s0 = (int64_t)blockIdx.x * kTM, x0 = (int64_t)blockIdx.y * kTN;

    if (warp == 0) {  // TMEM: 128 lanes x 256 FP32 columns
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_slot)),
                     "r"(kTN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int k = 0; k < NST; ++k) mbar_init(&bars[k], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base_slot;

    const int nchunks = (int)(Kp / TK);
    // one chunk of A (128 rows) and B (256 rows) into its stage by 16-byte asynchronous copies
    auto load_chunk = [&](int kc) {
        unsigned char* sA = base + (kc % NST) * stage_bytes<MODE>();  // A parts, then B parts
        unsigned char* sB = sA + parts * kAbytes;
        for (int t = tid; t < kTM * 8; t += kThreadsTC) {
            const int r = t >> 3, c = t & 7;
            const int64_t g = (s0 + r) * Kp + (int64_t)kc * TK + c * EPC;
            const uint32_t off = sw128(r, c);
            cp_async16(smem_u32(sA + off), A0 + g);
            if constexpr (parts == 2) cp_async16(smem_u32(sA + kAbytes + off), A1 + g);
        }
        for (int t = tid; t < kTN * 8; t += kThreadsTC) {
            const int r = t >> 3, c = t & 7;
            const int64_t g = (x0 + r) * Kp + (int64_t)kc * TK + c * EPC;
            const uint32_t off = sw128(r, c);
            cp_async16(smem_u32(sB + off), B0 + g);
            if constexpr (parts == 2) cp_async16(smem_u32(sB + kBbytes + off), B1 + g);
        }
    };
    // prologue: the first NST-1 chunks in flight (one commit group per chunk, empty past the end)
    for (int kc = 0; kc < NST - 1; ++kc) {
        if (kc < nchunks) load_chunk(kc);
        asm volatile("cp.async.commit_group;" ::: "memory");
    }
    bool ok = true;
    for (int kc = 0; kc < nchunks; ++kc) {
        // chunk kc has landed once at most NST-2 newer groups are pending
        asm volatile("cp.async.wait_group %0;" ::"n"(NST - 2) : "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // make the copies visible to the tensor cores
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a0 = smem_u32(base + (kc % NST) * stage_bytes<MODE>());
            const uint32_t b0 = a0 + parts * kAbytes;
#pragma unroll
            for (int ks = 0; ks < 4; ++ks) {  // 4 MMA K steps of 32 bytes per 128-byte row
                const uint32_t ko = ks * 32;
                const uint32_t first = (kc == 0 && ks == 0) ? 0u : 1u;
                mma<MODE>(tmem, smem_desc(a0 + ko), smem_desc(b0 + ko), first);
                if constexpr (MODE == TC_BF16X3) {
                    mma<MODE>(tmem, smem_desc(a0 + ko), smem_desc(b0 + kBbytes + ko), 1u);  // hi * lo
                    mma<MODE>(tmem, smem_desc(a0 + kAbytes + ko), smem_desc(b0 + ko), 1u);  // lo * hi
                }
            }
            mma_commit(&bars[kc % NST]);
        }
        // refill: chunk kc+NST-1 goes into the stage chunk kc-1 used, once its MMAs are done
        const int nk = kc + NST - 1;
        if (nk < nchunks) {
            if (kc >= 1) ok &= mbar_wait(&bars[(kc - 1) % NST], ((kc - 1) / NST) & 1);
            load_chunk(nk);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    }
    // the last commit completes after every MMA of the CTA
    if (nchunks >= 1) ok &= mbar_wait(&bars[(nchunks - 1) % NST], ((nchunks - 1) / NST) & 1);
    asm volatile("cp.async.wait_all;" ::: "memory");
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // every thread took part in the same waits; make the decision CTA-wide
    const int all_ok = __syncthreads_and(ok ? 1 : 0);
    if (!all_ok) {
        if (tid == 0) atomicExch(&g_tc_error, 1);
    } else {
        // epilogue: warp w reads TMEM lanes 32 (w % 4) .. +31 (samples), columns 128 (w / 4) .. +127
        // (points); each 32 x 32 block goes through a padded shared tile so that the stores of a
        // warp cover 32 consecutive points of one sample
        const int lane_base = 32 * (warp & 3), col_base = 128 * (warp >> 2);
        float* tile = reinterpret_cast<float*>(base) + warp * 32 * 33;  // the stages are free now
        for (int cb = 0; cb < 128; cb += 32) {
            float v[32];
            tmem_ld32(tmem + ((uint32_t)lane_base << 16) + (uint32_t)(col_base + cb), v);
#pragma unroll
            for (int k = 0; k < 32; ++k) tile[lane * 33 + k] = v[k];
            __syncwarp();
            const int64_t x = x0 + col_base + cb + lane;
            for (int rr = 0; rr < 32; ++rr) {
                const int64_t s = s0 + lane_base + rr;
                if (s < S && x < npts) Z[s * npts + x] = (TZ)tile[rr * 33 + lane];
            }
            __syncwarp();
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTN) : "memory");
}

struct TcLayout {
    int64_t Kp, Np;
    size_t p0, p1, sl, total;
};

TcLayout tc_layout(int64_t npts, int32_t M, int mode)
{
    TcLayout L{};
    const bool tf = mode == TC_TF32;
    L.Kp = round_up(M, tf ? TcCfg<TC_TF32>::TK : TcCfg<TC_BF16X3>::TK);
    L.Np = round_up(npts, kTN);
    const size_t part = (size_t)L.Np * L.Kp * (tf ? sizeof(float) : sizeof(__nv_bfloat16));
    L.p0 = 0;
    L.p1 = (part + 255) / 256 * 256;
    L.sl = tf ? L.p1 : 2 * L.p1;
    L.total = L.sl + ((sizeof(double) * M + 255) / 256 * 256);
    return L;
}

int tc_mode(int32_t gemm_mode) { return gemm_mode == MSG_GEMM_TF32 ? TC_TF32 : TC_BF16X3; }

template <int MODE, class TZ>
int tc_launch(const TcLayout& L, const char* b, int64_t npts, int32_t M, const double* xi, int64_t S, void* Z,
              cudaStream_t st)
{
    typedef typename TcCfg<MODE>::E E;
    constexpr int parts = TcCfg<MODE>::parts;
    const int64_t Sp = round_up(S, kTM);
    const size_t apart = (size_t)Sp * L.Kp * sizeof(E), apart_al = (apart + 255) / 256 * 256;
    // the converted A lives in a stream-ordered temporary, freed after the contraction
    char* abuf = nullptr;
    MSG_CUDA_TRY(cudaMallocAsync((void**)&abuf, parts * apart_al, st));
    E* A0 = (E*)abuf;
    E* A1 = parts == 2 ? (E*)(abuf + apart_al) : nullptr;
    k_prep_a<MODE><<<152 * 4, 256, 0, st>>>((const double*)(b + L.sl), xi, S, M, L.Kp, Sp, A0, A1);
    MSG_CHECK_LAUNCH();
    dim3 grid((unsigned)(Sp / kTM), (unsigned)(L.Np / kTN));
    MSG_CUDA_TRY(cudaFuncSetAttribute(k_kl_tc<MODE, TZ>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes<MODE>()));
    k_kl_tc<MODE, TZ><<<grid, kThreadsTC, smem_bytes<MODE>(), st>>>(A0, A1 ? A1 : A0, (const E*)(b + L.p0),
                                                                     (const E*)(b + (parts == 2 ? L.p1 : L.p0)), npts,
                                                                     L.Kp, S, (TZ*)Z);
    MSG_CHECK_LAUNCH();
    MSG_CUDA_TRY(cudaFreeAsync(abuf, st));
    return MSG_OK;
}

}  // namespace

size_t kl_tc_prepared_bytes(int64_t npts, int32_t M, int32_t mode) { return tc_layout(npts, M, tc_mode(mode)).total; }

int32_t kl_tc_prepare(const double* Phi, const double* sqrt_lambda, int64_t npts, int32_t M, int32_t mode,
                      void* prepared, cudaStream_t st)
{
    const int tm = tc_mode(mode);
    const TcLayout L = tc_layout(npts, M, tm);
    char* b = (char*)prepared;
    prof_begin(K_KL, st);
    if (tm == TC_TF32)
        k_tf32_phi<<<152 * 8, 256, 0, st>>>(Phi, npts, M, L.Kp, L.Np, (float*)(b + L.p0));
    else
        k_split_phi<<<152 * 8, 256, 0, st>>>(Phi, npts, M, L.Kp, L.Np, (__nv_bfloat16*)(b + L.p0),
                                              (__nv_bfloat16*)(b + L.p1));
    prof_end(K_KL, st, 8.0 * npts * M + 4.0 * L.Np * L.Kp, 0.0);
    MSG_CHECK_LAUNCH();
    MSG_CUDA_TRY(cudaMemcpyAsync(b + L.sl, sqrt_lambda, sizeof(double) * M, cudaMemcpyDeviceToDevice, st));
    return MSG_OK;
}

int32_t kl_tc_sample(const void* prepared, int64_t npts, int32_t M, int32_t mode, const double* xi, int64_t S, void* Z,
                     int32_t z_fp32, cudaStream_t st)
{
    const int tm = tc_mode(mode);
    const TcLayout L = tc_layout(npts, M, tm);
    if ((npts + kTN - 1) / kTN > 65535) { set_error("sample_field: too many points for one call"); return MSG_ERR_INVALID; }
    const char* b = (const char*)prepared;
    prof_begin(K_KL, st);
    int rc;
    if (tm == TC_TF32)
        rc = z_fp32 ? tc_launch<TC_TF32, float>(L, b, npts, M, xi, S, Z, st) : tc_launch<TC_TF32, double>(L, b, npts, M, xi, S, Z, st);
    else
        rc = z_fp32 ? tc_launch<TC_BF16X3, float>(L, b, npts, M, xi, S, Z, st)
                    : tc_launch<TC_BF16X3, double>(L, b, npts, M, xi, S, Z, st);
    if (rc != MSG_OK) return rc;
    // algorithmic work: (3 split products or 1) of 2 npts M S flops; bytes: Phi parts, xi, Z
    const double parts = tm == TC_TF32 ? 1.0 : 3.0, pbytes = tm == TC_TF32 ? 4.0 : 4.0;
    prof_end(K_KL, st, pbytes * npts * M + 8.0 * S * M + (z_fp32 ? 4.0 : 8.0) * S * npts, 2.0 * parts * npts * M * S);
    MSG_CHECK_LAUNCH();
    // a bounded wait that runs out sets g_tc_error (reported by msg_device_status)
    return MSG_OK;
}

}  // namespace msg

extern "C" int32_t msg_device_status(void)
{
    msg::clear_error();
    MSG_CUDA_TRY(cudaDeviceSynchronize());
    int err = 0, zero = 0;
    MSG_CUDA_TRY(cudaMemcpyFromSymbol(&err, msg::g_tc_error, sizeof(int)));
    MSG_CUDA_TRY(cudaMemcpyToSymbol(msg::g_tc_error, &zero, sizeof(int)));
    if (err) {
        msg::set_error("a bounded wait in a tensor-core kernel ran out; its output was not written");
        return MSG_ERR_TIMEOUT;
    }
    return MSG_OK;
}
