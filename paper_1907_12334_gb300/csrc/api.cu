// api.cu -- error state, version, launch counting and profiling of the C ABI.
#include <algorithm>
#include <atomic>
#include <cstdint>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "prof.cuh"

namespace msg {
namespace {
thread_local std::string g_last_error;
std::atomic<int64_t> g_launches{0};

struct Rec {
    cudaEvent_t a, b;
    int cls, level;
    double bytes, flops;
};
struct Prof {
    std::mutex mu;
    std::atomic<int> stride{0};              // 0: off; n: time a random 1/n of each class's launches
    std::atomic<int64_t> count[K_NCLASS];    // launches of each class since enable
    Prof() { for (auto& c : count) c = 0; }
    std::vector<cudaEvent_t> pool;
    size_t next = 0;
    std::vector<Rec> recs;
    cudaEvent_t take()
    {
        if (next == pool.size()) {
            cudaEvent_t e;
            cudaEventCreate(&e);
            pool.push_back(e);
        }
        return pool[next++];
    }
} g_prof;
thread_local cudaEvent_t t_pending_start[K_NCLASS];  // begin events of this thread's open launches
thread_local bool t_pending_timed[K_NCLASS];
thread_local uint64_t t_rng = 0;  // xorshift64 state of this thread's sampling decisions

// true with probability 1/n (n >= 1)
bool sample_one_in(int n)
{
    if (n <= 1) return true;
    if (t_rng == 0) t_rng = 0x9E3779B97F4A7C15ull ^ (uint64_t)(uintptr_t)&t_rng;
    t_rng ^= t_rng << 13;
    t_rng ^= t_rng >> 7;
    t_rng ^= t_rng << 17;
    return t_rng % (uint64_t)n == 0;
}
}  // namespace

namespace {
struct StagingSlot {
    void* p = nullptr;
    size_t bytes = 0;
    cudaEvent_t ev = nullptr;
    int dev = -1;
    bool pending = false;  // an event was recorded and may not have completed
    bool held = false;     // handed out, not yet released
};
std::mutex g_staging_mu;
std::vector<StagingSlot> g_staging;
}  // namespace

int staging_acquire(size_t bytes, void** ptr, int* token)
{
    int dev = 0;
    MSG_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_staging_mu);
    for (size_t k = 0; k < g_staging.size(); ++k) {
        StagingSlot& s = g_staging[k];
        if (s.held || s.bytes < bytes) continue;
        if (s.pending) {
            if (cudaEventQuery(s.ev) != cudaSuccess) continue;  // still being read by an earlier copy
            s.pending = false;
        }
        s.held = true;
        *ptr = s.p;
        *token = (int)k;
        return MSG_OK;
    }
    StagingSlot s;
    s.bytes = std::max<size_t>(bytes, 4096);
    MSG_CUDA_TRY(cudaHostAlloc(&s.p, s.bytes, cudaHostAllocPortable));
    s.held = true;
    g_staging.push_back(s);
    *ptr = s.p;
    *token = (int)g_staging.size() - 1;
    return MSG_OK;
}

int staging_release(int token, cudaStream_t st)
{
    int dev = 0;
    MSG_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_staging_mu);
    StagingSlot& s = g_staging[token];
    if (s.ev && s.dev != dev) {  // events belong to a device
        cudaEventDestroy(s.ev);
        s.ev = nullptr;
    }
    if (!s.ev) {
        MSG_CUDA_TRY(cudaEventCreateWithFlags(&s.ev, cudaEventDisableTiming));
        s.dev = dev;
    }
    MSG_CUDA_TRY(cudaEventRecord(s.ev, st));
    s.pending = true;
    s.held = false;
    return MSG_OK;
}

void set_error(const std::string& what) { g_last_error = what; }
void clear_error() { g_last_error.clear(); }

void prof_begin(int cls, cudaStream_t st)
{
    t_pending_timed[cls] = false;
    const int n = g_prof.stride.load(std::memory_order_relaxed);
    if (n <= 0) return;
    g_prof.count[cls].fetch_add(1, std::memory_order_relaxed);
    // the cycle's classes launch thousands of times per solve and are sampled;
    // the once-per-step or per-stage classes are always timed
    const bool cycle_class = cls == K_PRE || cls == K_POST || cls == K_LOW || cls == K_RESIDUAL || cls == K_UPDATE;
    if (cycle_class && !sample_one_in(n)) return;
    std::lock_guard<std::mutex> lk(g_prof.mu);
    cudaEvent_t e = g_prof.take();
    cudaEventRecord(e, st);
    t_pending_start[cls] = e;
    t_pending_timed[cls] = true;
}

void prof_end(int cls, cudaStream_t st, double bytes, double flops, int level)
{
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if (!t_pending_timed[cls]) return;
    t_pending_timed[cls] = false;
    std::lock_guard<std::mutex> lk(g_prof.mu);
    cudaEvent_t e = g_prof.take();
    cudaEventRecord(e, st);
    g_prof.recs.push_back(Rec{t_pending_start[cls], e, cls, level, bytes, flops});
}


}  // namespace msg

using namespace msg;

extern "C" const char* msg_last_error(void) { return g_last_error.c_str(); }
extern "C" const char* msg_version(void) { return "msg-mimc-gb300 0.1 (sm_103a)"; }
extern "C" int64_t msg_launch_count(void) { return g_launches.load(); }

extern "C" int32_t msg_profile_enable(int32_t on)
{
    clear_error();
    if (on < 0) {
        set_error("msg_profile_enable: on must be >= 0");
        return MSG_ERR_INVALID;
    }
    std::lock_guard<std::mutex> lk(g_prof.mu);
    g_prof.stride = 0;
    g_prof.recs.clear();
    g_prof.next = 0;
    for (auto& c : g_prof.count) c = 0;
    g_prof.stride = on;
    return MSG_OK;
}

// Sums over the timed launches of one class (and level, if level >= 0).
static int32_t profile_sum(int32_t cls, int32_t level, int64_t* timed, double* ms_out, double* by_out, double* fl_out)
{
    std::lock_guard<std::mutex> lk(g_prof.mu);
    int64_t n = 0;
    double ms = 0.0, by = 0.0, fl = 0.0;
    for (const Rec& r : g_prof.recs) {
        if (r.cls != cls || (level >= 0 && r.level != level)) continue;
        cudaError_t e = cudaEventSynchronize(r.b);
        if (e != cudaSuccess) { set_error(cudaGetErrorString(e)); return MSG_ERR_CUDA; }
        float t = 0.f;
        cudaEventElapsedTime(&t, r.a, r.b);
        ms += t;
        by += r.bytes;
        fl += r.flops;
        ++n;
    }
    *timed = n;
    *ms_out = ms;
    *by_out = by;
    *fl_out = fl;
    return MSG_OK;
}

extern "C" int32_t msg_profile_read(int32_t cls, int64_t* launches, double* total_ms, double* bytes, double* flops)
{
    clear_error();
    if (cls < 0 || cls >= K_NCLASS || !launches || !total_ms || !bytes || !flops) {
        set_error("msg_profile_read: bad arguments");
        return MSG_ERR_INVALID;
    }
    int64_t n = 0;
    double ms = 0.0, by = 0.0, fl = 0.0;
    const int32_t rc = profile_sum(cls, -1, &n, &ms, &by, &fl);
    if (rc != MSG_OK) return rc;
    // every launch is counted, a random 1/stride of them is timed: scale the timed sums
    const int64_t all = g_prof.count[cls].load();
    const double scale = n > 0 ? (double)all / (double)n : 0.0;
    *launches = all;
    *total_ms = ms * scale;
    *bytes = by * scale;
    *flops = fl * scale;
    return MSG_OK;
}

extern "C" int32_t msg_profile_read_level(int32_t cls, int32_t level, int64_t* timed, double* total_ms, double* bytes)
{
    clear_error();
    if (cls < 0 || cls >= K_NCLASS || level < 0 || !timed || !total_ms || !bytes) {
        set_error("msg_profile_read_level: bad arguments");
        return MSG_ERR_INVALID;
    }
    double fl = 0.0;
    return profile_sum(cls, level, timed, total_ms, bytes, &fl);
}
