// api.cu -- error state, version, launch counting and profiling of the C ABI.
#include <atomic>
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
    int cls;
    double bytes, flops;
};
struct Prof {
    std::mutex mu;
    bool on = false;
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
}  // namespace

void set_error(const std::string& what) { g_last_error = what; }
void clear_error() { g_last_error.clear(); }

void prof_begin(int cls, cudaStream_t st)
{
    if (!g_prof.on) return;
    std::lock_guard<std::mutex> lk(g_prof.mu);
    cudaEvent_t e = g_prof.take();
    cudaEventRecord(e, st);
    t_pending_start[cls] = e;
}

void prof_end(int cls, cudaStream_t st, double bytes, double flops)
{
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if (!g_prof.on) return;
    std::lock_guard<std::mutex> lk(g_prof.mu);
    cudaEvent_t e = g_prof.take();
    cudaEventRecord(e, st);
    g_prof.recs.push_back(Rec{t_pending_start[cls], e, cls, bytes, flops});
}

void prof_count() { g_launches.fetch_add(1, std::memory_order_relaxed); }

}  // namespace msg

using namespace msg;

extern "C" const char* msg_last_error(void) { return g_last_error.c_str(); }
extern "C" const char* msg_version(void) { return "msg-mimc-gb300 0.1 (sm_103a)"; }
extern "C" int64_t msg_launch_count(void) { return g_launches.load(); }

extern "C" int32_t msg_profile_enable(int32_t on)
{
    clear_error();
    std::lock_guard<std::mutex> lk(g_prof.mu);
    g_prof.on = on != 0;
    g_prof.recs.clear();
    g_prof.next = 0;
    return MSG_OK;
}

extern "C" int32_t msg_profile_read(int32_t cls, int64_t* launches, double* total_ms, double* bytes, double* flops)
{
    clear_error();
    if (cls < 0 || cls >= K_NCLASS || !launches || !total_ms || !bytes || !flops) {
        set_error("msg_profile_read: bad arguments");
        return MSG_ERR_INVALID;
    }
    std::lock_guard<std::mutex> lk(g_prof.mu);
    int64_t n = 0;
    double ms = 0.0, by = 0.0, fl = 0.0;
    for (const Rec& r : g_prof.recs) {
        if (r.cls != cls) continue;
        cudaError_t e = cudaEventSynchronize(r.b);
        if (e != cudaSuccess) { set_error(cudaGetErrorString(e)); return MSG_ERR_CUDA; }
        float t = 0.f;
        cudaEventElapsedTime(&t, r.a, r.b);
        ms += t;
        by += r.bytes;
        fl += r.flops;
        ++n;
    }
    *launches = n;
    *total_ms = ms;
    *bytes = by;
    *flops = fl;
    return MSG_OK;
}
