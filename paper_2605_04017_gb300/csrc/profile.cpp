// Per-kernel CUDA-event timing: when enabled, every kernel launch of the
// library is bracketed by two events recorded on the launch stream; reading
// the profile waits for them and sums the elapsed time per kernel name.
#include <cstring>
#include <mutex>
#include <vector>

#include "profile.h"

namespace lt {

namespace {
struct Rec {
    const char* name;
    cudaEvent_t a, b;
    int slot;
};
std::mutex g_mu;
bool g_on = false;
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_free;
unsigned long long g_dropped = 0;
constexpr size_t kMaxRecs = kProfMaxRecs;
// kProfShards device counters per record (record r, shard s at r + s * kMaxRecs),
// zeroed when profiling is enabled and at every reset
unsigned long long* g_work = nullptr;
int g_work_dev = -1;
size_t g_next_slot = 0;

cudaEvent_t get_event()
{
    if (!g_free.empty()) {
        cudaEvent_t e = g_free.back();
        g_free.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}
}  // namespace

bool prof_enabled() { return g_on; }

ProfScope::ProfScope(const char* name, cudaStream_t st) : name_(name), st_(st)
{
    if (!g_on) return;
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_recs.size() >= kMaxRecs) { ++g_dropped; return; }
    a_ = get_event();
    b_ = get_event();
    if (!a_ || !b_) return;
    int dev = -1;
    cudaGetDevice(&dev);
    if (g_work && dev == g_work_dev && g_next_slot < kMaxRecs) {
        slot_ = (int)g_next_slot++;
        work_ = g_work + slot_;
    }
    cudaEventRecord(a_, st_);
    active_ = true;
}

ProfScope::~ProfScope()
{
    if (!active_) return;
    std::lock_guard<std::mutex> lk(g_mu);
    cudaEventRecord(b_, st_);
    g_recs.push_back({name_, a_, b_, slot_});
}

}  // namespace lt

using namespace lt;

extern "C" {

lt_status lt_profile_enable(int32_t on)
{
    std::lock_guard<std::mutex> lk(g_mu);
    g_on = on != 0;
    if (g_on && !g_work) {
        const size_t bytes = kMaxRecs * kProfShards * sizeof(unsigned long long);
        if (cudaGetDevice(&g_work_dev) != cudaSuccess || cudaMalloc(&g_work, bytes) != cudaSuccess ||
            cudaMemset(g_work, 0, bytes) != cudaSuccess) {
            if (g_work) cudaFree(g_work);
            g_work = nullptr;
            g_work_dev = -1;   // timing still works; work counts read as 0
        }
    }
    return LT_OK;
}

lt_status lt_profile_read(lt_kernel_time* out, int32_t max, int32_t* n_out, int32_t reset)
{
    clear_error();
    if (!n_out || (max > 0 && !out)) return fail(LT_EINVAL, "lt_profile_read: NULL argument");
    std::lock_guard<std::mutex> lk(g_mu);
    std::vector<lt_kernel_time> agg;
    std::vector<unsigned long long> work;
    for (const Rec& r : g_recs) LT_CUDA_TRY(cudaEventSynchronize(r.b));
    if (g_work && g_next_slot > 0) {
        work.assign(g_next_slot, 0);
        std::vector<unsigned long long> shard(g_next_slot);
        for (int s = 0; s < kProfShards; ++s) {
            LT_CUDA_TRY(cudaMemcpy(shard.data(), g_work + (size_t)s * kMaxRecs,
                                   shard.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost));
            for (size_t r = 0; r < shard.size(); ++r) work[r] += shard[r];
        }
    }
    for (const Rec& r : g_recs) {
        float ms = 0.0f;
        LT_CUDA_TRY(cudaEventElapsedTime(&ms, r.a, r.b));
        lt_kernel_time* t = nullptr;
        for (auto& x : agg)
            if (std::strcmp(x.name, r.name) == 0) t = &x;
        if (!t) {
            lt_kernel_time z;
            std::memset(&z, 0, sizeof z);
            std::strncpy(z.name, r.name, sizeof z.name - 1);
            agg.push_back(z);
            t = &agg.back();
        }
        t->launches += 1;
        t->total_ms += ms;
        if (r.slot >= 0 && (size_t)r.slot < work.size()) t->work += (int64_t)work[r.slot];
    }
    *n_out = (int32_t)agg.size();
    for (int32_t i = 0; i < (int32_t)agg.size() && i < max; ++i) out[i] = agg[i];
    if (reset) {
        for (const Rec& r : g_recs) {
            g_free.push_back(r.a);
            g_free.push_back(r.b);
        }
        g_recs.clear();
        if (g_work && g_next_slot > 0) {
            // clear the used slots of every shard on the counters' device
            int cur = -1;
            LT_CUDA_TRY(cudaGetDevice(&cur));
            if (cur != g_work_dev) LT_CUDA_TRY(cudaSetDevice(g_work_dev));
            cudaError_t e = cudaSuccess;
            for (int s = 0; s < kProfShards && e == cudaSuccess; ++s)
                e = cudaMemset(g_work + (size_t)s * kMaxRecs, 0, g_next_slot * sizeof(unsigned long long));
            if (cur != g_work_dev) cudaSetDevice(cur);
            if (e != cudaSuccess) return cuda_fail(e, "lt_profile_read: clearing the work counters");
        }
        g_next_slot = 0;
        g_dropped = 0;
    }
    return LT_OK;
}

}  // extern "C"
