// Launch accounting and optional per-launch CUDA-event timing.
//
// Every kernel launch site calls note_launch(); the SpMV/SpMM and fixup
// launches of Algorithm 1 are bracketed by prof_begin/prof_end, which record
// a pair of CUDA events on the launch stream while timing is enabled, plus the
// algorithmic bytes of the launch, so a benchmark can report achieved
// bandwidth of a kernel from event durations taken inside its timed region.
#include <cuda_runtime.h>

#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "tpa_internal.cuh"

namespace tpa {

namespace {
std::atomic<uint64_t> g_launches{0};
std::mutex g_mu;
bool g_timing = false;

struct Stat {
    int64_t launches = 0;
    double total_ms = 0.0;
    double bytes = 0.0;
};
std::map<std::string, Stat> g_stats;

struct Pending {
    std::string name;
    cudaEvent_t a, b;
    double bytes;
};
std::vector<Pending> g_pending;
std::vector<cudaEvent_t> g_pool;

cudaEvent_t take_event()
{
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    TPA_CUDA(cudaEventCreate(&e));
    return e;
}
}  // namespace

void note_launch(const char *family, int count)
{
    g_launches += (uint64_t)count;
    std::lock_guard<std::mutex> lk(g_mu);
    g_stats[family].launches += count;
}

void note_launch_count(int count) { g_launches += (uint64_t)count; }

uint64_t launches_so_far() { return g_launches.load(); }

bool prof_pause()
{
    std::lock_guard<std::mutex> lk(g_mu);
    const bool was = g_timing;
    g_timing = false;
    return was;
}

void prof_resume(bool timing)
{
    std::lock_guard<std::mutex> lk(g_mu);
    g_timing = timing;
}

ProfMark prof_begin(cudaStream_t s)
{
    ProfMark m{nullptr};
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_timing) return m;
    m.a = take_event();
    TPA_CUDA(cudaEventRecord(m.a, s));
    return m;
}

void prof_end(const ProfMark &m, const char *family, double bytes, cudaStream_t s)
{
    std::lock_guard<std::mutex> lk(g_mu);
    if (!m.a) {
        g_stats[family].bytes += bytes;
        return;
    }
    cudaEvent_t b = take_event();
    TPA_CUDA(cudaEventRecord(b, s));
    g_pending.push_back(Pending{family, m.a, b, bytes});
}

}  // namespace tpa

using namespace tpa;

extern "C" {

uint64_t tpa_launch_count(void) { return g_launches.load(); }

tpa_status tpa_profile_reset(int timing)
{
    try {
        std::lock_guard<std::mutex> lk(g_mu);
        for (Pending &p : g_pending) {
            cudaEventSynchronize(p.b);
            g_pool.push_back(p.a);
            g_pool.push_back(p.b);
        }
        g_pending.clear();
        g_stats.clear();
        g_timing = timing != 0;
    } catch (const Fail &f) {
        return f.st;
    }
    return TPA_OK;
}

tpa_status tpa_profile_read(tpa_kernel_stat *out, int cap, int *count)
{
    try {
        std::lock_guard<std::mutex> lk(g_mu);
        for (Pending &p : g_pending) {
            TPA_CUDA(cudaEventSynchronize(p.b));
            float ms = 0.0f;
            TPA_CUDA(cudaEventElapsedTime(&ms, p.a, p.b));
            Stat &st = g_stats[p.name];
            st.total_ms += ms;
            st.bytes += p.bytes;
            g_pool.push_back(p.a);
            g_pool.push_back(p.b);
        }
        g_pending.clear();
        int i = 0;
        for (auto &kv : g_stats) {
            if (i < cap && out) {
                memset(&out[i], 0, sizeof(tpa_kernel_stat));
                strncpy(out[i].name, kv.first.c_str(), sizeof(out[i].name) - 1);
                out[i].launches = kv.second.launches;
                out[i].total_ms = kv.second.total_ms;
                out[i].alg_bytes = kv.second.bytes;
            }
            ++i;
        }
        if (count) *count = i;
    } catch (const Fail &f) {
        return f.st;
    }
    return TPA_OK;
}

}  // extern "C"
