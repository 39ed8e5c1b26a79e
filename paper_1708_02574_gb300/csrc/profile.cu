// Launch accounting and optional per-launch CUDA-event timing.
//
// Every kernel launch site calls note_launch(); the SpMV/SpMM and fixup
// launches of Algorithm 1 are bracketed by prof_begin/prof_end, which record
// a pair of CUDA events on the launch stream while timing is enabled, plus the
// algorithmic bytes of the launch, so a benchmark can report achieved
// bandwidth of a kernel from event durations taken inside its timed region.
#include <cuda_runtime.h>

#include <algorithm>
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

// Gather-rate probe: the column ids of CSR(A~^T) read in order and, for
// each, the row of KP floats of an iterate at that column gathered and
// summed, with no row structure, no carries and no epilogue: the cost of the
// gathers alone at the graph's column pattern, against which the SpMM
// kernels are compared.  Four gathers in flight per thread.
template <int KP>
__global__ void gather_probe_k(const int32_t *col, int64_t m, const float *x, float *out)
{
    constexpr int U = 4;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float acc = 0.0f;
    for (int64_t e0 = tid; e0 < m; e0 += U * stride) {
        float v[U][KP];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t e = e0 + u * stride;
#pragma unroll
            for (int j = 0; j < KP; ++j) v[u][j] = 0.0f;
            if (e < m) {
                const float *row = x + (int64_t)__ldcs(col + e) * KP;
                if constexpr (KP == 8) {
                    asm("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                        : "=f"(v[u][0]), "=f"(v[u][1]), "=f"(v[u][2]), "=f"(v[u][3]), "=f"(v[u][4]),
                          "=f"(v[u][5]), "=f"(v[u][6]), "=f"(v[u][7])
                        : "l"(row));
                } else {
                    v[u][0] = __ldg(row);
                }
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
#pragma unroll
            for (int j = 0; j < KP; ++j) acc += v[u][j];
        }
    }
    out[tid] = acc;
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

tpa_status tpa_probe_gather(tpa_graph *g, int kp, int reps, void *stream, double *ms)
{
    clear_error();
    try {
        TPA_REQUIRE(g && ms, "tpa_probe_gather: NULL argument");
        TPA_REQUIRE(kp == 1 || kp == 8, "tpa_probe_gather: kp = %d is neither 1 nor 8", kp);
        TPA_REQUIRE(reps >= 1, "tpa_probe_gather: reps = %d < 1", reps);
        cudaStream_t s = (cudaStream_t)stream;
        int dev = 0, sms = 0;
        TPA_CUDA(cudaGetDevice(&dev));
        TPA_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        const unsigned blocks = (unsigned)sms * 8, threads = 256;
        DevBuf x, out;
        x.ensure((size_t)std::max<int64_t>(1, g->n) * kp * sizeof(float), s);
        out.ensure((size_t)blocks * threads * sizeof(float), s);
        TPA_CUDA(cudaMemsetAsync(x.p, 0, x.bytes, s));
        cudaEvent_t a = nullptr, b = nullptr;
        TPA_CUDA(cudaEventCreate(&a));
        TPA_CUDA(cudaEventCreate(&b));
        auto pass = [&]() {
            if (kp == 8)
                gather_probe_k<8><<<blocks, threads, 0, s>>>(g->col_t.as<int32_t>(), g->m, x.as<float>(),
                                                             out.as<float>());
            else
                gather_probe_k<1><<<blocks, threads, 0, s>>>(g->col_t.as<int32_t>(), g->m, x.as<float>(),
                                                             out.as<float>());
            note_launch("probe");
        };
        pass();   // warm-up
        TPA_CUDA(cudaEventRecord(a, s));
        for (int i = 0; i < reps; ++i) pass();
        TPA_CUDA(cudaEventRecord(b, s));
        TPA_CUDA(cudaEventSynchronize(b));
        float t = 0.0f;
        TPA_CUDA(cudaEventElapsedTime(&t, a, b));
        cudaEventDestroy(a);
        cudaEventDestroy(b);
        TPA_CHECK_LAUNCH();
        x.release(s);
        out.release(s);
        *ms = (double)t / reps;
    } catch (const Fail &f) {
        return f.st;
    }
    return TPA_OK;
}

}  // extern "C"
