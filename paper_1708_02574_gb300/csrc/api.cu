// C-ABI entry points of libtpa (declared in include/tpa.h).
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <cmath>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "tpa_internal.cuh"

namespace tpa {

// Fixed per-thread buffer: recording an error never allocates.
static thread_local char g_err[1024];

void set_error(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

void clear_error() { g_err[0] = '\0'; }

// The library's stream-ordered memory pool on the current device.  Its release
// threshold is unlimited, so a freed block stays mapped (and is reused by the
// next allocation) until trim_pool() hands unused memory back to the driver;
// that happens only after a device-wide synchronisation (end of graph build,
// tpa_free_graph, tpa_server_free).  The default pool would unmap freed
// blocks at every synchronisation of any stream.
static cudaMemPool_t lib_pool()
{
    constexpr int kMaxDevices = 64;
    static std::mutex mu;
    static cudaMemPool_t pools[kMaxDevices];
    int dev = 0;
    TPA_CUDA(cudaGetDevice(&dev));
    TPA_REQUIRE(dev >= 0 && dev < kMaxDevices, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lk(mu);
    if (!pools[dev]) {
        cudaMemPoolProps props;
        memset(&props, 0, sizeof props);
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        TPA_CUDA(cudaMemPoolCreate(&pool, &props));
        uint64_t keep = UINT64_MAX;
        TPA_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep));
        pools[dev] = pool;
    }
    return pools[dev];
}

void trim_pool() noexcept
{
    try {
        cudaMemPoolTrimTo(lib_pool(), 0);
    } catch (...) {
        cudaGetLastError();
    }
}

// Growth of a buffer that exists frees the old block, which a captured graph,
// another stream or an earlier call may still be reading: wait for the whole
// device first (growth happens a few times per workspace, not per call).  No
// allocation may happen while a stream is being captured: the address would
// belong to the graph, not to the library.
void DevBuf::ensure(size_t b, cudaStream_t s)
{
    if (b <= bytes && p) return;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
        cudaGetLastError();
        cs = cudaStreamCaptureStatusNone;
    }
    if (cs != cudaStreamCaptureStatusNone) {
        set_error("a %zu-byte device buffer would be allocated while the stream is captured", b);
        throw Fail{TPA_ECUDA};
    }
    if (p) {
        TPA_CUDA(cudaDeviceSynchronize());
        release(s);
    }
    void *q = nullptr;
    cudaError_t e = cudaMallocFromPoolAsync(&q, b ? b : 16, lib_pool(), s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("device allocation of %zu bytes failed: %s", b, cudaGetErrorString(e));
        throw Fail{TPA_ENOMEM};
    }
    p = q;
    bytes = b;
}

void DevBuf::release(cudaStream_t s)
{
    if (p) cudaFreeAsync(p, s);
    p = nullptr;
    bytes = 0;
}

void need(const DevBuf &b, size_t bytes, const char *what)
{
    if (!b.p || b.bytes < bytes) {
        set_error("internal: %s holds %zu bytes, a launch indexes %zu", what, b.p ? b.bytes : (size_t)0, bytes);
        throw Fail{TPA_ECUDA};
    }
}

bool is_device_ptr(const void *p)
{
    if (!p) return false;
    cudaPointerAttributes attr;
    cudaError_t e = cudaPointerGetAttributes(&attr, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
}

// Device address of page-locked host memory the device can reach (allocated
// or registered with CUDA), else nullptr.
void *mapped_host_ptr(void *p)
{
    if (!p) return nullptr;
    cudaPointerAttributes attr;
    cudaError_t e = cudaPointerGetAttributes(&attr, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return attr.type == cudaMemoryTypeHost ? attr.devicePointer : nullptr;
}

void copy_in(void *dst_dev, const void *src_any, size_t bytes, cudaStream_t s)
{
    if (bytes) TPA_CUDA(cudaMemcpyAsync(dst_dev, src_any, bytes, cudaMemcpyDefault, s));
}

double alpha_of(double c, int S, int T)
{
    // Section III-B: ||r_neighbor||_1 / ||r_family||_1 by Lemma 2
    const double a = std::pow(1.0 - c, (double)S), b = std::pow(1.0 - c, (double)T);
    return (a - b) / (1.0 - a);
}

// Copy k seeds to the host (from host or device memory) and check 0 <= s < n.
static std::vector<int32_t> read_seeds(const int32_t *seeds, int k, int64_t n, cudaStream_t s)
{
    std::vector<int32_t> h((size_t)k);
    if (is_device_ptr(seeds)) {
        TPA_CUDA(cudaMemcpyAsync(h.data(), seeds, (size_t)k * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        TPA_CUDA(cudaStreamSynchronize(s));
    } else {
        memcpy(h.data(), seeds, (size_t)k * sizeof(int32_t));
    }
    for (int j = 0; j < k; ++j) TPA_REQUIRE(h[j] >= 0 && h[j] < n, "seed %d (index %d) is outside [0, %lld)", h[j], j, (long long)n);
    return h;
}

// Raise TPA_ETIMEOUT when a bounded device wait of the graph's kernels gave
// up since the last check (the flag lives in the control block and is
// cleared here).  Called where a call synchronises anyway.
static void check_waits(tpa_graph *g, cudaStream_t s)
{
    if (!g->ws.ctl.p) return;
    int32_t *flag = &static_cast<Ctl *>(g->ws.ctl.p)->error;
    int32_t e = 0;
    TPA_CUDA(cudaMemcpyAsync(&e, flag, sizeof e, cudaMemcpyDeviceToHost, s));
    TPA_CUDA(cudaStreamSynchronize(s));
    if (e) {
        TPA_CUDA(cudaMemsetAsync(flag, 0, sizeof e, s));
        TPA_CUDA(cudaStreamSynchronize(s));
        set_error("a bounded device wait gave up: the results of the calls since the last check are not valid");
        throw Fail{TPA_ETIMEOUT};
    }
}

}  // namespace tpa

using namespace tpa;

#define API_BEGIN \
    clear_error(); \
    try {
#define API_END                                   \
    }                                             \
    catch (const Fail &f) {                       \
        return f.st;                              \
    }                                             \
    catch (const std::bad_alloc &) {              \
        set_error("host allocation failed");      \
        return TPA_ENOMEM;                        \
    }                                             \
    catch (...) {                                 \
        set_error("unexpected C++ exception");    \
        return TPA_ECUDA;                         \
    }                                             \
    return TPA_OK;

// Columns per group when a query's scores go to page-locked host memory
// through device buffers (tpa_set_output_group_width): -1 makes the kernels
// write the host memory directly; 0, the default, takes 128 columns where
// two buffers of n x 128 floats fit in 8 GiB, else 64 where those fit, else
// direct writes.  Grouping applies from two groups on, so that a copy
// overlaps a computation.
static std::atomic<int> g_group_width{0};

static int stage_width(int64_t n, int k)
{
    int w = g_group_width.load();
    if (w < 0) return 0;
    if (w == 0) {
        w = 128;
        while (w >= 64 && 2.0 * (double)n * w * sizeof(float) > (double)(8ull << 30)) w /= 2;
        if (w < 64) return 0;
    }
    return k >= 2 * w ? w : 0;
}

// Algorithm 3 for the columns of a host output in groups of gw: group i is
// computed on s into stage[i & 1] and copied to the host on the copy stream,
// which group i + 2 waits for before it reuses the buffer.
static void query_in_groups(tpa_graph *g, const CpiArgs &a0, float *host, int gw, cudaStream_t s)
{
    Workspace &W = g->ws;
    if (!W.copy) TPA_CUDA(cudaStreamCreateWithFlags(&W.copy, cudaStreamNonBlocking));
    for (int b = 0; b < 2; ++b) {
        if (!W.ready[b]) TPA_CUDA(cudaEventCreateWithFlags(&W.ready[b], cudaEventDisableTiming));
        if (!W.copied[b]) TPA_CUDA(cudaEventCreateWithFlags(&W.copied[b], cudaEventDisableTiming));
        W.stage[b].ensure((size_t)g->n * gw * sizeof(float), s);
    }
    const int k = a0.k;
    int groups = 0;
    for (int g0 = 0; g0 < k; g0 += gw, ++groups) {
        const int b = groups & 1, kg = std::min(gw, k - g0);
        if (groups >= 2) TPA_CUDA(cudaStreamWaitEvent(s, W.copied[b], 0));
        CpiArgs a = a0;
        a.seeds = a0.seeds + g0;
        a.seed_outdeg = a0.seed_outdeg + g0;
        a.k = kg;
        a.out = W.stage[b].as<float>();
        a.ldo = kg;
        run_cpi(g, a, s);
        TPA_CUDA(cudaEventRecord(W.ready[b], s));
        TPA_CUDA(cudaStreamWaitEvent(W.copy, W.ready[b], 0));
        TPA_CUDA(cudaMemcpy2DAsync(host + g0, (size_t)k * sizeof(float), W.stage[b].p, (size_t)kg * sizeof(float),
                                   (size_t)kg * sizeof(float), (size_t)g->n, cudaMemcpyDeviceToHost, W.copy));
        TPA_CUDA(cudaEventRecord(W.copied[b], W.copy));
    }
    // the caller's stream completes after both copies (and the stage buffers
    // are freed on it only after them)
    for (int b = 0; b < std::min(groups, 2); ++b) TPA_CUDA(cudaStreamWaitEvent(s, W.copied[b], 0));
}

extern "C" {

const char *tpa_last_error(void) { return g_err; }

tpa_status tpa_build_graph(int64_t n, int64_t m_edges, const int32_t *src, const int32_t *dst, void *stream,
                           tpa_graph **out)
{
    API_BEGIN
    TPA_REQUIRE(out != nullptr, "tpa_build_graph: out is NULL");
    TPA_REQUIRE(n >= 1 && n < ((int64_t)1 << 31), "tpa_build_graph: n = %lld outside [1, 2^31)", (long long)n);
    TPA_REQUIRE(m_edges >= 0 && m_edges < ((int64_t)1 << 31) - 1, "tpa_build_graph: m_edges = %lld outside [0, 2^31-1)",
                (long long)m_edges);
    TPA_REQUIRE(m_edges == 0 || (src && dst), "tpa_build_graph: NULL edge arrays");
    cudaStream_t s = (cudaStream_t)stream;
    tpa_graph *g = new tpa_graph();
    try {
        TPA_CUDA(cudaGetDevice(&g->device));
        g->n = n;
        DevBuf dsrc, ddst;
        const int32_t *ps = src, *pd = dst;
        if (m_edges > 0 && !is_device_ptr(src)) {
            dsrc.ensure((size_t)m_edges * sizeof(int32_t), s);
            copy_in(dsrc.p, src, (size_t)m_edges * sizeof(int32_t), s);
            ps = dsrc.as<int32_t>();
        }
        if (m_edges > 0 && !is_device_ptr(dst)) {
            ddst.ensure((size_t)m_edges * sizeof(int32_t), s);
            copy_in(ddst.p, dst, (size_t)m_edges * sizeof(int32_t), s);
            pd = ddst.as<int32_t>();
        }
        build_csr(g, ps, pd, m_edges, s);
        dsrc.release(s);
        ddst.release(s);
        // the sort buffers of the build go back to the driver
        TPA_CUDA(cudaStreamSynchronize(s));
        trim_pool();
    } catch (...) {
        tpa_free_graph(g);
        throw;
    }
    *out = g;
    API_END
}

void tpa_free_graph(tpa_graph *g)
{
    if (!g) return;
    cudaStream_t s = 0;
    cudaDeviceSynchronize();
    DevBuf *bufs[] = {&g->rp_t, &g->col_t, &g->val_t, &g->rp_a, &g->col_a, &g->val_a, &g->outdeg, &g->inv_deg32,
                      &g->r_str,
                      &g->perm_a2t, &g->w_a, &g->inv_d, &g->row_a, &g->ws.u, &g->ws.touched, &g->ws.x2,
                      &g->ws.x, &g->ws.y, &g->ws.r, &g->ws.carry, &g->ws.head, &g->ws.tl1, &g->ws.fix,
                      &g->ws.ctl, &g->ws.seeds, &g->ws.sets, &g->ws.seeds_g, &g->ws.cols,
                      &g->ws.out, &g->ws.iters};
    for (DevBuf *b : bufs) b->release(s);
    g->ws.cpart.release(s);
    g->ws.agg.release(s);
    g->ws.lrec.release(s);
    g->ws.ltail.release(s);
    for (tpa::SegRows *R : {&g->seg_t, &g->seg_a})
        for (DevBuf *b : {&R->colf, &R->nz_rows, &R->empty_rows, &R->nzpos, &R->nzrp}) b->release(s);
    for (auto *tiles : {&g->segt_t, &g->segt_a})
        for (auto &kv : *tiles) kv.second.crow0.release(s);
    for (tpa::BinPlan *B : {&g->bins_t, &g->bins_a})
        for (DevBuf *b : {&B->rows_short, &B->rows_mid, &B->rows_long, &B->rows_empty, &B->long_first,
                          &B->chunk_row, &B->chunk_e0})
            b->release(s);
    for (auto *plans : {&g->plans_t, &g->plans_a})
        for (auto &kv : *plans) {
            kv.second.tile_x.release(s);
            kv.second.tile_y.release(s);
            kv.second.head_row.release(s);
            kv.second.head_first.release(s);
        }
    g->ws.stage[0].release(s);
    g->ws.stage[1].release(s);
    if (g->ws.hflag) cudaFreeHost(g->ws.hflag);
    for (int b = 0; b < 2; ++b) {
        if (g->ws.ready[b]) cudaEventDestroy(g->ws.ready[b]);
        if (g->ws.copied[b]) cudaEventDestroy(g->ws.copied[b]);
    }
    if (g->ws.copy) cudaStreamDestroy(g->ws.copy);
    cudaStreamSynchronize(s);
    trim_pool();
    delete g;
}

tpa_status tpa_graph_info(const tpa_graph *g, int64_t *n, int64_t *m)
{
    API_BEGIN
    TPA_REQUIRE(g != nullptr, "tpa_graph_info: NULL graph");
    if (n) *n = g->n;
    if (m) *m = g->m;
    API_END
}

tpa_status tpa_get_csr(const tpa_graph *g, int which, int64_t *row_ptr, int32_t *col, float *val, void *stream)
{
    API_BEGIN
    TPA_REQUIRE(g != nullptr, "tpa_get_csr: NULL graph");
    TPA_REQUIRE(which == 0 || which == 1, "tpa_get_csr: which must be 0 (A~^T) or 1 (A~)");
    cudaStream_t s = (cudaStream_t)stream;
    const DevBuf &rp = which ? g->rp_a : g->rp_t;
    const DevBuf &cl = which ? g->col_a : g->col_t;
    const DevBuf &vl = which ? g->val_a : g->val_t;
    bool host = false;
    if (row_ptr) {
        TPA_CUDA(cudaMemcpyAsync(row_ptr, rp.p, (size_t)(g->n + 1) * sizeof(int64_t), cudaMemcpyDefault, s));
        host |= !is_device_ptr(row_ptr);
    }
    if (col && g->m) {
        TPA_CUDA(cudaMemcpyAsync(col, cl.p, (size_t)g->m * sizeof(int32_t), cudaMemcpyDefault, s));
        host |= !is_device_ptr(col);
    }
    if (val && g->m) {
        TPA_CUDA(cudaMemcpyAsync(val, vl.p, (size_t)g->m * sizeof(float), cudaMemcpyDefault, s));
        host |= !is_device_ptr(val);
    }
    if (host) TPA_CUDA(cudaStreamSynchronize(s));
    API_END
}

tpa_status tpa_preprocess(tpa_graph *g, double c, int T, double eps, void *stream)
{
    API_BEGIN
    TPA_REQUIRE(g != nullptr, "tpa_preprocess: NULL graph");
    TPA_REQUIRE(c > 0.0 && c < 1.0, "tpa_preprocess: c = %g outside (0, 1)", c);
    TPA_REQUIRE(T >= 1, "tpa_preprocess: T = %d < 1", T);
    TPA_REQUIRE(eps > 0.0 && std::isfinite(eps), "tpa_preprocess: eps must be positive");
    cudaStream_t s = (cudaStream_t)stream;
    g->has_pre = false;
    g->r_str.ensure((size_t)g->n * sizeof(float), s);
    g->ws.iters.ensure(sizeof(int32_t), s);
    CpiArgs a;
    a.seeds = nullptr;
    a.k = 1;
    a.c = c;
    a.eps = eps;
    a.s_iter = T;
    a.t_iter = -1;
    a.r = g->r_str.as<float>();
    a.ldr = 1;
    a.iters_out = g->ws.iters.as<int32_t>();
    run_cpi(g, a, s);
    int32_t it = 0;
    TPA_CUDA(cudaMemcpyAsync(&it, a.iters_out, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    TPA_CUDA(cudaStreamSynchronize(s));
    check_waits(g, s);
    g->pre_iters = it;
    g->c = c;
    g->T = T;
    g->eps = eps;
    g->has_pre = true;
    API_END
}

tpa_status tpa_get_stranger(const tpa_graph *g, float *out, int64_t *iters, void *stream)
{
    API_BEGIN
    TPA_REQUIRE(g != nullptr, "tpa_get_stranger: NULL graph");
    if (!g->has_pre) {
        set_error("tpa_get_stranger: tpa_preprocess has not run");
        return TPA_ESTATE;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (out) {
        TPA_CUDA(cudaMemcpyAsync(out, g->r_str.p, (size_t)g->n * sizeof(float), cudaMemcpyDefault, s));
        if (!is_device_ptr(out)) TPA_CUDA(cudaStreamSynchronize(s));
    }
    if (iters) *iters = g->pre_iters;
    API_END
}

tpa_status tpa_query(tpa_graph *g, const int32_t *seeds, int k, int S, float *out, void *stream)
{
    API_BEGIN
    TPA_REQUIRE(g != nullptr, "tpa_query: NULL graph");
    if (!g->has_pre) {
        set_error("tpa_query: tpa_preprocess has not run");
        return TPA_ESTATE;
    }
    TPA_REQUIRE(k >= 1, "tpa_query: k = %d < 1", k);
    TPA_REQUIRE(S >= 1 && S <= g->T, "tpa_query: S = %d outside [1, T = %d]", S, g->T);
    TPA_REQUIRE(seeds && out, "tpa_query: NULL seeds or out");
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<int32_t> hs = read_seeds(seeds, k, g->n, s);
    g->ws.seeds.ensure((size_t)k * sizeof(int32_t), s);
    TPA_CUDA(cudaMemcpyAsync(g->ws.seeds.p, hs.data(), (size_t)k * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    // Host output.  Page-locked memory is filled by column groups: each group
    // is computed into a device buffer and copied to the host by the copy
    // engine while the next group computes (or, for few columns or
    // tpa_set_output_group_width(-1), written by the kernels directly).
    // Other host memory is staged and copied at the end.
    const bool host_out = !is_device_ptr(out);
    float *mapped = host_out ? static_cast<float *>(mapped_host_ptr(out)) : nullptr;
    // rows not 16-byte aligned would take 4-byte stores over the host link:
    // stage those in device memory and copy once
    if (mapped && (k * sizeof(float)) % 16 != 0) mapped = nullptr;
    const int gw = mapped ? stage_width(g->n, k) : 0;
    float *dout = out;
    if (host_out && !gw) {
        if (mapped) {
            dout = mapped;
        } else {
            g->ws.out.ensure((size_t)g->n * k * sizeof(float), s);
            dout = g->ws.out.as<float>();
        }
    }
    CpiArgs a;
    a.seeds = g->ws.seeds.as<int32_t>();
    a.k = k;
    a.c = g->c;
    a.eps = g->eps;
    a.s_iter = 0;
    a.t_iter = S - 1;
    a.r_internal = true;
    a.tpa_final = true;
    a.alpha = alpha_of(g->c, S, g->T);
    a.r_str = g->r_str.as<float>();
    a.out = dout;
    a.ldo = k;
    std::vector<int32_t> od = seed_outdegrees(g, a.seeds, k, s);   // the host picks each chunk's branch
    a.seed_outdeg = od.data();
    if (gw) {
        query_in_groups(g, a, out, gw, s);
    } else {
        run_cpi(g, a, s);
    }
    if (host_out) {
        if (!mapped)
            TPA_CUDA(cudaMemcpyAsync(out, dout, (size_t)g->n * k * sizeof(float), cudaMemcpyDeviceToHost, s));
        TPA_CUDA(cudaStreamSynchronize(s));
        check_waits(g, s);
    }
    API_END
}

tpa_status tpa_query_sets(tpa_graph *g, const int64_t *set_ptr, const int32_t *members, int nsets, int S,
                          float *out, void *stream)
{
    API_BEGIN
    TPA_REQUIRE(g != nullptr, "tpa_query_sets: NULL graph");
    if (!g->has_pre) {
        set_error("tpa_query_sets: tpa_preprocess has not run");
        return TPA_ESTATE;
    }
    TPA_REQUIRE(nsets >= 1, "tpa_query_sets: nsets = %d < 1", nsets);
    TPA_REQUIRE(S >= 1 && S <= g->T, "tpa_query_sets: S = %d outside [1, T = %d]", S, g->T);
    TPA_REQUIRE(set_ptr && members && out, "tpa_query_sets: NULL set_ptr, members or out");
    TPA_REQUIRE(is_device_ptr(out), "tpa_query_sets: out must be device memory");
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<int64_t> hp((size_t)nsets + 1);
    if (is_device_ptr(set_ptr)) {
        TPA_CUDA(cudaMemcpyAsync(hp.data(), set_ptr, hp.size() * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        TPA_CUDA(cudaStreamSynchronize(s));
    } else {
        memcpy(hp.data(), set_ptr, hp.size() * sizeof(int64_t));
    }
    TPA_REQUIRE(hp[0] == 0, "tpa_query_sets: set_ptr[0] = %lld, not 0", (long long)hp[0]);
    for (int j = 0; j < nsets; ++j)
        TPA_REQUIRE(hp[j + 1] > hp[j], "tpa_query_sets: seed set %d is empty or set_ptr decreases", j);
    const int64_t total = hp[nsets];
    TPA_REQUIRE(total <= ((int64_t)1 << 31) - 1, "tpa_query_sets: %lld members, more than 2^31 - 1",
                (long long)total);
    std::vector<int32_t> hm((size_t)total);
    if (is_device_ptr(members)) {
        TPA_CUDA(cudaMemcpyAsync(hm.data(), members, (size_t)total * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        TPA_CUDA(cudaStreamSynchronize(s));
    } else {
        memcpy(hm.data(), members, (size_t)total * sizeof(int32_t));
    }
    for (int64_t e = 0; e < total; ++e)
        TPA_REQUIRE(hm[e] >= 0 && hm[e] < g->n, "member %d (index %lld) is outside [0, %lld)", hm[e], (long long)e,
                    (long long)g->n);
    g->ws.seeds.ensure((size_t)total * sizeof(int32_t), s);
    g->ws.sets.ensure(hp.size() * sizeof(int64_t), s);
    TPA_CUDA(cudaMemcpyAsync(g->ws.seeds.p, hm.data(), (size_t)total * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    TPA_CUDA(cudaMemcpyAsync(g->ws.sets.p, hp.data(), hp.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    CpiArgs a;
    a.seeds = g->ws.seeds.as<int32_t>();
    a.set_ptr = g->ws.sets.as<int64_t>();
    a.k = nsets;
    a.c = g->c;
    a.eps = g->eps;
    a.s_iter = 0;
    a.t_iter = S - 1;
    a.r_internal = true;
    a.tpa_final = true;
    a.alpha = alpha_of(g->c, S, g->T);
    a.r_str = g->r_str.as<float>();
    a.out = out;
    a.ldo = nsets;
    run_cpi(g, a, s);
    // the host copies above read from pageable vectors: finish them before those go
    TPA_CUDA(cudaStreamSynchronize(s));
    API_END
}

tpa_status tpa_cpi(tpa_graph *g, const int32_t *seeds, int k, double c, double eps, int s_iter, int t_iter,
                   float *out, int32_t *iters, void *stream)
{
    API_BEGIN
    TPA_REQUIRE(g != nullptr, "tpa_cpi: NULL graph");
    TPA_REQUIRE(k >= 1, "tpa_cpi: k = %d < 1", k);
    TPA_REQUIRE(c > 0.0 && c < 1.0, "tpa_cpi: c = %g outside (0, 1)", c);
    TPA_REQUIRE(eps > 0.0 && std::isfinite(eps), "tpa_cpi: eps must be positive");
    TPA_REQUIRE(s_iter >= 0, "tpa_cpi: s_iter < 0");
    TPA_REQUIRE(seeds && out, "tpa_cpi: NULL seeds or out");
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<int32_t> hs = read_seeds(seeds, k, g->n, s);
    g->ws.seeds.ensure((size_t)k * sizeof(int32_t), s);
    TPA_CUDA(cudaMemcpyAsync(g->ws.seeds.p, hs.data(), (size_t)k * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    const bool host_out = !is_device_ptr(out);
    float *dout = out;
    if (host_out) {
        g->ws.out.ensure((size_t)g->n * k * sizeof(float), s);
        dout = g->ws.out.as<float>();
    }
    g->ws.iters.ensure((size_t)k * sizeof(int32_t), s);
    CpiArgs a;
    a.seeds = g->ws.seeds.as<int32_t>();
    a.k = k;
    a.c = c;
    a.eps = eps;
    a.s_iter = s_iter;
    a.t_iter = t_iter;
    a.r = dout;
    a.ldr = k;
    a.iters_out = g->ws.iters.as<int32_t>();
    run_cpi(g, a, s);
    if (iters) {
        TPA_CUDA(cudaMemcpyAsync(iters, a.iters_out, (size_t)k * sizeof(int32_t), cudaMemcpyDefault, s));
        if (!is_device_ptr(iters)) TPA_CUDA(cudaStreamSynchronize(s));
    }
    if (host_out) {
        TPA_CUDA(cudaMemcpyAsync(out, dout, (size_t)g->n * k * sizeof(float), cudaMemcpyDeviceToHost, s));
        TPA_CUDA(cudaStreamSynchronize(s));
        check_waits(g, s);
    }
    API_END
}

tpa_status tpa_cpi_exact(tpa_graph *g, int32_t seed, double c, double eps, float *out, int32_t *iters, void *stream)
{
    return tpa_cpi(g, &seed, 1, c, eps, 0, -1, out, iters, stream);
}

tpa_status tpa_set_edge_weights(tpa_graph *g, const float *w, void *stream)
{
    API_BEGIN
    TPA_REQUIRE(g != nullptr && (w != nullptr || g->m == 0), "tpa_set_edge_weights: NULL argument");
    set_edge_weights(g, w, (cudaStream_t)stream);
    if (!is_device_ptr(w)) TPA_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    API_END
}

tpa_status tpa_edge_weights(const float *feat, const float *theta, int d, int64_t m, float *w, void *stream)
{
    API_BEGIN
    TPA_REQUIRE(d >= 1 && d <= 16 && m >= 0, "tpa_edge_weights: d = %d outside [1, 16] or m < 0", d);
    TPA_REQUIRE(m == 0 || (is_device_ptr(feat) && is_device_ptr(theta) && is_device_ptr(w)),
                "tpa_edge_weights: feat, theta and w must be device memory");
    if (m) weights_from_features(feat, theta, d, m, w, (cudaStream_t)stream);
    API_END
}

tpa_status tpa_sync(tpa_graph *g, void *stream)
{
    API_BEGIN
    TPA_REQUIRE(g != nullptr, "tpa_sync: NULL graph");
    check_waits(g, (cudaStream_t)stream);
    API_END
}

tpa_status tpa_set_adjoint_budget(uint64_t bytes)
{
    g_adjoint_budget = (size_t)bytes;
    return TPA_OK;
}

tpa_status tpa_set_adjoint_batch_width(int width)
{
    clear_error();
    if (!(width == 0 || width == 8 || width == 16 || width == 32)) {
        set_error("tpa_set_adjoint_batch_width: %d is not 0, 8, 16 or 32", width);
        return TPA_EINVAL;
    }
    g_adjoint_batch = width;
    return TPA_OK;
}

int tpa_get_adjoint_batch_width(void) { return adjoint_batch_width(); }

tpa_status tpa_loss_grad(tpa_graph *g, const int32_t *seeds, const int32_t *pos, const int32_t *neg, int ntrip,
                         double c, int S, int T, int K, double *loss, float *grad_w, void *stream)
{
    API_BEGIN
    TPA_REQUIRE(g && seeds && pos && neg && loss, "tpa_loss_grad: NULL argument");
    TPA_REQUIRE(ntrip >= 1, "tpa_loss_grad: ntrip = %d < 1", ntrip);
    TPA_REQUIRE(c > 0.0 && c < 1.0, "tpa_loss_grad: c = %g outside (0, 1)", c);
    TPA_REQUIRE(S >= 1 && S <= T && T <= K && K <= 100000, "tpa_loss_grad: need 1 <= S <= T <= K");
    cudaStream_t s = (cudaStream_t)stream;
    if (!g->weighted) {
        // unit weights reproduce the unweighted A~ and give the inverse degrees
        DevBuf ones;
        ones.ensure((size_t)std::max<int64_t>(g->m, 1) * sizeof(float), s);
        std::vector<float> h((size_t)std::max<int64_t>(g->m, 1), 1.0f);
        TPA_CUDA(cudaMemcpyAsync(ones.p, h.data(), h.size() * sizeof(float), cudaMemcpyHostToDevice, s));
        set_edge_weights(g, ones.as<float>(), s, false);   // RN32(1/d) either way: preprocessing stays valid
        TPA_CUDA(cudaStreamSynchronize(s));
        ones.release(s);
    }
    std::vector<int32_t> hs = read_seeds(seeds, ntrip, g->n, s), hp = read_seeds(pos, ntrip, g->n, s),
                         hq = read_seeds(neg, ntrip, g->n, s);
    DevBuf trip;
    trip.ensure((size_t)3 * ntrip * sizeof(int32_t), s);
    TPA_CUDA(cudaMemcpyAsync(trip.as<int32_t>(), hs.data(), (size_t)ntrip * 4, cudaMemcpyHostToDevice, s));
    TPA_CUDA(cudaMemcpyAsync(trip.as<int32_t>() + ntrip, hp.data(), (size_t)ntrip * 4, cudaMemcpyHostToDevice, s));
    TPA_CUDA(cudaMemcpyAsync(trip.as<int32_t>() + 2 * ntrip, hq.data(), (size_t)ntrip * 4, cudaMemcpyHostToDevice, s));
    const bool host_out = grad_w && !is_device_ptr(grad_w);
    DevBuf gw;
    float *dgw = grad_w;
    if (host_out) {
        gw.ensure((size_t)std::max<int64_t>(g->m, 1) * sizeof(float), s);
        dgw = gw.as<float>();
    }
    *loss = loss_grad(g, trip.as<int32_t>(), trip.as<int32_t>() + ntrip, trip.as<int32_t>() + 2 * ntrip, ntrip, c, S,
                      T, K, dgw, s);
    if (host_out && g->m) {
        TPA_CUDA(cudaMemcpyAsync(grad_w, dgw, (size_t)g->m * sizeof(float), cudaMemcpyDeviceToHost, s));
        TPA_CUDA(cudaStreamSynchronize(s));
    }
    trip.release(s);
    gw.release(s);
    API_END
}

tpa_status tpa_theta_grad(const float *feat, const float *w, const float *grad_w, int d, int64_t m,
                          double *grad_theta, void *stream)
{
    API_BEGIN
    TPA_REQUIRE(d >= 1 && d <= 16 && m >= 1, "tpa_theta_grad: d = %d outside [1, 16] or m < 1", d);
    TPA_REQUIRE(is_device_ptr(feat) && is_device_ptr(w) && is_device_ptr(grad_w) && is_device_ptr(grad_theta),
                "tpa_theta_grad: every array must be device memory");
    theta_grad(feat, w, grad_w, d, m, grad_theta, (cudaStream_t)stream);
    API_END
}

struct PreHeader {
    char magic[8];
    int64_t n, m;
    double c;
    int64_t T;
    double eps;
    int64_t iters;
};

tpa_status tpa_save_preprocessed(const tpa_graph *g, const char *path)
{
    API_BEGIN
    TPA_REQUIRE(g && path, "tpa_save_preprocessed: NULL argument");
    if (!g->has_pre) {
        set_error("tpa_save_preprocessed: tpa_preprocess has not run");
        return TPA_ESTATE;
    }
    std::vector<float> h((size_t)g->n);
    TPA_CUDA(cudaMemcpy(h.data(), g->r_str.p, (size_t)g->n * sizeof(float), cudaMemcpyDeviceToHost));
    PreHeader hd;
    memcpy(hd.magic, "TPASTR01", 8);
    hd.n = g->n;
    hd.m = g->m;
    hd.c = g->c;
    hd.T = g->T;
    hd.eps = g->eps;
    hd.iters = g->pre_iters;
    FILE *f = fopen(path, "wb");
    TPA_REQUIRE(f != nullptr, "tpa_save_preprocessed: cannot open %s", path);
    const bool ok = fwrite(&hd, sizeof(hd), 1, f) == 1 && fwrite(h.data(), sizeof(float), h.size(), f) == h.size();
    const bool closed = fclose(f) == 0;
    TPA_REQUIRE(ok && closed, "tpa_save_preprocessed: write to %s failed", path);
    API_END
}

tpa_status tpa_load_preprocessed(tpa_graph *g, const char *path, void *stream)
{
    API_BEGIN
    TPA_REQUIRE(g && path, "tpa_load_preprocessed: NULL argument");
    FILE *f = fopen(path, "rb");
    TPA_REQUIRE(f != nullptr, "tpa_load_preprocessed: cannot open %s", path);
    PreHeader hd;
    std::vector<float> h;
    bool ok = fread(&hd, sizeof(hd), 1, f) == 1 && memcmp(hd.magic, "TPASTR01", 8) == 0 && hd.n == g->n &&
              hd.m == g->m && hd.c > 0 && hd.c < 1 && hd.T >= 1 && hd.T < (1 << 30);
    if (ok) {
        h.resize((size_t)g->n);
        ok = fread(h.data(), sizeof(float), h.size(), f) == h.size();
    }
    fclose(f);
    TPA_REQUIRE(ok, "tpa_load_preprocessed: %s is not preprocessed data for this graph", path);
    cudaStream_t s = (cudaStream_t)stream;
    g->r_str.ensure((size_t)g->n * sizeof(float), s);
    TPA_CUDA(cudaMemcpyAsync(g->r_str.p, h.data(), (size_t)g->n * sizeof(float), cudaMemcpyHostToDevice, s));
    TPA_CUDA(cudaStreamSynchronize(s));
    g->c = hd.c;
    g->T = (int)hd.T;
    g->eps = hd.eps;
    g->pre_iters = hd.iters;
    g->has_pre = true;
    API_END
}

tpa_status tpa_set_output_group_width(int width)
{
    clear_error();
    if (!(width == 0 || width == -1 || (width >= 8 && width <= 4096 && width % 8 == 0))) {
        set_error("tpa_set_output_group_width: %d is not 0, -1 or a multiple of 8 in [8, 4096]", width);
        return TPA_EINVAL;
    }
    g_group_width.store(width);
    return TPA_OK;
}

int tpa_get_output_group_width(void) { return g_group_width.load(); }

}  // extern "C"
