// Batched query serving (Algorithm 3 over a stream of request batches).
//
// A request batch of k seeds is answered by the launch sequence tpa_query
// would issue for it: the seeds too heavy for the push branch are moved into
// the last chunks (regrouping), every chunk's push/pull branch for x1 and x2
// is chosen on the host from the seeds' out-degrees (a host copy of them is
// kept), and the moved columns are swapped back at the end.  The sequence
// thus depends on k and on the string of chunk branches only; the seeds in
// run order and the swapped column pairs are data in the server's device
// buffers.  The first batch with a new (k, branches) key runs directly and
// its sequence is then captured into a CUDA graph; later batches with that
// key copy their seeds and pairs and replay the graph.  Results equal
// tpa_query's bit for bit.  The server owns a workspace of its own, swapped
// into the graph handle while a batch is issued, so the device addresses a
// captured graph holds stay valid whatever the graph handle does between
// batches.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <cstring>
#include <map>
#include <string>
#include <utility>
#include <vector>

#include "tpa_internal.cuh"

using namespace tpa;

struct tpa_server {
    tpa_graph *g = nullptr;
    int S = 0, max_k = 0;
    float *out = nullptr;
    int64_t ldo = 0;
    DevBuf out_buf;                 // when the server allocated out
    DevBuf seeds;                   // int32[max_k] seeds in run order, read by the captured graphs
    DevBuf pairs;                   // int32[1 + max_k]: count, then the column pairs to swap back
    int32_t *h_seeds = nullptr;     // pinned: the request's seeds as given
    int32_t *h_stage = nullptr;     // pinned: seeds in run order, count, pairs (one copy to the device)
    cudaEvent_t staged = nullptr;   // the last copy has left h_stage
    cudaStream_t cap = nullptr;     // capture stream
    std::vector<int32_t> h_outdeg;  // out-degrees of all nodes (branch choice on the host)
    Workspace ws;
    struct Entry {
        cudaGraphExec_t exec = nullptr;
        int64_t launches = 0;
        int k = 0;
        uint64_t used = 0;             // last use, for eviction
        std::vector<uint64_t> ident;   // what the graph refers to (see identity())
    };
    std::map<std::string, Entry> graphs;   // keyed by k and the chunk branches
    uint64_t epoch = 0, clock = 0;
    int64_t replays = 0;
    int64_t captures = 0;
};

namespace {


// The server's workspace stands in for the graph's while a batch is issued.
struct WorkspaceSwap {
    tpa_graph *g;
    Workspace *w;
    WorkspaceSwap(tpa_graph *g_, Workspace *w_) : g(g_), w(w_) { std::swap(g->ws, *w); }
    ~WorkspaceSwap() { std::swap(g->ws, *w); }
};

constexpr size_t SERVER_MAX_GRAPHS = 64;

// The launch sequence of a batch of k seeds already in run order in
// srv->seeds with out-degrees od_run (host), pairs in srv->pairs.
void issue_batch(tpa_server *srv, int k, const int32_t *od_run, cudaStream_t s)
{
    tpa_graph *g = srv->g;
    CpiArgs a;
    a.seeds = srv->seeds.as<int32_t>();
    a.k = k;
    a.c = g->c;
    a.eps = g->eps;
    a.s_iter = 0;
    a.t_iter = srv->S - 1;
    a.r_internal = true;
    a.tpa_final = true;
    a.alpha = alpha_of(g->c, srv->S, g->T);
    a.r_str = g->r_str.as<float>();
    a.out = srv->out;
    a.ldo = srv->ldo;
    a.seed_outdeg = od_run;   // the host picks each chunk's branch
    a.no_regroup = true;      // the seeds come regrouped
    a.dev_pairs = srv->pairs.as<int32_t>();
    a.max_pairs = k / 2;
    run_cpi(g, a, s);
}

// Everything a captured batch refers to besides the server's seed and output
// buffers: the device addresses of the workspace in use (a workspace buffer
// that has to grow for a larger batch is reallocated), of the graph's arrays,
// plans and row bins, and the graph's scalars.  A graph captured under another
// identity would touch freed memory, so it is never replayed.
std::vector<uint64_t> identity(const tpa_graph *g)
{
    std::vector<uint64_t> v;
    auto addr = [&v](const DevBuf &b) {
        v.push_back((uint64_t)(uintptr_t)b.p);
        v.push_back((uint64_t)b.bytes);
    };
    const Workspace &w = g->ws;
    for (const DevBuf *b : {&w.x, &w.y, &w.r, &w.carry, &w.head, &w.tl1, &w.fix, &w.ctl, &w.seeds, &w.sets,
                            &w.seeds_g, &w.cols, &w.out, &w.iters, &w.u, &w.touched, &w.x2, &w.cpart, &w.agg, &w.lrec, &w.ltail})
        addr(*b);
    v.push_back((uint64_t)(uintptr_t)w.hflag);
    for (const DevBuf *b : {&g->rp_t, &g->col_t, &g->val_t, &g->rp_a, &g->col_a, &g->val_a, &g->outdeg, &g->inv_deg32,
                            &g->perm_a2t,
                            &g->w_a, &g->inv_d, &g->row_a, &g->r_str})
        addr(*b);
    for (const auto *plans : {&g->plans_t, &g->plans_a})
        for (const auto &kv : *plans) {
            v.push_back((uint64_t)kv.first);
            for (const DevBuf *b : {&kv.second.tile_x, &kv.second.tile_y, &kv.second.head_row, &kv.second.head_first})
                addr(*b);
        }
    for (const SegRows *R : {&g->seg_t, &g->seg_a})
        for (const DevBuf *b : {&R->colf, &R->nz_rows, &R->empty_rows, &R->nzpos, &R->nzrp}) addr(*b);
    for (const auto *tiles : {&g->segt_t, &g->segt_a})
        for (const auto &kv : *tiles) {
            v.push_back((uint64_t)kv.first);
            addr(kv.second.crow0);
        }
    for (const BinPlan *B : {&g->bins_t, &g->bins_a})
        for (const DevBuf *b : {&B->rows_short, &B->rows_mid, &B->rows_long, &B->rows_empty, &B->long_first,
                                &B->chunk_row, &B->chunk_e0})
            addr(*b);
    uint64_t bits;
    memcpy(&bits, &g->c, sizeof bits);
    v.push_back(bits);
    memcpy(&bits, &g->eps, sizeof bits);
    v.push_back(bits);
    v.push_back((uint64_t)g->T);
    v.push_back((uint64_t)g->weighted);
    return v;
}

void drop_graphs(tpa_server *srv)
{
    for (auto &kv : srv->graphs)
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    srv->graphs.clear();
}

// Capture the launch sequence of a batch (the workspace already has its
// sizes for it, so nothing is allocated while capturing).
tpa_server::Entry capture(tpa_server *srv, int k, const int32_t *od_run)
{
    tpa_server::Entry e;
    e.k = k;
    const bool timing = prof_pause();
    const uint64_t l0 = launches_so_far();
    cudaGraph_t graph = nullptr;
    e.ident = identity(srv->g);
    TPA_CUDA(cudaStreamBeginCapture(srv->cap, cudaStreamCaptureModeThreadLocal));
    try {
        issue_batch(srv, k, od_run, srv->cap);
    } catch (...) {
        cudaStreamEndCapture(srv->cap, &graph);
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        prof_resume(timing);
        throw;
    }
    const cudaError_t ce = cudaStreamEndCapture(srv->cap, &graph);
    prof_resume(timing);
    e.launches = (int64_t)(launches_so_far() - l0);
    note_launch_count(-(int)e.launches);   // nothing ran while capturing
    if (ce != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        TPA_CUDA(ce);
    }
    const cudaError_t ie = cudaGraphInstantiate(&e.exec, graph, 0);
    cudaGraphDestroy(graph);
    TPA_CUDA(ie);
    if (identity(srv->g) != e.ident) {   // the direct run sized everything: nothing may move while capturing
        cudaGraphExecDestroy(e.exec);
        set_error("tpa_server_query: a buffer was reallocated while a batch was captured");
        throw Fail{TPA_ECUDA};
    }
    return e;
}

}  // namespace

#define SRV_BEGIN \
    clear_error(); \
    try {
#define SRV_END                                   \
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

extern "C" {

tpa_status tpa_server_create(tpa_graph *g, int S, int max_k, float *out, int64_t ldo, void *stream,
                             tpa_server **srv_out)
{
    SRV_BEGIN
    TPA_REQUIRE(g != nullptr && srv_out != nullptr, "tpa_server_create: NULL argument");
    if (!g->has_pre) {
        set_error("tpa_server_create: the graph is not preprocessed");
        throw Fail{TPA_ESTATE};
    }
    TPA_REQUIRE(S >= 1 && S <= g->T, "tpa_server_create: S = %d outside [1, T = %d]", S, g->T);
    TPA_REQUIRE(max_k >= 1, "tpa_server_create: max_k = %d < 1", max_k);
    TPA_REQUIRE(out == nullptr || is_device_ptr(out), "tpa_server_create: out must be device memory");
    TPA_REQUIRE(out == nullptr || ldo >= max_k, "tpa_server_create: ldo = %lld < max_k = %d", (long long)ldo, max_k);
    cudaStream_t s = (cudaStream_t)stream;
    tpa_server *srv = new tpa_server();
    try {
        srv->g = g;
        srv->S = S;
        srv->max_k = max_k;
        if (out) {
            srv->out = out;
            srv->ldo = ldo;
        } else {
            srv->out_buf.ensure((size_t)g->n * max_k * sizeof(float), s);
            srv->out = srv->out_buf.as<float>();
            srv->ldo = max_k;
        }
        srv->seeds.ensure((size_t)max_k * sizeof(int32_t), s);
        srv->pairs.ensure((size_t)(1 + max_k) * sizeof(int32_t), s);
        TPA_CUDA(cudaMemsetAsync(srv->pairs.p, 0, srv->pairs.bytes, s));
        TPA_CUDA(cudaHostAlloc((void **)&srv->h_seeds, (size_t)max_k * sizeof(int32_t), cudaHostAllocDefault));
        TPA_CUDA(cudaHostAlloc((void **)&srv->h_stage, (size_t)(2 * max_k + 1) * sizeof(int32_t),
                               cudaHostAllocDefault));
        srv->h_outdeg.resize((size_t)g->n);
        TPA_CUDA(cudaMemcpyAsync(srv->h_outdeg.data(), g->outdeg.p, (size_t)g->n * sizeof(int32_t),
                                 cudaMemcpyDeviceToHost, s));
        TPA_CUDA(cudaStreamSynchronize(s));
        TPA_CUDA(cudaEventCreateWithFlags(&srv->staged, cudaEventDisableTiming));
        TPA_CUDA(cudaStreamCreateWithFlags(&srv->cap, cudaStreamNonBlocking));
        srv->epoch = settings_epoch();
    } catch (...) {
        tpa_server_free(srv);
        throw;
    }
    *srv_out = srv;
    SRV_END
}

tpa_status tpa_server_query(tpa_server *srv, const int32_t *seeds, int k, void *stream)
{
    SRV_BEGIN
    TPA_REQUIRE(srv != nullptr && seeds != nullptr, "tpa_server_query: NULL argument");
    TPA_REQUIRE(k >= 1 && k <= srv->max_k, "tpa_server_query: k = %d outside [1, %d]", k, srv->max_k);
    cudaStream_t s = (cudaStream_t)stream;
    tpa_graph *g = srv->g;
    // read and check the ids
    TPA_CUDA(cudaEventSynchronize(srv->staged));
    if (is_device_ptr(seeds)) {
        TPA_CUDA(cudaMemcpyAsync(srv->h_seeds, seeds, (size_t)k * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        TPA_CUDA(cudaStreamSynchronize(s));
    } else {
        memcpy(srv->h_seeds, seeds, (size_t)k * sizeof(int32_t));
    }
    for (int j = 0; j < k; ++j)
        TPA_REQUIRE(srv->h_seeds[j] >= 0 && srv->h_seeds[j] < g->n, "seed %d (index %d) is outside [0, %lld)",
                    srv->h_seeds[j], j, (long long)g->n);
    if (srv->epoch != settings_epoch()) {   // a kernel setting changed: recapture
        TPA_CUDA(cudaStreamSynchronize(s));
        drop_graphs(srv);
        srv->epoch = settings_epoch();
    }
    // run order (heavy seeds into the last chunks, as tpa_query does), the
    // column pairs to swap back, and the chunk branches that key the graph
    std::vector<int32_t> od((size_t)k), perm, od_run((size_t)k);
    for (int j = 0; j < k; ++j) od[j] = srv->h_outdeg[srv->h_seeds[j]];
    regroup_seeds(od.data(), k, srv->S, perm);
    int32_t *st_seeds = srv->h_stage, *st_pairs = srv->h_stage + srv->max_k;
    int np = 0;
    for (int j = 0; j < k; ++j) {
        st_seeds[j] = srv->h_seeds[perm[j]];
        od_run[j] = od[perm[j]];
        if (perm[j] > j) {
            st_pairs[1 + 2 * np] = j;
            st_pairs[2 + 2 * np] = perm[j];
            ++np;
        }
    }
    st_pairs[0] = np;
    TPA_REQUIRE(np <= k / 2, "tpa_server_query: internal: %d column pairs for %d seeds", np, k);
    TPA_CUDA(cudaMemcpyAsync(srv->seeds.p, st_seeds, (size_t)k * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    TPA_CUDA(cudaMemcpyAsync(srv->pairs.p, st_pairs, (size_t)(1 + 2 * np) * sizeof(int32_t),
                             cudaMemcpyHostToDevice, s));
    TPA_CUDA(cudaEventRecord(srv->staged, s));
    const std::string key = std::to_string(k) + ":" + query_branches(od_run.data(), k, srv->S);

    WorkspaceSwap swap(g, &srv->ws);
    auto it = srv->graphs.find(key);
    if (it != srv->graphs.end() && it->second.ident != identity(g)) {
        TPA_CUDA(cudaStreamSynchronize(s));
        drop_graphs(srv);                       // stale: they refer to reallocated buffers
        it = srv->graphs.end();
    }
    if (it == srv->graphs.end()) {
        issue_batch(srv, k, od_run.data(), s);  // this batch's answer; sizes the workspace for it
        TPA_CUDA(cudaStreamSynchronize(s));     // the capture must not race the direct run
        const std::vector<uint64_t> now = identity(g);
        for (auto e = srv->graphs.begin(); e != srv->graphs.end();) {   // a buffer grew: older graphs are stale
            if (e->second.ident != now) {
                cudaGraphExecDestroy(e->second.exec);
                e = srv->graphs.erase(e);
            } else {
                ++e;
            }
        }
        if (srv->graphs.size() >= SERVER_MAX_GRAPHS) {   // evict the least recently used
            auto lru = srv->graphs.begin();
            for (auto e = srv->graphs.begin(); e != srv->graphs.end(); ++e)
                if (e->second.used < lru->second.used) lru = e;
            cudaGraphExecDestroy(lru->second.exec);
            srv->graphs.erase(lru);
        }
        tpa_server::Entry e = capture(srv, k, od_run.data());
        e.used = ++srv->clock;
        srv->graphs[key] = std::move(e);
        ++srv->captures;
    } else {
        TPA_CUDA(cudaGraphLaunch(it->second.exec, s));
        it->second.used = ++srv->clock;
        note_launch_count((int)it->second.launches);
        ++srv->replays;
    }
    SRV_END
}

tpa_status tpa_server_result(const tpa_server *srv, float **out, int64_t *ldo)
{
    SRV_BEGIN
    TPA_REQUIRE(srv != nullptr, "tpa_server_result: NULL server");
    if (out) *out = srv->out;
    if (ldo) *ldo = srv->ldo;
    SRV_END
}

tpa_status tpa_server_sync(tpa_server *srv, void *stream)
{
    SRV_BEGIN
    TPA_REQUIRE(srv != nullptr, "tpa_server_sync: NULL server");
    cudaStream_t s = (cudaStream_t)stream;
    TPA_CUDA(cudaStreamSynchronize(s));
    if (srv->ws.ctl.p) {
        int32_t *flag = &static_cast<Ctl *>(srv->ws.ctl.p)->error;
        int32_t e = 0;
        TPA_CUDA(cudaMemcpyAsync(&e, flag, sizeof e, cudaMemcpyDeviceToHost, s));
        TPA_CUDA(cudaStreamSynchronize(s));
        if (e) {
            TPA_CUDA(cudaMemsetAsync(flag, 0, sizeof e, s));
            TPA_CUDA(cudaStreamSynchronize(s));
            set_error("a bounded device wait gave up: the batches since the last check are not valid");
            throw Fail{TPA_ETIMEOUT};
        }
    }
    SRV_END
}

tpa_status tpa_server_stats(const tpa_server *srv, int k, int64_t *graphs, int64_t *replays,
                            int64_t *launches_per_replay, int64_t *captures)
{
    SRV_BEGIN
    TPA_REQUIRE(srv != nullptr, "tpa_server_stats: NULL server");
    if (graphs) *graphs = (int64_t)srv->graphs.size();
    if (replays) *replays = srv->replays;
    if (launches_per_replay) {   // the most recently used graph for batches of k seeds
        const tpa_server::Entry *best = nullptr;
        for (const auto &kv : srv->graphs)
            if (kv.second.k == k && (!best || kv.second.used > best->used)) best = &kv.second;
        *launches_per_replay = best ? best->launches : 0;
    }
    if (captures) *captures = srv->captures;
    SRV_END
}

void tpa_server_free(tpa_server *srv)
{
    if (!srv) return;
    cudaDeviceSynchronize();
    drop_graphs(srv);
    cudaStream_t s = 0;
    DevBuf *bufs[] = {&srv->out_buf, &srv->seeds, &srv->pairs, &srv->ws.x, &srv->ws.y, &srv->ws.r, &srv->ws.carry,
                      &srv->ws.head, &srv->ws.tl1, &srv->ws.fix, &srv->ws.ctl, &srv->ws.seeds, &srv->ws.sets,
                      &srv->ws.seeds_g, &srv->ws.cols, &srv->ws.out,
                      &srv->ws.iters, &srv->ws.u, &srv->ws.touched, &srv->ws.x2, &srv->ws.cpart, &srv->ws.agg};
    for (DevBuf *b : bufs) b->release(s);
    if (srv->ws.hflag) cudaFreeHost(srv->ws.hflag);
    if (srv->h_seeds) cudaFreeHost(srv->h_seeds);
    if (srv->h_stage) cudaFreeHost(srv->h_stage);
    if (srv->staged) cudaEventDestroy(srv->staged);
    if (srv->cap) cudaStreamDestroy(srv->cap);
    cudaDeviceSynchronize();
    trim_pool();
    delete srv;
}

}  // extern "C"
