// Cumulative power iteration (Algorithm 1) on the GPU: the host side that
// plans and launches it.  The kernels are in spmm_kernels.cuh (merge path)
// and spmm_binned.cuh (rows binned by length).
//
// One iteration computes x_i = (1-c) A~^T x_{i-1} for a chunk of k columns
// (node-major X[n][KP], KP = k padded to a power of two) with a merge-path
// SpMM over CSR(A~^T): the path interleaves the n row ends with the m
// nonzeros and is cut into equal tiles, so rows of hubs cost no imbalance.
// Several kernel variants exist per KP (warp walker, pipelined group walker,
// CTA walker, binned rows); the first of each width in kVariants is the
// default, and the autotuner or tpa_set_variant may pick another.  Each
// SpMM launch fuses the epilogue of Algorithm 1 (y stored, r += y for
// running columns, FP32 L1 partials of y) or, on the last family iteration
// of Algorithm 3, the finalize out = (1+alpha)(r + y) + r~_stranger.  A
// fixup kernel then finishes the rows split across tiles, adds the L1
// partials in a fixed order (FP64 across blocks) and applies the break test
// ||x_i||_1 < eps per column.  Tile orders are static, so results are
// deterministic run to run.
//
// Around the SpMM: query chunks of light seeds push x1 and x2 along CSR(A~)
// instead of pulling them (the host or, in captured launch sequences, the
// device picks the branch); unweighted graphs use pattern-only products
// (the iterate is kept scaled by 1/outdeg and the value array is not read);
// and a query whose scores go to device memory moves its seeds too heavy to
// push into its last chunks, swapping their columns back at the end.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <atomic>
#include <cstddef>
#include <cstring>
#include <cmath>
#include <numeric>
#include <string>
#include <vector>

#include "tpa_internal.cuh"

#include "spmm_kernels.cuh"
#include "spmm_binned.cuh"
#include "spmm_seg.cuh"
#include "spmm_lane.cuh"

namespace tpa {

static unsigned grid_1d(int64_t work, int threads)
{
    const int64_t b = (work + threads - 1) / threads;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 32));
}

const Plan &get_plan(tpa_graph *g, int L, cudaStream_t s, int which)
{
    std::map<int, Plan> &plans = which ? g->plans_a : g->plans_t;
    const int64_t *rp = which ? g->rp_a.as<int64_t>() : g->rp_t.as<int64_t>();
    auto it = plans.find(L);
    if (it != plans.end()) return it->second;
    Plan &P = plans[L];
    P.L = L;
    P.tiles = std::max<int64_t>(1, (g->n + g->m + L - 1) / L);
    TPA_REQUIRE(P.tiles < INT32_MAX, "merge-path plan: too many tiles");
    P.tile_x.ensure((size_t)(P.tiles + 1) * sizeof(int32_t), s);
    P.tile_y.ensure((size_t)(P.tiles + 1) * sizeof(int64_t), s);
    P.head_row.ensure((size_t)P.tiles * sizeof(int32_t), s);
    P.head_first.ensure((size_t)P.tiles * sizeof(int32_t), s);
    plan_tiles_k<<<grid_1d(P.tiles + 1, 256), 256, 0, s>>>(rp, g->n, g->m, L, P.tiles,
                                                            P.tile_x.as<int32_t>(), P.tile_y.as<int64_t>());
    plan_heads_k<<<grid_1d(P.tiles, 256), 256, 0, s>>>(rp, P.tile_x.as<int32_t>(),
                                                       P.tile_y.as<int64_t>(), P.tiles, P.head_row.as<int32_t>(),
                                                       P.head_first.as<int32_t>());
    note_launch("plan", 2);
    TPA_CHECK_LAUNCH();
    return P;
}

// Row bins of CSR(A~^T) (which = 0) or CSR(A~) for the binned-row kernels.
static const BinPlan &get_bin_plan(tpa_graph *g, int which, cudaStream_t s)
{
    BinPlan &B = which ? g->bins_a : g->bins_t;
    if (B.built) return B;
    const int64_t n = g->n;
    const int64_t *rp = which ? g->rp_a.as<int64_t>() : g->rp_t.as<int64_t>();
    DevBuf flags, pos, tmp, cnt;
    flags.ensure((size_t)4 * n * sizeof(int32_t), s);
    pos.ensure((size_t)4 * (n + 1) * sizeof(int64_t), s);
    bin_classify_k<<<grid_1d(n, 256), 256, 0, s>>>(rp, n, flags.as<int32_t>());
    TPA_CHECK_LAUNCH();
    for (int b = 0; b < 4; ++b)
        exclusive_scan_i32_i64(flags.as<int32_t>() + b * n, pos.as<int64_t>() + b * (n + 1), n, tmp, s);
    int64_t tot[4];
    for (int b = 0; b < 4; ++b)
        TPA_CUDA(cudaMemcpyAsync(&tot[b], pos.as<int64_t>() + b * (n + 1) + n, sizeof(int64_t),
                                 cudaMemcpyDeviceToHost, s));
    TPA_CUDA(cudaStreamSynchronize(s));
    B.n_short = tot[0];
    B.n_mid = tot[1];
    B.n_long = tot[2];
    B.n_empty = tot[3];
    B.rows_short.ensure((size_t)std::max<int64_t>(1, B.n_short) * sizeof(int32_t), s);
    B.rows_mid.ensure((size_t)std::max<int64_t>(1, B.n_mid) * sizeof(int32_t), s);
    B.rows_long.ensure((size_t)std::max<int64_t>(1, B.n_long) * sizeof(int32_t), s);
    B.rows_empty.ensure((size_t)std::max<int64_t>(1, B.n_empty) * sizeof(int32_t), s);
    cnt.ensure((size_t)std::max<int64_t>(1, B.n_long) * sizeof(int32_t), s);
    bin_scatter_k<<<grid_1d(n, 256), 256, 0, s>>>(rp, n, flags.as<int32_t>(), pos.as<int64_t>(),
                                                   B.rows_short.as<int32_t>(), B.rows_mid.as<int32_t>(),
                                                   B.rows_long.as<int32_t>(), B.rows_empty.as<int32_t>(),
                                                   cnt.as<int32_t>());
    TPA_CHECK_LAUNCH();
    B.long_first.ensure((size_t)(B.n_long + 1) * sizeof(int64_t), s);
    exclusive_scan_i32_i64(cnt.as<int32_t>(), B.long_first.as<int64_t>(), B.n_long, tmp, s);
    TPA_CUDA(cudaMemcpyAsync(&B.n_chunks, B.long_first.as<int64_t>() + B.n_long, sizeof(int64_t),
                             cudaMemcpyDeviceToHost, s));
    TPA_CUDA(cudaStreamSynchronize(s));
    B.chunk_row.ensure((size_t)std::max<int64_t>(1, B.n_chunks) * sizeof(int32_t), s);
    B.chunk_e0.ensure((size_t)std::max<int64_t>(1, B.n_chunks) * sizeof(int64_t), s);
    if (B.n_long)
        bin_chunks_k<<<grid_1d(B.n_long, 256), 256, 0, s>>>(rp, B.rows_long.as<int32_t>(), B.n_long,
                                                             B.long_first.as<int64_t>(), B.chunk_row.as<int32_t>(),
                                                             B.chunk_e0.as<int64_t>());
    note_launch("plan", 3 + (B.n_long ? 1 : 0));
    TPA_CHECK_LAUNCH();
    flags.release(s);
    pos.release(s);
    tmp.release(s);
    cnt.release(s);
    B.built = true;
    return B;
}

// Flag-walk data of CSR(A~^T) (which = 0) or CSR(A~), built once per graph.
static const SegRows &get_seg_rows(tpa_graph *g, int which, cudaStream_t s)
{
    SegRows &R = which ? g->seg_a : g->seg_t;
    if (R.built) return R;
    const int64_t n = g->n, m = g->m;
    const int64_t *rp = which ? g->rp_a.as<int64_t>() : g->rp_t.as<int64_t>();
    const int32_t *col = which ? g->col_a.as<int32_t>() : g->col_t.as<int32_t>();
    DevBuf nzf, ef, epos, tmp;
    nzf.ensure((size_t)n * sizeof(int32_t), s);
    ef.ensure((size_t)n * sizeof(int32_t), s);
    R.nzpos.ensure((size_t)(n + 1) * sizeof(int64_t), s);
    epos.ensure((size_t)(n + 1) * sizeof(int64_t), s);
    seg_row_flags_k<<<grid_1d(n, 256), 256, 0, s>>>(rp, n, nzf.as<int32_t>(), ef.as<int32_t>());
    TPA_CHECK_LAUNCH();
    exclusive_scan_i32_i64(nzf.as<int32_t>(), R.nzpos.as<int64_t>(), n, tmp, s);
    exclusive_scan_i32_i64(ef.as<int32_t>(), epos.as<int64_t>(), n, tmp, s);
    int64_t cnt[2];
    TPA_CUDA(cudaMemcpyAsync(&cnt[0], R.nzpos.as<int64_t>() + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    TPA_CUDA(cudaMemcpyAsync(&cnt[1], epos.as<int64_t>() + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    TPA_CUDA(cudaStreamSynchronize(s));
    R.n_nz = cnt[0];
    R.n_empty = cnt[1];
    R.nz_rows.ensure((size_t)std::max<int64_t>(1, R.n_nz) * sizeof(int32_t), s);
    R.empty_rows.ensure((size_t)std::max<int64_t>(1, R.n_empty) * sizeof(int32_t), s);
    seg_scatter_rows_k<<<grid_1d(n, 256), 256, 0, s>>>(rp, n, R.nzpos.as<int64_t>(), epos.as<int64_t>(),
                                                       R.nz_rows.as<int32_t>(), R.empty_rows.as<int32_t>());
    TPA_CHECK_LAUNCH();
    R.padded = (m + SEG_MAX_TN - 1) / SEG_MAX_TN * SEG_MAX_TN + SEG_MAX_TN;
    R.colf.ensure((size_t)R.padded * sizeof(uint32_t), s);
    seg_copy_cols_k<<<grid_1d(R.padded, 256), 256, 0, s>>>(col, m, R.padded, R.colf.as<uint32_t>());
    seg_mark_k<<<grid_1d(n, 256), 256, 0, s>>>(rp, n, R.colf.as<uint32_t>());
    note_launch("plan", 5);
    TPA_CHECK_LAUNCH();
    TPA_CUDA(cudaStreamSynchronize(s));
    nzf.release(s);
    ef.release(s);
    epos.release(s);
    tmp.release(s);
    R.built = true;
    return R;
}

// Tiles of tn nonzeros over CSR(A~^T) (which = 0) or CSR(A~).
static const SegTiles &get_seg_tiles(tpa_graph *g, int which, int64_t tn, cudaStream_t s)
{
    TPA_REQUIRE(tn >= 32 && tn <= SEG_MAX_TN, "segmented walk: tile of %lld nonzeros", (long long)tn);
    std::map<int, SegTiles> &M = which ? g->segt_a : g->segt_t;
    auto it = M.find((int)tn);
    if (it != M.end()) return it->second;
    const SegRows &R = get_seg_rows(g, which, s);
    const int64_t *rp = which ? g->rp_a.as<int64_t>() : g->rp_t.as<int64_t>();
    SegTiles &T = M[(int)tn];
    T.tn = tn;
    T.tiles = (g->m + tn - 1) / tn;
    TPA_REQUIRE(T.tiles * tn <= R.padded, "segmented walk: column copy too short");
    T.crow0.ensure((size_t)(T.tiles + 1) * sizeof(int32_t), s);
    seg_tiles_k<<<grid_1d(T.tiles + 1, 256), 256, 0, s>>>(rp, g->n, g->m, R.nzpos.as<int64_t>(), tn, T.tiles,
                                                          T.crow0.as<int32_t>());
    note_launch("plan");
    TPA_CHECK_LAUNCH();
    return T;
}

// Point the flag-walk fields of p at the data of a CSR; sizes the carry-out
// words of the workspace for kp columns (zeroed whenever allocated).
static void bind_seg(Params &p, tpa_graph *g, int which, int64_t tn, int kp, cudaStream_t s)
{
    const SegRows &R = get_seg_rows(g, which, s);
    const SegTiles &T = get_seg_tiles(g, which, tn, s);
    Workspace &W = g->ws;
    const size_t agg_bytes = (size_t)std::max<int64_t>(1, T.tiles) * kp * sizeof(unsigned long long);
    if (!W.agg.p || W.agg.bytes < agg_bytes) {
        W.agg.ensure(agg_bytes, s);
        TPA_CUDA(cudaMemsetAsync(W.agg.p, 0, W.agg.bytes, s));
    }
    need(W.agg, (size_t)T.tiles * kp * sizeof(unsigned long long), "carry-out words");
    need(R.colf, (size_t)T.tiles * tn * sizeof(uint32_t), "flagged columns");
    TPA_REQUIRE(T.tiles * tn <= csr_len(g->m), "segmented walk: value array shorter than the tiles");
    p.colf = R.colf.as<uint32_t>();
    p.nz_rows = R.nz_rows.as<int32_t>();
    p.empty_rows = R.empty_rows.as<int32_t>();
    p.n_empty = R.n_empty;
    p.tile_crow0 = T.crow0.as<int32_t>();
    p.seg_tiles = T.tiles;
    p.m = g->m;
    p.agg = W.agg.as<unsigned long long>();
}

// Point the binned-row fields of p at the bins of a CSR (and the chunk sums).
static void bind_bins(Params &p, tpa_graph *g, int which, int KP, cudaStream_t s)
{
    const BinPlan &B = get_bin_plan(g, which, s);
    p.rows_short = B.rows_short.as<int32_t>();
    p.rows_mid = B.rows_mid.as<int32_t>();
    p.rows_long = B.rows_long.as<int32_t>();
    p.rows_empty = B.rows_empty.as<int32_t>();
    p.chunk_row = B.chunk_row.as<int32_t>();
    p.chunk_e0 = B.chunk_e0.as<int64_t>();
    p.n_short = B.n_short;
    p.n_mid = B.n_mid;
    p.n_long = B.n_long;
    p.n_empty = B.n_empty;
    p.n_chunks = B.n_chunks;
    p.long_first64 = B.long_first.as<int64_t>();
    g->ws.cpart.ensure((size_t)std::max<int64_t>(1, B.n_chunks) * KP * sizeof(float), s);
    p.cpart = g->ws.cpart.as<float>();
}

// --------------------------------------------------------- dispatching ---
struct KCfg {
    int G, V, ITEMS, PF;
    int NT;   // threads per CTA
    int KP() const { return G * V; }
    int L() const { return (NT / G) * ITEMS; }
};

typedef void (*SpmmFn)(Params);
typedef void (*FixFn)(Params);

static int num_sms()
{
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        TPA_CUDA(cudaGetDevice(&dev));
        TPA_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    }
    return sms;
}

// Persistent grid: resident CTAs per SM x SMs, capped by the tile count.
template <int G, int V, int ITEMS, int PF>
static int64_t launch_spmm(const Params &p, cudaStream_t s)
{
    static int per_sm = 0;
    if (!per_sm) {
        TPA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, spmm_tile_k<G, V, ITEMS, PF>, CTA, 0));
        per_sm = std::max(per_sm, 1);
    }
    const int64_t grid = std::min<int64_t>(p.tiles, (int64_t)per_sm * num_sms());
    spmm_tile_k<G, V, ITEMS, PF><<<(unsigned)grid, CTA, 0, s>>>(p);
    return p.tiles;
}

template <int V, int ITEMS, int WARPS>
static int64_t launch_spmvw(const Params &p, cudaStream_t s)
{
    static int per_sm = 0;
    if (!per_sm) {
        TPA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, spmvw_tile_k<V, ITEMS, WARPS>, WARPS * 32, 0));
        per_sm = std::max(per_sm, 1);
    }
    const int64_t grid = std::min<int64_t>((p.tiles + WARPS - 1) / WARPS, (int64_t)per_sm * num_sms());
    spmvw_tile_k<V, ITEMS, WARPS><<<(unsigned)grid, WARPS * 32, 0, s>>>(p);
    return p.tiles;
}

template <int G, int V, int ITEMS, int PF, int WARPS>
static int64_t launch_spmvg(const Params &p, cudaStream_t s)
{
    static int per_sm = 0;
    if (!per_sm) {
        TPA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, spmvg_tile_k<G, V, ITEMS, PF, WARPS>,
                                                               WARPS * 32, 0));
        per_sm = std::max(per_sm, 1);
    }
    const int64_t grid = std::min<int64_t>((p.tiles + WARPS - 1) / WARPS, (int64_t)per_sm * num_sms());
    spmvg_tile_k<G, V, ITEMS, PF, WARPS><<<(unsigned)grid, WARPS * 32, 0, s>>>(p);
    return p.tiles;
}

// Returns the rows of tl1 written: one per warp of the grid (at most
// tiles + 7, the size the workspace reserves).
// Cooperative launch of a persistent grid (kernels whose CTAs wait on one
// another): the driver starts every CTA at once or refuses, and a refused
// grid is halved until it fits.
static int64_t launch_cooperative(void (*kern)(Params), const Params &p, int64_t grid, unsigned threads,
                                  size_t smem, cudaStream_t s)
{
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof cfg);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    for (;;) {
        cfg.gridDim = dim3((unsigned)grid);
        const cudaError_t e = cudaLaunchKernelEx(&cfg, kern, p);
        if (e == cudaSuccess) return grid;
        if (e != cudaErrorCooperativeLaunchTooLarge || grid == 1) TPA_CUDA(e);
        cudaGetLastError();
        grid = (grid + 1) / 2;
    }
}

// FUSE: the pipelined kernel that finishes its deferred rows itself (no
// fixup), launched cooperatively; returns the CTAs launched.  Otherwise the
// rows of tl1 written (one per warp).
template <int G, int V, int ITEMS, int PF, int WARPS, int MINB, bool FUSE = false>
static int64_t launch_spmvp(const Params &p, cudaStream_t s)
{
    // one instantiation per product mode, so the valued kernel carries no test of it
    constexpr size_t smem_v = WARPS * PipeSmem<G, V, ITEMS, false>::PER_WARP;
    constexpr size_t smem_p = WARPS * PipeSmem<G, V, ITEMS, true>::PER_WARP;
    static_assert(smem_v <= 227 * 1024 && smem_p <= 227 * 1024, "shared memory per block");
    auto *const valued = spmvp_tile_k<G, V, ITEMS, PF, WARPS, MINB, false, FUSE>;
    auto *const pattern = spmvp_tile_k<G, V, ITEMS, PF, WARPS, MINB, true, FUSE>;
    static int per_sm_v = 0, per_sm_p = 0;
    if (!per_sm_v) {
        TPA_CUDA(cudaFuncSetAttribute(valued, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_v));
        TPA_CUDA(cudaFuncSetAttribute(pattern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_p));
        TPA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_v, valued, WARPS * 32, smem_v));
        TPA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_p, pattern, WARPS * 32, smem_p));
        per_sm_v = std::max(per_sm_v, 1);
        per_sm_p = std::max(per_sm_p, 1);
    }
    const int per_sm = p.inv_deg ? per_sm_p : per_sm_v;
    const int64_t grid =
        std::max<int64_t>(1, std::min<int64_t>((p.tiles + WARPS - 1) / WARPS, (int64_t)per_sm * num_sms()));
    if constexpr (FUSE) {
        return launch_cooperative(p.inv_deg ? pattern : valued, p, grid, WARPS * 32, p.inv_deg ? smem_p : smem_v, s);
    } else {
        if (p.inv_deg) pattern<<<(unsigned)grid, WARPS * 32, smem_p, s>>>(p);
        else valued<<<(unsigned)grid, WARPS * 32, smem_v, s>>>(p);
        return grid * WARPS;
    }
}

// Segmented flag walk (spmm_seg.cuh; AHEAD: the gathers-ahead kernel):
// persistent grid of at most the kernel's occupancy times the SM count,
// launched cooperatively (its waits need every CTA resident); returns the
// CTAs launched (rows of the L1 partial buffer).
template <int V, int R, int PF, int NB, bool AHEAD>
static int64_t launch_seg(const Params &p, cudaStream_t s)
{
    constexpr size_t smem_v = AHEAD ? SegaSmem<V, R, NB, false>::BYTES : SegSmem<V, R, NB, false>::BYTES;
    constexpr size_t smem_p = AHEAD ? SegaSmem<V, R, NB, true>::BYTES : SegSmem<V, R, NB, true>::BYTES;
    static_assert(smem_v <= 200 * 1024 && smem_p <= 200 * 1024, "shared memory per block");
    void (*valued)(Params), (*pattern)(Params);
    if constexpr (AHEAD) {
        valued = spmm_sega_k<V, R, PF, NB, false>;
        pattern = spmm_sega_k<V, R, PF, NB, true>;
    } else {
        valued = spmm_seg_k<V, R, PF, NB, false>;
        pattern = spmm_seg_k<V, R, PF, NB, true>;
    }
    static int per_sm_v = 0, per_sm_p = 0;
    if (!per_sm_v) {
        TPA_CUDA(cudaFuncSetAttribute(valued, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_v));
        TPA_CUDA(cudaFuncSetAttribute(pattern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_p));
        TPA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_v, valued, SEG_WARPS * 32, smem_v));
        TPA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_p, pattern, SEG_WARPS * 32, smem_p));
        TPA_REQUIRE(per_sm_v >= 1 && per_sm_p >= 1, "segmented walk: the kernel does not fit on an SM");
        // ask for the shared-memory share those CTAs need (the rest stays L1)
        for (int k = 0; k < 2; ++k) {
            const size_t need = (size_t)(k ? per_sm_p : per_sm_v) * ((k ? smem_p : smem_v) + 3 * 1024);
            const int pct = (int)std::min<size_t>(100, (need * 100 + 228 * 1024 - 1) / (228 * 1024));
            TPA_CUDA(cudaFuncSetAttribute(k ? pattern : valued, cudaFuncAttributePreferredSharedMemoryCarveout, pct));
        }
    }
    const bool pat = p.inv_deg != nullptr;
    const int per_sm = pat ? per_sm_p : per_sm_v;
    int64_t grid =
        std::max<int64_t>(1, std::min<int64_t>((p.seg_tiles + SEG_WARPS - 1) / SEG_WARPS, (int64_t)per_sm * num_sms()));
    return launch_cooperative(pat ? pattern : valued, p, grid, SEG_WARPS * 32, pat ? smem_p : smem_v, s);
}

// Upper bound of the CTAs of any persistent grid (32 resident blocks per SM at most).
static int64_t seg_grid_bound() { return (int64_t)32 * num_sms(); }

// Lane-segment walk (spmm_lane.cuh): the walk over segments of R nonzeros,
// then the finishing launch (rows, epilogue, L1, break test) in the fixup's
// place; returns the CTAs of the walk.
template <int V, int R, int PF>
static int64_t launch_lane(const Params &p, cudaStream_t s)
{
    auto *const valued = spmm_lane_k<V, R, PF, false>;
    auto *const pattern = spmm_lane_k<V, R, PF, true>;
    static int per_sm_v = 0, per_sm_p = 0;
    if (!per_sm_v) {
        TPA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_v, valued, 256, 0));
        TPA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_p, pattern, 256, 0));
        per_sm_v = std::max(per_sm_v, 1);
        per_sm_p = std::max(per_sm_p, 1);
    }
    const int per_sm = p.inv_deg ? per_sm_p : per_sm_v;
    const int64_t grid =
        std::max<int64_t>(1, std::min<int64_t>((p.seg_tiles + 255) / 256, (int64_t)per_sm * num_sms()));
    if (p.inv_deg) pattern<<<(unsigned)grid, 256, 0, s>>>(p);
    else valued<<<(unsigned)grid, 256, 0, s>>>(p);
    return grid;
}

template <int V, int R>
static void launch_lane_finish(const Params &p, unsigned, cudaStream_t s)
{
    const int64_t rows = std::max<int64_t>(1, p.n - p.n_empty);
    const unsigned grid = (unsigned)std::min<int64_t>((rows + 255) / 256, (int64_t)8 * num_sms());
    lane_finish_k<V, R><<<grid, 256, 0, s>>>(p);
}

// Binned-row kernels (spmm_binned.cuh): short, medium, chunks of long rows,
// long-row combine, empty rows; returns the rows of tl1 written.
template <int KP>
static int64_t launch_binned(const Params &p0, cudaStream_t s)
{
    static int per_short = 0, per_mid = 0, per_chunk = 0;
    if (!per_short) {
        TPA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_short, bin_short_k<KP>, BIN_WARPS * 32, 0));
        TPA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_mid, bin_warp_k<KP, false>, BIN_WARPS * 32, 0));
        TPA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_chunk, bin_warp_k<KP, true>, BIN_WARPS * 32, 0));
        per_short = std::max(per_short, 1);
        per_mid = std::max(per_mid, 1);
        per_chunk = std::max(per_chunk, 1);
    }
    const int64_t sms = num_sms();
    auto blocks = [&](int64_t warps, int per) {
        return (unsigned)std::max<int64_t>(1, std::min<int64_t>((warps + BIN_WARPS - 1) / BIN_WARPS, per * sms));
    };
    Params p = p0;
    constexpr int RPW = 32 / (KP < 32 ? KP : 32);
    int64_t slot = 0;
    const unsigned gs = blocks((p.n_short + RPW - 1) / RPW, per_short);
    p.slot0 = slot;
    bin_short_k<KP><<<gs, BIN_WARPS * 32, 0, s>>>(p);
    slot += (int64_t)gs * BIN_WARPS;
    const unsigned gm = blocks(p.n_mid, per_mid);
    p.slot0 = slot;
    bin_warp_k<KP, false><<<gm, BIN_WARPS * 32, 0, s>>>(p);
    slot += (int64_t)gm * BIN_WARPS;
    int launches = 2;
    if (p.n_chunks) {
        bin_warp_k<KP, true><<<blocks(p.n_chunks, per_chunk), BIN_WARPS * 32, 0, s>>>(p);
        const unsigned gl = (unsigned)((p.n_long * KP + 255) / 256);
        p.slot0 = slot;
        bin_long_k<KP><<<gl, 256, 0, s>>>(p);
        slot += gl;
        launches += 2;
    }
    if (p.n_empty) {
        bin_empty_k<KP><<<grid_1d(p.n_empty * KP, 256), 256, 0, s>>>(p);
        ++launches;
    }
    note_launch_count(launches - 1);   // the caller counts one
    TPA_CHECK_LAUNCH();
    return slot;
}

// Upper bound of the tl1 rows launch_binned writes.
static int64_t binned_slots_bound(int64_t n_long, int KP)
{
    return 2 * (int64_t)32 * num_sms() * BIN_WARPS + (n_long * KP + 255) / 256 + 1;
}

template <int KP>
static void launch_bin_finish(const Params &p, unsigned blocks, cudaStream_t s)
{
    (void)blocks;
    bin_finish_k<KP><<<1, 256, 0, s>>>(p);
}

template <int KP>
static void launch_fix(const Params &p, unsigned blocks, cudaStream_t s)
{
    if constexpr (KP <= 8) {
        fixup_small_k<KP><<<blocks, 256, 0, s>>>(p);
    } else {
        fixup_k<KP><<<blocks, FIX_WARPS * 32, 0, s>>>(p);
    }
}

// Blocks of the fixup grid (the L1 partial buffer holds one row per block);
// the narrow fixup runs a persistent grid of FIX_SMALL_PER_SM blocks per SM.
constexpr int FIX_SMALL_PER_SM = 4;
static unsigned fix_grid(int KP, int64_t tiles)
{
    if (KP <= 8)
        return (unsigned)std::max<int64_t>(
            1, std::min<int64_t>((tiles + 255) / 256, (int64_t)FIX_SMALL_PER_SM * num_sms()));
    return (unsigned)std::min<int64_t>((tiles + FIX_WARPS - 1) / FIX_WARPS, (int64_t)4 * num_sms());
}

struct Variant {
    KCfg cfg;
    int64_t (*spmm)(const Params &, cudaStream_t);   // returns the rows of tl1 written
    void (*fix)(const Params &, unsigned, cudaStream_t);
    const char *name;
    bool binned = false;   // binned-row kernels (need the row bins bound to Params)
    bool seg = false;      // segmented flag walk: no fixup; tiles of cfg.L() nonzeros
    bool lane = false;     // lane-segment walk (with seg): segments of cfg.L() nonzeros, a finishing launch
};

#define TPA_VARIANT(G, V, I, PF) \
    {{G, V, I, PF, CTA}, launch_spmm<G, V, I, PF>, launch_fix<G * V>, "cta<" #G "," #V "," #I "," #PF ">"}
#define TPA_VARIANTW(V, I, W) \
    {{1, V, I, I, 32}, launch_spmvw<V, I, W>, launch_fix<V>, "warp<" #V "," #I "," #W ">"}
#define TPA_VARIANTG(G, V, I, PF) \
    {{G, V, I, PF, 32}, launch_spmvg<G, V, I, PF, 8>, launch_fix<G * V>, "walker<" #G "," #V "," #I "," #PF ">"}
#define TPA_VARIANTB(KP) {{1, KP, 4, 4, 32}, launch_binned<KP>, launch_bin_finish<KP>, "bins<" #KP ">", true}
#define TPA_VARIANTS(V, R, PF, NB) \
    {{1, V, R, PF, 32}, launch_seg<V, R, PF, NB, false>, nullptr, "seg<" #V "," #R "," #PF "," #NB ">", false, true}
#define TPA_VARIANTL(V, R, PF) \
    {{1, V, R, PF, 1}, launch_lane<V, R, PF>, launch_lane_finish<V, R>, "lane<" #V "," #R "," #PF ">", false, true, true}
#define TPA_VARIANTA(V, R, PF, NB) \
    {{1, V, R, PF, 32}, launch_seg<V, R, PF, NB, true>, nullptr, "sega<" #V "," #R "," #PF "," #NB ">", false, true}
#define TPA_VARIANTPF(G, V, I, PF, W, MB)                                \
    {{G, V, I, PF, 32}, launch_spmvp<G, V, I, PF, W, MB, true>, nullptr, \
     "pipef<" #G "," #V "," #I "," #PF "," #W "," #MB ">"}
#define TPA_VARIANTP(G, V, I, PF, W, MB)                                 \
    {{G, V, I, PF, 32}, launch_spmvp<G, V, I, PF, W, MB>, launch_fix<G * V>, \
     "pipe<" #G "," #V "," #I "," #PF "," #W "," #MB ">"}
// The first variant of each padded width is its default (the fastest measured
// on R-MAT scale 22 queries); the autotuner may pick any other.
static const Variant kVariants[] = {
    TPA_VARIANTL(1, 32, 8),
    TPA_VARIANTL(2, 32, 8),
    TPA_VARIANTL(4, 32, 4),
    TPA_VARIANTL(8, 32, 4),
    TPA_VARIANTW(1, 6, 8),
    TPA_VARIANTW(2, 6, 8),
    TPA_VARIANTP(1, 4, 4, 4, 8, 1),
    TPA_VARIANTP(2, 4, 8, 8, 4, 5),
    TPA_VARIANTP(4, 4, 8, 8, 4, 1),
    TPA_VARIANTS(1, 8, 8, 3),
    TPA_VARIANTS(2, 8, 8, 3),
    TPA_VARIANTS(4, 8, 8, 3),
    TPA_VARIANTPF(2, 4, 8, 8, 4, 5),
    TPA_VARIANTL(8, 32, 2),
    TPA_VARIANTS(8, 8, 4, 2),
    TPA_VARIANTS(1, 4, 4, 4),
    TPA_VARIANTS(8, 8, 8, 2),
    TPA_VARIANTA(1, 8, 8, 2),
    TPA_VARIANTA(2, 8, 8, 2),
    TPA_VARIANTA(4, 8, 8, 2),
    TPA_VARIANTA(8, 8, 4, 2),
    TPA_VARIANT(8, 4, 16, 8),
    TPA_VARIANT(16, 4, 16, 8),
    TPA_VARIANT(32, 4, 32, 8),
    TPA_VARIANT(32, 8, 32, 4),
    TPA_VARIANTW(1, 8, 8),
    TPA_VARIANTW(1, 7, 8),
    TPA_VARIANTW(2, 8, 4),
    TPA_VARIANTW(4, 6, 4),
    TPA_VARIANTW(4, 8, 4),
    TPA_VARIANTW(4, 4, 8),
    TPA_VARIANTW(8, 4, 4),
    TPA_VARIANTW(8, 6, 2),
    TPA_VARIANTW(8, 2, 8),
    TPA_VARIANTG(8, 1, 16, 16),
    TPA_VARIANTG(2, 4, 16, 8),
    TPA_VARIANTG(2, 2, 16, 16),
    TPA_VARIANTG(8, 4, 32, 8),
    TPA_VARIANT(1, 1, 8, 8),
    TPA_VARIANT(1, 2, 8, 8),
    TPA_VARIANT(1, 4, 8, 8),
    TPA_VARIANT(2, 4, 16, 8),
    TPA_VARIANT(8, 1, 16, 16),
    TPA_VARIANT(2, 2, 8, 8),
    TPA_VARIANTP(1, 2, 8, 8, 4, 1),
    TPA_VARIANTP(1, 4, 8, 8, 4, 1),
    TPA_VARIANTP(1, 4, 8, 8, 4, 6),
    TPA_VARIANTP(2, 2, 8, 8, 8, 1),
    TPA_VARIANTP(2, 4, 16, 8, 4, 1),
    TPA_VARIANTP(2, 4, 8, 8, 8, 3),
    TPA_VARIANTP(2, 4, 8, 4, 8, 1),
    TPA_VARIANTP(2, 4, 8, 4, 8, 3),
    TPA_VARIANTP(2, 4, 8, 8, 8, 1),
    TPA_VARIANT(4, 4, 16, 8),
    TPA_VARIANTP(2, 4, 8, 4, 4, 6),
    TPA_VARIANTP(2, 4, 8, 4, 4, 8),
    TPA_VARIANTP(2, 4, 4, 4, 8, 1),
    TPA_VARIANTP(2, 4, 8, 8, 4, 1),
    TPA_VARIANTP(1, 8, 4, 4, 8, 1),
    TPA_VARIANTP(1, 8, 4, 4, 4, 1),
    TPA_VARIANTP(1, 8, 8, 4, 4, 1),
    TPA_VARIANTP(1, 8, 4, 2, 8, 1),
    TPA_VARIANTP(4, 4, 8, 8, 8, 1),
    TPA_VARIANTP(2, 8, 8, 4, 8, 1),
    TPA_VARIANTP(2, 8, 8, 4, 4, 1),
    TPA_VARIANTB(1),
    TPA_VARIANTB(2),
    TPA_VARIANTB(4),
    TPA_VARIANTB(8),
    TPA_VARIANTB(16),
    TPA_VARIANTP(4, 4, 16, 8, 4, 1),
    TPA_VARIANTP(4, 4, 8, 4, 8, 2),
    TPA_VARIANTP(8, 4, 8, 8, 8, 1),
};
#undef TPA_VARIANT
#undef TPA_VARIANTW
#undef TPA_VARIANTG
#undef TPA_VARIANTP
#undef TPA_VARIANTB
#undef TPA_VARIANTS

// Padded width: the smallest power of two >= k (every power of two up to
// KP_MAX has at least one kernel variant).
int kp_for(int k)
{
    int kp = 1;
    while (kp < k) kp <<= 1;
    return std::max(1, std::min(kp, KP_MAX));
}

constexpr int NUM_VARIANTS = (int)(sizeof(kVariants) / sizeof(kVariants[0]));
// Variant chosen per padded width (index into kVariants, -1 = default).
static std::atomic<uint64_t> g_epoch{0};
uint64_t settings_epoch() { return g_epoch.load(); }
static int g_forced[KP_MAX + 1];
static bool g_forced_init = false;
// Seeds per CPI chunk in batched calls (a power of two <= KP_MAX).
// 0 selects the default: narrow chunks for queries (light seeds then take the
// push path and X[n][8] stays near L2 size), wide chunks for Algorithm 1 runs
// of many iterations (each streamed nonzero serves more seeds).
static int g_chunk_query = 0;
static int g_chunk_cpi = 0;
constexpr int DEFAULT_CHUNK_QUERY = 8;
constexpr int DEFAULT_CHUNK_CPI = 8;
// Push path for the first two family iterations of a query (on by default).
static bool g_push = true;
// Pattern-only products for unweighted graphs (on by default; see Params::inv_deg).
static bool g_pattern = true;
constexpr int PUSH_MAX_OUTDEG = 256;   // seeds with more out-edges keep the pull path
static_assert(PUSH_MAX_OUTDEG <= PUSH_THREADS, "push_x2_k takes one thread per out-edge of the seed");
constexpr int PUSH_BLOCKS = 32;        // blocks per column in push_x2_k
constexpr int PUSH_MAX_KP = 16;        // widest query chunk with the push branch

static void launch_convert(int KP, unsigned blocks, unsigned long long *U, uint32_t *touched, float *X, float *R,
                           int64_t n, int kc, float decay, double eps, double *part, void *ctl, int gate,
                           const float *inv_deg, cudaStream_t s)
{
#define TPA_CONVERT(W) \
    convert_x2_k<W><<<blocks, 256, 0, s>>>(U, touched, X, R, n, kc, decay, eps, part, ctl, gate, inv_deg)
    switch (KP) {
    case 1: TPA_CONVERT(1); break;
    case 2: TPA_CONVERT(2); break;
    case 4: TPA_CONVERT(4); break;
    case 16: TPA_CONVERT(16); break;
    default: TPA_CONVERT(8); break;
    }
#undef TPA_CONVERT
}

static void launch_clear_x2(int KP, uint32_t *touched, float *X, int64_t n, void *ctl, int gate, cudaStream_t s)
{
    const int64_t nwords = (n + 31) / 32;
    const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((nwords + 255) / 256, 8 * num_sms()));
    switch (KP) {
    case 1: clear_x2_k<1><<<blocks, 256, 0, s>>>(touched, X, nwords, ctl, gate); break;
    case 2: clear_x2_k<2><<<blocks, 256, 0, s>>>(touched, X, nwords, ctl, gate); break;
    case 4: clear_x2_k<4><<<blocks, 256, 0, s>>>(touched, X, nwords, ctl, gate); break;
    case 16: clear_x2_k<16><<<blocks, 256, 0, s>>>(touched, X, nwords, ctl, gate); break;
    default: clear_x2_k<8><<<blocks, 256, 0, s>>>(touched, X, nwords, ctl, gate); break;
    }
}

// The forced variant for a padded width, else the first listed with that width.
static const Variant &pick_variant(int KP)
{
    if (g_forced_init && KP <= KP_MAX && g_forced[KP] >= 0) return kVariants[g_forced[KP]];
    for (const Variant &v : kVariants)
        if (v.cfg.KP() == KP) return v;
    set_error("no SpMM kernel variant for padded width %d", KP);
    throw Fail{TPA_EINVAL};
}

// ------------------------------------------------------------ CPI loop ---
// Algorithmic bytes of one SpMV/SpMM launch over CSR(A~^T): row pointers
// (int64), columns and values once (columns only for pattern-only products),
// the iterate X[n][KP] read once and, in the accumulate mode, Y[n][KP]
// written (pattern-only: with inv_deg[n] read) and r[n][k] read and written;
// in the finalize mode r[n][k] and r~_stranger[n] read and out[n][k] written.
static double spmm_bytes(int64_t n, int64_t m, int KP, int k, int mode, int accumulate, bool pattern)
{
    double b = 8.0 * (double)(n + 1) + (pattern ? 4.0 : 8.0) * (double)m + 4.0 * (double)n * KP;
    if (mode == MODE_ACC)
        b += 4.0 * (double)n * KP + (accumulate ? 8.0 * (double)n * k : 0.0) + (pattern ? 4.0 * (double)n : 0.0);
    else
        b += 4.0 * (double)n * k + 4.0 * (double)n + 4.0 * (double)n * k;
    return b;
}

// Statistics family of the SpMV/SpMM launches of one padded width.
static const char *spmm_family(int KP)
{
    static const char *names[] = {"spmm_kp1", "spmm_kp2", "spmm_kp4", "spmm_kp8", "spmm_kp16",
                                  "spmm_kp32", "spmm_kp64", "spmm_kp128", "spmm_kp256"};
    int i = 0;
    while ((1 << i) < KP && i < 8) ++i;
    return names[i];
}

// The finishing launch of the lane-segment walk (the rows, their epilogue,
// the L1 norm and the break test), timed apart from the walk.
static const char *finish_family(int KP)
{
    static const char *names[] = {"finish_kp1", "finish_kp2", "finish_kp4", "finish_kp8", "finish_kp16",
                                  "finish_kp32", "finish_kp64", "finish_kp128", "finish_kp256"};
    int i = 0;
    while ((1 << i) < KP && i < 8) ++i;
    return names[i];
}

static int iteration_bound(double c, double eps)
{
    // first i with c (1-c)^i < eps, plus a margin for FP32 rounding of the norm
    const double b = std::log(eps / c) / std::log(1.0 - c);
    const double i = std::max(0.0, std::ceil(b));
    return (int)std::min(1.0e6, i) + 4;
}

// Sizes the workspace buffers that one SpMV/SpMM launch of variant var at
// padded width KP over CSR(A~^T) (which = 0) or CSR(A~) indexes, and checks
// them against what the launch indexes; fills the plan fields of p.  The
// control block is zeroed when first allocated (its launch counter must
// start below every tag in the carry-out words).  Returns the blocks of the
// fixup grid (0 for the segmented walk, which has no fixup).
static unsigned size_for_variant(tpa_graph *g, const Variant &var, int which, int KP, Params &p, cudaStream_t s)
{
    Workspace &W = g->ws;
    const bool fresh_ctl = !W.ctl.p;
    W.ctl.ensure(CTL_BYTES, s);
    if (fresh_ctl) TPA_CUDA(cudaMemsetAsync(W.ctl.p, 0, CTL_BYTES, s));
    if (var.seg) {
        const size_t fix_bytes = (size_t)seg_grid_bound() * KP * sizeof(double);
        W.fix.ensure(fix_bytes, s);
        need(W.fix, fix_bytes, "L1 partials");
        bind_seg(p, g, which, var.cfg.L(), KP, s);
        p.tiles = 0;
        if (var.lane) {   // row parts by rank, segment-end sums, row bounds by rank
            SegRows &SR = which ? g->seg_a : g->seg_t;
            if (!SR.nzrp.p) {
                SR.nzrp.ensure((size_t)(SR.n_nz + 1) * sizeof(int64_t), s);
                lane_bounds_k<<<grid_1d(SR.n_nz + 1, 256), 256, 0, s>>>(
                    which ? g->rp_a.as<int64_t>() : g->rp_t.as<int64_t>(), SR.nz_rows.as<int32_t>(), SR.n_nz, g->m,
                    SR.nzrp.as<int64_t>());
                note_launch("plan");
                TPA_CHECK_LAUNCH();
            }
            need(SR.nzrp, (size_t)(SR.n_nz + 1) * sizeof(int64_t), "row bounds");
            p.nzrp = SR.nzrp.as<int64_t>();
            const size_t rec_bytes = (size_t)std::max<int64_t>(1, g->n - p.n_empty) * KP * sizeof(float);
            const size_t tail_bytes = (size_t)std::max<int64_t>(1, (p.seg_tiles + 31) / 32) * KP * sizeof(float);
            W.lrec.ensure(rec_bytes, s);
            W.ltail.ensure(tail_bytes, s);
            need(W.lrec, rec_bytes, "row parts");
            need(W.ltail, tail_bytes, "segment sums");
            p.lrec = W.lrec.as<float>();
            p.ltail = W.ltail.as<float>();
        }
        return 0;
    }
    const Plan &P = get_plan(g, var.cfg.L(), s, which);
    const size_t tile_bytes = (size_t)P.tiles * KP * sizeof(float);
    W.carry.ensure(tile_bytes, s);
    W.head.ensure(tile_bytes, s);
    int64_t tl1_rows = P.tiles + 8;   // per tile, or per warp of a grid
    if (var.binned) tl1_rows = std::max(tl1_rows, binned_slots_bound(get_bin_plan(g, which, s).n_long, KP));
    W.tl1.ensure((size_t)tl1_rows * KP * sizeof(float), s);
    const unsigned fix_blocks = fix_grid(KP, P.tiles);
    W.fix.ensure((size_t)fix_blocks * KP * sizeof(double), s);
    need(W.carry, tile_bytes, "tile carries");
    need(W.head, tile_bytes, "deferred heads");
    need(W.tl1, (size_t)tl1_rows * KP * sizeof(float), "tile L1 partials");
    need(W.fix, (size_t)fix_blocks * KP * sizeof(double), "fixup partials");
    p.tile_x = P.tile_x.as<int32_t>();
    p.tile_y = P.tile_y.as<int64_t>();
    p.head_row = P.head_row.as<int32_t>();
    p.head_first = P.head_first.as<int32_t>();
    p.tiles = P.tiles;
    p.carry = W.carry.as<float>();
    p.head = W.head.as<float>();
    p.tl1 = W.tl1.as<float>();
    if (var.binned) bind_bins(p, g, which, KP, s);
    if (!var.fix) {   // finishes its deferred rows itself: tagged carry words, one L1 partial per CTA
        const size_t agg_bytes = (size_t)std::max<int64_t>(1, P.tiles) * KP * sizeof(unsigned long long);
        if (!W.agg.p || W.agg.bytes < agg_bytes) {
            W.agg.ensure(agg_bytes, s);
            TPA_CUDA(cudaMemsetAsync(W.agg.p, 0, W.agg.bytes, s));
        }
        need(W.agg, agg_bytes, "carry-out words");
        const size_t part_bytes = (size_t)seg_grid_bound() * KP * sizeof(double);
        if (W.fix.bytes < part_bytes) W.fix.ensure(part_bytes, s);
        need(W.fix, part_bytes, "CTA partials");
        p.agg = W.agg.as<unsigned long long>();
    }
    return fix_blocks;
}

// Iterate buffers of n rows of KP floats: y is zeroed when allocated (the
// segmented walk writes only rows with in-edges); a new x has unknown rows.
static void size_iterates(tpa_graph *g, int KP, cudaStream_t s)
{
    Workspace &W = g->ws;
    const size_t bytes = (size_t)g->n * KP * sizeof(float);
    if (!W.x.p || W.x.bytes < bytes) {
        W.x.ensure(bytes, s);
        W.x_zkp = 0;
        W.x_seeds = false;
    }
    if (!W.y.p || W.y.bytes < bytes) {
        W.y.ensure(bytes, s);
        TPA_CUDA(cudaMemsetAsync(W.y.p, 0, W.y.bytes, s));
        W.y_zkp = -1;
    }
    need(W.x, bytes, "iterate x");
    need(W.y, bytes, "iterate y");
}

void run_cpi_chunk(tpa_graph *g, const CpiArgs &a, int k0, int kc, cudaStream_t s)
{
    const int KP = kp_for(kc);
    const Variant &var = pick_variant(KP);
    const int64_t n = g->n;
    Workspace &W = g->ws;
    Params p{};
    size_iterates(g, KP, s);
    const unsigned fix_blocks = size_for_variant(g, var, 0, KP, p, s);
    if (W.x_seeds) {   // the seeds were another chunk's
        W.x_zkp = 0;
        W.x_seeds = false;
    }

    ctl_init_k<<<1, 256, 0, s>>>(W.ctl.p, kc);
    note_launch("init");
    // pattern-only products: x is kept scaled by the inverse out-degree
    const float *inv_deg = g_pattern && !g->weighted ? g->inv_deg32.as<float>() : nullptr;
    const float c_val = (float)a.c;
    const float pr_val = (float)(a.c * (1.0 / (double)n));
    float *r;
    int64_t ldr;
    if (a.r_internal) {
        W.r.ensure((size_t)n * KP * sizeof(float), s);
        need(W.r, (size_t)n * KP * sizeof(float), "accumulator r");
        r = W.r.as<float>();
        ldr = KP;
    } else {
        r = a.r + k0;
        ldr = a.ldr;
    }
    const int last = a.t_iter >= 0 ? a.t_iter : iteration_bound(a.c, a.eps);
    // Query chunks of at most 8 seeds have two branches for x1 and x2: push
    // along CSR(A~) when every seed is light, pull otherwise.  With the seeds'
    // out-degrees on the host the branch is chosen here and only its kernels
    // are launched; without them (a launch sequence being captured into a
    // CUDA graph) the device chooses (push_decide_k) and the kernels of the
    // other branch return at once.  On both branches x2 ends in the x2
    // buffer, which iteration 3 reads.
    const bool two_way =
        g_push && a.tpa_final && a.seeds && !a.set_ptr && last >= 3 && KP <= PUSH_MAX_KP && a.r_internal;
    bool host_decided = false, host_push = false;
    if (two_way && a.seed_outdeg) {
        host_decided = true;
        host_push = true;
        for (int j = 0; j < kc; ++j) host_push = host_push && a.seed_outdeg[k0 + j] <= PUSH_MAX_OUTDEG;
    }
    const bool run_push = two_way && (!host_decided || host_push);
    const bool run_pull = two_way && (!host_decided || !host_push);
    const int gate_push = host_decided ? GATE_NONE : GATE_PUSH;
    const int gate_pull = host_decided ? GATE_NONE : GATE_PULL;
    if (two_way) {
        const unsigned cblocks = (unsigned)std::min<int64_t>((n + 255) / 256, (int64_t)8 * num_sms());
        W.fix.ensure((size_t)std::max<unsigned>(fix_blocks, cblocks) * KP * sizeof(double), s);
        // U, the row marks and the x2 buffer are all zero between chunks
        if (!W.u.p || W.u.bytes < (size_t)n * KP * sizeof(unsigned long long) || !W.u_clean) {
            W.u.ensure((size_t)n * KP * sizeof(unsigned long long), s);
            W.touched.ensure((size_t)((n + 31) / 32) * sizeof(uint32_t), s);
            W.x2.ensure((size_t)n * PUSH_MAX_KP * sizeof(float), s);
            TPA_CUDA(cudaMemsetAsync(W.u.p, 0, W.u.bytes, s));
            TPA_CUDA(cudaMemsetAsync(W.touched.p, 0, W.touched.bytes, s));
            TPA_CUDA(cudaMemsetAsync(W.x2.p, 0, W.x2.bytes, s));
        }
        need(W.u, (size_t)n * KP * sizeof(unsigned long long), "push accumulator");
        need(W.touched, (size_t)((n + 31) / 32) * sizeof(uint32_t), "push row marks");
        need(W.x2, (size_t)n * KP * sizeof(float), "x2 buffer");
        need(W.fix, (size_t)cblocks * KP * sizeof(double), "conversion partials");
        W.u_clean = false;
        if (!host_decided) {
            push_decide_k<<<1, 32, 0, s>>>(a.seeds + k0, kc, g->outdeg.as<int32_t>(), PUSH_MAX_OUTDEG, W.ctl.p);
            note_launch("push");
        }
        if (run_push) {   // r = x0 + x1, x2 into the x2 buffer
            const float decay_f = (float)(1.0 - a.c);
            zero_k<<<grid_1d(n * KP / 4, 256), 256, 0, s>>>(r, n * KP, W.ctl.p, gate_push);
            push_x2_k<<<dim3(PUSH_BLOCKS, kc), PUSH_THREADS, 0, s>>>(
                g->rp_a.as<int64_t>(), g->col_a.as<int32_t>(), g->val_a.as<float>(), a.seeds + k0, KP, c_val,
                decay_f, W.u.as<unsigned long long>(), W.touched.as<uint32_t>(), r, W.ctl.p, gate_push);
            launch_convert(KP, cblocks, W.u.as<unsigned long long>(), W.touched.as<uint32_t>(), W.x2.as<float>(), r,
                           n, kc, decay_f, a.eps, W.fix.as<double>(), W.ctl.p, gate_push, inv_deg, s);
            note_launch("push", 3);
        }
        if (run_pull) {   // x0; iterations 1 and 2 are pulled below
            init_k<<<grid_1d(n * KP, 256), 256, 0, s>>>(W.x.as<float>(), KP, n, a.seeds + k0, kc, c_val, pr_val, r,
                                                         ldr, a.s_iter == 0 ? 1 : 0, W.ctl.p, gate_pull, inv_deg);
            note_launch("init");
            // x0 at the seeds, zero elsewhere; a gated launch may not run, then x keeps its state
            const bool was_clean = W.x_zkp == KP || W.x_zkp == -1;
            W.x_zkp = host_decided || was_clean ? KP : 0;
            W.x_seeds = W.x_zkp == KP;
        }
        TPA_CHECK_LAUNCH();
    } else if (a.set_ptr) {   // seed sets: zero, then scatter c / |S_j| over each set's members
        init_k<<<grid_1d(n * KP, 256), 256, 0, s>>>(W.x.as<float>(), KP, n, nullptr, kc, c_val, 0.0f, r, ldr,
                                                     a.s_iter == 0 ? 1 : 0, W.ctl.p, GATE_NONE, inv_deg);
        scatter_sets_k<<<kc, 256, 0, s>>>(W.x.as<float>(), KP, a.set_ptr + k0, a.seeds, c_val, r, ldr,
                                          a.s_iter == 0 ? 1 : 0, inv_deg);
        note_launch("init", 2);
        W.x_zkp = 0;   // the members' x0 may sit on rows without in-edges
        W.x_seeds = false;
        TPA_CHECK_LAUNCH();
    } else {
        init_k<<<grid_1d(n * KP, 256), 256, 0, s>>>(W.x.as<float>(), KP, n, a.seeds ? a.seeds + k0 : nullptr, kc,
                                                     c_val, pr_val, r, ldr, a.s_iter == 0 ? 1 : 0, W.ctl.p,
                                                     GATE_NONE, inv_deg);
        note_launch("init");
        TPA_CHECK_LAUNCH();
        W.x_zkp = a.seeds ? KP : 0;   // PageRank's x0 is c/n on every row
        W.x_seeds = a.seeds != nullptr;
    }
    if (last == 0) {
        if (a.tpa_final) {
            finalize_k<<<grid_1d(n * kc, 256), 256, 0, s>>>(r, ldr, a.r_str, (float)(1.0 + a.alpha), a.out + k0,
                                                           a.ldo, n, kc);
            note_launch("finalize");
        }
        if (a.iters_out) {
            copy_iters_k<<<1, 256, 0, s>>>(W.ctl.p, a.iters_out + k0, kc);
            note_launch("init");
        }
        TPA_CHECK_LAUNCH();
        return;
    }

    p.rp = g->rp_t.as<int64_t>();
    p.col = g->col_t.as<int32_t>();
    p.val = g->val_t.as<float>();
    p.n = n;
    p.r = r;
    p.ldr = ldr;
    p.out = a.out ? a.out + k0 : nullptr;
    p.ldo = a.ldo;
    p.r_str = a.r_str;
    p.one_plus_alpha = (float)(1.0 + a.alpha);
    p.decay = (float)(1.0 - a.c);
    p.k = kc;
    p.eps = a.eps;
    p.part = W.fix.as<double>();
    p.ctl = W.ctl.p;
    p.inv_deg = inv_deg;

    // x and y alternate; on a two-way chunk iteration 2 writes and iteration
    // 3 reads the x2 buffer
    float *cur = W.x.as<float>(), *nxt = W.y.as<float>();
    // Host-side early stop: every CHUNK iterations, read the device done flag
    // of the chunk before last, so launches never run far past convergence.
    const int CHUNK = 8;
    int32_t *hflag = nullptr;
    if (a.t_iter < 0) {
        if (!W.hflag) TPA_CUDA(cudaHostAlloc((void **)&W.hflag, 2 * sizeof(int32_t), cudaHostAllocDefault));
        hflag = W.hflag;
    }
    cudaEvent_t ev[2] = {nullptr, nullptr};
    try {
        if (hflag) {
            hflag[0] = hflag[1] = 0;
            TPA_CUDA(cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming));
            TPA_CUDA(cudaEventCreateWithFlags(&ev[1], cudaEventDisableTiming));
        }
        int chunk = 0;
        for (int i = two_way && !run_pull ? 3 : 1; i <= last; ++i) {
            if (two_way && i == 3) {   // iteration 3 reads x2 from the x2 buffer and writes y
                cur = W.x2.as<float>();
                nxt = W.y.as<float>();
            }
            p.x = cur;
            p.y = (two_way && i == 2) ? W.x2.as<float>() : nxt;
            p.gate = (two_way && i <= 2) ? gate_pull : GATE_NONE;
            p.iter = i;
            p.accumulate = i >= a.s_iter ? 1 : 0;
            p.mode = (a.tpa_final && i == last) ? MODE_FINAL : MODE_ACC;
            // the segmented walk writes only rows with in-edges: clear the
            // others in a buffer that held x0 (the seeds' rows, or every row)
            p.zero_mode = 0;
            const bool out_x = p.y == W.x.as<float>(), out_y = p.y == W.y.as<float>();
            if (p.mode == MODE_ACC && (out_x || out_y)) {
                int &zkp = out_x ? W.x_zkp : W.y_zkp;
                const bool clean = zkp == KP || zkp == -1;
                if (var.seg) {
                    p.zero_mode = !clean ? 2 : (out_x && W.x_seeds) ? 1 : 0;
                    p.zseeds = a.seeds ? a.seeds + k0 : nullptr;
                    p.zk = kc;
                    if (p.zero_mode == 1 && !p.zseeds) p.zero_mode = 2;
                }
                if (p.gate == GATE_NONE) {   // a gated launch may not run: the state stays
                    zkp = KP;
                    if (out_x) W.x_seeds = false;
                }
            }
            ProfMark pm = prof_begin(s);
            p.l1_slots = var.spmm(p, s);
            prof_end(pm, spmm_family(KP), spmm_bytes(n, g->m, KP, kc, p.mode, p.accumulate, p.inv_deg != nullptr), s);
            note_launch(spmm_family(KP));
            if (var.fix) {
                const char *fam = var.lane ? finish_family(KP) : "fixup";
                ProfMark pf = prof_begin(s);
                var.fix(p, fix_blocks, s);
                prof_end(pf, fam, 0.0, s);
                note_launch(fam);
            }
            if (p.mode == MODE_FINAL) {
                if (var.seg)
                    finalize_seg_k<<<grid_1d(n, 256), 256, 0, s>>>(W.ctl.p, p.empty_rows, p.n_empty, r, ldr,
                                                                        a.r_str, p.one_plus_alpha, p.out, p.ldo, n,
                                                                        kc);
                else   // usually returns at once: a grid of 8 blocks per SM (grid-stride when it works)
                    finalize_if_done_k<<<std::min<unsigned>(grid_1d(n * kc, 256), 8u * (unsigned)num_sms()), 256, 0,
                                         s>>>(W.ctl.p, r, ldr, a.r_str, p.one_plus_alpha, p.out, p.ldo, n, kc);
                note_launch("finalize");
            }
            TPA_CHECK_LAUNCH();
            if (two_way && i == 3) {
                // restore the x2 buffer: sparse on the push branch, whole on the pull branch
                if (run_push) {
                    launch_clear_x2(KP, W.touched.as<uint32_t>(), W.x2.as<float>(), n, W.ctl.p, gate_push, s);
                    note_launch("push");
                }
                if (run_pull) {
                    zero_k<<<grid_1d(n * KP / 4, 256), 256, 0, s>>>(W.x2.as<float>(), n * KP, W.ctl.p, gate_pull);
                    note_launch("push");
                }
                TPA_CHECK_LAUNCH();
                W.u_clean = true;
                cur = nxt;
                nxt = W.x.as<float>();
            } else if (!(two_way && i == 2)) {
                std::swap(cur, nxt);
            }
            if (hflag && i % CHUNK == 0) {
                const int slot = chunk & 1;
                if (chunk >= 2) {
                    TPA_CUDA(cudaEventSynchronize(ev[slot]));
                    if (hflag[slot]) break;
                }
                const CtlView cv = ctl_view(W.ctl.p);
                TPA_CUDA(cudaMemcpyAsync(&hflag[slot], &cv.hdr->done, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
                TPA_CUDA(cudaEventRecord(ev[slot], s));
                ++chunk;
            }
        }
        if (a.iters_out) {
            copy_iters_k<<<1, 256, 0, s>>>(W.ctl.p, a.iters_out + k0, kc);
            note_launch("init");
        }
        TPA_CHECK_LAUNCH();
    } catch (...) {
        if (hflag) cudaStreamSynchronize(s);
        if (ev[0]) cudaEventDestroy(ev[0]);
        if (ev[1]) cudaEventDestroy(ev[1]);
        throw;
    }
    if (hflag) TPA_CUDA(cudaStreamSynchronize(s));
    if (ev[0]) cudaEventDestroy(ev[0]);
    if (ev[1]) cudaEventDestroy(ev[1]);
}

// ------------------------------------------------ single step, no alloc ---
// One propagation step for one vector over caller-provided CSR(A~^T), with
// every scratch array carved out of a caller-provided device buffer.  Error
// reporting is by return value: this path throws nothing and allocates
// nothing (it backs the scratch-free entry point).
namespace {

constexpr int STEP_ITEMS = 8;
constexpr int STEP_WARPS = 8;
constexpr int STEP_L = 32 * STEP_ITEMS;
constexpr int STEP_FIX_BLOCKS = 256;

__host__ __device__ inline size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

struct StepLayout {
    size_t tile_x, tile_y, head_row, head_first, carry, head, tl1, part, ctl, total;
};

StepLayout step_layout(int64_t tiles)
{
    StepLayout L;
    size_t off = 0;
    L.tile_x = off;     off += align256((size_t)(tiles + 1) * sizeof(int32_t));
    L.tile_y = off;     off += align256((size_t)(tiles + 1) * sizeof(int64_t));
    L.head_row = off;   off += align256((size_t)tiles * sizeof(int32_t));
    L.head_first = off; off += align256((size_t)tiles * sizeof(int32_t));
    L.carry = off;      off += align256((size_t)tiles * sizeof(float));
    L.head = off;       off += align256((size_t)tiles * sizeof(float));
    L.tl1 = off;        off += align256((size_t)tiles * sizeof(float));
    L.part = off;       off += align256((size_t)STEP_FIX_BLOCKS * sizeof(double));
    L.ctl = off;        off += align256(CTL_BYTES);
    L.total = off;
    return L;
}

__global__ void copy_norm_k(const void *ctl, double *out)
{
    const CtlView cv = ctl_view(const_cast<void *>(ctl));
    out[0] = cv.norm[0];
}
}  // namespace

size_t step1_scratch_bytes(int64_t n, int64_t m)
{
    const int64_t tiles = std::max<int64_t>(1, (n + m + STEP_L - 1) / STEP_L);
    return step_layout(tiles).total;
}

cudaError_t run_step1(const int64_t *rp, const int32_t *col, const float *val, int64_t n, int64_t m, double c,
                      const float *x, float *y, float *r, double *l1, unsigned char *scratch, cudaStream_t s)
{
    const int64_t tiles = std::max<int64_t>(1, (n + m + STEP_L - 1) / STEP_L);
    const StepLayout L = step_layout(tiles);
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, spmvw_tile_k<1, STEP_ITEMS, STEP_WARPS>,
                                                          STEP_WARPS * 32, 0);
    if (e != cudaSuccess) return e;
    per_sm = std::max(per_sm, 1);

    Params p{};
    p.rp = rp;
    p.col = col;
    p.val = val;
    p.n = n;
    p.tile_x = reinterpret_cast<int32_t *>(scratch + L.tile_x);
    p.tile_y = reinterpret_cast<int64_t *>(scratch + L.tile_y);
    p.head_row = reinterpret_cast<int32_t *>(scratch + L.head_row);
    p.head_first = reinterpret_cast<int32_t *>(scratch + L.head_first);
    p.tiles = tiles;
    p.x = x;
    p.y = y;
    p.r = r;
    p.ldr = 1;
    p.decay = (float)(1.0 - c);
    p.k = 1;
    p.mode = MODE_ACC;
    p.accumulate = r ? 1 : 0;
    p.iter = 1;
    p.eps = 0.0;
    p.carry = reinterpret_cast<float *>(scratch + L.carry);
    p.head = reinterpret_cast<float *>(scratch + L.head);
    p.tl1 = reinterpret_cast<float *>(scratch + L.tl1);
    p.part = reinterpret_cast<double *>(scratch + L.part);
    p.ctl = scratch + L.ctl;

    plan_tiles_k<<<grid_1d(tiles + 1, 256), 256, 0, s>>>(rp, n, m, STEP_L, tiles, const_cast<int32_t *>(p.tile_x),
                                                          const_cast<int64_t *>(p.tile_y));
    plan_heads_k<<<grid_1d(tiles, 256), 256, 0, s>>>(rp, p.tile_x, p.tile_y, tiles, const_cast<int32_t *>(p.head_row),
                                                     const_cast<int32_t *>(p.head_first));
    ctl_init_k<<<1, 256, 0, s>>>(p.ctl, 1);   // done, ticket and alive start cleared for every call
    const int64_t grid = std::min<int64_t>((tiles + STEP_WARPS - 1) / STEP_WARPS, (int64_t)per_sm * sms);
    spmvw_tile_k<1, STEP_ITEMS, STEP_WARPS><<<(unsigned)grid, STEP_WARPS * 32, 0, s>>>(p);
    const unsigned fb = (unsigned)std::min<int64_t>((tiles + FIX_WARPS - 1) / FIX_WARPS, STEP_FIX_BLOCKS);
    fixup_k<1><<<fb, FIX_WARPS * 32, 0, s>>>(p);
    int launches = 5;
    if (l1) {
        copy_norm_k<<<1, 1, 0, s>>>(p.ctl, l1);
        ++launches;
    }
    note_launch_count(launches);
    return cudaGetLastError();
}

__global__ void gather_outdeg_k(const int32_t *outdeg, const int32_t *seeds, int k, int32_t *out)
{
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < k; j += gridDim.x * blockDim.x) out[j] = outdeg[seeds[j]];
}

std::vector<int32_t> seed_outdegrees(tpa_graph *g, const int32_t *d_seeds, int k, cudaStream_t s)
{
    std::vector<int32_t> h((size_t)k);
    DevBuf tmp;
    tmp.ensure((size_t)k * sizeof(int32_t), s);
    gather_outdeg_k<<<(unsigned)std::min(1024, (k + 255) / 256), 256, 0, s>>>(g->outdeg.as<int32_t>(), d_seeds, k,
                                                                            tmp.as<int32_t>());
    note_launch("init");
    TPA_CHECK_LAUNCH();
    TPA_CUDA(cudaMemcpyAsync(h.data(), tmp.p, (size_t)k * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    TPA_CUDA(cudaStreamSynchronize(s));
    tmp.release(s);
    return h;
}

void spmv_apply(tpa_graph *g, int which, const float *x, float *y, int kc, float decay, cudaStream_t s)
{
    TPA_REQUIRE(kc >= 1 && kc <= 32, "spmv_apply: %d columns (at most 32)", kc);
    const int KP = kp_for(kc);
    const Variant &var = pick_variant(KP);
    Workspace &W = g->ws;
    Params p{};
    const unsigned fix_blocks = size_for_variant(g, var, which, KP, p, s);
    ctl_init_k<<<1, 256, 0, s>>>(W.ctl.p, kc);
    p.rp = which ? g->rp_a.as<int64_t>() : g->rp_t.as<int64_t>();
    p.col = which ? g->col_a.as<int32_t>() : g->col_t.as<int32_t>();
    p.val = which ? g->val_a.as<float>() : g->val_t.as<float>();
    p.n = g->n;
    p.x = x;
    p.y = y;
    p.decay = decay;
    p.k = kc;
    p.mode = MODE_ACC;
    p.accumulate = 0;
    p.iter = 1;
    p.eps = 0.0;   // no break test: every column stays alive
    p.part = W.fix.as<double>();
    p.ctl = W.ctl.p;
    p.zero_mode = var.seg ? 2 : 0;   // y is the caller's: its rows without nonzeros are cleared
    ProfMark pm = prof_begin(s);
    p.l1_slots = var.spmm(p, s);
    prof_end(pm, spmm_family(KP), spmm_bytes(g->n, g->m, KP, kc, MODE_ACC, 0, false), s);
    note_launch("init");
    note_launch(spmm_family(KP));
    if (var.fix) {
        const char *fam = var.lane ? finish_family(KP) : "fixup";
        ProfMark pf = prof_begin(s);
        var.fix(p, fix_blocks, s);
        prof_end(pf, fam, 0.0, s);
        note_launch(fam);
    }
    TPA_CHECK_LAUNCH();
}

// Reorder of a query's seeds that gathers the seeds too heavy for the push
// branch (more out-edges than it takes) into the last positions, swapping
// each with a light seed from there, so that fewer chunks fall back to
// pulling x1 and x2.  od: host out-degrees of the k seeds.  perm[j] is the
// original position of the seed placed at j.  False (nothing moves) when no
// chunk can push, or the query is one chunk.
static bool group_heavy_seeds(const int32_t *od, int k, int chunk, std::vector<int32_t> &perm)
{
    perm.resize((size_t)k);
    for (int j = 0; j < k; ++j) perm[j] = j;
    if (!g_push || chunk > PUSH_MAX_KP || k <= chunk) return false;
    std::vector<int> heavy;
    for (int j = 0; j < k; ++j)
        if (od[j] > PUSH_MAX_OUTDEG) heavy.push_back(j);
    const int nh = (int)heavy.size();
    if (nh == 0 || nh == k) return false;
    const int r0 = k - nh;
    int l = r0;
    bool moved = false;
    for (int h : heavy) {
        if (h >= r0) continue;
        while (od[perm[l]] > PUSH_MAX_OUTDEG) ++l;   // a light seed in the last nh positions
        std::swap(perm[h], perm[l]);
        ++l;
        moved = true;
    }
    return moved;
}

bool regroup_seeds(const int32_t *od, int k, int S, std::vector<int32_t> &perm)
{
    const int chunk = g_chunk_query ? g_chunk_query : DEFAULT_CHUNK_QUERY;
    perm.resize((size_t)k);
    for (int j = 0; j < k; ++j) perm[j] = j;
    if (S - 1 < 3) return false;   // the push branch exists from S = 4
    return group_heavy_seeds(od, k, chunk, perm);
}

std::string query_branches(const int32_t *od, int k, int S)
{
    const int chunk = g_chunk_query ? g_chunk_query : DEFAULT_CHUNK_QUERY;
    std::string key;
    for (int k0 = 0; k0 < k; k0 += chunk) {
        const int kc = std::min(chunk, k - k0);
        // the conditions of run_cpi_chunk's two-way chunks for a query
        if (!g_push || S - 1 < 3 || kp_for(kc) > PUSH_MAX_KP) {
            key.push_back('-');
            continue;
        }
        bool light = true;
        for (int j = 0; j < kc; ++j) light = light && od[k0 + j] <= PUSH_MAX_OUTDEG;
        key.push_back(light ? 'p' : 'l');
    }
    return key;
}

// After a regrouped query has written every chunk in place, swap back the
// column pairs listed in device memory: pairs[0] = count, then the pairs.
// Grid-stride over n x count, so a captured launch serves any count.
__global__ void swap_cols_dev_k(float *out, int64_t ldo, int64_t n, const int32_t *pairs)
{
    const int np = __ldg(pairs);
    const int64_t total = n * np;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = i / np;
        const int q = (int)(i % np);
        float *row = out + v * ldo;
        const int32_t a = __ldg(pairs + 1 + 2 * q), b = __ldg(pairs + 2 + 2 * q);
        const float ta = row[a], tb = row[b];
        row[a] = tb;
        row[b] = ta;
    }
}

__global__ void gather_seeds_k(const int32_t *seeds, const int32_t *perm, int k, int32_t *out)
{
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < k; j += gridDim.x * blockDim.x) out[j] = seeds[perm[j]];
}

// After a regrouped query has written every chunk in place, column pairs
// (a, b) of out hold each other's scores: swap them back.
__global__ void swap_cols_k(float *out, int64_t ldo, int64_t n, const int32_t *pairs, int np)
{
    const int64_t total = n * np;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = i / np;
        const int q = (int)(i % np);
        float *row = out + v * ldo;
        const int32_t a = __ldg(pairs + 2 * q), b = __ldg(pairs + 2 * q + 1);
        const float ta = row[a], tb = row[b];
        row[a] = tb;
        row[b] = ta;
    }
}

void run_cpi(tpa_graph *g, const CpiArgs &a0, cudaStream_t s)
{
    const int chunk = a0.tpa_final ? (g_chunk_query ? g_chunk_query : DEFAULT_CHUNK_QUERY)
                                   : (g_chunk_cpi ? g_chunk_cpi : DEFAULT_CHUNK_CPI);
    CpiArgs a = a0;
    // what x holds is not known across calls (graph replays run the sequence
    // captured here on whatever a previous call left)
    g->ws.x_zkp = 0;
    g->ws.y_zkp = 0;
    g->ws.x_seeds = false;
    // A query whose chunk branches the host picks (it has the seeds' out-degrees)
    // and whose output is in device memory swaps the seeds too heavy for the
    // push branch into its last chunks, runs every chunk in place, and swaps
    // the moved columns back at the end.
    std::vector<int32_t> perm, od;
    bool grouped = false;
    if (!a.no_regroup && a.tpa_final && a.seed_outdeg && a.seeds && !a.set_ptr && a.r_internal && a.t_iter >= 3 &&
        a.out && is_device_ptr(a.out))
        grouped = group_heavy_seeds(a.seed_outdeg, a.k, chunk, perm);
    Workspace &W = g->ws;
    std::vector<int32_t> pairs;
    if (grouped) {
        od.resize((size_t)a.k);
        for (int j = 0; j < a.k; ++j) od[j] = a.seed_outdeg[perm[j]];
        for (int j = 0; j < a.k; ++j)
            if (perm[j] > j) {   // positions j and perm[j] traded seeds
                pairs.push_back(j);
                pairs.push_back(perm[j]);
            }
        W.cols.ensure(((size_t)a.k + pairs.size()) * sizeof(int32_t), s);
        W.seeds_g.ensure((size_t)a.k * sizeof(int32_t), s);
        TPA_CUDA(cudaMemcpyAsync(W.cols.p, perm.data(), (size_t)a.k * sizeof(int32_t), cudaMemcpyHostToDevice, s));
        TPA_CUDA(cudaMemcpyAsync(W.cols.as<int32_t>() + a.k, pairs.data(), pairs.size() * sizeof(int32_t),
                                 cudaMemcpyHostToDevice, s));
        gather_seeds_k<<<(unsigned)std::min(1024, (a.k + 255) / 256), 256, 0, s>>>(a.seeds, W.cols.as<int32_t>(),
                                                                                   a.k, W.seeds_g.as<int32_t>());
        note_launch("init");
        TPA_CHECK_LAUNCH();
        a.seeds = W.seeds_g.as<int32_t>();
        a.seed_outdeg = od.data();
    }
    for (int k0 = 0; k0 < a.k; k0 += chunk) run_cpi_chunk(g, a, k0, std::min(chunk, a.k - k0), s);
    if (a.dev_pairs && a.max_pairs > 0) {
        swap_cols_dev_k<<<grid_1d(g->n * a.max_pairs, 256), 256, 0, s>>>(a.out, a.ldo, g->n, a.dev_pairs);
        note_launch("finalize");
        TPA_CHECK_LAUNCH();
    }
    if (grouped) {
        const int np = (int)(pairs.size() / 2);
        swap_cols_k<<<grid_1d(g->n * np, 256), 256, 0, s>>>(a.out, a.ldo, g->n, W.cols.as<int32_t>() + a.k, np);
        note_launch("finalize");
        TPA_CHECK_LAUNCH();
    }
}

}  // namespace tpa

using namespace tpa;

extern "C" {

int tpa_variant_count(void) { return NUM_VARIANTS; }

tpa_status tpa_variant_info(int idx, int *kp, int *lanes, int *cols_per_lane, int *items, int *threads)
{
    if (idx < 0 || idx >= NUM_VARIANTS) {
        set_error("tpa_variant_info: index %d outside [0, %d)", idx, NUM_VARIANTS);
        return TPA_EINVAL;
    }
    const KCfg &c = kVariants[idx].cfg;
    if (kp) *kp = c.KP();
    if (lanes) *lanes = c.G;
    if (cols_per_lane) *cols_per_lane = c.V;
    if (items) *items = c.ITEMS;
    if (threads) *threads = c.NT;
    return TPA_OK;
}

int tpa_get_variant(int kp)
{
    if (kp < 1 || kp > KP_MAX || (kp & (kp - 1))) return -1;
    if (g_forced_init && g_forced[kp] >= 0) return g_forced[kp];
    for (int i = 0; i < NUM_VARIANTS; ++i)
        if (kVariants[i].cfg.KP() == kp) return i;
    return -1;
}

const char *tpa_variant_name(int idx)
{
    if (idx < 0 || idx >= NUM_VARIANTS) return nullptr;
    return kVariants[idx].name;
}

tpa_status tpa_set_variant(int kp, int idx)
{
    if (kp < 1 || kp > KP_MAX || (kp & (kp - 1))) {
        set_error("tpa_set_variant: width %d is not a power of two in [1, %d]", kp, KP_MAX);
        return TPA_EINVAL;
    }
    if (idx >= NUM_VARIANTS || (idx >= 0 && kVariants[idx].cfg.KP() != kp)) {
        set_error("tpa_set_variant: variant %d does not have width %d", idx, kp);
        return TPA_EINVAL;
    }
    if (!g_forced_init) {
        for (int i = 0; i <= KP_MAX; ++i) g_forced[i] = -1;
        g_forced_init = true;
    }
    g_forced[kp] = idx < 0 ? -1 : idx;
    ++g_epoch;
    return TPA_OK;
}

static bool valid_width(int width) { return width == 0 || (width >= 1 && width <= KP_MAX && !(width & (width - 1))); }

tpa_status tpa_set_batch_width(int width)
{
    if (!valid_width(width)) {
        set_error("tpa_set_batch_width: %d is neither 0 nor a power of two in [1, %d]", width, KP_MAX);
        return TPA_EINVAL;
    }
    g_chunk_query = width;
    ++g_epoch;
    return TPA_OK;
}

int tpa_get_batch_width(void) { return g_chunk_query ? g_chunk_query : DEFAULT_CHUNK_QUERY; }

tpa_status tpa_set_cpi_batch_width(int width)
{
    if (!valid_width(width)) {
        set_error("tpa_set_cpi_batch_width: %d is neither 0 nor a power of two in [1, %d]", width, KP_MAX);
        return TPA_EINVAL;
    }
    g_chunk_cpi = width;
    ++g_epoch;
    return TPA_OK;
}

int tpa_get_cpi_batch_width(void) { return g_chunk_cpi ? g_chunk_cpi : DEFAULT_CHUNK_CPI; }

tpa_status tpa_set_push(int enable)
{
    g_push = enable != 0;
    ++g_epoch;
    return TPA_OK;
}

tpa_status tpa_seed_order(const int32_t *outdeg, int k, int S, int32_t *perm)
{
    if (!outdeg || !perm || k < 1) {
        set_error("tpa_seed_order: NULL argument or k < 1");
        return TPA_EINVAL;
    }
    std::vector<int32_t> p((size_t)k);
    std::iota(p.begin(), p.end(), 0);
    const int chunk = g_chunk_query ? g_chunk_query : DEFAULT_CHUNK_QUERY;
    if (S - 1 >= 3) group_heavy_seeds(outdeg, k, chunk, p);   // the push branch exists from S = 4
    std::copy(p.begin(), p.end(), perm);
    return TPA_OK;
}

tpa_status tpa_set_pattern(int enable)
{
    g_pattern = enable != 0;
    ++g_epoch;
    return TPA_OK;
}

}  // extern "C"

namespace tpa {

}  // namespace tpa
