// Segmented flag walk: the SpMV/SpMM of one CPI iteration (Algorithm 1,
// x_i = (1-c) A~^T x_{i-1}) with its epilogue, L1 norm and break test in a
// single launch.  Included once, by cpi.cu, after spmm_kernels.cuh.
//
// The nonzeros of CSR(A~^T) are cut into tiles of TN = 32 * R consecutive
// nonzeros, one warp per tile in a static strided order (tile t on warp
// t mod W, so the warps in flight work on one band of rows and their gathers
// share L2).  Lane l of a tile owns nonzeros [t*TN + R*l, t*TN + R*l + R):
//   1. its R column ids come from a copy of the column array whose bit 31
//      marks the first nonzero of a row (no row pointer is read); each warp
//      keeps its next NB tiles of column words (and values) in flight with
//      1-D bulk copies (cp.async.bulk) into a ring of shared-memory stages,
//      each completing on its own mbarrier, so the copies cost no load
//      instructions and the tile's words are there when its turn comes;
//   2. it gathers the R rows X[col][0..V) (V = padded batch width, one lane
//      holds a whole row: one 32-byte load at V = 8) and walks them in order,
//      closing a row sum at every row start;
//   3. a shuffle segmented scan over the lanes adds the partials of rows that
//      span lanes; rows that start and end in the tile are parked in shared
//      memory and finished by one coalesced pass (lane per row: y stored,
//      r += y by a vector atomic, or the TPA finalize in the last family
//      iteration);
//   4. a row that spans tiles is finished by the tile where it ends: each tile
//      publishes its carry-out (the sum after its last row start, or of the
//      whole tile when no row starts in it) as 64-bit words that pair the
//      value with a launch tag, so a reader needs no fence: it waits (bounded)
//      until the word carries this launch's tag, then adds the carry-outs of
//      the tiles before it, nearest first, back to the tile where the row
//      started.  The fixed order keeps results identical run to run.
// The per-warp L1 partials are reduced by the last CTA to finish (one fence
// and one ticket per CTA), which applies the break test ||x_i||_1 < eps.
// Rows without nonzeros are never visited: their y stays zero (the rows a
// launch must clear are listed in Params::zero_mode), and the TPA finalize
// of those rows runs in finalize_seg_k.
//
// The waits assume every CTA of the grid is resident at once: the grid is at
// most the occupancy of the kernel times the SM count.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace tpa {

constexpr int SEG_WARPS = 8;                 // 256 threads: block_sum_partials runs on them
constexpr uint32_t SEG_ROW_START = 0x80000000u;
// Sum of the carry-outs of tiles t-1, t-2, ... back to and including the
// nearest one in which a row starts (all of them down to tile 0 if none),
// nearest first.  Warp-cooperative: tile t-1 first (lane j reads its word j),
// which ends the search in the common case of a row that started one tile
// back; then 32 tiles per round (lane l reads tile base - l), lanes past the
// first tile with a row start contributing zero, lanes added in a fixed
// shuffle tree.  Every lane returns the same sums.
template <int V>
__device__ __forceinline__ void seg_lookback(const Params &p, int64_t t, uint32_t want, Ctl *hdr, int lane,
                                             float (&sum)[V])
{
    const unsigned FULL = 0xffffffffu;
    float v1 = 0.0f;
    int st1 = 0;
    if (lane < V) {
        const unsigned long long w = seg_wait(p.agg + (t - 1) * V + lane, want, hdr);
        v1 = __uint_as_float((uint32_t)w);
        st1 = (int)((w >> 32) & 1ull);
    }
#pragma unroll
    for (int j = 0; j < V; ++j) sum[j] = __shfl_sync(FULL, v1, j);
    if (__shfl_sync(FULL, st1, 0)) return;
    for (int64_t base = t - 2; base >= 0; base -= 32) {
        const int64_t u = base - lane;
        float v[V];
        bool start = false;
#pragma unroll
        for (int j = 0; j < V; ++j) v[j] = 0.0f;
        if (u >= 0) {
#pragma unroll
            for (int j = 0; j < V; ++j) {
                const unsigned long long w = seg_wait(p.agg + u * V + j, want, hdr);
                v[j] = __uint_as_float((uint32_t)w);
                start = (w >> 32) & 1ull;
            }
        }
        const unsigned starts = __ballot_sync(FULL, start);
        const int stop = starts ? __ffs(starts) - 1 : 31;   // last lane that contributes
        if (lane > stop) {
#pragma unroll
            for (int j = 0; j < V; ++j) v[j] = 0.0f;
        }
#pragma unroll
        for (int j = 0; j < V; ++j) {
            float a = v[j];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(FULL, a, o);
            sum[j] += a;
        }
        if (starts) break;
    }
}

// Epilogue of one finished row for the segmented kernel (lane holds the row;
// w_row: RN32(1/outdeg) of the row for pattern-only products).
template <int V, bool PAT>
__device__ __forceinline__ void seg_emit_w(const Params &p, int64_t v, const float (&sv)[V], const int (&alive)[V],
                                           float (&l1)[V], float w_row)
{
    if (p.mode == MODE_ACC)
        epilogue_red<V, V, PAT ? PM_PATTERN : PM_VALUED>(p, v, 0, sv, alive, l1, w_row);
    else
        epilogue<V, V, PAT ? PM_PATTERN : PM_VALUED>(p, v, 0, sv, alive, l1);
}

template <int V, bool PAT>
__device__ __forceinline__ void seg_emit(const Params &p, int64_t v, const float (&sv)[V], const int (&alive)[V],
                                         float (&l1)[V])
{
    seg_emit_w<V, PAT>(p, v, sv, alive, l1, PAT && p.mode == MODE_ACC ? __ldg(p.inv_deg + v) : 0.0f);
}

// Finish row `row`, whose part in tile t is `part`, with the carry-outs of
// the tiles before t (warp-cooperative; lane 0 runs the epilogue).
template <int V, bool PAT>
__device__ __forceinline__ void seg_finish(const Params &p, int64_t t, int32_t row, const float (&part)[V],
                                           uint32_t want, Ctl *hdr, int lane, const int (&alive)[V], float (&l1)[V])
{
    float back[V];
    seg_lookback<V>(p, t, want, hdr, lane, back);
    if (lane == 0) {
        float tot[V];
#pragma unroll
        for (int j = 0; j < V; ++j) tot[j] = part[j] + back[j];
        seg_emit<V, PAT>(p, (int64_t)row, tot, alive, l1);
    }
}

// ------------------------------------------ bulk copies and mbarriers ---
__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
}

// One expected arrival that also expects `bytes` from bulk copies.
__device__ __forceinline__ void mbar_expect(uint64_t *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t *bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for phase `parity` of a barrier; false (and the error flag
// raised) when it gives up.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity, Ctl *hdr)
{
    long long spins = 0;
    while (!mbar_test(bar, parity)) {
        if (++spins > SEG_SPIN_LIMIT) {
            atomicOr(&hdr->error, 1);
            return false;
        }
    }
    return true;
}

// 1-D bulk copy global -> shared (16-byte aligned, size a multiple of 16),
// completing on the barrier.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Shared memory of the segmented kernel, per warp: NB stages of one tile's
// column words (and values), the sums of the rows finished in the tile (slot
// TN-1 holds the part of the row that ends at the tile's first row start),
// and one barrier per stage.
template <int V, int R, int NB, bool PAT>
struct SegSmem {
    static constexpr int TN = 32 * R;
    static constexpr size_t STAGE = (size_t)TN * sizeof(uint32_t) * (PAT ? 1 : 2);
    static constexpr size_t RS = (size_t)TN * V * sizeof(float);
    static constexpr size_t PER_WARP = NB * STAGE + RS + 16 * NB;
    static constexpr size_t BYTES = SEG_WARPS * PER_WARP;
};

template <int V, int R, int NB, bool PAT>
__device__ __forceinline__ void seg_issue(const Params &p, unsigned char *stage, uint64_t *bar, int64_t t)
{
    using SM = SegSmem<V, R, NB, PAT>;
    constexpr unsigned CB = SM::TN * sizeof(uint32_t);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // earlier reads of the stage come first
    mbar_expect(bar, PAT ? CB : 2 * CB);
    bulk_g2s(stage, p.colf + t * SM::TN, CB, bar);
    if constexpr (!PAT) bulk_g2s(stage + CB, p.val + t * SM::TN, CB, bar);
}

// Rows of y that the walk never writes but that must read as zero: the
// empty seed rows (zero_mode 1) or every empty row (zero_mode 2).
template <int V>
__device__ __forceinline__ void seg_zero_rows(const Params &p)
{
    if (p.zero_mode == 1) {
        for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < p.zk; j += gridDim.x * blockDim.x) {
            const int64_t s = p.zseeds[j];
            if (p.rp[s + 1] == p.rp[s]) {
                float z[V];
#pragma unroll
                for (int q = 0; q < V; ++q) z[q] = 0.0f;
                st_row<V>(p.y + s * V, z);
            }
        }
    } else if (p.zero_mode == 2) {
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < p.n_empty;
             i += (int64_t)gridDim.x * blockDim.x) {
            float z[V];
#pragma unroll
            for (int q = 0; q < V; ++q) z[q] = 0.0f;
            st_row<V>(p.y + (int64_t)p.empty_rows[i] * V, z);
        }
    }
}

// End of a segmented launch: the CTA's L1 partial; the last CTA to finish
// sums the partials in a fixed order and applies the break test of
// Algorithm 1 per column, then opens the next launch's epoch.
template <int V>
__device__ __forceinline__ void seg_close_launch(const Params &p, const CtlView &cv, const float (&l1)[V],
                                                 uint32_t ep_raw, int lane, int warp)
{
    __shared__ double s_fin[256];
    __shared__ float s_l1[SEG_WARPS][V];
    __shared__ int s_last;
    const unsigned FULL = 0xffffffffu;
#pragma unroll
    for (int j = 0; j < V; ++j) {
        float a = l1[j];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(FULL, a, o);
        if (lane == 0) s_l1[warp][j] = a;
    }
    __syncthreads();
    if (threadIdx.x < V) {
        float a = 0.0f;
#pragma unroll
        for (int w = 0; w < SEG_WARPS; ++w) a += s_l1[w][threadIdx.x];
        p.part[(int64_t)blockIdx.x * V + threadIdx.x] = (double)a;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(&cv.hdr->ticket, 1) == (int)gridDim.x - 1);
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    block_sum_partials<V>(p.part, gridDim.x, s_fin);
    if (threadIdx.x < V) {
        const int c = threadIdx.x;
        const double a = s_fin[c];
        if (c < p.k && cv.alive[c]) {
            cv.norm[c] = a;
            cv.iters[c] = p.iter;
            if (a < p.eps && p.mode == MODE_ACC) cv.alive[c] = 0;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int any = 0;
        for (int c = 0; c < p.k && c < V; ++c) any |= cv.alive[c];
        cv.hdr->done = any ? 0 : 1;
        cv.hdr->ticket = 0;
        cv.hdr->epoch = ep_raw + 1u;
    }
}

template <int V, int R, int PF, int NB, bool PAT>
__global__ void __launch_bounds__(SEG_WARPS * 32) spmm_seg_k(Params p)
{
    using SM = SegSmem<V, R, NB, PAT>;
    static_assert(R % 4 == 0 && R % PF == 0 && R <= 32, "R");
    static_assert(V == 1 || V == 2 || V == 4 || V == 8, "V");
    constexpr int TN = SM::TN;
    extern __shared__ __align__(128) unsigned char seg_smem[];
    const CtlView cv = ctl_view(p.ctl);
    if (gate_off(p.gate, p.ctl) || *(volatile int32_t *)&cv.hdr->done) return;
    const uint32_t ep_raw = *(volatile uint32_t *)&cv.hdr->epoch;
    const uint32_t ep = (ep_raw + 1u) & 0x7fffffffu;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned FULL = 0xffffffffu;
    unsigned char *wbase = seg_smem + (size_t)warp * SM::PER_WARP;
    float *rs = reinterpret_cast<float *>(wbase + NB * SM::STAGE);
    uint64_t *bars = reinterpret_cast<uint64_t *>(wbase + NB * SM::STAGE + SM::RS);

    seg_zero_rows<V>(p);

    unsigned amask = 0;
    float l1[V];
#pragma unroll
    for (int j = 0; j < V; ++j) {
        amask |= (cv.alive[j] ? 1u : 0u) << j;
        l1[j] = 0.0f;
    }
    int alive[V];
#pragma unroll
    for (int j = 0; j < V; ++j) alive[j] = (amask >> j) & 1u;

    const int64_t nw = (int64_t)gridDim.x * SEG_WARPS;
    const int64_t t0 = (int64_t)blockIdx.x * SEG_WARPS + warp;
    // prologue: barriers, and the first NB tiles of this warp in flight
    if (lane == 0) {
#pragma unroll
        for (int b = 0; b < NB; ++b) mbar_init(bars + b);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
#pragma unroll
        for (int b = 0; b < NB; ++b)
            if (t0 + b * nw < p.seg_tiles) seg_issue<V, R, NB, PAT>(p, wbase + b * SM::STAGE, bars + b, t0 + b * nw);
    }
    __syncwarp();
    int32_t crow_next = t0 < p.seg_tiles ? __ldg(p.tile_crow0 + t0) : 0;

    // the row a tile finishes through the carry-outs of earlier tiles, held
    // until the warp's next tile is under way
    bool pend = false;
    int64_t pend_t = 0;
    int32_t pend_row = 0;
    float pend_part[V];
#pragma unroll
    for (int j = 0; j < V; ++j) pend_part[j] = 0.0f;

    int it = 0;
    bool broke = false;
    for (int64_t t = t0; t < p.seg_tiles; t += nw, ++it) {
        const int b = it % NB;
        const int64_t crow0 = crow_next;
        if (t + nw < p.seg_tiles) crow_next = __ldg(p.tile_crow0 + t + nw);
        // the carry-out the pending row needs first, loaded early
        unsigned long long probe = 0ull;
        if (pend && lane < V) probe = ld_relaxed_u64(p.agg + (pend_t - 1) * V + lane);

        // 1. column words (and values) of the tile from its stage
        unsigned char *stage = wbase + b * SM::STAGE;
        if (!mbar_wait(bars + b, (unsigned)(it / NB) & 1u, cv.hdr)) {
            broke = true;
            break;
        }
        uint32_t cw[R];
        float vv[PAT ? 1 : R];
#pragma unroll
        for (int q = 0; q < R / 4; ++q) {
            const uint4 c = reinterpret_cast<const uint4 *>(stage)[lane * (R / 4) + q];
            cw[4 * q] = c.x;
            cw[4 * q + 1] = c.y;
            cw[4 * q + 2] = c.z;
            cw[4 * q + 3] = c.w;
            if constexpr (!PAT) {
                const float4 v4 = reinterpret_cast<const float4 *>(stage + TN * sizeof(uint32_t))[lane * (R / 4) + q];
                vv[4 * q] = v4.x;
                vv[4 * q + 1] = v4.y;
                vv[4 * q + 2] = v4.z;
                vv[4 * q + 3] = v4.w;
            }
        }
        const int64_t e0 = t * TN + (int64_t)lane * R;
        const bool full = (t + 1) * TN <= p.m;
        const int64_t left = p.m - e0;
        const unsigned vm = left >= R ? (R == 32 ? FULL : (1u << R) - 1u) : left > 0 ? (1u << left) - 1u : 0u;
        unsigned fm = 0;
#pragma unroll
        for (int i = 0; i < R; ++i) fm |= (cw[i] >> 31) << i;
        fm &= vm;
        __syncwarp();   // every lane has its words: the stage takes the warp's tile NB rounds ahead
        if (lane == 0 && t + NB * nw < p.seg_tiles) seg_issue<V, R, NB, PAT>(p, stage, bars + b, t + NB * nw);

        const int nf = __popc(fm);
        int incl = nf;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += y;
        }
        const int excl = incl - nf;
        const int q = __shfl_sync(FULL, incl, 31);
        // ids of the rows the epilogue pass finishes (lane k: row k), loaded early
        const int32_t vk = lane < q - 1 ? __ldg(p.nz_rows + crow0 + lane) : 0;

        // 2. gathers and the walk: at a row start the running sum goes to its
        //    slot (the row that ends there) and restarts; one FFMA per column
        float acc[V];
#pragma unroll
        for (int j = 0; j < V; ++j) acc[j] = 0.0f;
        int slot = excl - 1;   // row ending at this lane's next row start (-1: the tile's first row)
#pragma unroll
        for (int c0 = 0; c0 < R; c0 += PF) {
            float xv[PF][V];
            if (full) {   // every nonzero of the tile exists: no masks on the gathers
#pragma unroll
                for (int u = 0; u < PF; ++u) ld_row<V>(p.x + (int64_t)(cw[c0 + u] & ~SEG_ROW_START) * V, xv[u]);
            } else {
#pragma unroll
                for (int u = 0; u < PF; ++u) {
                    const int i = c0 + u;
                    if ((vm >> i) & 1u) {
                        ld_row<V>(p.x + (int64_t)(cw[i] & ~SEG_ROW_START) * V, xv[u]);
                    } else {
#pragma unroll
                        for (int j = 0; j < V; ++j) xv[u][j] = 0.0f;
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < PF; ++u) {
                const int i = c0 + u;
                const bool f = (fm >> i) & 1u;
                if (f) {
                    st_row<V>(rs + (slot >= 0 ? slot : TN - 1) * V, acc);
                    ++slot;
                }
                const float keep = f ? 0.0f : 1.0f;
                if constexpr (PAT) {
#pragma unroll
                    for (int j = 0; j < V; ++j) acc[j] = fmaf(acc[j], keep, xv[u][j]);
                } else {
#pragma unroll
                    for (int j = 0; j < V; ++j) acc[j] = fmaf(vv[i], xv[u][j], acc[j] * keep);
                }
            }
        }

        // 3. segmented scan of the lanes' trailing sums, restarting at lanes in
        //    which a row starts; acc of lane l becomes the sum from the last
        //    row start at or before lane l through the end of lane l
        int key = nf > 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            float up[V];
#pragma unroll
            for (int j = 0; j < V; ++j) up[j] = __shfl_up_sync(FULL, acc[j], o);
            const int kup = __shfl_up_sync(FULL, key, o);
            if (lane >= o) {
                if (!key) {
#pragma unroll
                    for (int j = 0; j < V; ++j) acc[j] += up[j];
                }
                key |= kup;
            }
        }
        // the row that ends at this lane's first row start: add what earlier lanes hold
        {
            float cin[V];
#pragma unroll
            for (int j = 0; j < V; ++j) {
                cin[j] = __shfl_up_sync(FULL, acc[j], 1);
                if (lane == 0) cin[j] = 0.0f;
            }
            if (nf > 0) {
                float *sp = rs + (excl > 0 ? excl - 1 : TN - 1) * V;
                float h[V];
                ld_row_smem<V>(sp, h);
#pragma unroll
                for (int j = 0; j < V; ++j) h[j] += cin[j];
                st_row<V>(sp, h);
            }
        }
        // carry-out of the tile, tagged with this launch and whether a row starts in it
        if (lane == 31) {
            const uint32_t tag = (ep << 1) | (q > 0 ? 1u : 0u);
#pragma unroll
            for (int j = 0; j < V; ++j) st_relaxed_u64(p.agg + t * V + j, seg_pack(acc[j], tag));
        }
        __syncwarp();

        // 4. the pending row of the warp's previous tile
        if (pend) {
            float back[V];
            const unsigned long long w = lane < V ? probe : 0ull;
            const bool ready = __all_sync(FULL, lane >= V || (uint32_t)(w >> 33) == ep);
            const bool start = __shfl_sync(FULL, (int)((w >> 32) & 1ull), 0) != 0;
            if (ready && start) {
#pragma unroll
                for (int j = 0; j < V; ++j) back[j] = __shfl_sync(FULL, __uint_as_float((uint32_t)w), j);
            } else {
                seg_lookback<V>(p, pend_t, ep, cv.hdr, lane, back);
            }
            if (lane == 0) {
                float tot[V];
#pragma unroll
                for (int j = 0; j < V; ++j) tot[j] = pend_part[j] + back[j];
                seg_emit<V, PAT>(p, (int64_t)pend_row, tot, alive, l1);
            }
            pend = false;
        }
        // the row that ends in this tile after starting in an earlier one (or
        // runs to the end of the matrix from an earlier tile) waits for the
        // warp's next tile
        const bool last = t == p.seg_tiles - 1;
        if ((q > 0 && t > 0) || (q == 0 && last)) {
            if (q > 0) {
                ld_row_smem<V>(rs + (TN - 1) * V, pend_part);
            } else {
#pragma unroll
                for (int j = 0; j < V; ++j) pend_part[j] = __shfl_sync(FULL, acc[j], 31);
            }
            pend = true;
            pend_t = t;
            pend_row = __ldg(p.nz_rows + crow0 - 1);
        }

        // 5. rows that start and end in the tile: lane per row, coalesced
        if (lane < q - 1) {
            float sv[V];
            ld_row_smem<V>(rs + lane * V, sv);
            seg_emit<V, PAT>(p, (int64_t)vk, sv, alive, l1);
        }
        for (int k = lane + 32; k < q - 1; k += 32) {
            float sv[V];
            ld_row_smem<V>(rs + k * V, sv);
            seg_emit<V, PAT>(p, (int64_t)__ldg(p.nz_rows + crow0 + k), sv, alive, l1);
        }
        // 6. the last row that starts in the last tile ends with the matrix
        if (last && q > 0 && lane == 31) seg_emit<V, PAT>(p, (int64_t)__ldg(p.nz_rows + crow0 + q - 1), acc, alive, l1);
        __syncwarp();   // rs is rewritten by the next tile
    }
    if (broke) {   // a stage never arrived: wait (bounded) for the copies still in flight before leaving
        const int64_t mine = t0 < p.seg_tiles ? (p.seg_tiles - 1 - t0) / nw + 1 : 0;
        for (int k = it; k < it + NB && k < mine; ++k) mbar_wait(bars + k % NB, (unsigned)(k / NB) & 1u, cv.hdr);
        pend = false;
    }
    if (pend) {
        float back[V];
        seg_lookback<V>(p, pend_t, ep, cv.hdr, lane, back);
        if (lane == 0) {
            float tot[V];
#pragma unroll
            for (int j = 0; j < V; ++j) tot[j] = pend_part[j] + back[j];
            seg_emit<V, PAT>(p, (int64_t)pend_row, tot, alive, l1);
        }
    }

    seg_close_launch<V>(p, cv, l1, ep_raw, lane, warp);
}

// ------------------------------------- segmented walk, gathers ahead ---
// The same walk with the gathers of a warp's next tile in flight while its
// current tile is summed: each lane copies the rows X[col] of its R nonzeros
// of the next tile into a shared-memory buffer with cp.async, which holds no
// register while the copies fly (two buffers per warp).  The walk then reads
// its rows from shared memory.  A row sum that a lane finishes is parked in
// the cell of a nonzero the lane has already consumed, and a table of cell
// positions (slot -> cell) lets the coalesced pass find the finished rows.
//
// Cell layout: the row of nonzero i of lane l is cell i*32 + l; a row of
// V <= 4 floats is one 4V-byte cell, a row of 8 floats two 16-byte halves TN
// cells apart, so the 16-byte reads of consecutive lanes hit consecutive
// banks.
template <int V, int R, int NB, bool PAT>
struct SegaSmem {
    static constexpr int TN = 32 * R;
    static constexpr size_t STAGE = (size_t)TN * sizeof(uint32_t) * (PAT ? 1 : 2);
    static constexpr size_t XB = (size_t)TN * V * sizeof(float);
    static constexpr size_t POS = (size_t)TN * sizeof(uint16_t);
    static constexpr size_t PER_WARP = NB * STAGE + 2 * XB + POS + 16 * NB;
    static constexpr size_t BYTES = SEG_WARPS * PER_WARP;
    static_assert(STAGE % 16 == 0 && XB % 16 == 0 && POS % 16 == 0, "16-byte sections");
};

template <int V, int TN>
__device__ __forceinline__ void sega_ld(const float *xb, int c, float (&o)[V])
{
    if constexpr (V == 8) {
        const float4 a = reinterpret_cast<const float4 *>(xb)[c];
        const float4 b = reinterpret_cast<const float4 *>(xb)[TN + c];
        o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w;
        o[4] = b.x; o[5] = b.y; o[6] = b.z; o[7] = b.w;
    } else {
        ld_row_smem<V>(xb + c * V, o);
    }
}

template <int V, int TN>
__device__ __forceinline__ void sega_st(float *xb, int c, const float (&v)[V])
{
    if constexpr (V == 8) {
        reinterpret_cast<float4 *>(xb)[c] = make_float4(v[0], v[1], v[2], v[3]);
        reinterpret_cast<float4 *>(xb)[TN + c] = make_float4(v[4], v[5], v[6], v[7]);
    } else {
        st_row<V>(xb + c * V, v);
    }
}

// cp.async of one row of V floats (global, 4V-byte aligned) into cell c.
template <int V, int TN>
__device__ __forceinline__ void sega_fetch(float *xb, int c, const float *src)
{
    const unsigned d = smem_u32(xb);
    if constexpr (V == 8) {
        asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(d + c * 16), "l"(src) : "memory");
        asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(d + (TN + c) * 16), "l"(src + 4) : "memory");
    } else {
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(d + c * V * 4), "l"(src), "n"(V * 4)
                     : "memory");
    }
}

__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

template <int N>
__device__ __forceinline__ void cpa_wait()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Take tile t from its stage: wait (bounded) for the stage, read the lane's
// R column words (and values), return the row-start flags of its existing
// nonzeros in fm, and send the gathers of their rows into buffer xb as one
// commit group.  False (the error flag raised) when the stage never arrived.
template <int V, int R, bool PAT>
__device__ __forceinline__ bool sega_take(const Params &p, const unsigned char *stage, uint64_t *bar,
                                          unsigned parity, Ctl *hdr, int64_t t, float *xb, int lane, unsigned &fm,
                                          float (&vv)[PAT ? 1 : R])
{
    constexpr int TN = 32 * R;
    if (!__all_sync(0xffffffffu, mbar_wait(bar, parity, hdr))) return false;
    uint32_t cw[R];
#pragma unroll
    for (int q = 0; q < R / 4; ++q) {
        const uint4 c = reinterpret_cast<const uint4 *>(stage)[lane * (R / 4) + q];
        cw[4 * q] = c.x;
        cw[4 * q + 1] = c.y;
        cw[4 * q + 2] = c.z;
        cw[4 * q + 3] = c.w;
        if constexpr (!PAT) {
            const float4 v4 = reinterpret_cast<const float4 *>(stage + TN * sizeof(uint32_t))[lane * (R / 4) + q];
            vv[4 * q] = v4.x;
            vv[4 * q + 1] = v4.y;
            vv[4 * q + 2] = v4.z;
            vv[4 * q + 3] = v4.w;
        }
    }
    const int64_t left = p.m - (t * TN + (int64_t)lane * R);
    const unsigned vm = left >= R ? (R == 32 ? 0xffffffffu : (1u << R) - 1u) : left > 0 ? (1u << left) - 1u : 0u;
    unsigned f = 0;
#pragma unroll
    for (int i = 0; i < R; ++i) {
        f |= (cw[i] >> 31) << i;
        if ((vm >> i) & 1u) sega_fetch<V, TN>(xb, i * 32 + lane, p.x + (int64_t)(cw[i] & ~SEG_ROW_START) * V);
    }
    fm = f & vm;
    cpa_commit();
    return true;
}

template <int V, int R, int PF, int NB, bool PAT>
__global__ void __launch_bounds__(SEG_WARPS * 32) spmm_sega_k(Params p)
{
    using SM = SegaSmem<V, R, NB, PAT>;
    static_assert(R % 4 == 0 && R % PF == 0 && R <= 32 && NB >= 2, "R");
    static_assert(V == 1 || V == 2 || V == 4 || V == 8, "V");
    static_assert(SM::TN <= 65536, "cell index in 16 bits");
    constexpr int TN = SM::TN;
    constexpr int XBF = (int)(SM::XB / sizeof(float));
    extern __shared__ __align__(128) unsigned char seg_smem[];
    const CtlView cv = ctl_view(p.ctl);
    if (gate_off(p.gate, p.ctl) || *(volatile int32_t *)&cv.hdr->done) return;
    const uint32_t ep_raw = *(volatile uint32_t *)&cv.hdr->epoch;
    const uint32_t ep = (ep_raw + 1u) & 0x7fffffffu;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned FULL = 0xffffffffu;
    unsigned char *wbase = seg_smem + (size_t)warp * SM::PER_WARP;
    float *xbuf = reinterpret_cast<float *>(wbase + NB * SM::STAGE);
    uint16_t *pos = reinterpret_cast<uint16_t *>(wbase + NB * SM::STAGE + 2 * SM::XB);
    uint64_t *bars = reinterpret_cast<uint64_t *>(wbase + NB * SM::STAGE + 2 * SM::XB + SM::POS);

    seg_zero_rows<V>(p);

    unsigned amask = 0;
    float l1[V];
#pragma unroll
    for (int j = 0; j < V; ++j) {
        amask |= (cv.alive[j] ? 1u : 0u) << j;
        l1[j] = 0.0f;
    }
    int alive[V];
#pragma unroll
    for (int j = 0; j < V; ++j) alive[j] = (amask >> j) & 1u;

    const int64_t nw = (int64_t)gridDim.x * SEG_WARPS;
    const int64_t t0 = (int64_t)blockIdx.x * SEG_WARPS + warp;
    const int64_t mine = t0 < p.seg_tiles ? (p.seg_tiles - 1 - t0) / nw + 1 : 0;   // tiles of this warp
    if (lane == 0) {
#pragma unroll
        for (int b = 0; b < NB; ++b) mbar_init(bars + b);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
#pragma unroll
        for (int b = 0; b < NB; ++b)
            if (b < mine) seg_issue<V, R, NB, PAT>(p, wbase + b * SM::STAGE, bars + b, t0 + b * nw);
    }
    __syncwarp();
    int32_t crow_next = mine > 0 ? __ldg(p.tile_crow0 + t0) : 0;

    bool pend = false;
    int64_t pend_t = 0;
    int32_t pend_row = 0;
    float pend_part[V];
#pragma unroll
    for (int j = 0; j < V; ++j) pend_part[j] = 0.0f;

    // the warp's first tile: flags, values and gathers
    unsigned fm = 0;
    float vv[PAT ? 1 : R];
    int64_t broke_at = -1;   // index of the warp tile whose stage never arrived
    if (mine > 0) {
        if (!sega_take<V, R, PAT>(p, wbase, bars, 0u, cv.hdr, t0, xbuf, lane, fm, vv)) {
            broke_at = 0;
        } else {
            __syncwarp();
            if (lane == 0 && NB < mine) seg_issue<V, R, NB, PAT>(p, wbase, bars, t0 + NB * nw);
        }
    }

    int it = 0;
    for (int64_t t = t0; broke_at < 0 && t < p.seg_tiles; t += nw, ++it) {
        float *xb = xbuf + (it & 1) * XBF;
        const int64_t crow0 = crow_next;
        if (t + nw < p.seg_tiles) crow_next = __ldg(p.tile_crow0 + t + nw);
        unsigned long long probe = 0ull;
        if (pend && lane < V) probe = ld_relaxed_u64(p.agg + (pend_t - 1) * V + lane);

        // 1. the next tile's gathers go out before this one is summed
        unsigned fm_nx = 0;
        float vv_nx[PAT ? 1 : R];
        if (it + 1 < mine) {
            const int k = it + 1, b = k % NB;
            if (!sega_take<V, R, PAT>(p, wbase + b * SM::STAGE, bars + b, (unsigned)(k / NB) & 1u, cv.hdr, t + nw,
                                      xbuf + (k & 1) * XBF, lane, fm_nx, vv_nx)) {
                cpa_wait<0>();
                broke_at = k;
                break;
            }
            __syncwarp();   // every lane has its words: the stage takes the warp's tile NB rounds ahead
            if (lane == 0 && k + NB < mine) seg_issue<V, R, NB, PAT>(p, wbase + b * SM::STAGE, bars + b, t + (NB + 1) * nw);
        } else {
            cpa_commit();   // an empty group: one group per tile
        }
        cpa_wait<1>();      // this lane's rows of tile t have landed

        const bool full = (t + 1) * TN <= p.m;
        const int64_t left = p.m - (t * TN + (int64_t)lane * R);
        const unsigned vm = left >= R ? (R == 32 ? FULL : (1u << R) - 1u) : left > 0 ? (1u << left) - 1u : 0u;
        const int nf = __popc(fm);
        int incl = nf;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += y;
        }
        const int excl = incl - nf;
        const int q = __shfl_sync(FULL, incl, 31);
        // ids (and pattern-only weights) of the rows the coalesced pass finishes, loaded early
        const int32_t vk = lane < q - 1 ? __ldg(p.nz_rows + crow0 + lane) : 0;
        const float wk = (PAT && p.mode == MODE_ACC && lane < q - 1) ? __ldg(p.inv_deg + vk) : 0.0f;

        // 2. the walk over the rows in shared memory: at a row start the
        //    running sum is parked in the cell of the lane's previous nonzero
        float acc[V];
#pragma unroll
        for (int j = 0; j < V; ++j) acc[j] = 0.0f;
        int seen = 0;   // row starts passed in this lane
#pragma unroll
        for (int c0 = 0; c0 < R; c0 += PF) {
            float xv[PF][V];
#pragma unroll
            for (int u = 0; u < PF; ++u) {
                const int i = c0 + u;
                sega_ld<V, TN>(xb, i * 32 + lane, xv[u]);
                if (!full && !((vm >> i) & 1u)) {
#pragma unroll
                    for (int j = 0; j < V; ++j) xv[u][j] = 0.0f;
                }
            }
#pragma unroll
            for (int u = 0; u < PF; ++u) {
                const int i = c0 + u;
                const bool f = (fm >> i) & 1u;
                if (i > 0 && f) {
                    sega_st<V, TN>(xb, (i - 1) * 32 + lane, acc);
                    if (seen > 0) pos[excl + seen - 1] = (uint16_t)((i - 1) * 32 + lane);
                }
                seen += f ? 1 : 0;
                const float keep = f ? 0.0f : 1.0f;
                if constexpr (PAT) {
#pragma unroll
                    for (int j = 0; j < V; ++j) acc[j] = fmaf(acc[j], keep, xv[u][j]);
                } else {
#pragma unroll
                    for (int j = 0; j < V; ++j) acc[j] = fmaf(vv[i], xv[u][j], acc[j] * keep);
                }
            }
        }

        // 3. segmented scan of the lanes' trailing sums (as in spmm_seg_k)
        int key = nf > 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            float up[V];
#pragma unroll
            for (int j = 0; j < V; ++j) up[j] = __shfl_up_sync(FULL, acc[j], o);
            const int kup = __shfl_up_sync(FULL, key, o);
            if (lane >= o) {
                if (!key) {
#pragma unroll
                    for (int j = 0; j < V; ++j) acc[j] += up[j];
                }
                key |= kup;
            }
        }
        // the row that ends at this lane's first row start: its part in this
        // lane (cell of the nonzero before the start; none when the start is
        // the lane's first nonzero, whose sum then parks in the lane's last
        // cell, never a parking cell) plus what earlier lanes hold
        {
            float cin[V];
#pragma unroll
            for (int j = 0; j < V; ++j) {
                cin[j] = __shfl_up_sync(FULL, acc[j], 1);
                if (lane == 0) cin[j] = 0.0f;
            }
            if (nf > 0) {
                const int i0 = __ffs(fm) - 1;
                const int c = (i0 > 0 ? i0 - 1 : R - 1) * 32 + lane;
                float h[V];
                if (i0 > 0) {
                    sega_ld<V, TN>(xb, c, h);
                } else {
#pragma unroll
                    for (int j = 0; j < V; ++j) h[j] = 0.0f;
                }
#pragma unroll
                for (int j = 0; j < V; ++j) h[j] += cin[j];
                sega_st<V, TN>(xb, c, h);
                pos[excl > 0 ? excl - 1 : TN - 1] = (uint16_t)c;
            }
        }
        // carry-out of the tile, tagged with this launch and whether a row starts in it
        if (lane == 31) {
            const uint32_t tag = (ep << 1) | (q > 0 ? 1u : 0u);
#pragma unroll
            for (int j = 0; j < V; ++j) st_relaxed_u64(p.agg + t * V + j, seg_pack(acc[j], tag));
        }
        __syncwarp();

        // 4. the pending row of the warp's previous tile
        if (pend) {
            float back[V];
            const unsigned long long w = lane < V ? probe : 0ull;
            const bool ready = __all_sync(FULL, lane >= V || (uint32_t)(w >> 33) == ep);
            const bool start = __shfl_sync(FULL, (int)((w >> 32) & 1ull), 0) != 0;
            if (ready && start) {
#pragma unroll
                for (int j = 0; j < V; ++j) back[j] = __shfl_sync(FULL, __uint_as_float((uint32_t)w), j);
            } else {
                seg_lookback<V>(p, pend_t, ep, cv.hdr, lane, back);
            }
            if (lane == 0) {
                float tot[V];
#pragma unroll
                for (int j = 0; j < V; ++j) tot[j] = pend_part[j] + back[j];
                seg_emit<V, PAT>(p, (int64_t)pend_row, tot, alive, l1);
            }
            pend = false;
        }
        const bool last = t == p.seg_tiles - 1;
        if ((q > 0 && t > 0) || (q == 0 && last)) {
            if (q > 0) {
                sega_ld<V, TN>(xb, pos[TN - 1], pend_part);
            } else {
#pragma unroll
                for (int j = 0; j < V; ++j) pend_part[j] = __shfl_sync(FULL, acc[j], 31);
            }
            pend = true;
            pend_t = t;
            pend_row = __ldg(p.nz_rows + crow0 - 1);
        }

        // 5. rows that start and end in the tile: lane per row, coalesced
        if (lane < q - 1) {
            float sv[V];
            sega_ld<V, TN>(xb, pos[lane], sv);
            seg_emit_w<V, PAT>(p, (int64_t)vk, sv, alive, l1, wk);
        }
        for (int k = lane + 32; k < q - 1; k += 32) {
            float sv[V];
            sega_ld<V, TN>(xb, pos[k], sv);
            seg_emit<V, PAT>(p, (int64_t)__ldg(p.nz_rows + crow0 + k), sv, alive, l1);
        }
        // 6. the last row that starts in the last tile ends with the matrix
        if (last && q > 0 && lane == 31) seg_emit<V, PAT>(p, (int64_t)__ldg(p.nz_rows + crow0 + q - 1), acc, alive, l1);
        fm = fm_nx;
        if constexpr (!PAT) {
#pragma unroll
            for (int i = 0; i < R; ++i) vv[i] = vv_nx[i];
        }
        __syncwarp();   // the buffer and the cell table are rewritten two tiles on
    }
    if (broke_at >= 0) {   // a stage never arrived: wait (bounded) for the copies still in flight before leaving
        for (int64_t k = broke_at; k < broke_at + NB && k < mine; ++k)
            mbar_wait(bars + k % NB, (unsigned)(k / NB) & 1u, cv.hdr);
        pend = false;
    }
    if (pend) {
        float back[V];
        seg_lookback<V>(p, pend_t, ep, cv.hdr, lane, back);
        if (lane == 0) {
            float tot[V];
#pragma unroll
            for (int j = 0; j < V; ++j) tot[j] = pend_part[j] + back[j];
            seg_emit<V, PAT>(p, (int64_t)pend_row, tot, alive, l1);
        }
    }
    seg_close_launch<V>(p, cv, l1, ep_raw, lane, warp);
}

// The TPA finalize r_TPA = (1+alpha) r_family + r~_stranger for the rows the
// segmented kernel does not visit: the rows without nonzeros, or every row
// when all columns stopped before the last family iteration (that launch
// then returned at once).
__global__ void finalize_seg_k(const void *ctl, const int32_t *empty_rows, int64_t n_empty, const float *r,
                               int64_t ldr, const float *r_str, float opa, float *out, int64_t ldo, int64_t n, int k)
{
    const CtlView cv = ctl_view(const_cast<void *>(ctl));
    const bool all = *(volatile int32_t *)&cv.hdr->done != 0;
    const int64_t rows = all ? n : n_empty;
    // thread per row; 16-byte loads and stores when the rows allow them
    const bool vec = k % 4 == 0 && ldr % 4 == 0 && ldo % 4 == 0 && (reinterpret_cast<uintptr_t>(r) & 15) == 0 &&
                     (reinterpret_cast<uintptr_t>(out) & 15) == 0;
    for (int64_t rr = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; rr < rows; rr += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = all ? rr : (int64_t)empty_rows[rr];
        const float rs = r_str[v];
        if (vec) {
            for (int j = 0; j < k; j += 4) {
                const float4 a = *reinterpret_cast<const float4 *>(r + v * ldr + j);
                *reinterpret_cast<float4 *>(out + v * ldo + j) =
                    make_float4(fmaf(opa, a.x, rs), fmaf(opa, a.y, rs), fmaf(opa, a.z, rs), fmaf(opa, a.w, rs));
            }
        } else {
            for (int j = 0; j < k; ++j) out[v * ldo + j] = fmaf(opa, r[v * ldr + j], rs);
        }
    }
}

// ---------------------------------------------------- plan of the walk ---
// nzf[v] = 1 when row v has a nonzero, ef[v] = 1 when it has none.
__global__ void seg_row_flags_k(const int64_t *rp, int64_t n, int32_t *nzf, int32_t *ef)
{
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const int nz = rp[v + 1] > rp[v] ? 1 : 0;
        nzf[v] = nz;
        ef[v] = 1 - nz;
    }
}

__global__ void seg_scatter_rows_k(const int64_t *rp, int64_t n, const int64_t *nzpos, const int64_t *epos,
                                   int32_t *nz_rows, int32_t *empty_rows)
{
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        if (rp[v + 1] > rp[v]) nz_rows[nzpos[v]] = (int32_t)v;
        else empty_rows[epos[v]] = (int32_t)v;
    }
}

// colf[e] = col[e] for e < m, 0 in the padding up to total.
__global__ void seg_copy_cols_k(const int32_t *col, int64_t m, int64_t total, uint32_t *colf)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
        colf[e] = e < m ? (uint32_t)col[e] : 0u;
}

// Mark the first nonzero of every nonempty row.
__global__ void seg_mark_k(const int64_t *rp, int64_t n, uint32_t *colf)
{
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        if (rp[v + 1] > rp[v]) colf[rp[v]] |= SEG_ROW_START;
}

// crow0[t] = number of nonempty rows whose first nonzero precedes t * tn,
// for t = 0 .. tiles (nzpos: exclusive prefix of the nonempty-row flags and
// their total at n).
__global__ void seg_tiles_k(const int64_t *rp, int64_t n, int64_t m, const int64_t *nzpos, int64_t tn, int64_t tiles,
                            int32_t *crow0)
{
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t <= tiles; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t X = t * tn;
        if (X >= m) {
            crow0[t] = (int32_t)nzpos[n];
            continue;
        }
        int64_t lo = 0, hi = n;   // first v with rp[v] >= X (rp[n] = m > X)
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (rp[mid] >= X) hi = mid; else lo = mid + 1;
        }
        crow0[t] = (int32_t)nzpos[lo];
    }
}

}  // namespace tpa
