// Binned-row SpMV/SpMM of one CPI iteration (Algorithm 1), the alternative to
// the merge path for narrow batches.  Rows of A~^T are binned once per graph
// by their number of nonzeros (in-degree):
//   short  (1..BIN_SHORT)  : LPR = KP lanes per row, 32 / KP rows per warp;
//   medium (..BIN_MEDIUM)  : one warp per row;
//   long   (> BIN_MEDIUM)  : cut into chunks of BIN_CHUNK nonzeros, one warp
//                            per chunk writes its partial sums, which a
//                            combine pass adds per row in chunk order;
//   empty                  : y = 0 (r unchanged), or the finalize alone.
// In every bin a lane owns whole nonzeros: it gathers the full row
// X[col][0..KP) (one 32-byte sector for KP = 8) and multiplies by the value,
// so a row is summed by plain loads and FMAs in registers with no merge-path
// search, step test or carry.  The lanes of a row then reduce-scatter their
// KP-vectors (log2 rounds of shuffles that halve the vector), after which
// each lane holds one finished column and the epilogue writes consecutive
// columns from consecutive lanes.  L1 partials of the break test are kept per
// lane and written once per warp (or block) to fixed rows of tl1; the finish
// kernel sums them in a fixed order and applies the test.  Every row is
// finished by exactly one kernel, so r gets one add per element per launch
// (deterministic), and summation orders are fixed by the lane layout.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "tpa_internal.cuh"

namespace tpa {

constexpr int BIN_SHORT = 32;
constexpr int BIN_MEDIUM = 512;
constexpr int BIN_CHUNK = 512;
constexpr int BIN_WARPS = 8;   // warps per block of the binned kernels

// Sum a KP-vector over the LPR lanes of a lane group (LPR a power of two,
// aligned in the warp) by recursive halving: at the rounds with offsets
// LPR/2, LPR/4, ... a lane keeps one half of its vector (the upper half when
// the offset bit of its sub-lane index is set), sends the other half to its
// partner and adds what it receives; once the vector has one element, the
// remaining rounds add across the lanes that hold the same column.  Returns
// the lane's finished column sum; col is its column index.  Fixed order.
template <int KP, int LPR>
__device__ __forceinline__ float reduce_scatter(const float (&a)[KP], int sub, int &col)
{
    float v[KP];
#pragma unroll
    for (int j = 0; j < KP; ++j) v[j] = a[j];
    col = 0;
    int len = KP;
#pragma unroll
    for (int o = LPR / 2; o > 0; o >>= 1) {
        if (len > 1) {
            const int h = len / 2;
            const bool up = (sub & o) != 0;
#pragma unroll
            for (int i = 0; i < (KP > 1 ? KP / 2 : 1); ++i) {
                if (i < h) {
                    const float send = up ? v[i] : v[i + h];
                    const float keep = up ? v[i + h] : v[i];
                    v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
                }
            }
            if (up) col += h;
            len = h;
        } else {
            v[0] += __shfl_xor_sync(0xffffffffu, v[0], o);
        }
    }
    return v[0];
}

// Epilogue of Algorithm 1 for column c of a finished row whose sum is s.
__device__ __forceinline__ void epilogue_col(const Params &p, int64_t row, int c, int KP, float s, bool alive_c,
                                             float &l1)
{
    const float y = p.decay * s;
    const bool valid = c < p.k;
    const bool run = valid && alive_c;
    if (p.mode == MODE_ACC) {
        p.y[row * KP + c] = p.inv_deg ? y * __ldg(p.inv_deg + row) : y;   // the next product's x
        if (p.accumulate && run) atomicAdd(p.r + row * p.ldr + c, y);
    } else if (valid) {
        float fam = p.r[row * p.ldr + c];
        if (alive_c) fam += y;
        p.out[row * p.ldo + c] = fmaf(p.one_plus_alpha, fam, p.r_str[row]);
    }
    l1 += run ? fabsf(y) : 0.0f;
}

// Short rows: LPR = KP lanes per row, the lanes of a row take its nonzeros
// round-robin (at most BIN_SHORT / KP each).
template <int KP>
__global__ void __launch_bounds__(BIN_WARPS * 32) bin_short_k(Params p)
{
    constexpr int LPR = KP < 32 ? KP : 32;
    constexpr int RPW = 32 / LPR;
    const CtlView cv = ctl_view(p.ctl);
    if (gate_off(p.gate, p.ctl) || *(volatile int32_t *)&cv.hdr->done) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int sub = lane % LPR, grp = lane / LPR;
    int col = 0;
    {
        float dummy[KP];
#pragma unroll
        for (int j = 0; j < KP; ++j) dummy[j] = 0.0f;
        (void)reduce_scatter<KP, LPR>(dummy, sub, col);   // column layout only
    }
    const bool alive_c = col < p.k && cv.alive[col];
    float l1 = 0.0f;
    const int64_t groups = (p.n_short + RPW - 1) / RPW;
    for (int64_t gi = (int64_t)blockIdx.x * BIN_WARPS + warp; gi < groups; gi += (int64_t)gridDim.x * BIN_WARPS) {
        const int64_t idx = gi * RPW + grp;
        int64_t row = -1, e0 = 0, e1 = 0;
        if (idx < p.n_short) {
            row = __ldg(p.rows_short + idx);
            e0 = __ldg(p.rp + row);
            e1 = __ldg(p.rp + row + 1);
        }
        float acc[KP];
#pragma unroll
        for (int j = 0; j < KP; ++j) acc[j] = 0.0f;
#pragma unroll 4
        for (int64_t e = e0 + sub; e < e1; e += LPR) {
            const int32_t c = __ldcs(p.col + e);
            const float v = p.inv_deg ? 1.0f : __ldcs(p.val + e);
            float xv[KP];
            ld_row<KP>(p.x + (int64_t)c * KP, xv);
#pragma unroll
            for (int j = 0; j < KP; ++j) acc[j] = fmaf(v, xv[j], acc[j]);
        }
        int c;
        const float s = reduce_scatter<KP, LPR>(acc, sub, c);
        if (row >= 0 && sub < KP) epilogue_col(p, row, c, KP, s, alive_c, l1);
    }
    // one column per lane: add over the row groups of the warp, write per warp
#pragma unroll
    for (int o = LPR; o < 32; o <<= 1) l1 += __shfl_xor_sync(0xffffffffu, l1, o);
    if (lane < LPR && sub < KP) p.tl1[(p.slot0 + (int64_t)blockIdx.x * BIN_WARPS + warp) * KP + col] = l1;
}

// Medium rows (CHUNK = false: one warp per row, epilogue) and the chunks of
// long rows (CHUNK = true: one warp per chunk, partial sums to cpart).
template <int KP, bool CHUNK>
__global__ void __launch_bounds__(BIN_WARPS * 32) bin_warp_k(Params p)
{
    static_assert(KP <= 32, "KP");
    constexpr int SPAN = 32 / KP;   // lanes left holding the same column
    const CtlView cv = ctl_view(p.ctl);
    if (gate_off(p.gate, p.ctl) || *(volatile int32_t *)&cv.hdr->done) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int col = 0;
    {
        float dummy[KP];
#pragma unroll
        for (int j = 0; j < KP; ++j) dummy[j] = 0.0f;
        (void)reduce_scatter<KP, 32>(dummy, lane, col);   // column layout only
    }
    const bool writer = lane % SPAN == 0;
    const bool alive_c = col < p.k && cv.alive[col];
    float l1 = 0.0f;
    const int64_t count = CHUNK ? p.n_chunks : p.n_mid;
    for (int64_t i = (int64_t)blockIdx.x * BIN_WARPS + warp; i < count; i += (int64_t)gridDim.x * BIN_WARPS) {
        int64_t row, e0, e1;
        if (CHUNK) {
            row = __ldg(p.rows_long + __ldg(p.chunk_row + i));
            e0 = __ldg(p.chunk_e0 + i);
            e1 = min(e0 + (int64_t)BIN_CHUNK, __ldg(p.rp + row + 1));
        } else {
            row = __ldg(p.rows_mid + i);
            e0 = __ldg(p.rp + row);
            e1 = __ldg(p.rp + row + 1);
        }
        float acc[KP];
#pragma unroll
        for (int j = 0; j < KP; ++j) acc[j] = 0.0f;
#pragma unroll 4
        for (int64_t e = e0 + lane; e < e1; e += 32) {
            const int32_t c = __ldcs(p.col + e);
            const float v = p.inv_deg ? 1.0f : __ldcs(p.val + e);
            float xv[KP];
            ld_row<KP>(p.x + (int64_t)c * KP, xv);
#pragma unroll
            for (int j = 0; j < KP; ++j) acc[j] = fmaf(v, xv[j], acc[j]);
        }
        int c;
        const float s = reduce_scatter<KP, 32>(acc, lane, c);
        if (writer) {
            if (CHUNK) p.cpart[i * KP + c] = s;
            else epilogue_col(p, row, c, KP, s, alive_c, l1);
        }
    }
    if (!CHUNK && writer) p.tl1[(p.slot0 + (int64_t)blockIdx.x * BIN_WARPS + warp) * KP + col] = l1;
}

// Long rows: one thread per (row, column) adds the row's chunk sums in chunk
// order, then the epilogue; L1 partial per block.
template <int KP>
__global__ void __launch_bounds__(256) bin_long_k(Params p)
{
    static_assert(256 % KP == 0, "KP");
    __shared__ float s_l1[256];
    const CtlView cv = ctl_view(p.ctl);
    if (gate_off(p.gate, p.ctl) || *(volatile int32_t *)&cv.hdr->done) return;
    const int64_t t = (int64_t)blockIdx.x * 256 + threadIdx.x;
    const int64_t j = t / KP;
    const int c = (int)(t % KP);
    float l1 = 0.0f;
    if (j < p.n_long) {
        const int64_t f0 = __ldg(p.long_first64 + j), f1 = __ldg(p.long_first64 + j + 1);
        float s = 0.0f;
        for (int64_t f = f0; f < f1; ++f) s += p.cpart[f * KP + c];
        epilogue_col(p, __ldg(p.rows_long + j), c, KP, s, c < p.k && cv.alive[c], l1);
    }
    s_l1[threadIdx.x] = l1;
    __syncthreads();
    if (threadIdx.x < KP) {
        float a = 0.0f;
        for (int g = 0; g < 256 / KP; ++g) a += s_l1[g * KP + threadIdx.x];
        p.tl1[(p.slot0 + blockIdx.x) * KP + threadIdx.x] = a;
    }
}

// Rows without nonzeros: y = 0 (r unchanged), or the finalize alone.
template <int KP>
__global__ void bin_empty_k(Params p)
{
    const CtlView cv = ctl_view(p.ctl);
    if (gate_off(p.gate, p.ctl) || *(volatile int32_t *)&cv.hdr->done) return;
    const int64_t total = p.n_empty * KP;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = __ldg(p.rows_empty + t / KP);
        const int c = (int)(t % KP);
        if (p.mode == MODE_ACC)
            p.y[row * KP + c] = 0.0f;
        else if (c < p.k)
            p.out[row * p.ldo + c] = fmaf(p.one_plus_alpha, p.r[row * p.ldr + c], p.r_str[row]);
    }
}

// One block: the L1 norms of the iterate from the l1_slots rows of tl1 (fixed
// order), and the break test of Algorithm 1 per column.
template <int KP>
__global__ void __launch_bounds__(256) bin_finish_k(Params p)
{
    __shared__ double s_fin[256];
    const CtlView cv = ctl_view(p.ctl);
    if (gate_off(p.gate, p.ctl) || *(volatile int32_t *)&cv.hdr->done) return;
    block_sum_partials_t<KP, float>(p.tl1, (unsigned)p.l1_slots, s_fin);
    if (threadIdx.x < KP) {
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
        for (int c = 0; c < p.k && c < KP; ++c) any |= cv.alive[c];
        cv.hdr->done = any ? 0 : 1;
    }
}

// ---------------------------------------------------- binning the rows ---
// flags[b * n + v] = 1 when row v falls in bin b (0 short, 1 medium, 2 long,
// 3 empty).
__global__ void bin_classify_k(const int64_t *rp, int64_t n, int32_t *flags)
{
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const int64_t d = rp[v + 1] - rp[v];
        const int b = d == 0 ? 3 : d <= BIN_SHORT ? 0 : d <= BIN_MEDIUM ? 1 : 2;
#pragma unroll
        for (int q = 0; q < 4; ++q) flags[q * n + v] = q == b;
    }
}

// Row ids of each bin in ascending order, from the exclusive prefix sums of
// the flags (pos[b * (n + 1) + v]); chunk counts of the long rows.
__global__ void bin_scatter_k(const int64_t *rp, int64_t n, const int32_t *flags, const int64_t *pos,
                              int32_t *rows_short, int32_t *rows_mid, int32_t *rows_long, int32_t *rows_empty,
                              int32_t *long_cnt)
{
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        if (flags[v]) rows_short[pos[v]] = (int32_t)v;
        if (flags[n + v]) rows_mid[pos[(n + 1) + v]] = (int32_t)v;
        if (flags[2 * n + v]) {
            const int64_t j = pos[2 * (n + 1) + v];
            rows_long[j] = (int32_t)v;
            long_cnt[j] = (int32_t)((rp[v + 1] - rp[v] + BIN_CHUNK - 1) / BIN_CHUNK);
        }
        if (flags[3 * n + v]) rows_empty[pos[3 * (n + 1) + v]] = (int32_t)v;
    }
}

// Chunk list of the long rows from their exclusive chunk offsets.
__global__ void bin_chunks_k(const int64_t *rp, const int32_t *rows_long, int64_t n_long, const int64_t *first,
                             int32_t *chunk_row, int64_t *chunk_e0)
{
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n_long; j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e0 = rp[rows_long[j]];
        for (int64_t q = first[j]; q < first[j + 1]; ++q) {
            chunk_row[q] = (int32_t)j;
            chunk_e0[q] = e0 + (q - first[j]) * BIN_CHUNK;
        }
    }
}

}  // namespace tpa
