// Lane-segment walk: the SpMV/SpMM of one CPI iteration (Algorithm 1,
// x_i = (1-c) A~^T x_{i-1}) as two launches, with no waits between warps.
// Included once, by cpi.cu, after spmm_seg.cuh.
//
//   1. spmm_lane_k: a warp takes a tile of 32 R consecutive nonzeros of
//      CSR(A~^T), lane l the R nonzeros [l*R, l*R + R) of it.  The lane reads
//      their column words (bit 31 marks a row's first nonzero), gathers the
//      rows of x and keeps one running sum; a row that begins and ends in the
//      lane goes to lrec[rank of the row among the nonempty rows] at once.
//      One segmented shuffle scan over the lanes then adds the parts of rows
//      that cross lanes: the row ending at a lane's first row start gets its
//      part in the tile in lrec, and lane 31 writes the part of the row open
//      at the tile's end to ltail[tile].
//   2. lane_finish_k: thread per nonempty row (rank k), nonzeros [q0, q1]:
//      the row's parts are ltail[q0/W .. q1/W - 1] (W = 32 R) and, last,
//      lrec[k] when the row ends inside a tile (else ltail[q1/W]), added in
//      that order; then the epilogue of Algorithm 1 (y, r += y, or the TPA
//      finalize), the L1 partials, and in the last block the break test.
//      Rows spanning more than LANE_SHORT tiles (hubs) are summed by the
//      whole warp in a fixed lane-strided order.  Rows without nonzeros are
//      cleared (zero_mode) as for the segmented walk.
// Every sum has a fixed order, so results are identical run to run.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace tpa {

constexpr int LANE_SHORT = 32;

template <int V, int R, int PF, bool PAT>
__global__ void __launch_bounds__(256) spmm_lane_k(Params p)
{
    static_assert(R % 16 == 0 && 16 % PF == 0, "R, PF");
    static_assert(V == 1 || V == 2 || V == 4 || V == 8, "V");
    const CtlView cv = ctl_view(p.ctl);
    if (gate_off(p.gate, p.ctl) || *(volatile int32_t *)&cv.hdr->done) return;
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // a warp takes 32 consecutive segments (a warp tile of 32 R nonzeros) per round
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < p.seg_tiles;
         base += stride) {
        const int64_t L = base + lane;
        const bool live = L < p.seg_tiles;
        const int64_t e0 = L * R;
        const bool full = live && e0 + R <= p.m;      // every nonzero of the segment exists
        const int32_t c0 = live ? __ldg(p.tile_crow0 + L) : 0;   // nonempty rows begun before the segment
        float acc[V], hd[V];
#pragma unroll
        for (int j = 0; j < V; ++j) acc[j] = hd[j] = 0.0f;
        int nf = 0;   // row starts seen in the segment
        if (live) {
#pragma unroll
            for (int h = 0; h < R; h += 16) {
                uint32_t cw[16];
                float vv[PAT ? 1 : 16];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const uint4 c = __ldg(reinterpret_cast<const uint4 *>(p.colf + e0 + h) + q);
                    cw[4 * q] = c.x;
                    cw[4 * q + 1] = c.y;
                    cw[4 * q + 2] = c.z;
                    cw[4 * q + 3] = c.w;
                    if constexpr (!PAT) {
                        const float4 w = __ldg(reinterpret_cast<const float4 *>(p.val + e0 + h) + q);
                        vv[4 * q] = w.x;
                        vv[4 * q + 1] = w.y;
                        vv[4 * q + 2] = w.z;
                        vv[4 * q + 3] = w.w;
                    }
                }
#pragma unroll
                for (int c = 0; c < 16; c += PF) {
                    float xv[PF][V];
                    if (full) {   // no masks: the PF gathers go out together
#pragma unroll
                        for (int u = 0; u < PF; ++u)
                            ld_row<V>(p.x + (int64_t)(cw[c + u] & ~SEG_ROW_START) * V, xv[u]);
                    } else {
#pragma unroll
                        for (int u = 0; u < PF; ++u) {
                            if (e0 + h + c + u < p.m) {
                                ld_row<V>(p.x + (int64_t)(cw[c + u] & ~SEG_ROW_START) * V, xv[u]);
                            } else {
#pragma unroll
                                for (int j = 0; j < V; ++j) xv[u][j] = 0.0f;
                            }
                        }
                    }
#pragma unroll
                    for (int u = 0; u < PF; ++u) {
                        const int i = h + c + u;
                        const bool f = (cw[c + u] >> 31) != 0u && (full || e0 + i < p.m);
                        if (f) {
                            // the row that ends before this start: a row begun in
                            // this segment is complete; the first one keeps its
                            // part here for the warp's scan below
                            if (nf > 0) {
                                st_row<V>(p.lrec + (int64_t)(c0 + nf - 1) * V, acc);
                            } else {
#pragma unroll
                                for (int j = 0; j < V; ++j) hd[j] = acc[j];
                            }
                        }
                        nf += f ? 1 : 0;
                        const float keep = f ? 0.0f : 1.0f;
                        if constexpr (PAT) {
#pragma unroll
                            for (int j = 0; j < V; ++j) acc[j] = fmaf(acc[j], keep, xv[u][j]);
                        } else {
#pragma unroll
                            for (int j = 0; j < V; ++j) acc[j] = fmaf(vv[c + u], xv[u][j], acc[j] * keep);
                        }
                    }
                }
            }
        }
        // segmented scan of the lanes' end sums over the warp tile, restarting
        // at lanes in which a row starts: acc of lane l becomes the part, in
        // the tile, of the row open at the end of lane l
        const int key = nf > 0;
        int k = key;
        float cin[V];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            float up[V];
#pragma unroll
            for (int j = 0; j < V; ++j) up[j] = __shfl_up_sync(FULL, acc[j], o);
            const int kup = __shfl_up_sync(FULL, k, o);
            if (lane >= o) {
                if (!k) {
#pragma unroll
                    for (int j = 0; j < V; ++j) acc[j] += up[j];
                }
                k |= kup;
            }
        }
#pragma unroll
        for (int j = 0; j < V; ++j) {
            cin[j] = __shfl_up_sync(FULL, acc[j], 1);
            if (lane == 0) cin[j] = 0.0f;
        }
        // the row that ends at this lane's first row start: its part in the tile
        if (key && c0 > 0) {   // (no row ends before the matrix's first nonzero)
#pragma unroll
            for (int j = 0; j < V; ++j) hd[j] += cin[j];
            st_row<V>(p.lrec + (int64_t)(c0 - 1) * V, hd);
        }
        if (lane == 31) st_row<V>(p.ltail + (base / 32) * V, acc);
    }
}

// Epilogue of one finished row: with accumulation, y stored and r += y by a
// vector atomic (the row has this one writer, so the sum is the same every
// run), w = RN32(1/outdeg) of the row for pattern-only products; otherwise
// the TPA finalize, which reads r.
template <int V>
__device__ __forceinline__ void lane_emit(const Params &p, int64_t v, const float (&s)[V], const int (&alive)[V],
                                          float (&l1)[V], float w)
{
    if (p.mode == MODE_ACC) {
        if (p.inv_deg)
            epilogue_red<V, V, PM_PATTERN>(p, v, 0, s, alive, l1, w);
        else
            epilogue_red<V, V, PM_VALUED>(p, v, 0, s, alive, l1, w);
    } else {
        epilogue<V, V>(p, v, 0, s, alive, l1);
    }
}

template <int V, int R>
__global__ void __launch_bounds__(256) lane_finish_k(Params p)
{
    constexpr int64_t W = 32 * R;   // nonzeros per warp tile
    __shared__ float s_red[8][V];
    __shared__ double s_fin[256];
    __shared__ int s_last;
    const CtlView cv = ctl_view(p.ctl);
    if (gate_off(p.gate, p.ctl) || *(volatile int32_t *)&cv.hdr->done) return;
    seg_zero_rows<V>(p);
    int alive[V];
#pragma unroll
    for (int q = 0; q < V; ++q) alive[q] = cv.alive[q];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float l1[V];
#pragma unroll
    for (int q = 0; q < V; ++q) l1[q] = 0.0f;
    const int64_t nnz_rows = p.n - p.n_empty;
    const int64_t step = (int64_t)gridDim.x * 256;
    // two rows per thread in flight: ranks k and k + step
    for (int64_t base = (int64_t)blockIdx.x * 256; base < nnz_rows; base += 2 * step) {
        int32_t v[2] = {0, 0};
        int64_t L0[2] = {0, 0}, L1[2] = {0, 0};
        const float *last[2];
        bool mine[2], longspan[2];
        float w[2] = {0.0f, 0.0f};
#pragma unroll
        for (int h = 0; h < 2; ++h) {   // row, first and last nonzero: independent loads
            const int64_t k = base + threadIdx.x + h * step;
            mine[h] = k < nnz_rows;
            bool inside = false;
            if (mine[h]) {
                v[h] = __ldg(p.nz_rows + k);
                const int64_t q0 = __ldg(p.nzrp + k), q1 = __ldg(p.nzrp + k + 1) - 1;
                L0[h] = q0 / W;
                L1[h] = q1 / W;
                inside = q1 % W != W - 1 && q1 != p.m - 1;
            }
            last[h] = inside ? p.lrec + (mine[h] ? k : 0) * V : p.ltail + L1[h] * V;
            longspan[h] = mine[h] && L1[h] - L0[h] > LANE_SHORT;
        }
#pragma unroll
        for (int h = 0; h < 2; ++h)
            if (mine[h] && p.inv_deg && p.mode == MODE_ACC) w[h] = __ldg(p.inv_deg + v[h]);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            if (mine[h] && !longspan[h]) {
                float sum[V];
#pragma unroll
                for (int q = 0; q < V; ++q) sum[q] = 0.0f;
                for (int64_t u = L0[h]; u < L1[h]; ++u) {
                    float t[V];
                    ld_row<V>(p.ltail + u * V, t);
#pragma unroll
                    for (int q = 0; q < V; ++q) sum[q] += t[q];
                }
                float t[V];
                ld_row<V>(last[h], t);
#pragma unroll
                for (int q = 0; q < V; ++q) sum[q] += t[q];
                lane_emit<V>(p, (int64_t)v[h], sum, alive, l1, w[h]);
            }
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            unsigned lm = __ballot_sync(0xffffffffu, longspan[h]);
            while (lm) {
                const int src = __ffs(lm) - 1;
                lm &= lm - 1;
                const int64_t a = __shfl_sync(0xffffffffu, L0[h], src);
                const int64_t b = __shfl_sync(0xffffffffu, L1[h], src);
                float part[V];
#pragma unroll
                for (int q = 0; q < V; ++q) part[q] = 0.0f;
                for (int64_t u = a + lane; u < b; u += 32) {
                    float t[V];
                    ld_row<V>(p.ltail + u * V, t);
#pragma unroll
                    for (int q = 0; q < V; ++q) part[q] += t[q];
                }
#pragma unroll
                for (int q = 0; q < V; ++q) {
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) part[q] += __shfl_xor_sync(0xffffffffu, part[q], o);
                }
                if (lane == src) {
                    float t[V];
                    ld_row<V>(last[h], t);
#pragma unroll
                    for (int q = 0; q < V; ++q) part[q] += t[q];
                    lane_emit<V>(p, (int64_t)v[h], part, alive, l1, w[h]);
                }
            }
        }
    }
    // block partial of the L1 norm (fixed order); the last block applies the break test
#pragma unroll
    for (int q = 0; q < V; ++q) {
        float a = l1[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if (lane == 0) s_red[warp][q] = a;
    }
    __syncthreads();
    if (threadIdx.x < V) {
        float a = 0.0f;
#pragma unroll
        for (int w = 0; w < 8; ++w) a += s_red[w][threadIdx.x];
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
    }
}

// nzrp[k] = first nonzero of the k-th nonempty row, nzrp[n_nz] = m (the next
// nonempty row's first nonzero is the end of row k: rows between are empty).
__global__ void lane_bounds_k(const int64_t *rp, const int32_t *nz_rows, int64_t n_nz, int64_t m, int64_t *nzrp)
{
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k <= n_nz; k += (int64_t)gridDim.x * blockDim.x)
        nzrp[k] = k < n_nz ? rp[nz_rows[k]] : m;
}

}  // namespace tpa
