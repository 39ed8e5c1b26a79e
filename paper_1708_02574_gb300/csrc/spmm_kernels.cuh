// Device code of the CPI propagation (Algorithm 1): the SpMV/SpMM kernel
// families, their fixups, the push path of the first family iterates, and
// the merge-path planning kernels.  Included once, by cpi.cu; the host
// dispatch lives there.  Kept apart so that a change of host code leaves
// this file, and the identity of the kernels, untouched.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstddef>

#include "tpa_internal.cuh"

namespace tpa {


constexpr int KP_MAX = 256;
constexpr int CTA = 256;

// Control buffer layout (bytes): Ctl header, int32 alive[KP_MAX], int32 iters[KP_MAX], double norm[KP_MAX]
struct CtlView {
    Ctl *hdr;
    int32_t *alive;   // column still running (its iterate is accumulated)
    int32_t *iters;   // last iteration computed per column
    int32_t *own;     // reserved
    int32_t *pad;
    double *norm;     // last ||x_i||_1 per column
    double *norm1;    // push path: ||x1||_1 per column
};
__host__ __device__ inline CtlView ctl_view(void *base)
{
    CtlView v;
    v.hdr = reinterpret_cast<Ctl *>(base);
    v.alive = reinterpret_cast<int32_t *>(v.hdr + 1);
    v.iters = v.alive + KP_MAX;
    v.own = v.iters + KP_MAX;
    v.pad = v.own + KP_MAX;
    v.norm = reinterpret_cast<double *>(v.pad + KP_MAX);
    v.norm1 = v.norm + KP_MAX;
    return v;
}
constexpr size_t CTL_BYTES = sizeof(Ctl) + 4 * KP_MAX * sizeof(int32_t) + 2 * KP_MAX * sizeof(double);

struct Params {
    // CSR(A~^T)
    const int64_t *rp;
    const int32_t *col;
    const float *val;
    int64_t n;
    // merge-path plan
    const int32_t *tile_x;
    const int64_t *tile_y;
    const int32_t *head_row;
    const int32_t *head_first;
    int64_t tiles;
    // iterates [n][KP]
    const float *x;
    float *y;
    // accumulator and finalize
    float *r;
    int64_t ldr;
    float *out;
    int64_t ldo;
    const float *r_str;
    float one_plus_alpha;
    float decay;
    int k;
    int mode;
    int accumulate;
    int iter;
    double eps;
    // per-tile scratch
    float *carry;    // [tiles][KP]
    float *head;     // [tiles][KP]
    float *tl1;      // [tiles][KP] per-tile L1 partials (FP32; FP64 only across blocks)
    double *part;    // [fix blocks][KP]
    void *ctl;
    // number of [KP] rows of tl1 the SpMM wrote (0 = one per tile); the
    // pipelined kernel writes one per warp of its grid
    int64_t l1_slots;
    // branch gate of a query chunk whose path the device chooses:
    // GATE_NONE runs always, GATE_PULL / GATE_PUSH only on that branch
    int gate;
    // rows binned by length (binned-row kernels): ids of rows with 1..32,
    // 33..512, more than 512 and no nonzeros; the long rows are cut into
    // chunks of 512 nonzeros (chunk i: long row chunk_row[i], first nonzero
    // chunk_e0[i]; long row j owns chunks long_first64[j] .. long_first64[j+1])
    const int32_t *rows_short, *rows_mid, *rows_long, *rows_empty, *chunk_row;
    const int64_t *chunk_e0, *long_first64;
    int64_t n_short, n_mid, n_long, n_empty, n_chunks;
    float *cpart;       // [n_chunks][KP] chunk sums
    int64_t slot0;      // first row of tl1 this launch writes its L1 partials to
    // Pattern-only products over an unweighted CSR(A~^T), whose value at
    // (v, u) is RN32(1/outdeg(u)) for every v: when inv_deg (that value per
    // node u) is set, the value array is not read, x holds x_u * inv_deg[u],
    // and the accumulate epilogue stores y_v * inv_deg[v] as the next x.
    // r, the L1 norms and the outputs keep the unscaled iterate.
    const float *inv_deg;
    // Segmented flag walk (spmm_seg.cuh): the columns of the CSR with bit 31
    // set on the first nonzero of every row, the nonempty rows in order, the
    // number of row starts before each tile of seg_tn nonzeros, and one
    // tagged carry-out word per tile and column.
    const uint32_t *colf;
    const int32_t *nz_rows;
    const int32_t *tile_crow0;
    const int32_t *empty_rows;   // n_empty of them (the field the binned kernels use too)
    int64_t m;
    int64_t seg_tiles;
    unsigned long long *agg;
    // rows of y to clear before the walk (the walk writes nonempty rows only):
    // 0 none, 1 those of the zk seeds zseeds[] that have no in-edge, 2 every
    // empty row
    int zero_mode;
    int zk;
    const int32_t *zseeds;
    // Lane-segment walk (spmm_lane.cuh): the part of every row that ends
    // inside a segment, by the row's rank among the nonempty rows, and the
    // running sum at the end of every segment ([n_nz][KP] and [segments][KP]).
    float *lrec;
    float *ltail;
    const int64_t *nzrp;   // first nonzero of each nonempty row by rank, then m
};

enum Gate : int { GATE_NONE = 0, GATE_PULL = 1, GATE_PUSH = 2 };

// Whether a launch of a gated branch is off for the chunk (Ctl::push is set
// by push_decide_k before the branch kernels run).
__device__ __forceinline__ bool gate_off(int gate, const void *ctl)
{
    if (gate == GATE_NONE) return false;
    const int32_t push = *(volatile const int32_t *)&reinterpret_cast<const Ctl *>(ctl)->push;
    return gate == GATE_PUSH ? push == 0 : push != 0;
}

// ------------------------------------------- tagged carry-out words ---
// A tile publishes its carry-out as 64-bit words that pair the value with a
// launch tag, written and read relaxed: a reader needs no fence, it polls
// (bounded) until the word carries its launch's tag.
constexpr long long SEG_SPIN_LIMIT = 1ll << 22;   // polls of one carry-out word (about a second)

__device__ __forceinline__ void st_relaxed_u64(unsigned long long *p, unsigned long long v)
{
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long seg_pack(float v, uint32_t tag)
{
    return ((unsigned long long)tag << 32) | (unsigned long long)__float_as_uint(v);
}

// Streaming 16-byte load of four column words (read once per launch).
__device__ __forceinline__ uint4 ld_cols4(const uint32_t *p)
{
    uint4 r;
    asm volatile("ld.global.cs.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
                 : "l"(p));
    return r;
}

__device__ __forceinline__ float4 ld_vals4(const float *p)
{
    float4 r;
    asm volatile("ld.global.cs.v4.f32 {%0,%1,%2,%3}, [%4];"
                 : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w)
                 : "l"(p));
    return r;
}

// Wait (bounded) for the carry-out word w of the current launch (tag `want`
// in bits 33.., row-start flag in bit 32); returns the word, or a zero value
// with the error flag raised when the wait gives up.  Once any wait of the
// launch has given up, every other wait returns at once, so a launch ends
// within about one wait limit whatever happens.
__device__ __forceinline__ unsigned long long seg_wait(const unsigned long long *w, uint32_t want, Ctl *hdr)
{
    unsigned long long v = ld_relaxed_u64(w);
    long long spins = 0;
    unsigned ns = 32;
    while ((uint32_t)(v >> 33) != want) {
        if (++spins > SEG_SPIN_LIMIT || *(volatile int32_t *)&hdr->error) {
            atomicOr(&hdr->error, 1);
            return 0ull;
        }
        __nanosleep(ns);
        if (ns < 256) ns <<= 1;
        v = ld_relaxed_u64(w);
    }
    return v;
}


// ------------------------------------------------------------- helpers ---
template <int V>
__device__ __forceinline__ void ld_row(const float *p, float (&o)[V])
{
    if constexpr (V == 1) {
        o[0] = __ldg(p);
    } else if constexpr (V == 2) {
        const float2 t = __ldg(reinterpret_cast<const float2 *>(p));
        o[0] = t.x; o[1] = t.y;
    } else if constexpr (V == 4) {
        const float4 t = __ldg(reinterpret_cast<const float4 *>(p));
        o[0] = t.x; o[1] = t.y; o[2] = t.z; o[3] = t.w;
    } else {
        // 256-bit read-only loads (32-byte aligned: every caller's row is)
        static_assert(V % 8 == 0, "V");
#pragma unroll
        for (int q = 0; q < V / 8; ++q)
            asm("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                : "=f"(o[8 * q]), "=f"(o[8 * q + 1]), "=f"(o[8 * q + 2]), "=f"(o[8 * q + 3]), "=f"(o[8 * q + 4]),
                  "=f"(o[8 * q + 5]), "=f"(o[8 * q + 6]), "=f"(o[8 * q + 7])
                : "l"(p + 8 * q));
    }
}

template <int V>
__device__ __forceinline__ void st_row(float *p, const float (&v)[V])
{
    if constexpr (V == 1) {
        p[0] = v[0];
    } else if constexpr (V == 2) {
        *reinterpret_cast<float2 *>(p) = make_float2(v[0], v[1]);
    } else {
        static_assert(V % 4 == 0, "V");
#pragma unroll
        for (int q = 0; q < V / 4; ++q)
            reinterpret_cast<float4 *>(p)[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
    }
}

template <int V>
__device__ __forceinline__ void ld_row_smem(const float *p, float (&o)[V])
{
    if constexpr (V == 1) {
        o[0] = p[0];
    } else if constexpr (V == 2) {
        const float2 t = *reinterpret_cast<const float2 *>(p);
        o[0] = t.x; o[1] = t.y;
    } else if constexpr (V == 4) {
        const float4 t = *reinterpret_cast<const float4 *>(p);
        o[0] = t.x; o[1] = t.y; o[2] = t.z; o[3] = t.w;
    } else {
        const float4 a = reinterpret_cast<const float4 *>(p)[0];
        const float4 b = reinterpret_cast<const float4 *>(p)[1];
        o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w;
        o[4] = b.x; o[5] = b.y; o[6] = b.z; o[7] = b.w;
    }
}

// Plain (read-write path) vector load of V floats.
template <int V>
__device__ __forceinline__ void ld_row_rw(const float *p, float (&o)[V])
{
    if constexpr (V == 1) {
        o[0] = p[0];
    } else if constexpr (V == 2) {
        const float2 t = *reinterpret_cast<const float2 *>(p);
        o[0] = t.x; o[1] = t.y;
    } else if constexpr (V == 4) {
        const float4 t = *reinterpret_cast<const float4 *>(p);
        o[0] = t.x; o[1] = t.y; o[2] = t.z; o[3] = t.w;
    } else {
        const float4 a = reinterpret_cast<const float4 *>(p)[0];
        const float4 b = reinterpret_cast<const float4 *>(p)[1];
        o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w;
        o[4] = b.x; o[5] = b.y; o[6] = b.z; o[7] = b.w;
    }
}

// Asynchronous global -> shared copies (cp.async, no register staging).
template <int BYTES>
__device__ __forceinline__ void cp_async(void *smem, const void *gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(sa), "l"(gmem), "n"(BYTES));
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::); }

// Copy one row of V floats of the iterate into its swizzled shared-memory slot.
template <int V>
__device__ __forceinline__ void cp_async_row(float *base, int elem, const float *src);

// Product mode of a kernel: read from Params at run time, or fixed when the
// kernel is compiled for one of them (valued: x_u and the value array;
// pattern-only: x_u * inv_deg[u], see Params::inv_deg).
enum ProductMode : int { PM_RUNTIME = 0, PM_VALUED = 1, PM_PATTERN = 2 };

// Store one finished row of the iterate as the next product's x: scaled by
// the row's inverse out-degree in pattern-only mode.
template <int V, int PM = PM_RUNTIME>
__device__ __forceinline__ void st_next_row(const Params &p, int64_t row, float *dst, const float (&y)[V],
                                            float w_row)
{
    const bool pattern = PM == PM_PATTERN || (PM == PM_RUNTIME && p.inv_deg != nullptr);
    if (pattern) {
        // a kernel compiled for pattern-only products passes inv_deg[row] (staged)
        const float w = PM == PM_PATTERN ? w_row : __ldg(p.inv_deg + row);
        float xs[V];
#pragma unroll
        for (int j = 0; j < V; ++j) xs[j] = y[j] * w;
        st_row<V>(dst, xs);
    } else {
        st_row<V>(dst, y);
    }
}

// Epilogue of Algorithm 1 for one finished row and V consecutive columns.
template <int KP, int V, int PM = PM_RUNTIME>
__device__ __forceinline__ void epilogue(const Params &p, int64_t row, int col0, const float (&s)[V],
                                         const int (&alive)[V], float (&l1)[V], float w_row = 0.0f)
{
    float yv[V];
#pragma unroll
    for (int j = 0; j < V; ++j) yv[j] = p.decay * s[j];
    if (p.mode == MODE_ACC) {
        st_next_row<V, PM>(p, row, p.y + row * KP + col0, yv, w_row);
        if (p.accumulate) {
            if (p.ldr == KP && V > 1) {
                // whole padded row contiguous: vector read-modify-write
                float rv[V];
                ld_row_rw<V>(p.r + row * KP + col0, rv);
#pragma unroll
                for (int j = 0; j < V; ++j)
                    if (col0 + j < p.k && alive[j]) rv[j] += yv[j];
                st_row<V>(p.r + row * KP + col0, rv);
            } else {
#pragma unroll
                for (int j = 0; j < V; ++j)
                    if (col0 + j < p.k && alive[j]) p.r[row * p.ldr + col0 + j] += yv[j];
            }
        }
    } else {
        const float rs = p.r_str[row];
        float fam[V], o[V];
        if (p.ldr == KP && V > 1) {
            ld_row_rw<V>(p.r + row * KP + col0, fam);
        } else {
#pragma unroll
            for (int j = 0; j < V; ++j) fam[j] = col0 + j < p.k ? p.r[row * p.ldr + col0 + j] : 0.0f;
        }
#pragma unroll
        for (int j = 0; j < V; ++j) o[j] = fmaf(p.one_plus_alpha, alive[j] ? fam[j] + yv[j] : fam[j], rs);
        float *dst = p.out + row * p.ldo + col0;
        bool vec = false;
        if constexpr (V == 4 || V == 8)   // whole aligned rows go as 16-byte stores (fewer host-link writes)
            vec = col0 + V <= p.k && (reinterpret_cast<uintptr_t>(dst) & 15) == 0;
        if (vec) {
            st_row<V>(dst, o);
        } else {
#pragma unroll
            for (int j = 0; j < V; ++j)
                if (col0 + j < p.k) dst[j] = o[j];
        }
    }
#pragma unroll
    for (int j = 0; j < V; ++j) l1[j] += alive[j] ? fabsf(yv[j]) : 0.0f;
}

// --------------------------------------------------------- main kernel ---
template <int G, int V, int ITEMS, int PF>
struct SpmmSmem {
    static constexpr int NVT = CTA / G;
    static constexpr int L = NVT * ITEMS;
    static constexpr int KP = G * V;
    int32_t end[L + 1];
    int32_t col[L];
    float val[L];
    int32_t crow[NVT];
    float carry[NVT][KP];
    float l1[CTA / 32][KP];
};

template <int G, int V, int ITEMS, int PF>
__global__ void __launch_bounds__(CTA) spmm_tile_k(Params p)
{
    using Sm = SpmmSmem<G, V, ITEMS, PF>;
    constexpr int NVT = Sm::NVT, L = Sm::L, KP = Sm::KP;
    static_assert(ITEMS % PF == 0, "PF");
    static_assert(L <= (1 << 20), "L");
    __shared__ Sm S;

    const CtlView cv = ctl_view(p.ctl);
    if (gate_off(p.gate, p.ctl) || *(volatile int32_t *)&cv.hdr->done) return;

    const int vt = threadIdx.x / G, g = threadIdx.x % G;
    const int col0 = g * V;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int alive[V];
#pragma unroll
    for (int j = 0; j < V; ++j) alive[j] = cv.alive[col0 + j];

    // persistent CTA: static round-robin over tiles (deterministic)
    for (int64_t t = blockIdx.x; t < p.tiles; t += gridDim.x) {
        const int32_t x0 = p.tile_x[t], x1 = p.tile_x[t + 1];
        const int64_t y0 = p.tile_y[t], y1 = p.tile_y[t + 1];
        const int nrows = x1 - x0, nnz = (int)(y1 - y0);
        __syncthreads();   // the previous tile is done with shared memory

        for (int i = threadIdx.x; i < nrows; i += CTA) S.end[i] = (int)(__ldcs(p.rp + x0 + i + 1) - y0);
        if (threadIdx.x == 0) S.end[nrows] = 0x7fffffff;
        for (int i = threadIdx.x; i < nnz; i += CTA) {
            S.col[i] = __ldcs(p.col + y0 + i);
            S.val[i] = p.inv_deg ? 1.0f : __ldcs(p.val + y0 + i);
        }
        __syncthreads();

        // merge-path search for this virtual thread's diagonal
        const int d = min(vt * ITEMS, nrows + nnz);
        int lo = max(0, d - nnz), hi = min(d, nrows);
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (S.end[mid] + mid + 1 <= d) lo = mid + 1; else hi = mid;
        }
        int xs = lo, ys = d - lo;
        const int avail = nrows + nnz - d;

        float acc[V];
        float l1[V];
        float first_val[V];
#pragma unroll
        for (int j = 0; j < V; ++j) {
            acc[j] = 0.0f;
            l1[j] = 0.0f;
            first_val[j] = 0.0f;
        }
        int first_row = -1;

#pragma unroll
        for (int c0 = 0; c0 < ITEMS; c0 += PF) {
            float xv[PF][V];
            float vv[PF];
            unsigned nzmask = 0;
            // pass 1: decide each step and issue the gathers
            {
                int xa = xs, ya = ys;
#pragma unroll
                for (int it = 0; it < PF; ++it) {
                    if (c0 + it < avail) {
                        if (ya < S.end[xa]) {
                            const int c = S.col[ya];
                            vv[it] = S.val[ya];
                            ld_row<V>(p.x + (int64_t)c * KP + col0, xv[it]);
                            nzmask |= 1u << it;
                            ++ya;
                        } else {
                            ++xa;
                        }
                    }
                }
            }
            // pass 2: accumulate and emit
#pragma unroll
            for (int it = 0; it < PF; ++it) {
                if (c0 + it < avail) {
                    if (nzmask & (1u << it)) {
#pragma unroll
                        for (int j = 0; j < V; ++j) acc[j] = fmaf(vv[it], xv[it][j], acc[j]);
                        ++ys;
                    } else {
                        if (first_row < 0) {
                            first_row = xs;
#pragma unroll
                            for (int j = 0; j < V; ++j) first_val[j] = acc[j];
                        } else {
                            epilogue<KP, V>(p, (int64_t)(x0 + xs), col0, acc, alive, l1);
                        }
#pragma unroll
                        for (int j = 0; j < V; ++j) acc[j] = 0.0f;
                        ++xs;
                    }
                }
            }
        }

        // segmented inclusive scan of the virtual threads' carries (key = row)
        if (g == 0) S.crow[vt] = xs;
#pragma unroll
        for (int j = 0; j < V; ++j) S.carry[vt][col0 + j] = acc[j];
        __syncthreads();
#pragma unroll 1
        for (int off = 1; off < NVT; off <<= 1) {
            float add[V];
            const bool take = vt >= off && S.crow[vt - off] == S.crow[vt];
#pragma unroll
            for (int j = 0; j < V; ++j) add[j] = take ? S.carry[vt - off][col0 + j] : 0.0f;
            __syncthreads();
#pragma unroll
            for (int j = 0; j < V; ++j) S.carry[vt][col0 + j] += add[j];
            __syncthreads();
        }

        if (first_row >= 0) {
            float tot[V];
#pragma unroll
            for (int j = 0; j < V; ++j) tot[j] = first_val[j] + (vt > 0 ? S.carry[vt - 1][col0 + j] : 0.0f);
            if (first_row == 0 && p.head_row[t] >= 0) {
                st_row<V>(p.head + t * KP + col0, tot);
            } else {
                epilogue<KP, V>(p, (int64_t)(x0 + first_row), col0, tot, alive, l1);
            }
        }
        if (vt == NVT - 1) {
            float cv2[V];
#pragma unroll
            for (int j = 0; j < V; ++j) cv2[j] = S.carry[vt][col0 + j];
            st_row<V>(p.carry + t * KP + col0, cv2);
        }

        // per-column L1 of this tile, fixed reduction order
#pragma unroll
        for (int j = 0; j < V; ++j) {
            float v = l1[j];
#pragma unroll
            for (int o = G; o < 32; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            l1[j] = v;
        }
        if (lane < G) {
#pragma unroll
            for (int j = 0; j < V; ++j) S.l1[warp][col0 + j] = l1[j];
        }
        __syncthreads();
        for (int c = threadIdx.x; c < KP; c += CTA) {
            float sum = 0.0f;
#pragma unroll
            for (int w = 0; w < CTA / 32; ++w) sum += S.l1[w][c];
            p.tl1[t * KP + c] = sum;
        }
    }
}

// ------------------------------------------------ narrow-batch kernel ---
// Warp-level merge-path SpMV/SpMM for V <= 8 columns per lane (V = 1: one
// vector; V = 2..8: the block of iterates X[n][V] of a small batch stays in
// L2 while the CSR streams once per V seeds).  Every warp owns whole tiles of
// L = 32 * ITEMS path steps and needs no block-wide barrier:
//   1. stage the tile's row ends and the products val * X[col][0..V) of its
//      nonzeros (coalesced, branch-free, ITEMS gathers in flight per lane)
//      into the warp's shared-memory slice;
//   2. each lane walks its ITEMS steps, keeping the current row end in a
//      register, and writes finished row sums to shared memory;
//   3. a shuffle segmented scan adds the carry of earlier lanes to each
//      lane's first row and yields the tile carry;
//   4. the epilogue runs lane-per-row over the tile's rows (coalesced y, r,
//      out); the tile's first row is deferred to the fixup when it started
//      in an earlier tile.
// Shared-memory rows of V floats, stored as chunks of CB bytes (16 for V >= 4,
// else 4V) whose position inside each 128-byte bank row is XOR-swizzled by the
// row number.  Lanes of a merge-path walk read elements about ITEMS apart,
// which without the swizzle lands every lane in the same banks.
template <int V>
struct Swz {
    static constexpr int CB = V >= 4 ? 16 : 4 * V;   // chunk bytes
    static constexpr int CPE = (4 * V) / CB;          // chunks per element (1 or 2)
    static constexpr int R = 128 / CB;                // chunks per 128-byte bank row
    static constexpr int CF = CB / 4;                 // floats per chunk
    __device__ __forceinline__ static int slot(int elem, int h)
    {
        const int c = elem * CPE + h;
        return (c & ~(R - 1)) | ((c ^ (c / R)) & (R - 1));
    }
};

template <int V>
__device__ __forceinline__ void lds_row(const float *base, int elem, float (&o)[V])
{
    using Z = Swz<V>;
#pragma unroll
    for (int h = 0; h < Z::CPE; ++h) {
        const float *p = base + Z::slot(elem, h) * Z::CF;
        if constexpr (Z::CF == 4) {
            const float4 t = *reinterpret_cast<const float4 *>(p);
            o[4 * h] = t.x; o[4 * h + 1] = t.y; o[4 * h + 2] = t.z; o[4 * h + 3] = t.w;
        } else if constexpr (Z::CF == 2) {
            const float2 t = *reinterpret_cast<const float2 *>(p);
            o[0] = t.x; o[1] = t.y;
        } else {
            o[0] = p[0];
        }
    }
}

template <int V>
__device__ __forceinline__ void sts_row(float *base, int elem, const float (&v)[V])
{
    using Z = Swz<V>;
#pragma unroll
    for (int h = 0; h < Z::CPE; ++h) {
        float *p = base + Z::slot(elem, h) * Z::CF;
        if constexpr (Z::CF == 4) {
            *reinterpret_cast<float4 *>(p) = make_float4(v[4 * h], v[4 * h + 1], v[4 * h + 2], v[4 * h + 3]);
        } else if constexpr (Z::CF == 2) {
            *reinterpret_cast<float2 *>(p) = make_float2(v[0], v[1]);
        } else {
            p[0] = v[0];
        }
    }
}

template <int V>
__device__ __forceinline__ void cp_async_row(float *base, int elem, const float *src)
{
    using Z = Swz<V>;
#pragma unroll
    for (int h = 0; h < Z::CPE; ++h) cp_async<Z::CB>(base + Z::slot(elem, h) * Z::CF, src + h * Z::CF);
}

// Vector arrays first: every row of prod/rowsum starts on a V*4-byte boundary
// (float2/float4 shared-memory accesses), and the slice size is a multiple of
// 16 bytes so every warp's slice starts aligned too.
template <int V, int ITEMS>
struct __align__(16) WarpTile {
    static constexpr int L = 32 * ITEMS;
    // V <= 2: prod holds the products val * X[col]; V >= 4: prod holds the
    // gathered rows X[col] (copied by cp.async) and val the A~ values
    static constexpr bool ASYNC = V >= 4;
    float prod[L * V];               // swizzled (see Swz)
    float rowsum[L * V];             // finished row sums, swizzled
    float val[ASYNC ? L : 4];        // swizzled as V = 1 rows
    int32_t end[L + 4];
};

template <int V, int ITEMS, int WARPS>
__global__ void __launch_bounds__(WARPS * 32, (V == 1 ? 1536 : V == 2 ? 1280 : V == 4 ? 1024 : 768) / (WARPS * 32))
spmvw_tile_k(Params p)
{
    using WT = WarpTile<V, ITEMS>;
    static_assert(offsetof(WT, prod) % 16 == 0 && offsetof(WT, rowsum) % 16 == 0, "vector rows must be aligned");
    static_assert((V * sizeof(float)) % (V == 1 ? 4 : V == 2 ? 8 : 16) == 0, "row width");
    static_assert(sizeof(WT) % 16 == 0, "warp slices must stay 16-byte aligned");
    static_assert(sizeof(WT) * WARPS <= 48 * 1024, "static shared memory is limited to 48 KB per block");
    __shared__ WT S_all[WARPS];
    const CtlView cv = ctl_view(p.ctl);
    if (gate_off(p.gate, p.ctl) || *(volatile int32_t *)&cv.hdr->done) return;
    int alive[V];
#pragma unroll
    for (int j = 0; j < V; ++j) alive[j] = cv.alive[j];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    WT &S = S_all[warp];

    for (int64_t t = (int64_t)blockIdx.x * WARPS + warp; t < p.tiles; t += (int64_t)gridDim.x * WARPS) {
        const int32_t x0 = p.tile_x[t], x1 = p.tile_x[t + 1];
        const int64_t y0 = p.tile_y[t], y1 = p.tile_y[t + 1];
        const int nrows = x1 - x0, nnz = (int)(y1 - y0);
        const bool defer_first = p.head_row[t] >= 0;
        __syncwarp();   // the previous tile is done with this warp's slice

        // 1. row ends and products
        for (int i = lane; i < nrows; i += 32) S.end[i] = (int)(__ldcs(p.rp + x0 + i + 1) - y0);
        if (lane == 0) S.end[nrows] = 0x7fffffff;
        {
            int32_t c[ITEMS];
            float v[ITEMS];
#pragma unroll
            for (int j = 0; j < ITEMS; ++j) {
                const int i = lane + j * 32;
                c[j] = i < nnz ? __ldcs(p.col + y0 + i) : 0;
                v[j] = i < nnz ? (p.inv_deg ? 1.0f : __ldcs(p.val + y0 + i)) : 0.0f;
            }
            if constexpr (WT::ASYNC) {
                // wide rows: gathers go straight to shared memory, all in flight at once
#pragma unroll
                for (int j = 0; j < ITEMS; ++j)
                    if (lane + j * 32 < nnz) cp_async_row<V>(S.prod, lane + j * 32, p.x + (int64_t)c[j] * V);
#pragma unroll
                for (int j = 0; j < ITEMS; ++j)
                    if (lane + j * 32 < nnz) S.val[Swz<1>::slot(lane + j * 32, 0)] = v[j];
                cp_async_wait_all();
            } else {
                // narrow rows: gather into registers, stage the products
                float xv[ITEMS][V];
#pragma unroll
                for (int j = 0; j < ITEMS; ++j) {
                    if (lane + j * 32 < nnz) {
                        ld_row<V>(p.x + (int64_t)c[j] * V, xv[j]);
                    } else {
#pragma unroll
                        for (int q = 0; q < V; ++q) xv[j][q] = 0.0f;
                    }
                }
#pragma unroll
                for (int j = 0; j < ITEMS; ++j)
                    if (lane + j * 32 < nnz) {
                        float pr[V];
#pragma unroll
                        for (int q = 0; q < V; ++q) pr[q] = v[j] * xv[j][q];
                        sts_row<V>(S.prod, lane + j * 32, pr);
                    }
            }
        }
        __syncwarp();

        // 2. merge-path walk in shared memory
        const int d = min(lane * ITEMS, nrows + nnz);
        int lo = max(0, d - nnz), hi = min(d, nrows);
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (S.end[mid] + mid + 1 <= d) lo = mid + 1; else hi = mid;
        }
        int xs = lo, ys = d - lo;
        const int avail = nrows + nnz - d;
        int row_end = S.end[xs];
        float acc[V];
#pragma unroll
        for (int q = 0; q < V; ++q) acc[q] = 0.0f;
        int first = -1;
#pragma unroll
        for (int it = 0; it < ITEMS; ++it) {
            if (it < avail) {
                if (ys < row_end) {
                    float xr[V];
                    lds_row<V>(S.prod, ys, xr);
                    if constexpr (WT::ASYNC) {
                        const float vv = S.val[Swz<1>::slot(ys, 0)];
#pragma unroll
                        for (int q = 0; q < V; ++q) acc[q] = fmaf(vv, xr[q], acc[q]);
                    } else {
#pragma unroll
                        for (int q = 0; q < V; ++q) acc[q] += xr[q];
                    }
                    ++ys;
                } else {
                    sts_row<V>(S.rowsum, xs, acc);
                    if (first < 0) first = xs;
#pragma unroll
                    for (int q = 0; q < V; ++q) acc[q] = 0.0f;
                    ++xs;
                    row_end = S.end[xs];
                }
            }
        }

        // 3. segmented inclusive scan of (row, partial) over the lanes
        const int key = xs;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int k2 = __shfl_up_sync(0xffffffffu, key, off);
            const bool take = lane >= off && k2 == key;
#pragma unroll
            for (int q = 0; q < V; ++q) {
                const float v2 = __shfl_up_sync(0xffffffffu, acc[q], off);
                if (take) acc[q] += v2;
            }
        }
        float prev[V];
#pragma unroll
        for (int q = 0; q < V; ++q) prev[q] = __shfl_up_sync(0xffffffffu, acc[q], 1);
        __syncwarp();   // rowsum writes of the walk are visible
        if (first >= 0 && lane > 0) {
            float cur[V];
            lds_row<V>(S.rowsum, first, cur);
#pragma unroll
            for (int q = 0; q < V; ++q) cur[q] += prev[q];
            sts_row<V>(S.rowsum, first, cur);
        }
        if (lane == 31) st_row<V>(p.carry + t * V, acc);
        __syncwarp();

        // 4. coalesced epilogue, lane per row
        float l1[V];
#pragma unroll
        for (int q = 0; q < V; ++q) l1[q] = 0.0f;
        for (int i = lane; i < nrows; i += 32) {
            float sum[V];
            lds_row<V>(S.rowsum, i, sum);
            if (i == 0 && defer_first) {
                st_row<V>(p.head + t * V, sum);
                continue;
            }
            epilogue<V, V>(p, (int64_t)(x0 + i), 0, sum, alive, l1);
        }
#pragma unroll
        for (int q = 0; q < V; ++q) {
            float a = l1[q];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
            l1[q] = a;
        }
        if (lane == 0) {
#pragma unroll
            for (int q = 0; q < V; ++q) p.tl1[t * V + q] = l1[q];
        }
    }
}

// --------------------------------------------------- group-walker kernel ---
// Warp-level merge path where each walker is a group of G lanes and each lane
// owns V consecutive columns of a batch of KP = G*V seeds: for a nonzero the
// group gathers one contiguous row X[col][0..KP) (G*V*4 bytes, one or a few
// sectors), so a gathered byte is a useful byte.  Only the tile's row ends,
// columns and values are staged in shared memory (coalesced), which keeps
// tiles long and occupancy high.  Per warp tile of L = (32/G) * ITEMS steps:
//   1. stage row ends, col, val;
//   2. each walker finds its diagonal, then walks ITEMS steps in chunks of
//      PF: first it decides the steps and issues the PF gathers, then it
//      accumulates and emits finished rows (epilogue fused, coalesced within
//      the group);
//   3. a shuffle segmented scan over the walkers resolves carries; the
//      tile's first row is deferred to the fixup when it started earlier.
template <int G, int V, int ITEMS>
struct GroupTile {
    static constexpr int NW = 32 / G;
    static constexpr int L = NW * ITEMS;
    int32_t col[L];
    float val[L];
    int32_t end[L + 4];
};

template <int G, int V, int ITEMS, int PF, int WARPS>
__global__ void __launch_bounds__(WARPS * 32) spmvg_tile_k(Params p)
{
    using GT = GroupTile<G, V, ITEMS>;
    constexpr int NW = GT::NW, KP = G * V;
    static_assert(ITEMS % PF == 0, "PF");
    static_assert(sizeof(GT) * WARPS <= 48 * 1024, "static shared memory is limited to 48 KB per block");
    __shared__ GT S_all[WARPS];
    const CtlView cv = ctl_view(p.ctl);
    if (gate_off(p.gate, p.ctl) || *(volatile int32_t *)&cv.hdr->done) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int w = lane / G, gl = lane % G, col0 = gl * V;
    int alive[V];
#pragma unroll
    for (int j = 0; j < V; ++j) alive[j] = cv.alive[col0 + j];
    GT &S = S_all[warp];

    for (int64_t t = (int64_t)blockIdx.x * WARPS + warp; t < p.tiles; t += (int64_t)gridDim.x * WARPS) {
        const int32_t x0 = p.tile_x[t], x1 = p.tile_x[t + 1];
        const int64_t y0 = p.tile_y[t], y1 = p.tile_y[t + 1];
        const int nrows = x1 - x0, nnz = (int)(y1 - y0);
        const bool defer_first = p.head_row[t] >= 0;
        __syncwarp();
        for (int i = lane; i < nrows; i += 32) S.end[i] = (int)(__ldcs(p.rp + x0 + i + 1) - y0);
        if (lane == 0) S.end[nrows] = 0x7fffffff;
        for (int i = lane; i < nnz; i += 32) {
            S.col[i] = __ldcs(p.col + y0 + i);
            S.val[i] = p.inv_deg ? 1.0f : __ldcs(p.val + y0 + i);
        }
        __syncwarp();

        const int d = min(w * ITEMS, nrows + nnz);
        int lo = max(0, d - nnz), hi = min(d, nrows);
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (S.end[mid] + mid + 1 <= d) lo = mid + 1; else hi = mid;
        }
        int xs = lo, ys = d - lo;
        const int avail = nrows + nnz - d;
        float acc[V], first_val[V];
        float l1[V];
#pragma unroll
        for (int j = 0; j < V; ++j) {
            acc[j] = 0.0f;
            first_val[j] = 0.0f;
            l1[j] = 0.0f;
        }
        int first_row = -1;
#pragma unroll
        for (int c0 = 0; c0 < ITEMS; c0 += PF) {
            float xv[PF][V];
            float vv[PF];
            unsigned nzmask = 0;
            {
                int xa = xs, ya = ys;
#pragma unroll
                for (int it = 0; it < PF; ++it) {
                    if (c0 + it < avail) {
                        if (ya < S.end[xa]) {
                            vv[it] = S.val[ya];
                            ld_row<V>(p.x + (int64_t)S.col[ya] * KP + col0, xv[it]);
                            nzmask |= 1u << it;
                            ++ya;
                        } else {
                            ++xa;
                        }
                    }
                }
            }
#pragma unroll
            for (int it = 0; it < PF; ++it) {
                if (c0 + it < avail) {
                    if (nzmask & (1u << it)) {
#pragma unroll
                        for (int j = 0; j < V; ++j) acc[j] = fmaf(vv[it], xv[it][j], acc[j]);
                        ++ys;
                    } else {
                        if (first_row < 0) {
                            first_row = xs;
#pragma unroll
                            for (int j = 0; j < V; ++j) first_val[j] = acc[j];
                        } else {
                            epilogue<KP, V>(p, (int64_t)(x0 + xs), col0, acc, alive, l1);
                        }
#pragma unroll
                        for (int j = 0; j < V; ++j) acc[j] = 0.0f;
                        ++xs;
                    }
                }
            }
        }

        // segmented inclusive scan of the walkers' carries (key = row)
        const int key = xs;
#pragma unroll
        for (int off = 1; off < NW; off <<= 1) {
            const int k2 = __shfl_up_sync(0xffffffffu, key, off * G);
            const bool take = w >= off && k2 == key;
#pragma unroll
            for (int j = 0; j < V; ++j) {
                const float v2 = __shfl_up_sync(0xffffffffu, acc[j], off * G);
                if (take) acc[j] += v2;
            }
        }
        float prev[V];
#pragma unroll
        for (int j = 0; j < V; ++j) prev[j] = __shfl_up_sync(0xffffffffu, acc[j], G);
        if (first_row >= 0) {
            float tot[V];
#pragma unroll
            for (int j = 0; j < V; ++j) tot[j] = first_val[j] + (w > 0 ? prev[j] : 0.0f);
            if (first_row == 0 && defer_first) {
                st_row<V>(p.head + t * KP + col0, tot);
            } else {
                epilogue<KP, V>(p, (int64_t)(x0 + first_row), col0, tot, alive, l1);
            }
        }
        if (w == NW - 1) st_row<V>(p.carry + t * KP + col0, acc);
#pragma unroll
        for (int j = 0; j < V; ++j) {
            float a = l1[j];
#pragma unroll
            for (int o = G; o < 32; o <<= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
            l1[j] = a;
        }
        if (lane < G) {
#pragma unroll
            for (int j = 0; j < V; ++j) p.tl1[t * KP + col0 + j] = l1[j];
        }
    }
}

// ------------------------------------------ pipelined group-walker kernel ---
// The group walker above, reorganised so that no walker waits on memory other
// than its own prefetched gathers:
//  - a warp's next tile (row ends, columns, values) is staged into the second
//    of two shared-memory buffers while the walkers work on the current tile;
//    columns and values of the tile after that are already in registers and
//    its bounds are loading, so a tile's own loads are never on its critical
//    path (see stage_tile);
//  - walkers park the sums of finished rows in shared memory; after the walk
//    one coalesced pass over the tile's rows (consecutive rows on consecutive
//    walkers) runs the epilogue.  In accumulate mode it reads nothing: y is
//    stored and r gets y by a vector atomic add; each element of r receives
//    exactly one add per launch, so the sum equals the read-modify-write and
//    is deterministic.  The final family iteration reads r and r~_str for all
//    the tile's rows at once and writes the TPA scores;
//  - the L1 partial of the break test is accumulated per lane over all of a
//    warp's tiles and reduced once per warp (one row of tl1 per warp).
// The first row of a tile, when it started in an earlier tile, is still
// finished by the fixup.
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait_group() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// r[0..V) += v[0..V) with vector atomics (the result is not read back).
template <int V>
__device__ __forceinline__ void red_row(float *p, const float (&v)[V])
{
    if constexpr (V == 1) {
        atomicAdd(p, v[0]);
    } else if constexpr (V == 2) {
        atomicAdd(reinterpret_cast<float2 *>(p), make_float2(v[0], v[1]));
    } else if constexpr (V == 4) {
        atomicAdd(reinterpret_cast<float4 *>(p), make_float4(v[0], v[1], v[2], v[3]));
    } else {
        static_assert(V == 8, "V");
        atomicAdd(reinterpret_cast<float4 *>(p), make_float4(v[0], v[1], v[2], v[3]));
        atomicAdd(reinterpret_cast<float4 *>(p) + 1, make_float4(v[4], v[5], v[6], v[7]));
    }
}

// Epilogue of Algorithm 1 for one finished row in accumulate mode without
// loads: y stored, r += y by a vector atomic add.
template <int KP, int V, int PM = PM_RUNTIME>
__device__ __forceinline__ void epilogue_red(const Params &p, int64_t row, int col0, const float (&s)[V],
                                             const int (&alive)[V], float (&l1)[V], float w_row = 0.0f)
{
    float yv[V];
#pragma unroll
    for (int j = 0; j < V; ++j) yv[j] = p.decay * s[j];
    if (p.mode == MODE_ACC) {
        st_next_row<V, PM>(p, row, p.y + row * KP + col0, yv, w_row);
        if (p.accumulate) {
            if (p.ldr == KP) {
                float add[V];
#pragma unroll
                for (int j = 0; j < V; ++j) add[j] = (col0 + j < p.k && alive[j]) ? yv[j] : 0.0f;
                red_row<V>(p.r + row * KP + col0, add);
            } else {
#pragma unroll
                for (int j = 0; j < V; ++j)
                    if (col0 + j < p.k && alive[j]) atomicAdd(p.r + row * p.ldr + col0 + j, yv[j]);
            }
        }
    }
#pragma unroll
    for (int j = 0; j < V; ++j) l1[j] += alive[j] ? fabsf(yv[j]) : 0.0f;
}

// Sum over b in [0, nb) of part[b * KP + c] for every column c < KP, by the
// NT threads of one block in a fixed order (so the result is deterministic):
// group grp of the NG = NT / KP groups adds b = grp, grp + NG, ... in increasing b
// (loads issued eight at a time), then thread c adds the group sums in group
// order.  The result for column c is left in s_fin[c] (s_fin holds 256).
template <int KP, class T, int NT = 256>
__device__ __forceinline__ void block_sum_partials_t(const T *part, unsigned nb, double *s_fin)
{
    static_assert(KP >= 1 && KP <= NT && NT % KP == 0 && NT <= 256, "KP");
    constexpr unsigned NG = NT / KP;
    const int c = threadIdx.x % KP, grp = threadIdx.x / KP;
    double a = 0.0;
    unsigned b = grp;
    for (; b + 7u * NG < nb; b += 8u * NG) {
        double v[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) v[i] = __ldcg(&part[(int64_t)(b + i * NG) * KP + c]);
#pragma unroll
        for (int i = 0; i < 8; ++i) a += v[i];
    }
    for (; b < nb; b += NG) a += __ldcg(&part[(int64_t)b * KP + c]);
    __syncthreads();
    s_fin[grp * KP + c] = a;
    __syncthreads();
    if (threadIdx.x < KP) {
        double t = 0.0;
        for (unsigned g = 0; g < NG; ++g) t += s_fin[g * KP + threadIdx.x];
        s_fin[threadIdx.x] = t;   // only this thread reads or writes column c's group-0 slot
    }
    __syncthreads();
}

template <int KP>
__device__ __forceinline__ void block_sum_partials(const double *part, unsigned nb, double *s_fin)
{
    block_sum_partials_t<KP, double>(part, nb, s_fin);
}

template <int G, int V, int ITEMS, bool PAT>
struct __align__(16) PipeTile {
    static constexpr int NW = 32 / G;
    static constexpr int L = NW * ITEMS;
    static constexpr int CH = (L + 6) / 4 + 1;      // 4-nonzero chunks a tile's nonzeros can span
    static constexpr int PCH = (2 * CH + 7) & ~7;   // 16-byte pair chunks, whole swizzle groups
    static constexpr int CCH = (CH + 7) & ~7;       // 16-byte column chunks (pattern-only)
    int64_t rp[L + 2];   // row_ptr[x0+1 .. x1], then a sentinel y0 + INT_MAX
    // Valued products: (column, value bits) of nonzeros y0a .. y0a + 4 * chunks,
    // y0a = y0 rounded down to a multiple of 4; nonzero e of the slice is the
    // pair at word pair_word(e): one 8-byte shared load per step.
    // Pattern-only products: the columns alone, nonzero e at col_word(e).
    int32_t cv[PAT ? 4 * CCH : 4 * PCH];
    // pattern-only: inv_deg of the tile's rows x0 .. x1-1
    float inv[PAT ? ((L + 3) & ~3) : 4];
};

// Slot of 16-byte chunk q: an XOR swizzle inside each group of 8 chunks (one
// 128-byte bank row), so walkers a few chunks apart share banks less often.
__device__ __forceinline__ int chunk_slot(int q) { return (q & ~7) | ((q ^ (q >> 3)) & 7); }
// First word of the (column, value) pair of nonzero e (two pairs per chunk).
__device__ __forceinline__ int pair_word(int e) { return 4 * chunk_slot(e >> 1) + 2 * (e & 1); }
// Word of the column of nonzero e when only columns are staged (four per chunk).
__device__ __forceinline__ int col_word(int e) { return 4 * chunk_slot(e >> 2) + (e & 3); }

struct TileMeta {
    int64_t y0, y1;
    int32_t x0, x1;
    int defer;           // the tile's first row started in an earlier tile
};

__device__ __forceinline__ TileMeta tile_meta(const Params &p, int64_t t)
{
    TileMeta m;
    if (t < p.tiles) {
        m.x0 = __ldg(p.tile_x + t);
        m.x1 = __ldg(p.tile_x + t + 1);
        m.y0 = __ldg(p.tile_y + t);
        m.y1 = __ldg(p.tile_y + t + 1);
        m.defer = __ldg(p.head_row + t) >= 0;
    } else {
        m.x0 = m.x1 = 0;
        m.y0 = m.y1 = 0;
        m.defer = 0;
    }
    return m;
}

// 16-byte global -> shared copy that bypasses L1 (the CSR is streamed once).
__device__ __forceinline__ void cp_async16_cg(void *smem, const void *gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem));
}

// A tile's CSR slice is staged in two parts.  The row ends (a few per tile)
// go by 8-byte cp.async.  Columns and values (8 bytes per nonzero, the bulk)
// are loaded with coalesced 16-byte loads into registers one tile ahead and
// stored to shared memory just before that tile is walked: a cp.async costs an
// L1 wavefront per 32-byte sector on each side, a coalesced load one per
// 128-byte line.  Chunks beyond 32 * RC (at most a few per tile) go by cp.async.
// Columns and values run from y0 rounded down to a multiple of 4 up to y1
// rounded up: at most 3 elements past m, inside the CSR padding.
__device__ __forceinline__ int tile_chunks(const TileMeta &m)
{
    return m.y1 > m.y0 ? (int)((m.y1 - (m.y0 & ~(int64_t)3) + 3) >> 2) : 0;
}

template <int RC>
struct ChunkRegs {
    int4 c[RC > 0 ? RC : 1];
    float4 v[RC > 0 ? RC : 1];
};

template <int RC, bool PAT>
__device__ __forceinline__ void load_chunks(const Params &p, const TileMeta &m, ChunkRegs<RC> &r, int lane)
{
    const int chunks = tile_chunks(m);
    const int64_t y0a = m.y0 & ~(int64_t)3;
#pragma unroll
    for (int k = 0; k < RC; ++k) {
        const int q = lane + 32 * k;
        if (q < chunks) {
            r.c[k] = __ldcs(reinterpret_cast<const int4 *>(p.col + y0a) + q);
            if constexpr (!PAT) r.v[k] = __ldcs(reinterpret_cast<const float4 *>(p.val + y0a) + q);
        }
    }
}

// Store the register chunks of tile m interleaved as (column, value) pairs,
// and issue the cp.async copies of its row ends and of the elements of chunks
// past 32 * RC (a few per tile at most; the caller commits).
template <int RC, bool PAT>
__device__ __forceinline__ void stage_tile(const Params &p, const TileMeta &m, const ChunkRegs<RC> &r,
                                           int64_t *rp_s, int32_t *cv_s, float *inv_s, int lane)
{
    const int chunks = tile_chunks(m);
    const int64_t y0a = m.y0 & ~(int64_t)3;
#pragma unroll
    for (int k = 0; k < RC; ++k) {
        const int q = lane + 32 * k;
        if (q < chunks) {
            const int4 c = r.c[k];
            if constexpr (PAT) {
                *reinterpret_cast<int4 *>(cv_s + 4 * chunk_slot(q)) = c;
            } else {
                const float4 v = r.v[k];
                *reinterpret_cast<int4 *>(cv_s + 4 * chunk_slot(2 * q)) =
                    make_int4(c.x, __float_as_int(v.x), c.y, __float_as_int(v.y));
                *reinterpret_cast<int4 *>(cv_s + 4 * chunk_slot(2 * q + 1)) =
                    make_int4(c.z, __float_as_int(v.z), c.w, __float_as_int(v.w));
            }
        }
    }
    for (int e = 128 * RC + lane; e < 4 * chunks; e += 32) {
        if constexpr (PAT) {
            cp_async<4>(cv_s + col_word(e), p.col + y0a + e);
        } else {
            cp_async<4>(cv_s + pair_word(e), p.col + y0a + e);
            cp_async<4>(cv_s + pair_word(e) + 1, p.val + y0a + e);
        }
    }
    const int nrows = m.x1 - m.x0;
    for (int i = lane; i < nrows; i += 32) cp_async<8>(rp_s + i, p.rp + m.x0 + i + 1);
    if constexpr (PAT)
        for (int i = lane; i < nrows; i += 32) cp_async<4>(inv_s + i, p.inv_deg + m.x0 + i);
    if (lane == 0) rp_s[nrows] = m.y0 + 0x7fffffff;
}

// FUSE: the carry-out goes to the tagged words p.agg instead of p.carry.
template <int G, int V, int ITEMS, int PF, bool PAT, bool FUSE = false>
__device__ __forceinline__ void walk_tile(const Params &p, const TileMeta &m, int64_t t, const int64_t *rp_s,
                                          const int32_t *cv_s, const float *inv_s, float *rs_s, int lane,
                                          const int (&alive)[V], float (&l1)[V], uint32_t tag = 0)
{
    constexpr int NW = 32 / G, KP = G * V;
    const int w = lane / G, col0 = (lane % G) * V;
    const int nrows = m.x1 - m.x0, nnz = (int)(m.y1 - m.y0);
    const int off = (int)(m.y0 & 3);   // position of nonzero y0 in the staged chunks
    // this walker's diagonal on the tile's merge path
    const int d = min(w * ITEMS, nrows + nnz);
    int lo = max(0, d - nnz), hi = min(d, nrows);
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if ((int)(rp_s[mid] - m.y0) + mid + 1 <= d) lo = mid + 1; else hi = mid;
    }
    int xs = lo, ys = d - lo;
    int row_end = (int)(rp_s[xs] - m.y0);
    const int avail = nrows + nnz - d;
    float acc[V], first_val[V];
#pragma unroll
    for (int j = 0; j < V; ++j) {
        acc[j] = 0.0f;
        first_val[j] = 0.0f;
    }
    int first_row = -1;
#pragma unroll
    for (int c0 = 0; c0 < ITEMS; c0 += PF) {
        // decide PF steps and issue their gathers
        float xv[PF][V];
        float vv[PF];
        unsigned nzmask = 0;
        int xa = xs;
#pragma unroll
        for (int it = 0; it < PF; ++it) {
            if (c0 + it < avail) {
                if (ys < row_end) {
                    if constexpr (PAT) {   // every value is folded into x
                        vv[it] = 1.0f;
                        ld_row<V>(p.x + (int64_t)cv_s[col_word(off + ys)] * KP + col0, xv[it]);
                    } else {
                        const int2 e = *reinterpret_cast<const int2 *>(cv_s + pair_word(off + ys));
                        vv[it] = __int_as_float(e.y);
                        ld_row<V>(p.x + (int64_t)e.x * KP + col0, xv[it]);
                    }
                    nzmask |= 1u << it;
                    ++ys;
                } else {
                    ++xa;
                    row_end = (int)(rp_s[xa] - m.y0);
                }
            }
        }
        // accumulate, emit finished rows
#pragma unroll
        for (int it = 0; it < PF; ++it) {
            if (c0 + it < avail) {
                if (nzmask & (1u << it)) {
#pragma unroll
                    for (int j = 0; j < V; ++j) acc[j] = fmaf(vv[it], xv[it][j], acc[j]);
                } else {
                    if (first_row < 0) {
                        first_row = xs;
#pragma unroll
                        for (int j = 0; j < V; ++j) first_val[j] = acc[j];
                    } else {
                        st_row<V>(rs_s + xs * KP + col0, acc);   // finished: epilogue after the walk
                    }
#pragma unroll
                    for (int j = 0; j < V; ++j) acc[j] = 0.0f;
                    ++xs;
                }
            }
        }
    }

    // segmented inclusive scan of the walkers' trailing partials (key = row)
    const int key = xs;
#pragma unroll
    for (int off = 1; off < NW; off <<= 1) {
        const int k2 = __shfl_up_sync(0xffffffffu, key, off * G);
        const bool take = w >= off && k2 == key;
#pragma unroll
        for (int j = 0; j < V; ++j) {
            const float v2 = __shfl_up_sync(0xffffffffu, acc[j], off * G);
            if (take) acc[j] += v2;
        }
    }
    float prev[V];
#pragma unroll
    for (int j = 0; j < V; ++j) prev[j] = __shfl_up_sync(0xffffffffu, acc[j], G);
    if (first_row >= 0) {
        float tot[V];
#pragma unroll
        for (int j = 0; j < V; ++j) tot[j] = first_val[j] + (w > 0 ? prev[j] : 0.0f);
        if (first_row == 0 && m.defer)
            st_row<V>(p.head + t * KP + col0, tot);
        else
            st_row<V>(rs_s + first_row * KP + col0, tot);
    }
    if (w == NW - 1) {
        if constexpr (FUSE) {
#pragma unroll
            for (int j = 0; j < V; ++j) st_relaxed_u64(p.agg + t * KP + col0 + j, seg_pack(acc[j], tag));
        } else {
            st_row<V>(p.carry + t * KP + col0, acc);
        }
    }
    __syncwarp();
    // epilogue of the tile's finished rows, consecutive rows on consecutive
    // walkers (coalesced): accumulate by atomics (no load), the final family
    // iteration reads r and r~_str for all rows of the tile at once
    for (int r = w; r < nrows; r += NW) {
        if (r == 0 && m.defer) continue;   // finished by the fixup
        float sv[V];
        ld_row_smem<V>(rs_s + r * KP + col0, sv);
        if (p.mode == MODE_ACC)
            epilogue_red<KP, V, PAT ? PM_PATTERN : PM_VALUED>(p, (int64_t)(m.x0 + r), col0, sv, alive, l1,
                                                              PAT ? inv_s[r] : 0.0f);
        else
            epilogue<KP, V, PAT ? PM_PATTERN : PM_VALUED>(p, (int64_t)(m.x0 + r), col0, sv, alive, l1);
    }
}

// Shared memory per warp: two tile buffers and the row sums of one tile.
template <int G, int V, int ITEMS, bool PAT>
struct PipeSmem {
    using PT = PipeTile<G, V, ITEMS, PAT>;
    static constexpr size_t RS = (size_t)PT::L * G * V * sizeof(float);
    static constexpr size_t PER_WARP = 2 * sizeof(PT) + RS;
};

// The deferred rows of one warp's tiles, finished after its last tile (the
// fixup's work, inside the SpMM): lane l takes the warp's tiles l, l+32, ...
// in turn; a row whose part began at most TAIL_SHORT tiles back is summed by
// its lane (head part, then the carry-outs of the tiles it spans, in tile
// order), a longer one (a hub's) by the whole warp in a fixed lane-strided
// order.  Carry-outs are read from the tagged words (bounded waits; by now
// nearly all of them are published).  The same sums in the same order as
// fixup_small_k, so rows come out bit-identical to the launch with a fixup.
constexpr int TAIL_SHORT = 32;

// Add the KP carry-out words of tile u to acc: the loads first (all in
// flight together), then the tag checks; a word of an earlier launch is
// waited for (bounded).
template <int KP>
__device__ __forceinline__ void add_tagged_row(const Params &p, int64_t u, uint32_t ep, Ctl *hdr, float (&acc)[KP])
{
    unsigned long long w[KP];
#pragma unroll
    for (int c = 0; c < KP; ++c) w[c] = ld_relaxed_u64(p.agg + u * KP + c);
#pragma unroll
    for (int c = 0; c < KP; ++c) {
        if ((uint32_t)(w[c] >> 33) != ep) w[c] = seg_wait(p.agg + u * KP + c, ep, hdr);
        acc[c] += __uint_as_float((uint32_t)w[c]);
    }
}

template <int KP>
__device__ __forceinline__ void pipe_tail(const Params &p, int64_t t0, int64_t stride, uint32_t ep, const CtlView &cv,
                                          int lane, float (&l1)[KP])
{
    int alive[KP];
#pragma unroll
    for (int c = 0; c < KP; ++c) alive[c] = cv.alive[c];
    const int64_t mine = t0 < p.tiles ? (p.tiles - 1 - t0) / stride + 1 : 0;
    for (int64_t j0 = 0; j0 < mine; j0 += 32) {
        const int64_t j = j0 + lane;
        const int64_t t = t0 + j * stride;
        int32_t h = -1;
        int64_t first = 0;
        if (j < mine) {
            h = __ldg(p.head_row + t);
            if (h >= 0) first = __ldg(p.head_first + t);
        }
        const bool longspan = h >= 0 && t - first > TAIL_SHORT;
        if (h >= 0 && !longspan) {
            float sum[KP];
            ld_row_rw<KP>(p.head + t * KP, sum);
            for (int64_t u = first; u < t; ++u) add_tagged_row<KP>(p, u, ep, cv.hdr, sum);
            epilogue<KP, KP>(p, (int64_t)h, 0, sum, alive, l1);
        }
        unsigned lm = __ballot_sync(0xffffffffu, longspan);
        while (lm) {
            const int src = __ffs(lm) - 1;
            lm &= lm - 1;
            const int64_t tt = __shfl_sync(0xffffffffu, t, src);
            const int64_t ff = __shfl_sync(0xffffffffu, first, src);
            float part[KP];
#pragma unroll
            for (int c = 0; c < KP; ++c) part[c] = 0.0f;
            for (int64_t u = ff + lane; u < tt; u += 32) add_tagged_row<KP>(p, u, ep, cv.hdr, part);
#pragma unroll
            for (int c = 0; c < KP; ++c) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) part[c] += __shfl_xor_sync(0xffffffffu, part[c], o);
            }
            if (lane == src) {
                float sum[KP];
                ld_row_rw<KP>(p.head + tt * KP, sum);
#pragma unroll
                for (int c = 0; c < KP; ++c) sum[c] += part[c];
                epilogue<KP, KP>(p, (int64_t)h, 0, sum, alive, l1);
            }
        }
    }
}

// MINB: resident blocks per SM requested from the register allocator.
// FUSE: no fixup launch.  Tiles publish their carry-outs as tagged words;
// after its last tile each warp finishes the rows its tiles deferred
// (pipe_tail), and the last CTA to finish reduces the L1 partials and
// applies the break test.  The waits need every CTA resident: the grid is
// launched cooperatively.
template <int G, int V, int ITEMS, int PF, int WARPS, int MINB, bool PAT, bool FUSE = false>
__global__ void __launch_bounds__(WARPS * 32, MINB) spmvp_tile_k(Params p)
{
    using PT = PipeTile<G, V, ITEMS, PAT>;
    using SM = PipeSmem<G, V, ITEMS, PAT>;
    constexpr int KP = G * V;
    static_assert(ITEMS % PF == 0, "PF");
    static_assert(PF <= 32, "PF");
    static_assert(sizeof(PT) % 16 == 0 && offsetof(PT, cv) % 16 == 0, "layout");
    static_assert(SM::PER_WARP % 16 == 0, "warp slices must stay 16-byte aligned");
    extern __shared__ __align__(16) unsigned char pipe_smem[];
    const CtlView cv = ctl_view(p.ctl);
    if (gate_off(p.gate, p.ctl) || *(volatile int32_t *)&cv.hdr->done) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int col0 = (lane % G) * V;
    unsigned char *base = pipe_smem + (size_t)warp * SM::PER_WARP;
    PT *buf = reinterpret_cast<PT *>(base);
    float *rs_s = reinterpret_cast<float *>(base + 2 * sizeof(PT));
    uint32_t ep_raw = 0, ep = 0;
    if constexpr (FUSE) {
        ep_raw = *(volatile uint32_t *)&cv.hdr->epoch;
        ep = (ep_raw + 1u) & 0x7fffffffu;
    }
    int alive[V];
    float l1[V];
#pragma unroll
    for (int j = 0; j < V; ++j) {
        alive[j] = cv.alive[col0 + j];
        l1[j] = 0.0f;
    }
    constexpr int RC = PT::CH / 32;   // chunks per lane held in registers
    const int64_t stride = (int64_t)gridDim.x * WARPS;
    int64_t t = (int64_t)blockIdx.x * WARPS + warp;
    TileMeta cur = tile_meta(p, t);
    ChunkRegs<RC> rg;
    if (t < p.tiles) {
        load_chunks<RC, PAT>(p, cur, rg, lane);   // the first tile waits for its loads
        stage_tile<RC, PAT>(p, cur, rg, buf[0].rp, buf[0].cv, buf[0].inv, lane);
    }
    cp_async_commit();
    TileMeta nxt = tile_meta(p, t + stride);
    load_chunks<RC, PAT>(p, nxt, rg, lane);
    int b = 0;
    for (; t < p.tiles; t += stride) {
        if (t + stride < p.tiles) stage_tile<RC, PAT>(p, nxt, rg, buf[b ^ 1].rp, buf[b ^ 1].cv, buf[b ^ 1].inv, lane);
        cp_async_commit();
        const TileMeta after = tile_meta(p, t + 2 * stride);
        load_chunks<RC, PAT>(p, after, rg, lane);   // in flight during this walk
        cp_async_wait_group<1>();              // this tile's copies have landed
        __syncwarp();
        walk_tile<G, V, ITEMS, PF, PAT, FUSE>(p, cur, t, buf[b].rp, buf[b].cv, buf[b].inv, rs_s, lane, alive, l1,
                                              ep << 1);
        __syncwarp();                          // buffers and row sums are rewritten next iteration
        cur = nxt;
        nxt = after;
        b ^= 1;
    }
    cp_async_wait_group<0>();
    if constexpr (FUSE) {
        // the rows this warp's tiles deferred (the head parts it stored are
        // visible to its own lanes after the barrier)
        __syncwarp();
        float l1t[KP];
#pragma unroll
        for (int c = 0; c < KP; ++c) l1t[c] = 0.0f;
        pipe_tail<KP>(p, (int64_t)blockIdx.x * WARPS + warp, stride, ep, cv, lane, l1t);
        // L1 partial of the CTA; the last CTA to finish sums the partials in a
        // fixed order and applies the break test of Algorithm 1 per column
        __shared__ float s_l1[WARPS][KP];
        __shared__ double s_fin[256];
        __shared__ int s_last;
#pragma unroll
        for (int c = 0; c < KP; ++c) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) l1t[c] += __shfl_xor_sync(0xffffffffu, l1t[c], o);
        }
        if (lane == 0) {
#pragma unroll
            for (int c = 0; c < KP; ++c) s_l1[warp][c] = l1t[c];
        }
        __syncwarp();
#pragma unroll
        for (int j = 0; j < V; ++j) {
            float a = l1[j];
#pragma unroll
            for (int o = G; o < 32; o <<= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
            if (lane < G) s_l1[warp][col0 + j] += a;
        }
        __syncthreads();
        if (threadIdx.x < KP) {
            float a = 0.0f;
#pragma unroll
            for (int w = 0; w < WARPS; ++w) a += s_l1[w][threadIdx.x];
            p.part[(int64_t)blockIdx.x * KP + threadIdx.x] = (double)a;
        }
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) s_last = (atomicAdd(&cv.hdr->ticket, 1) == (int)gridDim.x - 1);
        __syncthreads();
        if (!s_last) return;
        __threadfence();
        block_sum_partials_t<KP, double, WARPS * 32>(p.part, gridDim.x, s_fin);
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
            cv.hdr->ticket = 0;
            cv.hdr->epoch = ep_raw + 1u;
        }
    } else {
        // this warp's L1 partial over all its tiles (fixed order: deterministic
        // for a given grid), one row of tl1 per warp of the grid
#pragma unroll
        for (int j = 0; j < V; ++j) {
            float a = l1[j];
#pragma unroll
            for (int o = G; o < 32; o <<= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
            l1[j] = a;
        }
        if (lane < G) {
            const int64_t slot = (int64_t)blockIdx.x * WARPS + warp;
#pragma unroll
            for (int j = 0; j < V; ++j) p.tl1[slot * (G * V) + col0 + j] = l1[j];
        }
    }
}


// --------------------------------------------------------------- fixup ---
constexpr int FIX_WARPS = 8;

// Persistent grid: each warp takes tiles in a fixed round-robin order, adds the
// carries of earlier tiles to the tile's deferred row (unrolled, fixed order),
// applies the epilogue and accumulates the per-tile L1; the last block to
// finish reduces the block partials in parallel in a fixed order and applies
// the break test.
template <int KP>
__global__ void __launch_bounds__(FIX_WARPS * 32) fixup_k(Params p)
{
    constexpr int CW = KP < 32 ? KP : 32;    // columns per lane group
    constexpr int SUB = 32 / CW;             // lanes sharing one column
    constexpr int NCH = KP / CW;             // column chunks per lane
    static_assert(FIX_WARPS * 32 == 256, "block_sum_partials runs on 256 threads");
    __shared__ float s_l1[FIX_WARPS][KP];
    __shared__ double s_red[256];
    __shared__ int s_last;
    const CtlView cv = ctl_view(p.ctl);
    if (gate_off(p.gate, p.ctl) || *(volatile int32_t *)&cv.hdr->done) return;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int cl = lane % CW, sub = lane / CW;
    float l1acc[NCH];
#pragma unroll
    for (int i = 0; i < NCH; ++i) l1acc[i] = 0.0f;

    for (int64_t t = (int64_t)blockIdx.x * FIX_WARPS + warp; t < p.tiles; t += (int64_t)gridDim.x * FIX_WARPS) {
        const int32_t h = p.head_row[t];
        const int64_t first = p.head_first[t];
#pragma unroll
        for (int i = 0; i < NCH; ++i) {
            const int c = i * CW + cl;
            float l1 = (sub == 0 && t < (p.l1_slots ? p.l1_slots : p.tiles)) ? p.tl1[t * KP + c] : 0.0f;
            if (h >= 0) {
                float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f, s3 = 0.0f;
                int64_t u = first + sub;
                for (; u + 3 * SUB < t; u += 4 * SUB) {
                    s0 += p.carry[u * KP + c];
                    s1 += p.carry[(u + SUB) * KP + c];
                    s2 += p.carry[(u + 2 * SUB) * KP + c];
                    s3 += p.carry[(u + 3 * SUB) * KP + c];
                }
                for (; u < t; u += SUB) s0 += p.carry[u * KP + c];
                float s = (s0 + s1) + (s2 + s3);
#pragma unroll
                for (int o = CW; o < 32; o <<= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
                if (sub == 0) {
                    float tot[1] = {p.head[t * KP + c] + s};
                    int al[1] = {cv.alive[c]};
                    float e[1] = {0.0f};
                    epilogue<KP, 1>(p, (int64_t)h, c, tot, al, e);
                    l1 += e[0];
                }
            }
            l1acc[i] += l1;
        }
    }
    if (sub == 0) {
#pragma unroll
        for (int i = 0; i < NCH; ++i) s_l1[warp][i * CW + cl] = l1acc[i];
    }
    __syncthreads();
    for (int c = threadIdx.x; c < KP; c += FIX_WARPS * 32) {
        float sum = 0.0f;
#pragma unroll
        for (int w = 0; w < FIX_WARPS; ++w) sum += s_l1[w][c];
        p.part[(int64_t)blockIdx.x * KP + c] = (double)sum;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(&cv.hdr->ticket, 1) == (int)gridDim.x - 1);
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    block_sum_partials<KP>(p.part, gridDim.x, s_red);
    for (int c = threadIdx.x; c < KP; c += FIX_WARPS * 32) {
        const double sum = s_red[c];
        if (c < p.k && cv.alive[c]) {
            cv.norm[c] = sum;
            cv.iters[c] = p.iter;
            // the break test; the finalize iteration is the last one, so the
            // break state stays as it was for finalize_if_done_k
            if (sum < p.eps && p.mode == MODE_ACC) cv.alive[c] = 0;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int any = 0;
        for (int c = 0; c < p.k && c < KP; ++c) any |= cv.alive[c];
        cv.hdr->done = any ? 0 : 1;
        cv.hdr->ticket = 0;
    }
}

// Fixup for narrow widths (KP <= 8): one thread per tile, so the dependent
// loads of many tiles are in flight at once.  A deferred row whose carries
// span at most FIX_SHORT earlier tiles is summed by its thread in tile order;
// longer spans (rows of hubs) are summed by the whole warp in a fixed
// lane-strided order.  The last block reduces the block partials of the L1
// norm in a fixed order and applies the break test.
constexpr int FIX_SHORT = 32;

template <int V>
__global__ void __launch_bounds__(256) fixup_small_k(Params p)
{
    __shared__ float s_red[8][V];
    __shared__ double s_fin[256];
    __shared__ int s_last;
    const CtlView cv = ctl_view(p.ctl);
    if (gate_off(p.gate, p.ctl) || *(volatile int32_t *)&cv.hdr->done) return;
    int alive[V];
#pragma unroll
    for (int q = 0; q < V; ++q) alive[q] = cv.alive[q];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float l1[V];
#pragma unroll
    for (int q = 0; q < V; ++q) l1[q] = 0.0f;
    // a persistent grid: each thread takes tiles blockIdx*256 + tid, then one
    // grid further on (the block's loop count is uniform)
    for (int64_t base = (int64_t)blockIdx.x * 256; base < p.tiles; base += (int64_t)gridDim.x * 256) {
        const int64_t t = base + threadIdx.x;
        const bool mine = t < p.tiles;
        const int32_t h = mine ? p.head_row[t] : -1;
        const int64_t first = mine ? (int64_t)p.head_first[t] : 0;
        const bool has_l1 = mine && t < (p.l1_slots ? p.l1_slots : p.tiles);
#pragma unroll
        for (int q = 0; q < V; ++q) l1[q] += has_l1 ? p.tl1[t * V + q] : 0.0f;
        const bool longspan = h >= 0 && t - first > FIX_SHORT;
        if (h >= 0 && !longspan) {
            float sum[V];
            ld_row<V>(p.head + t * V, sum);
            for (int64_t u = first; u < t; ++u) {
                float c[V];
                ld_row<V>(p.carry + u * V, c);
#pragma unroll
                for (int q = 0; q < V; ++q) sum[q] += c[q];
            }
            epilogue<V, V>(p, (int64_t)h, 0, sum, alive, l1);
        }
        unsigned lm = __ballot_sync(0xffffffffu, longspan);
        while (lm) {
            const int src = __ffs(lm) - 1;
            lm &= lm - 1;
            const int64_t tt = __shfl_sync(0xffffffffu, t, src);
            const int64_t ff = __shfl_sync(0xffffffffu, first, src);
            float part[V];
#pragma unroll
            for (int q = 0; q < V; ++q) part[q] = 0.0f;
            for (int64_t u = ff + lane; u < tt; u += 32) {
                float c[V];
                ld_row<V>(p.carry + u * V, c);
#pragma unroll
                for (int q = 0; q < V; ++q) part[q] += c[q];
            }
#pragma unroll
            for (int q = 0; q < V; ++q) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) part[q] += __shfl_xor_sync(0xffffffffu, part[q], o);
            }
            if (lane == src) {
                float sum[V];
                ld_row<V>(p.head + t * V, sum);
#pragma unroll
                for (int q = 0; q < V; ++q) sum[q] += part[q];
                epilogue<V, V>(p, (int64_t)h, 0, sum, alive, l1);
            }
        }
    }
    // block partial of the L1 norm, fixed order
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

// ---------------------------------------------------------- init / misc ---
// x0 = c q per column (one-hot at seeds[j], or c/n everywhere when seeds is null);
// r = x0 when s_iter == 0, else 0.
// With inv_deg (pattern-only products) x holds x0 scaled by the row's inverse
// out-degree; r gets x0 itself.
__global__ void init_k(float *x, int KP, int64_t n, const int32_t *seeds, int k, float c_val, float pr_val,
                       float *r, int64_t ldr, int acc0, const void *ctl, int gate, const float *inv_deg)
{
    if (gate_off(gate, ctl)) return;
    const int64_t total = n * KP;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = i / KP;
        const int j = (int)(i % KP);
        float x0 = 0.0f;
        if (j < k) x0 = seeds ? (seeds[j] == v ? c_val : 0.0f) : pr_val;
        x[i] = inv_deg ? x0 * __ldg(inv_deg + v) : x0;
        if (r && j < k) r[v * ldr + j] = acc0 ? x0 : 0.0f;
    }
}

// x0 of seed-set columns (x and r zeroed before): block j adds c / |S_j| for
// each member of set j (scaled by inv_deg in x for pattern-only products;
// unscaled into r when acc0).  Repeated members add equal values, so the
// order of the atomics does not change the sums.
__global__ void scatter_sets_k(float *x, int KP, const int64_t *set_ptr, const int32_t *members, float c_val,
                               float *r, int64_t ldr, int acc0, const float *inv_deg)
{
    const int j = blockIdx.x;
    const int64_t e0 = set_ptr[j], e1 = set_ptr[j + 1];
    const float w = c_val / (float)(e1 - e0);
    for (int64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
        const int64_t v = members[e];
        atomicAdd(x + v * KP + j, inv_deg ? w * __ldg(inv_deg + v) : w);
        if (r && acc0) atomicAdd(r + v * ldr + j, w);
    }
}

__global__ void ctl_init_k(void *ctl, int k)
{
    const CtlView cv = ctl_view(ctl);
    for (int j = threadIdx.x; j < KP_MAX; j += blockDim.x) {
        cv.alive[j] = j < k ? 1 : 0;
        cv.iters[j] = 0;
        cv.own[j] = 0;
        cv.norm[j] = 0.0;
        cv.norm1[j] = 0.0;
    }
    if (threadIdx.x == 0) {
        cv.hdr->done = 0;
        cv.hdr->ticket = 0;
        cv.hdr->iter = 0;
        cv.hdr->push = 0;
    }
}

// r_TPA = (1+alpha) r_family + r_str, used when the family has no SpMV (S = 1)
__global__ void finalize_k(const float *r, int64_t ldr, const float *r_str, float opa, float *out, int64_t ldo,
                           int64_t n, int k)
{
    const int64_t total = n * k;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = i / k;
        const int j = (int)(i % k);
        out[v * ldo + j] = fmaf(opa, r[v * ldr + j], r_str[v]);
    }
}

// The finalize of Algorithm 3 when every column broke before the last family
// iteration (the SpMM of that iteration then returned early):
// r_TPA = (1+alpha) r_family + r_str.
__global__ void finalize_if_done_k(const void *ctl, const float *r, int64_t ldr, const float *r_str, float opa,
                                   float *out, int64_t ldo, int64_t n, int k)
{
    const CtlView cv = ctl_view(const_cast<void *>(ctl));
    if (!*(volatile int32_t *)&cv.hdr->done) return;
    const int64_t total = n * k;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = i / k;
        const int j = (int)(i % k);
        out[v * ldo + j] = fmaf(opa, r[v * ldr + j], r_str[v]);
    }
}

__global__ void copy_iters_k(const void *ctl, int32_t *out, int k)
{
    const CtlView cv = ctl_view(const_cast<void *>(ctl));
    for (int j = threadIdx.x; j < k; j += blockDim.x) out[j] = cv.iters[j];
}

// ---------------------------------------------------------- push path ---
// The first family iterates of a query are sparse: x1 lives on the
// out-neighbours of the seed and x2 on their out-neighbours (about 0.2% of the
// edges are touched), while a pull iteration streams the whole CSR.  So for
// light seeds x1 and x2 are pushed along CSR(A~) and only iterations 3.. are
// pulled:
//   x1[u] = (1-c) (A~_su c)                 for u in out(s)
//   x2[v] = (1-c) sum_u A~_uv x1[u]
// x2 is accumulated in 64-bit fixed point (scale 2^63; every term is
// non-negative and the total mass is below 1), so the integer atomics make the
// sum independent of their order: the result is deterministic and rounded to
// FP32 once.  r starts as x0 + x1; the conversion adds x2 to r for the
// columns that passed the break test after x1.
constexpr float FX_SCALE_F = 9223372036854775808.0f;      // 2^63, exact in FP32
constexpr float FX_INV_F = 1.0842021724855044e-19f;       // 2^-63, exact in FP32

// One block per (column j, slice): the block loads the seed's out-edges (at
// most PUSH_THREADS, one per thread) with the out-degree of each neighbour,
// takes an exclusive prefix sum of those degrees, and then treats the edges
// of all neighbours as one flat range split over the column's blocks (a
// binary search in the prefix finds each edge's neighbour), so the work of a
// seed is spread evenly whatever its neighbours' degrees.  Block 0 also
// writes x0 and x1 into r and ||x1||_1 (summed in out-edge order).
constexpr int PUSH_THREADS = 256;

__global__ void __launch_bounds__(PUSH_THREADS) push_x2_k(const int64_t *rp_a, const int32_t *col_a,
                                                          const float *val_a, const int32_t *seeds, int KP, float c_f,
                                                          float decay, unsigned long long *U, uint32_t *touched,
                                                          float *R, void *ctl, int gate)
{
    if (gate_off(gate, ctl)) return;
    __shared__ int64_t s_start[PUSH_THREADS];     // first out-edge of neighbour k
    __shared__ int64_t s_pref[PUSH_THREADS + 1];  // exclusive prefix of the neighbours' out-degrees
    __shared__ float s_x1[PUSH_THREADS];
    __shared__ int64_t s_warp[PUSH_THREADS / 32];
    const CtlView cv = ctl_view(ctl);
    const int j = blockIdx.y, k = threadIdx.x, lane = k & 31, warp = k >> 5;
    const int32_t s = seeds[j];
    const int64_t e0 = rp_a[s];
    const int deg_s = (int)(rp_a[s + 1] - e0);    // <= PUSH_THREADS (checked by the host)
    int64_t dk = 0;
    if (k < deg_s) {
        const int32_t u = col_a[e0 + k];
        const float x1u = decay * (val_a[e0 + k] * c_f);   // x1, as the pull computes it
        const int64_t f0 = rp_a[u];
        s_x1[k] = x1u;
        s_start[k] = f0;
        dk = rp_a[u + 1] - f0;
        if (blockIdx.x == 0) R[(int64_t)u * KP + j] = x1u;
    }
    // exclusive prefix of dk over the block
    int64_t v = dk;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    if (lane == 31) s_warp[warp] = v;
    __syncthreads();
    if (warp == 0) {
        int64_t w = lane < PUSH_THREADS / 32 ? s_warp[lane] : 0;
#pragma unroll
        for (int o = 1; o < PUSH_THREADS / 32; o <<= 1) {
            const int64_t t = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += t;
        }
        if (lane < PUSH_THREADS / 32) s_warp[lane] = w;
    }
    __syncthreads();
    s_pref[k + 1] = v + (warp > 0 ? s_warp[warp - 1] : 0);
    if (k == 0) s_pref[0] = 0;
    __syncthreads();
    if (blockIdx.x == 0 && k == 0) {
        R[(int64_t)s * KP + j] = c_f;                   // x0
        float nrm = 0.0f;
        for (int i = 0; i < deg_s; ++i) nrm += s_x1[i];
        cv.norm1[j] = (double)nrm;
    }
    const int64_t E = s_pref[deg_s];
    for (int64_t f = (int64_t)blockIdx.x * PUSH_THREADS + k; f < E; f += (int64_t)gridDim.x * PUSH_THREADS) {
        int lo = 0, hi = deg_s - 1;                     // the last neighbour whose range starts at or before f
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s_pref[mid] <= f) lo = mid; else hi = mid - 1;
        }
        const int64_t edge = s_start[lo] + (f - s_pref[lo]);
        const int32_t w = col_a[edge];
        const float q = val_a[edge] * s_x1[lo];
        atomicAdd(&U[(int64_t)w * KP + j], __float2ull_rn(q * FX_SCALE_F));
        atomicOr(&touched[w >> 5], 1u << (w & 31));     // rows the conversion must read
    }
}

// x2 in FP32 into X, a buffer that is zero outside the rows marked in
// `touched` (clear_x2_k restores that after the first pulled iteration): a
// warp covers 32 consecutive rows, i.e. one mark word, and skips an empty
// word without touching memory; marked rows read U (then cleared) and store
// their KP columns (padding columns zero).  x2 is added to r for the columns
// that passed the test after x1; ||x2||_1 per column; the last block applies
// the break tests after x1 and x2.
template <int KP>
__global__ void __launch_bounds__(256) convert_x2_k(unsigned long long *U, const uint32_t *touched, float *X,
                                                    float *R, int64_t n, int kc, float decay, double eps,
                                                    double *part, void *ctl, int gate, const float *inv_deg)
{
    if (gate_off(gate, ctl)) return;
    __shared__ float s_red[8][KP];
    __shared__ double s_fin[256];
    __shared__ int s_last;
    const CtlView cv = ctl_view(ctl);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    bool own[KP];
#pragma unroll
    for (int j = 0; j < KP; ++j) own[j] = j < kc && cv.norm1[j] >= eps;
    float nrm[KP];
#pragma unroll
    for (int j = 0; j < KP; ++j) nrm[j] = 0.0f;
    const int64_t step = (int64_t)gridDim.x * 256;
    for (int64_t base = (int64_t)blockIdx.x * 256; base < n; base += step) {
        const int64_t v = base + threadIdx.x;
        const uint32_t word = v < n ? touched[v >> 5] : 0u;   // the same word in the whole warp
        if ((word >> (v & 31)) & 1u) {
            float x[KP];
#pragma unroll
            for (int j = 0; j < KP; ++j) {
                x[j] = 0.0f;
                if (j < kc) {
                    const unsigned long long a = U[v * KP + j];
                    if (a) {
                        U[v * KP + j] = 0ull;
                        x[j] = decay * (__ull2float_rn(a) * FX_INV_F);
                        if (own[j]) R[v * KP + j] += x[j];
                    }
                }
                nrm[j] += x[j];
            }
            if (inv_deg) {   // pattern-only products gather x2 scaled by the inverse out-degree
                const float w = __ldg(inv_deg + v);
                float xs[KP];
#pragma unroll
                for (int j = 0; j < KP; ++j) xs[j] = x[j] * w;
                st_row<KP>(X + v * KP, xs);
            } else {
                st_row<KP>(X + v * KP, x);
            }
        }
    }
#pragma unroll
    for (int j = 0; j < KP; ++j) {
        float a = nrm[j];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if (lane == 0) s_red[warp][j] = a;
    }
    __syncthreads();
    if (threadIdx.x < KP) {
        float a = 0.0f;
#pragma unroll
        for (int w = 0; w < 8; ++w) a += s_red[w][threadIdx.x];
        part[(int64_t)blockIdx.x * KP + threadIdx.x] = (double)a;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(&cv.hdr->ticket, 1) == (int)gridDim.x - 1);
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    block_sum_partials<KP>(part, gridDim.x, s_fin);
    if (threadIdx.x < KP) {
        const int c = threadIdx.x;
        const double a = s_fin[c];
        if (c < kc) {
            const bool a1 = cv.norm1[c] >= eps;          // Algorithm 1 breaks after x1 when ||x1|| < eps
            const bool a2 = a1 && a >= eps;              // ... or after x2
            cv.alive[c] = a2 ? 1 : 0;
            cv.iters[c] = a1 ? 2 : 1;
            cv.norm[c] = a1 ? a : cv.norm1[c];
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) cv.hdr->ticket = 0;   // done stays 0: iteration 3 is pulled
}

// Per query chunk: the push branch is taken when every seed has at most
// PUSH_MAX_OUTDEG out-edges (the push kernel takes one thread per out-edge).
__global__ void push_decide_k(const int32_t *seeds, int kc, const int32_t *outdeg, int max_outdeg, void *ctl)
{
    const int lane = threadIdx.x;
    bool ok = true;
    for (int j = lane; j < kc; j += 32) ok = ok && outdeg[seeds[j]] <= max_outdeg;
    ok = __all_sync(0xffffffffu, ok);
    if (lane == 0) reinterpret_cast<Ctl *>(ctl)->push = ok ? 1 : 0;
}

// x[0..count) = 0 on a gated branch.
__global__ void zero_k(float *x, int64_t count, const void *ctl, int gate)
{
    if (gate_off(gate, ctl)) return;
    const int64_t n4 = count / 4;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x)
        reinterpret_cast<float4 *>(x)[i] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    for (int64_t i = 4 * n4 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x)
        x[i] = 0.0f;
}

// Restore the x2 buffer to zero and clear the row marks after the first pulled
// iteration has read x2: one thread per mark word.
template <int KP>
__global__ void clear_x2_k(uint32_t *touched, float *X, int64_t nwords, const void *ctl, int gate)
{
    if (gate_off(gate, ctl)) return;
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < nwords; w += (int64_t)gridDim.x * blockDim.x) {
        uint32_t word = touched[w];
        if (!word) continue;
        touched[w] = 0u;
        float z[KP];
#pragma unroll
        for (int j = 0; j < KP; ++j) z[j] = 0.0f;
        while (word) {
            const int b = __ffs(word) - 1;
            word &= word - 1;
            st_row<KP>(X + (w * 32 + b) * KP, z);
        }
    }
}

// ------------------------------------------------------------- planning ---
__global__ void plan_tiles_k(const int64_t *rp, int64_t n, int64_t m, int64_t L, int64_t tiles, int32_t *tx, int64_t *ty)
{
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t <= tiles; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t D = min(t * L, n + m);
        int64_t lo = max((int64_t)0, D - m), hi = min(D, n);
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if (rp[mid + 1] + mid + 1 <= D) lo = mid + 1; else hi = mid;
        }
        tx[t] = (int32_t)lo;
        ty[t] = D - lo;
    }
}

__global__ void plan_heads_k(const int64_t *rp, const int32_t *tx, const int64_t *ty, int64_t tiles, int32_t *hr, int32_t *hf)
{
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < tiles; t += (int64_t)gridDim.x * blockDim.x) {
        const int32_t x0 = tx[t], x1 = tx[t + 1];
        const int64_t y0 = ty[t];
        if (x0 < x1 && rp[x0] < y0) {
            hr[t] = x0;
            // last tile whose start is at or before the row's first nonzero
            const int64_t s = rp[x0];
            int64_t lo = 0, hi = t;
            while (lo < hi) {
                const int64_t mid = (lo + hi + 1) >> 1;
                if (ty[mid] <= s) lo = mid; else hi = mid - 1;
            }
            hf[t] = (int32_t)lo;
        } else {
            hr[t] = -1;
            hf[t] = (int32_t)t;
        }
    }
}

}  // namespace tpa
