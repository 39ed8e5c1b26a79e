// CSR construction of the row-normalised adjacency A~ (Table 1) on the GPU.
//
// Raw edges (src, dst) -> 64-bit keys dst<<32|src -> stable LSD radix sort
// over the bits that node ids use -> drop self-loops and duplicates ->
// CSR(A~^T) (rows = dst, sources ascending).  A second stable radix pass over
// the source bits gives CSR(A~) (rows = src, destinations ascending) and the
// out-degrees; A~_uv = RN32(1 / outdeg(u)) with IEEE division.
//
// Every step is deterministic: the sorted, de-duplicated key list is unique,
// so the CSR arrays are bit-identical to any other correct construction.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "tpa_internal.cuh"

namespace tpa {
namespace {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 16;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

constexpr int SORT_THREADS = 256;
constexpr int SORT_WARPS = SORT_THREADS / 32;
constexpr int SORT_ITEMS = 16;
constexpr int SORT_TILE = SORT_THREADS * SORT_ITEMS;
constexpr int RADIX = 256;

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Block-wide exclusive scan of one value per thread (SCAN_THREADS threads).
template <class T>
__device__ T block_exclusive_scan(T v, T *total, T *s_warp)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        T w = lane < (int)(blockDim.x >> 5) ? s_warp[lane] : T(0);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < (int)(blockDim.x >> 5)) s_warp[lane] = w;   // inclusive warp totals
    }
    __syncthreads();
    T before = warp > 0 ? s_warp[warp - 1] : T(0);
    *total = s_warp[(blockDim.x >> 5) - 1];
    __syncthreads();
    return before + x - v;
}

// ---------------------------------------------------------------- scans ---
template <class Tin, class Tout>
__global__ void __launch_bounds__(SCAN_THREADS) scan_reduce_k(const Tin *in, int64_t len, Tout *part)
{
    __shared__ Tout s_warp[32];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    Tout sum = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i)
        if (base + i < len) sum += (Tout)in[base + i];
    Tout total;
    block_exclusive_scan<Tout>(sum, &total, s_warp);
    if (threadIdx.x == 0) part[blockIdx.x] = total;
}

// Single block: exclusive scan of part[0..nb) in place, part[nb] = total.
template <class Tout>
__global__ void __launch_bounds__(SCAN_THREADS) scan_partials_k(Tout *part, int64_t nb)
{
    __shared__ Tout s_warp[32];
    Tout carry = 0;
    for (int64_t b0 = 0; b0 < nb; b0 += SCAN_THREADS) {
        const int64_t i = b0 + threadIdx.x;
        Tout v = i < nb ? part[i] : Tout(0);
        Tout total;
        Tout ex = block_exclusive_scan<Tout>(v, &total, s_warp);
        if (i < nb) part[i] = carry + ex;
        carry += total;
    }
    if (threadIdx.x == 0) part[nb] = carry;
}

template <class Tin, class Tout>
__global__ void __launch_bounds__(SCAN_THREADS) scan_down_k(const Tin *in, int64_t len, const Tout *part, Tout *out)
{
    __shared__ Tout s_warp[32];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    Tout v[SCAN_ITEMS];
    Tout sum = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        v[i] = base + i < len ? (Tout)in[base + i] : Tout(0);
        sum += v[i];
    }
    Tout total;
    Tout run = part[blockIdx.x] + block_exclusive_scan<Tout>(sum, &total, s_warp);
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i)
        if (base + i < len) {
            out[base + i] = run;
            run += v[i];
        }
}

// out[0..len) = exclusive scan of in; out[len] = total if with_total.
template <class Tin, class Tout>
void exclusive_scan(const Tin *in, Tout *out, int64_t len, bool with_total, DevBuf &tmp, cudaStream_t s)
{
    const int64_t nb = std::max<int64_t>(1, (len + SCAN_TILE - 1) / SCAN_TILE);
    tmp.ensure((size_t)(nb + 1) * sizeof(Tout), s);
    Tout *part = tmp.as<Tout>();
    scan_reduce_k<Tin, Tout><<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, len, part);
    scan_partials_k<Tout><<<1, SCAN_THREADS, 0, s>>>(part, nb);
    scan_down_k<Tin, Tout><<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, len, part, out);
    note_launch("scan", 3);
    if (with_total) TPA_CUDA(cudaMemcpyAsync(out + len, part + nb, sizeof(Tout), cudaMemcpyDeviceToDevice, s));
    TPA_CHECK_LAUNCH();
}

// ----------------------------------------------------------- radix sort ---
__global__ void __launch_bounds__(SORT_THREADS) radix_hist_k(const uint64_t *keys, int64_t len, int shift,
                                                             uint32_t *hist, int64_t ntiles)
{
    __shared__ uint32_t h[RADIX];
    for (int i = threadIdx.x; i < RADIX; i += SORT_THREADS) h[i] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * SORT_TILE;
    const int lane = threadIdx.x & 31;
    for (int j = 0; j < SORT_ITEMS; ++j) {
        const int64_t idx = base + (int64_t)j * SORT_THREADS + threadIdx.x;
        const bool valid = idx < len;
        const unsigned d = valid ? (unsigned)((keys[idx] >> shift) & (RADIX - 1)) : RADIX;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        if (valid && lane == __ffs(peers) - 1) atomicAdd(&h[d], (uint32_t)__popc(peers));
    }
    __syncthreads();
    for (int i = threadIdx.x; i < RADIX; i += SORT_THREADS) hist[(int64_t)i * ntiles + blockIdx.x] = h[i];
}

struct SortSmem {
    uint64_t keys[SORT_TILE];
    uint32_t vals[SORT_TILE];
    uint32_t wcnt[SORT_WARPS][RADIX];
    uint32_t dofs[RADIX];
    uint32_t gofs[RADIX];
    uint32_t warp_tmp[32];
};

// Stable scatter of one tile by digit.  Warp w owns tile items [w*512, (w+1)*512)
// in rounds of 32 consecutive keys, so (warp, round, lane) is the input order.
template <bool HAS_VAL>
__global__ void __launch_bounds__(SORT_THREADS) radix_scatter_k(const uint64_t *kin, const uint32_t *vin,
                                                                uint64_t *kout, uint32_t *vout, int64_t len,
                                                                int shift, const uint32_t *gofs, int64_t ntiles)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SortSmem &S = *reinterpret_cast<SortSmem *>(smem_raw);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t base = (int64_t)blockIdx.x * SORT_TILE;
    const int count = (int)std::min<int64_t>(SORT_TILE, len - base);

    for (int i = lane; i < RADIX; i += 32) S.wcnt[warp][i] = 0;
    __syncwarp();

    uint64_t k[SORT_ITEMS];
    uint32_t v[SORT_ITEMS];
    uint32_t rank[SORT_ITEMS];
    const unsigned lt = lanemask_lt();
#pragma unroll
    for (int j = 0; j < SORT_ITEMS; ++j) {
        const int idx = warp * (32 * SORT_ITEMS) + j * 32 + lane;
        const bool valid = idx < count;
        k[j] = valid ? kin[base + idx] : 0ull;
        if (HAS_VAL) v[j] = valid ? vin[base + idx] : 0u;
        const unsigned d = valid ? (unsigned)((k[j] >> shift) & (RADIX - 1)) : RADIX;
        const unsigned peers = __match_any_sync(0xffffffffu, d);
        const uint32_t before = valid ? S.wcnt[warp][d] : 0u;
        __syncwarp();
        if (valid && (peers & lt) == 0) S.wcnt[warp][d] = before + (uint32_t)__popc(peers);
        __syncwarp();
        rank[j] = before + (uint32_t)__popc(peers & lt);
    }
    __syncthreads();
    // per digit: exclusive prefix over warps, then over digits
    {
        const int d = threadIdx.x;   // SORT_THREADS == RADIX
        uint32_t run = 0;
#pragma unroll
        for (int w = 0; w < SORT_WARPS; ++w) {
            const uint32_t c = S.wcnt[w][d];
            S.wcnt[w][d] = run;
            run += c;
        }
        uint32_t total;
        const uint32_t ex = block_exclusive_scan<uint32_t>(run, &total, S.warp_tmp);
        S.dofs[d] = ex;
        S.gofs[d] = gofs[(int64_t)d * ntiles + blockIdx.x];
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < SORT_ITEMS; ++j) {
        const int idx = warp * (32 * SORT_ITEMS) + j * 32 + lane;
        if (idx < count) {
            const unsigned d = (unsigned)((k[j] >> shift) & (RADIX - 1));
            const uint32_t pos = S.dofs[d] + S.wcnt[warp][d] + rank[j];
            S.keys[pos] = k[j];
            if (HAS_VAL) S.vals[pos] = v[j];
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < count; i += SORT_THREADS) {
        const uint64_t key = S.keys[i];
        const unsigned d = (unsigned)((key >> shift) & (RADIX - 1));
        const uint64_t dst = (uint64_t)S.gofs[d] + (uint64_t)(i - (int)S.dofs[d]);
        kout[dst] = key;
        if (HAS_VAL) vout[dst] = S.vals[i];
    }
}

// Stable LSD sort of keys over the given digit shifts.  Returns the buffer
// index (0 = a, 1 = b) that holds the result.
int radix_sort(uint64_t *ka, uint64_t *kb, uint32_t *va, uint32_t *vb, int64_t len,
               const std::vector<int> &shifts, DevBuf &hist, DevBuf &tmp, cudaStream_t s)
{
    if (len == 0 || shifts.empty()) return 0;
    TPA_REQUIRE(len < (int64_t)UINT32_MAX, "radix sort: %lld keys exceed the 32-bit offset range", (long long)len);
    const int64_t ntiles = (len + SORT_TILE - 1) / SORT_TILE;
    hist.ensure((size_t)ntiles * RADIX * sizeof(uint32_t), s);
    const size_t smem = sizeof(SortSmem);
    static bool attr_done = false;
    if (!attr_done) {
        TPA_CUDA(cudaFuncSetAttribute(radix_scatter_k<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        TPA_CUDA(cudaFuncSetAttribute(radix_scatter_k<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        attr_done = true;
    }
    int cur = 0;
    for (int sh : shifts) {
        uint64_t *kin = cur ? kb : ka, *kout = cur ? ka : kb;
        uint32_t *vin = cur ? vb : va, *vout = cur ? va : vb;
        radix_hist_k<<<(unsigned)ntiles, SORT_THREADS, 0, s>>>(kin, len, sh, hist.as<uint32_t>(), ntiles);
        exclusive_scan<uint32_t, uint32_t>(hist.as<uint32_t>(), hist.as<uint32_t>(), ntiles * RADIX, false, tmp, s);
        if (va)
            radix_scatter_k<true><<<(unsigned)ntiles, SORT_THREADS, smem, s>>>(kin, vin, kout, vout, len, sh,
                                                                                 hist.as<uint32_t>(), ntiles);
        else
            radix_scatter_k<false><<<(unsigned)ntiles, SORT_THREADS, smem, s>>>(kin, nullptr, kout, nullptr, len, sh,
                                                                                  hist.as<uint32_t>(), ntiles);
        TPA_CHECK_LAUNCH();
        note_launch("sort", 2);
        cur ^= 1;
    }
    return cur;
}

// ------------------------------------------------------- graph assembly ---
__global__ void check_ids_k(const int32_t *src, const int32_t *dst, int64_t m, int64_t n, int *bad)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t a = src[e], b = dst[e];
        if (a < 0 || a >= n || b < 0 || b >= n) atomicOr(bad, 1);
    }
}

__global__ void encode_k(const int32_t *src, const int32_t *dst, int64_t m, uint64_t *key)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x)
        key[e] = ((uint64_t)(uint32_t)dst[e] << 32) | (uint32_t)src[e];
}

// keep[i] = first of its run and not a self-loop
__global__ void keep_flags_k(const uint64_t *key, int64_t m, uint32_t *keep)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t k = key[i];
        const bool self = (uint32_t)(k >> 32) == (uint32_t)k;
        keep[i] = (!self && (i == 0 || key[i - 1] != k)) ? 1u : 0u;
    }
}

__global__ void compact_k(const uint64_t *key, const uint32_t *keep, const uint32_t *pos, int64_t m, uint64_t *out)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
        if (keep[i]) out[pos[i]] = key[i];
}

// Row lengths from a key list sorted by its high 32 bits: count[row] = run length.
__global__ void run_lengths_k(const uint64_t *key, int64_t m, int32_t *count)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t r = (uint32_t)(key[i] >> 32);
        if (i == 0 || (uint32_t)(key[i - 1] >> 32) != r) atomicSub(&count[r], (int32_t)i);
        if (i == m - 1 || (uint32_t)(key[i + 1] >> 32) != r) atomicAdd(&count[r], (int32_t)(i + 1));
    }
}

// CSR(A~^T) columns from keys dst<<32|src; also the swapped keys src<<32|dst.
__global__ void split_t_k(const uint64_t *key, int64_t m, int32_t *col, uint64_t *swapped)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t k = key[i];
        col[i] = (int32_t)(uint32_t)k;
        swapped[i] = (k << 32) | (k >> 32);
    }
}

// Sort keys for the edge map: key[i] = source of CSR(A~^T) edge i, idx[i] = i.
__global__ void src_keys_k(const int32_t *col_t, int64_t m, uint64_t *key, uint32_t *idx)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        key[i] = (uint64_t)(uint32_t)col_t[i];
        idx[i] = (uint32_t)i;
    }
}

__global__ void fill_vals_t_k(const int32_t *col, int64_t m, const int32_t *outdeg, float *val)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
        val[i] = 1.0f / (float)outdeg[col[i]];
}

// RN32(1/outdeg(u)) per node, the value every edge out of u carries in both
// CSRs (same expression as the edge values, so bit-identical); 0 for deadends.
__global__ void inv_deg_k(const int32_t *outdeg, int64_t n, float *inv)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t d = outdeg[i];
        inv[i] = d > 0 ? 1.0f / (float)d : 0.0f;
    }
}

__global__ void split_a_k(const uint64_t *key, int64_t m, const int32_t *outdeg, int32_t *col, float *val)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t k = key[i];
        col[i] = (int32_t)(uint32_t)k;
        val[i] = 1.0f / (float)outdeg[(uint32_t)(k >> 32)];
    }
}

unsigned grid_for(int64_t work, int threads)
{
    int64_t b = (work + threads - 1) / threads;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 64));
}

std::vector<int> digit_shifts(int nbits, int base)
{
    std::vector<int> v;
    for (int b = 0; b < nbits; b += 8) v.push_back(base + b);
    return v;
}

}  // namespace

void build_csr(tpa_graph *g, const int32_t *d_src, const int32_t *d_dst, int64_t m_in, cudaStream_t s)
{
    const int64_t n = g->n;
    int nbits = 0;
    while (nbits < 31 && ((int64_t)1 << nbits) < n) ++nbits;
    DevBuf ka, kb, hist, tmp, flags, pos, cnt;

    // 1. validate ids
    {
        DevBuf bad;
        bad.ensure(sizeof(int), s);
        TPA_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(int), s));
        if (m_in > 0) {
            check_ids_k<<<grid_for(m_in, 256), 256, 0, s>>>(d_src, d_dst, m_in, n, bad.as<int>());
            note_launch("build");
        }
        TPA_CHECK_LAUNCH();
        int h = 0;
        TPA_CUDA(cudaMemcpyAsync(&h, bad.p, sizeof(int), cudaMemcpyDeviceToHost, s));
        TPA_CUDA(cudaStreamSynchronize(s));
        bad.release(s);
        TPA_REQUIRE(h == 0, "tpa_build_graph: an edge endpoint is outside [0, n)");
    }

    // 2. sort raw keys by (dst, src)
    const size_t kbytes = (size_t)std::max<int64_t>(m_in, 1) * sizeof(uint64_t);
    ka.ensure(kbytes, s);
    kb.ensure(kbytes, s);
    if (m_in > 0) {
        encode_k<<<grid_for(m_in, 256), 256, 0, s>>>(d_src, d_dst, m_in, ka.as<uint64_t>());
        note_launch("build");
    }
    TPA_CHECK_LAUNCH();
    std::vector<int> sh = digit_shifts(nbits, 0);
    for (int x : digit_shifts(nbits, 32)) sh.push_back(x);
    int cur = radix_sort(ka.as<uint64_t>(), kb.as<uint64_t>(), nullptr, nullptr, m_in, sh, hist, tmp, s);
    uint64_t *sorted = cur ? kb.as<uint64_t>() : ka.as<uint64_t>();
    uint64_t *other = cur ? ka.as<uint64_t>() : kb.as<uint64_t>();

    // 3. drop self-loops and duplicates
    flags.ensure((size_t)std::max<int64_t>(m_in, 1) * sizeof(uint32_t) + sizeof(uint32_t), s);
    pos.ensure((size_t)(m_in + 1) * sizeof(uint32_t), s);
    if (m_in > 0) {
        keep_flags_k<<<grid_for(m_in, 256), 256, 0, s>>>(sorted, m_in, flags.as<uint32_t>());
        note_launch("build");
    }
    TPA_CHECK_LAUNCH();
    exclusive_scan<uint32_t, uint32_t>(flags.as<uint32_t>(), pos.as<uint32_t>(), m_in, true, tmp, s);
    uint32_t m32 = 0;
    TPA_CUDA(cudaMemcpyAsync(&m32, pos.as<uint32_t>() + m_in, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    TPA_CUDA(cudaStreamSynchronize(s));
    const int64_t m = m32;
    g->m = m;
    uint64_t *uk = other;   // unique keys, sorted by (dst, src)
    if (m_in > 0) {
        compact_k<<<grid_for(m_in, 256), 256, 0, s>>>(sorted, flags.as<uint32_t>(), pos.as<uint32_t>(), m_in, uk);
        note_launch("build");
    }
    TPA_CHECK_LAUNCH();
    flags.release(s);
    pos.release(s);

    // 4. allocate the graph arrays
    const size_t mp = (size_t)csr_len(m);
    g->rp_t.ensure((size_t)(n + 1) * sizeof(int64_t), s);
    g->col_t.ensure(mp * sizeof(int32_t), s);
    g->val_t.ensure(mp * sizeof(float), s);
    g->rp_a.ensure((size_t)(n + 1) * sizeof(int64_t), s);
    g->col_a.ensure(mp * sizeof(int32_t), s);
    g->val_a.ensure(mp * sizeof(float), s);
    for (DevBuf *b : {&g->col_t, &g->val_t, &g->col_a, &g->val_a})
        TPA_CUDA(cudaMemsetAsync(static_cast<char *>(b->p) + (size_t)m * 4, 0, (mp - (size_t)m) * 4, s));
    g->outdeg.ensure((size_t)n * sizeof(int32_t), s);
    g->inv_deg32.ensure((size_t)n * sizeof(float), s);
    cnt.ensure((size_t)n * sizeof(int32_t), s);

    // 5. CSR(A~^T) row pointers from run lengths of dst
    TPA_CUDA(cudaMemsetAsync(cnt.p, 0, (size_t)n * sizeof(int32_t), s));
    if (m > 0) {
        run_lengths_k<<<grid_for(m, 256), 256, 0, s>>>(uk, m, cnt.as<int32_t>());
        note_launch("build");
    }
    TPA_CHECK_LAUNCH();
    exclusive_scan<int32_t, int64_t>(cnt.as<int32_t>(), g->rp_t.as<int64_t>(), n, true, tmp, s);

    // 6. columns of A~^T and swapped keys (src, dst)
    uint64_t *sw = sorted;   // raw sorted keys are no longer needed
    if (m > 0) {
        split_t_k<<<grid_for(m, 256), 256, 0, s>>>(uk, m, g->col_t.as<int32_t>(), sw);
        note_launch("build");
    }
    TPA_CHECK_LAUNCH();

    // 7. stable sort by source -> CSR(A~) (within a source, destinations stay ascending)
    std::vector<int> sh_src = digit_shifts(nbits, 32);
    int cur2 = radix_sort(sw, uk, nullptr, nullptr, m, sh_src, hist, tmp, s);
    uint64_t *ak = cur2 ? uk : sw;
    TPA_CUDA(cudaMemsetAsync(g->outdeg.p, 0, (size_t)n * sizeof(int32_t), s));
    if (m > 0) {
        run_lengths_k<<<grid_for(m, 256), 256, 0, s>>>(ak, m, g->outdeg.as<int32_t>());
        note_launch("build");
    }
    TPA_CHECK_LAUNCH();
    exclusive_scan<int32_t, int64_t>(g->outdeg.as<int32_t>(), g->rp_a.as<int64_t>(), n, true, tmp, s);
    if (m > 0) {
        split_a_k<<<grid_for(m, 256), 256, 0, s>>>(ak, m, g->outdeg.as<int32_t>(), g->col_a.as<int32_t>(),
                                                   g->val_a.as<float>());
        fill_vals_t_k<<<grid_for(m, 256), 256, 0, s>>>(g->col_t.as<int32_t>(), m, g->outdeg.as<int32_t>(),
                                                       g->val_t.as<float>());
        note_launch("build", 2);
    }
    if (n > 0) {
        inv_deg_k<<<grid_for(n, 256), 256, 0, s>>>(g->outdeg.as<int32_t>(), n, g->inv_deg32.as<float>());
        note_launch("build");
    }
    TPA_CHECK_LAUNCH();
    // the edge map between the two CSRs is built when edge weights first need it
    g->perm_a2t.release(s);
    TPA_CUDA(cudaStreamSynchronize(s));
    ka.release(s); kb.release(s); hist.release(s); tmp.release(s); cnt.release(s);
}

void ensure_perm_a2t(tpa_graph *g, cudaStream_t s)
{
    if (g->perm_a2t.p) return;
    const int64_t n = g->n, m = g->m;
    int nbits = 0;
    while (nbits < 31 && ((int64_t)1 << nbits) < n) ++nbits;
    // CSR(A~^T) lists the edges by (dst, src); a stable sort by src puts them
    // in CSR(A~)'s (src, dst) order, carrying each edge's CSR(A~^T) index
    DevBuf ka, kb, ia, ib, hist, tmp;
    const size_t mb = (size_t)std::max<int64_t>(m, 1);
    ka.ensure(mb * sizeof(uint64_t), s);
    kb.ensure(mb * sizeof(uint64_t), s);
    ia.ensure(mb * sizeof(uint32_t), s);
    ib.ensure(mb * sizeof(uint32_t), s);
    if (m > 0) {
        src_keys_k<<<grid_for(m, 256), 256, 0, s>>>(g->col_t.as<int32_t>(), m, ka.as<uint64_t>(), ia.as<uint32_t>());
        note_launch("build");
    }
    TPA_CHECK_LAUNCH();
    const int cur = radix_sort(ka.as<uint64_t>(), kb.as<uint64_t>(), ia.as<uint32_t>(), ib.as<uint32_t>(), m,
                               digit_shifts(nbits, 0), hist, tmp, s);
    DevBuf &perm = cur ? ib : ia;
    g->perm_a2t = perm;
    perm.p = nullptr;
    perm.bytes = 0;
    ka.release(s); kb.release(s); ia.release(s); ib.release(s); hist.release(s); tmp.release(s);
}

void exclusive_scan_i32_i64(const int32_t *in, int64_t *out, int64_t len, DevBuf &tmp, cudaStream_t s)
{
    exclusive_scan<int32_t, int64_t>(in, out, len, true, tmp, s);
}

}  // namespace tpa
