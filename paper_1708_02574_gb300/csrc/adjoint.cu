// Gradient of a link-prediction loss on TPA scores with respect to edge
// weights (supervised random walks); not part of the paper's method.
//
// A~_uv = w_uv / d_u (d_u = sum_v w_uv), P = (1-c) A~^T.  For triples
// (s, p, q): r = (1+alpha) r_family(s) + r~_stranger (Algorithms 2-3 with the
// stranger chain run for a fixed K iterations), L = sum softplus(r[q] - r[p]).
// With g = dL/dr (two nonzeros per triple):
//   family   l_{S-1} = (1+alpha) g, l_i = (1+alpha) g + P^T l_{i+1}
//   stranger m_K = G, m_i = [i >= T] G + P^T m_{i+1}, G = sum over triples of g
//   dL/dA~_uv = (1-c) (sum_i l_i[v] x_{i-1}[u] + sum_i m_i[v] x'_{i-1}[u])
//   dL/dw_uv  = (dL/dA~_uv - sum_v' dL/dA~_uv' A~_uv') / d_u
// P x runs the merge-path SpMV over CSR(A~^T); P^T y the same kernel over
// CSR(A~) (rows = sources), i.e. the non-transposed A~.  The edge gradient is
// an SDDMM over CSR(A~) edges.  Every reduction has a fixed order; the
// stranger seed G is accumulated in 64-bit fixed point.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "tpa_internal.cuh"

namespace tpa {
namespace {

constexpr int KB_DEFAULT = 8;   // triples per family batch (8, 16 or 32; 8 measured fastest at scale 20)
constexpr double G_SCALE = 1099511627776.0;            // 2^40, fixed point of G

unsigned grid_for(int64_t work, int threads = 256)
{
    const int64_t b = (work + threads - 1) / threads;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 32));
}

__global__ void weights_k(const float *feat, const float *theta, int d, int64_t m, float *w)
{
    extern __shared__ float s_theta[];
    for (int j = threadIdx.x; j < d; j += blockDim.x) s_theta[j] = theta[j];
    __syncthreads();
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        float z = 0.0f;
        for (int j = 0; j < d; ++j) z = fmaf(s_theta[j], feat[e * d + j], z);
        w[e] = expf(z);
    }
}

// Warp per source row: d_u in FP64 (lane-strided, fixed shuffle tree), then
// A~ = w / d_u in both CSR orders.
__global__ void normalise_k(const int64_t *rp_a, const float *w, const uint32_t *perm, int64_t n, float *val_a,
                            float *val_t, double *inv_d)
{
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < n; u += warps) {
        const int64_t e0 = rp_a[u], e1 = rp_a[u + 1];
        double sum = 0.0;
        for (int64_t e = e0 + lane; e < e1; e += 32) sum += (double)w[e];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
        const double inv = sum > 0.0 ? 1.0 / sum : 0.0;
        if (lane == 0) inv_d[u] = inv;
        for (int64_t e = e0 + lane; e < e1; e += 32) {
            const float v = (float)((double)w[e] * inv);
            val_a[e] = v;
            val_t[perm[e]] = v;
        }
    }
}

__global__ void row_ids_k(const int64_t *rp_a, int64_t n, int32_t *row)
{
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < n; u += warps)
        for (int64_t e = rp_a[u] + lane; e < rp_a[u + 1]; e += 32) row[e] = (int32_t)u;
}

__global__ void fill_k(float *x, int64_t len, float v)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x) x[i] = v;
}

// r~_stranger = sum_{i=T}^{K} x'_i, summed in iteration order
__global__ void stranger_sum_k(const float *xs, int64_t n, int T, int K, float *rs)
{
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        float s = 0.0f;
        for (int i = T; i <= K; ++i) s += xs[(int64_t)i * n + v];
        rs[v] = s;
    }
}

// F_0 = c e_s for the batch's columns (padding columns stay zero)
template <int KB>
__global__ void family_init_k(float *F0, const int32_t *seeds, int kb, float c)
{
    const int j = threadIdx.x;
    if (j < kb) F0[(int64_t)seeds[j] * KB + j] = c;
}

// Scores at (p, q), loss and sigma per triple; G (stranger seed) in fixed point.
template <int KB>
__global__ void pair_k(const float *F, int64_t n, int S, const int32_t *pos, const int32_t *neg, int kb, float opa,
                       const float *rs, double *loss, double *sg, unsigned long long *gacc)
{
    const int j = threadIdx.x;
    if (j >= kb) return;
    const int32_t p = pos[j], q = neg[j];
    float fp = 0.0f, fq = 0.0f;
    for (int i = 0; i < S; ++i) {
        fp += F[((int64_t)i * n + p) * KB + j];
        fq += F[((int64_t)i * n + q) * KB + j];
    }
    const double rp = (double)fmaf(opa, fp, rs[p]);
    const double rq = (double)fmaf(opa, fq, rs[q]);
    const double z = rq - rp;
    loss[j] = z > 0 ? z + log1p(exp(-z)) : log1p(exp(z));
    const double s = 1.0 / (1.0 + exp(-z));
    sg[j] = s;
    const long long fx = __double2ll_rn(s * G_SCALE);
    atomicAdd(&gacc[q], (unsigned long long)fx);
    atomicAdd(&gacc[p], (unsigned long long)(-fx));
}

// lam[q][j] += (1+alpha) sg_j, lam[p][j] -= (1+alpha) sg_j  (one thread per column)
template <int KB>
__global__ void scatter_g_k(float *lam, const int32_t *pos, const int32_t *neg, const double *sg, int kb, float opa)
{
    const int j = threadIdx.x;
    if (j >= kb) return;
    const float a = (float)((double)opa * sg[j]);
    lam[(int64_t)neg[j] * KB + j] += a;
    lam[(int64_t)pos[j] * KB + j] -= a;
}

// sum of the per-triple losses in triple order
__global__ void loss_sum_k(const double *loss, int ntrip, double *out)
{
    double s = 0.0;
    for (int t = 0; t < ntrip; ++t) s += loss[t];
    out[0] = s;
}

__global__ void gacc_to_float_k(const unsigned long long *gacc, int64_t n, float *G)
{
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        G[v] = (float)((double)(long long)gacc[v] / G_SCALE);
}

__global__ void axpy_k(float *y, const float *x, int64_t n)
{
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) y[v] += x[v];
}

// GE[e] += coef * sum_j lam[v][j] * X[u][j] over CSR(A~) edges (u = row, v = col)
template <int W>
__global__ void sddmm_k(const int32_t *row, const int32_t *col, int64_t m, const float *lam, const float *X, int kc,
                        float coef, float *GE)
{
    // the padding columns kc .. W-1 of lam and X are zero, so summing all W
    // columns in order gives the same FP32 dot as stopping at kc
    (void)kc;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t u = row[e], v = col[e];
        float dot = 0.0f;
        if constexpr (W % 4 == 0) {
            const float4 *lv = reinterpret_cast<const float4 *>(lam + v * W);
            const float4 *xu = reinterpret_cast<const float4 *>(X + u * W);
#pragma unroll
            for (int q = 0; q < W / 4; ++q) {
                const float4 a = __ldg(lv + q), b = __ldg(xu + q);
                dot = fmaf(a.x, b.x, dot);
                dot = fmaf(a.y, b.y, dot);
                dot = fmaf(a.z, b.z, dot);
                dot = fmaf(a.w, b.w, dot);
            }
        } else {
#pragma unroll
            for (int j = 0; j < W; ++j) dot = fmaf(__ldg(lam + v * W + j), __ldg(X + u * W + j), dot);
        }
        GE[e] += coef * dot;
    }
}

// dL/dw_e = (GE_e - sum_{e' in row} GE_e' A~_e') / d_u  (warp per row, fixed order)
__global__ void jacobian_k(const int64_t *rp_a, const float *GE, const float *val_a, const double *inv_d, int64_t n,
                           float *grad_w)
{
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < n; u += warps) {
        const int64_t e0 = rp_a[u], e1 = rp_a[u + 1];
        float s = 0.0f;
        for (int64_t e = e0 + lane; e < e1; e += 32) s = fmaf(GE[e], val_a[e], s);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        const float inv = (float)inv_d[u];
        for (int64_t e = e0 + lane; e < e1; e += 32) grad_w[e] = (GE[e] - s) * inv;
    }
}

// dL/dtheta_j = sum_e grad_w_e w_e f_ej: block partials (FP32), then the last
// block sums them in FP64 in block order.
__global__ void theta_grad_k(const float *feat, const float *w, const float *gw, int d, int64_t m, double *part,
                             unsigned *ticket, double *out)
{
    extern __shared__ float s_acc[];   // [blockDim.x / 32][d]
    __shared__ int s_last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    float acc[16];
    for (int j = 0; j < 16; ++j) acc[j] = 0.0f;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        const float a = gw[e] * w[e];
        for (int j = 0; j < d; ++j) acc[j] = fmaf(a, feat[e * d + j], acc[j]);
    }
    for (int j = 0; j < d; ++j) {
        float v = acc[j];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) s_acc[warp * d + j] = v;
    }
    __syncthreads();
    if (threadIdx.x < d) {
        float v = 0.0f;
        for (int i = 0; i < nw; ++i) v += s_acc[i * d + threadIdx.x];
        part[(int64_t)blockIdx.x * d + threadIdx.x] = (double)v;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    if (threadIdx.x < d) {
        double v = 0.0;
        for (unsigned b = 0; b < gridDim.x; ++b) v += __ldcg(&part[(int64_t)b * d + threadIdx.x]);
        out[threadIdx.x] = v;
    }
    if (threadIdx.x == 0) *ticket = 0;
}

}  // namespace

void ensure_row_ids(tpa_graph *g, cudaStream_t s)
{
    if (g->row_a.p) return;
    g->row_a.ensure((size_t)std::max<int64_t>(g->m, 1) * sizeof(int32_t), s);
    row_ids_k<<<grid_for(g->n * 32), 256, 0, s>>>(g->rp_a.as<int64_t>(), g->n, g->row_a.as<int32_t>());
    note_launch("adjoint");
    TPA_CHECK_LAUNCH();
}

void set_edge_weights(tpa_graph *g, const float *w_any, cudaStream_t s, bool drop_preprocessing)
{
    const int64_t m = g->m, n = g->n;
    g->w_a.ensure((size_t)std::max<int64_t>(m, 1) * sizeof(float), s);
    g->inv_d.ensure((size_t)n * sizeof(double), s);
    if (m) copy_in(g->w_a.p, w_any, (size_t)m * sizeof(float), s);
    ensure_perm_a2t(g, s);
    normalise_k<<<grid_for(n * 32), 256, 0, s>>>(g->rp_a.as<int64_t>(), g->w_a.as<float>(), g->perm_a2t.as<uint32_t>(),
                                                n, g->val_a.as<float>(), g->val_t.as<float>(), g->inv_d.as<double>());
    note_launch("adjoint");
    TPA_CHECK_LAUNCH();
    g->weighted = true;
    if (drop_preprocessing) g->has_pre = false;   // the stranger vector belongs to the old weights
}

void weights_from_features(const float *feat, const float *theta, int d, int64_t m, float *w, cudaStream_t s)
{
    weights_k<<<grid_for(m), 256, (size_t)d * sizeof(float), s>>>(feat, theta, d, m, w);
    note_launch("adjoint");
    TPA_CHECK_LAUNCH();
}

void theta_grad(const float *feat, const float *w, const float *gw, int d, int64_t m, double *out, cudaStream_t s)
{
    const unsigned blocks = std::min<unsigned>(grid_for(m), 1024);
    DevBuf part, tick;
    part.ensure((size_t)blocks * d * sizeof(double), s);
    tick.ensure(sizeof(unsigned), s);
    TPA_CUDA(cudaMemsetAsync(tick.p, 0, sizeof(unsigned), s));
    theta_grad_k<<<blocks, 256, (size_t)8 * d * sizeof(float), s>>>(feat, w, gw, d, m, part.as<double>(),
                                                                   tick.as<unsigned>(), out);
    note_launch("adjoint");
    TPA_CHECK_LAUNCH();
    part.release(s);
    tick.release(s);
}

// Iterates x'_0 .. x'_{K-1} of the stranger chain as the reverse sweep asks
// for them (in decreasing order).  Either all are kept (K+1 vectors of n), or
// only every C-th one is, C = ceil(sqrt(K+1)), and the C iterates of a segment
// are recomputed from its checkpoint when the sweep enters it: about
// 2 sqrt(K) vectors instead of K+1, for K extra SpMVs.  The recomputation runs
// the same deterministic kernel on the same input, so the iterates, and the
// gradient, are bit-identical either way.
struct StrangerIterates {
    tpa_graph *g = nullptr;
    int64_t n = 0;
    int K = 0, C = 0;           // C = 0: every iterate is kept
    float decay = 0.0f;
    DevBuf all, ck, seg;
    int seg_base = -1;

    // Bytes of device memory each way keeps.
    static size_t full_bytes(int64_t n, int K) { return (size_t)(K + 1) * n * sizeof(float); }
    static int stride(int K) { return (int)std::ceil(std::sqrt((double)(K + 1))); }
    static size_t checkpoint_bytes(int64_t n, int K)
    {
        const int C = stride(K);
        return ((size_t)(K / C + 1) + (size_t)C) * n * sizeof(float);
    }

    void init(tpa_graph *g_, int K_, float decay_, bool checkpoint, cudaStream_t s)
    {
        g = g_;
        n = g->n;
        K = K_;
        decay = decay_;
        if (checkpoint) {
            C = stride(K);
            ck.ensure((size_t)(K / C + 1) * n * sizeof(float), s);
            seg.ensure((size_t)C * n * sizeof(float), s);
        } else {
            all.ensure(full_bytes(n, K), s);
        }
    }
    // Buffer the forward sweep writes x'_i into (a segment slot when checkpointing).
    float *fwd_slot(int i)
    {
        if (!C) return all.as<float>() + (int64_t)i * n;
        return seg.as<float>() + (int64_t)(i % C) * n;
    }
    // After x'_i is written: keep it when it is a checkpoint.
    void fwd_done(int i, cudaStream_t s)
    {
        if (C && i % C == 0)
            TPA_CUDA(cudaMemcpyAsync(ck.as<float>() + (int64_t)(i / C) * n, fwd_slot(i), (size_t)n * sizeof(float),
                                     cudaMemcpyDeviceToDevice, s));
    }
    const float *get(int i, cudaStream_t s)
    {
        if (!C) return all.as<float>() + (int64_t)i * n;
        const int base = (i / C) * C;
        if (base != seg_base) {
            float *S0 = seg.as<float>();
            TPA_CUDA(cudaMemcpyAsync(S0, ck.as<float>() + (int64_t)(base / C) * n, (size_t)n * sizeof(float),
                                     cudaMemcpyDeviceToDevice, s));
            for (int t = 1; t < C && base + t <= K - 1; ++t)
                spmv_apply(g, 0, S0 + (int64_t)(t - 1) * n, S0 + (int64_t)t * n, 1, decay, s);
            seg_base = base;
        }
        return seg.as<float>() + (int64_t)(i - base) * n;
    }
    void release(cudaStream_t s)
    {
        all.release(s);
        ck.release(s);
        seg.release(s);
    }
};

int g_adjoint_batch = 0;   // triples per family batch (tpa_set_adjoint_batch_width; 0: the default)

int adjoint_batch_width() { return g_adjoint_batch ? g_adjoint_batch : KB_DEFAULT; }

namespace {

// The family chains of all triples in batches of KB (columns [n][KB], padding
// columns zero): forward x_1 .. x_{S-1} from c e_seed, the scores at the
// positive and negative nodes with the loss and its sigma, and (want_grad)
// the backward chain lam_{S-1} .. lam_1 with the edge products of each step
// added into GE.
template <int KB>
void family_batches(tpa_graph *g, const int32_t *seeds, const int32_t *pos, const int32_t *neg, int ntrip, int S,
                    float c, float decay, float opa, bool want_grad, DevBuf &rs, DevBuf &F, DevBuf &lamA, DevBuf &lamB,
                    DevBuf &GE, DevBuf &loss, DevBuf &sg, DevBuf &gacc, cudaStream_t s)
{
    const int64_t n = g->n, m = g->m;
    need(F, (size_t)S * n * KB * sizeof(float), "family iterates");
    need(lamA, (size_t)n * KB * sizeof(float), "family adjoint");
    need(lamB, (size_t)n * KB * sizeof(float), "family adjoint");
    float *Fp = F.as<float>();
    for (int t0 = 0; t0 < ntrip; t0 += KB) {
        const int kb = std::min(KB, ntrip - t0);
        TPA_CUDA(cudaMemsetAsync(Fp, 0, (size_t)n * KB * sizeof(float), s));
        family_init_k<KB><<<1, 32, 0, s>>>(Fp, seeds + t0, kb, c);
        for (int i = 1; i < S; ++i)
            spmv_apply(g, 0, Fp + (int64_t)(i - 1) * n * KB, Fp + (int64_t)i * n * KB, KB, decay, s);
        pair_k<KB><<<1, 32, 0, s>>>(Fp, n, S, pos + t0, neg + t0, kb, opa, rs.as<float>(), loss.as<double>() + t0,
                                    sg.as<double>() + t0, gacc.as<unsigned long long>());
        note_launch("adjoint", 2);
        if (!want_grad) continue;
        float *lam = lamA.as<float>(), *nxt = lamB.as<float>();
        TPA_CUDA(cudaMemsetAsync(lam, 0, (size_t)n * KB * sizeof(float), s));
        scatter_g_k<KB><<<1, 32, 0, s>>>(lam, pos + t0, neg + t0, sg.as<double>() + t0, kb, opa);
        for (int i = S - 1; i >= 1; --i) {
            sddmm_k<KB><<<grid_for(m), 256, 0, s>>>(g->row_a.as<int32_t>(), g->col_a.as<int32_t>(), m, lam,
                                                    Fp + (int64_t)(i - 1) * n * KB, kb, decay, GE.as<float>());
            if (i > 1) {
                spmv_apply(g, 1, lam, nxt, KB, decay, s);
                std::swap(lam, nxt);
                scatter_g_k<KB><<<1, 32, 0, s>>>(lam, pos + t0, neg + t0, sg.as<double>() + t0, kb, opa);
            }
        }
        note_launch("adjoint", 1 + 2 * (S - 1));
        TPA_CHECK_LAUNCH();
    }
}

}  // namespace

size_t g_adjoint_budget = (size_t)16 << 30;   // iterate bytes kept before checkpointing starts

// Loss and dL/dw (device float[m], CSR(A~) order; grad_w = nullptr: the loss
// only, without the reverse sweep or stored iterates).  seeds/pos/neg are
// device arrays.
double loss_grad(tpa_graph *g, const int32_t *seeds, const int32_t *pos, const int32_t *neg, int ntrip, double c,
                 int S, int T, int K, float *grad_w, cudaStream_t s)
{
    const int64_t n = g->n, m = g->m;
    const float decay = (float)(1.0 - c);
    const float opa = (float)(1.0 + alpha_of(c, S, T));
    const bool want_grad = grad_w != nullptr;
    ensure_row_ids(g, s);
    DevBuf rs, F, lamA, lamB, GE, loss, sg, gacc, Gs, two;
    StrangerIterates X;
    rs.ensure((size_t)n * sizeof(float), s);
    const int KBW = adjoint_batch_width();
    F.ensure((size_t)S * n * KBW * sizeof(float), s);
    lamA.ensure((size_t)n * KBW * sizeof(float), s);
    lamB.ensure((size_t)n * KBW * sizeof(float), s);
    loss.ensure((size_t)ntrip * sizeof(double), s);
    sg.ensure((size_t)ntrip * sizeof(double), s);
    gacc.ensure((size_t)n * sizeof(unsigned long long), s);
    TPA_CUDA(cudaMemsetAsync(gacc.p, 0, gacc.bytes, s));
    TPA_CUDA(cudaMemsetAsync(rs.p, 0, rs.bytes, s));
    if (want_grad) {
        X.init(g, K, decay, StrangerIterates::full_bytes(n, K) > g_adjoint_budget, s);
        GE.ensure((size_t)std::max<int64_t>(m, 1) * sizeof(float), s);
        Gs.ensure((size_t)n * sizeof(float), s);
        TPA_CUDA(cudaMemsetAsync(GE.p, 0, GE.bytes, s));
    } else {
        two.ensure((size_t)2 * n * sizeof(float), s);
    }

    // stranger chain, K fixed: r~_stranger = x'_T + ... + x'_K, added in
    // iteration order (the same FP32 sums whether or not iterates are kept)
    auto slot = [&](int i) { return want_grad ? X.fwd_slot(i) : two.as<float>() + (int64_t)(i & 1) * n; };
    fill_k<<<grid_for(n), 256, 0, s>>>(slot(0), n, (float)(c * (1.0 / (double)n)));
    note_launch("adjoint");
    TPA_CHECK_LAUNCH();
    if (want_grad) X.fwd_done(0, s);
    if (T == 0) axpy_k<<<grid_for(n), 256, 0, s>>>(rs.as<float>(), slot(0), n);
    for (int i = 1; i <= K; ++i) {
        spmv_apply(g, 0, slot(i - 1), slot(i), 1, decay, s);
        if (want_grad) X.fwd_done(i, s);
        if (i >= T) {
            axpy_k<<<grid_for(n), 256, 0, s>>>(rs.as<float>(), slot(i), n);
            note_launch("adjoint");
        }
    }
    TPA_CHECK_LAUNCH();

    // family chains in batches of kb triples: forward, scores, backward
    switch (adjoint_batch_width()) {
    case 16:
        family_batches<16>(g, seeds, pos, neg, ntrip, S, (float)c, decay, opa, want_grad, rs, F, lamA, lamB, GE,
                           loss, sg, gacc, s);
        break;
    case 32:
        family_batches<32>(g, seeds, pos, neg, ntrip, S, (float)c, decay, opa, want_grad, rs, F, lamA, lamB, GE,
                           loss, sg, gacc, s);
        break;
    default:
        family_batches<8>(g, seeds, pos, neg, ntrip, S, (float)c, decay, opa, want_grad, rs, F, lamA, lamB, GE,
                          loss, sg, gacc, s);
        break;
    }

    if (want_grad) {
        // stranger backward: m_K = G, m_i = [i >= T] G + P^T m_{i+1}
        gacc_to_float_k<<<grid_for(n), 256, 0, s>>>(gacc.as<unsigned long long>(), n, Gs.as<float>());
        float *mu = lamA.as<float>(), *mn = lamB.as<float>();   // [n] vectors now
        TPA_CUDA(cudaMemcpyAsync(mu, Gs.p, (size_t)n * sizeof(float), cudaMemcpyDeviceToDevice, s));
        for (int i = K; i >= 1; --i) {
            sddmm_k<1><<<grid_for(m), 256, 0, s>>>(g->row_a.as<int32_t>(), g->col_a.as<int32_t>(), m, mu,
                                                   X.get(i - 1, s), 1, decay, GE.as<float>());
            if (i > 1) {
                spmv_apply(g, 1, mu, mn, 1, decay, s);
                std::swap(mu, mn);
                if (i - 1 >= T) axpy_k<<<grid_for(n), 256, 0, s>>>(mu, Gs.as<float>(), n);
            }
        }
        note_launch("adjoint", 1 + 2 * K);
        jacobian_k<<<grid_for(n * 32), 256, 0, s>>>(g->rp_a.as<int64_t>(), GE.as<float>(), g->val_a.as<float>(),
                                                   g->inv_d.as<double>(), n, grad_w);
        note_launch("adjoint");
        TPA_CHECK_LAUNCH();
    }

    loss_sum_k<<<1, 1, 0, s>>>(loss.as<double>(), ntrip, sg.as<double>());
    note_launch("adjoint");
    TPA_CHECK_LAUNCH();
    double L = 0.0;
    TPA_CUDA(cudaMemcpyAsync(&L, sg.p, sizeof(double), cudaMemcpyDeviceToHost, s));
    TPA_CUDA(cudaStreamSynchronize(s));
    X.release(s);
    rs.release(s); F.release(s); lamA.release(s); lamB.release(s); GE.release(s);
    loss.release(s); sg.release(s); gacc.release(s); Gs.release(s); two.release(s);
    return L;
}

}  // namespace tpa
