/*
 * FP64 CPU oracle for TPA (Yoon, Jung and Kang, "TPA: Fast, Scalable, and
 * Accurate Method for Approximate Random Walk with Restart on Billion Scale
 * Graphs", ICDE 2018, arXiv 1708.02574).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow reference that the
 * CUDA path is checked against.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load it; the product path never calls it
 * and shares no code with it.
 *
 * Everything is double precision and written straight from the paper's
 * definitions; the loops over rows may run on several threads (each row's
 * sum keeps its sequential order, norms are summed sequentially), which
 * changes no result:
 *   - Table 1: A~ is the row-normalised adjacency matrix (A~_uv = 1/outdeg(u)
 *     for an edge u->v of the simple graph); the propagation operator is
 *     (1-c) A~^T.
 *   - Algorithm 1 (CPI, Section II-C): x0 = c q, x_i = (1-c) A~^T x_{i-1},
 *     r = sum of x_i for s_iter <= i <= t_iter, stop once ||x_i||_1 < eps.
 *   - Algorithm 2 (preprocessing): r~_stranger = CPI(all nodes, T, inf).
 *   - Algorithm 3 (online) with the neighbour scale of Section III-B:
 *     r_TPA = r_family + alpha r_family + r~_stranger,
 *     alpha = ((1-c)^S - (1-c)^T) / (1 - (1-c)^S).
 *
 * Readings of points the paper leaves open:
 *   - Graph: self-loops are dropped and duplicate edges are kept once.
 *     Nodes without out-edges (deadends) keep an all-zero row of A~, so mass
 *     leaks there.
 *   - Algorithm 1 starts its loop at i = 1; x0 is added to r when s_iter = 0
 *     (Table 1 defines r_family as x0 + ... + x_{S-1}).
 *   - t_iter is inclusive; t_iter < 0 stands for infinity.
 *   - x_i is added before its norm is tested, and the test runs at every i.
 *   - PageRank's seed vector is q = (1/n) 1 over all n nodes.
 *
 * Parity pins (tests/test_oracle_*.py): dense LU of the RWR equation
 * (Theorem 1), closed forms on the directed cycle and the bidirectional star,
 * the L1-mass identities of Lemma 2, the error bounds of Lemmas 1 and 3 and
 * Theorem 2, the bound constants printed in Table 3, the iteration count of
 * Lemma 4, and brute-force CSR construction on tiny graphs.
 */
#include <math.h>
#include <stdint.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stdlib.h>
#include <string.h>

/* Planted-mistake switch used only by the oracle's own pin-strength tests.
 * 0 = correct oracle.  Each nonzero value plants one plausible mistake. */
static int g_fault = 0;
void orc_set_fault(int f) { g_fault = f; }
int orc_get_fault(void) { return g_fault; }

static int cmp_i32(const void *a, const void *b)
{
    const int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* Threads of the parallel loops below (0 = the OpenMP default, all cores).
 * Every parallel loop runs over independent rows and keeps each row's own
 * sums in their sequential order, so results do not depend on it. */
static int g_threads = 0;
void orc_set_threads(int t) { g_threads = t; }
static int nthreads(void)
{
#ifdef _OPENMP
    return g_threads > 0 ? g_threads : omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * Build the simple directed graph from a raw edge list and return its
 * row-normalised adjacency A~ (Table 1) in two CSR forms:
 *   CSR(A~^T): row v lists the in-neighbours u of v in ascending order,
 *              value 1/outdeg(u)                 (rp_t, col_t, val_t)
 *   CSR(A~):   row u lists the out-neighbours v of u in ascending order,
 *              value 1/outdeg(u)                 (rp_a, col_a, val_a)
 * plus outdeg[u].  Arrays sized for m_in entries; any output may be NULL
 * (CSR(A~) is built only when rp_a is given).  The edges are bucketed by
 * destination (counting sort), each bucket is sorted and its duplicates
 * dropped; CSR(A~) is then a counting sort of CSR(A~^T) by source, which
 * keeps each row's destinations ascending.
 * Returns the number m of distinct non-self-loop edges, or -1.
 */
int64_t orc_build(int64_t n, int64_t m_in, const int32_t *src, const int32_t *dst,
                  int64_t *rp_t, int32_t *col_t, double *val_t,
                  int64_t *rp_a, int32_t *col_a, double *val_a, int32_t *outdeg)
{
    int64_t *off = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    int64_t *len = (int64_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(int64_t));
    int32_t *deg = (int32_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(int32_t));
    if (!off || !len || !deg) { free(off); free(len); free(deg); return -1; }
    /* bucket the sources of the non-self-loop edges by destination */
    for (int64_t e = 0; e < m_in; ++e) {
        if (src[e] < 0 || src[e] >= n || dst[e] < 0 || dst[e] >= n) { free(off); free(len); free(deg); return -1; }
        if (src[e] != dst[e]) off[dst[e] + 1]++;
    }
    for (int64_t v = 0; v < n; ++v) off[v + 1] += off[v];
    const int64_t k = off[n];
    int32_t *bucket = (int32_t *)malloc((size_t)(k > 0 ? k : 1) * sizeof(int32_t));
    int64_t *fill = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    if (!bucket || !fill) { free(off); free(len); free(deg); free(bucket); free(fill); return -1; }
    memcpy(fill, off, (size_t)n * sizeof(int64_t));
    for (int64_t e = 0; e < m_in; ++e)
        if (src[e] != dst[e]) bucket[fill[dst[e]]++] = src[e];
    free(fill);
    /* sort each bucket and keep its distinct sources at its front */
#pragma omp parallel for schedule(dynamic, 1024) num_threads(nthreads())
    for (int64_t v = 0; v < n; ++v) {
        int32_t *b = bucket + off[v];
        const int64_t cnt = off[v + 1] - off[v];
        if (cnt > 1) qsort(b, (size_t)cnt, sizeof(int32_t), cmp_i32);
        int64_t u = 0;
        for (int64_t i = 0; i < cnt; ++i)
            if (i == 0 || b[i] != b[i - 1]) b[u++] = b[i];
        len[v] = u;
    }
    int64_t m = 0;
    for (int64_t v = 0; v < n; ++v) m += len[v];

    for (int64_t v = 0; v < n; ++v)
        for (int64_t i = 0; i < len[v]; ++i) deg[bucket[off[v] + i]]++;
    if (g_fault == 6) {               /* planted: normalise by in-degree */
        for (int64_t v = 0; v < n; ++v) deg[v] = (int32_t)len[v];
    }
    if (outdeg) memcpy(outdeg, deg, (size_t)n * sizeof(int32_t));

    int64_t *rpt = rp_t;
    int64_t *tmp_rp = NULL;
    if (!rpt && rp_a) {               /* CSR(A~) is built from CSR(A~^T)'s rows */
        tmp_rp = (int64_t *)malloc((size_t)(n + 1) * sizeof(int64_t));
        if (!tmp_rp) { free(off); free(len); free(deg); free(bucket); return -1; }
        rpt = tmp_rp;
    }
    if (rpt) {
        rpt[0] = 0;
        for (int64_t v = 0; v < n; ++v) rpt[v + 1] = rpt[v] + len[v];
    }
    if (rp_t) {
#pragma omp parallel for schedule(dynamic, 1024) num_threads(nthreads())
        for (int64_t v = 0; v < n; ++v)
            for (int64_t i = 0; i < len[v]; ++i) {
                const int32_t u = bucket[off[v] + i];
                if (col_t) col_t[rp_t[v] + i] = u;
                if (val_t) val_t[rp_t[v] + i] = deg[u] > 0 ? 1.0 / (double)deg[u] : 0.0;
            }
    }
    if (rp_a) {
        /* counting sort of the edges by source; rows v are visited in
         * ascending order, so each source's destinations come out ascending */
        memset(rp_a, 0, (size_t)(n + 1) * sizeof(int64_t));
        for (int64_t v = 0; v < n; ++v)
            for (int64_t i = 0; i < len[v]; ++i) rp_a[bucket[off[v] + i] + 1]++;
        for (int64_t u = 0; u < n; ++u) rp_a[u + 1] += rp_a[u];
        int64_t *pos = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
        if (!pos) { free(off); free(len); free(deg); free(bucket); free(tmp_rp); return -1; }
        memcpy(pos, rp_a, (size_t)n * sizeof(int64_t));
        for (int64_t v = 0; v < n; ++v)
            for (int64_t i = 0; i < len[v]; ++i) {
                const int32_t u = bucket[off[v] + i];
                const int64_t at = pos[u]++;
                if (col_a) col_a[at] = (int32_t)v;
                if (val_a) val_a[at] = deg[u] > 0 ? 1.0 / (double)deg[u] : 0.0;
            }
        free(pos);
    }
    free(tmp_rp);
    free(off);
    free(len);
    free(deg);
    free(bucket);
    return m;
}

/* One propagation step of Algorithm 1: y = (1-c) (A~^T x), with A~^T given
 * in CSR (row v = in-neighbours of v). */
static void propagate(int64_t n, const int64_t *rp, const int32_t *col, const double *val,
                      double c, const double *x, double *y)
{
    const double decay = (g_fault == 3) ? 1.0 : (1.0 - c);   /* planted: no decay */
    if (g_fault == 1) {                                       /* planted: A~ instead of A~^T */
        for (int64_t v = 0; v < n; ++v) y[v] = 0.0;
        for (int64_t v = 0; v < n; ++v)
            for (int64_t e = rp[v]; e < rp[v + 1]; ++e) y[col[e]] += val[e] * x[v];
        for (int64_t v = 0; v < n; ++v) y[v] *= decay;
        return;
    }
#pragma omp parallel for schedule(dynamic, 4096) num_threads(nthreads())
    for (int64_t v = 0; v < n; ++v) {
        double s = 0.0;
        for (int64_t e = rp[v]; e < rp[v + 1]; ++e) s += val[e] * x[col[e]];
        y[v] = decay * s;
    }
}

/*
 * Algorithm 1 (CPI).  q is the seed vector (length n).  Returns r in `r`
 * and the last iteration index i that was computed (0 if the loop never
 * ran).  norms[i-1] receives ||x_i||_1 for i = 1..min(iters, norms_cap).
 * t_iter < 0 means no terminal iteration.  Returns -1 on bad input.
 */
int64_t orc_cpi(int64_t n, const int64_t *rp, const int32_t *col, const double *val,
                const double *q, double c, double eps, int64_t s_iter, int64_t t_iter,
                double *r, double *norms, int64_t norms_cap)
{
    if (n <= 0 || !(c > 0.0 && c < 1.0) || s_iter < 0) return -1;
    double *x = (double *)malloc((size_t)n * sizeof(double));
    double *y = (double *)malloc((size_t)n * sizeof(double));
    if (!x || !y) { free(x); free(y); return -1; }

    for (int64_t v = 0; v < n; ++v) { x[v] = c * q[v]; r[v] = 0.0; }
    if (s_iter == 0 && g_fault != 2)                          /* planted: drop x0 */
        for (int64_t v = 0; v < n; ++v) r[v] += x[v];

    const int64_t hard_cap = 100000;                          /* guards c ~ 0 */
    const int64_t last = (g_fault == 5 && t_iter > 0) ? t_iter - 1 : t_iter;  /* planted: exclusive t_iter */
    int64_t i;
    for (i = 1; (last < 0 || i <= last) && i <= hard_cap; ++i) {
        propagate(n, rp, col, val, c, x, y);
        double norm = 0.0;
        for (int64_t v = 0; v < n; ++v) norm += fabs(y[v]);
        if (g_fault == 7 && norm < eps) break;                /* planted: test before adding */
        if (i >= s_iter)
            for (int64_t v = 0; v < n; ++v) r[v] += y[v];
        if (norms && i <= norms_cap) norms[i - 1] = norm;
        double *t = x; x = y; y = t;
        if (norm < eps) break;
    }
    if (last >= 0 && i > last) i = last;   /* loop ran to its terminal iteration */
    free(x);
    free(y);
    return i;
}

/* Neighbour-approximation scale of Section III-B (closed form from Lemma 2). */
double orc_alpha(double c, int64_t S, int64_t T)
{
    const double a = pow(1.0 - c, (double)S), b = pow(1.0 - c, (double)T);
    if (g_fault == 4) return (b - a) / (1.0 - a);             /* planted: sign flip */
    return (a - b) / (1.0 - a);
}

/* Algorithm 2: PageRank CPI from q = (1/n) 1, keeping iterations T.. . */
int64_t orc_preprocess(int64_t n, const int64_t *rp, const int32_t *col, const double *val,
                       double c, double eps, int64_t T, double *r_stranger)
{
    double *q = (double *)malloc((size_t)n * sizeof(double));
    if (!q) return -1;
    const double w = (g_fault == 8) ? 1.0 : 1.0 / (double)n;  /* planted: unnormalised q */
    for (int64_t v = 0; v < n; ++v) q[v] = w;
    const int64_t it = orc_cpi(n, rp, col, val, q, c, eps, T, -1, r_stranger, NULL, 0);
    free(q);
    return it;
}

/* Algorithm 3 for one seed s: r_family from iterations 0..S-1, then
 * r_TPA = r_family + alpha r_family + r~_stranger.  If fam_out is not NULL
 * it receives r_family.  Returns the CPI iteration count or -1. */
int64_t orc_query(int64_t n, const int64_t *rp, const int32_t *col, const double *val,
                  double c, double eps, int64_t S, int64_t T, int32_t s,
                  const double *r_stranger, double *out, double *fam_out)
{
    if (s < 0 || s >= n || S < 1 || T < S) return -1;
    double *q = (double *)calloc((size_t)n, sizeof(double));
    double *fam = (double *)malloc((size_t)n * sizeof(double));
    if (!q || !fam) { free(q); free(fam); return -1; }
    q[s] = 1.0;
    const int64_t it = orc_cpi(n, rp, col, val, q, c, eps, 0, S - 1, fam, NULL, 0);
    const double alpha = orc_alpha(c, S, T);
    for (int64_t v = 0; v < n; ++v) {
        const double nb = alpha * fam[v];
        out[v] = fam[v] + nb + r_stranger[v];
    }
    if (fam_out) memcpy(fam_out, fam, (size_t)n * sizeof(double));
    free(q);
    free(fam);
    return it;
}

/* Algorithm 3 for a seed set (the seed vector of Algorithm 1 with
 * q_s = 1/|S| for s in S, Section II-C): members[0..len) lists the set, a
 * node listed twice counting twice.  r_family from iterations 0..S-1 of CPI
 * from that q, then r_TPA = r_family + alpha r_family + r~_stranger.
 * Returns the CPI iteration count or -1. */
int64_t orc_query_set(int64_t n, const int64_t *rp, const int32_t *col, const double *val,
                      double c, double eps, int64_t S, int64_t T, int64_t len, const int32_t *members,
                      const double *r_stranger, double *out)
{
    if (len < 1 || S < 1 || T < S) return -1;
    for (int64_t j = 0; j < len; ++j)
        if (members[j] < 0 || members[j] >= n) return -1;
    double *q = (double *)calloc((size_t)n, sizeof(double));
    double *fam = (double *)malloc((size_t)n * sizeof(double));
    if (!q || !fam) { free(q); free(fam); return -1; }
    const double w = (g_fault == 9) ? 1.0 : 1.0 / (double)len;   /* planted: unnormalised q */
    for (int64_t j = 0; j < len; ++j) q[members[j]] += w;
    const int64_t it = orc_cpi(n, rp, col, val, q, c, eps, 0, S - 1, fam, NULL, 0);
    const double alpha = orc_alpha(c, S, T);
    for (int64_t v = 0; v < n; ++v) out[v] = fam[v] + alpha * fam[v] + r_stranger[v];
    free(q);
    free(fam);
    return it;
}

/* Exact RWR by CPI (Algorithm 1 with s_iter = 0 and no terminal iteration). */
int64_t orc_cpi_exact(int64_t n, const int64_t *rp, const int32_t *col, const double *val,
                      double c, double eps, int32_t s, double *out)
{
    if (s < 0 || s >= n) return -1;
    double *q = (double *)calloc((size_t)n, sizeof(double));
    if (!q) return -1;
    q[s] = 1.0;
    const int64_t it = orc_cpi(n, rp, col, val, q, c, eps, 0, -1, out, NULL, 0);
    free(q);
    return it;
}
