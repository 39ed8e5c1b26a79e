/*
 * FP64 oracle for the gradient of a link-prediction loss on TPA scores with
 * respect to edge weights (supervised random walks).  TEST INFRASTRUCTURE
 * ONLY: the CUDA path never calls it and shares no code with it.
 *
 * The paper defines TPA on the row-normalised adjacency A~ (Table 1).  Here
 * A~ comes from positive edge weights: A~_uv = w_uv / d_u, d_u = sum_v w_uv.
 * With P = (1-c) A~^T, for a seed s (Algorithms 1-3, Section III-B):
 *   x_0 = c e_s, x_i = P x_{i-1},  r_family = x_0 + ... + x_{S-1}
 *   x'_0 = (c/n) 1, x'_i = P x'_{i-1},  r~_stranger = x'_T + ... + x'_K
 *   r_TPA = (1 + alpha) r_family + r~_stranger,
 *   alpha = ((1-c)^S - (1-c)^T) / (1 - (1-c)^S).
 * K, the last stranger iteration, is fixed (the forward pass's count), so the
 * loss is a smooth function of w.  Over triples (s, p, q):
 *   L = sum softplus(r_TPA^(s)[q] - r_TPA^(s)[p]).
 *
 * The gradient follows by the chain rule (not in the paper):
 *   g = dL/dr_TPA (two nonzeros per triple: sigma(z) at q, -sigma(z) at p)
 *   family:   l_{S-1} = (1+alpha) g,  l_i = (1+alpha) g + P^T l_{i+1}
 *   stranger: m_K = G,  m_i = [i >= T] G + P^T m_{i+1},  G = sum over triples of g
 *   dL/dA~_uv = (1-c) ( sum_{i=1}^{S-1} l_i[v] x_{i-1}[u] + sum_{i=1}^{K} m_i[v] x'_{i-1}[u] )
 *   dL/dw_uv  = ( dL/dA~_uv - sum_v' dL/dA~_uv' A~_uv' ) / d_u
 * Pins: central finite differences of L on w and on theta (w = exp(theta.f)),
 * and a dense-matrix forward written independently in the tests.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Planted-mistake switch for the pin-strength tests of this file (0 = none). */
static int g_adj_fault = 0;
void orc_adj_set_fault(int f) { g_adj_fault = f; }

/*
 * val_a[e] = w[e] / d_u over CSR(A~) (rows = sources), and val_t, the same
 * values in CSR(A~^T) order (rows = destinations, sources ascending).
 */
int orc_weighted_csr(int64_t n, const int64_t *rp_a, const int32_t *col_a, const double *w,
                     const int64_t *rp_t, int64_t m, double *val_a, double *val_t, int64_t *pos_t)
{
    int64_t *cur = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    if (!cur) return -1;
    for (int64_t v = 0; v < n; ++v) cur[v] = rp_t[v];
    for (int64_t u = 0; u < n; ++u) {
        double d = 0.0;
        for (int64_t e = rp_a[u]; e < rp_a[u + 1]; ++e) d += w[e];
        for (int64_t e = rp_a[u]; e < rp_a[u + 1]; ++e) {
            val_a[e] = w[e] / d;
            /* rows u arrive in ascending order, so each destination's cursor
             * walks its in-neighbours in ascending order */
            const int64_t pt = cur[col_a[e]]++;
            val_t[pt] = val_a[e];
            if (pos_t) pos_t[e] = pt;
        }
    }
    free(cur);
    (void)m;
    return 0;
}

static void prop(int64_t n, const int64_t *rp_t, const int32_t *col_t, const double *val_t, double c,
                 const double *x, double *y)
{
    for (int64_t v = 0; v < n; ++v) {
        double s = 0.0;
        for (int64_t e = rp_t[v]; e < rp_t[v + 1]; ++e) s += val_t[e] * x[col_t[e]];
        y[v] = (1.0 - c) * s;
    }
}

/* (P^T y)[u] = (1-c) sum_v A~_uv y[v], over CSR(A~) */
static void prop_t(int64_t n, const int64_t *rp_a, const int32_t *col_a, const double *val_a, double c,
                   const double *y, double *out)
{
    for (int64_t u = 0; u < n; ++u) {
        double s = 0.0;
        for (int64_t e = rp_a[u]; e < rp_a[u + 1]; ++e) s += val_a[e] * y[col_a[e]];
        out[u] = (1.0 - c) * s;
    }
}

static double softplus(double z) { return z > 0 ? z + log1p(exp(-z)) : log1p(exp(z)); }
static double sigmoid(double z) { return 1.0 / (1.0 + exp(-z)); }

static double alpha_of(double c, int64_t S, int64_t T)
{
    const double a = pow(1.0 - c, (double)S), b = pow(1.0 - c, (double)T);
    return (a - b) / (1.0 - a);
}

/*
 * Loss and (if grad_w is not NULL) dL/dw in CSR(A~) order.  w in CSR(A~)
 * order.  Returns the loss, or NAN on bad input.
 */
double orc_adjoint_grad(int64_t n, int64_t m, const int64_t *rp_a, const int32_t *col_a, const int64_t *rp_t,
                        const int32_t *col_t, const double *w, double c, int64_t S, int64_t T, int64_t K,
                        int64_t ntrip, const int32_t *seeds, const int32_t *pos, const int32_t *neg,
                        double *grad_w, double *r_out, double *stranger_out, double *val_a_out)
{
    if (n < 1 || S < 1 || T < S || K < T || !(c > 0 && c < 1)) return NAN;
    double *val_a = (double *)malloc((size_t)(m > 0 ? m : 1) * sizeof(double));
    double *val_t = (double *)malloc((size_t)(m > 0 ? m : 1) * sizeof(double));
    double *xs = (double *)malloc((size_t)(K + 1) * (size_t)n * sizeof(double));   /* stranger iterates */
    double *xf = (double *)malloc((size_t)S * (size_t)n * sizeof(double));         /* one family */
    double *rstr = (double *)calloc((size_t)n, sizeof(double));
    double *gsum = (double *)calloc((size_t)n, sizeof(double));
    double *gA = grad_w ? (double *)calloc((size_t)(m > 0 ? m : 1), sizeof(double)) : NULL;
    double *lam = (double *)malloc((size_t)n * sizeof(double));
    double *tmp = (double *)malloc((size_t)n * sizeof(double));
    if (!val_a || !val_t || !xs || !xf || !rstr || !gsum || (grad_w && !gA) || !lam || !tmp) {
        free(val_a); free(val_t); free(xs); free(xf); free(rstr); free(gsum); free(gA); free(lam); free(tmp);
        return NAN;
    }
    orc_weighted_csr(n, rp_a, col_a, w, rp_t, m, val_a, val_t, NULL);
    if (val_a_out) memcpy(val_a_out, val_a, (size_t)m * sizeof(double));
    const double alpha = alpha_of(c, S, T);

    /* stranger chain, K fixed */
    for (int64_t v = 0; v < n; ++v) xs[v] = c / (double)n;
    for (int64_t i = 1; i <= K; ++i) prop(n, rp_t, col_t, val_t, c, xs + (i - 1) * n, xs + i * n);
    for (int64_t i = T; i <= K; ++i)
        for (int64_t v = 0; v < n; ++v) rstr[v] += xs[i * n + v];
    if (stranger_out) memcpy(stranger_out, rstr, (size_t)n * sizeof(double));

    double loss = 0.0;
    for (int64_t t = 0; t < ntrip; ++t) {
        const int32_t s = seeds[t];
        for (int64_t v = 0; v < n; ++v) xf[v] = 0.0;
        xf[s] = c;
        for (int64_t i = 1; i < S; ++i) prop(n, rp_t, col_t, val_t, c, xf + (i - 1) * n, xf + i * n);
        double rp = 0.0, rq = 0.0;
        for (int64_t i = 0; i < S; ++i) {
            rp += xf[i * n + pos[t]];
            rq += xf[i * n + neg[t]];
        }
        rp = (1.0 + alpha) * rp + rstr[pos[t]];
        rq = (1.0 + alpha) * rq + rstr[neg[t]];
        if (r_out) { r_out[2 * t] = rp; r_out[2 * t + 1] = rq; }
        const double z = rq - rp;
        loss += softplus(z);
        if (!gA) continue;
        const double sg = sigmoid(z);
        gsum[neg[t]] += sg;
        gsum[pos[t]] -= sg;
        /* family adjoint: l_{S-1} = (1+alpha) g, l_i = (1+alpha) g + P^T l_{i+1} */
        for (int64_t v = 0; v < n; ++v) lam[v] = 0.0;
        for (int64_t i = S - 1; i >= 1; --i) {
            if (i == S - 1) {
                for (int64_t v = 0; v < n; ++v) lam[v] = 0.0;
            } else {
                prop_t(n, rp_a, col_a, val_a, c, lam, tmp);
                memcpy(lam, tmp, (size_t)n * sizeof(double));
            }
            lam[neg[t]] += (1.0 + alpha) * sg;
            lam[pos[t]] -= (1.0 + alpha) * sg;
            /* dL/dA~_uv += (1-c) l_i[v] x_{i-1}[u] */
            for (int64_t u = 0; u < n; ++u)
                for (int64_t e = rp_a[u]; e < rp_a[u + 1]; ++e)
                    gA[e] += (1.0 - c) * lam[col_a[e]] * xf[(i - 1) * n + u];
        }
    }
    if (gA) {
        /* stranger adjoint: m_K = G, m_i = [i >= T] G + P^T m_{i+1} */
        for (int64_t i = K; i >= 1; --i) {
            if (i == K) {
                for (int64_t v = 0; v < n; ++v) lam[v] = 0.0;
            } else {
                prop_t(n, rp_a, col_a, val_a, c, lam, tmp);
                memcpy(lam, tmp, (size_t)n * sizeof(double));
            }
            if (i >= T && g_adj_fault != 2)                       /* planted: drop the direct term */
                for (int64_t v = 0; v < n; ++v) lam[v] += gsum[v];
            for (int64_t u = 0; u < n; ++u)
                for (int64_t e = rp_a[u]; e < rp_a[u + 1]; ++e)
                    gA[e] += (1.0 - c) * lam[col_a[e]] * xs[(i - 1) * n + u];
        }
        /* row-normalisation Jacobian */
        for (int64_t u = 0; u < n; ++u) {
            double d = 0.0, su = 0.0;
            for (int64_t e = rp_a[u]; e < rp_a[u + 1]; ++e) {
                d += w[e];
                su += gA[e] * val_a[e];
            }
            if (g_adj_fault == 1) su = 0.0;                       /* planted: no Jacobian term */
            for (int64_t e = rp_a[u]; e < rp_a[u + 1]; ++e) grad_w[e] = (gA[e] - su) / d;
        }
    }
    free(val_a); free(val_t); free(xs); free(xf); free(rstr); free(gsum); free(gA); free(lam); free(tmp);
    return loss;
}
