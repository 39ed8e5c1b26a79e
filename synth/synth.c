/*
 * Seeded synthetic inputs: R-MAT edge lists, query seeds, batch sizes,
 * edge features, parameter vectors and link-prediction triples.
 *
 * This module is shared by the FP64 oracle and by the CUDA path.  It holds
 * none of the method's arithmetic (no normalisation, no propagation): it only
 * draws random numbers and turns them into integer ids or N(0,1) samples.
 *
 * Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast
 * splittable pseudorandom number generators", OOPSLA 2014) used as a
 * counter-based generator: the value for counter i under stream key s is the
 * SplitMix64 output after i+1 increments of the golden gamma starting at s.
 * A uniform double in [0,1) takes the top 53 bits.
 *
 * R-MAT (Chakrabarti, Zhan and Faloutsos, SDM 2004): every edge e chooses,
 * for each of `scale` levels from the most significant bit down, one of four
 * quadrants with probabilities (a, b, c, d).  Quadrant a sets (src bit, dst
 * bit) = (0,0), b = (0,1), c = (1,0), d = (1,1).  The uniform for edge e at
 * level l uses counter e*scale + l.  No vertex permutation is applied.
 *
 * Host C only (builds on x86-64 and aarch64 alike); work is split across
 * POSIX threads by edge ranges, so the output does not depend on the thread
 * count.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static inline uint64_t sm64(uint64_t key, uint64_t ctr)
{
    uint64_t z = key + (ctr + 1u) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static inline double u01(uint64_t key, uint64_t ctr)
{
    return (double)(sm64(key, ctr) >> 11) * 0x1.0p-53;
}

uint64_t synth_splitmix64(uint64_t key, uint64_t ctr) { return sm64(key, ctr); }
double synth_uniform(uint64_t key, uint64_t ctr) { return u01(key, ctr); }

typedef struct {
    int scale;
    int64_t e0, e1;
    double ta, tab, tabc;
    uint64_t key;
    int32_t *src, *dst;
} rmat_job;

static void *rmat_worker(void *arg)
{
    rmat_job *j = (rmat_job *)arg;
    const int L = j->scale;
    for (int64_t e = j->e0; e < j->e1; ++e) {
        uint32_t s = 0, d = 0;
        const uint64_t base = (uint64_t)e * (uint64_t)L;
        for (int l = 0; l < L; ++l) {
            const double u = u01(j->key, base + (uint64_t)l);
            uint32_t sb, db;
            if (u < j->ta) { sb = 0; db = 0; }
            else if (u < j->tab) { sb = 0; db = 1; }
            else if (u < j->tabc) { sb = 1; db = 0; }
            else { sb = 1; db = 1; }
            s = (s << 1) | sb;
            d = (d << 1) | db;
        }
        j->src[e] = (int32_t)s;
        j->dst[e] = (int32_t)d;
    }
    return NULL;
}

/* Generate m R-MAT edges over 2^scale nodes.  Returns 0 on success. */
int synth_rmat(int scale, int64_t m, double a, double b, double c, uint64_t key,
               int32_t *src, int32_t *dst, int nthreads)
{
    if (scale < 1 || scale > 30 || m < 0 || !src || !dst) return -1;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if ((int64_t)nthreads > m) nthreads = m > 0 ? (int)m : 1;
    rmat_job jobs[256];
    pthread_t th[256];
    const double ta = a, tab = a + b, tabc = a + b + c;
    for (int t = 0; t < nthreads; ++t) {
        jobs[t].scale = scale;
        jobs[t].e0 = m * t / nthreads;
        jobs[t].e1 = m * (t + 1) / nthreads;
        jobs[t].ta = ta; jobs[t].tab = tab; jobs[t].tabc = tabc;
        jobs[t].key = key; jobs[t].src = src; jobs[t].dst = dst;
    }
    for (int t = 1; t < nthreads; ++t)
        if (pthread_create(&th[t], NULL, rmat_worker, &jobs[t]) != 0) {
            rmat_worker(&jobs[t]); th[t] = 0;
        }
    rmat_worker(&jobs[0]);
    for (int t = 1; t < nthreads; ++t)
        if (th[t]) pthread_join(th[t], NULL);
    return 0;
}

/* Planted-partition graph: n nodes in `blocks` equal contiguous blocks
 * (block of v = v * blocks / n), m directed edges.  Edge e draws its source
 * uniformly over all nodes and, with probability p_in, its destination
 * uniformly inside the source's block, else uniformly over all nodes.
 * Counter-based: edge e uses counters 3e, 3e+1, 3e+2 of `key`.
 * Returns -1 on bad arguments. */
int synth_planted(int64_t n, int64_t m, int64_t blocks, double p_in, uint64_t key, int32_t *src, int32_t *dst)
{
    if (n < 1 || n > ((int64_t)1 << 31) - 1 || m < 0 || blocks < 1 || blocks > n || !(p_in >= 0.0 && p_in <= 1.0) ||
        !src || !dst)
        return -1;
    for (int64_t e = 0; e < m; ++e) {
        const uint64_t c = 3 * (uint64_t)e;
        int64_t s = (int64_t)(u01(key, c) * (double)n);
        if (s >= n) s = n - 1;
        int64_t d;
        if (u01(key, c + 1) < p_in) {
            const int64_t b = s * blocks / n;
            const int64_t lo = (b * n + blocks - 1) / blocks, hi = ((b + 1) * n + blocks - 1) / blocks;
            d = lo + (int64_t)(u01(key, c + 2) * (double)(hi - lo));
            if (d >= hi) d = hi - 1;
        } else {
            d = (int64_t)(u01(key, c + 2) * (double)n);
            if (d >= n) d = n - 1;
        }
        src[e] = (int32_t)s;
        dst[e] = (int32_t)d;
    }
    return 0;
}

/* Mark nodes with at least one out-edge to another node (not a self-loop).
 * flag must hold n bytes; it is overwritten. */
void synth_has_out_edge(int64_t n, int64_t m, const int32_t *src, const int32_t *dst, uint8_t *flag)
{
    memset(flag, 0, (size_t)n);
    for (int64_t e = 0; e < m; ++e)
        if (src[e] != dst[e]) flag[src[e]] = 1;
}

/* Draw `count` ids uniformly (with replacement) from cand[0..ncand). */
void synth_pick_uniform(int64_t ncand, const int32_t *cand, int64_t count, uint64_t key, int32_t *out)
{
    for (int64_t i = 0; i < count; ++i) {
        int64_t j = (int64_t)(u01(key, (uint64_t)i) * (double)ncand);
        if (j >= ncand) j = ncand - 1;
        out[i] = cand[j];
    }
}

/* Standard normal samples by the Box-Muller transform: sample i uses the two
 * uniforms at counters 2i and 2i+1 (the first mapped to (0,1]). */
void synth_normal(int64_t count, uint64_t key, double mean, double sd, float *out)
{
    const double two_pi = 6.283185307179586476925286766559;
    for (int64_t i = 0; i < count; ++i) {
        const double u1 = 1.0 - u01(key, 2u * (uint64_t)i);
        const double u2 = u01(key, 2u * (uint64_t)i + 1u);
        out[i] = (float)(mean + sd * sqrt(-2.0 * log(u1)) * cos(two_pi * u2));
    }
}

/* Triples (seed, pos, neg) for link prediction: seed uniform over the ids in
 * cand, pos the head of a uniformly chosen non-self-loop out-edge of the seed
 * in the raw edge list, neg a uniform node.  Out-edges are grouped by a
 * counting pass over the raw list.  Returns 0 on success. */
int synth_triples(int64_t n, int64_t m, const int32_t *src, const int32_t *dst,
                  int64_t ncand, const int32_t *cand, int64_t count, uint64_t key,
                  int32_t *seed, int32_t *pos, int32_t *neg)
{
    int64_t *start = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    if (!start) return -1;
    for (int64_t e = 0; e < m; ++e)
        if (src[e] != dst[e]) start[src[e] + 1]++;
    for (int64_t v = 0; v < n; ++v) start[v + 1] += start[v];
    int32_t *heads = (int32_t *)malloc((size_t)(start[n] > 0 ? start[n] : 1) * sizeof(int32_t));
    int64_t *fill = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    if (!heads || !fill) { free(start); free(heads); free(fill); return -1; }
    memcpy(fill, start, (size_t)n * sizeof(int64_t));
    for (int64_t e = 0; e < m; ++e)
        if (src[e] != dst[e]) heads[fill[src[e]]++] = dst[e];
    for (int64_t i = 0; i < count; ++i) {
        int64_t j = (int64_t)(u01(key, 3u * (uint64_t)i) * (double)ncand);
        if (j >= ncand) j = ncand - 1;
        const int32_t s = cand[j];
        const int64_t deg = start[s + 1] - start[s];
        int64_t k = deg > 0 ? (int64_t)(u01(key, 3u * (uint64_t)i + 1u) * (double)deg) : 0;
        if (k >= deg) k = deg - 1;
        int64_t v = (int64_t)(u01(key, 3u * (uint64_t)i + 2u) * (double)n);
        if (v >= n) v = n - 1;
        seed[i] = s;
        pos[i] = deg > 0 ? heads[start[s] + k] : s;
        neg[i] = (int32_t)v;
    }
    free(start); free(heads); free(fill);
    return 0;
}
