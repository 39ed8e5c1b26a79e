/*
 * tpa.h -- C ABI of libtpa, a GB300 (sm_103a) implementation of the
 * data-parallel hot path of TPA (Yoon, Jung and Kang, "TPA: Fast, Scalable,
 * and Accurate Method for Approximate Random Walk with Restart on Billion
 * Scale Graphs", arXiv 1708.02574).
 *
 * Notation (Table 1): n nodes, m edges, c restart probability, eps
 * convergence tolerance, A~ the row-normalised adjacency matrix, S and T the
 * first iterations of the neighbour and stranger parts.
 *
 * Conventions shared by every entry point
 *   - Pointers may be host or device memory; the kind is detected with
 *     cudaPointerGetAttributes.  Inputs are copied; the caller keeps
 *     ownership of every array it passes.  Outputs are written into
 *     caller-provided buffers.  When an output is in host memory the call
 *     returns after the data has arrived; otherwise it is stream-ordered.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  All device
 *     work of a call is issued on that stream.
 *   - Calls on one tpa_graph must not overlap (the graph owns one workspace);
 *     different graphs are independent.
 *   - Every call returns a tpa_status and never aborts.  On failure,
 *     tpa_last_error() returns a message for the calling thread.
 *   - Score vectors are float32, laid out node-major: out[v * k + j] is the
 *     score of node v for seed j.
 */
#ifndef TPA_H
#define TPA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tpa_graph tpa_graph;

typedef enum {
    TPA_OK = 0,
    TPA_EINVAL = 1,    /* argument out of range (ids, sizes, c, S, T, eps) */
    TPA_ENOMEM = 2,    /* device or host allocation failed */
    TPA_ECUDA = 3,     /* a CUDA call failed (message in tpa_last_error) */
    TPA_ESTATE = 4,    /* call out of order, e.g. tpa_query before tpa_preprocess */
    TPA_ETIMEOUT = 5   /* a bounded device wait gave up */
} tpa_status;

/* Message for the last failed call on this thread ("" if none). */
const char *tpa_last_error(void);

/*
 * Build the row-normalised adjacency A~ of Table 1 from a raw edge list
 * (src[e] -> dst[e], 0 <= id < n, m_edges entries, int32).  Self-loops are
 * dropped and duplicate edges are kept once; A~_uv = 1/outdeg(u) rounded to
 * float32, and nodes without out-edges keep an all-zero row.  The graph
 * holds CSR(A~^T) (rows = destinations, sources ascending) for the pull
 * products of Algorithm 1 and CSR(A~) (rows = sources) for the push step
 * and the adjoint, both on the device of `stream`.
 * The build is unweighted; a weighted graph takes a second call,
 * tpa_set_edge_weights (weights in CSR(A~) edge order, after duplicates
 * are merged, so a weight belongs to one distinct edge).
 * Errors: TPA_EINVAL for n < 1, n >= 2^31, m_edges < 0, an id out of range;
 * TPA_ENOMEM, TPA_ECUDA.  *out is set only on success.
 */
tpa_status tpa_build_graph(int64_t n, int64_t m_edges, const int32_t *src, const int32_t *dst,
                           void *stream, tpa_graph **out);

/* Release a graph and all device memory it owns.  NULL is ignored. */
void tpa_free_graph(tpa_graph *g);

/* Number of nodes and of distinct non-self-loop edges. */
tpa_status tpa_graph_info(const tpa_graph *g, int64_t *n, int64_t *m);

/*
 * Copy one CSR of the graph out: which = 0 for A~^T, 1 for A~.
 * row_ptr holds n+1 int64, col m int32, val m float32; any may be NULL.
 */
tpa_status tpa_get_csr(const tpa_graph *g, int which, int64_t *row_ptr, int32_t *col,
                       float *val, void *stream);

/*
 * Algorithm 2 (preprocessing phase): PageRank by CPI from x0 = (c/n) 1,
 * keeping the sum of iterations i >= T until ||x_i||_1 < eps.  The result
 * r~_stranger (float32[n]) stays resident in the graph together with c, T
 * and eps.  Requires 0 < c < 1, T >= 1, eps > 0.
 */
tpa_status tpa_preprocess(tpa_graph *g, double c, int T, double eps, void *stream);

/* Copy r~_stranger out (float32[n]) and the CPI iteration count. */
tpa_status tpa_get_stranger(const tpa_graph *g, float *out, int64_t *iters, void *stream);

/*
 * Algorithm 3 (online phase) for k independent single-seed queries:
 * for each seed s_j, r_family = x0 + ... + x_{S-1} by CPI from x0 = c e_s
 * (with the preprocessing eps), then
 *   r_TPA = (1 + alpha) r_family + r~_stranger,
 *   alpha = ((1-c)^S - (1-c)^T) / (1 - (1-c)^S)   (Section III-B),
 * using the c and T of tpa_preprocess.  out is float32[n * k], node-major.
 * Seeds run in chunks (tpa_set_batch_width).  With out in device memory (or
 * host memory that is not page-locked), seeds with more out-edges than the
 * push branch takes (256) are swapped into the last chunks of the query, so
 * that the other chunks push x1 and x2, and the swapped columns are put back
 * at the end; results then agree with unmoved seeds to FP32 rounding.
 * With out in page-locked host memory and k >= 2w (w = 128 columns where
 * two device buffers of n x 128 floats fit in 8 GiB, else 64 where those
 * fit; see tpa_set_output_group_width), the seeds run in column groups of w:
 * each group is computed into one of two device buffers (n x w floats
 * each), with the swap above inside the group, and copied to out by the copy
 * engine while the next group computes.  Otherwise the kernels write the
 * scores into page-locked memory directly (no swap) when its rows are
 * 16-byte aligned (k a multiple of 4), else the scores are staged in device
 * memory and copied once.  Host outputs are complete when the call returns.
 * Requires 1 <= S <= T, k >= 1, 0 <= seeds[j] < n.
 * Errors: TPA_ESTATE before tpa_preprocess; TPA_EINVAL.
 */
tpa_status tpa_query(tpa_graph *g, const int32_t *seeds, int k, int S, float *out, void *stream);

/*
 * Algorithm 3 for nsets seed sets (personalised PageRank with the seed vector
 * q_s = 1/|S| of Section II-C): column j starts from x0 = c q_j with
 * q_j = 1/|S_j| on each member of set j, members[set_ptr[j] .. set_ptr[j+1])
 * (a node listed twice counts twice), then r_TPA as for tpa_query.  By
 * linearity each column equals the mean of its members' single-seed TPA
 * vectors.  set_ptr: int64[nsets + 1], set_ptr[0] = 0, strictly increasing
 * (no empty set); members: int32, 0 <= id < n; both host or device.  out:
 * device float32[n * nsets], node-major.  The first two iterations are pulled
 * (the push path starts from single seeds).
 * Errors: TPA_ESTATE before tpa_preprocess; TPA_EINVAL.
 */
tpa_status tpa_query_sets(tpa_graph *g, const int64_t *set_ptr, const int32_t *members, int nsets, int S,
                          float *out, void *stream);

/*
 * Algorithm 1 (CPI) for k single-seed vectors q = e_{s_j}: returns
 * r_j = sum of x_i for s_iter <= i <= t_iter (t_iter < 0: no limit), each
 * column stopping after the first i with ||x_i||_1 < eps.  out is
 * float32[n * k], node-major; iters (int32[k], may be NULL) receives the
 * last iteration computed for each column.
 */
tpa_status tpa_cpi(tpa_graph *g, const int32_t *seeds, int k, double c, double eps, int s_iter,
                   int t_iter, float *out, int32_t *iters, void *stream);

/*
 * Wait for the graph's work on `stream` and report whether a bounded device
 * wait of its kernels gave up since the last check (TPA_ETIMEOUT; the
 * results of those calls are not valid).  The SpMV/SpMM of a CPI iteration
 * finishes rows that span tiles by waiting, with a limit of about a second,
 * for the partial sums of earlier tiles; calls that synchronise anyway
 * (host outputs, tpa_preprocess) check by themselves.
 */
tpa_status tpa_sync(tpa_graph *g, void *stream);

/* Exact RWR by CPI for one seed (Algorithm 1 with s_iter = 0, t_iter = inf). */
tpa_status tpa_cpi_exact(tpa_graph *g, int32_t seed, double c, double eps, float *out,
                         int32_t *iters, void *stream);

/*
 * Save / load the preprocessed data (Theorem 4: O(n) floats) as a binary
 * file: magic, n, m, c, T, eps, iteration count, then float32[n].  Loading
 * checks that n and m match the graph.
 */
tpa_status tpa_save_preprocessed(const tpa_graph *g, const char *path);
tpa_status tpa_load_preprocessed(tpa_graph *g, const char *path, void *stream);

/*
 * One propagation step of CPI for a single vector that allocates nothing.
 * The paper has no counterpart: this is an extra entry point for callers that
 * cannot allocate device memory when they want a step -- for example a
 * serving process whose GPU memory is all reserved by another allocator, or a
 * latency-critical loop that must avoid cudaMalloc/cudaFree and the
 * synchronisation they imply.
 *
 * Computes y = (1-c) A~^T x over the caller's CSR of A~^T (row_ptr int64[n+1],
 * col int32[m], val float32[m]; rows = destinations), adds y into r when r is
 * not NULL, and writes ||y||_1 (FP64) to l1[0] when l1 is not NULL.  Every
 * array must be device memory; the call is stream-ordered on `stream`.
 * The CSR is not validated on the device: row_ptr[0] = 0, row_ptr[n] = m,
 * row_ptr non-decreasing and 0 <= col[e] < n are the caller's to guarantee
 * (an id out of range makes the step read out of bounds).  x, y and r must
 * be three distinct arrays (TPA_EINVAL otherwise): the step is not in place.
 *
 * Scratch lives in a file-scope device array of TPA_NOALLOC_SCRATCH_BYTES
 * (16 MiB) that every GPU loading the library holds until the process exits.
 * Its layout takes 32 bytes per merge-path tile of 256 steps plus about
 * 10 KB, so it fits graphs with n + m up to about 134 million (TPA_EINVAL
 * beyond, with the needed size in tpa_last_error).  The first call on each device looks up
 * the array's device address (cudaGetSymbolAddress); make that first call
 * before any stream capture.  All calls share the one array, so calls whose
 * GPU work overlaps (other streams, other threads) race and give wrong
 * results; serialise them.  Each call clears the counters it needs before use.
 */
#define TPA_NOALLOC_SCRATCH_BYTES ((size_t)16 << 20)
tpa_status tpa_cpi_step_noalloc(int64_t n, int64_t m, const int64_t *row_ptr, const int32_t *col,
                                const float *val, double c, const float *x, float *y, float *r,
                                double *l1, void *stream);

/* ------------------------------------------------------ differentiation ---
 * Not part of the paper's method: gradients of a link-prediction loss on TPA
 * scores with respect to positive edge weights (supervised random walks).
 * With weights w, A~_uv = w_uv / sum_v' w_uv'. */

/* Use weights w (float32[m], device or host, in CSR(A~) edge order as
 * returned by tpa_get_csr(g, 1, ...)).  Recomputes A~ in both CSR orders;
 * the previous preprocessing result is dropped (TPA_ESTATE until
 * tpa_preprocess runs again).  The first call on a graph also builds, and
 * keeps, the map from CSR(A~) edges to their CSR(A~^T) positions (uint32[m],
 * allocated on `stream`). */
tpa_status tpa_set_edge_weights(tpa_graph *g, const float *w, void *stream);

/* w_e = exp(theta . f_e) for m edges with d <= 16 features (feat row-major
 * [m][d]); all arrays device memory. */
tpa_status tpa_edge_weights(const float *feat, const float *theta, int d, int64_t m, float *w, void *stream);

/*
 * Bytes of stranger-chain iterates the reverse sweep of tpa_loss_grad keeps
 * (default 16 GiB).  When the K+1 iterates of n floats need more, only every
 * C-th one is kept, C = ceil(sqrt(K+1)), and each segment of C iterates is
 * recomputed from its checkpoint when the sweep reaches it (about 2 sqrt(K)
 * vectors instead of K+1, for K more SpMVs); the gradient is bit-identical.
 */
tpa_status tpa_set_adjoint_budget(uint64_t bytes);

/* Triples per family batch of tpa_loss_grad: the forward and reverse family
 * chains of `width` triples run as one [n][width] SpMM per step (8, 16 or
 * 32; 0 restores the default).  Wider batches stream the CSR fewer times per
 * triple.  The gradient differs between widths only by FP32 rounding.
 * TPA_EINVAL for another value; the getter returns the width in effect. */
tpa_status tpa_set_adjoint_batch_width(int width);
int tpa_get_adjoint_batch_width(void);

/*
 * L = sum over ntrip triples (s, p, q) of softplus(r[q] - r[p]), where
 * r = (1+alpha) r_family(s) + r~_stranger follows Algorithms 2-3 on the
 * current weights with the stranger chain run for exactly K >= T iterations
 * (take K from tpa_get_stranger after tpa_preprocess on the same weights so
 * the loss matches the served scores).  Writes L to *loss (host) and
 * dL/dw (float32[m], CSR(A~) order, device or host) to grad_w, computed by the
 * adjoint recursions l_i = (1+alpha) g + P^T l_{i+1} (family, S-1 steps) and
 * m_i = [i >= T] G + P^T m_{i+1} (stranger, K steps) with P^T = (1-c) A~ and
 * the row-normalisation Jacobian.  grad_w = NULL computes the loss alone (no
 * reverse sweep, no stored iterates).  Unweighted graphs use unit weights.
 */
tpa_status tpa_loss_grad(tpa_graph *g, const int32_t *seeds, const int32_t *pos, const int32_t *neg, int ntrip,
                         double c, int S, int T, int K, double *loss, float *grad_w, void *stream);

/* dL/dtheta_j = sum_e grad_w_e w_e f_ej (FP64 out[d]); device arrays. */
tpa_status tpa_theta_grad(const float *feat, const float *w, const float *grad_w, int d, int64_t m,
                          double *grad_theta, void *stream);

/* ---------------------------------------------------- kernel tuning ---
 * Not part of the paper's method.  Process-wide settings of the SpMV/SpMM
 * that runs each CPI iteration; an autotuner times the variants on a graph
 * and keeps the fastest.  Results do not depend on the choice beyond FP32
 * rounding order. */

/* Number of compiled SpMV/SpMM variants. */
int tpa_variant_count(void);

/* Shape of variant idx: padded batch width kp (columns per CPI chunk), lanes
 * per merge-path walker, columns per lane, path steps per walker, threads per
 * CTA.  TPA_EINVAL for an index out of range. */
tpa_status tpa_variant_info(int idx, int *kp, int *lanes, int *cols_per_lane, int *items, int *threads);

/* Static name of variant idx (kernel family and template shape, e.g.
 * "pipe<2,4,16,8,4>"); NULL for an index out of range.  Owned by the
 * library, valid for the life of the process. */
const char *tpa_variant_name(int idx);

/* Index of the variant in effect for padded width kp (the forced one, else
 * the default); -1 if kp is not a power of two in [1, 256]. */
int tpa_get_variant(int kp);

/* Use variant idx for padded width kp (a power of two <= 256); idx = -1
 * restores the default.  TPA_EINVAL if the variant has another width. */
tpa_status tpa_set_variant(int kp, int idx);

/* Seeds per chunk when tpa_query gets k seeds: chunks of `width` columns run
 * one after another (a power of two <= 256; 0 restores the default, 8).  In a
 * chunk of at most 8 light seeds x1 and x2 are pushed; a narrow chunk keeps its
 * iterates X[n][width] near L2 size.  TPA_EINVAL for another value.  The
 * getter returns the width in effect. */
tpa_status tpa_set_batch_width(int width);
int tpa_get_batch_width(void);

/* The same for tpa_cpi and the many-iteration runs behind it (default 128:
 * every streamed nonzero serves more seeds). */
tpa_status tpa_set_cpi_batch_width(int width);
int tpa_get_cpi_batch_width(void);

/* Column groups of a tpa_query whose output is page-locked host memory (see
 * tpa_query): width = 0 (the default) picks 128 or 64 columns from the graph
 * size, -1 has the kernels write the host memory directly, and a multiple of
 * 8 in [8, 4096] fixes the group width (for k >= 2 x width).  TPA_EINVAL for
 * another value.  The getter returns the setting. */
tpa_status tpa_set_output_group_width(int width);
int tpa_get_output_group_width(void);

/* Direction choice in tpa_query (default on): for chunks of up to 8 seeds,
 * each with at most 256 out-edges, and S >= 4, the sparse iterates x1 and x2
 * are pushed along CSR(A~) instead of pulled over all of A~^T; results differ
 * only by FP32 rounding order.  enable = 0 pulls every iteration. */
tpa_status tpa_set_push(int enable);

/* Pattern-only products (default on) for unweighted graphs: every edge out of
 * node u carries the same value RN32(1/outdeg(u)), so the propagation gathers
 * x_u * RN32(1/outdeg(u)), kept scaled in the iterate buffer, instead of
 * reading the value array: 4 instead of 8 bytes per nonzero (Section III-A's
 * row-normalised A~ is unchanged).  Results differ from the valued products
 * only by FP32 rounding.  Weighted graphs always read their values.
 * enable = 0 reads the value array everywhere. */
tpa_status tpa_set_pattern(int enable);

/* The order in which tpa_query runs the k seeds of one call (with its output
 * in device memory), from their out-degrees outdeg[0..k) (host int32) and the
 * settings in effect: perm[j] (host int32[k]) is the position of the seed
 * run at place j.  Seeds with more than 256 out-edges are swapped into the
 * last places, each with a light seed from there, when some chunk can push
 * (push on, S >= 4, chunks of at most 16, more than one chunk); otherwise
 * perm is the identity.  Host only: no GPU work.  TPA_EINVAL for NULL
 * arguments or k < 1. */
tpa_status tpa_seed_order(const int32_t *outdeg, int k, int S, int32_t *perm);

/* ---------------------------------------------------- batched serving ---
 * Algorithm 3 for a stream of request batches of uneven size, with the launch
 * sequence of each kind of batch captured once in a CUDA graph and replayed.
 * Not part of the paper (its online phase answers one seed at a time).
 *
 * A server answers into one caller-owned device buffer out (float32, node-
 * major, row stride ldo >= max_k): after tpa_server_query with k seeds,
 * out[v * ldo + j] for j < k is the TPA score of node v for seeds[j].  Each
 * batch runs as tpa_query would run it: seeds of more than 256 out-edges go
 * to the last chunks, every chunk's push or pull branch for x1 and x2 is
 * chosen on the host from the seeds' out-degrees (the server keeps a host
 * copy of them, 4n bytes), and the moved columns are swapped back at the
 * end; results equal tpa_query's bit for bit.  A captured graph is keyed by
 * k and the string of chunk branches, so batches of the same size share
 * graphs whatever their seeds; at most 64 graphs are kept (least recently
 * used dropped).  A server keeps its own workspace (about 6 n * 8 floats for
 * chunks of 8 seeds) and graphs that point at it and at the graph's CSR: it
 * must be freed before the graph, and calls on one server must not overlap.
 * A change of a kernel setting (tpa_set_variant, tpa_set_batch_width,
 * tpa_set_push, tpa_set_pattern) makes the server capture again, and so does
 * a batch that needs more workspace than any before it (its buffers are
 * reallocated, and graphs captured over the old ones are dropped, never
 * replayed).  Validated with oracle parity up to R-MAT scale 24 (16.8 M
 * nodes, 8,192 seeds in uneven batches). */
typedef struct tpa_server tpa_server;

/* Create a server for queries with S family steps and at most max_k seeds
 * per batch on a preprocessed graph.  out: device buffer of n rows of ldo
 * floats, or NULL to let the server allocate one (ldo is then max_k; see
 * tpa_server_result).  Errors: TPA_ESTATE before tpa_preprocess; TPA_EINVAL
 * for S outside [1, T], max_k < 1, ldo < max_k, or a host out. */
tpa_status tpa_server_create(tpa_graph *g, int S, int max_k, float *out, int64_t ldo, void *stream,
                             tpa_server **srv);

/* Answer one batch of k <= max_k seeds (host or device int32, 0 <= id < n;
 * ids are checked on the host, so device ids cost one small copy and a wait).
 * The first batch of a kind (k and chunk branches) runs directly and its
 * sequence is captured; later batches of that kind replay it.  Work is
 * issued on stream. */
tpa_status tpa_server_query(tpa_server *srv, const int32_t *seeds, int k, void *stream);

/* The output buffer and its row stride. */
tpa_status tpa_server_result(const tpa_server *srv, float **out, int64_t *ldo);

/* Graphs held now, graph replays, kernel launches per replay of the most
 * recently used graph for batch size k (0 if none), and captures so far
 * (every batch is either a replay or a direct run followed by a capture).
 * NULL outputs are skipped. */
tpa_status tpa_server_stats(const tpa_server *srv, int k, int64_t *graphs, int64_t *replays,
                            int64_t *launches_per_replay, int64_t *captures);

/* Wait for the server's work on `stream`; TPA_ETIMEOUT when a bounded
 * device wait of its kernels gave up since the last check (see tpa_sync). */
tpa_status tpa_server_sync(tpa_server *srv, void *stream);

/* Release the server (waits for its work). */
void tpa_server_free(tpa_server *srv);

/* ------------------------------------------------------ measurement ---
 * Not part of the paper's method: launch accounting and kernel timing for
 * benchmarks.  The statistics are process-wide and thread-safe. */
typedef struct {
    char name[32];        /* kernel family, e.g. "spmm", "fixup", "sort" */
    int64_t launches;     /* launches since the last tpa_profile_reset */
    double total_ms;      /* summed CUDA-event durations (0 unless timing is on) */
    double alg_bytes;     /* algorithmic bytes of the timed launches */
} tpa_kernel_stat;

/* Number of CUDA kernel launches issued by the library since it was loaded. */
uint64_t tpa_launch_count(void);

/* Clear the per-family statistics.  With timing != 0, every SpMV/SpMM and
 * fixup launch of Algorithm 1 is bracketed by CUDA events recorded on its
 * own stream until the next reset. */
tpa_status tpa_profile_reset(int timing);

/* Read the statistics (waits for the recorded events).  Writes up to cap
 * entries to out and the number of families to *count. */
tpa_status tpa_profile_read(tpa_kernel_stat *out, int cap, int *count);

/* Milliseconds per pass of a gather-only probe over the graph's CSR(A~^T):
 * every column id read in order and the row of kp floats (1 or 8) of an
 * iterate at that column gathered, with no rows, carries or epilogue - the
 * floor the SpMV/SpMM kernels' gathers set at this column pattern.  Averaged
 * over reps passes after one warm-up, on `stream` (synchronises it).  Uses
 * a temporary n x kp buffer.  TPA_EINVAL for another kp or reps < 1. */
tpa_status tpa_probe_gather(tpa_graph *g, int kp, int reps, void *stream, double *ms);

#ifdef __cplusplus
}
#endif

#endif /* TPA_H */
