// Internal declarations shared by the libtpa translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <string>
#include <vector>

#include "../../include/tpa.h"

namespace tpa {

// ---------------------------------------------------------------- errors ---
void set_error(const char *fmt, ...);
void clear_error();

struct Fail {
    tpa_status st;
};

#define TPA_CUDA(call)                                                                    \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) {                                                          \
            ::tpa::set_error("%s:%d %s: %s", __FILE__, __LINE__, #call, cudaGetErrorString(e_)); \
            throw ::tpa::Fail{e_ == cudaErrorMemoryAllocation ? TPA_ENOMEM : TPA_ECUDA}; \
        }                                                                                 \
    } while (0)

#define TPA_REQUIRE(cond, ...)                 \
    do {                                       \
        if (!(cond)) {                         \
            ::tpa::set_error(__VA_ARGS__);     \
            throw ::tpa::Fail{TPA_EINVAL};     \
        }                                      \
    } while (0)

#define TPA_CHECK_LAUNCH() TPA_CUDA(cudaGetLastError())

// profile.cu: launch accounting and optional event timing
void note_launch(const char *family, int count = 1);
void note_launch_count(int count);   // counter only; never allocates
uint64_t launches_so_far();
bool prof_pause();                   // stop event timing (during graph capture); returns the previous state
void prof_resume(bool timing);
struct ProfMark {
    cudaEvent_t a;
};
ProfMark prof_begin(cudaStream_t s);
void prof_end(const ProfMark &m, const char *family, double bytes, cudaStream_t s);

// --------------------------------------------------------------- memory ---
// Device buffer owned by the library (cudaMallocAsync on the call's stream).
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    void ensure(size_t b, cudaStream_t s);   // grow-only
    void release(cudaStream_t s);
    template <class T> T *as() const { return static_cast<T *>(p); }
};

bool is_device_ptr(const void *p);

// Check before a launch that a buffer holds the bytes the launch indexes
// (TPA_ECUDA with a message otherwise).
void need(const DevBuf &b, size_t bytes, const char *what);

// Hand unused blocks of the library's memory pool back to the driver (call
// after a device or stream synchronisation that retired the frees).
void trim_pool() noexcept;

// Copy `bytes` from a host or device pointer into device memory (stream-ordered).
void copy_in(void *dst_dev, const void *src_any, size_t bytes, cudaStream_t s);

// ------------------------------------------------------ merge-path plans ---
// A tile of the merge path between the row-end offsets of a CSR and the
// nonzero indices.  Tile t covers path diagonals [t*L, (t+1)*L).
struct Plan {
    int L = 0;              // path steps per tile
    int64_t tiles = 0;
    DevBuf tile_x;          // int32[tiles+1]  rows fully consumed before the tile
    DevBuf tile_y;          // int64[tiles+1]  nonzeros consumed before the tile
    DevBuf head_row;        // int32[tiles]    row whose end falls in the tile but that started before it, or -1
    DevBuf head_first;      // int32[tiles]    first tile holding a nonzero of that row
};

// Rows of a CSR binned by length for the binned-row kernels (built once per
// graph and CSR; see spmm_binned.cuh).
struct BinPlan {
    bool built = false;
    int64_t n_short = 0, n_mid = 0, n_long = 0, n_empty = 0, n_chunks = 0;
    DevBuf rows_short, rows_mid, rows_long, rows_empty;   // int32 row ids
    DevBuf long_first;    // int64[n_long + 1] first chunk of each long row
    DevBuf chunk_row;     // int32[n_chunks]
    DevBuf chunk_e0;      // int64[n_chunks]
};

// The segmented flag walk (spmm_seg.cuh) over one CSR: a copy of the column
// ids with bit 31 set on the first nonzero of every row (zero-padded to whole
// tiles of the widest tile), the rows with and without nonzeros, and the
// exclusive prefix of the nonempty-row flags (int64[n + 1]).
struct SegRows {
    bool built = false;
    int64_t n_nz = 0, n_empty = 0, padded = 0;
    DevBuf colf, nz_rows, empty_rows, nzpos;
    DevBuf nzrp;   // lane-segment walk: first nonzero of every nonempty row, then m (int64[n_nz + 1])
};
// Tiles of tn nonzeros: crow0[t] (int32[tiles + 1]) is the number of rows
// that start before tile t.
struct SegTiles {
    int64_t tn = 0, tiles = 0;
    DevBuf crow0;
};
constexpr int64_t SEG_MAX_TN = 1024;   // the padding of the column arrays covers tiles up to this size

// ---------------------------------------------------------------- graph ---
// The column and value arrays of both CSRs hold at least CSR_PAD extra zero
// elements after the m real ones, so kernels may stage a tile's nonzeros in
// 16-byte chunks rounded outward; they are allocated to csr_len(m) elements,
// which also covers the whole last tile of a segmented walk (tiles of at
// most SEG_MAX_TN nonzeros, whose bulk copies read whole tiles).
constexpr int64_t CSR_PAD = 4;
constexpr int64_t CSR_TILE_PAD = 1024;
inline int64_t csr_len(int64_t m) { return (m + CSR_TILE_PAD - 1) / CSR_TILE_PAD * CSR_TILE_PAD + CSR_TILE_PAD; }
static_assert(CSR_TILE_PAD >= SEG_MAX_TN, "CSR padding covers a whole tile");

struct Workspace {
    DevBuf x, y, r;         // iterates and accumulator
    DevBuf carry, head, tl1;   // per-tile carries, deferred heads, per-tile L1
    DevBuf fix;             // fixup partials
    DevBuf ctl;             // control block (see Ctl)
    DevBuf seeds;           // int32 seeds (or seed-set members)
    DevBuf sets;            // int64 seed-set offsets
    DevBuf seeds_g, cols;   // a query's seeds regrouped; their positions, then the swapped column pairs
    DevBuf out;             // device staging for host outputs
    DevBuf stage[2];        // column groups of a host output, computed in turn while the other is copied
    cudaStream_t copy = nullptr;                   // the copies of staged column groups to the host
    cudaEvent_t ready[2] = {nullptr, nullptr};     // a group's scores are in stage[b]
    cudaEvent_t copied[2] = {nullptr, nullptr};    // stage[b] has reached the host
    DevBuf iters;           // int32 per-column iteration counts
    DevBuf u;               // push path: 64-bit fixed-point accumulator [n][KP]
    DevBuf touched;         // push path: one bit per row reached by the push
    DevBuf x2;              // push path: x2 [n][KP <= 16], zero outside the marked rows
    DevBuf cpart;           // binned-row kernels: chunk sums of long rows [chunks][KP]
    DevBuf agg;             // segmented kernel: tagged carry-out words [tiles][KP] (zeroed when allocated)
    DevBuf lrec, ltail;     // lane-segment walk: row parts [n_nz][KP], segment-end sums [segments][KP]
    bool u_clean = false;   // u, touched and x2 are known to be all zero
    // The segmented walk never writes the rows of y without in-edges, so they
    // must already read as zero.  x_zkp / y_zkp: the padded width KP for
    // whose layout [n][KP] the rows without in-edges of x / y are known to be
    // zero (-1: the whole buffer is zero; 0: not known).  x_seeds: those rows
    // of x are zero except the current chunk's seeds, which hold x0.
    int x_zkp = 0, y_zkp = 0;
    bool x_seeds = false;
    int32_t *hflag = nullptr;   // pinned host mirror of the done flag (2 slots)
};

}  // namespace tpa

struct tpa_graph {
    int64_t n = 0, m = 0;
    int device = 0;
    // CSR(A~^T): rows = destinations
    tpa::DevBuf rp_t, col_t, val_t;
    // CSR(A~): rows = sources
    tpa::DevBuf rp_a, col_a, val_a;
    tpa::DevBuf outdeg;
    tpa::DevBuf inv_deg32;  // float[n] RN32(1/outdeg), 0 for deadends: the value of every edge out of a node
    tpa::DevBuf perm_a2t;   // uint32[m]: position in CSR(A~^T) of each CSR(A~) edge (ensure_perm_a2t)
    // weighted graphs (tpa_set_edge_weights)
    tpa::DevBuf w_a;        // float[m] edge weights, CSR(A~) order
    tpa::DevBuf inv_d;      // double[n] 1 / weighted out-degree
    tpa::DevBuf row_a;      // int32[m] source of each CSR(A~) edge (made on first use)
    bool weighted = false;
    // preprocessing result
    tpa::DevBuf r_str;
    bool has_pre = false;
    double c = 0, eps = 0;
    int T = 0;
    int64_t pre_iters = 0;
    std::map<int, tpa::Plan> plans_t;   // merge-path plans over CSR(A~^T) keyed by L
    std::map<int, tpa::Plan> plans_a;   // merge-path plans over CSR(A~) keyed by L
    tpa::BinPlan bins_t, bins_a;        // row bins of CSR(A~^T) and CSR(A~)
    tpa::SegRows seg_t, seg_a;          // flag-walk data of CSR(A~^T) and CSR(A~)
    std::map<int, tpa::SegTiles> segt_t, segt_a;   // flag-walk tiles keyed by tile size
    tpa::Workspace ws;
};

namespace tpa {

// Control block living in device memory, one per CPI run.
struct Ctl {
    int32_t done;           // 1 once no column is alive
    int32_t ticket;         // last-block-done counter for the fixup reduction
    int32_t iter;           // current iteration index (written by the host-side schedule)
    int32_t push;           // 1: this query chunk takes the push path for x1, x2 (decided on the device)
    uint32_t epoch;         // launches of the segmented SpMM so far (tags its carry-out words; never reset)
    int32_t error;          // 1: a bounded device wait gave up (kept until the host reads and clears it)
    int32_t pad_[2];
};
// Per-column state follows the Ctl header in the control buffer:
//   int32 alive[kpad], int32 iters[kpad], double norm[kpad]

// build.cu
void build_csr(tpa_graph *g, const int32_t *d_src, const int32_t *d_dst, int64_t m_in,
               cudaStream_t s);
// g->perm_a2t (position in CSR(A~^T) of each CSR(A~) edge), built on first use
void ensure_perm_a2t(tpa_graph *g, cudaStream_t s);
// out[0..len] = exclusive prefix sums of in[0..len) and the total (device arrays)
void exclusive_scan_i32_i64(const int32_t *in, int64_t *out, int64_t len, DevBuf &tmp, cudaStream_t s);

// cpi.cu
const Plan &get_plan(tpa_graph *g, int L, cudaStream_t s, int which = 0);   // which: 0 = A~^T, 1 = A~

// One SpMV/SpMM step y = decay * M x for kc <= 32 columns (x, y node-major
// [n][kp_for(kc)], padding columns of x zero) with M = A~^T (which = 0) or
// M = A~ (which = 1).
int kp_for(int k);
void spmv_apply(tpa_graph *g, int which, const float *x, float *y, int kc, float decay, cudaStream_t s);

enum Mode : int {
    MODE_ACC = 0,     // y written; r += y for alive columns when i >= s_iter
    MODE_FINAL = 1    // TPA: out = (1+alpha) (r + y) + r_str; y and r not written
};

struct CpiArgs {
    // seeds for single-seed columns (device int32[k]); nullptr = PageRank (k = 1)
    const int32_t *seeds = nullptr;
    int k = 1;
    double c = 0.15, eps = 1e-9;
    int s_iter = 0, t_iter = -1;
    // output: accumulation target (float32, row stride ldr, columns offset by the
    // chunk start), or an internal [n][KP] buffer when r_internal is set
    float *r = nullptr;
    int64_t ldr = 1;
    bool r_internal = false;
    // TPA online: finalize into out with (1+alpha) and r_str on the last iteration
    bool tpa_final = false;
    double alpha = 0.0;
    const float *r_str = nullptr;
    float *out = nullptr;
    int64_t ldo = 1;
    int32_t *iters_out = nullptr;   // device int32[k] or nullptr
    // host int32[k]: out-degrees of the seeds.  Given, query chunks choose
    // their push/pull branch on the host; absent (graph capture), on the device.
    const int32_t *seed_outdeg = nullptr;
    // seed sets (device int64[k+1]): column j starts from q = 1/|S_j| on the
    // members seeds[set_ptr[j] .. set_ptr[j+1]) instead of one seed
    const int64_t *set_ptr = nullptr;
    // the caller has ordered the seeds already (no regrouping here); when
    // dev_pairs is set (device int32: a count, then that many column pairs,
    // at most max_pairs), the paired columns of out are swapped at the end
    bool no_regroup = false;
    const int32_t *dev_pairs = nullptr;
    int max_pairs = 0;
};

// adjoint.cu
void set_edge_weights(tpa_graph *g, const float *w_any, cudaStream_t s, bool drop_preprocessing = true);
void weights_from_features(const float *feat, const float *theta, int d, int64_t m, float *w, cudaStream_t s);
void theta_grad(const float *feat, const float *w, const float *gw, int d, int64_t m, double *out, cudaStream_t s);
double loss_grad(tpa_graph *g, const int32_t *seeds, const int32_t *pos, const int32_t *neg, int ntrip, double c,
                 int S, int T, int K, float *grad_w, cudaStream_t s);
// Bytes of stranger-chain iterates the reverse sweep keeps before it switches
// to checkpoints every ceil(sqrt(K+1)) iterations (tpa_set_adjoint_budget).
extern size_t g_adjoint_budget;
// Triples per family batch of tpa_loss_grad (tpa_set_adjoint_batch_width;
// 0: the default) and the width in effect.
extern int g_adjoint_batch;
int adjoint_batch_width();


// Out-degrees of k device-resident seeds, copied to the host (one small copy and a wait).
std::vector<int32_t> seed_outdegrees(tpa_graph *g, const int32_t *d_seeds, int k, cudaStream_t s);

void run_cpi(tpa_graph *g, const CpiArgs &a, cudaStream_t s);

// The order tpa_query runs the k seeds of a call in, from their out-degrees
// od (host): perm[j] is the original position of the seed placed at j.
// False when nothing moves.
bool regroup_seeds(const int32_t *od, int k, int S, std::vector<int32_t> &perm);

// The branch each query chunk of k seeds with out-degrees od (in run order,
// host) takes for x1 and x2: one character per chunk, 'p' push, 'l' pull,
// '-' neither (the chunk pulls every iteration); a captured launch sequence
// is valid for the seeds of any batch with the same string.
std::string query_branches(const int32_t *od, int k, int S);

// Counter bumped by every change of a kernel setting (variant, chunk widths,
// push path): launch sequences captured before a change are stale.
uint64_t settings_epoch();

// TPA's neighbor scale alpha (Section III-B, Lemma 2).
double alpha_of(double c, int S, int T);

// One CPI propagation step for a single vector with all scratch taken from
// `scratch` (at least step1_scratch_bytes(n, m) bytes of device memory).
// Throws nothing and allocates nothing; returns the first CUDA error.
size_t step1_scratch_bytes(int64_t n, int64_t m);
cudaError_t run_step1(const int64_t *rp, const int32_t *col, const float *val, int64_t n, int64_t m, double c,
                      const float *x, float *y, float *r, double *l1, unsigned char *scratch, cudaStream_t s);

}  // namespace tpa
