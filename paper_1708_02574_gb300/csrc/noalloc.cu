// tpa_cpi_step_noalloc: one CPI propagation step that allocates nothing.
//
// Some callers cannot allocate device memory at the moment they want a
// propagation step: a serving loop whose memory is fully reserved up front by
// another allocator, a caller that must not pay the implicit synchronisation
// and latency of cudaMalloc/cudaFree on its critical path, or code running
// under a fixed memory budget.  For them this entry point takes its scratch
// (merge-path plan, tile carries, L1 partials, control block) from a
// file-scope __device__ array of TPA_NOALLOC_SCRATCH_BYTES bytes.  That array
// is part of the library image, so every GPU that loads libtpa holds it until
// the process exits.  The caller still provides the inputs and outputs.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "tpa_internal.cuh"

namespace {

constexpr int kMaxDevices = 64;

// The scratch itself.  In host code `g_step_scratch` names a host-side
// stand-in, never the device memory: host code must use the address returned
// by cudaGetSymbolAddress for the current device.
__device__ __align__(256) unsigned char g_step_scratch[TPA_NOALLOC_SCRATCH_BYTES];

unsigned char *g_scratch_addr[kMaxDevices];
std::mutex g_scratch_mu;

// Device address of the scratch on the current device, looked up once per
// device (the first call on a device does this set-up).
cudaError_t scratch_for_current_device(unsigned char **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_step_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

}  // namespace

using namespace tpa;

extern "C" tpa_status tpa_cpi_step_noalloc(int64_t n, int64_t m, const int64_t *row_ptr, const int32_t *col,
                                           const float *val, double c, const float *x, float *y, float *r,
                                           double *l1, void *stream)
{
    clear_error();
    // the walk gathers x while other tiles store y and add into r: an output
    // that is also an input would be read half-updated
    if ((x && (x == y || x == r)) || (y && y == r)) {
        set_error("tpa_cpi_step_noalloc: x, y and r must be distinct arrays (in-place steps are not supported)");
        return TPA_EINVAL;
    }
    if (n < 1 || n >= ((int64_t)1 << 31) || m < 0 || m >= ((int64_t)1 << 31)) {
        set_error("tpa_cpi_step_noalloc: n = %lld or m = %lld out of range", (long long)n, (long long)m);
        return TPA_EINVAL;
    }
    const size_t need = step1_scratch_bytes(n, m);
    if (need > TPA_NOALLOC_SCRATCH_BYTES) {
        set_error("tpa_cpi_step_noalloc: n + m = %lld needs %zu bytes of scratch, more than the %zu-byte limit",
                  (long long)(n + m), need, (size_t)TPA_NOALLOC_SCRATCH_BYTES);
        return TPA_EINVAL;
    }
    if (!(c > 0.0 && c < 1.0)) {
        set_error("tpa_cpi_step_noalloc: c = %g outside (0, 1)", c);
        return TPA_EINVAL;
    }
    if (!row_ptr || !x || !y || (m > 0 && (!col || !val))) {
        set_error("tpa_cpi_step_noalloc: NULL array");
        return TPA_EINVAL;
    }
    const void *must_be_device[] = {row_ptr, x, y, m > 0 ? (const void *)col : (const void *)row_ptr,
                                    m > 0 ? (const void *)val : (const void *)row_ptr, r ? (const void *)r : (const void *)y,
                                    l1 ? (const void *)l1 : (const void *)y};
    for (const void *q : must_be_device)
        if (!is_device_ptr(q)) {
            set_error("tpa_cpi_step_noalloc: every array must be device memory");
            return TPA_EINVAL;
        }
    unsigned char *scratch = nullptr;
    cudaError_t e = scratch_for_current_device(&scratch);
    if (e == cudaSuccess)
        e = run_step1(row_ptr, col, val, n, m, c, x, y, r, l1, scratch, (cudaStream_t)stream);
    if (e != cudaSuccess) {
        set_error("tpa_cpi_step_noalloc: %s", cudaGetErrorString(e));
        return TPA_ECUDA;
    }
    return TPA_OK;
}
