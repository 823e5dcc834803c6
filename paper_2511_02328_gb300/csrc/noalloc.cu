// noalloc.cu -- allocation-free variant of the boxcar S/N call.
//
// Some callers cannot call cudaMalloc at all: a real-time receiver thread
// whose every device allocation would implicitly synchronise the device and
// stall the data stream, or a host application whose memory pool has already
// reserved all of the GPU's memory for itself, so that a library-side
// cudaMalloc fails or fragments its pool.  Such a caller cannot create an
// af_plan (the plan uploads its delay table and sizes its scratch with
// cudaMalloc).  af_boxcar_snr_noalloc needs no plan: its scratch -- the
// per-row sums and per-row, per-width normalisation constants -- lives in
// the file-scope device array below, which every GPU that loads this library
// holds until the process exits.
//
// The first call on each device looks up the array's device address with
// cudaGetSymbolAddress (once per device, with that device current); make that
// first call before any stream capture.  Every call uses the same array, so
// calls whose work overlaps on the GPU (different streams, or different host
// threads) race on it: serialise them.  Each call overwrites every scratch
// entry it reads, so nothing has to start at zero.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <mutex>

#include "internal.h"

namespace {

// Room for AF_NOALLOC_MAX_ROWS rows: one af_rowstats_t plus AF_MAX_WIDTHS
// af_rowconst_t per row (16 + 32*16 bytes), 2.1 MiB in total.
constexpr size_t kStatsBytes = (size_t)AF_NOALLOC_MAX_ROWS * sizeof(af_rowstats_t);
constexpr size_t kConstBytes = (size_t)AF_NOALLOC_MAX_ROWS * AF_MAX_WIDTHS * sizeof(af_rowconst_t);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kStatsBytes + kConstBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices];

// Device address of g_noalloc_scratch on the current device (looked up once).
int scratch_address(void** out)
{
    int dev = 0;
    if (int rc = af_cuda_check(cudaGetDevice(&dev), "af_boxcar_snr_noalloc: cudaGetDevice")) return rc;
    if (dev < 0 || dev >= kMaxDevices) return af_set_error(AF_EINVAL, "af_boxcar_snr_noalloc: device %d", dev);
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return af_cuda_check(e, "af_boxcar_snr_noalloc: cudaGetSymbolAddress");
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return AF_OK;
}

}  // namespace

extern "C" int af_boxcar_snr_noalloc(const int32_t* d_plane, int ndm, int64_t nout, int nchan,
                                     const int32_t* widths, int nw, float* d_best_snr, uint8_t* d_best_w,
                                     void* stream)
try {
    if (!d_plane || !d_best_snr) return af_set_error(AF_EINVAL, "af_boxcar_snr_noalloc: NULL buffer");
    if (ndm < 1 || ndm > AF_NOALLOC_MAX_ROWS)
        return af_set_error(AF_EINVAL, "af_boxcar_snr_noalloc: ndm %d outside 1..%d (the static scratch holds %d rows)",
                            ndm, AF_NOALLOC_MAX_ROWS, AF_NOALLOC_MAX_ROWS);
    if (nout < 1 || nout > INT32_MAX) return af_set_error(AF_EINVAL, "af_boxcar_snr_noalloc: bad nout");
    if (nchan < 1 || nchan > 65536) return af_set_error(AF_EINVAL, "af_boxcar_snr_noalloc: bad nchan %d", nchan);
    // the same width checks (and the same choice of the 32-bit boxcar kernel) as af_boxcar_snr
    af_widths_t w;
    if (int rc = af_check_widths_nchan(nchan, widths, nw, nout, &w)) return rc;
    void* base = nullptr;
    if (int rc = scratch_address(&base)) return rc;
    af_rowstats_t* stats = (af_rowstats_t*)base;
    af_rowconst_t* rconst = (af_rowconst_t*)((unsigned char*)base + kStatsBytes);
    cudaStream_t s = (cudaStream_t)stream;
    if (int rc = af_launch_rowstats(d_plane, ndm, nout, stats, s)) return rc;
    return af_launch_boxcar(d_plane, ndm, nout, stats, w, rconst, d_best_snr, d_best_w, s);
} catch (...) {
    return af_host_exception("af_boxcar_snr_noalloc");
}
