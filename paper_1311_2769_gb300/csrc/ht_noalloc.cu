// ht_noalloc.cu — peak finding that allocates nothing.
//
// Some callers cannot allocate device memory at the point where they need
// peaks: code running inside a framework that owns every allocation (a
// caching allocator or a fixed memory pool), code on a real-time path where
// cudaMalloc's implicit synchronisation and latency are not allowed, or code
// that has no context object to keep buffers in.  ht_peaks_noalloc serves
// them: the caller passes the accumulators and the output buffers, and the
// per-column scratch (peak counts, bitmasks, scan partials) lives in one
// fixed file-scope device array that every GPU loading the library holds
// until the process exits.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <mutex>

#include "ht_internal.h"

using namespace ht;

namespace {

// Shared by every call on a device; see ht_peaks_noalloc in ht.h.
static __device__ __align__(256) unsigned char g_noalloc_scratch[HT_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Device address of the scratch array for the current device (first use on
// a device looks it up; a host-side use of the symbol itself would be wrong).
cudaError_t scratch_for_current_device(unsigned char** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = p;
    }
    *out = static_cast<unsigned char*>(g_addr[dev]);
    return cudaSuccess;
}

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

struct Layout {
    size_t scal, npk, colbase, mask, wpre, part, total;
};

Layout layout(int64_t cols, int nkw) {
    Layout L{};
    size_t o = 0;
    L.scal = o;
    o = align256(o + 8 * sizeof(int64_t));
    L.npk = o;
    o = align256(o + (size_t)cols * sizeof(int32_t));
    L.colbase = o;
    o = align256(o + (size_t)(cols + 1) * sizeof(int64_t));
    L.mask = o;
    o = align256(o + (size_t)cols * nkw * sizeof(uint32_t));
    L.wpre = o;
    o = align256(o + (size_t)cols * nkw * sizeof(uint16_t));
    L.part = o;
    o = align256(o + 2 * kScanBlocks * sizeof(int64_t));
    L.total = o;
    return L;
}

bool grid_valid(const ht_grid* g) {
    return g && g->n_phi >= 1 && g->n_phi <= 65535 && g->n_d0 >= 1 && g->n_d0 <= 65535 && g->n_kappa >= 1 &&
           g->n_kappa <= 4096 && (int64_t)g->n_d0 * g->n_kappa <= (1 << 24);
}

}  // namespace

extern "C" int ht_peaks_noalloc(const ht_grid* grid, const uint32_t* acc, int32_t n_events, uint32_t threshold,
                                ht_peak* peaks, int64_t cap, int64_t* count, void* stream) {
    if (!grid_valid(grid) || !acc || n_events < 0 || !count || cap < 0 || (cap > 0 && !peaks))
        return HT_ERR_INVALID_ARG;
    // the detection stages whole kappa rows with 16-byte loads when n_kappa is
    // a multiple of 4; the count is one 8-byte store, the peaks 4-byte fields
    if (((uintptr_t)count & 7u) != 0 || ((uintptr_t)peaks & 3u) != 0 || ((uintptr_t)acc & 3u) != 0 ||
        (grid->n_kappa % 4 == 0 && ((uintptr_t)acc & 15u) != 0))
        return HT_ERR_INVALID_ARG;
    const int nkw = (grid->n_kappa + 31) / 32;
    const int64_t cols = (int64_t)n_events * grid->n_phi * grid->n_d0;
    // each column takes 12 + 6 nkw bytes of scratch (count, base, mask, word
    // prefixes): refuse before the layout's size arithmetic could wrap
    if (cols > (int64_t)(HT_NOALLOC_SCRATCH_BYTES / (12u + 6u * (unsigned)nkw))) return HT_ERR_BUDGET;
    const Layout L = layout(cols, nkw);
    if (L.total > (size_t)HT_NOALLOC_SCRATCH_BYTES) return HT_ERR_BUDGET;
    unsigned char* base = nullptr;
    if (scratch_for_current_device(&base) != cudaSuccess) return HT_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    int64_t* scal = reinterpret_cast<int64_t*>(base + L.scal);
    // the scratch keeps the previous call's contents: clear what must start at zero
    if (cudaMemsetAsync(scal, 0, 8 * sizeof(int64_t), s) != cudaSuccess) return HT_ERR_CUDA;
    if (cols > 0) {
        PeakParams p{};
        p.acc = acc;
        p.cells = (int64_t)grid->n_phi * grid->n_d0 * grid->n_kappa;
        p.n_events = n_events;
        p.event0 = 0;
        p.thr = threshold;
        p.nphi = grid->n_phi;
        p.nd = grid->n_d0;
        p.nk = grid->n_kappa;
        p.nkw = nkw;
        p.mask = reinterpret_cast<uint32_t*>(base + L.mask);
        p.wpre = reinterpret_cast<uint16_t*>(base + L.wpre);
        p.npk = reinterpret_cast<int32_t*>(base + L.npk);
        p.colbase = reinterpret_cast<int64_t*>(base + L.colbase);
        p.peaks = peaks;
        p.peak_cap = cap;
        p.window = -1;
        p.paircnt = nullptr;
        p.extra_pairs = nullptr;
        if (launch_detect(p, s) != cudaSuccess) return HT_ERR_CUDA;
        ScanRange r{};
        r.in = p.npk;
        r.out = p.colbase;
        r.lo = 0;
        r.hi = cols;
        r.cap = cols;
        r.base_dev = scal + 2;  // zero
        r.total = scal + 0;
        r.write_end = 0;
        if (launch_scan(r, reinterpret_cast<int64_t*>(base + L.part), s) != cudaSuccess) return HT_ERR_CUDA;
        if (launch_emit(p, s) != cudaSuccess) return HT_ERR_CUDA;
    }
    if (cudaMemcpyAsync(count, scal, sizeof(int64_t), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        return HT_ERR_CUDA;
    return HT_OK;
}
