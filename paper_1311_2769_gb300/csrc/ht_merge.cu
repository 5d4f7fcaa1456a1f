// ht_merge.cu — duplicate and mirror merging of fitted candidates.
//
// Section 3 hands the transform's candidates to a confirmation step.  Every
// track leaves a mirror candidate (phi0 + pi, -d0, -kappa: the same circle
// travelled the other way) and nearby cells that its hits also fill above
// threshold.  After the circle fit:
//  * a candidate whose fit has status != 1 is UNFITTED;
//  * a fitted candidate is BACKWARD unless its hits lie ahead of its perigee
//    along t = (cos phi0, sin phi0): the binary64 sum over its row, in row
//    order, of x cos phi0 + y sin phi0 must be > 0 (the perigee d0 n is
//    orthogonal to t);
//  * a forward fitted candidate is a DUPLICATE when a better one (more
//    votes, or as many and a smaller index) of the same event lies within
//    `radius` cells in phi0 (periodic), d0 and kappa; otherwise KEPT.
// Two kernels, one thread per candidate.  The first sums the direction test
// with one IEEE binary64 operation per step, as the definition orders it.
// The second searches the event's peaks, which are sorted by linear index:
// for each phi0 row within the radius one binary search finds the first
// peak at or after (row, j - r, k - r), and a scan runs to (row, j + r,
// k + r), checking the kappa distance of the peaks in between.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "ht_internal.h"

namespace ht {
namespace {

__device__ __forceinline__ int64_t merge_count(const MergeParams& p) {
    int64_t n = *p.n_peaks;
    if (n > p.peak_cap) n = p.peak_cap;
    if (n > p.cap) n = p.cap;
    return n;
}

__global__ void merge_direction_kernel(const MergeParams p) {
    const int64_t n = merge_count(p);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += stride) {
        const ht_track& f = p.fits[c];
        // a row cut by pair_cap is never fitted; the check also keeps the
        // reads inside hit_idx whatever fits the caller passes
        if (f.status != 1 || p.po[c + 1] > p.pair_cap) {
            p.state[c] = HT_MERGE_UNFITTED;
            continue;
        }
        const double cs = f.cos_phi0, sn = f.sin_phi0;
        double t = 0.0;
        for (int64_t k = p.po[c]; k < p.po[c + 1]; ++k) {
            const int32_t h = p.hidx[k];
            t = __dadd_rn(t, __dadd_rn(__dmul_rn((double)p.x[h], cs), __dmul_rn((double)p.y[h], sn)));
        }
        p.state[c] = t > 0.0 ? HT_MERGE_KEPT : HT_MERGE_BACKWARD;
    }
}

__device__ __forceinline__ int64_t peak_lin(const ht_peak& q, int32_t nd, int32_t nk) {
    return ((int64_t)q.i_phi * nd + q.i_d0) * nk + q.i_kappa;
}

// first index in [lo, hi) whose event is >= ev
__device__ int64_t lower_event(const ht_peak* pk, int64_t lo, int64_t hi, int32_t ev) {
    while (lo < hi) {
        const int64_t m = lo + ((hi - lo) >> 1);
        if (pk[m].event < ev) lo = m + 1;
        else hi = m;
    }
    return lo;
}

// first index in [lo, hi) whose linear index is >= key
__device__ int64_t lower_lin(const ht_peak* pk, int64_t lo, int64_t hi, int64_t key, int32_t nd, int32_t nk) {
    while (lo < hi) {
        const int64_t m = lo + ((hi - lo) >> 1);
        if (peak_lin(pk[m], nd, nk) < key) lo = m + 1;
        else hi = m;
    }
    return lo;
}

__global__ void merge_suppress_kernel(const MergeParams p) {
    const int64_t n = merge_count(p);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int32_t nphi = p.n_phi, nd = p.n_d0, nk = p.n_kappa, r = p.radius;
    for (int64_t c0 = (int64_t)blockIdx.x * blockDim.x; c0 < n; c0 += stride) {
        const int64_t c = c0 + threadIdx.x;
        bool kept = false;
        if (c < n && p.state[c] >= 0) {
            const ht_peak a = p.peaks[c];
            const int64_t b = lower_event(p.peaks, 0, n, a.event);
            const int64_t e = lower_event(p.peaks, b, n, a.event + 1);
            const int32_t jlo = max(a.i_d0 - r, 0), jhi = min(a.i_d0 + r, nd - 1);
            const int32_t klo = max(a.i_kappa - r, 0), khi = min(a.i_kappa + r, nk - 1);
            const bool all_rows = 2 * r + 1 >= nphi;
            const int32_t rows = all_rows ? nphi : 2 * r + 1;
            bool dup = false;
            for (int32_t t = 0; t < rows && !dup; ++t) {
                int32_t i = all_rows ? t : a.i_phi - r + t;
                if (i < 0) i += nphi;
                if (i >= nphi) i -= nphi;
                const int64_t key_lo = ((int64_t)i * nd + jlo) * nk + klo;
                const int64_t key_hi = ((int64_t)i * nd + jhi) * nk + khi;
                for (int64_t q = lower_lin(p.peaks, b, e, key_lo, nd, nk); q < e; ++q) {
                    const ht_peak o = p.peaks[q];
                    if (peak_lin(o, nd, nk) > key_hi) break;
                    if (q == c || o.i_kappa < klo || o.i_kappa > khi) continue;
                    if (p.state[q] < 0) continue;  // unfitted or backward: never suppresses
                    if (o.votes > a.votes || (o.votes == a.votes && q < c)) {
                        dup = true;
                        break;
                    }
                }
            }
            // Only KEPT -> DUPLICATE is written; readers test state >= 0, which
            // both values satisfy, so the order of these writes does not matter.
            if (dup) p.state[c] = HT_MERGE_DUPLICATE;
            kept = !dup;
        }
        const unsigned m = __ballot_sync(0xffffffffu, kept);
        if (m && (threadIdx.x & 31) == (unsigned)(__ffs(m) - 1))
            atomicAdd(p.kept, (unsigned long long)__popc(m));
    }
}

}  // namespace

cudaError_t launch_merge(const MergeParams& p, cudaStream_t s) {
    if (p.cap <= 0 || p.peak_cap <= 0) return cudaSuccess;
    const int64_t want = (std::min(p.cap, p.peak_cap) + 255) / 256;
    const int grid = (int)(want < 152 * 16 ? (want > 0 ? want : 1) : 152 * 16);
    merge_direction_kernel<<<grid, 256, 0, s>>>(p);
    if (cudaError_t e = cudaGetLastError()) return e;
    merge_suppress_kernel<<<grid, 256, 0, s>>>(p);
    return cudaGetLastError();
}

}  // namespace ht
