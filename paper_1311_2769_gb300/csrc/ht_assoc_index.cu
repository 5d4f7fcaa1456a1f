// ht_assoc_index.cu — association through a per-layer angular index.
//
// The association rule (a hit joins peak (i, j, k) when its kappa bin in
// column (i, j) lies within `window` of k) is evaluated here only for the
// hits that can satisfy it, found geometrically, instead of for every hit of
// the event in every column:
//  * For a fixed column, kappa = 2 (q - d) / (r^2 + d^2 - 2 d q) is monotone
//    in q = y cos phi - x sin phi whenever r != |d| (dkappa/dq has the sign of
//    r^2 - d^2), with inverse q = (kappa (r^2 + d^2) + 2 d) / (2 (1 + kappa d)).
//    So the hits of radius r whose exact kappa lies in [kappa_lo, kappa_hi]
//    have s = q / r in an interval, and s = sin(theta - phi) for the hit's
//    polar angle theta: at most two angular windows per radius.
//  * Hits are bucketed by (event, layer); each bucket holds its hits sorted
//    by angle and the range of their radii.  Over a bucket's radius range
//    the interval of s is bounded by its values at the two ends and at the
//    one interior stationary point r* = sqrt(d^2 + 2 d / kappa) (s is monotone
//    in kappa for fixed r, so the kappa ends suffice).
//  * The kappa range is the peak's window widened by one bin on each side,
//    far more than the difference between the method's binned kappa and the
//    exact one; s and the angles are widened by 1e-4, far more than the
//    float errors of these bounds.  A bucket whose radius range comes within
//    5 % of |d| (where kappa is not monotone or its bin is ill-conditioned),
//    or where |kappa d| > 1/2, takes all its hits.
// Every candidate is then binned exactly as the scanning association bins it
// (same stage-1 certificate, same slow path), so the rows are the same; the
// matches of a row are marked in a per-warp bitmap over the event's hit range
// and written in ascending hit order.  The row length is known beforehand
// (the window sum of the accumulator), and a row that comes out with another
// length raises an error flag instead of passing silently.
#include <cuda_runtime.h>

#include <cstdint>

#include "ht_internal.h"
#include "ht_kbin.cuh"

namespace ht {
namespace {

constexpr int kIdxSortCap = 4096;   // bucket size sorted in shared memory
constexpr int kIdxCapWords = 512;   // bitmap words per warp: 16384 hits per segment
constexpr int kIdxRanges = 4;       // angle ranges per layer lane
constexpr int kIdxWarps = 8;
constexpr int kIdxBins = 256;       // coarse angle table per bucket: first position at or after each bin start
constexpr int kIdxChunk = 256;      // consecutive peaks per block step (one event's buckets stay in L1)

__device__ __forceinline__ float bin_start(int t) {
    return -3.14159265358979323846f + (float)t * (6.28318530717958647692f / (float)kIdxBins);
}

__device__ __forceinline__ int clamp_layer(int l, int nl) { return l < 0 ? 0 : (l >= nl ? nl - 1 : l); }

// bucket counts and radius ranges (r^2 as float bits: non-negative floats
// order like their bit patterns)
__global__ void index_count_kernel(const IndexParams p) {
    extern __shared__ uint32_t hist[];  // [nl] counts, [nl] r2 min, [nl] r2 max
    const int nl = p.nl;
    for (int e = blockIdx.x; e < p.n_events; e += gridDim.x) {
        for (int l = threadIdx.x; l < nl; l += blockDim.x) {
            hist[l] = 0;
            hist[nl + l] = 0x7F800000u;
            hist[2 * nl + l] = 0;
        }
        __syncthreads();
        const int h0 = p.offs[e], h1 = p.offs[e + 1];
        for (int h = h0 + threadIdx.x; h < h1; h += blockDim.x) {
            const int l = clamp_layer(p.layer[h], nl);
            const float x = p.x[h], y = p.y[h];
            const uint32_t r2 = __float_as_uint(__fadd_rn(__fmul_rn(x, x), __fmul_rn(y, y)));
            atomicAdd(&hist[l], 1u);
            atomicMin(&hist[nl + l], r2);
            atomicMax(&hist[2 * nl + l], r2);
        }
        __syncthreads();
        for (int l = threadIdx.x; l < nl; l += blockDim.x) {
            const int64_t b = (int64_t)e * nl + l;
            p.bcount[b] = (int32_t)hist[l];
            p.r2min[b] = hist[nl + l];
            p.r2max[b] = hist[2 * nl + l];
            p.bcursor[b] = 0;
        }
        __syncthreads();
    }
}

__global__ void index_scatter_kernel(const IndexParams p) {
    const int nl = p.nl;
    for (int e = blockIdx.x; e < p.n_events; e += gridDim.x) {
        const int h0 = p.offs[e], h1 = p.offs[e + 1];
        for (int h = h0 + threadIdx.x; h < h1; h += blockDim.x) {
            const int64_t b = (int64_t)e * nl + clamp_layer(p.layer[h], nl);
            const int64_t pos = p.bstart[b] + atomicAdd(&p.bcursor[b], 1);
            p.theta[pos] = atan2f(p.y[h], p.x[h]);
            p.hid[pos] = h;
        }
    }
}

__device__ __forceinline__ bool pair_less(float ka, int32_t va, float kb, int32_t vb) {
    return ka < kb || (ka == kb && va < vb);
}

// Ascending bitonic sort of n (key, value) pairs by the block, in shared or
// global memory (generic pointers).  Positions n .. pow2 - 1 act as +infinity:
// every comparator puts the smaller element at the lower index, so those
// virtual elements never move and are never touched.
__device__ void block_sort_pairs(float* key, int32_t* val, int n) {
    int N = 1, lg = 0;
    while (N < n) {
        N <<= 1;
        ++lg;
    }
    for (int kl = 1; kl <= lg; ++kl) {
        const int k = 1 << kl;
        for (int jl = kl - 1; jl >= 0; --jl) {
            const int j = 1 << jl;
            const bool flip = jl == kl - 1;
            for (int i = threadIdx.x; i < (N >> 1); i += blockDim.x) {
                const int a = ((i >> jl) << (jl + 1)) + (i & (j - 1));
                const int b = flip ? (a ^ (k - 1)) : (a + j);
                if (b < n) {
                    const float ka = key[a], kb = key[b];
                    const int32_t va = val[a], vb = val[b];
                    if (pair_less(kb, vb, ka, va)) {
                        key[a] = kb;
                        key[b] = ka;
                        val[a] = vb;
                        val[b] = va;
                    }
                }
            }
            __syncthreads();
        }
    }
}

__global__ void index_sort_kernel(const IndexParams p) {
    extern __shared__ __align__(16) unsigned char sraw[];
    float* sk = reinterpret_cast<float*>(sraw);
    int32_t* sv = reinterpret_cast<int32_t*>(sk + kIdxSortCap);
    const int64_t nb = (int64_t)p.n_events * p.nl;
    for (int64_t b = blockIdx.x; b < nb; b += gridDim.x) {
        const int64_t base = p.bstart[b];
        const int n = (int)(p.bstart[b + 1] - base);
        int32_t* tab = p.tab + b * (kIdxBins + 1);
        if (n <= 1) {
            for (int t = threadIdx.x; t <= kIdxBins; t += blockDim.x)
                tab[t] = (n == 1 && t > 0 && p.theta[base] < bin_start(t)) || t == kIdxBins ? n : 0;
            continue;
        }
        if (n <= kIdxSortCap) {
            for (int t = threadIdx.x; t < n; t += blockDim.x) {
                sk[t] = p.theta[base + t];
                sv[t] = p.hid[base + t];
            }
            __syncthreads();
            block_sort_pairs(sk, sv, n);
            for (int t = threadIdx.x; t < n; t += blockDim.x) {
                p.theta[base + t] = sk[t];
                p.hid[base + t] = sv[t];
            }
            __syncthreads();
        } else {
            block_sort_pairs(p.theta + base, p.hid + base, n);
        }
        // coarse table: first sorted position with angle >= each bin start
        for (int t = threadIdx.x; t <= kIdxBins; t += blockDim.x) {
            int lo = 0, hi = n;
            if (t == kIdxBins) {
                lo = n;
            } else {
                const float v = bin_start(t);
                while (lo < hi) {
                    const int m = (lo + hi) >> 1;
                    if (p.theta[base + m] < v) lo = m + 1;
                    else hi = m;
                }
            }
            tab[t] = lo;
        }
        __syncthreads();
    }
}

// first position in [lo, hi) of sorted t with t[pos] >= v
__device__ __forceinline__ int64_t lower_theta(const float* t, int64_t lo, int64_t hi, float v) {
    while (lo < hi) {
        const int64_t m = lo + ((hi - lo) >> 1);
        if (t[m] < v) lo = m + 1;
        else hi = m;
    }
    return lo;
}

// conservative range of s = q / r over the bucket's radii for kappa in
// [klo, khi]; false when the bucket must take all its hits
__device__ __forceinline__ bool s_range(float rlo, float rhi, float d, float klo, float khi, float& slo,
                                        float& shi) {
    const float ad = fabsf(d);
    if (!(rlo > 1e-6f) || !(rhi >= rlo)) return false;
    if (rlo <= ad * 1.05f + 1e-3f && rhi >= ad * 0.95f - 1e-3f) return false;
    if (fabsf(klo * d) > 0.5f || fabsf(khi * d) > 0.5f) return false;
    slo = 3.0f;
    shi = -3.0f;
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        const float kap = t ? khi : klo;
        const float num0 = kap * d * d + 2.0f * d, den0 = 2.0f * (1.0f + kap * d);
        float rs[3] = {rlo, rhi, rlo};
        const float st = d * d + (kap != 0.0f ? 2.0f * d / kap : -1.0f);
        if (kap != 0.0f && st > 0.0f) {
            const float r = sqrtf(st);
            if (r > rlo && r < rhi) rs[2] = r;
        }
#pragma unroll
        for (int u = 0; u < 3; ++u) {
            const float r = rs[u];
            const float s = (kap * r * r + num0) / (den0 * r);
            slo = fminf(slo, s);
            shi = fmaxf(shi, s);
        }
    }
    if (!(slo <= shi)) return false;  // NaN on the way: take every hit
    slo -= 1e-4f;
    shi += 1e-4f;
    return true;
}

struct Ranges {
    int64_t a[kIdxRanges], b[kIdxRanges];
    int n;
};

// first position in [lo, hi) of sorted t with t[pos] > v
__device__ __forceinline__ int64_t upper_theta(const float* t, int64_t lo, int64_t hi, float v) {
    while (lo < hi) {
        const int64_t m = lo + ((hi - lo) >> 1);
        if (t[m] <= v) lo = m + 1;
        else hi = m;
    }
    return lo;
}

// The part of a bucket that can hold the first angle >= v (or > v): the
// table's bins around v's bin (one bin of slack on each side absorbs the
// rounding of the bin index)
__device__ __forceinline__ void table_window(const int32_t* tab, int64_t lo, float v, int64_t& a, int64_t& b) {
    int t = (int)floorf((v + 3.14159265358979323846f) * ((float)kIdxBins / 6.28318530717958647692f));
    const int t0 = min(max(t - 1, 0), kIdxBins), t1 = min(max(t + 2, 0), kIdxBins);
    a = lo + tab[t0];
    b = lo + tab[t1];
}

// add the angle interval [u, v] (radians, v >= u, any branch), widened by
// 1e-4, as ranges of the bucket's sorted angles (which lie in [-pi, pi])
__device__ __forceinline__ void add_interval(Ranges& R, const float* th, const int32_t* tab, int64_t lo, int64_t hi,
                                             float u, float v) {
    const float twopi = 6.28318530717958647692f, pi = 3.14159265358979323846f;
    u -= 1e-4f;
    v += 1e-4f;
    if (!(v - u < twopi - 1e-3f)) {  // (also NaN) the whole bucket
        R.a[0] = lo;
        R.b[0] = hi;
        R.n = 1;
        return;
    }
    while (u < -pi) {
        u += twopi;
        v += twopi;
    }
    while (u >= pi) {
        u -= twopi;
        v -= twopi;
    }
    float iu[2], iv[2];
    int m = 1;
    iu[0] = u;
    iv[0] = v;
    if (v > pi) {  // wraps past +pi: [u, pi] and [-pi, v - 2 pi]
        iv[0] = pi + 1.0f;
        iu[1] = -pi - 1.0f;
        iv[1] = v - twopi;
        m = 2;
    }
    for (int t = 0; t < m && R.n < kIdxRanges; ++t) {
        int64_t wa, wb, va, vb;  // the two searches are independent: their loads overlap
        table_window(tab, lo, iu[t], wa, wb);
        table_window(tab, lo, iv[t], va, vb);
        const int64_t a = lower_theta(th, wa, wb, iu[t]);
        const int64_t b = upper_theta(th, va, vb, iv[t]);
        if (b > a) {
            R.a[R.n] = a;
            R.b[R.n] = b;
            ++R.n;
        }
    }
}

// the bin of one (hit, column) cell exactly as the scanning association
// computes it: nk for no vote
__device__ __forceinline__ unsigned cell_bin(float x, float y, float c, float s, float4 dt, const KConsts& K,
                                             unsigned long long* stats) {
    const HitFast hf = hit_fast(x, y, K);
    const float q = q_of(x, y, c, s);
    const float qs = q * K.S2;
    const float Rj = hf.r2 + dt.z;
    const S1 o = stage1_fast(qs, q, dt, Rj, hf.G, K.H, K.T0);
    const unsigned nk = (unsigned)K.nk;
    if (o.flo == o.fhi) return min(o.kb, nk);
    if (!stage1_pending(o, hf.dmin, K.wlo, K.whi)) return nk;
    const int ks = cell_slow(x, y, c, s, dt.x, hf.R1, K, stats);
    return ks >= 0 ? (unsigned)ks : nk;
}

__global__ void __launch_bounds__(kIdxWarps * 32) assoc_index_kernel(const AssocIndexParams P) {
    __shared__ uint32_t bitmap[kIdxWarps][kIdxCapWords];
    __shared__ int64_t rstart[kIdxWarps][32 * kIdxRanges + 1];  // flattened candidate ranges: prefix starts
    __shared__ int64_t rfrom[kIdxWarps][32 * kIdxRanges];
    const AssocParams& A = P.a;
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int64_t lo = *P.lo_dev;
    int64_t hi = *P.hi_dev;
    if (hi > A.peak_cap) hi = A.peak_cap;
    const int nl = P.nl, win = A.window;
    // blocks take chunks of consecutive peaks (same event, nearby columns),
    // warps the chunk's peaks in turn
    for (int64_t chunk = lo + (int64_t)blockIdx.x * kIdxChunk; chunk < hi; chunk += (int64_t)gridDim.x * kIdxChunk)
    for (int64_t p = chunk + wib; p < min(hi, chunk + kIdxChunk); p += kIdxWarps) {
        const ht_peak pk = P.peaks[p];
        const int e = pk.event, i = pk.i_phi, j = pk.i_d0, k = pk.i_kappa;
        const int64_t row0 = A.peak_offsets[p], nrow = A.peak_offsets[p + 1] - row0;
        const float c = A.cphi[i], s = A.sphi[i];
        const float4 dt = A.dtab[j];
        const float phi = atan2f(s, c);
        const float klo = P.kmin + (float)(k - win - 1) * P.dk, khi = P.kmin + (float)(k + win + 2) * P.dk;
        // this lane's layer: candidate ranges of its bucket
        Ranges R;
        R.n = 0;
        if (lane < nl) {
            const int64_t b = (int64_t)e * nl + lane;
            const int64_t blo = P.bstart[b], bhi = P.bstart[b + 1];
            if (bhi > blo) {
                const float rlo = sqrtf(__uint_as_float(P.r2min[b])) * (1.0f - 1e-5f);
                const float rhi = sqrtf(__uint_as_float(P.r2max[b])) * (1.0f + 1e-5f);
                float sl, sh;
                if (!s_range(rlo, rhi, dt.x, klo, khi, sl, sh) || (sl <= -1.0f && sh >= 1.0f)) {
                    R.a[0] = blo;
                    R.b[0] = bhi;
                    R.n = 1;
                } else if (!(sl > 1.0f || sh < -1.0f)) {
                    const float pi = 3.14159265358979323846f;
                    if (sh >= 1.0f) {
                        const float a0 = asinf(sl);
                        add_interval(R, P.theta, P.tab + b * (kIdxBins + 1), blo, bhi, phi + a0, phi + pi - a0);
                    } else if (sl <= -1.0f) {
                        const float b0 = asinf(sh);
                        add_interval(R, P.theta, P.tab + b * (kIdxBins + 1), blo, bhi, phi - pi - b0, phi + b0);
                    } else {
                        const float a0 = asinf(sl), b0 = asinf(sh);
                        add_interval(R, P.theta, P.tab + b * (kIdxBins + 1), blo, bhi, phi + a0, phi + b0);
                        add_interval(R, P.theta, P.tab + b * (kIdxBins + 1), blo, bhi, phi + pi - b0, phi + pi - a0);
                    }
                }
            }
        }
        // flatten the ranges of all lanes: lane l's ranges start at its prefix
        int64_t cnt = 0;
        for (int t = 0; t < R.n; ++t) cnt += R.b[t] - R.a[t];
        int64_t incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        const int64_t total = __shfl_sync(0xffffffffu, incl, 31);
        {
            int64_t at = incl - cnt;
            for (int t = 0; t < kIdxRanges; ++t) {
                rstart[wib][lane * kIdxRanges + t] = at;
                rfrom[wib][lane * kIdxRanges + t] = t < R.n ? R.a[t] : 0;
                if (t < R.n) at += R.b[t] - R.a[t];
            }
            if (lane == 31) rstart[wib][32 * kIdxRanges] = total;
        }
        __syncwarp();
        // segments of the event's hits, each marked in the bitmap and written
        const int h0 = A.offs[e], h1 = A.offs[e + 1];
        int64_t written = 0;
        for (int seg = h0; seg < h1; seg += 32 * kIdxCapWords) {
            const int nwords = min(kIdxCapWords, (h1 - seg + 31) >> 5);
            for (int w = lane; w < nwords; w += 32) bitmap[wib][w] = 0;
            __syncwarp();
            for (int64_t t0 = 0; t0 < total; t0 += 32) {
                const int64_t t = t0 + lane;
                if (t < total) {
                    // the range holding flattened position t (ranges with no
                    // candidates share a start; take the last of them)
                    int lo_r = 0, hi_r = 32 * kIdxRanges - 1;
                    while (lo_r < hi_r) {
                        const int m = (lo_r + hi_r + 1) >> 1;
                        if (rstart[wib][m] <= t) lo_r = m;
                        else hi_r = m - 1;
                    }
                    const int64_t pos = rfrom[wib][lo_r] + (t - rstart[wib][lo_r]);
                    const int h = P.hid[pos];
                    if (h >= seg && h < seg + 32 * kIdxCapWords) {
                        const unsigned kb = cell_bin(A.x[h], A.y[h], c, s, dt, A.K, A.stats);
                        if (kb < (unsigned)A.K.nk && abs((int)kb - k) <= win)
                            atomicOr(&bitmap[wib][(h - seg) >> 5], 1u << ((h - seg) & 31));
                    }
                }
            }
            __syncwarp();
            for (int w0 = 0; w0 < nwords; w0 += 32) {
                const int w = w0 + lane;
                uint32_t bits = w < nwords ? bitmap[wib][w] : 0u;
                const int n = __popc(bits);
                int ex = n;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int v = __shfl_up_sync(0xffffffffu, ex, o);
                    if (lane >= o) ex += v;
                }
                const int all = __shfl_sync(0xffffffffu, ex, 31);
                int64_t out = row0 + written + (ex - n);
                while (bits) {
                    const int bit = __ffs(bits) - 1;
                    bits &= bits - 1u;
                    if (out < A.pair_cap) A.hit_idx[out] = seg + (w << 5) + bit;
                    ++out;
                }
                written += all;
            }
            __syncwarp();
        }
        if (lane == 0 && written != nrow) atomicOr(P.err, 8);
    }
}

}  // namespace

cudaError_t launch_index_build(const IndexParams& p, cudaStream_t s) {
    if (p.n_events <= 0) return cudaSuccess;
    const int grid = (int)std::min<int64_t>(p.n_events, 152 * 8);
    index_count_kernel<<<grid, 256, 3 * p.nl * sizeof(uint32_t), s>>>(p);
    if (cudaError_t e = cudaGetLastError()) return e;
    ScanRange r{};
    r.in = p.bcount;
    r.out = p.bstart;
    r.lo = 0;
    r.hi = (int64_t)p.n_events * p.nl;
    r.cap = r.hi;
    r.write_end = 1;
    if (cudaError_t e = launch_scan(r, p.scratch, s)) return e;
    index_scatter_kernel<<<grid, 256, 0, s>>>(p);
    if (cudaError_t e = cudaGetLastError()) return e;
    const int64_t nb = (int64_t)p.n_events * p.nl;
    const int sgrid = (int)std::min<int64_t>(nb, 152 * 8);
    index_sort_kernel<<<sgrid, 256, kIdxSortCap * 8, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_assoc_index(const AssocIndexParams& p, cudaStream_t s) {
    assoc_index_kernel<<<152 * 8, kIdxWarps * 32, 0, s>>>(p);
    return cudaGetLastError();
}

}  // namespace ht
