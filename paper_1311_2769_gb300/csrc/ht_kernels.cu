// ht_kernels.cu — sm_103a kernels of the Hough-transform track finder.
//
// Section 4 of the paper observes that each hit's parameter-space computation
// is independent of every other hit.  The vote kernel maps that onto GB300 as
// (phi0, d0)-slab tiles: one CTA owns a tile of tile_phi x tile_d columns with
// all kappa bins in shared memory, streams every hit of the tile's event
// through it (one hit per thread, coalesced SoA loads), bins each (hit, column)
// with the certified float32 filter of ht_kbin.cuh and counts with shared
// atomics, then flushes the tile to HBM as uint32 rows (kappa contiguous).
// Batched launches are persistent: CTAs pull (event, tile) items from an
// atomic queue whose events are ordered largest first.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstdint>

#include "ht_internal.h"

namespace ht {

namespace {

__device__ __forceinline__ int64_t clamp64(int64_t v, int64_t lo, int64_t hi) {
    return v < lo ? lo : (v > hi ? hi : v);
}

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// ---------------------------------------------------------------------------
// vote
// ---------------------------------------------------------------------------
// Shared tile layout: [d0 column j][phi row r][kappa k], kappa contiguous, so
// a row's offset r * NK is a compile-time immediate of the atomic.

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared reduction when stage 1 certified a bin in range (flo == fhi and
// kb < n_kappa [and the lane holds a hit]); the test lives in the same PTX
// block so no branch or predicate round trip surrounds the atomic.
__device__ __forceinline__ void red_if_vote(uint32_t addr, float flo, float fhi, unsigned kb, unsigned nk) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.eq.f32 p, %1, %2;\n\tsetp.lt.and.u32 p, %3, %4, p;\n\t"
        "@p red.shared.add.u32 [%0], 1;\n\t}" ::"r"(addr),
        "f"(flo), "f"(fhi), "r"(kb), "r"(nk));
}
__device__ __forceinline__ void red_if_vote(uint32_t addr, float flo, float fhi, unsigned kb, unsigned nk,
                                            bool valid) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.eq.f32 p, %1, %2;\n\tsetp.lt.and.u32 p, %3, %4, p;\n\t"
        "setp.ne.and.u32 p, %5, 0, p;\n\t@p red.shared.add.u32 [%0], 1;\n\t}" ::"r"(addr),
        "f"(flo), "f"(fhi), "r"(kb), "r"(nk), "r"((unsigned)valid));
}

struct TileHit {
    float x, y;
    HitFast hf;
};

// One hit against every column of the tile.  TAIL: lanes past the event's
// last hit stay in the loop (the full-mask vote needs all 32) but are masked.
template <int SPHI, int NK, bool TAIL>
__device__ __forceinline__ void vote_one_hit(const VoteParams& p, const float* cp, const float* sp,
                                             const float4* dt_s, uint32_t* acc_s, uint32_t acc_sh, int nj, int nk,
                                             int64_t h, bool valid) {
    const float x = (!TAIL || valid) ? p.x[h] : 0.0f;
    const float y = (!TAIL || valid) ? p.y[h] : 0.0f;
    const HitFast hf = hit_fast(x, y, p.K);
    const float S2 = p.K.S2, H = p.K.H, T0 = p.K.T0;
    float q[SPHI], qs[SPHI];
#pragma unroll
    for (int r = 0; r < SPHI; ++r) {
        q[r] = q_of(x, y, cp[r], sp[r]);
        qs[r] = q[r] * S2;
    }
    const unsigned nku = (unsigned)nk;
    const int col_words = SPHI * nk;
    uint32_t col_sh = acc_sh;
    for (int j = 0; j < nj; ++j, col_sh += 4u * col_words) {
        const float4 dt = dt_s[j];
        const float Rj = hf.r2 + dt.z;
        bool und = false;
#pragma unroll
        for (int r = 0; r < SPHI; ++r) {
            const S1 o = stage1_fast(qs[r], q[r], dt, Rj, hf.G, H, T0);
            const uint32_t addr = col_sh + 4u * ((unsigned)(r * nk) + o.kb);
            if (TAIL) {
                red_if_vote(addr, o.flo, o.fhi, o.kb, nku, valid);
                und |= (o.flo != o.fhi) & valid;
            } else {
                red_if_vote(addr, o.flo, o.fhi, o.kb, nku);
                und |= o.flo != o.fhi;
            }
        }
        if (__any_sync(0xffffffffu, und)) {
#pragma unroll
            for (int r = 0; r < SPHI; ++r) {
                const S1 o = stage1_fast(qs[r], q[r], dt, Rj, hf.G, H, T0);
                if ((o.flo != o.fhi) && (!TAIL || valid) && stage1_pending(o, hf.dmin, p.K.wlo, p.K.whi)) {
                    const int kk = cell_slow(x, y, cp[r], sp[r], dt.x, hf.R1, p.K, p.stats);
                    if (kk >= 0) atomicAdd(acc_s + j * col_words + r * nk + kk, 1u);
                }
            }
        }
    }
}

template <int SPHI, int NK>
__global__ void __launch_bounds__(256, 3) vote_kernel(const VoteParams p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float4* dt_s = reinterpret_cast<float4*>(smem_raw);
    uint32_t* acc_s = reinterpret_cast<uint32_t*>(smem_raw + 16 * p.tile_d);
    __shared__ int s_item;

    const int nk = NK ? NK : p.K.nk;
    const int nthr = blockDim.x;
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int tiles = p.tiles_phi * p.tiles_d;
    const int col_words = SPHI * nk;
    const uint32_t acc_sh = smem_addr(acc_s);

    for (int it = 0;; ++it) {
        int item;
        if (p.queue) {
            if (tid == 0) s_item = atomicAdd(p.queue, 1);
            __syncthreads();
            item = s_item;
        } else {
            if (it > 0) break;
            item = p.item0 + blockIdx.x;
        }
        if (item >= p.n_items) break;
        const int el = item / tiles;
        const int t = item - el * tiles;
        const int e = p.order ? p.order[el] : el;
        const int tp = t / p.tiles_d;
        const int td = t - tp * p.tiles_d;
        const int i0 = tp * SPHI;
        const int j0 = td * p.tile_d;
        const int nj = min(p.tile_d, p.K.nd - j0);
        const int nrows = min(SPHI, p.K.nphi - i0);
        const int64_t hb = clamp64(p.offs[p.event0 + e], 0, p.n_hits);
        const int64_t he = clamp64(p.offs[p.event0 + e + 1], hb, p.n_hits);

        for (int w = tid; w < nj * col_words; w += nthr) acc_s[w] = 0u;
        for (int j = tid; j < nj; j += nthr) dt_s[j] = p.dtab[j0 + j];
        // rows past a ragged phi edge vote into tile slots that are never flushed
        float cp[SPHI], sp[SPHI];
#pragma unroll
        for (int r = 0; r < SPHI; ++r) {
            const int i = r < nrows ? i0 + r : i0;
            cp[r] = p.cphi[i];
            sp[r] = p.sphi[i];
        }
        if (p.stats && tid == 0) atomicAdd(&p.stats[0], (unsigned long long)((he - hb) * nrows * nj));
        __syncthreads();

        const int64_t nfull = ((he - hb) / nthr) * nthr;
        for (int64_t h = hb + tid; h < hb + nfull; h += nthr)
            vote_one_hit<SPHI, NK, false>(p, cp, sp, dt_s, acc_s, acc_sh, nj, nk, h, true);
        {
            const int64_t h = hb + nfull + tid;
            if (hb + nfull + (tid - lane) < he)  // warps with at least one hit left
                vote_one_hit<SPHI, NK, true>(p, cp, sp, dt_s, acc_s, acc_sh, nj, nk, h, h < he);
        }
        __syncthreads();

        uint32_t* dst_e = p.acc + (int64_t)e * p.cells;
        const int warp = tid >> 5, nw = nthr >> 5;
        const int nrj = nrows * nj;
        for (int row = warp; row < nrj; row += nw) {
            const int r = row / nj;
            const int j = row - r * nj;
            const uint32_t* src = acc_s + j * col_words + r * nk;
            uint32_t* dst = dst_e + ((int64_t)(i0 + r) * p.K.nd + (j0 + j)) * nk;
            if ((nk & 3) == 0) {
                const uint4* s4 = reinterpret_cast<const uint4*>(src);
                uint4* d4 = reinterpret_cast<uint4*>(dst);
                for (int kk = lane; kk < (nk >> 2); kk += 32) d4[kk] = s4[kk];
            } else {
                for (int kk = lane; kk < nk; kk += 32) dst[kk] = src[kk];
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// pruned vote: only the d0 band of each (hit, phi row) is evaluated
// ---------------------------------------------------------------------------
// Per chunk of blockDim hits: every thread computes its hit's band over the
// tile's rows (the union of the rows' d0_band) and files the hit into one of
// four buckets by band length (<= nj/8, nj/4, nj/2, nj).  Warps then take 32
// hits of one bucket at a time; each lane walks its own band from its own
// first column, the warp for as many steps as the longest band among its 32
// lanes, so lanes of a warp do similar amounts of work.  Cells outside every
// band cannot vote (they are out of the kappa range in binary64), so the
// accumulator is the same as the full vote's.
constexpr int kBuckets = 4;

template <int SPHI, int NK>
__global__ void __launch_bounds__(256, 3) vote_band_kernel(const VoteParams p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float4* dt_s = reinterpret_cast<float4*>(smem_raw);
    const int nthr = blockDim.x;
    // chunk records follow the d0 table; the accumulator tile follows them
    float* sx = reinterpret_cast<float*>(smem_raw + 16 * p.tile_d);
    float* sy = sx + nthr;
    int* sband = reinterpret_cast<int*>(sy + nthr);           // jlo | (len << 16)
    uint16_t* slist = reinterpret_cast<uint16_t*>(sband + nthr);  // [kBuckets][nthr]
    uint32_t* acc_s = reinterpret_cast<uint32_t*>(slist + kBuckets * nthr + (nthr & 1 ? 2 : 0));
    __shared__ int s_item;
    __shared__ int s_cnt[kBuckets];

    const int nk = NK ? NK : p.K.nk;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = nthr >> 5;
    const int tiles = p.tiles_phi * p.tiles_d;
    const int col_words = SPHI * nk;
    const uint32_t acc_sh = smem_addr(acc_s);
    const float S2 = p.K.S2, H = p.K.H, T0 = p.K.T0;
    const unsigned nku = (unsigned)nk;

    for (int it = 0;; ++it) {
        int item;
        if (p.queue) {
            if (tid == 0) s_item = atomicAdd(p.queue, 1);
            __syncthreads();
            item = s_item;
        } else {
            if (it > 0) break;
            item = p.item0 + blockIdx.x;
        }
        if (item >= p.n_items) break;
        const int el = item / tiles;
        const int t = item - el * tiles;
        const int e = p.order ? p.order[el] : el;
        const int tp = t / p.tiles_d;
        const int td = t - tp * p.tiles_d;
        const int i0 = tp * SPHI;
        const int j0 = td * p.tile_d;
        const int nj = min(p.tile_d, p.K.nd - j0);
        const int nrows = min(SPHI, p.K.nphi - i0);
        const int64_t hb = clamp64(p.offs[p.event0 + e], 0, p.n_hits);
        const int64_t he = clamp64(p.offs[p.event0 + e + 1], hb, p.n_hits);

        for (int w = tid; w < nj * col_words; w += nthr) acc_s[w] = 0u;
        for (int j = tid; j < nj; j += nthr) dt_s[j] = p.dtab[j0 + j];
        float cp[SPHI], sp[SPHI];
#pragma unroll
        for (int r = 0; r < SPHI; ++r) {
            const int i = r < nrows ? i0 + r : i0;
            cp[r] = p.cphi[i];
            sp[r] = p.sphi[i];
        }
        const float dlo = p.dtab[j0].x, dhi = p.dtab[j0 + nj - 1].x;
        int lim[kBuckets];
        lim[0] = max(1, nj / 8);
        lim[1] = max(1, nj / 4);
        lim[2] = max(1, nj / 2);
        lim[3] = nj;
        if (p.stats && tid == 0) atomicAdd(&p.stats[0], (unsigned long long)((he - hb) * nrows * nj));

        for (int64_t cb = hb; cb < he; cb += nthr) {
            if (tid < kBuckets) s_cnt[tid] = 0;
            __syncthreads();
            // phase 1: band of this thread's hit over the tile's rows, filed by length
            const int64_t h = cb + tid;
            int jlo = j0 + nj, jhi = j0 - 1;
            float x = 0.0f, y = 0.0f;
            if (h < he) {
                x = p.x[h];
                y = p.y[h];
                if (p.K.band_ok) {
                    const float r2 = fmaf(x, x, __fmul_rn(y, y));
#pragma unroll
                    for (int r = 0; r < SPHI; ++r) {
                        if (r >= nrows) break;
                        int a, b;
                        d0_band(r2, q_of(x, y, cp[r], sp[r]), dlo, dhi, j0, nj, p.K, a, b);
                        if (b >= a) {
                            jlo = min(jlo, a);
                            jhi = max(jhi, b);
                        }
                    }
                } else {
                    jlo = j0;
                    jhi = j0 + nj - 1;
                }
            }
            const int len = jhi >= jlo ? jhi - jlo + 1 : 0;
            sx[tid] = x;
            sy[tid] = y;
            sband[tid] = (jlo - j0) | (len << 16);
#pragma unroll
            for (int bk = 0; bk < kBuckets; ++bk) {
                const bool in = len > 0 && len <= lim[bk] && (bk == 0 || len > lim[bk - 1]);
                const unsigned m = __ballot_sync(0xffffffffu, in);
                int base = 0;
                if (lane == 0 && m) base = atomicAdd(&s_cnt[bk], __popc(m));
                base = __shfl_sync(0xffffffffu, base, 0);
                if (in) slist[bk * nthr + base + __popc(m & lanemask_lt())] = (uint16_t)tid;
            }
            __syncthreads();
            // phase 2: warps take 32 hits of one bucket at a time
            int groups = 0;
            int gstart[kBuckets + 1];
#pragma unroll
            for (int bk = 0; bk < kBuckets; ++bk) {
                gstart[bk] = groups;
                groups += (s_cnt[bk] + 31) >> 5;
            }
            gstart[kBuckets] = groups;
            for (int g = warp; g < groups; g += nw) {
                int bk = 0;
#pragma unroll
                for (int b2 = 1; b2 < kBuckets; ++b2) bk += g >= gstart[b2];
                const int idx = (g - gstart[bk]) * 32 + lane;
                const bool has = idx < s_cnt[bk];
                const int ht = has ? slist[bk * nthr + idx] : 0;
                const int bd = has ? sband[ht] : 0;
                const int jl = bd & 0xFFFF, ln = bd >> 16;
                const float hx = sx[ht], hy = sy[ht];
                const HitFast hf = hit_fast(hx, hy, p.K);
                float q[SPHI], qs[SPHI];
#pragma unroll
                for (int r = 0; r < SPHI; ++r) {
                    q[r] = q_of(hx, hy, cp[r], sp[r]);
                    qs[r] = q[r] * S2;
                }
                const int steps = __reduce_max_sync(0xffffffffu, ln);
                for (int s = 0; s < steps; ++s) {
                    const bool live = s < ln;
                    const int j = live ? jl + s : 0;
                    const float4 dt = dt_s[j];
                    const float Rj = hf.r2 + dt.z;
                    const uint32_t col_sh = acc_sh + 4u * (unsigned)(j * col_words);
                    bool und = false;
#pragma unroll
                    for (int r = 0; r < SPHI; ++r) {
                        const S1 o = stage1_fast(qs[r], q[r], dt, Rj, hf.G, H, T0);
                        red_if_vote(col_sh + 4u * ((unsigned)(r * nk) + o.kb), o.flo, o.fhi, o.kb, nku, live);
                        und |= (o.flo != o.fhi) & live;
                    }
                    if (__any_sync(0xffffffffu, und)) {
#pragma unroll
                        for (int r = 0; r < SPHI; ++r) {
                            const S1 o = stage1_fast(qs[r], q[r], dt, Rj, hf.G, H, T0);
                            if ((o.flo != o.fhi) && live && stage1_pending(o, hf.dmin, p.K.wlo, p.K.whi)) {
                                const int kk = cell_slow(hx, hy, cp[r], sp[r], dt.x, hf.R1, p.K, p.stats);
                                if (kk >= 0) atomicAdd(acc_s + j * col_words + r * nk + kk, 1u);
                            }
                        }
                    }
                }
            }
            __syncthreads();
        }

        uint32_t* dst_e = p.acc + (int64_t)e * p.cells;
        const int nrj = nrows * nj;
        for (int row = warp; row < nrj; row += nw) {
            const int r = row / nj;
            const int j = row - r * nj;
            const uint32_t* src = acc_s + j * col_words + r * nk;
            uint32_t* dst = dst_e + ((int64_t)(i0 + r) * p.K.nd + (j0 + j)) * nk;
            if ((nk & 3) == 0) {
                const uint4* s4 = reinterpret_cast<const uint4*>(src);
                uint4* d4 = reinterpret_cast<uint4*>(dst);
                for (int kk = lane; kk < (nk >> 2); kk += 32) d4[kk] = s4[kk];
            } else {
                for (int kk = lane; kk < nk; kk += 32) dst[kk] = src[kk];
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// input validation (device-resident batches)
// bit 1: non-finite or |coordinate| > 1e4; bit 2: layer out of range; bit 4: offsets
// ---------------------------------------------------------------------------
__global__ void validate_kernel(const float* x, const float* y, const int8_t* layer, int64_t n_hits,
                                const int32_t* offs, int32_t n_events, int32_t n_layers, int32_t* err) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int bad = 0;
    for (int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; h < n_hits; h += stride) {
        const float xv = x[h], yv = y[h];
        if (!(fabsf(xv) <= 1.0e4f) || !(fabsf(yv) <= 1.0e4f)) bad |= 1;
        if (layer) {
            const int l = layer[h];
            if (l < 0 || l >= n_layers) bad |= 2;
        }
    }
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n_events; e += stride) {
        if (offs[e] > offs[e + 1]) bad |= 4;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (offs[0] != 0 || (int64_t)offs[n_events] != n_hits) bad |= 4;
    }
    if (bad) atomicOr(err, bad);
}

// ---------------------------------------------------------------------------
// event order: counting sort by size class (floor(log2(hits))), largest first
// ---------------------------------------------------------------------------
__global__ void order_kernel(const int32_t* offs, int32_t event0, int32_t n_events, int64_t n_hits,
                             int32_t* order) {
    __shared__ int hist[33];
    __shared__ int start[33];
    if (threadIdx.x < 33) hist[threadIdx.x] = 0;
    __syncthreads();
    for (int e = threadIdx.x; e < n_events; e += blockDim.x) {
        const int64_t a = clamp64(offs[event0 + e], 0, n_hits);
        const int64_t b = clamp64(offs[event0 + e + 1], a, n_hits);
        const int cls = 32 - __clz((unsigned)(b - a));
        atomicAdd(&hist[32 - cls], 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        for (int c = 0; c < 33; ++c) {
            start[c] = run;
            run += hist[c];
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < n_events; e += blockDim.x) {
        const int64_t a = clamp64(offs[event0 + e], 0, n_hits);
        const int64_t b = clamp64(offs[event0 + e + 1], a, n_hits);
        const int cls = 32 - __clz((unsigned)(b - a));
        order[atomicAdd(&start[32 - cls], 1)] = e;
    }
}

// ---------------------------------------------------------------------------
// peaks: detection (warp per (event, phi0, d0) column, lanes over kappa)
// ---------------------------------------------------------------------------
// A CTA stages rows i0-1 .. i0+R (phi wraps) x columns j0-1 .. j0+TD of one
// event in shared memory, cells outside the d0 range marked absent, and tests
// every interior cell at or above the threshold against its 26 neighbours
// with the linear-order tie rule, leaving at the first failure.
constexpr uint32_t kAbsent = 0xFFFFFFFFu;

__global__ void __launch_bounds__(512) detect_kernel(const PeakParams p, const int R, const int TD) {
    extern __shared__ __align__(16) uint32_t tile[];
    const int nk = p.nk, nkw = p.nkw;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int tcols = TD + 2;
    const int tiles_i = (p.nphi + R - 1) / R, tiles_j = (p.nd + TD - 1) / TD;
    const int64_t items = (int64_t)p.n_events * tiles_i * tiles_j;
    for (int64_t item = blockIdx.x; item < items; item += gridDim.x) {
        const int e = (int)(item / ((int64_t)tiles_i * tiles_j));
        const int t = (int)(item - (int64_t)e * tiles_i * tiles_j);
        const int ti = t / tiles_j, tj = t - (t / tiles_j) * tiles_j;
        const int i0 = ti * R, j0 = tj * TD;
        const int nr = min(R, p.nphi - i0), nj = min(TD, p.nd - j0);
        const uint32_t* A = p.acc + (int64_t)e * p.cells;
        __syncthreads();
        // stage (nr + 2) x (nj + 2) columns
        const int ncolumns = (nr + 2) * (nj + 2);
        for (int cc = warp; cc < ncolumns; cc += nw) {
            const int ri = cc / (nj + 2), cj = cc - (cc / (nj + 2)) * (nj + 2);
            int ii = i0 - 1 + ri;
            ii = ((ii % p.nphi) + p.nphi) % p.nphi;
            const int jj = j0 - 1 + cj;
            uint32_t* dst = tile + ((int64_t)ri * tcols + cj) * nk;
            if (jj < 0 || jj >= p.nd) {
                for (int kk = lane; kk < nk; kk += 32) dst[kk] = kAbsent;
            } else {
                const uint32_t* src = A + ((int64_t)ii * p.nd + jj) * nk;
                if ((nk & 3) == 0) {
                    const uint4* s4 = reinterpret_cast<const uint4*>(src);
                    uint4* d4 = reinterpret_cast<uint4*>(dst);
                    for (int kk = lane; kk < (nk >> 2); kk += 32) d4[kk] = s4[kk];
                } else {
                    for (int kk = lane; kk < nk; kk += 32) dst[kk] = src[kk];
                }
            }
        }
        __syncthreads();
        // interior columns: warp per (row, column), lanes over kappa.  Every lane
        // reads its 3x3x3 box (absent neighbours read as -1 in int32, so they
        // never reject) and compares against the maximum of the neighbours that
        // precede it in linear order (strictly) and of those that follow it.
        for (int cc = warp; cc < nr * nj; cc += nw) {
            const int r = cc / nj, j = cc - (cc / nj) * nj;
            const int i = i0 + r;
            const int64_t col = ((int64_t)e * p.nphi + i) * p.nd + (j0 + j);
            // row di = -1 / +1 precedes row i unless the phi wrap makes it follow
            // (one row only: those rows are the row itself, covered by di = 0)
            const bool single = p.nphi == 1;
            const bool m_earlier = i > 0, p_earlier = i == p.nphi - 1;
            int count = 0;
            for (int k0 = 0, w = 0; k0 < nk; k0 += 32, ++w) {
                const int kk = k0 + lane;
                bool pk = false;
                if (kk < nk) {
                    const int v = (int)tile[((int64_t)(r + 1) * tcols + (j + 1)) * nk + kk];
                    int mE = -1, mL = -1;
#pragma unroll
                    for (int di = -1; di <= 1; ++di) {
                        if (single && di != 0) continue;
                        const int* rowp = reinterpret_cast<const int*>(tile) + ((int64_t)(r + 1 + di) * tcols) * nk;
#pragma unroll
                        for (int dj = -1; dj <= 1; ++dj) {
                            const int* cp2 = rowp + (j + 1 + dj) * nk;
                            const int u0 = cp2[kk];
                            const int um = kk > 0 ? cp2[kk - 1] : -1;
                            const int up = kk + 1 < nk ? cp2[kk + 1] : -1;
                            if (di == 0) {
                                if (dj < 0) {
                                    mE = max(mE, max(u0, max(um, up)));
                                } else if (dj > 0) {
                                    mL = max(mL, max(u0, max(um, up)));
                                } else {
                                    mE = max(mE, um);
                                    mL = max(mL, up);
                                }
                            } else {
                                const int m3 = max(u0, max(um, up));
                                const bool earlier = di < 0 ? m_earlier : p_earlier;
                                if (earlier) mE = max(mE, m3);
                                else mL = max(mL, m3);
                            }
                        }
                    }
                    pk = (uint32_t)v >= p.thr && v > mE && v >= mL;
                }
                const unsigned b = __ballot_sync(0xffffffffu, pk);
                if (lane == 0) {
                    p.mask[col * nkw + w] = b;
                    p.wpre[col * nkw + w] = (uint16_t)count;
                }
                count += __popc(b);
            }
            if (lane == 0) p.npk[col] = count;
        }
    }
}

// peaks: emission in (event, linear index) order + per-peak pair counts
__global__ void emit_kernel(const PeakParams p) {
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwt = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t per_ev = (int64_t)p.nphi * p.nd;
    const int64_t ncols = per_ev * p.n_events;
    for (int64_t col = gw; col < ncols; col += nwt) {
        if (p.npk[col] == 0) continue;
        const int64_t base = p.colbase[col];
        if (base >= p.peak_cap && p.window < 0) continue;
        const int e = (int)(col / per_ev);
        const int ij = (int)(col - e * per_ev);
        const int i = ij / p.nd;
        const int j = ij - i * p.nd;
        const uint32_t* colp = p.acc + (int64_t)e * p.cells + ((int64_t)i * p.nd + j) * p.nk;
        for (int w = 0; w < p.nkw; ++w) {
            const unsigned m = p.mask[col * p.nkw + w];
            if (!m) continue;
            if (!((m >> lane) & 1u)) continue;
            const int k = w * 32 + lane;
            const int64_t pid = base + p.wpre[col * p.nkw + w] + __popc(m & lanemask_lt());
            if (pid >= p.peak_cap) {
                if (p.window >= 0 && p.extra_pairs) {
                    const int lo = max(0, k - p.window), hi = min(p.nk - 1, k + p.window);
                    unsigned long long s = 0;
                    for (int kk = lo; kk <= hi; ++kk) s += colp[kk];
                    atomicAdd(reinterpret_cast<unsigned long long*>(p.extra_pairs), s);
                }
                continue;
            }
            ht_peak pk;
            pk.event = p.event0 + e;
            pk.i_phi = i;
            pk.i_d0 = j;
            pk.i_kappa = k;
            pk.votes = colp[k];
            p.peaks[pid] = pk;
            if (p.window >= 0) {
                const int lo = max(0, k - p.window), hi = min(p.nk - 1, k + p.window);
                uint32_t s = 0;
                for (int kk = lo; kk <= hi; ++kk) s += colp[kk];
                p.paircnt[pid] = (int32_t)s;
            }
        }
    }
}

// per-peak pair counts for peaks [lo, hi) already emitted (separate ht_associate)
__global__ void paircount_kernel(const PeakParams p, const int64_t* lo_dev, const int64_t* hi_dev) {
    const int64_t lo = *lo_dev;
    const int64_t hi = min(*hi_dev, p.peak_cap);
    for (int64_t pid = lo + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; pid < hi;
         pid += (int64_t)gridDim.x * blockDim.x) {
        const ht_peak pk = p.peaks[pid];
        const int e = pk.event - p.event0;
        const uint32_t* colp = p.acc + (int64_t)e * p.cells + ((int64_t)pk.i_phi * p.nd + pk.i_d0) * p.nk;
        const int lo_k = max(0, pk.i_kappa - p.window), hi_k = min(p.nk - 1, pk.i_kappa + p.window);
        uint32_t s = 0;
        for (int kk = lo_k; kk <= hi_k; ++kk) s += colp[kk];
        p.paircnt[pid] = (int32_t)s;
    }
}

// ---------------------------------------------------------------------------
// scan (reduce, spine, down-sweep over contiguous per-block segments)
// ---------------------------------------------------------------------------
// [lo, hi) clamped to [0, cap]: both ends, so that out[hi] (write_end) stays
// inside an output of cap + 1 entries even when a whole wave lies past the cap
__device__ void scan_bounds(const ScanRange& r, int64_t& lo, int64_t& hi) {
    lo = r.lo_dev ? *r.lo_dev : r.lo;
    hi = r.hi_dev ? *r.hi_dev : r.hi;
    if (lo > r.cap) lo = r.cap;
    if (lo < 0) lo = 0;
    if (hi > r.cap) hi = r.cap;
    if (hi < lo) hi = lo;
}

__device__ __forceinline__ int64_t block_sum64(int64_t v, int64_t* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    int64_t t = 0;
    if (threadIdx.x == 0) {
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
        sh[32] = t;
    }
    __syncthreads();
    return sh[32];
}

// exclusive block scan; returns the exclusive prefix of this thread, *total = block sum
__device__ __forceinline__ int64_t block_exscan64(int64_t v, int64_t* sh, int64_t* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int64_t incl = v;
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t n = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += n;
    }
    __syncthreads();
    if (lane == 31) sh[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int64_t ws = lane < nw ? sh[lane] : 0;
        int64_t wi = ws;
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t n = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += n;
        }
        if (lane < nw) sh[lane] = wi - ws;
        if (lane == 31) sh[32] = wi;
    }
    __syncthreads();
    *total = sh[32];
    return sh[warp] + incl - v;
}

__global__ void scan_reduce_kernel(const ScanRange r, int64_t* partial) {
    __shared__ int64_t sh[33];
    int64_t lo, hi;
    scan_bounds(r, lo, hi);
    const int64_t n = hi - lo;
    const int64_t seg = (n + gridDim.x - 1) / gridDim.x;
    const int64_t a = lo + min(n, seg * blockIdx.x), b = lo + min(n, seg * (blockIdx.x + 1));
    int64_t s = 0;
    for (int64_t i = a + threadIdx.x; i < b; i += blockDim.x) s += r.in[i];
    s = block_sum64(s, sh);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void scan_spine_kernel(const ScanRange r, int64_t* partial, int nblocks) {
    __shared__ int64_t sh[33];
    int64_t lo, hi;
    scan_bounds(r, lo, hi);
    const int64_t base = r.base_dev ? *r.base_dev : r.base;
    int64_t carry = base;
    for (int c = 0; c < nblocks; c += blockDim.x) {
        const int idx = c + threadIdx.x;
        const int64_t v = idx < nblocks ? partial[idx] : 0;
        int64_t tot;
        const int64_t ex = block_exscan64(v, sh, &tot);
        if (idx < nblocks) partial[nblocks + idx] = carry + ex;
        carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (r.total) *r.total = carry;
        if (r.write_end) r.out[hi] = carry;
    }
}

__global__ void scan_down_kernel(const ScanRange r, const int64_t* partial, int nblocks) {
    __shared__ int64_t sh[33];
    int64_t lo, hi;
    scan_bounds(r, lo, hi);
    const int64_t n = hi - lo;
    const int64_t seg = (n + gridDim.x - 1) / gridDim.x;
    const int64_t a = lo + min(n, seg * blockIdx.x), b = lo + min(n, seg * (blockIdx.x + 1));
    int64_t carry = partial[nblocks + blockIdx.x];
    for (int64_t c = a; c < b; c += blockDim.x) {
        const int64_t i = c + threadIdx.x;
        const int64_t v = i < b ? r.in[i] : 0;
        int64_t tot;
        const int64_t ex = block_exscan64(v, sh, &tot);
        if (i < b) r.out[i] = carry + ex;
        carry += tot;
    }
}

// ---------------------------------------------------------------------------
// association: the vote's tiling again.  A CTA owns a (phi0, d0) tile of one
// event, loads the tile's peak bitmasks, marks the kappa bins that lie within
// `window` of a peak ("near" bits), and streams the event's hits through the
// same certified binning as the vote.  A hit whose bin is near a peak is
// appended to each such peak's CSR row through a shared-memory cursor; rows
// are then put in ascending hit order (most already are) by a warp rank sort.
// ---------------------------------------------------------------------------
constexpr int kSortCap = 1024;  // per-warp shared sort buffer (hit indices)
constexpr int kQueue = 64;      // per-warp candidate queue (drained at >= 32)

struct AssocSmem {
    float4* dt;        // [tile_d]
    uint32_t* mask;    // [tile_cols][nkw] peak bits
    uint32_t* nearb;   // [tile_cols][nkw] near-peak bits
    int32_t* lpre;     // [tile_cols][nkw] first local peak slot of the word
    int64_t* gpre;     // [tile_cols][nkw] first global peak id of the word
    unsigned long long* wpos;  // [tile_cols * ceil(nk/2)] next CSR write position per local peak
    uint2* queue;      // [warps][kQueue] (column << 16 | kappa bin, hit)
    int32_t* sortbuf;  // [warps][kSortCap]
    int32_t* active;   // [tile_d] d0 columns of the tile holding any peak
    float* sx;         // [threads] band bucketing records of the current hit chunk
    float* sy;
    int* sband;
    uint16_t* slist;   // [kBuckets][threads]
    int* cnt;          // [kBuckets] bucket fill counts
};

__host__ __device__ inline size_t assoc_smem_bytes(int tile_phi, int tile_d, int nk, int threads, bool band) {
    const size_t cols = (size_t)tile_phi * tile_d, nkw = (nk + 31) / 32;
    return 16 * (size_t)tile_d + cols * nkw * (4 + 4 + 4 + 8) + cols * ((nk + 1) / 2) * 8 +
           (size_t)(threads / 32) * (kQueue * 8 + kSortCap * 4) + 4 * (size_t)tile_d +
           (band ? (size_t)threads * (4 + 4 + 4 + 2 * kBuckets) : 0) + 64;
}

// One queued candidate (column c of the tile, kappa bin kb, hit h): append h
// to every peak within `window` bins of kb.
__device__ __forceinline__ void assoc_append(const AssocParams& p, const AssocSmem& S, int nkw, int nk, uint2 ent) {
    const int c = (int)(ent.x >> 16), kb = (int)(ent.x & 0xFFFFu);
    for (int o = -p.window; o <= p.window; ++o) {
        const int kk = kb + o;
        if (kk < 0 || kk >= nk) continue;
        const int wd = kk >> 5;
        const uint32_t bits = S.mask[c * nkw + wd];
        if (!((bits >> (kk & 31)) & 1u)) continue;
        const int below = __popc(bits & ((1u << (kk & 31)) - 1u));
        const int64_t pid = S.gpre[c * nkw + wd] + below;
        if (pid >= p.peak_cap) continue;
        const unsigned long long pos = atomicAdd(&S.wpos[S.lpre[c * nkw + wd] + below], 1ull);
        if ((int64_t)pos < p.pair_cap) p.hit_idx[pos] = (int32_t)ent.y;
    }
}

// Push this lane's candidate (if any) into the warp queue; drain 32 at a time.
__device__ __forceinline__ void queue_push(const AssocParams& p, const AssocSmem& S, uint2* q, int& qn, int nkw,
                                           int nk, bool cand, uint2 ent, int lane) {
    const unsigned m = __ballot_sync(0xffffffffu, cand);
    if (!m) return;
    if (cand) q[qn + __popc(m & lanemask_lt())] = ent;
    qn += __popc(m);
    if (qn >= 32) {
        __syncwarp();
        assoc_append(p, S, nkw, nk, q[qn - 32 + lane]);
        __syncwarp();
        qn -= 32;
    }
}

__device__ __forceinline__ void queue_drain(const AssocParams& p, const AssocSmem& S, uint2* q, int& qn, int nkw,
                                            int nk, int lane) {
    __syncwarp();
    if (lane < qn) assoc_append(p, S, nkw, nk, q[lane]);
    __syncwarp();
    qn = 0;
}

template <int SPHI, int NK, bool TAIL>
__device__ __forceinline__ void assoc_one_hit(const AssocParams& p, const AssocSmem& S, uint2* q, int& qn,
                                              const float* cp, const float* sp, int n_active, int nk, int nkw,
                                              int64_t h, bool valid, int lane) {
    const float x = (!TAIL || valid) ? p.x[h] : 0.0f;
    const float y = (!TAIL || valid) ? p.y[h] : 0.0f;
    const HitFast hf = hit_fast(x, y, p.K);
    const float S2 = p.K.S2, H = p.K.H, T0 = p.K.T0;
    float q_[SPHI], qs[SPHI];
#pragma unroll
    for (int r = 0; r < SPHI; ++r) {
        q_[r] = q_of(x, y, cp[r], sp[r]);
        qs[r] = q_[r] * S2;
    }
    const unsigned nku = (unsigned)nk;
    for (int ja = 0; ja < n_active; ++ja) {
        const int j = S.active[ja];
        const float4 dt = S.dt[j];
        const float Rj = hf.r2 + dt.z;
        bool und = false;
#pragma unroll
        for (int r = 0; r < SPHI; ++r) {
            const int c = j * SPHI + r;
            const S1 o = stage1_fast(qs[r], q_[r], dt, Rj, hf.G, H, T0);
            bool vote = (o.flo == o.fhi) & (o.kb < nku);
            if (TAIL) vote &= valid;
            // kb is only meaningful (< n_kappa) when vote; other lanes read word 0
            const uint32_t nb = S.nearb[c * nkw + (vote ? (o.kb >> 5) : 0u)];
            const bool cand = vote && ((nb >> (o.kb & 31)) & 1u);
            queue_push(p, S, q, qn, nkw, nk, cand, make_uint2(((unsigned)c << 16) | o.kb, (unsigned)h), lane);
            und |= (o.flo != o.fhi) & (!TAIL || valid);
        }
        if (__any_sync(0xffffffffu, und)) {
#pragma unroll
            for (int r = 0; r < SPHI; ++r) {
                const int c = j * SPHI + r;
                const S1 o = stage1_fast(qs[r], q_[r], dt, Rj, hf.G, H, T0);
                int kk = -1;
                if ((o.flo != o.fhi) && (!TAIL || valid) && stage1_pending(o, hf.dmin, p.K.wlo, p.K.whi))
                    kk = cell_slow(x, y, cp[r], sp[r], dt.x, hf.R1, p.K, p.stats);
                const bool cand = kk >= 0 && ((S.nearb[c * nkw + (kk >> 5)] >> (kk & 31)) & 1u);
                queue_push(p, S, q, qn, nkw, nk, cand, make_uint2(((unsigned)c << 16) | (unsigned)kk, (unsigned)h),
                           lane);
            }
        }
    }
}

// Association over d0 bands: the vote's bucketing (see vote_band_kernel),
// bands clipped to the tile's columns [ja, ja + nja) that hold peaks.
template <int SPHI, int NK>
__device__ __forceinline__ void assoc_band_hits(const AssocParams& p, const AssocSmem& S, uint2* q, int& qn,
                                                const float* cp, const float* sp, int ja, int nja, int j0,
                                                int nrows, int nk, int nkw, int64_t hb, int64_t he, int lane) {
    const int nthr = blockDim.x, tid = threadIdx.x, warp = tid >> 5, nw = nthr >> 5;
    const float S2 = p.K.S2, H = p.K.H, T0 = p.K.T0;
    const unsigned nku = (unsigned)nk;
    const float dlo = S.dt[ja - j0].x, dhi = S.dt[ja - j0 + nja - 1].x;
    int lim[kBuckets];
    lim[0] = max(1, nja / 8);
    lim[1] = max(1, nja / 4);
    lim[2] = max(1, nja / 2);
    lim[3] = nja;
    for (int64_t cb = hb; cb < he; cb += nthr) {
        if (tid < kBuckets) S.cnt[tid] = 0;
        __syncthreads();
        const int64_t h = cb + tid;
        int jlo = ja + nja, jhi = ja - 1;
        float x = 0.0f, y = 0.0f;
        if (h < he) {
            x = p.x[h];
            y = p.y[h];
            const float r2 = fmaf(x, x, __fmul_rn(y, y));
#pragma unroll
            for (int r = 0; r < SPHI; ++r) {
                if (r >= nrows) break;
                int a, b;
                d0_band(r2, q_of(x, y, cp[r], sp[r]), dlo, dhi, ja, nja, p.K, a, b);
                if (b >= a) {
                    jlo = min(jlo, a);
                    jhi = max(jhi, b);
                }
            }
        }
        const int len = jhi >= jlo ? jhi - jlo + 1 : 0;
        S.sx[tid] = x;
        S.sy[tid] = y;
        S.sband[tid] = (jlo - j0) | (len << 16);
#pragma unroll
        for (int bk = 0; bk < kBuckets; ++bk) {
            const bool in = len > 0 && len <= lim[bk] && (bk == 0 || len > lim[bk - 1]);
            const unsigned m = __ballot_sync(0xffffffffu, in);
            int base = 0;
            if (lane == 0 && m) base = atomicAdd(&S.cnt[bk], __popc(m));
            base = __shfl_sync(0xffffffffu, base, 0);
            if (in) S.slist[bk * nthr + base + __popc(m & lanemask_lt())] = (uint16_t)tid;
        }
        __syncthreads();
        int groups = 0;
        int gstart[kBuckets + 1];
#pragma unroll
        for (int bk = 0; bk < kBuckets; ++bk) {
            gstart[bk] = groups;
            groups += (S.cnt[bk] + 31) >> 5;
        }
        gstart[kBuckets] = groups;
        for (int g = warp; g < groups; g += nw) {
            int bk = 0;
#pragma unroll
            for (int b2 = 1; b2 < kBuckets; ++b2) bk += g >= gstart[b2];
            const int idx = (g - gstart[bk]) * 32 + lane;
            const bool has = idx < S.cnt[bk];
            const int ht = has ? S.slist[bk * nthr + idx] : 0;
            const int bd = has ? S.sband[ht] : 0;
            const int jl = bd & 0xFFFF, ln = bd >> 16;
            const float hx = S.sx[ht], hy = S.sy[ht];
            const int64_t hh = cb + ht;
            const HitFast hf = hit_fast(hx, hy, p.K);
            float q_[SPHI], qs[SPHI];
#pragma unroll
            for (int r = 0; r < SPHI; ++r) {
                q_[r] = q_of(hx, hy, cp[r], sp[r]);
                qs[r] = q_[r] * S2;
            }
            const int steps = __reduce_max_sync(0xffffffffu, ln);
            for (int s = 0; s < steps; ++s) {
                const bool live = s < ln;
                const int j = live ? jl + s : ja - j0;
                const float4 dt = S.dt[j];
                const float Rj = hf.r2 + dt.z;
                bool und = false;
#pragma unroll
                for (int r = 0; r < SPHI; ++r) {
                    const int c = j * SPHI + r;
                    const S1 o = stage1_fast(qs[r], q_[r], dt, Rj, hf.G, H, T0);
                    const bool vote = live & (o.flo == o.fhi) & (o.kb < nku);
                    const uint32_t nb = S.nearb[c * nkw + (vote ? (o.kb >> 5) : 0u)];
                    const bool cand = vote && ((nb >> (o.kb & 31)) & 1u);
                    queue_push(p, S, q, qn, nkw, nk, cand, make_uint2(((unsigned)c << 16) | o.kb, (unsigned)hh), lane);
                    und |= (o.flo != o.fhi) & live;
                }
                if (__any_sync(0xffffffffu, und)) {
#pragma unroll
                    for (int r = 0; r < SPHI; ++r) {
                        const int c = j * SPHI + r;
                        const S1 o = stage1_fast(qs[r], q_[r], dt, Rj, hf.G, H, T0);
                        int kk = -1;
                        if ((o.flo != o.fhi) && live && stage1_pending(o, hf.dmin, p.K.wlo, p.K.whi))
                            kk = cell_slow(hx, hy, cp[r], sp[r], dt.x, hf.R1, p.K, p.stats);
                        const bool cand = kk >= 0 && ((S.nearb[c * nkw + (kk >> 5)] >> (kk & 31)) & 1u);
                        queue_push(p, S, q, qn, nkw, nk, cand,
                                   make_uint2(((unsigned)c << 16) | (unsigned)kk, (unsigned)hh), lane);
                    }
                }
            }
        }
        __syncthreads();
    }
}

// Ascending order of one CSR row (distinct hit indices) by rank sort.
__device__ void sort_row(int32_t* seg, int n, int32_t* buf, int lane) {
    if (n <= 1) return;
    if (n > kSortCap) {  // rare: long rows sorted in place by one lane
        if (lane == 0) {
            for (int a = 1; a < n; ++a) {
                const int32_t v = seg[a];
                int b = a - 1;
                while (b >= 0 && seg[b] > v) {
                    seg[b + 1] = seg[b];
                    --b;
                }
                seg[b + 1] = v;
            }
        }
        __syncwarp();
        return;
    }
    bool unsorted = false;
    for (int t = lane; t < n; t += 32) {
        buf[t] = seg[t];
        if (t + 1 < n) unsorted |= seg[t] > seg[t + 1];
    }
    if (!__any_sync(0xffffffffu, unsorted)) return;
    __syncwarp();
    for (int t = lane; t < n; t += 32) {
        const int32_t v = buf[t];
        int rank = 0;
        for (int u = 0; u < n; ++u) rank += buf[u] < v;
        seg[rank] = v;
    }
    __syncwarp();
}

template <int SPHI, int NK, bool BAND>
__global__ void __launch_bounds__(256, 3) assoc_kernel(const AssocParams p, const int tile_d) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nk = NK ? NK : p.K.nk;
    const int nkw = (nk + 31) >> 5;
    const int tcols = SPHI * tile_d;
    const int nthr = blockDim.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = nthr >> 5;
    AssocSmem S;
    {
        unsigned char* ptr = smem_raw;
        S.dt = reinterpret_cast<float4*>(ptr);
        ptr += 16 * tile_d;
        S.gpre = reinterpret_cast<int64_t*>(ptr);
        ptr += 8 * tcols * nkw;
        S.wpos = reinterpret_cast<unsigned long long*>(ptr);
        ptr += 8 * tcols * ((nk + 1) / 2);
        S.queue = reinterpret_cast<uint2*>(ptr);
        ptr += 8 * nw * kQueue;
        S.mask = reinterpret_cast<uint32_t*>(ptr);
        ptr += 4 * tcols * nkw;
        S.nearb = reinterpret_cast<uint32_t*>(ptr);
        ptr += 4 * tcols * nkw;
        S.lpre = reinterpret_cast<int32_t*>(ptr);
        ptr += 4 * tcols * nkw;
        S.sortbuf = reinterpret_cast<int32_t*>(ptr);
        ptr += 4 * nw * kSortCap;
        S.active = reinterpret_cast<int32_t*>(ptr);
        ptr += 4 * tile_d;
        if (BAND) {
            S.sx = reinterpret_cast<float*>(ptr);
            S.sy = S.sx + nthr;
            S.sband = reinterpret_cast<int*>(S.sy + nthr);
            S.slist = reinterpret_cast<uint16_t*>(S.sband + nthr);
        } else {
            S.sx = S.sy = nullptr;
            S.sband = nullptr;
            S.slist = nullptr;
        }
    }
    __shared__ int s_cnt[kBuckets];
    S.cnt = s_cnt;
    __shared__ int s_nactive;
    uint2* q = S.queue + warp * kQueue;
    __shared__ int64_t sh[33];
    const int tiles_phi = (p.K.nphi + SPHI - 1) / SPHI;
    const int tiles_d = (p.K.nd + tile_d - 1) / tile_d;
    const int64_t items = (int64_t)p.n_events * tiles_phi * tiles_d;
    for (int64_t item = blockIdx.x; item < items; item += gridDim.x) {
        const int e = (int)(item / ((int64_t)tiles_phi * tiles_d));
        const int t = (int)(item - (int64_t)e * tiles_phi * tiles_d);
        const int tp = t / tiles_d, td = t - (t / tiles_d) * tiles_d;
        const int i0 = tp * SPHI, j0 = td * tile_d;
        const int nj = min(tile_d, p.K.nd - j0);
        const int nrows = min(SPHI, p.K.nphi - i0);
        // tile columns c = j * SPHI + r; first-peak ids and local slots
        int64_t carry = 0;
        bool any = false;
        __syncthreads();
        for (int c0 = 0; c0 < tcols; c0 += nthr) {
            const int c = c0 + tid;
            const int j = c / SPHI, r = c - (c / SPHI) * SPHI;
            const bool live = c < tcols && j < nj && r < nrows;
            const int64_t col = live ? ((int64_t)e * p.K.nphi + i0 + r) * p.K.nd + j0 + j : 0;
            const int n = live ? p.npk[col] : 0;
            int64_t tot;
            const int64_t ex = block_exscan64(n, sh, &tot);
            if (c < tcols) {
                const int64_t cb = live ? p.colbase[col] : 0;
                for (int w = 0; w < nkw; ++w) {
                    const uint32_t m = live ? p.mask[col * nkw + w] : 0u;
                    const int wp = live ? p.wpre[col * nkw + w] : 0;
                    S.mask[c * nkw + w] = m;
                    S.lpre[c * nkw + w] = (int)(carry + ex) + wp;
                    S.gpre[c * nkw + w] = cb + wp;
                }
                any |= n > 0 && cb < p.peak_cap;
            }
            carry += tot;
        }
        if (!__syncthreads_or(any)) continue;
        for (int j = tid; j < nj; j += nthr) S.dt[j] = p.dtab[j0 + j];
        // compacted list of the d0 columns that hold a peak in any of the tile's rows
        if (warp == 0) {
            int na = 0;
            for (int jb = 0; jb < nj; jb += 32) {
                const int j = jb + lane;
                bool act = false;
                if (j < nj)
                    for (int r = 0; r < SPHI; ++r)
                        for (int w = 0; w < nkw; ++w) act |= S.mask[(j * SPHI + r) * nkw + w] != 0u;
                const unsigned b = __ballot_sync(0xffffffffu, act);
                if (act) S.active[na + __popc(b & lanemask_lt())] = j;
                na += __popc(b);
            }
            if (lane == 0) s_nactive = na;
        }
        // near bits (a peak within `window`) and each peak's first CSR position
        for (int v = tid; v < tcols * nkw; v += nthr) {
            const int c = v / nkw, w = v - (v / nkw) * nkw;
            const uint32_t* m = S.mask + c * nkw;
            uint32_t nb = m[w];
            for (int o = 1; o <= p.window; ++o) {
                const uint32_t hi_w = w + 1 < nkw ? m[w + 1] : 0u, lo_w = w > 0 ? m[w - 1] : 0u;
                nb |= (m[w] >> o) | (hi_w << (32 - o)) | (m[w] << o) | (lo_w >> (32 - o));
            }
            S.nearb[v] = nb;
            uint32_t bits = m[w];
            int below = 0;
            while (bits) {
                bits &= bits - 1;
                const int64_t pid = S.gpre[v] + below;
                S.wpos[S.lpre[v] + below] =
                    pid < p.peak_cap ? (unsigned long long)p.peak_offsets[pid] : ~0ull >> 1;
                ++below;
            }
        }
        float cp[SPHI], sp[SPHI];
#pragma unroll
        for (int r = 0; r < SPHI; ++r) {
            const int i = r < nrows ? i0 + r : i0;
            cp[r] = p.cphi[i];
            sp[r] = p.sphi[i];
        }
        const int64_t hb = clamp64(p.offs[p.event0 + e], 0, p.n_hits);
        const int64_t he = clamp64(p.offs[p.event0 + e + 1], hb, p.n_hits);
        int qn = 0;
        __syncthreads();
        const int na = s_nactive;
        if (BAND && na > 0) {
            // the active columns span [S.active[0], S.active[na-1]]: bands are clipped to it
            const int ja = j0 + S.active[0], jb = j0 + S.active[na - 1];
            assoc_band_hits<SPHI, NK>(p, S, q, qn, cp, sp, ja, jb - ja + 1, j0, nrows, nk, nkw, hb, he, lane);
        } else {
            const int64_t nfull = ((he - hb) / nthr) * nthr;
            for (int64_t h = hb + tid; h < hb + nfull; h += nthr)
                assoc_one_hit<SPHI, NK, false>(p, S, q, qn, cp, sp, na, nk, nkw, h, true, lane);
            {
                const int64_t h = hb + nfull + tid;
                if (hb + nfull + (tid - lane) < he)
                    assoc_one_hit<SPHI, NK, true>(p, S, q, qn, cp, sp, na, nk, nkw, h, h < he, lane);
            }
        }
        queue_drain(p, S, q, qn, nkw, nk, lane);
        __syncthreads();
        // ascending hit order within every complete row of the tile's peaks
        int32_t* buf = S.sortbuf + warp * kSortCap;
        for (int c = warp; c < tcols; c += nw) {
            for (int w = 0; w < nkw; ++w) {
                uint32_t m = S.mask[c * nkw + w];
                int below = 0;
                while (m) {
                    m &= m - 1;
                    const int64_t pid = S.gpre[c * nkw + w] + below;
                    const int local = S.lpre[c * nkw + w] + below;
                    ++below;
                    if (pid >= p.peak_cap) continue;
                    const int64_t off = p.peak_offsets[pid];
                    const int64_t end = (int64_t)S.wpos[local];
                    if (end > p.pair_cap) continue;  // row cut by the output cap
                    sort_row(p.hit_idx + off, (int)(end - off), buf, lane);
                }
            }
        }
    }
}

// counts[0..1] = {peaks, pairs of stored peaks + pairs of peaks beyond the cap}
__global__ void finalize_kernel(int64_t* scal) {
    scal[6] = scal[0];
    scal[7] = scal[1] + scal[4];
}

// rcp.approx.ftz.f32 accuracy over a range of float bit patterns: out[0] = max
// |rcp(x) * x - 1| scaled by 2^40 (as an integer), out[1] = patterns checked.
__global__ void rcp_check_kernel(uint32_t first_bits, uint32_t count, unsigned long long* out) {
    unsigned long long worst = 0, n = 0;
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < count; t += gridDim.x * blockDim.x) {
        const float x = __uint_as_float(first_bits + t);
        const float r = rcp_approx(x);
        const double err = fabs((double)r * (double)x - 1.0);
        const unsigned long long e = (unsigned long long)(err * 1099511627776.0);
        worst = e > worst ? e : worst;
        ++n;
    }
    atomicMax(&out[0], worst);
    atomicAdd(&out[1], n);
}

}  // namespace

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
int vote_smem_bytes(int tile_phi, int tile_d, int nk, int threads, bool band) {
    const int chunk = band ? threads * (4 + 4 + 4 + 2 * kBuckets) + 4 : 0;
    return 16 * tile_d + chunk + 4 * tile_phi * tile_d * nk;
}


template <int S>
static cudaError_t prep_one(int smem) {
    return cudaFuncSetAttribute(vote_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

template <int S, int N>
static void* vote_fn() {
    return reinterpret_cast<void*>(vote_kernel<S, N>);
}
template <int S, int N>
static void* vote_band_fn() {
    return reinterpret_cast<void*>(vote_band_kernel<S, N>);
}

static void* vote_band_instance(int tile_phi, int nk) {
#define HT_VOTEB_NK(S)                             \
    switch (nk) {                                  \
        case 64: return vote_band_fn<S, 64>();     \
        case 128: return vote_band_fn<S, 128>();   \
        case 256: return vote_band_fn<S, 256>();   \
        case 512: return vote_band_fn<S, 512>();   \
        default: return vote_band_fn<S, 0>();      \
    }
    switch (tile_phi) {
        case 1: HT_VOTEB_NK(1)
        case 2: HT_VOTEB_NK(2)
        case 4: HT_VOTEB_NK(4)
        case 8: HT_VOTEB_NK(8)
    }
#undef HT_VOTEB_NK
    return nullptr;
}

// kernel instance for (tile_phi, n_kappa): compile-time n_kappa for the common widths
static void* vote_instance(int tile_phi, int nk) {
#define HT_VOTE_NK(S)                         \
    switch (nk) {                             \
        case 64: return vote_fn<S, 64>();     \
        case 128: return vote_fn<S, 128>();   \
        case 256: return vote_fn<S, 256>();   \
        case 512: return vote_fn<S, 512>();   \
        default: return vote_fn<S, 0>();      \
    }
    switch (tile_phi) {
        case 1: HT_VOTE_NK(1)
        case 2: HT_VOTE_NK(2)
        case 4: HT_VOTE_NK(4)
        case 8: HT_VOTE_NK(8)
    }
#undef HT_VOTE_NK
    return nullptr;
}

cudaError_t vote_occupancy(int tile_phi, int nk, int threads, int smem, int* blocks, bool band) {
    void* f = band ? vote_band_instance(tile_phi, nk) : vote_instance(tile_phi, nk);
    if (!f) return cudaErrorInvalidValue;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, f, threads, smem);
}

cudaError_t launch_finalize(int64_t* scal, cudaStream_t s) {
    finalize_kernel<<<1, 1, 0, s>>>(scal);
    return cudaGetLastError();
}

cudaError_t vote_prepare(int tile_phi, int nk, int smem, bool band) {
    void* f = band ? vote_band_instance(tile_phi, nk) : vote_instance(tile_phi, nk);
    if (!f) return cudaErrorInvalidValue;
    return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

cudaError_t launch_vote(int tile_phi, const VoteParams& p, int grid, int threads, int smem, cudaStream_t s,
                        bool band) {
    if (grid <= 0) return cudaSuccess;
    void* f = band ? vote_band_instance(tile_phi, p.K.nk) : vote_instance(tile_phi, p.K.nk);
    if (!f) return cudaErrorInvalidValue;
    void* args[] = {const_cast<VoteParams*>(&p)};
    return cudaLaunchKernel(f, dim3(grid), dim3(threads), args, smem, s);
}

cudaError_t launch_validate(const float* x, const float* y, const int8_t* layer, int64_t n_hits,
                            const int32_t* offs, int32_t n_events, int32_t n_layers, int32_t* err,
                            cudaStream_t s) {
    int64_t work = n_hits > n_events ? n_hits : n_events;
    int grid = (int)((work + 255) / 256);
    if (grid > 1216) grid = 1216;
    if (grid < 1) grid = 1;
    validate_kernel<<<grid, 256, 0, s>>>(x, y, layer, n_hits, offs, n_events, n_layers, err);
    return cudaGetLastError();
}

cudaError_t launch_order(const int32_t* offs, int32_t event0, int32_t n_events, int64_t n_hits,
                         int32_t* order, cudaStream_t s) {
    order_kernel<<<1, 1024, 0, s>>>(offs, event0, n_events, n_hits, order);
    return cudaGetLastError();
}

static int warp_grid(int64_t ncols, int threads) {
    int64_t blocks = (ncols * 32 + threads - 1) / threads;
    if (blocks > 152 * 16) blocks = 152 * 16;
    return blocks < 1 ? 1 : (int)blocks;
}

// detect tile: R interior rows x TD interior columns, halo included, ~96 KB
void detect_tile(int nphi, int nd, int nk, int* R, int* TD) {
    const int64_t budget = 96 * 1024 / 4;  // words
    int td = nd;
    while (td > 1 && (int64_t)3 * (td + 2) * nk > budget) td = (td + 1) / 2;
    int r = (int)(budget / ((int64_t)(td + 2) * nk)) - 2;
    r = std::max(1, std::min(r, nphi));
    *R = r;
    *TD = td;
}

size_t detect_smem(int nphi, int nd, int nk) {
    int R, TD;
    detect_tile(nphi, nd, nk, &R, &TD);
    return (size_t)(R + 2) * (TD + 2) * nk * 4;
}

cudaError_t detect_prepare(int nphi, int nd, int nk) {
    return cudaFuncSetAttribute(detect_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)detect_smem(nphi, nd, nk));
}

cudaError_t launch_detect(const PeakParams& p, cudaStream_t s) {
    if ((int64_t)p.n_events * p.nphi * p.nd == 0) return cudaSuccess;
    int R, TD;
    detect_tile(p.nphi, p.nd, p.nk, &R, &TD);
    const int64_t items = (int64_t)p.n_events * ((p.nphi + R - 1) / R) * ((p.nd + TD - 1) / TD);
    const int grid = (int)std::min<int64_t>(items, 152 * 8);
    detect_kernel<<<grid, 512, detect_smem(p.nphi, p.nd, p.nk), s>>>(p, R, TD);
    return cudaGetLastError();
}

cudaError_t launch_emit(const PeakParams& p, cudaStream_t s) {
    const int64_t ncols = (int64_t)p.n_events * p.nphi * p.nd;
    if (ncols == 0) return cudaSuccess;
    emit_kernel<<<warp_grid(ncols, 256), 256, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_paircount(const PeakParams& p, const int64_t* lo_dev, const int64_t* hi_dev,
                             cudaStream_t s) {
    paircount_kernel<<<152 * 8, 256, 0, s>>>(p, lo_dev, hi_dev);
    return cudaGetLastError();
}

cudaError_t launch_scan(const ScanRange& r, int64_t* scratch, cudaStream_t s) {
    scan_reduce_kernel<<<kScanBlocks, kScanThreads, 0, s>>>(r, scratch);
    scan_spine_kernel<<<1, kScanThreads, 0, s>>>(r, scratch, kScanBlocks);
    scan_down_kernel<<<kScanBlocks, kScanThreads, 0, s>>>(r, scratch, kScanBlocks);
    return cudaGetLastError();
}

template <int S, int N>
static void* assoc_fn(bool band) {
    return band ? reinterpret_cast<void*>(assoc_kernel<S, N, true>) : reinterpret_cast<void*>(assoc_kernel<S, N, false>);
}

static void* assoc_instance(int tile_phi, int nk, bool band) {
#define HT_ASSOC_NK(S)                             \
    switch (nk) {                                  \
        case 64: return assoc_fn<S, 64>(band);     \
        case 128: return assoc_fn<S, 128>(band);   \
        case 256: return assoc_fn<S, 256>(band);   \
        case 512: return assoc_fn<S, 512>(band);   \
        default: return assoc_fn<S, 0>(band);      \
    }
    switch (tile_phi) {
        case 1: HT_ASSOC_NK(1)
        case 2: HT_ASSOC_NK(2)
        case 4: HT_ASSOC_NK(4)
        case 8: HT_ASSOC_NK(8)
    }
#undef HT_ASSOC_NK
    return nullptr;
}

size_t assoc_smem(int tile_phi, int tile_d, int nk, int threads, bool band) {
    return assoc_smem_bytes(tile_phi, tile_d, nk, threads, band);
}

cudaError_t assoc_prepare(int tile_phi, int nk, int smem, bool band) {
    void* f = assoc_instance(tile_phi, nk, band);
    if (!f) return cudaErrorInvalidValue;
    return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

cudaError_t launch_assoc(const AssocParams& p, int tile_phi, int tile_d, int threads, cudaStream_t s) {
    if ((int64_t)p.n_events * p.K.nphi == 0) return cudaSuccess;
    void* f = assoc_instance(tile_phi, p.K.nk, p.band != 0);
    if (!f) return cudaErrorInvalidValue;
    const int tiles = ((p.K.nphi + tile_phi - 1) / tile_phi) * ((p.K.nd + tile_d - 1) / tile_d);
    const int64_t items = (int64_t)p.n_events * tiles;
    const int grid = (int)std::min<int64_t>(items, 152 * 32);
    const int smem = (int)assoc_smem_bytes(tile_phi, tile_d, p.K.nk, threads, p.band != 0);
    int td = tile_d;
    void* args[] = {const_cast<AssocParams*>(&p), &td};
    return cudaLaunchKernel(f, dim3(grid), dim3(threads), args, smem, s);
}

cudaError_t launch_rcp_check(uint32_t first_bits, uint32_t count, unsigned long long* out, cudaStream_t s) {
    rcp_check_kernel<<<152 * 4, 256, 0, s>>>(first_bits, count, out);
    return cudaGetLastError();
}

}  // namespace ht
