// ht_assoc_rec.cu — hit-to-candidate association over the vote's records.
//
// Section 3 attaches to each maximum the hits that voted for it: hit h joins
// peak (i, j, k) of its event when its bin in column (i, j) lies within
// `window` of k.  The band vote has already binned every (hit, cell) pair of
// each tile whose d0 band the hit meets, and written those bins as one byte
// per cell (255: no vote) into a record per (hit, tile), plus one bit per
// (hit, tile) saying that the record exists.  A hit without a record has no
// bin in any of the tile's columns, so it joins none of their peaks.
//
// Here one warp owns one (event, vote tile) item and walks the tile's
// recorded hits in increasing order.  Lane L owns the record's bytes
// [L * CPL, (L + 1) * CPL), i.e. CPL cells, and therefore every peak of
// those cells: no other lane ever touches their row cursors, so rows come out
// in ascending hit order with no ranking, atomics or sort.  A cell whose bin
// is near a peak (a bit table per cell) queues (hit, cell, bin) in the lane's
// own small queue; the warp empties the queues together when one fills, each
// lane writing its entries in order.
#include <cuda_runtime.h>

#include <climits>
#include <cstdint>

#include "ht_internal.h"

namespace ht {

namespace {

constexpr int kRecQueue = 16;  // queued candidates per lane

__device__ __forceinline__ int64_t clamp64r(int64_t v, int64_t lo, int64_t hi) {
    return v < lo ? lo : (v > hi ? hi : v);
}

// CPL record bytes per lane
template <int CPL> struct RecLane { using T = uint32_t; };
template <> struct RecLane<1> { using T = uint8_t; };
template <> struct RecLane<2> { using T = uint16_t; };
template <> struct RecLane<8> { using T = unsigned long long; };

// hits per step of the walk; the next step's record loads are issued before
// this step's records are tested
constexpr int kRecStep = 8;
constexpr int kRecBlock = 1024;  // hits whose bitmap words are read at once (32 words, one per lane)

struct RecWarp {
    // cell tables, one row per cell in lane-major order (row tt * 32 + L holds
    // cell L * CPL + tt), so the lanes' lookups fall in different banks
    uint32_t* mask;   // [cells][nkw] peak bits of the tile's cells (0 outside the grid)
    int32_t* lpre;    // [cells][nkw] item-local id of the first peak of each word
    uint32_t* nearb;  // [cells][nkn] bins within `window` of a peak; bin nk (no bin) is 0
    long long* cur;   // [cap] row cursors (absolute positions) of the pass's peaks
    uint32_t* q;      // [kRecQueue][32] (cell in lane << 18) | (bin << 10) | hit offset in the block
    uint16_t* list;   // [kRecBlock] recorded hits of the current block (offsets in the block)
};

__host__ __device__ inline size_t rec_warp_bytes(int cells, int nk, int cap) {
    const size_t nkw = (nk + 31) / 32, nkn = nk / 32 + 1;
    return (4 * (size_t)cells * (2 * nkw + nkn) + 8 * (size_t)cap + 4 * (size_t)kRecQueue * 32 +
            2 * (size_t)kRecBlock + 15) &
           ~size_t(15);
}

// Write the queued candidates of every lane (each lane its own, in order);
// hbase is the first hit of the block the entries belong to.
template <int CPL>
__device__ __forceinline__ void rec_flush(const AssocParams& p, const RecWarp& S, int nkw, int nk, int qn, int L0,
                                          int L1, int64_t hbase, int lane) {
    const int mx = (int)__reduce_max_sync(0xffffffffu, (unsigned)qn);
    const int w = p.window;
    for (int s = 0; s < mx; ++s) {
        if (s < qn) {
            const uint32_t ent = S.q[s * 32 + lane];
            const int row = (int)(ent >> 18) * 32 + lane;
            const int b = (int)((ent >> 10) & 0xFFu);
            const uint32_t* m = S.mask + row * nkw;
            const int lo = max(b - w, 0), hi = min(b + w, nk - 1);
            const int a = lo >> 5, bw = hi >> 5;  // bw <= a + 1 since 2w < 32
            const unsigned long long two =
                ((unsigned long long)(bw > a ? m[bw] : 0u) << 32) | (unsigned long long)m[a];
            unsigned pend = (unsigned)(two >> (lo & 31)) & (0xFFFFFFFFu >> (31 - (hi - lo)));
            for (; pend; pend &= pend - 1u) {
                const int kk = lo + __ffs(pend) - 1;
                const uint32_t word = m[kk >> 5];
                const int local = S.lpre[row * nkw + (kk >> 5)] + __popc(word & ((1u << (kk & 31)) - 1u));
                if (local >= L0 && local < L1) {
                    const long long pos = S.cur[local - L0];
                    S.cur[local - L0] = pos + 1;
                    if (pos < p.pair_cap) p.hit_idx[pos] = (int32_t)(hbase + (int64_t)(ent & 0x3FFu));
                }
            }
        }
    }
    __syncwarp();
}

// Test CPL cells of one recorded hit (`off` in its block) and queue the near ones.
template <int CPL, typename LT>
__device__ __forceinline__ void rec_test(const RecWarp& S, LT v, uint32_t off, int nk, int nkn, int lane, int& qn) {
#pragma unroll
    for (int tt = 0; tt < CPL; ++tt) {
        const unsigned b = (unsigned)(v >> (8 * tt)) & 0xFFu;
        const unsigned bb = min(b, (unsigned)nk);
        const int row = tt * 32 + lane;
        if ((S.nearb[row * nkn + (bb >> 5)] >> (bb & 31)) & 1u) {
            S.q[qn * 32 + lane] = ((unsigned)tt << 18) | (b << 10) | off;
            ++qn;
        }
    }
}

template <int SPHI, int CPL>
__global__ void __launch_bounds__(128, 4) assoc_rec_kernel(const AssocParams p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using LT = typename RecLane<CPL>::T;
    constexpr int CELLS = 32 * CPL;
    constexpr int TD = CELLS / SPHI;  // record columns (the vote tile's d0 width)
    constexpr int U = kRecStep;
    constexpr int kRecCheck = 8 / CPL;  // hits between queue checks (<= 8 new entries per lane)
    const int nk = p.K.nk;
    const int nkw = (nk + 31) >> 5;
    const int nkn = (nk >> 5) + 1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    RecWarp S;
    {
        unsigned char* ptr = smem_raw + (size_t)warp * p.warp_bytes;
        S.cur = reinterpret_cast<long long*>(ptr);
        ptr += 8 * (size_t)p.cap;
        S.q = reinterpret_cast<uint32_t*>(ptr);
        ptr += 4 * kRecQueue * 32;
        S.list = reinterpret_cast<uint16_t*>(ptr);
        ptr += 2 * kRecBlock;
        S.mask = reinterpret_cast<uint32_t*>(ptr);
        S.lpre = reinterpret_cast<int32_t*>(S.mask + CELLS * nkw);
        S.nearb = reinterpret_cast<uint32_t*>(S.lpre + CELLS * nkw);
    }
    const int64_t tiles = (int64_t)p.rtiles_phi * p.rtiles_d;
    const int64_t n_items = (int64_t)p.n_events * tiles;
    const int64_t whb = clamp64r(p.offs[p.event0], 0, p.n_hits);
    const int64_t wend = clamp64r(p.offs[p.event0 + p.n_events], whb, p.n_hits);
    for (;;) {
        unsigned long long it = 0;
        if (lane == 0) it = atomicAdd(p.queue, 1ull);
        const int64_t item = (int64_t)__shfl_sync(0xffffffffu, it, 0);
        if (item >= n_items) break;
        const int el = (int)(item / tiles);
        const int64_t t = item - (int64_t)el * tiles;
        const int e = p.order ? p.order[el] : el;
        const int tp = (int)(t / p.rtiles_d), td = (int)(t - (int64_t)tp * p.rtiles_d);
        const int i0 = tp * SPHI, j0 = td * TD;
        const int nj = min(TD, p.K.nd - j0);
        const int nrows = min(SPHI, p.K.nphi - i0);
        // peaks of the item: row r of the tile holds a consecutive run of
        // global ids starting at its first column's base
        int64_t rg = 0;  // lane r < nrows: first global id of run r
        int rn = 0;      // its length
        if (lane < nrows) {
            const int64_t c0 = ((int64_t)e * p.K.nphi + i0 + lane) * p.K.nd + j0;
            rg = p.colbase[c0];
            rn = (int)(p.colbase[c0 + nj - 1] + p.npk[c0 + nj - 1] - rg);
        }
        // run bases (item-local ids) and the stored peaks (global id < peak_cap)
        int run_base = 0, tot = 0, stored = 0;
        int64_t RG[SPHI];
        int RB0[SPHI];
#pragma unroll
        for (int r = 0; r < SPHI; ++r) {
            const int rn_r = __shfl_sync(0xffffffffu, rn, r);
            const int n_r = r < nrows ? rn_r : 0;
            RG[r] = __shfl_sync(0xffffffffu, rg, r);
            RB0[r] = tot;
            if (lane == r) run_base = tot;
            tot += n_r;
            stored += (int)clamp64r(p.peak_cap - RG[r], 0, n_r);
        }
        if (stored == 0) continue;
        const int64_t hb = clamp64r(p.offs[p.event0 + e], 0, p.n_hits);
        const int64_t he = clamp64r(p.offs[p.event0 + e + 1], hb, p.n_hits);
        if (hb < whb || he > wend) continue;  // offsets the validation rejects: no records were written
        __syncwarp();  // the previous item's tables are no longer read
        for (int v = lane; v < CELLS * nkw; v += 32) {
            const int row = v / nkw, wd = v - (v / nkw) * nkw;
            const int c = (row & 31) * CPL + (row >> 5);
            const int j = c / SPHI, r = c - (c / SPHI) * SPHI;
            const bool ok = r < nrows && j < nj;
            const int64_t col = ((int64_t)e * p.K.nphi + i0 + r) * p.K.nd + j0 + j;
            const int64_t g_r = __shfl_sync(0xffffffffu, rg, r & 31);
            const int b_r = __shfl_sync(0xffffffffu, run_base, r & 31);
            S.mask[v] = ok ? p.mask[col * nkw + wd] : 0u;
            S.lpre[v] = ok ? b_r + (int)(p.colbase[col] - g_r) + p.wpre[col * nkw + wd] : 0;
        }
        __syncwarp();
        for (int v = lane; v < CELLS * nkn; v += 32) {
            const int row = v / nkn, wd = v - (v / nkn) * nkn;
            const uint32_t* m = S.mask + row * nkw;
            const uint32_t mw = wd < nkw ? m[wd] : 0u;
            const uint32_t hi_w = wd + 1 < nkw ? m[wd + 1] : 0u, lo_w = wd > 0 && wd - 1 < nkw ? m[wd - 1] : 0u;
            uint32_t nb = mw;
            for (int o = 1; o <= p.window; ++o) nb |= (mw >> o) | (hi_w << (32 - o)) | (mw << o) | (lo_w >> (32 - o));
            if (wd == (nk >> 5)) nb &= (1u << (nk & 31)) - 1u;  // no bins from nk on
            S.nearb[v] = nb;
        }
        const int64_t n_e = he - hb;
        const uint8_t* recb = p.rec + ((hb - whb) * tiles + t * n_e) * p.rec_bytes + lane * CPL;
        const uint32_t* bits_t = p.rbits + (((hb - whb) >> 5) + e) * tiles + t * ((n_e + 31) >> 5);
        const int nwords = (int)((n_e + 31) >> 5);
        for (int L0 = 0; L0 < tot; L0 += p.cap) {
            const int L1 = min(tot, L0 + p.cap);
            __syncwarp();
            for (int l = L0 + lane; l < L1; l += 32) {
                // run of l: the last run whose base is <= l
                int64_t g = RG[0] + l;
#pragma unroll
                for (int q = 1; q < SPHI; ++q)
                    if (q < nrows && RB0[q] <= l) g = RG[q] + (l - RB0[q]);
                S.cur[l - L0] = g < p.peak_cap ? (long long)p.peak_offsets[g] : LLONG_MAX / 2;
            }
            __syncwarp();
            for (int cw0 = 0; cw0 < nwords; cw0 += 32) {
                // the block's recorded hits, in order, as offsets from its first hit
                const uint32_t myw = cw0 + lane < nwords ? bits_t[cw0 + lane] : 0u;
                const int cnt = __popc(myw);
                int pre = cnt;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int v = __shfl_up_sync(0xffffffffu, pre, o);
                    if (lane >= o) pre += v;
                }
                const int n = __shfl_sync(0xffffffffu, pre, 31);
                pre -= cnt;
                __syncwarp();  // the previous block's list is no longer read
                for (unsigned b = myw; b; b &= b - 1u) S.list[pre++] = (uint16_t)(lane * 32 + __ffs(b) - 1);
                __syncwarp();
                const uint8_t* blk = recb + (int64_t)cw0 * 32 * p.rec_bytes;
                // two buffers of U hits: the loads of one are in flight while
                // the other's records are tested
                uint32_t ha[U], hb2[U];
                LT va[U], vb[U];
                auto load = [&](uint32_t* hh, LT* vv, int first) {
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        const bool hv = first + u < n;
                        hh[u] = hv ? S.list[first + u] : 0u;
                        vv[u] = hv ? *reinterpret_cast<const LT*>(blk + (int64_t)hh[u] * p.rec_bytes) : (LT)~(LT)0;
                    }
                };
                int qn = 0;
                auto test = [&](const uint32_t* hh, const LT* vv) {
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        rec_test<CPL>(S, vv[u], hh[u], nk, nkn, lane, qn);
                        if ((u + 1) % kRecCheck == 0 && __any_sync(0xffffffffu, qn > kRecQueue - 8)) {
                            rec_flush<CPL>(p, S, nkw, nk, qn, L0, L1, hb + (int64_t)cw0 * 32, lane);
                            qn = 0;
                        }
                    }
                };
                load(ha, va, 0);
                for (int s0 = 0; s0 < n; s0 += 2 * U) {
                    load(hb2, vb, s0 + U);
                    test(ha, va);
                    if (s0 + U >= n) break;
                    load(ha, va, s0 + 2 * U);
                    test(hb2, vb);
                }
                rec_flush<CPL>(p, S, nkw, nk, qn, L0, L1, hb + (int64_t)cw0 * 32, lane);
            }
        }
    }
}

template <int S, int C>
void* rec_fn() {
    return reinterpret_cast<void*>(assoc_rec_kernel<S, C>);
}

void* rec_instance(int tile_phi, int cpl) {
#define HT_REC_CPL(S)                       \
    switch (cpl) {                          \
        case 1: return rec_fn<S, 1>();      \
        case 2: return rec_fn<S, 2>();      \
        case 4: return rec_fn<S, 4>();      \
        case 8: return rec_fn<S, 8>();      \
    }                                       \
    return nullptr;
    switch (tile_phi) {
        case 1: HT_REC_CPL(1)
        case 2: HT_REC_CPL(2)
        case 4: HT_REC_CPL(4)
        case 8: HT_REC_CPL(8)
    }
#undef HT_REC_CPL
    return nullptr;
}

}  // namespace

bool assoc_rec_supported(int tile_phi, int tile_d, int nk) {
    const int rb = tile_phi * tile_d;
    return nk >= 1 && nk <= 255 && (tile_phi == 1 || tile_phi == 2 || tile_phi == 4 || tile_phi == 8) &&
           (rb == 32 || rb == 64 || rb == 128 || rb == 256);
}

size_t assoc_rec_warp_smem(int tile_phi, int tile_d, int nk, int cap) {
    return rec_warp_bytes(tile_phi * tile_d, nk, cap);
}

cudaError_t assoc_rec_prepare(int tile_phi, int tile_d, int nk, int smem, int threads, int* blocks_per_sm) {
    void* f = rec_instance(tile_phi, tile_phi * tile_d / 32);
    if (!f) return cudaErrorInvalidValue;
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    if (smem > optin) return cudaErrorInvalidValue;
    cudaFuncAttributes fa{};
    e = cudaFuncGetAttributes(&fa, f);
    if (e != cudaSuccess) return e;
    // the limit is only ever raised (shared by every context in the process)
    if (fa.maxDynamicSharedSizeBytes < optin - (int)fa.sharedSizeBytes) {
        e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
        if (e != cudaSuccess) return e;
    }
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, f, threads, smem);
}

cudaError_t launch_assoc_rec(const AssocParams& p, int tile_phi, int threads, int grid, cudaStream_t s) {
    if ((int64_t)p.n_events * p.K.nphi == 0) return cudaSuccess;
    void* f = rec_instance(tile_phi, p.rec_bytes / 32);
    if (!f) return cudaErrorInvalidValue;
    const int smem = (int)(p.warp_bytes * (threads / 32));
    void* args[] = {const_cast<AssocParams*>(&p)};
    return cudaLaunchKernel(f, dim3(grid), dim3(threads), args, smem, s);
}

}  // namespace ht
