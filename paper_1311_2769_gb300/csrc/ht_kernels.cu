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

// red_if_vote (TAIL form) that also sets byte `r` of a record word to the
// certified bin, or 255 when the cell casts no certified vote (out of range,
// undecided, or an idle lane): one predicate for both.
__device__ __forceinline__ uint32_t red_and_byte(uint32_t addr, float flo, float fhi, unsigned kb, unsigned nk,
                                                 bool valid, uint32_t word, unsigned pos) {
    uint32_t out;
    asm volatile(
        "{\n\t.reg .pred p;\n\t.reg .b32 b;\n\tsetp.eq.f32 p, %2, %3;\n\tsetp.lt.and.u32 p, %4, %5, p;\n\t"
        "setp.ne.and.u32 p, %6, 0, p;\n\t@p red.shared.add.u32 [%1], 1;\n\tselp.b32 b, %4, 255, p;\n\t"
        "bfi.b32 %0, b, %7, %8, 8;\n\t}"
        : "=r"(out)
        : "r"(addr), "f"(flo), "f"(fhi), "r"(kb), "r"(nk), "r"((unsigned)valid), "r"(word), "r"(pos));
    return out;
}

struct TileHit {
    float x, y;
    HitFast hf;
};

// One hit against the tile's columns ja..jb (warp-uniform).  TAIL: lanes
// without a hit stay in the loop (the full-mask vote needs all 32) but are
// masked.
template <int SPHI, int NK, bool TAIL>
__device__ __forceinline__ void vote_xy(const VoteParams& p, const float* cp, const float* sp, const float4* dt_s,
                                        uint32_t* acc_s, uint32_t acc_sh, int ja, int jb, int nk, float x, float y,
                                        bool valid) {
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
    uint32_t col_sh = acc_sh + 4u * (unsigned)(ja * col_words);
    for (int j = ja; j <= jb; ++j, col_sh += 4u * col_words) {
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

template <int SPHI, int NK, bool TAIL>
__device__ __forceinline__ void vote_one_hit(const VoteParams& p, const float* cp, const float* sp,
                                             const float4* dt_s, uint32_t* acc_s, uint32_t acc_sh, int ja, int jb,
                                             int nk, int64_t h, bool valid) {
    const float x = (!TAIL || valid) ? p.x[h] : 0.0f;
    const float y = (!TAIL || valid) ? p.y[h] : 0.0f;
    vote_xy<SPHI, NK, TAIL>(p, cp, sp, dt_s, acc_s, acc_sh, ja, jb, nk, x, y, valid);
}

// Packed bins of one column's SPHI cells (one byte per phi row, row 0 in
// the lowest byte; 255: no vote).
template <int SPHI> struct RecWord { using T = uint32_t; };
template <> struct RecWord<1> { using T = uint8_t; };
template <> struct RecWord<2> { using T = uint16_t; };
template <> struct RecWord<8> { using T = unsigned long long; };

// vote_one_hit (TAIL form) that also writes the hit's record for the tile:
// every column of [ja, jb] gets its rows' certified (or stage 2/3) bins, the
// columns outside the warp's hull 255 (a hit votes nowhere outside its own
// band, and the hull contains it).  `rec` is the lane's record (valid lanes).
template <int SPHI, int NK>
__device__ __forceinline__ void vote_xy_rec(const VoteParams& p, const float* cp, const float* sp, const float4* dt_s,
                                            uint32_t* acc_s, uint32_t acc_sh, int ja, int jb, int nk, float x, float y,
                                            bool valid, uint8_t* rec) {
    using W = typename RecWord<SPHI>::T;
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
    W* rw = reinterpret_cast<W*>(rec);
    if (valid) {
        const W none = (W)~(W)0;
        for (int j = 0; j < ja; ++j) rw[j] = none;
        for (int j = jb + 1; j < p.tile_d; ++j) rw[j] = none;
    }
    uint32_t col_sh = acc_sh + 4u * (unsigned)(ja * col_words);
    for (int j = ja; j <= jb; ++j, col_sh += 4u * col_words) {
        const float4 dt = dt_s[j];
        const float Rj = hf.r2 + dt.z;
        bool und = false;
        uint32_t wlo = 0, whi = 0;  // rows 0-3 and 4-7
#pragma unroll
        for (int r = 0; r < SPHI; ++r) {
            const S1 o = stage1_fast(qs[r], q[r], dt, Rj, hf.G, H, T0);
            const uint32_t addr = col_sh + 4u * ((unsigned)(r * nk) + o.kb);
            if (r < 4)
                wlo = red_and_byte(addr, o.flo, o.fhi, o.kb, nku, valid, wlo, 8u * r);
            else
                whi = red_and_byte(addr, o.flo, o.fhi, o.kb, nku, valid, whi, 8u * (r - 4));
            und |= (o.flo != o.fhi) & valid;
        }
        W word = (W)(SPHI == 8 ? ((unsigned long long)whi << 32) | wlo : wlo);
        if (__any_sync(0xffffffffu, und)) {
#pragma unroll
            for (int r = 0; r < SPHI; ++r) {
                const S1 o = stage1_fast(qs[r], q[r], dt, Rj, hf.G, H, T0);
                if ((o.flo != o.fhi) && valid && stage1_pending(o, hf.dmin, p.K.wlo, p.K.whi)) {
                    const int kk = cell_slow(x, y, cp[r], sp[r], dt.x, hf.R1, p.K, p.stats);
                    if (kk >= 0) atomicAdd(acc_s + j * col_words + r * nk + kk, 1u);
                    word = (word & ~((W)0xFF << (8 * r))) | ((W)(kk >= 0 ? (unsigned)kk : 255u) << (8 * r));
                }
            }
        }
        if (valid) rw[j] = word;
    }
}

// vote_xy (TAIL form), optionally writing the hit's record, with each lane
// walking its own band [lo, hi] from its first column: step s evaluates
// column lo + s, so `steps` (the widest band of the warp) replaces the hull
// of the warp's bands.  Lanes past their band idle.  With REC the whole
// record is first set to 255 (16-byte stores), then the band's columns are
// written.  Idle and invalid lanes have lo in range (the dt load stays
// inside the tile table) and hi < lo.
template <int SPHI, int NK, bool REC>
__device__ __forceinline__ void vote_xy_al(const VoteParams& p, const float* cp, const float* sp, const float4* dt_s,
                                           uint32_t* acc_s, uint32_t acc_sh, int lo, int hi, int steps, int nk,
                                           float x, float y, bool valid, uint8_t* rec) {
    using W = typename RecWord<SPHI>::T;
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
    W* rw = reinterpret_cast<W*>(rec);
    if (REC && valid) {
        uint4* r4 = reinterpret_cast<uint4*>(rec);
        const uint4 none = make_uint4(~0u, ~0u, ~0u, ~0u);
        for (int b = 0; b < (p.rec_bytes >> 4); ++b) r4[b] = none;
    }
    for (int s = 0; s < steps; ++s) {
        const int j = lo + s;
        const bool act = valid & (j <= hi);
        const int jc = act ? j : lo;
        const float4 dt = dt_s[jc];
        const float Rj = hf.r2 + dt.z;
        const uint32_t col_sh = acc_sh + 4u * (unsigned)(jc * col_words);
        bool und = false;
        uint32_t wlo = 0, whi = 0;
#pragma unroll
        for (int r = 0; r < SPHI; ++r) {
            const S1 o = stage1_fast(qs[r], q[r], dt, Rj, hf.G, H, T0);
            const uint32_t addr = col_sh + 4u * ((unsigned)(r * nk) + o.kb);
            if (REC) {
                if (r < 4)
                    wlo = red_and_byte(addr, o.flo, o.fhi, o.kb, nku, act, wlo, 8u * r);
                else
                    whi = red_and_byte(addr, o.flo, o.fhi, o.kb, nku, act, whi, 8u * (r - 4));
            } else {
                red_if_vote(addr, o.flo, o.fhi, o.kb, nku, act);
            }
            und |= (o.flo != o.fhi) & act;
        }
        W word = (W)(SPHI == 8 ? ((unsigned long long)whi << 32) | wlo : wlo);
        if (__any_sync(0xffffffffu, und)) {
#pragma unroll
            for (int r = 0; r < SPHI; ++r) {
                const S1 o = stage1_fast(qs[r], q[r], dt, Rj, hf.G, H, T0);
                if ((o.flo != o.fhi) && act && stage1_pending(o, hf.dmin, p.K.wlo, p.K.whi)) {
                    const int kk = cell_slow(x, y, cp[r], sp[r], dt.x, hf.R1, p.K, p.stats);
                    if (kk >= 0) atomicAdd(acc_s + jc * col_words + r * nk + kk, 1u);
                    if (REC) word = (word & ~((W)0xFF << (8 * r))) | ((W)(kk >= 0 ? (unsigned)kk : 255u) << (8 * r));
                }
            }
        }
        if (REC && act) rw[j] = word;
    }
}

template <int SPHI, int NK>
__device__ __forceinline__ void vote_one_hit_rec(const VoteParams& p, const float* cp, const float* sp,
                                                 const float4* dt_s, uint32_t* acc_s, uint32_t acc_sh, int ja, int jb,
                                                 int nk, int64_t h, bool valid, uint8_t* rec) {
    const float x = valid ? p.x[h] : 0.0f;
    const float y = valid ? p.y[h] : 0.0f;
    vote_xy_rec<SPHI, NK>(p, cp, sp, dt_s, acc_s, acc_sh, ja, jb, nk, x, y, valid, rec);
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
            vote_one_hit<SPHI, NK, false>(p, cp, sp, dt_s, acc_s, acc_sh, 0, nj - 1, nk, h, true);
        {
            const int64_t h = hb + nfull + tid;
            if (hb + nfull + (tid - lane) < he)  // warps with at least one hit left
                vote_one_hit<SPHI, NK, true>(p, cp, sp, dt_s, acc_s, acc_sh, 0, nj - 1, nk, h, h < he);
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
// pruned vote: hits without a band in the tile are dropped first
// ---------------------------------------------------------------------------
// Each warp takes its hits 32 at a time and computes, per hit, the union of
// the tile rows' d0 bands (d0_band: a proven superset of the columns where
// the hit can vote).  Hits with an empty union are dropped; the others enter
// a per-warp queue, and every 32 queued hits run the ordinary cell loop over
// the hull of their 32 bands.  Cells outside a hit's band cannot vote (they
// are out of the kappa range in binary64), so the accumulator is the full
// vote's.  On the batch workload about two thirds of the (hit, tile) pairs
// of a 4 x 16 tile have an empty band.
constexpr int kHitQueue = 64;  // per-warp queue of banded hits (run 32 at a time)

// ---- staged hit blocks: 1-D bulk copies (TMA) into shared memory ----------
// One thread arms an mbarrier with the block's byte count and issues
// cp.async.bulk copies of the block's 16-byte-aligned interior of x and of
// y; every thread waits on the barrier's phase (a bounded wait), and a few
// threads load the block's ragged ends (at most three hits each) directly.
constexpr int kStageHits = 512;                 // hits per staged block
constexpr int kStageBuf = kStageHits + 4;       // floats per array buffer (block start rounded down to 4)
constexpr int kStageBytes = 2 * 2 * kStageBuf * 4;  // two buffers of x and y
constexpr unsigned kStageWaitLimit = 1u << 20;  // try_wait rounds before a copy counts as lost

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}
// bounded wait for the completion of the barrier phase with parity `par`
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned par) {
    for (unsigned i = 0; i < kStageWaitLimit; ++i) {
        unsigned done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(smem_addr(bar)), "r"(par)
            : "memory");
        if (done) return true;
    }
    return false;
}

struct StageBlock {
    int64_t b0, b1, base, a0, a1;  // hits [b0, b1); smem index h - base; bulk part [a0, a1)
};

__device__ __forceinline__ StageBlock stage_block(int64_t hb, int64_t he, int b) {
    StageBlock k;
    k.b0 = hb + (int64_t)b * kStageHits;
    k.b1 = clamp64(k.b0 + kStageHits, k.b0, he);
    k.base = k.b0 & ~(int64_t)3;
    k.a0 = clamp64((k.b0 + 3) & ~(int64_t)3, k.b0, k.b1);
    k.a1 = clamp64(k.b1 & ~(int64_t)3, k.a0, k.b1);
    return k;
}

// issued by one thread: block b of [hb, he) into buffer b & 1
__device__ __forceinline__ void stage_issue(const VoteParams& p, float* stg, uint64_t* bars, int64_t hb, int64_t he,
                                            int b) {
    const StageBlock k = stage_block(hb, he, b);
    uint64_t* bar = bars + (b & 1);
    float* xs = stg + (b & 1) * 2 * kStageBuf;
    float* ys = xs + kStageBuf;
    if (k.a1 > k.a0) {
        const unsigned bytes = (unsigned)((k.a1 - k.a0) * 4);
        // the buffer's previous contents were read through the generic proxy
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(bar, 2 * bytes);
        bulk_g2s(xs + (k.a0 - k.base), p.x + k.a0, bytes, bar);
        bulk_g2s(ys + (k.a0 - k.base), p.y + k.a0, bytes, bar);
    } else {
        mbar_arrive(bar);
    }
}

template <int SPHI, int NK, bool REC>
__device__ __forceinline__ void vote_queued_xy(const VoteParams& p, const float* cp, const float* sp,
                                               const float4* dt_s, uint32_t* acc_s, uint32_t acc_sh, const uint4* hq,
                                               unsigned head, int n, int nj, int nk, int lane, uint8_t* rec_t,
                                               int64_t hb) {
    __syncwarp();
    const bool valid = lane < n;
    const uint4 ent = valid ? hq[(head + lane) & (kHitQueue - 1)] : make_uint4(0u, 0u, 0u, 0u);
    const int lo = valid ? (int)(ent.y & 0xFFFFu) : nj, hi = valid ? (int)(ent.y >> 16) : -1;
    const int ja = __reduce_min_sync(0xffffffffu, lo), jb = __reduce_max_sync(0xffffffffu, hi);
    __syncwarp();  // entries read before their slots are reused
    const float x = __uint_as_float(ent.z), y = __uint_as_float(ent.w);
    if (REC)
        vote_xy_rec<SPHI, NK>(p, cp, sp, dt_s, acc_s, acc_sh, ja, jb, nk, x, y, valid,
                              rec_t + ((int64_t)ent.x - hb) * p.rec_bytes);
    else
        vote_xy<SPHI, NK, true>(p, cp, sp, dt_s, acc_s, acc_sh, ja, jb, nk, x, y, valid);
}

// Per-warp band queues of the directly loaded band vote: two rings of
// kHitQueue entries, ring 0 the narrow bands (at most p.narrow columns),
// ring 1 the rest.  An entry is the hit's offset in its event and its band
// (lo | hi << 8, tile columns).
struct BandRings {
    uint32_t* off;   // [2][kHitQueue]
    uint16_t* band;  // [2][kHitQueue]
};

__host__ __device__ constexpr int band_ring_bytes() { return 2 * kHitQueue * 6; }

// One batch of up to 32 queued hits: lanes [0, n0) take ring c0 from head
// h0, lanes [n0, n0 + n1) ring 1 from head h1.  ALIGNED: each lane walks its
// own band (narrow or mixed batches); otherwise the hull of the bands.
template <int SPHI, int NK, bool REC, bool ALIGNED>
__device__ __forceinline__ void vote_batch(const VoteParams& p, const float* cp, const float* sp, const float4* dt_s,
                                           uint32_t* acc_s, uint32_t acc_sh, const BandRings& q, int c0, unsigned h0,
                                           int n0, unsigned h1, int n1, int nj, int nk, int lane, uint8_t* rec_t,
                                           int64_t hb) {
    __syncwarp();
    const bool valid = lane < n0 + n1;
    const int slot = lane < n0 ? c0 * kHitQueue + (int)((h0 + lane) & (kHitQueue - 1))
                               : kHitQueue + (int)((h1 + (lane - n0)) & (kHitQueue - 1));
    const uint32_t off = valid ? q.off[slot] : 0u;
    const unsigned bd = valid ? q.band[slot] : 0u;
    __syncwarp();  // entries read before their slots are reused
    const float x = valid ? p.x[hb + off] : 0.0f;
    const float y = valid ? p.y[hb + off] : 0.0f;
    uint8_t* rec = REC ? rec_t + (int64_t)off * p.rec_bytes : nullptr;
    if (ALIGNED) {
        const int lo = valid ? (int)(bd & 0xFFu) : 0, hi = valid ? (int)(bd >> 8) : -1;
        const int steps = __reduce_max_sync(0xffffffffu, (unsigned)(hi - lo + 1));
        vote_xy_al<SPHI, NK, REC>(p, cp, sp, dt_s, acc_s, acc_sh, lo, hi, steps, nk, x, y, valid, rec);
    } else {
        const int lo = valid ? (int)(bd & 0xFFu) : nj, hi = valid ? (int)(bd >> 8) : -1;
        const int ja = __reduce_min_sync(0xffffffffu, lo), jb = __reduce_max_sync(0xffffffffu, hi);
        if (REC)
            vote_xy_rec<SPHI, NK>(p, cp, sp, dt_s, acc_s, acc_sh, ja, jb, nk, x, y, valid, rec);
        else
            vote_xy<SPHI, NK, true>(p, cp, sp, dt_s, acc_s, acc_sh, ja, jb, nk, x, y, valid);
    }
}

template <int SPHI, int NK, bool REC, bool STAGE>
__global__ void __launch_bounds__(256, 3) vote_band_kernel(const VoteParams p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float4* dt_s = reinterpret_cast<float4*>(smem_raw);
    const int nthr = blockDim.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = nthr >> 5;
    // queues: staged, one ring of (hit, band, x, y); direct, two band rings
    const int qbytes = STAGE ? 16 * kHitQueue : band_ring_bytes();
    uint4* hq4 = reinterpret_cast<uint4*>(smem_raw + 16 * p.tile_d) + warp * kHitQueue;
    BandRings rings;
    rings.off = reinterpret_cast<uint32_t*>(smem_raw + 16 * p.tile_d) + warp * 2 * kHitQueue;
    rings.band = reinterpret_cast<uint16_t*>(smem_raw + 16 * p.tile_d + 8 * kHitQueue * nw) + warp * 2 * kHitQueue;
    float* stg = reinterpret_cast<float*>(smem_raw + 16 * p.tile_d + qbytes * nw);
    uint32_t* acc_s =
        reinterpret_cast<uint32_t*>(smem_raw + 16 * p.tile_d + qbytes * nw + (STAGE ? kStageBytes : 0));
    __shared__ int s_item;
    __shared__ __align__(8) uint64_t s_bar[2];
    unsigned par[2] = {0u, 0u};
    if (STAGE) {
        if (tid == 0) {
            mbar_init(&s_bar[0], 1);
            mbar_init(&s_bar[1], 1);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        __syncthreads();
    }

    const int nk = NK ? NK : p.K.nk;
    const int tiles = p.tiles_phi * p.tiles_d;
    const int col_words = SPHI * nk;
    const uint32_t acc_sh = smem_addr(acc_s);
    const unsigned lt = lanemask_lt();

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
        if (p.stats && tid == 0) atomicAdd(&p.stats[0], (unsigned long long)((he - hb) * nrows * nj));
        __syncthreads();

        const float dlo = dt_s[0].x, dhi = dt_s[nj - 1].x;
        // this tile's records and in-band bitmap words (REC)
        uint8_t* rec_t = nullptr;
        uint32_t* bits_t = nullptr;
        if (REC) {
            // within the wave's hits even for offsets the validation rejects
            // (the records are sized for the wave)
            const int64_t whb = clamp64(p.offs[p.event0], 0, p.n_hits);
            const int64_t wend = clamp64(p.offs[p.event0 + p.n_events], whb, p.n_hits);
            if (hb < whb || he > wend) {
                __syncthreads();
                continue;
            }
            rec_t = p.rec + ((hb - whb) * tiles + (int64_t)t * (he - hb)) * p.rec_bytes;
            bits_t = p.rbits + (((hb - whb) >> 5) + e) * (int64_t)tiles + (int64_t)t * ((he - hb + 31) >> 5);
        }
        unsigned head = 0, tail = 0;     // staged ring; direct: the wide ring
        unsigned nhead = 0, ntail = 0;   // direct: the narrow ring
        // one chunk of 32 hits: bands, the bitmap word, queueing and votes
        auto chunk = [&](int64_t c0, int64_t cend, const float* xs, const float* ys, int64_t base) {
            const int64_t h = c0 + lane;
            const bool valid = h < cend;
            const float x = valid ? (STAGE ? xs[h - base] : p.x[h]) : 0.0f;
            const float y = valid ? (STAGE ? ys[h - base] : p.y[h]) : 0.0f;
            const float r2 = fmaf(x, x, __fmul_rn(y, y));
            int lo = nj, hi = -1;
#pragma unroll
            for (int r = 0; r < SPHI; ++r) {
                int jl, jh;
                d0_band(r2, q_of(x, y, cp[r], sp[r]), dlo, dhi, j0, nj, p.K, jl, jh);
                if (jh >= jl) {
                    lo = min(lo, jl - j0);
                    hi = max(hi, jh - j0);
                }
            }
            const bool keep = valid && hi >= lo;
            const unsigned m = __ballot_sync(0xffffffffu, keep);
            if (REC && lane == 0) bits_t[(c0 - hb) >> 5] = m;
            if (STAGE) {
                const unsigned slot = (tail + __popc(m & lt)) & (kHitQueue - 1);
                const unsigned band = (unsigned)lo | ((unsigned)hi << 16);
                if (keep) hq4[slot] = make_uint4((unsigned)h, band, __float_as_uint(x), __float_as_uint(y));
                tail += __popc(m);
                if (tail - head >= 32) {
                    vote_queued_xy<SPHI, NK, REC>(p, cp, sp, dt_s, acc_s, acc_sh, hq4, head, 32, nj, nk, lane, rec_t, hb);
                    head += 32;
                }
            } else {
                const bool nar = keep && hi - lo < p.narrow;
                const unsigned mn = __ballot_sync(0xffffffffu, nar);
                const unsigned mw = m & ~mn;
                if (keep) {
                    const int slot = nar ? (int)((ntail + __popc(mn & lt)) & (kHitQueue - 1))
                                         : kHitQueue + (int)((tail + __popc(mw & lt)) & (kHitQueue - 1));
                    rings.off[slot] = (uint32_t)(h - hb);
                    rings.band[slot] = (uint16_t)(lo | (hi << 8));
                }
                ntail += __popc(mn);
                tail += __popc(mw);
                if (tail - head >= 32) {
                    vote_batch<SPHI, NK, REC, false>(p, cp, sp, dt_s, acc_s, acc_sh, rings, 1, head, 32, 0u, 0, nj, nk,
                                                     lane, rec_t, hb);
                    head += 32;
                }
                if (ntail - nhead >= 32) {
                    vote_batch<SPHI, NK, REC, true>(p, cp, sp, dt_s, acc_s, acc_sh, rings, 0, nhead, 32, 0u, 0, nj, nk,
                                                    lane, rec_t, hb);
                    nhead += 32;
                }
            }
        };
        if (!STAGE) {
            for (int64_t c0 = hb + warp * 32; c0 < he; c0 += nthr) chunk(c0, he, nullptr, nullptr, 0);
        } else {
            const int nblk = (int)((he - hb + kStageHits - 1) / kStageHits);
            if (tid == 0) {
                if (nblk > 0) stage_issue(p, stg, s_bar, hb, he, 0);
                if (nblk > 1) stage_issue(p, stg, s_bar, hb, he, 1);
            }
            for (int b = 0; b < nblk; ++b) {
                const int buf = b & 1;
                const bool ok = mbar_wait(&s_bar[buf], par[buf]);
                par[buf] ^= 1u;
                const StageBlock k = stage_block(hb, he, b);
                float* xs = stg + buf * 2 * kStageBuf;
                float* ys = xs + kStageBuf;
                if (tid < 3) {  // ragged head and tail, loaded directly
                    const int64_t h = k.b0 + tid;
                    if (h < k.a0) {
                        xs[h - k.base] = p.x[h];
                        ys[h - k.base] = p.y[h];
                    }
                } else if (tid < 6) {
                    const int64_t h = k.a1 + (tid - 3);
                    if (h < k.b1) {
                        xs[h - k.base] = p.x[h];
                        ys[h - k.base] = p.y[h];
                    }
                }
                if (__syncthreads_or(!ok)) {
                    // a copy never completed: report it, wait (bounded) for the
                    // copies still in flight into this block's memory, leave
                    if (tid == 0) {
                        atomicOr(p.err, 16);
                        mbar_wait(&s_bar[0], par[0]);
                        mbar_wait(&s_bar[1], par[1]);
                    }
                    __syncthreads();
                    return;
                }
                for (int64_t c0 = k.b0 + warp * 32; c0 < k.b1; c0 += nthr) chunk(c0, k.b1, xs, ys, k.base);
                __syncthreads();  // the block's buffer is no longer read
                if (tid == 0 && b + 2 < nblk) stage_issue(p, stg, s_bar, hb, he, b + 2);
            }
        }
        if (STAGE) {
            if (tail != head)
                vote_queued_xy<SPHI, NK, REC>(p, cp, sp, dt_s, acc_s, acc_sh, hq4, head, (int)(tail - head), nj, nk, lane,
                                              rec_t, hb);
        } else {
            // the rings' remainders: one batch walking each lane's own band
            // when they fit in 32 lanes together, else one batch each
            const int nn = (int)(ntail - nhead), nw2 = (int)(tail - head);
            if (nn + nw2 <= 32) {
                if (nn + nw2 > 0)
                    vote_batch<SPHI, NK, REC, true>(p, cp, sp, dt_s, acc_s, acc_sh, rings, 0, nhead, nn, head, nw2, nj,
                                                    nk, lane, rec_t, hb);
            } else {
                vote_batch<SPHI, NK, REC, true>(p, cp, sp, dt_s, acc_s, acc_sh, rings, 0, nhead, nn, 0u, 0, nj, nk, lane,
                                                rec_t, hb);
                vote_batch<SPHI, NK, REC, false>(p, cp, sp, dt_s, acc_s, acc_sh, rings, 1, head, nw2, 0u, 0, nj, nk,
                                                 lane, rec_t, hb);
            }
        }
        __syncthreads();

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
// pruned vote over (hit, column) items
// ---------------------------------------------------------------------------
// Each warp takes 32 consecutive hits of the item's event and computes their
// d0 bands for the tile (the union over the tile's rows, as above).  The
// band columns of those hits, in hit order, are the warp's work items; lanes
// take them 32 at a time.  Every lane leaves its hit's per-hit values in the
// warp's shared slot table and writes its lane number into the item map over
// its band's items, so an item's lane reads its hit with one byte load and
// four 16-byte loads.  No lane evaluates a column outside its hit's band,
// whatever the mix of band widths.
struct FlatHit {
    float4 a;        // x, y, r2, G
    float4 b;        // dmin, R1, (lo, first item) as int bits
    float q[8];      // q per row (up to 8 rows)
    float qs[8];     // q * S2 per row
};

__host__ __device__ constexpr int flat_slot_bytes(int sphi) { return 32 + 8 * ((sphi + 3) / 4 * 4); }

template <int SPHI, int NK, bool REC>
__global__ void __launch_bounds__(256, 3) vote_flat_kernel(const VoteParams p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float4* dt_s = reinterpret_cast<float4*>(smem_raw);
    const int nthr = blockDim.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = nthr >> 5;
    constexpr int QW = (SPHI + 3) / 4;  // float4s of q (and of qs) per slot
    constexpr int SLOT = flat_slot_bytes(SPHI) / 16;  // float4s per slot
    float4* slots = reinterpret_cast<float4*>(smem_raw + 16 * p.tile_d) + warp * 32 * SLOT;
    uint8_t* imap = smem_raw + 16 * p.tile_d + 16 * SLOT * 32 * nw + warp * 32 * p.tile_d;
    uint32_t* acc_s =
        reinterpret_cast<uint32_t*>(smem_raw + 16 * p.tile_d + 16 * SLOT * 32 * nw + ((32 * p.tile_d * nw + 15) & ~15));
    __shared__ int s_item;
    using W = typename RecWord<SPHI>::T;

    const int nk = NK ? NK : p.K.nk;
    const int tiles = p.tiles_phi * p.tiles_d;
    const int col_words = SPHI * nk;
    const uint32_t acc_sh = smem_addr(acc_s);
    const unsigned nku = (unsigned)nk;
    const float S2 = p.K.S2, H = p.K.H, T0 = p.K.T0;

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
        if (p.stats && tid == 0) atomicAdd(&p.stats[0], (unsigned long long)((he - hb) * nrows * nj));
        __syncthreads();

        const float dlo = dt_s[0].x, dhi = dt_s[nj - 1].x;
        uint8_t* rec_t = nullptr;
        uint32_t* bits_t = nullptr;
        if (REC) {
            // within the wave's hits even for offsets the validation rejects
            // (the records are sized for the wave)
            const int64_t whb = clamp64(p.offs[p.event0], 0, p.n_hits);
            const int64_t wend = clamp64(p.offs[p.event0 + p.n_events], whb, p.n_hits);
            if (hb < whb || he > wend) {
                __syncthreads();
                continue;
            }
            rec_t = p.rec + ((hb - whb) * tiles + (int64_t)t * (he - hb)) * p.rec_bytes;
            bits_t = p.rbits + (((hb - whb) >> 5) + e) * (int64_t)tiles + (int64_t)t * ((he - hb + 31) >> 5);
        }
        for (int64_t c0 = hb + warp * 32; c0 < he; c0 += nthr) {
            const int64_t h = c0 + lane;
            const bool valid = h < he;
            const float x = valid ? p.x[h] : 0.0f;
            const float y = valid ? p.y[h] : 0.0f;
            const float r2 = fmaf(x, x, __fmul_rn(y, y));
            float q[SPHI], qs[SPHI];
            int lo = nj, hi = -1;
#pragma unroll
            for (int r = 0; r < SPHI; ++r) {
                q[r] = q_of(x, y, cp[r], sp[r]);
                qs[r] = q[r] * S2;
                int jl, jh;
                d0_band(r2, q[r], dlo, dhi, j0, nj, p.K, jl, jh);
                if (jh >= jl) {
                    lo = min(lo, jl - j0);
                    hi = max(hi, jh - j0);
                }
            }
            const bool keep = valid && hi >= lo;
            const unsigned m = __ballot_sync(0xffffffffu, keep);
            if (REC && lane == 0) bits_t[(c0 - hb) >> 5] = m;
            if (m == 0u) continue;
            const int width = keep ? hi - lo + 1 : 0;
            int P = width;  // inclusive prefix of the band widths
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, P, o);
                if (lane >= o) P += v;
            }
            const int Wtot = __shfl_sync(0xffffffffu, P, 31);
            P -= width;  // exclusive
            const HitFast hf = hit_fast(x, y, p.K);
            __syncwarp();  // the previous chunk's slots and map are no longer read
            {
                float4* sl = slots + lane * SLOT;
                sl[0] = make_float4(x, y, hf.r2, hf.G);
                sl[1] = make_float4(hf.dmin, hf.R1, __int_as_float(lo), __int_as_float(P));
#pragma unroll
                for (int w4 = 0; w4 < QW; ++w4) {
                    float4 a, b;
                    a.x = 4 * w4 + 0 < SPHI ? q[4 * w4 + 0] : 0.0f;
                    a.y = 4 * w4 + 1 < SPHI ? q[4 * w4 + 1] : 0.0f;
                    a.z = 4 * w4 + 2 < SPHI ? q[4 * w4 + 2] : 0.0f;
                    a.w = 4 * w4 + 3 < SPHI ? q[4 * w4 + 3] : 0.0f;
                    b.x = 4 * w4 + 0 < SPHI ? qs[4 * w4 + 0] : 0.0f;
                    b.y = 4 * w4 + 1 < SPHI ? qs[4 * w4 + 1] : 0.0f;
                    b.z = 4 * w4 + 2 < SPHI ? qs[4 * w4 + 2] : 0.0f;
                    b.w = 4 * w4 + 3 < SPHI ? qs[4 * w4 + 3] : 0.0f;
                    sl[2 + w4] = a;
                    sl[2 + QW + w4] = b;
                }
                for (int k = 0; k < width; ++k) imap[P + k] = (uint8_t)lane;
            }
            W* rw_own = REC ? reinterpret_cast<W*>(rec_t + (h - hb) * p.rec_bytes) : nullptr;
            if (REC && keep) {
                const W none = (W)~(W)0;
                for (int j = 0; j < lo; ++j) rw_own[j] = none;
                for (int j = hi + 1; j < p.tile_d; ++j) rw_own[j] = none;
            }
            __syncwarp();
            for (int s0 = 0; s0 < Wtot; s0 += 32) {
                const int itm = s0 + lane;
                const bool act = itm < Wtot;
                const int o = act ? imap[itm] : 0;
                const float4* sl = slots + o * SLOT;
                const float4 A0 = sl[0], A1 = sl[1];
                const int j = act ? __float_as_int(A1.z) + (itm - __float_as_int(A1.w)) : 0;
                float oq[SPHI], oqs[SPHI];
#pragma unroll
                for (int w4 = 0; w4 < QW; ++w4) {
                    const float4 a = sl[2 + w4], b = sl[2 + QW + w4];
                    if (4 * w4 + 0 < SPHI) { oq[4 * w4 + 0] = a.x; oqs[4 * w4 + 0] = b.x; }
                    if (4 * w4 + 1 < SPHI) { oq[4 * w4 + 1] = a.y; oqs[4 * w4 + 1] = b.y; }
                    if (4 * w4 + 2 < SPHI) { oq[4 * w4 + 2] = a.z; oqs[4 * w4 + 2] = b.z; }
                    if (4 * w4 + 3 < SPHI) { oq[4 * w4 + 3] = a.w; oqs[4 * w4 + 3] = b.w; }
                }
                const float4 dt = dt_s[j];
                const float Rj = A0.z + dt.z;
                const uint32_t col_sh = acc_sh + 4u * (unsigned)(j * col_words);
                bool und = false;
                uint32_t wlo = 0, whi = 0;
#pragma unroll
                for (int r = 0; r < SPHI; ++r) {
                    const S1 c = stage1_fast(oqs[r], oq[r], dt, Rj, A0.w, H, T0);
                    const uint32_t addr = col_sh + 4u * ((unsigned)(r * nk) + c.kb);
                    if (REC) {
                        if (r < 4)
                            wlo = red_and_byte(addr, c.flo, c.fhi, c.kb, nku, act, wlo, 8u * r);
                        else
                            whi = red_and_byte(addr, c.flo, c.fhi, c.kb, nku, act, whi, 8u * (r - 4));
                    } else {
                        red_if_vote(addr, c.flo, c.fhi, c.kb, nku, act);
                    }
                    und |= (c.flo != c.fhi) & act;
                }
                W word = (W)(SPHI == 8 ? ((unsigned long long)whi << 32) | wlo : wlo);
                if (__any_sync(0xffffffffu, und)) {
#pragma unroll
                    for (int r = 0; r < SPHI; ++r) {
                        const S1 c = stage1_fast(oqs[r], oq[r], dt, Rj, A0.w, H, T0);
                        if ((c.flo != c.fhi) && act && stage1_pending(c, A1.x, p.K.wlo, p.K.whi)) {
                            const int kk = cell_slow(A0.x, A0.y, cp[r], sp[r], dt.x, A1.y, p.K, p.stats);
                            if (kk >= 0) atomicAdd(acc_s + j * col_words + r * nk + kk, 1u);
                            if (REC)
                                word = (word & ~((W)0xFF << (8 * r))) |
                                       ((W)(kk >= 0 ? (unsigned)kk : 255u) << (8 * r));
                        }
                    }
                }
                if (REC && act) {
                    W* rw = reinterpret_cast<W*>(rec_t + (c0 + o - hb) * p.rec_bytes);
                    rw[j] = word;
                }
            }
        }
        __syncthreads();

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
// range vote: every kappa bin between a cell's corner bins
// ---------------------------------------------------------------------------
// The tile's corners are its SPHI + 1 phi0 edges by nj + 1 d0 edges.  Each
// thread sweeps its hit across the d0 edges, binning the SPHI + 1 corners of
// one edge (stage 1, stages 2 and 3 for undecided corners) while keeping the
// previous edge's codes, and votes each cell between the two edges for the
// bins from its lowest to its highest corner code.  A vote for bins [lo, hi]
// adds 1 at lo and subtracts 1 at hi + 1 of the column in shared memory (two
// atomics whatever the width: an inner-layer hit can span tens of bins); the
// flush turns each column into counts by a prefix sum over kappa.
template <int SPHI, int NK, bool TAIL>
__device__ __forceinline__ void vote_range_one_hit(const VoteParams& p, const float* ce, const float* se,
                                                   const float4* dte_s, uint32_t* acc_s, int nj, int nk, int64_t h,
                                                   bool valid) {
    const float x = (!TAIL || valid) ? p.x[h] : 0.0f;
    const float y = (!TAIL || valid) ? p.y[h] : 0.0f;
    const HitFast hf = hit_fast(x, y, p.K);
    const float S2 = p.K.S2, H = p.K.H, T0 = p.K.T0;
    float qe[SPHI + 1], qse[SPHI + 1];
#pragma unroll
    for (int m = 0; m <= SPHI; ++m) {
        qe[m] = q_of(x, y, ce[m], se[m]);
        qse[m] = qe[m] * S2;
    }
    int prev[SPHI + 1], cur[SPHI + 1];
    const int col_words = SPHI * nk;
    for (int n = 0; n <= nj; ++n) {
        const float4 dt = dte_s[n];
        const float Rj = hf.r2 + dt.z;
        bool und = false;
#pragma unroll
        for (int m = 0; m <= SPHI; ++m) {
            const S1 o = stage1_fast(qse[m], qe[m], dt, Rj, hf.G, H, T0);
            cur[m] = (!TAIL || valid) ? code_stage1(o, hf.dmin, nk) : kCodeUndef;
            und |= cur[m] == kCodeUndecided;
        }
        if (__any_sync(0xffffffffu, und)) {
#pragma unroll
            for (int m = 0; m <= SPHI; ++m)
                if (cur[m] == kCodeUndecided) cur[m] = code_slow(x, y, ce[m], se[m], dt.x, hf.R1, p.K, p.stats);
        }
        if (n > 0) {
            uint32_t* col = acc_s + (n - 1) * col_words;
#pragma unroll
            for (int r = 0; r < SPHI; ++r) {
                const int a = min(min(prev[r], prev[r + 1]), min(cur[r], cur[r + 1]));
                const int b = max(max(prev[r], prev[r + 1]), max(cur[r], cur[r + 1]));
                const bool undef = prev[r] == kCodeUndef || prev[r + 1] == kCodeUndef || cur[r] == kCodeUndef ||
                                   cur[r + 1] == kCodeUndef;
                if (!undef && b >= 0 && a < nk) {
                    const int lo = max(a, 0), hi = min(b, nk - 1);
                    atomicAdd(col + r * nk + lo, 1u);
                    if (hi + 1 < nk) atomicAdd(col + r * nk + hi + 1, 0xFFFFFFFFu);  // -1 mod 2^32
                }
            }
        }
#pragma unroll
        for (int m = 0; m <= SPHI; ++m) prev[m] = cur[m];
    }
}

template <int SPHI, int NK>
__global__ void __launch_bounds__(256, 3) vote_range_kernel(const VoteParams p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float4* dte_s = reinterpret_cast<float4*>(smem_raw);
    uint32_t* acc_s = reinterpret_cast<uint32_t*>(smem_raw + 16 * (p.tile_d + 1));
    __shared__ int s_item;

    const int nk = NK ? NK : p.K.nk;
    const int nthr = blockDim.x;
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int tiles = p.tiles_phi * p.tiles_d;
    const int col_words = SPHI * nk;

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
        for (int n = tid; n <= nj; n += nthr) dte_s[n] = p.edtab[j0 + n];
        // phi0 edges of the tile (periodic); rows past a ragged edge vote into
        // tile slots that are never flushed
        float ce[SPHI + 1], se[SPHI + 1];
#pragma unroll
        for (int m = 0; m <= SPHI; ++m) {
            const int i = (i0 + m) % p.K.nphi;
            ce[m] = p.ecos[i];
            se[m] = p.esin[i];
        }
        if (p.stats && tid == 0) atomicAdd(&p.stats[0], (unsigned long long)((he - hb) * nrows * nj));
        __syncthreads();

        const int64_t nfull = ((he - hb) / nthr) * nthr;
        for (int64_t h = hb + tid; h < hb + nfull; h += nthr)
            vote_range_one_hit<SPHI, NK, false>(p, ce, se, dte_s, acc_s, nj, nk, h, true);
        {
            const int64_t h = hb + nfull + tid;
            if (hb + nfull + (tid - lane) < he)
                vote_range_one_hit<SPHI, NK, true>(p, ce, se, dte_s, acc_s, nj, nk, h, h < he);
        }
        __syncthreads();

        // counts = prefix sums of the differences along kappa, 32 bins a step
        uint32_t* dst_e = p.acc + (int64_t)e * p.cells;
        const int warp = tid >> 5, nw = nthr >> 5;
        const int nrj = nrows * nj;
        for (int row = warp; row < nrj; row += nw) {
            const int r = row / nj;
            const int j = row - r * nj;
            const uint32_t* src = acc_s + j * col_words + r * nk;
            uint32_t* dst = dst_e + ((int64_t)(i0 + r) * p.K.nd + (j0 + j)) * nk;
            uint32_t carry = 0;
            for (int k0 = 0; k0 < nk; k0 += 32) {
                const int kk = k0 + lane;
                uint32_t v = kk < nk ? src[kk] : 0u;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t u = __shfl_up_sync(0xffffffffu, v, o);
                    if (lane >= o) v += u;
                }
                v += carry;
                if (kk < nk) dst[kk] = v;
                carry = __shfl_sync(0xffffffffu, v, 31);
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// line vote (the kappa = 0 model): every hit, every phi0 row, one d0 bin
// ---------------------------------------------------------------------------
// q = y cos phi_i - x sin phi_i from exact binary64 products of the float
// inputs (rounded once), its bin floor((q - d0_min) n_d0 / (d0_max - d0_min))
// in binary64; a block per event, global atomics into the zeroed
// accumulator [phi][d0] (one kappa bin).
__global__ void vote_line_kernel(const VoteParams p, double d0min, double d0max) {
    const int nphi = p.K.nphi, nd = p.K.nd;
    const double ndr = (double)nd;
    const double scale = __ddiv_rn(ndr, __dsub_rn(d0max, d0min));
    for (int e = blockIdx.x; e < p.n_events; e += gridDim.x) {
        const int64_t hb = clamp64(p.offs[p.event0 + e], 0, p.n_hits);
        const int64_t he = clamp64(p.offs[p.event0 + e + 1], hb, p.n_hits);
        uint32_t* a1 = p.acc + (int64_t)e * p.cells;
        const int64_t work = (he - hb) * nphi;
        for (int64_t t = threadIdx.x; t < work; t += blockDim.x) {
            const int64_t h = hb + t / nphi;
            const int i = (int)(t - (t / nphi) * nphi);
            const double q = __dsub_rn(__dmul_rn((double)p.y[h], (double)p.cphi[i]),
                                       __dmul_rn((double)p.x[h], (double)p.sphi[i]));
            const double u = __dmul_rn(__dsub_rn(q, d0min), scale);
            if (u >= 0.0 && u < ndr) atomicAdd(a1 + (int64_t)i * nd + (int)u, 1u);
        }
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
// peaks: detection by running maxima
// ---------------------------------------------------------------------------
// The 26 neighbours of cell (i, j, k) split into the plane of row i - 1, the
// plane of row i + 1, the columns (i, j - 1) and (i, j + 1), and the bins
// k - 1 and k + 1 of the cell's own column.  With K(r, c) the maximum of
// bins k - 1..k + 1 of column (r, c) and P(r) = max(K(r, j - 1), K(r, j),
// K(r, j + 1)), the earlier neighbours' maximum is
//   max(P(i - 1) if row i - 1 precedes row i, P(i + 1) if row i + 1 precedes
//       row i (the phi wrap at the last row), K(i, j - 1), A(i, j, k - 1))
// and the later neighbours' maximum the same with the other rows, K(i, j + 1)
// and A(i, j, k + 1); absent neighbours read -1.  A warp takes one (event,
// phi row, 32-bin kappa chunk), lanes over kappa, and walks the d0 columns
// in order, keeping K of rows i - 1, i, i + 1 at three consecutive columns in
// registers: each step loads one new column of each row (one coalesced load
// plus the chunk's two halo bins).  It writes the chunk's peak word and its
// population count; detect_words_kernel turns the counts into per-word
// prefixes and the column's total.
// One column of one row, a warp's 32-bin kappa chunk: the raw loads (issued
// a step ahead) and their 3-bin maxima.  Lane 0 and lane 31 also load the
// chunk's halo bins k0 - 1 and k0 + 32.
struct ColRaw {
    int a, h;
};

__device__ __forceinline__ ColRaw col_load(const uint32_t* colp, int k, int nk, int lane) {
    ColRaw r;
    r.a = k < nk ? (int)__ldg(colp + k) : -1;
    const int hk = lane == 0 ? k - 1 : k + 1;
    r.h = ((lane == 0 || lane == 31) && hk >= 0 && hk < nk) ? (int)__ldg(colp + hk) : -1;
    return r;
}

// a, its kappa neighbours am / ap (-1 when absent) and kx = max(am, a, ap)
__device__ __forceinline__ void col_max(ColRaw r, int k, int nk, int lane, int& a, int& am, int& ap, int& kx) {
    a = r.a;
    am = __shfl_up_sync(0xffffffffu, a, 1);
    ap = __shfl_down_sync(0xffffffffu, a, 1);
    if (lane == 0) am = r.h;
    if (lane == 31) ap = r.h;
    if (k + 1 >= nk) ap = -1;
    kx = max(a, max(am, ap));
}

// RB output rows per warp (rows i0 .. i0 + RB - 1 and their two neighbour
// rows, loaded once per column step for all of them).
template <int RB>
__global__ void __launch_bounds__(256) detect_slide_kernel(const PeakParams p) {
    constexpr int NR = RB + 2;  // rows i0 - 1 .. i0 + RB
    const int lane = threadIdx.x & 31;
    const int nk = p.nk, nkw = p.nkw, nd = p.nd, nphi = p.nphi;
    const int nblk = (nphi + RB - 1) / RB;
    const int64_t items = (int64_t)p.n_events * nblk * nkw;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t item = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); item < items; item += nwarps) {
        const int kc = (int)(item % nkw);
        const int64_t eb = item / nkw;
        const int ib = (int)(eb % nblk);
        const int e = (int)(eb / nblk);
        const int i0 = ib * RB;
        const int nout = min(RB, nphi - i0);
        const int k = kc * 32 + lane;
        const uint32_t* A = p.acc + (int64_t)e * p.cells;
        const uint32_t* R[NR];
#pragma unroll
        for (int t = 0; t < NR; ++t) {
            int r = i0 - 1 + t;
            r = ((r % nphi) + nphi) % nphi;
            R[t] = A + (int64_t)r * nd * nk;
        }
        // window per row: K at columns j - 1, j, j + 1; own bins at column j
        int K0[NR], K1[NR], K2[NR];
        int a1[NR], am1[NR], ap1[NR];
        ColRaw nx[NR];
#pragma unroll
        for (int t = 0; t < NR; ++t) {
            K0[t] = -1;
            col_max(col_load(R[t], k, nk, lane), k, nk, lane, a1[t], am1[t], ap1[t], K1[t]);
            nx[t] = nd > 1 ? col_load(R[t] + nk, k, nk, lane) : ColRaw{-1, -1};
        }
        const int64_t col0 = ((int64_t)e * nphi + i0) * nd;
        for (int j = 0; j < nd; ++j) {
            int a2[NR], am2[NR], ap2[NR];
#pragma unroll
            for (int t = 0; t < NR; ++t) {
                if (j + 1 < nd) {
                    col_max(nx[t], k, nk, lane, a2[t], am2[t], ap2[t], K2[t]);
                } else {
                    a2[t] = am2[t] = ap2[t] = K2[t] = -1;
                }
                // the loads of column j + 2 are in flight during this step
                nx[t] = j + 2 < nd ? col_load(R[t] + (int64_t)(j + 2) * nk, k, nk, lane) : ColRaw{-1, -1};
            }
#pragma unroll
            for (int o = 0; o < RB; ++o) {
                if (o < nout) {  // warp-uniform
                    const int i = i0 + o;
                    const int c = o + 1;  // window row of output row i
                    const bool planes = nphi > 1;  // one row: the planes are the cell's own column
                    const int Pm = planes ? max(K0[c - 1], max(K1[c - 1], K2[c - 1])) : -1;
                    const int Pp = planes ? max(K0[c + 1], max(K1[c + 1], K2[c + 1])) : -1;
                    const bool m_earlier = i > 0, p_earlier = i == nphi - 1;
                    const int E = max(max(m_earlier ? Pm : -1, p_earlier ? Pp : -1), max(K0[c], am1[c]));
                    const int L = max(max(m_earlier ? -1 : Pm, p_earlier ? -1 : Pp), max(K2[c], ap1[c]));
                    const int v = a1[c];
                    const bool pk = k < nk && (uint32_t)v >= p.thr && v > E && v >= L;
                    const unsigned b = __ballot_sync(0xffffffffu, pk);
                    if (lane == 0) {
                        const int64_t col = col0 + (int64_t)o * nd + j;
                        p.mask[col * nkw + kc] = b;
                        p.wpre[col * nkw + kc] = (uint16_t)__popc(b);
                    }
                }
            }
#pragma unroll
            for (int t = 0; t < NR; ++t) {
                K0[t] = K1[t];
                K1[t] = K2[t];
                a1[t] = a2[t];
                am1[t] = am2[t];
                ap1[t] = ap2[t];
            }
        }
    }
}

// The same rule with 16-byte loads (n_kappa a multiple of 4): lane L holds
// bins c*128 + 4L .. c*128 + 4L + 3 of a 128-bin chunk c, so a warp covers
// a 128-bin chunk of a column with one load; a bin's kappa neighbours come
// from the lane's own registers and one shuffle each way (lanes 0 and 31
// load the chunk's halo bins).  Peak bits are gathered into 32-bit words by
// three xor shuffles over each group of eight lanes.  RB output rows per
// warp, loads a column ahead.
struct Col4 {
    int v[4];
    int h;  // halo: lane 0 bin c*128 - 1, lane 31 bin c*128 + 128
};

__device__ __forceinline__ Col4 col4_load(const uint32_t* colp, int kb, int nk, int lane) {
    Col4 r;
    if (kb < nk) {
        const uint4 q = __ldg(reinterpret_cast<const uint4*>(colp + kb));
        r.v[0] = (int)q.x;
        r.v[1] = (int)q.y;
        r.v[2] = (int)q.z;
        r.v[3] = (int)q.w;
    } else {
        r.v[0] = r.v[1] = r.v[2] = r.v[3] = -1;
    }
    const int hk = lane == 0 ? kb - 1 : kb + 4;
    r.h = ((lane == 0 || lane == 31) && hk >= 0 && hk < nk) ? (int)__ldg(colp + hk) : -1;
    return r;
}

// kappa 3-bin maxima of the lane's four bins; lf / rt: the bins just left
// of the first and right of the last (-1 when absent)
__device__ __forceinline__ void col4_max(const Col4& c, int lane, int* K, int& lf, int& rt) {
    lf = __shfl_up_sync(0xffffffffu, c.v[3], 1);
    rt = __shfl_down_sync(0xffffffffu, c.v[0], 1);
    if (lane == 0) lf = c.h;
    if (lane == 31) rt = c.h;
    const int m01 = max(c.v[0], c.v[1]), m12 = max(c.v[1], c.v[2]), m23 = max(c.v[2], c.v[3]);
    K[0] = max(lf, m01);
    K[1] = max(m01, c.v[2]);
    K[2] = max(c.v[1], m23);
    K[3] = max(m23, rt);
}

template <int RB>
__global__ void __launch_bounds__(128) detect_vec_kernel(const PeakParams p) {
    constexpr int NR = RB + 2;  // rows i0 - 1 .. i0 + RB
    const int lane = threadIdx.x & 31;
    const int nk = p.nk, nkw = p.nkw, nd = p.nd, nphi = p.nphi;
    const int nch = (nk + 127) >> 7;
    const int nblk = (nphi + RB - 1) / RB;
    const int64_t items = (int64_t)p.n_events * nblk * nch;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t item = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); item < items; item += nwarps) {
        const int ch = (int)(item % nch);
        const int64_t eb = item / nch;
        const int ib = (int)(eb % nblk);
        const int e = (int)(eb / nblk);
        const int i0 = ib * RB;
        const int nout = min(RB, nphi - i0);
        const int kb = ch * 128 + 4 * lane;
        const uint32_t* A = p.acc + (int64_t)e * p.cells;
        const uint32_t* R[NR];
#pragma unroll
        for (int t = 0; t < NR; ++t) {
            int r = i0 - 1 + t;
            r = ((r % nphi) + nphi) % nphi;
            R[t] = A + (int64_t)r * nd * nk;
        }
        const bool planes = nphi > 1;  // one row: the planes are the cell's own column
        // window: K at columns j - 1 (0), j (1), j + 1 (2) for every row;
        // the own bins' neighbours of the output rows at column j
        int K[3][NR][4];
        int own[RB][4], lfo[RB], rto[RB];
        Col4 nx[NR];
#pragma unroll
        for (int t = 0; t < NR; ++t) {
#pragma unroll
            for (int q = 0; q < 4; ++q) K[0][t][q] = -1;
            const Col4 c0 = col4_load(R[t], kb, nk, lane);
            int lf, rt;
            col4_max(c0, lane, K[1][t], lf, rt);
            if (t >= 1 && t <= RB) {
#pragma unroll
                for (int q = 0; q < 4; ++q) own[t - 1][q] = c0.v[q];
                lfo[t - 1] = lf;
                rto[t - 1] = rt;
            }
            nx[t] = nd > 1 ? col4_load(R[t] + nk, kb, nk, lane) : Col4{{-1, -1, -1, -1}, -1};
        }
        const int64_t col0 = ((int64_t)e * nphi + i0) * nd;
        for (int j = 0; j < nd; ++j) {
            int own2[RB][4], lf2[RB], rt2[RB];
#pragma unroll
            for (int t = 0; t < NR; ++t) {
                int lf = -1, rt = -1;
                if (j + 1 < nd) {
                    col4_max(nx[t], lane, K[2][t], lf, rt);
                } else {
#pragma unroll
                    for (int q = 0; q < 4; ++q) K[2][t][q] = -1;
                }
                if (t >= 1 && t <= RB) {
#pragma unroll
                    for (int q = 0; q < 4; ++q) own2[t - 1][q] = j + 1 < nd ? nx[t].v[q] : -1;
                    lf2[t - 1] = lf;
                    rt2[t - 1] = rt;
                }
                // the loads of column j + 2 are in flight during this step
                nx[t] = j + 2 < nd ? col4_load(R[t] + (int64_t)(j + 2) * nk, kb, nk, lane)
                                   : Col4{{-1, -1, -1, -1}, -1};
            }
#pragma unroll
            for (int o = 0; o < RB; ++o) {
                if (o < nout) {  // warp-uniform
                    const int i = i0 + o;
                    const int c = o + 1;
                    const bool m_earlier = i > 0, p_earlier = i == nphi - 1;
                    unsigned nib = 0;
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int Pm = planes ? max(K[0][c - 1][q], max(K[1][c - 1][q], K[2][c - 1][q])) : -1;
                        const int Pp = planes ? max(K[0][c + 1][q], max(K[1][c + 1][q], K[2][c + 1][q])) : -1;
                        const int km = q == 0 ? lfo[o] : own[o][q - 1];   // bin k - 1 of the own column
                        const int kp = q == 3 ? rto[o] : own[o][q + 1];   // bin k + 1
                        const int E = max(max(m_earlier ? Pm : -1, p_earlier ? Pp : -1), max(K[0][c][q], km));
                        const int L = max(max(m_earlier ? -1 : Pm, p_earlier ? -1 : Pp), max(K[2][c][q], kp));
                        const int v = own[o][q];
                        const bool pk = kb + q < nk && (uint32_t)v >= p.thr && v > E && v >= L;
                        nib |= (unsigned)pk << q;
                    }
                    // lanes 8w .. 8w + 7 hold word ch * 4 + w
                    unsigned word = nib << (4 * (lane & 7));
                    word |= __shfl_xor_sync(0xffffffffu, word, 1);
                    word |= __shfl_xor_sync(0xffffffffu, word, 2);
                    word |= __shfl_xor_sync(0xffffffffu, word, 4);
                    const int w = ch * 4 + (lane >> 3);
                    if ((lane & 7) == 0 && w < nkw) {
                        const int64_t col = col0 + (int64_t)o * nd + j;
                        p.mask[col * nkw + w] = word;
                        p.wpre[col * nkw + w] = (uint16_t)__popc(word);
                    }
                }
            }
#pragma unroll
            for (int t = 0; t < NR; ++t)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    K[0][t][q] = K[1][t][q];
                    K[1][t][q] = K[2][t][q];
                }
#pragma unroll
            for (int o = 0; o < RB; ++o) {
#pragma unroll
                for (int q = 0; q < 4; ++q) own[o][q] = own2[o][q];
                lfo[o] = lf2[o];
                rto[o] = rt2[o];
            }
        }
    }
}

// Per column: the words' peak counts (left in wpre by detect_slide_kernel)
// become the count of peaks in the column's earlier words; npk the total.
__global__ void detect_words_kernel(const PeakParams p) {
    const int64_t ncols = (int64_t)p.n_events * p.nphi * p.nd;
    const int nkw = p.nkw;
    for (int64_t col = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; col < ncols;
         col += (int64_t)gridDim.x * blockDim.x) {
        uint16_t* w = p.wpre + col * nkw;
        int run = 0;
        for (int t = 0; t < nkw; ++t) {
            const int c = w[t];
            w[t] = (uint16_t)run;
            run += c;
        }
        p.npk[col] = run;
    }
}

// peaks: emission in (event, linear index) order + per-peak pair counts.
// One lane per column: the column's peaks (few) are walked in bin order;
// pairs of peaks past the capacity are summed per lane and added once per
// warp.
__global__ void emit_kernel(const PeakParams p) {
    const int64_t per_ev = (int64_t)p.nphi * p.nd;
    const int64_t ncols = per_ev * p.n_events;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t c0 = (int64_t)blockIdx.x * blockDim.x; c0 < ncols; c0 += stride) {
        const int64_t col = c0 + threadIdx.x;
        unsigned long long extra = 0;
        const int npk = col < ncols ? p.npk[col] : 0;
        if (npk > 0) {
            const int64_t base = p.colbase[col];
            if (!(base >= p.peak_cap && p.window < 0)) {
                const int e = (int)(col / per_ev);
                const int ij = (int)(col - e * per_ev);
                const int i = ij / p.nd;
                const int j = ij - i * p.nd;
                const uint32_t* colp = p.acc + (int64_t)e * p.cells + ((int64_t)i * p.nd + j) * p.nk;
                int64_t pid = base;
                for (int w = 0; w < p.nkw; ++w) {
                    for (unsigned m = p.mask[col * p.nkw + w]; m; m &= m - 1u, ++pid) {
                        const int k = w * 32 + __ffs(m) - 1;
                        if (pid >= p.peak_cap) {
                            if (p.window >= 0 && p.extra_pairs) {
                                const int lo = max(0, k - p.window), hi = min(p.nk - 1, k + p.window);
                                for (int kk = lo; kk <= hi; ++kk) extra += colp[kk];
                            }
                            continue;
                        }
                        ht_peak pk;
                        pk.event = p.event0 + e;
                        pk.i_phi = i;
                        pk.i_d0 = p.line ? k : j;  // line voting runs peaks on the [phi][1][d0] view
                        pk.i_kappa = p.line ? 0 : k;
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
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) extra += __shfl_xor_sync(0xffffffffu, extra, o);
        if (extra && (threadIdx.x & 31) == 0)
            atomicAdd(reinterpret_cast<unsigned long long*>(p.extra_pairs), extra);
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
// association: rows in hit order, one warp per item.  An item is SPHI phi
// rows x up to `wd` d0 columns of one event (at most 32 columns; SPHI > 1
// only with wd == n_d0, so the item's columns, and therefore its peaks, are
// consecutive in the peak numbering).  The warp loads the item's peak
// bitmasks, marks the kappa bins within `window` of a peak ("near" bits) and
// walks the event's hits 32 at a time in increasing order through the same
// certified binning as the vote.  Cells whose bin is near a peak enter a
// per-warp FIFO ring by ballot rank, so for every column the ring holds hits
// in increasing order.  A drain hands 32 entries to the 32 lanes, which rank
// themselves among the lanes holding the same peak (a match over peak ids);
// one lane per peak moves the row's cursor.  A row is written by one warp
// only, drain after drain, so it comes out in ascending hit order with no
// atomics and no sort.  Cursors live in shared memory, `cap` per warp; an
// item with more peaks is walked once per block of `cap` peaks.
// ---------------------------------------------------------------------------
// Columns per step of the cell loop (each with SPHI rows), and the ring
// size: a step pushes at most 32 entries per cell on top of < 32 waiting.
__host__ __device__ constexpr int assoc_unroll(int sphi) { return sphi >= 2 ? 1 : 2; }
__host__ __device__ constexpr int assoc_ring(int sphi) {
    int r = 64;
    while (r < 32 * (assoc_unroll(sphi) * sphi + 1)) r <<= 1;
    return r;
}

struct AssocWarp {
    float4* dt;      // [wd] d0 table of the item's columns
    uint32_t* cur;   // [cap] row cursors of the pass's peaks (offsets from the pass's first row)
    uint2* ring;     // [assoc_ring(rows)] (column << 16 | kappa bin, hit)
    uint2* hq;       // [kHitQueue] (hit, d0 band bits) of banded hits
    uint32_t* mask;  // [rows * wd][nkw] peak bits of the item's columns
    uint32_t* nearb; // [rows * wd][nk / 32 + 1] bins within `window` of a peak; bin nk (no bin) is 0
    int32_t* lpre;   // [rows * wd][nkw] item-local id of the first peak of each word
};

__host__ __device__ inline size_t assoc_warp_bytes(int rows, int wd, int nk, int cap) {
    const size_t nkw = (nk + 31) / 32, nkn = nk / 32 + 1;
    return ((16 * (size_t)wd + 4 * (size_t)cap + 8 * (size_t)(assoc_ring(rows) + kHitQueue) +
             4 * (size_t)rows * wd * (2 * nkw + nkn)) +
            15) &
           ~size_t(15);
}

struct AssocPass {
    int L0, L1;     // item-local peak ids of this pass
    bool whole;     // the pass holds all of the item's stored peaks
    int64_t Q;      // first row offset of the pass
};

// Rows of the n (<= 32) ring entries from `head`, lane i taking entry i.  An
// entry's peaks lie within `window` of its bin and at least two bins apart
// (a peak is strictly above its lower kappa neighbour and not below its
// upper one), so the peak at bin k can be given round (k >> 1) mod R, R the
// power of two >= window + 1: no entry has two peaks in one round, and every
// entry holding a given peak meets it in the same round.  In a round, lanes
// with equal peaks match; each takes its rank among them (lane order, which
// is hit order for a column) and the group's lowest lane moves the row's
// cursor.  When no entry holds two peaks, one round over all of them does.
template <int RING>
__device__ __forceinline__ void assoc_drain(const AssocParams& p, const AssocWarp& S, int nkw, int nk, unsigned head,
                                            int n, const AssocPass& ps, int lane) {
    __syncwarp();
    const bool has = lane < n;
    const uint2 ent = has ? S.ring[(head + lane) & (RING - 1)] : make_uint2(0u, 0u);
    const int c = (int)(ent.x >> 16), kb = (int)(ent.x & 0xFFFFu);
    const int w = p.window;
    const int k0 = kb - w;
    // pending: the peaks of column c (of this pass) at k0 + rel, rel in [0, 2w]
    unsigned pend = 0;
    if (has) {
        const uint32_t* m = S.mask + c * nkw;
        const int lo = max(k0, 0), hi = min(kb + w, nk - 1);
        const int a = lo >> 5, b = hi >> 5;  // b <= a + 1 since 2w < 32
        const unsigned long long two =
            ((unsigned long long)(b > a ? m[b] : 0u) << 32) | (unsigned long long)m[a];
        const unsigned span = (unsigned)(two >> (lo & 31)) & (0xFFFFFFFFu >> (31 - (hi - lo)));
        pend = span << (lo - k0);
        if (!ps.whole) {
            for (unsigned bits = pend; bits; bits &= bits - 1u) {
                const int rel = __ffs(bits) - 1;
                const int kk = k0 + rel;
                const uint32_t word = m[kk >> 5];
                const int local = S.lpre[c * nkw + (kk >> 5)] + __popc(word & ((1u << (kk & 31)) - 1u));
                if (local < ps.L0 || local >= ps.L1) pend &= ~(1u << rel);
            }
        }
    }
    const unsigned lt = lanemask_lt();
    const bool multi = __any_sync(0xffffffffu, (pend & (pend - 1u)) != 0u);
    int R = 1;
    if (multi)
        while (R < w + 1) R <<= 1;
    for (int s = 0; s < R; ++s) {
        int loc = -1;  // this lane's peak of round s, id within the pass
        for (unsigned bits = pend; bits; bits &= bits - 1u) {
            const int rel = __ffs(bits) - 1;
            const int kk = k0 + rel;
            if (multi && (((kk >> 1) & (R - 1)) != s)) continue;
            const uint32_t word = S.mask[c * nkw + (kk >> 5)];
            loc = S.lpre[c * nkw + (kk >> 5)] + __popc(word & ((1u << (kk & 31)) - 1u)) - ps.L0;
            break;
        }
        if (!__any_sync(0xffffffffu, loc >= 0)) continue;
        const unsigned key = loc >= 0 ? (unsigned)loc : (0x80000000u | (unsigned)lane);
        const unsigned grp = __match_any_sync(0xffffffffu, key);
        const int leader = __ffs(grp) - 1;
        uint32_t base = 0;
        if (loc >= 0 && lane == leader) {  // the only lane touching this row's cursor in this drain
            base = S.cur[loc];
            S.cur[loc] = base + (uint32_t)__popc(grp);
        }
        base = __shfl_sync(0xffffffffu, base, leader);
        if (loc >= 0) {
            const int64_t pos = ps.Q + (int64_t)base + __popc(grp & lt);
            if (pos < p.pair_cap) p.hit_idx[pos] = (int32_t)ent.y;
        }
    }
    __syncwarp();  // entries read before the ring slots are reused
}

// One warp's 32 hits (lane i: hit hh, `valid`) against the item's columns in
// jm: certified bins, near test, and ring pushes with drains.
template <int SPHI, int NK, int RING>
__device__ __forceinline__ void assoc_cells(const AssocParams& p, const AssocWarp& S, const AssocPass& ps,
                                            const float* cp, const float* sp, float x, float y, int64_t hh,
                                            bool valid, unsigned jm, unsigned cmask, int WD, int nk, int nkw, int nkn,
                                            int lane, unsigned lt, unsigned& head, unsigned& tail) {
    constexpr int U = assoc_unroll(SPHI);
    const unsigned nku = (unsigned)nk;
    const float S2 = p.K.S2, H = p.K.H, T0 = p.K.T0;
    const HitFast hf = hit_fast(x, y, p.K);
    float q_[SPHI], qs[SPHI];
#pragma unroll
    for (int r = 0; r < SPHI; ++r) {
        q_[r] = q_of(x, y, cp[r], sp[r]);
        qs[r] = q_[r] * S2;
    }
    // U columns per step, SPHI rows each: independent cells for the
    // pipelines; steps past the last active column repeat column
    // jj[0] with its cells masked off
    while (jm) {
        int jj[U];
        bool jv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            jv[u] = jm != 0u;
            jj[u] = jv[u] ? __ffs(jm) - 1 : jj[0];
            jm &= jm - 1u;
        }
        unsigned kb[U][SPHI];  // the bin, or nk for none
        bool und_any = false;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const float4 dt = S.dt[jj[u]];
            const float Rj = hf.r2 + dt.z;
#pragma unroll
            for (int r = 0; r < SPHI; ++r) {
                const int c = r * WD + jj[u];
                const bool on = valid && jv[u] && (SPHI == 1 || ((cmask >> c) & 1u));
                const S1 o = stage1_fast(qs[r], q_[r], dt, Rj, hf.G, H, T0);
                kb[u][r] = ((o.flo == o.fhi) & on) ? min(o.kb, nku) : nku;
                und_any |= (o.flo != o.fhi) & on;
            }
        }
        if (__any_sync(0xffffffffu, und_any)) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const float4 dt = S.dt[jj[u]];
                const float Rj = hf.r2 + dt.z;
#pragma unroll
                for (int r = 0; r < SPHI; ++r) {
                    const int c = r * WD + jj[u];
                    const bool on = valid && jv[u] && (SPHI == 1 || ((cmask >> c) & 1u));
                    const S1 o = stage1_fast(qs[r], q_[r], dt, Rj, hf.G, H, T0);
                    if ((o.flo != o.fhi) && on && stage1_pending(o, hf.dmin, p.K.wlo, p.K.whi)) {
                        const int ks = cell_slow(x, y, cp[r], sp[r], dt.x, hf.R1, p.K, p.stats);
                        kb[u][r] = ks >= 0 ? (unsigned)ks : nku;
                    }
                }
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
#pragma unroll
            for (int r = 0; r < SPHI; ++r) {
                const int c = r * WD + jj[u];
                const unsigned b = kb[u][r];
                const bool cand = (S.nearb[c * nkn + (b >> 5)] >> (b & 31)) & 1u;
                const unsigned m = __ballot_sync(0xffffffffu, cand);
                if (cand)
                    S.ring[(tail + __popc(m & lt)) & (RING - 1)] =
                        make_uint2(((unsigned)c << 16) | b, (unsigned)hh);
                tail += __popc(m);
            }
        }
        while (tail - head >= 32) {
            assoc_drain<RING>(p, S, nkw, nk, head, 32, ps, lane);
            head += 32;
        }
    }
}

template <int SPHI, int NK, bool BAND>
__global__ void __launch_bounds__(256, 3) assoc_kernel(const AssocParams p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nk = NK ? NK : p.K.nk;
    const int nkw = (nk + 31) >> 5;
    const int nkn = (nk >> 5) + 1;  // near words per column, the last holding bin nk
    const int WD = p.wd;
    const int ncols = SPHI * WD;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int RING = assoc_ring(SPHI);
    AssocWarp S;
    {
        unsigned char* ptr = smem_raw + (size_t)warp * p.warp_bytes;
        S.dt = reinterpret_cast<float4*>(ptr);
        ptr += 16 * WD;
        S.ring = reinterpret_cast<uint2*>(ptr);
        ptr += 8 * RING;
        S.hq = reinterpret_cast<uint2*>(ptr);
        ptr += 8 * kHitQueue;
        S.cur = reinterpret_cast<uint32_t*>(ptr);
        ptr += 4 * p.cap;
        S.mask = reinterpret_cast<uint32_t*>(ptr);
        S.lpre = reinterpret_cast<int32_t*>(S.mask + ncols * nkw);
        S.nearb = reinterpret_cast<uint32_t*>(S.lpre + ncols * nkw);
    }
    const int tiles_phi = (p.K.nphi + SPHI - 1) / SPHI;
    const int tiles_d = (p.K.nd + WD - 1) / WD;
    const int64_t tiles = (int64_t)tiles_phi * tiles_d;
    const int64_t n_items = (int64_t)p.n_events * tiles;
    const unsigned lt = lanemask_lt();
    for (;;) {
        unsigned long long it = 0;
        if (lane == 0) it = atomicAdd(p.queue, 1ull);
        const int64_t item = (int64_t)__shfl_sync(0xffffffffu, it, 0);
        if (item >= n_items) break;
        const int el = (int)(item / tiles);
        const int64_t t = item - (int64_t)el * tiles;
        const int e = p.order ? p.order[el] : el;
        const int tp = (int)(t / tiles_d), td = (int)(t - (int64_t)tp * tiles_d);
        const int i0 = tp * SPHI, j0 = td * WD;
        const int nj = min(WD, p.K.nd - j0);
        const int nrows = min(SPHI, p.K.nphi - i0);
        const int nvalid = nrows * nj;  // columns c = r * WD + j, consecutive in the column numbering
        const int64_t colA = ((int64_t)e * p.K.nphi + i0) * p.K.nd + j0;
        const bool live = lane < nvalid;
        const int n = live ? p.npk[colA + lane] : 0;
        const int64_t cb = live ? p.colbase[colA + lane] : 0;
        const int64_t P0 = __shfl_sync(0xffffffffu, cb, 0);
        const int tot = (int)__reduce_add_sync(0xffffffffu, (unsigned)n);
        // peaks of the item that are stored (id < peak_cap)
        const int npk = (int)clamp64(p.peak_cap - P0, 0, tot);
        if (npk == 0) continue;
        const int lo_c = (int)(cb - P0), hi_c = lo_c + n;  // this lane's column: local ids [lo_c, hi_c)
        __syncwarp();  // the previous item's tables are no longer read
        for (int v = lane; v < ncols * nkw; v += 32) {
            const int c = v / nkw, w = v - (v / nkw) * nkw;
            const bool ok = c < nvalid;
            const int64_t col = colA + c;
            S.mask[v] = ok ? p.mask[col * nkw + w] : 0u;
            S.lpre[v] = ok ? (int)(p.colbase[col] - P0) + p.wpre[col * nkw + w] : 0;
        }
        if (lane < nj) S.dt[lane] = p.dtab[j0 + lane];
        __syncwarp();
        for (int v = lane; v < ncols * nkn; v += 32) {
            const int c = v / nkn, w = v - (v / nkn) * nkn;
            const uint32_t* m = S.mask + c * nkw;
            const uint32_t mw = w < nkw ? m[w] : 0u;
            const uint32_t hi_w = w + 1 < nkw ? m[w + 1] : 0u, lo_w = w > 0 && w - 1 < nkw ? m[w - 1] : 0u;
            uint32_t nb = mw;
            for (int o = 1; o <= p.window; ++o) nb |= (mw >> o) | (hi_w << (32 - o)) | (mw << o) | (lo_w >> (32 - o));
            if (w == (nk >> 5)) nb &= (1u << (nk & 31)) - 1u;  // no bins from nk on
            S.nearb[v] = nb;
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
        // a pass's rows span at most cap * (event hits) pairs: keep that below 2^32
        const int64_t eh = he - hb > 1 ? he - hb : 1;
        const int step = (int)clamp64(0xFFFFFFFFll / eh, 1, p.cap);
        const float dlo = S.dt[0].x, dhi = S.dt[nj - 1].x;
        for (int L0 = 0; L0 < npk; L0 += step) {
            AssocPass ps;
            ps.L0 = L0;
            ps.L1 = min(npk, L0 + step);
            ps.whole = L0 == 0 && ps.L1 == tot;
            ps.Q = p.peak_offsets[P0 + L0];
            __syncwarp();
            for (int l = lane; l < ps.L1 - L0; l += 32)
                S.cur[l] = (uint32_t)(p.peak_offsets[P0 + L0 + l] - ps.Q);
            // columns holding a peak of this pass, and the d0 columns among them
            const unsigned cmask = __ballot_sync(0xffffffffu, live && hi_c > ps.L0 && lo_c < ps.L1);
            unsigned jmask = 0;
#pragma unroll
            for (int r = 0; r < SPHI; ++r) jmask |= (unsigned)((unsigned long long)cmask >> (r * WD));
            jmask &= (unsigned)((1ull << nj) - 1ull);
            unsigned head = 0, tail = 0;
            __syncwarp();
            if (!BAND) {
                int64_t hh = hb + lane;
                float xn = hh < he ? p.x[hh] : 0.0f;
                float yn = hh < he ? p.y[hh] : 0.0f;
                for (int64_t h0 = hb; h0 < he; h0 += 32, hh += 32) {
                    const float x = xn, y = yn;
                    if (hh + 32 < he) {  // next chunk's coordinates
                        xn = p.x[hh + 32];
                        yn = p.y[hh + 32];
                    }
                    assoc_cells<SPHI, NK, RING>(p, S, ps, cp, sp, x, y, hh, hh < he, jmask, cmask, WD, nk, nkw, nkn,
                                                lane, lt, head, tail);
                }
            } else {
                // hits whose d0 band misses the pass's columns are dropped; the
                // rest queue in hit order and run 32 at a time over the union
                // of their bands
                unsigned qh = 0, qt = 0;
                for (int64_t h0 = hb; h0 < he; h0 += 32) {
                    const int64_t hh = h0 + lane;
                    const bool valid = hh < he;
                    const float x = valid ? p.x[hh] : 0.0f;
                    const float y = valid ? p.y[hh] : 0.0f;
                    const float r2 = fmaf(x, x, __fmul_rn(y, y));
                    int lo = nj, hi = -1;
#pragma unroll
                    for (int r = 0; r < SPHI; ++r) {
                        int jl, jh;
                        d0_band(r2, q_of(x, y, cp[r], sp[r]), dlo, dhi, j0, nj, p.K, jl, jh);
                        if (jh >= jl) {
                            lo = min(lo, jl - j0);
                            hi = max(hi, jh - j0);
                        }
                    }
                    const unsigned bits =
                        hi >= lo ? (0xFFFFFFFFu >> (31 - (hi - lo))) << lo & jmask : 0u;
                    const bool keep = valid && bits != 0u;
                    const unsigned m = __ballot_sync(0xffffffffu, keep);
                    if (keep) S.hq[(qt + __popc(m & lt)) & (kHitQueue - 1)] = make_uint2((unsigned)hh, bits);
                    qt += __popc(m);
                    if (qt - qh >= 32) {
                        const int n = 32;
                        __syncwarp();
                        const bool has = lane < n;
                        const uint2 ent = has ? S.hq[(qh + lane) & (kHitQueue - 1)] : make_uint2(0u, 0u);
                        const unsigned jm = __reduce_or_sync(0xffffffffu, ent.y);
                        __syncwarp();  // entries read before their slots are reused
                        qh += n;
                        const float qx = has ? p.x[ent.x] : 0.0f;
                        const float qy = has ? p.y[ent.x] : 0.0f;
                        assoc_cells<SPHI, NK, RING>(p, S, ps, cp, sp, qx, qy, (int64_t)ent.x, has, jm, cmask, WD, nk,
                                                    nkw, nkn, lane, lt, head, tail);
                    }
                }
                // at most 31 left once the last chunk was queued
                if (qt != qh) {
                    const int n = (int)(qt - qh);
                    __syncwarp();
                    const bool has = lane < n;
                    const uint2 ent = has ? S.hq[(qh + lane) & (kHitQueue - 1)] : make_uint2(0u, 0u);
                    const unsigned jm = __reduce_or_sync(0xffffffffu, ent.y);
                    __syncwarp();
                    qh += n;
                    const float qx = has ? p.x[ent.x] : 0.0f;
                    const float qy = has ? p.y[ent.x] : 0.0f;
                    assoc_cells<SPHI, NK, RING>(p, S, ps, cp, sp, qx, qy, (int64_t)ent.x, has, jm, cmask, WD, nk,
                                                nkw, nkn, lane, lt, head, tail);
                }
            }
            if (tail != head) assoc_drain<RING>(p, S, nkw, nk, head, (int)(tail - head), ps, lane);
        }
    }
}

// ---------------------------------------------------------------------------
// range association: one warp per item (one phi0 row x up to wd d0 columns),
// hits 32 at a time in increasing order
// ---------------------------------------------------------------------------
// For every column that holds a peak, each lane forms its hit's range from
// the cell's four corner codes (the d0 edge shared with the previous column
// is kept); when some lane's range reaches a bin within `window` of a peak,
// every peak of the column in reach takes the qualifying lanes at its row
// cursor by ballot rank.  Rows thus come out in hit order.  The counting
// instance only moves the cursors and leaves each peak's row length (the
// hits whose range reaches it, which the window sums of a range-voted
// accumulator over-count) in paircnt, or in extra_pairs past the peak cap;
// the writing instance then fills the rows the scan of those counts opened.
struct RangeWarp {
    float4* dte;     // [wd + 1] d0 edges of the item
    uint32_t* cur;   // [cap] row cursors (COUNT: counts) of the pass's peaks
    uint32_t* mask;  // [wd][nkw] peak bits
    int32_t* lpre;   // [wd][nkw] item-local id of the first peak of each word
    uint32_t* nearb; // [wd][nkw] bins within `window` of a peak
};

__host__ __device__ inline size_t assoc_range_warp_bytes(int wd, int nk, int cap) {
    const size_t nkw = (nk + 31) / 32;
    return (16 * (size_t)(wd + 1) + 4 * (size_t)cap + 12 * (size_t)wd * nkw + 15) & ~size_t(15);
}

// Corner codes of the item's two phi0 edges at d0 edge n.
__device__ __forceinline__ void range_edge_codes(const AssocParams& p, float x, float y, const HitFast& hf,
                                                 const float* qe, const float* qse, const float* ce, const float* se,
                                                 float4 dt, bool valid, int nk, int* code) {
    const float Rj = hf.r2 + dt.z;
    bool und = false;
#pragma unroll
    for (int m = 0; m < 2; ++m) {
        const S1 o = stage1_fast(qse[m], qe[m], dt, Rj, hf.G, p.K.H, p.K.T0);
        code[m] = valid ? code_stage1(o, hf.dmin, nk) : kCodeUndef;
        und |= code[m] == kCodeUndecided;
    }
    if (__any_sync(0xffffffffu, und)) {
#pragma unroll
        for (int m = 0; m < 2; ++m)
            if (code[m] == kCodeUndecided) code[m] = code_slow(x, y, ce[m], se[m], dt.x, hf.R1, p.K, p.stats);
    }
}

template <int NK, bool COUNT, bool LINE>
__global__ void __launch_bounds__(256, 3) assoc_range_kernel(const AssocParams p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nk = NK ? NK : p.K.nk;
    const int nkw = (nk + 31) >> 5;
    const int WD = p.wd;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    RangeWarp S;
    {
        unsigned char* ptr = smem_raw + (size_t)warp * p.warp_bytes;
        S.dte = reinterpret_cast<float4*>(ptr);
        ptr += 16 * (WD + 1);
        S.cur = reinterpret_cast<uint32_t*>(ptr);
        ptr += 4 * p.cap;
        S.mask = reinterpret_cast<uint32_t*>(ptr);
        S.lpre = reinterpret_cast<int32_t*>(S.mask + WD * nkw);
        S.nearb = reinterpret_cast<uint32_t*>(S.lpre + WD * nkw);
    }
    const int tiles_d = (p.K.nd + WD - 1) / WD;
    const int64_t tiles = (int64_t)p.K.nphi * tiles_d;
    const int64_t n_items = (int64_t)p.n_events * tiles;
    const unsigned lt = lanemask_lt();
    const float S2 = p.K.S2;
    const int w = p.window;
    for (;;) {
        unsigned long long it = 0;
        if (lane == 0) it = atomicAdd(p.queue, 1ull);
        const int64_t item = (int64_t)__shfl_sync(0xffffffffu, it, 0);
        if (item >= n_items) break;
        const int el = (int)(item / tiles);
        const int64_t t = item - (int64_t)el * tiles;
        const int e = p.order ? p.order[el] : el;
        const int i0 = (int)(t / tiles_d), td = (int)(t - (int64_t)i0 * tiles_d);
        const int j0 = td * WD;
        const int nj = min(WD, p.K.nd - j0);
        const int64_t colA = ((int64_t)e * p.K.nphi + i0) * p.K.nd + j0;
        const bool live = lane < nj;
        const int n = live ? p.npk[colA + lane] : 0;
        const int64_t cb = live ? p.colbase[colA + lane] : 0;
        const int64_t P0 = __shfl_sync(0xffffffffu, cb, 0);
        const int tot = (int)__reduce_add_sync(0xffffffffu, (unsigned)n);
        // counting takes every peak (those past the cap add to extra_pairs);
        // writing only the stored ones (id < peak_cap)
        const int npk = COUNT ? tot : (int)clamp64(p.peak_cap - P0, 0, tot);
        if (npk == 0) continue;
        const int lo_c = (int)(cb - P0), hi_c = lo_c + n;
        __syncwarp();  // the previous item's tables are no longer read
        for (int v = lane; v < WD * nkw; v += 32) {
            const int c = v / nkw, wd = v - (v / nkw) * nkw;
            const bool ok = c < nj;
            const int64_t col = colA + c;
            S.mask[v] = ok ? p.mask[col * nkw + wd] : 0u;
            S.lpre[v] = ok ? (int)(p.colbase[col] - P0) + p.wpre[col * nkw + wd] : 0;
        }
        if (!LINE)
            for (int v = lane; v <= nj; v += 32) S.dte[v] = p.edtab[j0 + v];
        __syncwarp();
        for (int v = lane; v < WD * nkw; v += 32) {
            const int wd = v - (v / nkw) * nkw;
            const uint32_t* m = S.mask + (v - wd);
            uint32_t nb = m[wd];
            const uint32_t hi_w = wd + 1 < nkw ? m[wd + 1] : 0u, lo_w = wd > 0 ? m[wd - 1] : 0u;
            for (int o = 1; o <= w; ++o) nb |= (m[wd] >> o) | (hi_w << (32 - o)) | (m[wd] << o) | (lo_w >> (32 - o));
            S.nearb[v] = nb;
        }
        const int i1 = (i0 + 1) % p.K.nphi;
        const float ce[2] = {LINE ? 0.0f : p.ecos[i0], LINE ? 0.0f : p.ecos[i1]};
        const float se[2] = {LINE ? 0.0f : p.esin[i0], LINE ? 0.0f : p.esin[i1]};
        // line voting: the row's centre tables and the d0 binning
        const double lc = LINE ? (double)p.cphi[i0] : 0.0, ls = LINE ? (double)p.sphi[i0] : 0.0;
        const double lscale = LINE ? __ddiv_rn((double)p.line_nd, __dsub_rn(p.line_d0max, p.line_d0min)) : 0.0;
        const int64_t hb = clamp64(p.offs[p.event0 + e], 0, p.n_hits);
        const int64_t he = clamp64(p.offs[p.event0 + e + 1], hb, p.n_hits);
        const int64_t eh = he - hb > 1 ? he - hb : 1;
        const int step = COUNT ? p.cap : (int)clamp64(0xFFFFFFFFll / eh, 1, p.cap);
        for (int L0 = 0; L0 < npk; L0 += step) {
            const int L1 = min(npk, L0 + step);
            const int64_t Q = COUNT ? 0 : p.peak_offsets[P0 + L0];
            __syncwarp();
            for (int l = lane; l < L1 - L0; l += 32)
                S.cur[l] = COUNT ? 0u : (uint32_t)(p.peak_offsets[P0 + L0 + l] - Q);
            const unsigned jmask = __ballot_sync(0xffffffffu, live && hi_c > L0 && lo_c < L1);
            __syncwarp();
            for (int64_t h0 = hb; h0 < he; h0 += 32) {
                const int64_t hh = h0 + lane;
                const bool valid = hh < he;
                const float x = valid ? p.x[hh] : 0.0f;
                const float y = valid ? p.y[hh] : 0.0f;
                const HitFast hf = hit_fast(x, y, p.K);
                float qe[2], qse[2];
#pragma unroll
                for (int m = 0; m < 2; ++m) {
                    qe[m] = q_of(x, y, ce[m], se[m]);
                    qse[m] = qe[m] * S2;
                }
                int jline = -1;
                if (LINE && valid) {
                    const double q = __dsub_rn(__dmul_rn((double)y, lc), __dmul_rn((double)x, ls));
                    const double u = __dmul_rn(__dsub_rn(q, p.line_d0min), lscale);
                    if (u >= 0.0 && u < (double)p.line_nd) jline = (int)u;
                }
                int left[2], right[2];
                int ln = -2;  // d0 edge whose codes are in `right`
                unsigned jm = jmask;
                while (jm) {
                    const int j = __ffs(jm) - 1;
                    jm &= jm - 1u;
                    int a, b;
                    bool def;
                    if (LINE) {  // the row's single column: the hit's d0 bin
                        a = b = jline;
                        def = jline >= 0;
                    } else {
                        if (j == ln) {
                            left[0] = right[0];
                            left[1] = right[1];
                        } else {
                            range_edge_codes(p, x, y, hf, qe, qse, ce, se, S.dte[j], valid, nk, left);
                        }
                        range_edge_codes(p, x, y, hf, qe, qse, ce, se, S.dte[j + 1], valid, nk, right);
                        ln = j + 1;
                        a = min(min(left[0], left[1]), min(right[0], right[1]));
                        b = max(max(left[0], left[1]), max(right[0], right[1]));
                        def = left[0] != kCodeUndef && left[1] != kCodeUndef && right[0] != kCodeUndef &&
                              right[1] != kCodeUndef && b >= 0 && a < nk;
                    }
                    const int lo = max(a, 0), hi = min(b, nk - 1);
                    // near-peak bins inside [lo, hi]
                    bool cand = false;
                    if (def) {
                        const uint32_t* nb = S.nearb + j * nkw;
                        for (int wd = lo >> 5; wd <= (hi >> 5); ++wd) {
                            uint32_t bits = nb[wd];
                            if (wd == (lo >> 5)) bits &= ~0u << (lo & 31);
                            if (wd == (hi >> 5)) bits &= ~0u >> (31 - (hi & 31));
                            cand |= bits != 0u;
                        }
                    }
                    if (!__any_sync(0xffffffffu, cand)) continue;
                    const int kmin = __reduce_min_sync(0xffffffffu, cand ? lo : 0x7fffffff);
                    const int kmax = __reduce_max_sync(0xffffffffu, cand ? hi : -1);
                    const int plo = max(kmin - w, 0), phi = min(kmax + w, nk - 1);
                    const uint32_t* mw = S.mask + j * nkw;
                    const int32_t* lp = S.lpre + j * nkw;
                    for (int wd = plo >> 5; wd <= (phi >> 5); ++wd) {
                        const uint32_t full = mw[wd];
                        uint32_t bits = full;
                        if (wd == (plo >> 5)) bits &= ~0u << (plo & 31);
                        if (wd == (phi >> 5)) bits &= ~0u >> (31 - (phi & 31));
                        while (bits) {
                            const int bt = __ffs(bits) - 1;
                            bits &= bits - 1u;
                            const int local = lp[wd] + __popc(full & ((1u << bt) - 1u));
                            if (local < L0 || local >= L1) continue;
                            const int kp = (wd << 5) + bt;
                            const bool sel = cand && lo <= kp + w && hi >= kp - w;
                            const unsigned bb = __ballot_sync(0xffffffffu, sel);
                            if (!bb) continue;
                            uint32_t v = 0;
                            if (lane == 0) v = S.cur[local - L0];  // only lane 0 moves cursors
                            const uint32_t base = __shfl_sync(0xffffffffu, v, 0);
                            if (!COUNT && sel) {
                                const int64_t pos = Q + (int64_t)base + __popc(bb & lt);
                                if (pos < p.pair_cap) p.hit_idx[pos] = (int32_t)hh;
                            }
                            if (lane == 0) S.cur[local - L0] = base + (uint32_t)__popc(bb);
                        }
                    }
                }
            }
            if (COUNT) {
                __syncwarp();
                for (int l = lane; l < L1 - L0; l += 32) {
                    const int64_t pid = P0 + L0 + l;
                    if (pid < p.peak_cap)
                        p.paircnt[pid] = (int32_t)S.cur[l];
                    else if (S.cur[l])
                        atomicAdd(reinterpret_cast<unsigned long long*>(p.extra_pairs), (unsigned long long)S.cur[l]);
                }
            }
        }
    }
}

// counts[0..1] = {peaks, pairs of stored peaks + pairs of peaks beyond the cap}
// Device-to-host copy of results into page-locked host memory by the SMs
// (each thread moves 16-byte words, four in flight).  Straight after the
// step's kernels the copy engines ran at a quarter of the host link's rate
// or less, where SM stores kept it.  Blocks of 64 threads with few registers
// fit beside the persistent vote and association blocks, so a wave's copy
// overlaps the next wave's kernels.  Source and destination sharing their
// offset mod 16 take the 16-byte path (a byte head and tail), mod 4 a
// 4-byte path, otherwise bytes.
__global__ void __launch_bounds__(64) host_copy_kernel(unsigned char* __restrict__ dst,
                                                       const unsigned char* __restrict__ src, size_t n) {
    const size_t tid = blockIdx.x * (size_t)blockDim.x + threadIdx.x, nth = (size_t)gridDim.x * blockDim.x;
    const uintptr_t mis = (uintptr_t)dst ^ (uintptr_t)src;
    const int unit = (mis & 15) == 0 ? 16 : ((mis & 3) == 0 ? 4 : 1);
    size_t head = (size_t)((unit - ((uintptr_t)dst & (unit - 1))) & (unit - 1));
    if (head > n) head = n;
    for (size_t i = tid; i < head; i += nth) dst[i] = src[i];
    const size_t nv = (n - head) / unit;
    if (unit == 16) {
        uint4* d = reinterpret_cast<uint4*>(dst + head);
        const uint4* v = reinterpret_cast<const uint4*>(src + head);
        size_t i = tid;
        for (; i + 3 * nth < nv; i += 4 * nth) {
            const uint4 a = v[i], b = v[i + nth], c = v[i + 2 * nth], e = v[i + 3 * nth];
            d[i] = a;
            d[i + nth] = b;
            d[i + 2 * nth] = c;
            d[i + 3 * nth] = e;
        }
        for (; i < nv; i += nth) d[i] = v[i];
    } else if (unit == 4) {
        uint32_t* d = reinterpret_cast<uint32_t*>(dst + head);
        const uint32_t* v = reinterpret_cast<const uint32_t*>(src + head);
        for (size_t i = tid; i < nv; i += nth) d[i] = v[i];
    } else {
        for (size_t i = tid; i < nv; i += nth) dst[head + i] = src[head + i];
    }
    for (size_t i = head + nv * unit + tid; i < n; i += nth) dst[i] = src[i];
}

// The running totals after a wave, stored straight into pinned host memory
// (device-accessible under unified addressing).  A 16-byte copy-engine copy
// on the compute stream would wait behind the copy stream's result copies,
// which share the device-to-host engine, and stall the next wave.
__global__ void publish_kernel(const int64_t* scal, int64_t* host) {
    host[0] = scal[0];
    host[1] = scal[1];
    __threadfence_system();
}

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
int vote_smem_bytes(int tile_phi, int tile_d, int nk, int threads, int variant) {
    const int warps = threads / 32;
    int queues = variant == 1 || variant == 3 ? warps * band_ring_bytes() : 0;
    if (variant == 6 || variant == 7) queues = warps * kHitQueue * 16 + kStageBytes;
    // item vote: a slot per lane and an item map of 32 * tile_d bytes per warp
    if (variant == 4 || variant == 5) queues = warps * 32 * flat_slot_bytes(tile_phi) + ((32 * tile_d * warps + 15) & ~15);
    const int table = variant == 2 ? 16 * (tile_d + 1) : 16 * tile_d;
    return table + queues + 4 * tile_phi * tile_d * nk;
}

// The dynamic shared-memory limit of a kernel is a property of the function,
// shared by every context and call in the process.  It is only ever raised,
// to what the device allows beside the kernel's static shared memory, and
// never set to one call's size: a context (or an allocation-free call) with a
// smaller tile must not lower the limit that another context's launches rely
// on.  `smem` is checked against that ceiling.
static cudaError_t allow_dynamic_smem(const void* f, int smem) {
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    cudaFuncAttributes fa{};
    e = cudaFuncGetAttributes(&fa, f);
    if (e != cudaSuccess) return e;
    const int room = optin - (int)fa.sharedSizeBytes;
    if (smem > room) return cudaErrorInvalidValue;
    if (fa.maxDynamicSharedSizeBytes >= room) return cudaSuccess;
    return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, room);
}

template <int S, int N>
static void* vote_fn() {
    return reinterpret_cast<void*>(vote_kernel<S, N>);
}
template <int S, int N>
static void* vote_band_fn(bool rec, bool stage) {
    if (stage)
        return rec ? reinterpret_cast<void*>(vote_band_kernel<S, N, true, true>)
                   : reinterpret_cast<void*>(vote_band_kernel<S, N, false, true>);
    return rec ? reinterpret_cast<void*>(vote_band_kernel<S, N, true, false>)
               : reinterpret_cast<void*>(vote_band_kernel<S, N, false, false>);
}

// records hold one byte per bin: only grids with n_kappa <= 255 write them
static void* vote_band_instance(int tile_phi, int nk, bool rec, bool stage = false) {
#define HT_VOTEB_NK(S)                                              \
    switch (nk) {                                                   \
        case 64: return vote_band_fn<S, 64>(rec, stage);            \
        case 128: return vote_band_fn<S, 128>(rec, stage);          \
        case 256: return vote_band_fn<S, 256>(false, stage);        \
        case 512: return vote_band_fn<S, 512>(false, stage);        \
        default: return vote_band_fn<S, 0>(rec && nk <= 255, stage); \
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

template <int S, int N>
static void* vote_range_fn() {
    return reinterpret_cast<void*>(vote_range_kernel<S, N>);
}

static void* vote_range_instance(int tile_phi, int nk) {
#define HT_VOTER_NK(S)                             \
    switch (nk) {                                  \
        case 64: return vote_range_fn<S, 64>();    \
        case 128: return vote_range_fn<S, 128>();  \
        case 256: return vote_range_fn<S, 256>();  \
        case 512: return vote_range_fn<S, 512>();  \
        default: return vote_range_fn<S, 0>();     \
    }
    switch (tile_phi) {
        case 1: HT_VOTER_NK(1)
        case 2: HT_VOTER_NK(2)
        case 4: HT_VOTER_NK(4)
        case 8: HT_VOTER_NK(8)
    }
#undef HT_VOTER_NK
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

template <int S, int N>
static void* vote_flat_fn(bool rec) {
    return rec ? reinterpret_cast<void*>(vote_flat_kernel<S, N, true>)
               : reinterpret_cast<void*>(vote_flat_kernel<S, N, false>);
}

static void* vote_flat_instance(int tile_phi, int nk, bool rec) {
#define HT_VOTEF_NK(S)                                     \
    switch (nk) {                                          \
        case 64: return vote_flat_fn<S, 64>(rec);          \
        case 128: return vote_flat_fn<S, 128>(rec);        \
        case 256: return vote_flat_fn<S, 256>(false);      \
        case 512: return vote_flat_fn<S, 512>(false);      \
        default: return vote_flat_fn<S, 0>(rec && nk <= 255); \
    }
    switch (tile_phi) {
        case 1: HT_VOTEF_NK(1)
        case 2: HT_VOTEF_NK(2)
        case 4: HT_VOTEF_NK(4)
        case 8: HT_VOTEF_NK(8)
    }
#undef HT_VOTEF_NK
    return nullptr;
}

// variants: 0 full sweep, 1 band (hull of queued hits), 2 range, 3 = 1 writing
// records, 4 band over (hit, column) items, 5 = 4 writing records
static void* vote_variant(int tile_phi, int nk, int variant) {
    switch (variant) {
        case 1: case 3: return vote_band_instance(tile_phi, nk, variant == 3);
        case 6: case 7: return vote_band_instance(tile_phi, nk, variant == 7, true);
        case 2: return vote_range_instance(tile_phi, nk);
        case 4: case 5: return vote_flat_instance(tile_phi, nk, variant == 5);
        default: return vote_instance(tile_phi, nk);
    }
}

cudaError_t vote_occupancy(int tile_phi, int nk, int threads, int smem, int* blocks, int variant) {
    void* f = vote_variant(tile_phi, nk, variant);
    if (!f) return cudaErrorInvalidValue;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, f, threads, smem);
}

cudaError_t launch_host_copy(void* dst, const void* src, size_t bytes, int blocks, cudaStream_t s) {
    if (bytes == 0) return cudaSuccess;
    host_copy_kernel<<<blocks, 64, 0, s>>>(static_cast<unsigned char*>(dst), static_cast<const unsigned char*>(src),
                                           bytes);
    return cudaGetLastError();
}

cudaError_t launch_publish(const int64_t* scal, int64_t* host, cudaStream_t s) {
    publish_kernel<<<1, 1, 0, s>>>(scal, host);
    return cudaGetLastError();
}

cudaError_t launch_finalize(int64_t* scal, cudaStream_t s) {
    finalize_kernel<<<1, 1, 0, s>>>(scal);
    return cudaGetLastError();
}

cudaError_t vote_prepare(int tile_phi, int nk, int smem, int variant) {
    void* f = vote_variant(tile_phi, nk, variant);
    if (!f) return cudaErrorInvalidValue;
    return allow_dynamic_smem(f, smem);
}

cudaError_t launch_vote(int tile_phi, const VoteParams& p, int grid, int threads, int smem, cudaStream_t s,
                        int variant) {
    if (grid <= 0) return cudaSuccess;
    void* f = vote_variant(tile_phi, p.K.nk, variant);
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

cudaError_t launch_detect(const PeakParams& p, cudaStream_t s) {
    const int64_t ncols = (int64_t)p.n_events * p.nphi * p.nd;
    if (ncols == 0) return cudaSuccess;
    if ((p.nk & 3) == 0 && ((uintptr_t)p.acc & 15) == 0) {
        constexpr int RB = 2;  // output phi rows per warp
        const int64_t items = (int64_t)p.n_events * ((p.nphi + RB - 1) / RB) * ((p.nk + 127) / 128);
        const int grid = (int)std::min<int64_t>((items + 3) / 4, 152 * 16);
        detect_vec_kernel<RB><<<grid, 128, 0, s>>>(p);
    } else {
        constexpr int RB = 4;  // output phi rows per warp
        const int64_t items = (int64_t)p.n_events * ((p.nphi + RB - 1) / RB) * p.nkw;  // one warp each
        const int grid = (int)std::min<int64_t>((items + 7) / 8, 152 * 8);
        detect_slide_kernel<RB><<<grid, 256, 0, s>>>(p);
    }
    detect_words_kernel<<<(int)std::min<int64_t>((ncols + 255) / 256, 152 * 8), 256, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_emit(const PeakParams& p, cudaStream_t s) {
    const int64_t ncols = (int64_t)p.n_events * p.nphi * p.nd;
    if (ncols == 0) return cudaSuccess;
    const int64_t blocks = (ncols + 255) / 256;
    emit_kernel<<<(int)std::min<int64_t>(blocks, 152 * 16), 256, 0, s>>>(p);
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

size_t assoc_warp_smem(int rows, int wd, int nk, int cap) { return assoc_warp_bytes(rows, wd, nk, cap); }

cudaError_t assoc_prepare(int tile_phi, int nk, int smem, bool band, int threads, int* blocks_per_sm) {
    void* f = assoc_instance(tile_phi, nk, band);
    if (!f) return cudaErrorInvalidValue;
    cudaError_t e = allow_dynamic_smem(f, smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, f, threads, smem);
}

cudaError_t launch_assoc(const AssocParams& p, int tile_phi, int threads, int grid, cudaStream_t s) {
    if ((int64_t)p.n_events * p.K.nphi == 0) return cudaSuccess;
    void* f = assoc_instance(tile_phi, p.K.nk, p.band != 0);
    if (!f) return cudaErrorInvalidValue;
    const int smem = (int)(p.warp_bytes * (threads / 32));
    void* args[] = {const_cast<AssocParams*>(&p)};
    return cudaLaunchKernel(f, dim3(grid), dim3(threads), args, smem, s);
}

template <int N, bool C>
static void* assoc_range_fn() {
    return reinterpret_cast<void*>(assoc_range_kernel<N, C, false>);
}

static void* assoc_range_instance(int nk, bool count, bool line = false) {
    if (line)
        return count ? reinterpret_cast<void*>(assoc_range_kernel<0, true, true>)
                     : reinterpret_cast<void*>(assoc_range_kernel<0, false, true>);
    switch (nk) {
        case 64: return count ? assoc_range_fn<64, true>() : assoc_range_fn<64, false>();
        case 128: return count ? assoc_range_fn<128, true>() : assoc_range_fn<128, false>();
        case 256: return count ? assoc_range_fn<256, true>() : assoc_range_fn<256, false>();
        case 512: return count ? assoc_range_fn<512, true>() : assoc_range_fn<512, false>();
        default: return count ? assoc_range_fn<0, true>() : assoc_range_fn<0, false>();
    }
}

size_t assoc_range_warp_smem(int wd, int nk, int cap) { return assoc_range_warp_bytes(wd, nk, cap); }

cudaError_t assoc_range_prepare(int nk, int smem, int threads, int* blocks_per_sm, bool line) {
    int b[2] = {0, 0};
    for (int c = 0; c < 2; ++c) {
        void* f = assoc_range_instance(nk, c != 0, line);
        cudaError_t e = allow_dynamic_smem(f, smem);
        if (e != cudaSuccess) return e;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b[c], f, threads, smem);
        if (e != cudaSuccess) return e;
    }
    *blocks_per_sm = std::min(b[0], b[1]);
    return cudaSuccess;
}

cudaError_t launch_assoc_range(const AssocParams& p, bool count, int threads, int grid, cudaStream_t s) {
    if ((int64_t)p.n_events * p.K.nphi == 0) return cudaSuccess;
    void* f = assoc_range_instance(p.K.nk, count, p.line_nd > 0);
    const int smem = (int)(p.warp_bytes * (threads / 32));
    void* args[] = {const_cast<AssocParams*>(&p)};
    return cudaLaunchKernel(f, dim3(grid), dim3(threads), args, smem, s);
}

cudaError_t launch_vote_line(const VoteParams& p, double d0min, double d0max, cudaStream_t s) {
    if (p.n_events <= 0) return cudaSuccess;
    const int grid = p.n_events < 152 * 8 ? p.n_events : 152 * 8;
    vote_line_kernel<<<grid, 256, 0, s>>>(p, d0min, d0max);
    return cudaGetLastError();
}

cudaError_t launch_rcp_check(uint32_t first_bits, uint32_t count, unsigned long long* out, cudaStream_t s) {
    rcp_check_kernel<<<152 * 4, 256, 0, s>>>(first_bits, count, out);
    return cudaGetLastError();
}

}  // namespace ht
