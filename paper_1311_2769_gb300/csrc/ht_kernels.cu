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
template <int SPHI>
__global__ void __launch_bounds__(512) vote_kernel(const VoteParams p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float4* dt_s = reinterpret_cast<float4*>(smem_raw);
    uint32_t* acc_s = reinterpret_cast<uint32_t*>(smem_raw + 16 * p.tile_d);
    __shared__ int s_item;

    const int nk = p.K.nk;
    const int nthr = blockDim.x;
    const int tid = threadIdx.x;
    const int tiles = p.tiles_phi * p.tiles_d;
    const int row_words = p.tile_d * nk;

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

        for (int w = tid; w < SPHI * row_words; w += nthr) acc_s[w] = 0u;
        for (int j = tid; j < nj; j += nthr) dt_s[j] = p.dtab[j0 + j];
        float cp[SPHI], sp[SPHI];
#pragma unroll
        for (int r = 0; r < SPHI; ++r) {
            cp[r] = r < nrows ? p.cphi[i0 + r] : 0.0f;
            sp[r] = r < nrows ? p.sphi[i0 + r] : 0.0f;
        }
        if (p.stats && tid == 0) atomicAdd(&p.stats[0], (unsigned long long)((he - hb) * nrows * nj));
        __syncthreads();

        for (int64_t h = hb + tid; h < he; h += nthr) {
            const float x = p.x[h];
            const float y = p.y[h];
            const HitFast hf = hit_fast(x, y, p.K);
            float q[SPHI];
#pragma unroll
            for (int r = 0; r < SPHI; ++r) q[r] = q_of(x, y, cp[r], sp[r]);
            for (int j = 0; j < nj; ++j) {
                const float4 dt = dt_s[j];
                const float Rj = hf.r2 + dt.z;
                uint32_t* col = acc_s + j * nk;
#pragma unroll
                for (int r = 0; r < SPHI; ++r) {
                    if (r < nrows) {
                        int k = cell_fast(q[r], dt.x, dt.y, Rj, hf.G, hf.dmin, p.K);
                        if (k == -2) k = cell_slow(x, y, cp[r], sp[r], dt.x, hf.R1, p.K, p.stats);
                        if (k >= 0) atomicAdd(col + r * row_words + k, 1u);
                    }
                }
            }
        }
        __syncthreads();

        uint32_t* dst_e = p.acc + (int64_t)e * p.cells;
        const int lane = tid & 31, warp = tid >> 5, nw = nthr >> 5;
        const int nrj = nrows * nj;
        for (int row = warp; row < nrj; row += nw) {
            const int r = row / nj;
            const int j = row - r * nj;
            const uint32_t* src = acc_s + r * row_words + j * nk;
            uint32_t* dst = dst_e + ((int64_t)(i0 + r) * p.K.nd + (j0 + j)) * nk;
            if ((nk & 3) == 0) {
                const uint4* s4 = reinterpret_cast<const uint4*>(src);
                uint4* d4 = reinterpret_cast<uint4*>(dst);
                for (int k = lane; k < (nk >> 2); k += 32) d4[k] = s4[k];
            } else {
                for (int k = lane; k < nk; k += 32) dst[k] = src[k];
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
__device__ __forceinline__ bool is_peak_cell(const uint32_t* A, const PeakParams& p, int i, int j, int k,
                                             uint32_t v) {
    const int64_t self = ((int64_t)i * p.nd + j) * p.nk + k;
    for (int di = -1; di <= 1; ++di) {
        int ii = i + di;
        ii = ii < 0 ? ii + p.nphi : (ii >= p.nphi ? ii - p.nphi : ii);
        for (int dj = -1; dj <= 1; ++dj) {
            const int jj = j + dj;
            if (jj < 0 || jj >= p.nd) continue;
            for (int dk = -1; dk <= 1; ++dk) {
                const int kk = k + dk;
                if (kk < 0 || kk >= p.nk) continue;
                const int64_t other = ((int64_t)ii * p.nd + jj) * p.nk + kk;
                if (other == self) continue;
                const uint32_t u = A[other];
                if (other < self ? !(v > u) : !(v >= u)) return false;
            }
        }
    }
    return true;
}

__global__ void detect_kernel(const PeakParams p) {
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwt = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t per_ev = (int64_t)p.nphi * p.nd;
    const int64_t ncols = per_ev * p.n_events;
    for (int64_t col = gw; col < ncols; col += nwt) {
        const int e = (int)(col / per_ev);
        const int ij = (int)(col - e * per_ev);
        const int i = ij / p.nd;
        const int j = ij - i * p.nd;
        const uint32_t* A = p.acc + (int64_t)e * p.cells;
        const uint32_t* colp = A + ((int64_t)i * p.nd + j) * p.nk;
        int count = 0;
        for (int k0 = 0, w = 0; k0 < p.nk; k0 += 32, ++w) {
            const int k = k0 + lane;
            bool pk = false;
            if (k < p.nk) {
                const uint32_t v = colp[k];
                if (v >= p.thr) pk = is_peak_cell(A, p, i, j, k, v);
            }
            const unsigned b = __ballot_sync(0xffffffffu, pk);
            if (lane == 0) {
                p.mask[col * p.nkw + w] = b;
                p.wpre[col * p.nkw + w] = (uint16_t)count;
            }
            count += __popc(b);
        }
        if (lane == 0) p.npk[col] = count;
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
__device__ void scan_bounds(const ScanRange& r, int64_t& lo, int64_t& hi) {
    lo = r.lo_dev ? *r.lo_dev : r.lo;
    hi = r.hi_dev ? *r.hi_dev : r.hi;
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
// association: CTA per (event, phi0 row), warps split the d0 columns that hold
// peaks, each warp sweeps the event's hits in ascending order (32 per step) so
// that every peak's hit list comes out ascending without a sort.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128) assoc_kernel(const AssocParams p) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int nkw = (p.K.nk + 31) >> 5;
    const int64_t nrows = (int64_t)p.n_events * p.K.nphi;
    for (int64_t row = blockIdx.x; row < nrows; row += gridDim.x) {
        const int e = (int)(row / p.K.nphi);
        const int i = (int)(row - (int64_t)e * p.K.nphi);
        const int64_t col0 = row * p.K.nd;
        // any peaks in this warp's columns?
        bool any = false;
        for (int j = warp; j < p.K.nd; j += nw)
            if (p.npk[col0 + j] > 0 && p.colbase[col0 + j] < p.peak_cap) any = true;
        if (!any) continue;
        const float c = p.cphi[i], s = p.sphi[i];
        const int64_t hb = clamp64(p.offs[p.event0 + e], 0, p.n_hits);
        const int64_t he = clamp64(p.offs[p.event0 + e + 1], hb, p.n_hits);
        for (int64_t h0 = hb; h0 < he; h0 += 32) {
            const int64_t h = h0 + lane;
            const bool valid = h < he;
            const float x = valid ? p.x[h] : 0.0f;
            const float y = valid ? p.y[h] : 0.0f;
            const HitFast hf = hit_fast(x, y, p.K);
            const float q = q_of(x, y, c, s);
            for (int j = warp; j < p.K.nd; j += nw) {
                const int64_t col = col0 + j;
                if (p.npk[col] == 0) continue;
                const int64_t pid0 = p.colbase[col];
                if (pid0 >= p.peak_cap) continue;
                const float4 dt = p.dtab[j];
                int kb = -1;
                if (valid) {
                    kb = cell_fast(q, dt.x, dt.y, hf.r2 + dt.z, hf.G, hf.dmin, p.K);
                    if (kb == -2) kb = cell_slow(x, y, c, s, dt.x, hf.R1, p.K, p.stats);
                }
                const uint32_t* mcol = p.mask + col * nkw;
                unsigned pend = 0;
                if (kb >= 0) {
                    for (int o = -p.window; o <= p.window; ++o) {
                        const int kk = kb + o;
                        if (kk >= 0 && kk < p.K.nk && ((mcol[kk >> 5] >> (kk & 31)) & 1u))
                            pend |= 1u << (o + p.window);
                    }
                }
                while (__any_sync(0xffffffffu, pend != 0)) {
                    const int my = pend ? kb - p.window + (__ffs(pend) - 1) : INT_MAX;
                    const int kmin = __reduce_min_sync(0xffffffffu, my);
                    const int rel = kmin - (kb - p.window);
                    const bool in = pend && rel >= 0 && rel <= 2 * p.window && ((pend >> rel) & 1u);
                    const unsigned b = __ballot_sync(0xffffffffu, in);
                    const int64_t pid = pid0 + p.wpre[col * nkw + (kmin >> 5)] +
                                        __popc(mcol[kmin >> 5] & ((1u << (kmin & 31)) - 1u));
                    if (pid < p.peak_cap) {
                        const int64_t base = p.peak_offsets[pid] + p.cursor[pid];
                        if (in) {
                            const int64_t pos = base + __popc(b & lanemask_lt());
                            if (pos < p.pair_cap) p.hit_idx[pos] = (int32_t)h;
                        }
                        __syncwarp();
                        if (lane == 0) p.cursor[pid] += __popc(b);
                        __syncwarp();
                    }
                    if (in) pend &= ~(1u << rel);
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
int vote_smem_bytes(int tile_phi, int tile_d, int nk) {
    return 16 * tile_d + 4 * tile_phi * tile_d * nk;
}

template <int S>
static cudaError_t prep_one(int smem) {
    return cudaFuncSetAttribute(vote_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

template <int S>
static cudaError_t occ_one(int threads, int smem, int* blocks) {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, vote_kernel<S>, threads, smem);
}

cudaError_t vote_occupancy(int tile_phi, int threads, int smem, int* blocks) {
    switch (tile_phi) {
        case 1: return occ_one<1>(threads, smem, blocks);
        case 2: return occ_one<2>(threads, smem, blocks);
        case 4: return occ_one<4>(threads, smem, blocks);
        case 8: return occ_one<8>(threads, smem, blocks);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_finalize(int64_t* scal, cudaStream_t s) {
    finalize_kernel<<<1, 1, 0, s>>>(scal);
    return cudaGetLastError();
}

cudaError_t vote_prepare(int tile_phi, int smem) {
    switch (tile_phi) {
        case 1: return prep_one<1>(smem);
        case 2: return prep_one<2>(smem);
        case 4: return prep_one<4>(smem);
        case 8: return prep_one<8>(smem);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_vote(int tile_phi, const VoteParams& p, int grid, int threads, int smem, cudaStream_t s) {
    if (grid <= 0) return cudaSuccess;
    switch (tile_phi) {
        case 1: vote_kernel<1><<<grid, threads, smem, s>>>(p); break;
        case 2: vote_kernel<2><<<grid, threads, smem, s>>>(p); break;
        case 4: vote_kernel<4><<<grid, threads, smem, s>>>(p); break;
        case 8: vote_kernel<8><<<grid, threads, smem, s>>>(p); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
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

cudaError_t launch_detect(const PeakParams& p, cudaStream_t s) {
    const int64_t ncols = (int64_t)p.n_events * p.nphi * p.nd;
    if (ncols == 0) return cudaSuccess;
    detect_kernel<<<warp_grid(ncols, 256), 256, 0, s>>>(p);
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

cudaError_t launch_assoc(const AssocParams& p, cudaStream_t s) {
    const int64_t nrows = (int64_t)p.n_events * p.K.nphi;
    if (nrows == 0) return cudaSuccess;
    int64_t grid = nrows < (1 << 20) ? nrows : (1 << 20);
    assoc_kernel<<<(int)grid, 128, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_rcp_check(uint32_t first_bits, uint32_t count, unsigned long long* out, cudaStream_t s) {
    rcp_check_kernel<<<152 * 4, 256, 0, s>>>(first_bits, count, out);
    return cudaGetLastError();
}

}  // namespace ht
