// ht_api.cu — host side of libht.so: contexts, validation, staging, waves,
// CUDA-graph replay of the batched step, autotuning, and the C ABI of ht.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "ht_internal.h"

using namespace ht;

namespace {

template <class T>
struct DBuf {
    T* p = nullptr;
    size_t n = 0;
    // Grow to at least `want` elements (contents are not preserved).  Bumps *gen
    // on reallocation so captured graphs that hold the old pointer are dropped.
    // slack = false: a quarter more, but at most 4 GiB more (record buffers
    // reach 100+ GB; growth by small steps would reallocate, and cudaFree /
    // cudaMalloc synchronise the device, on every new maximum)
    cudaError_t ensure(size_t want, int* gen, bool slack = true) {
        if (want <= n && p) return cudaSuccess;
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
        size_t alloc = slack ? want + want / 4 + 16 : want + std::min(want / 4, (size_t(4) << 30) / sizeof(T));
        cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&p), alloc * sizeof(T));
        if (e != cudaSuccess) {
            p = nullptr;
            cudaGetLastError();
            return e;
        }
        n = alloc;
        if (gen) ++*gen;
        return cudaSuccess;
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
    DBuf() = default;
    DBuf(const DBuf&) = delete;
    DBuf& operator=(const DBuf&) = delete;
    ~DBuf() { release(); }  // every buffer of a destroyed context is freed, listed below or not
};

struct GraphKey {
    const void* ptrs[8];
    int64_t vals[13];
    bool operator==(const GraphKey& o) const {
        return std::memcmp(ptrs, o.ptrs, sizeof(ptrs)) == 0 && std::memcmp(vals, o.vals, sizeof(vals)) == 0;
    }
};

constexpr int64_t kDefaultBudget = 40LL << 30;
constexpr int64_t kDefaultRecBudget = 72LL << 30;
constexpr size_t kRecWarpBudget = 9728;  // shared memory per warp of the record association

}  // namespace

struct ht_ctx {
    int device = 0;
    int sms = 152;
    ht_grid grid{};
    int n_layers = 0;
    KConsts K{};
    std::vector<float> h_cphi, h_sphi, h_d0;
    std::vector<float> h_ecos, h_esin, h_de;  // range voting: phi0 and d0 edges
    float* d_ecos = nullptr;
    float* d_esin = nullptr;
    float4* d_edtab = nullptr;
    float* d_cphi = nullptr;
    float* d_sphi = nullptr;
    float4* d_dtab = nullptr;
    int64_t cells = 0;
    int64_t cols_per_event = 0;
    int nkw = 0;
    // peak geometry: the accumulator as the peak and association stages see
    // it, [phi][d0][kappa], or [phi][1][d0] for line voting (same memory)
    int pnd = 0, pnk = 0;
    KConsts Kp{};

    // options
    int mode = HT_MODE_BATCHED;
    int tile_phi = 0, tile_d = 0, threads = 0;
    int atile_phi = 0, atile_d = 0;  // association item (0 = auto)
    int prune = 3;                   // bit 0: vote, bit 1: association drop hits without a d0 band
    int vote_mode = HT_VOTE_POINT;
    int acap = 0;  // association row cursors per warp (0 = auto)
    int host_chunks = 8;   // host results: minimum waves, each copied out while the next computes
    int assoc_index = 0;   // 1: point association through the per-layer angular index when hits carry layers
    bool use_index = false;           // the staged batch uses it (set before each step)
    const int8_t* clayer = nullptr;   // layer ids of the staged batch (device)
    const ht_peak* cur_peaks = nullptr;  // the step's peak array (device)
    DBuf<int32_t> ibcount, ibcursor, ihid, itab;
    DBuf<int64_t> ibstart;
    DBuf<uint32_t> ir2min, ir2max;
    DBuf<float> itheta;
    int64_t budget = kDefaultBudget;
    bool count_stages = false;
    bool use_graph = true;

    // resolved tile configuration
    int r_tile_phi = 1, r_tile_d = 1, r_threads = 256, r_smem = 0, r_blocks_per_sm = 1;
    bool r_band = false, a_band = false;
    int r_variant = 0;  // vote kernel: 0 full sweep, 1 band compaction, 2 range
    int a_tile_phi = 1, a_tile_d = 1, a_threads = 256, a_cap = 0, a_blocks_per_sm = 1;  // association item
    size_t a_warp_bytes = 0;
    // association over vote records (items are the vote's tiles)
    int records = 1;
    int64_t rec_budget = kDefaultRecBudget;
    bool r_rec = false;                    // the resolved vote tile supports records
    int r_rec_blocks_per_sm = 1;           // the record-writing vote's occupancy
    int r_rec_variant = 3;                 // the record-writing vote kernel
    int vote_items = 0;                    // band vote over (hit, column) items (1) or the hull of queued hits (0)
    int hit_staging = 0;                   // hull band vote: hits staged into shared memory by bulk copies
    int band_split = -1;                   // hull band vote: narrow-band queue threshold (-1 auto, 0 off)
    int host_copy = 32;                    // host results in page-locked memory: copy-kernel blocks (0: the copy engine)
    int r_narrow = 0;                      // resolved threshold passed to the kernel
    bool r_stage = false;                  // staged variants prepared for the resolved tile
    int r_stage_blocks_per_sm = 1, r_stage_rec_blocks_per_sm = 1, r_stage_smem = 0;
    int rc_threads = 128, rc_cap = 256, rc_blocks_per_sm = 1;
    size_t rc_warp_bytes = 0;
    bool use_rec = false;                  // the current ht_process associates through records
    std::vector<int32_t> wave_start;       // the current ht_process's waves: first events, then c_events
    std::vector<int32_t> h_offs;           // host copy of device event offsets (wave planning)
    std::vector<int32_t> gwaves;           // the wave plan the captured graph was made with
    DBuf<uint8_t> rec;
    DBuf<uint32_t> rbits;

    int gen = 0;  // buffer generation (graph invalidation)
    DBuf<float> sx, sy;
    DBuf<int8_t> slayer;
    DBuf<int32_t> soffs;
    DBuf<uint32_t> acc;
    DBuf<uint32_t> mask;
    DBuf<uint16_t> wpre;
    DBuf<int32_t> npk;
    DBuf<int64_t> colbase;
    DBuf<int32_t> order;
    DBuf<int32_t> paircnt;  // doubles as the association cursor after the pair scan
    DBuf<ht_peak> peaks;
    DBuf<int64_t> peakoff;
    DBuf<int32_t> hitidx;
    DBuf<int64_t> scratch;
    int64_t* d_scal = nullptr;  // [0] peak total [1] pair total [2] wave peak base [3] wave pair base [4] extra pairs
    int32_t* d_err = nullptr;   // validation bits
    int32_t* d_queue = nullptr; // persistent vote queue (int32) and association queue (u64 at byte 8)
    unsigned long long* d_aqueue = nullptr;
    unsigned long long* d_stats = nullptr;
    int64_t* h_pinned = nullptr;  // pinned mirror of a few scalars

    // current batch (device pointers)
    const float* cx = nullptr;
    const float* cy = nullptr;
    const int32_t* coffs = nullptr;
    int64_t c_hits = 0;
    int32_t c_events = 0;
    int32_t c_event0 = 0;  // first event of the accumulators held (ht_vote: 0)
    int32_t c_wave_events = 0;
    bool have_votes = false, have_peaks = false, have_results = false;
    DBuf<ht_track> fits;  // device staging of fits for host results
    DBuf<int32_t> mstate;               // device staging of merge states for host results
    DBuf<unsigned long long> mkept;     // merge: kept counter
    // second Hough transform: accumulators, per-row counts and bases, scalars, staging
    DBuf<uint32_t> vacc;
    DBuf<int32_t> vrow;
    DBuf<int64_t> vbase;
    DBuf<int64_t> vscal;
    DBuf<ht_vertex> vout;
    int64_t n_peaks_held = 0;
    uint32_t last_threshold = 0;

    cudaStream_t stream = nullptr;
    cudaStream_t own_stream = nullptr;  // used when the caller passes the legacy NULL stream
    // host results copied wave by wave: per-wave running totals {peaks, pairs}
    // (pinned, written by the step), an event after each wave, a copy stream
    bool wave_marks = false;
    std::vector<cudaEvent_t> wave_ev;
    int64_t* h_wave = nullptr;      // pinned, mapped: per-wave running totals written by publish_kernel
    int64_t* d_h_wave = nullptr;    // its device address
    int h_wave_n = 0;
    cudaStream_t copy_stream = nullptr;
    bool pending_check = false;
    const ht_results* pending_res = nullptr;
    ht_results pending_copy{};

    cudaGraphExec_t gexec = nullptr;
    GraphKey gkey{};
    bool gvalid = false;

    // optional per-phase device timing (external events, also inside graphs)
    bool timing = false;
    // five per wave: vote start, vote end, association end, step end, association start
    std::vector<cudaEvent_t> tev;
    int tev_waves = 0;  // waves timed by the last ht_process
    float phase_ms[4] = {0, 0, 0, 0};
    int64_t launches = 0;  // kernels issued by the last ht_process

    std::string last_error;
};

namespace {

int fail(ht_ctx* c, int code, const char* fmt, ...) {
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        c->last_error = buf;
    }
    return code;
}

#define CU(call)                                                                          \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) {                                                          \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? HT_ERR_OOM : HT_ERR_CUDA,  \
                        "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
        }                                                                                 \
    } while (0)

const double kPi = 3.14159265358979323846;

// Bin-centre tables (Section 3 parameter grid): phi0_i = (i + 1/2) 2 pi / n_phi,
// d0_j = d0_min + (j + 1/2)(d0_max - d0_min) / n_d0, rounded to float once.
// Range voting's cell edges: phi0 edges m 2pi/n_phi (cell i spans edges i and
// i + 1 mod n_phi) and the n_d0 + 1 d0 edges, each rounded to float once.
void build_edges(const ht_grid& g, std::vector<float>& c, std::vector<float>& s, std::vector<float>& d) {
    c.resize(g.n_phi);
    s.resize(g.n_phi);
    d.resize(g.n_d0 + 1);
    const double dphi = 2.0 * kPi / (double)g.n_phi;
    for (int m = 0; m < g.n_phi; ++m) {
        const double phi = (double)m * dphi;
        c[m] = (float)std::cos(phi);
        s[m] = (float)std::sin(phi);
    }
    const double wd = ((double)g.d0_max - (double)g.d0_min) / (double)g.n_d0;
    for (int n = 0; n <= g.n_d0; ++n) d[n] = (float)((double)g.d0_min + (double)n * wd);
}

void build_tables(const ht_grid& g, std::vector<float>& c, std::vector<float>& s, std::vector<float>& d) {
    c.resize(g.n_phi);
    s.resize(g.n_phi);
    d.resize(g.n_d0);
    const double dphi = 2.0 * kPi / (double)g.n_phi;
    for (int i = 0; i < g.n_phi; ++i) {
        const double phi = ((double)i + 0.5) * dphi;
        c[i] = (float)std::cos(phi);
        s[i] = (float)std::sin(phi);
    }
    const double wd = ((double)g.d0_max - (double)g.d0_min) / (double)g.n_d0;
    for (int j = 0; j < g.n_d0; ++j) d[j] = (float)((double)g.d0_min + ((double)j + 0.5) * wd);
}

// Constants of the three-stage bin evaluation (see ht_kbin.cuh for the bounds).
KConsts make_consts(const ht_grid& g, const std::vector<float>& d0) {
    KConsts K{};
    const double u = std::ldexp(1.0, -24), er = std::ldexp(1.0, -22);
    const int nk = g.n_kappa;
    K.nphi = g.n_phi;
    K.nd = g.n_d0;
    K.nk = nk;
    const double scale = (double)nk / ((double)g.kappa_max - (double)g.kappa_min);
    const double Hd = -(double)g.kappa_min * scale;
    K.kmin = (double)g.kappa_min;
    K.scale = scale;
    K.S2 = (float)(2.0 * scale);
    K.H = (float)Hd;
    double dabs = 0.0;
    for (float v : d0) dabs = std::max(dabs, (double)std::fabs(v));
    K.dabs = (float)dabs;
    const double V0 = std::max(std::fabs(Hd), std::fabs((double)nk - Hd));
    const double ev = er + 4.0 * u + 1.0 / 63.0;
    const double m = std::ceil(2.0 * (ev * ((double)nk + std::fabs(Hd)) + 0.3) / (1.0 - ev)) + 1.0;
    const double Vmax = V0 + m;
    K.wlo = (float)(-m);
    K.whi = (float)((double)nk + m);
    const double S2 = (double)K.S2;
    K.T0 = (float)(2.0 * ((er + 3.0 * u) * Vmax + u * (std::fabs(Hd) + 2.0 * ((double)nk + m)) + u));
    K.cG1 = (float)(2.0 * (64.0 / 63.0) * 4.03 * u * Vmax * (1.0 + er) * (1.0 + er + 4.0 * u));
    K.cG2 = (float)(2.0 * 1.01 * S2 * u * (1.0 + er));
    K.cD1 = (float)(64.0 * 4.03 * u);
    K.cD2 = (float)(3.6 * 1.01 * S2 * u * (1.0 + er));
    // stage 2
    const double two_scale = 2.0 * scale;
    K.S2hi = (float)two_scale;
    K.S2lo = (float)(two_scale - (double)K.S2hi);
    K.Hhi = (float)Hd;
    K.Hlo = (float)(Hd - (double)K.Hhi);
    const double V2 = V0 + 2.0;
    K.T0b = (float)(std::ldexp(1.0, -34) * (V2 + (double)nk + std::fabs(Hd)));
    K.cGb1 = (float)(64.0 * u * u * V2);
    K.cGb2 = (float)(20.0 * u * u * S2);
    K.cDb = (float)std::ldexp(1.0, -23);
    // d0 bands (pruned vote and association): kappa window widened by two
    // bins.  The band's u bounds carry relative errors of a few ulps (|u| <=
    // 1.5e4 + |d0| for hits within the validated 1e4 box), so a column must
    // be wide enough for the one-column margin to absorb them.
    {
        const double kmn = (double)g.kappa_min, kmx = (double)g.kappa_max, dk = (kmx - kmn) / nk;
        const double A = kmn - 2.0 * dk, B = kmx + 2.0 * dk;
        const double colw = ((double)g.d0_max - (double)g.d0_min) / g.n_d0;
        K.band_ok = (A < 0.0 && B > 0.0 && colw >= 1e-5 * (2e4 + (double)K.dabs)) ? 1 : 0;
        K.bA2 = (float)(A * A);
        K.bB2 = (float)(B * B);
        K.biA = (float)(1.0 / std::fabs(A));
        K.biB = (float)(1.0 / B);
        K.bdfirst = d0.empty() ? 0.0f : d0[0];
        K.bidd = (float)((double)g.n_d0 / ((double)g.d0_max - (double)g.d0_min));
    }
    return K;
}

bool grid_ok(const ht_grid& g) {
    if (g.n_phi < 1 || g.n_phi > 65535 || g.n_d0 < 1 || g.n_d0 > 65535) return false;
    if (g.n_kappa < 1 || g.n_kappa > 4096) return false;
    if ((int64_t)g.n_d0 * g.n_kappa > (1 << 24)) return false;
    if (!std::isfinite(g.d0_min) || !std::isfinite(g.d0_max) || !(g.d0_min < g.d0_max)) return false;
    if (!std::isfinite(g.kappa_min) || !std::isfinite(g.kappa_max) || !(g.kappa_min < g.kappa_max)) return false;
    if (std::fabs(g.d0_min) > 1.0e4f || std::fabs(g.d0_max) > 1.0e4f) return false;
    const double scale = (double)g.n_kappa / ((double)g.kappa_max - (double)g.kappa_min);
    if (!(scale < 1.0e30) || std::fabs(-(double)g.kappa_min * scale) > 1.0e6) return false;
    return true;
}

// Resolve the vote tile shape: explicit options win, otherwise ~64 KB of
// shared accumulator per CTA (three CTAs per SM).
int resolve_tiles(ht_ctx* ctx) {
    const int nk = ctx->grid.n_kappa, nd = ctx->grid.n_d0;
    int td = ctx->tile_d > 0 ? std::min(ctx->tile_d, nd) : std::min(nd, std::max(1, 65536 / (4 * nk)));
    int tp = ctx->tile_phi;
    if (tp <= 0) {
        tp = 1;
        for (int c : {8, 4, 2})
            if ((int64_t)c * td * nk * 4 <= 65536 && c <= ctx->grid.n_phi) {
                tp = c;
                break;
            }
    }
    int thr = ctx->threads > 0 ? ctx->threads : 256;
    const bool line = ctx->vote_mode == HT_VOTE_LINE;
    const bool range = ctx->vote_mode == HT_VOTE_RANGE || line;
    // bands bound point votes only: range and line voting sweep every cell
    // queued bands keep their ends in one byte each: tiles of at most 256 columns
    const bool band = !range && (ctx->prune & 1) && ctx->K.band_ok && td <= 256;
    ctx->a_band = !range && (ctx->prune & 2) && ctx->K.band_ok;
    const int variant = ctx->vote_mode == HT_VOTE_RANGE ? 2 : (band ? (ctx->vote_items ? 4 : 1) : 0);
    const int smem = vote_smem_bytes(tp, td, nk, thr, variant);
    if (smem > 227 * 1024)
        return fail(ctx, HT_ERR_INVALID_ARG, "vote tile %dx%dx%d needs %d B of shared memory", tp, td, nk, smem);
    CU(vote_prepare(tp, nk, smem, variant));
    int per_sm = 0;
    CU(vote_occupancy(tp, nk, thr, smem, &per_sm, variant));
    ctx->r_band = band;
    ctx->r_variant = variant;
    ctx->r_narrow = variant == 1 ? (ctx->band_split >= 0 ? ctx->band_split : std::max(3, td * 5 / 16)) : 0;
    if (per_sm < 1) return fail(ctx, HT_ERR_INVALID_ARG, "vote tile %dx%dx%d with %d threads cannot launch", tp, td, nk, thr);
    ctx->r_tile_phi = tp;
    ctx->r_tile_d = td;
    ctx->r_threads = thr;
    ctx->r_smem = smem;
    ctx->r_blocks_per_sm = per_sm;
    // staged hit loads (hull band vote): the same vote with 512-hit blocks
    // copied into shared memory; chosen per call when x and y are 16-byte aligned
    ctx->r_stage = false;
    if (ctx->hit_staging && variant == 1) {
        const int ssm = vote_smem_bytes(tp, td, nk, thr, 6);
        int b6 = 0, b7 = 0;
        if (ssm <= 227 * 1024 && vote_prepare(tp, nk, ssm, 6) == cudaSuccess &&
            vote_occupancy(tp, nk, thr, ssm, &b6, 6) == cudaSuccess && b6 >= 1) {
            ctx->r_stage = true;
            ctx->r_stage_smem = ssm;
            ctx->r_stage_blocks_per_sm = b6;
            if (nk <= 255 && vote_prepare(tp, nk, ssm, 7) == cudaSuccess &&
                vote_occupancy(tp, nk, thr, ssm, &b7, 7) == cudaSuccess)
                ctx->r_stage_rec_blocks_per_sm = std::max(b7, 1);
        }
        cudaGetLastError();
    }
    // records: the band vote writes each tile's bins, the association reads them
    ctx->r_rec = false;
    if (ctx->records && (variant == 1 || variant == 4) && ctx->vote_mode == HT_VOTE_POINT &&
        assoc_rec_supported(tp, td, nk)) {
        int rper = 0;
        const int rv = variant == 4 ? 5 : 3;
        CU(vote_prepare(tp, nk, smem, rv));
        CU(vote_occupancy(tp, nk, thr, smem, &rper, rv));
        // row cursors: about four peaks per cell before a tile needs a second
        // pass over its records (the batch workload averages under two)
        const size_t fixed = assoc_rec_warp_smem(tp, td, nk, 0);
        int cap = fixed + 8 * 64 <= kRecWarpBudget ? (int)((kRecWarpBudget - fixed) / 8) & ~31 : 64;
        cap = std::max(cap, std::min(4 * tp * td, 1024));
        cap = ctx->acap > 0 ? ctx->acap : std::min(std::max(cap, 64), 1024);
        const size_t wbytes = assoc_rec_warp_smem(tp, td, nk, cap);
        const int athr_r = 128;
        int ablocks = 0;
        if (rper >= 1 && wbytes * (athr_r / 32) <= 227 * 1024 &&
            assoc_rec_prepare(tp, td, nk, (int)(wbytes * (athr_r / 32)), athr_r, &ablocks) == cudaSuccess &&
            ablocks >= 1) {
            ctx->r_rec = true;
            ctx->r_rec_blocks_per_sm = rper;
            ctx->r_rec_variant = rv;
            ctx->rc_threads = athr_r;
            ctx->rc_cap = cap;
            ctx->rc_warp_bytes = wbytes;
            ctx->rc_blocks_per_sm = ablocks;
        }
        cudaGetLastError();
    }
    // association items: a_tile_phi rows x a_tile_d d0 columns, at most 32
    // columns, several rows only over all d0 columns (so an item's peaks are
    // consecutive).  Per warp: the d0 table, the item's peak tables and row
    // cursors, within 9 KB (three 8-warp blocks per SM) where possible.
    // Default: 32 d0 columns of one row, or as many whole rows as fit in 32
    // columns, fewer columns while the tables and 256 cursors exceed 9 KB;
    // then as many cursors as fit, 256 to 1024.
    const int nphi = ctx->grid.n_phi;
    constexpr size_t kWarpBudget = 9216;
    const int athr = std::min(thr, 256);
    if (range) {
        // range (and line) association: one row x up to 32 columns per item
        // of the peak geometry (line voting: one column of n_d0 bins)
        const int gnd = ctx->pnd, gnk = ctx->pnk;
        int atd = std::min(ctx->atile_d > 0 ? ctx->atile_d : 32, std::min(gnd, 32));
        while (atd > 1 && assoc_range_warp_smem(atd, gnk, 256) > kWarpBudget) atd = (atd + 1) / 2;
        const size_t fixed = assoc_range_warp_smem(atd, gnk, 0);
        int cap = fixed + 4 * 256 <= kWarpBudget ? (int)((kWarpBudget - fixed) / 4) & ~31 : 256;
        cap = ctx->acap > 0 ? ctx->acap : std::min(cap, 1024);
        const size_t wbytes = assoc_range_warp_smem(atd, gnk, cap);
        const int asmem = (int)(wbytes * (athr / 32));
        if (asmem > 227 * 1024) return fail(ctx, HT_ERR_INVALID_ARG, "association item does not fit shared memory");
        int ablocks = 0;
        CU(assoc_range_prepare(gnk, asmem, athr, &ablocks, line));
        if (ablocks < 1) return fail(ctx, HT_ERR_INVALID_ARG, "association kernel cannot launch");
        ctx->a_tile_phi = 1;
        ctx->a_tile_d = atd;
        ctx->a_threads = athr;
        ctx->a_cap = cap;
        ctx->a_warp_bytes = wbytes;
        ctx->a_blocks_per_sm = ablocks;
        return HT_OK;
    }
    auto fits = [&](int rows, int cols) { return assoc_warp_smem(rows, cols, nk, 256) <= kWarpBudget; };
    int atp = ctx->atile_phi, atd = ctx->atile_d;
    if (atp == 0 && atd == 0) {
        atp = 1;
        if (nd >= 32) {
            atd = 32;
        } else {
            atd = nd;
            for (int c : {8, 4, 2})
                if (c * nd <= 32 && c <= nphi && fits(c, nd)) {
                    atp = c;
                    break;
                }
        }
        if (atp == 1)
            while (atd > 1 && !fits(1, atd)) atd = (atd + 1) / 2;
    } else if (atp == 0) {
        atp = 1;
    } else if (atd == 0) {
        atd = atp > 1 ? nd : std::min(nd, 32);
    }
    atd = std::min(atd, nd);
    if (atp * atd > 32 || (atp > 1 && atd != nd))
        return fail(ctx, HT_ERR_INVALID_ARG,
                    "association item %d x %d: at most 32 columns, and more than one row needs all %d d0 columns",
                    atp, atd, nd);
    const bool aband = ctx->a_band;
    const size_t fixed = assoc_warp_smem(atp, atd, nk, 0);
    int cap = fixed + 4 * 256 <= kWarpBudget ? (int)((kWarpBudget - fixed) / 4) & ~31 : 256;
    cap = ctx->acap > 0 ? ctx->acap : std::min(cap, 1024);
    const size_t wbytes = assoc_warp_smem(atp, atd, nk, cap);
    const int asmem = (int)(wbytes * (athr / 32));
    if (asmem > 227 * 1024) return fail(ctx, HT_ERR_INVALID_ARG, "association item does not fit shared memory");
    int ablocks = 0;
    CU(assoc_prepare(atp, nk, asmem, aband, athr, &ablocks));
    if (ablocks < 1) return fail(ctx, HT_ERR_INVALID_ARG, "association kernel cannot launch");
    ctx->a_tile_phi = atp;
    ctx->a_tile_d = atd;
    ctx->a_threads = athr;
    ctx->a_cap = cap;
    ctx->a_warp_bytes = wbytes;
    ctx->a_blocks_per_sm = ablocks;
    return HT_OK;
}

int check_hits(ht_ctx* ctx, const ht_hits* h) {
    if (!h) return fail(ctx, HT_ERR_INVALID_ARG, "hits is NULL");
    if (h->mem != HT_HOST && h->mem != HT_DEVICE) return fail(ctx, HT_ERR_INVALID_ARG, "hits.mem must be HT_HOST or HT_DEVICE");
    if (h->n_events < 0) return fail(ctx, HT_ERR_INVALID_ARG, "n_events < 0");
    if (h->n_hits < 0 || h->n_hits > INT32_MAX) return fail(ctx, HT_ERR_INVALID_ARG, "n_hits out of range");
    if (!h->event_offsets) return fail(ctx, HT_ERR_INVALID_ARG, "event_offsets is NULL");
    if (h->n_hits > 0 && (!h->x || !h->y)) return fail(ctx, HT_ERR_INVALID_ARG, "x/y is NULL");
    if (h->n_hits > 0 && ctx->n_layers > 0 && !h->layer) return fail(ctx, HT_ERR_INVALID_ARG, "layer is NULL");
    if (h->mem == HT_HOST) {
        const int32_t* o = h->event_offsets;
        if (o[0] != 0 || (int64_t)o[h->n_events] != h->n_hits)
            return fail(ctx, HT_ERR_INVALID_ARG, "event_offsets must start at 0 and end at n_hits");
        for (int32_t e = 0; e < h->n_events; ++e)
            if (o[e] > o[e + 1]) return fail(ctx, HT_ERR_INVALID_ARG, "event_offsets decrease at event %d", e);
    }
    return HT_OK;
}

// Make the batch device-resident (host inputs are copied into context buffers)
// and queue its device-side validation.
int stage_hits(ht_ctx* ctx, const ht_hits* h, cudaStream_t s) {
    int st = check_hits(ctx, h);
    if (st) return st;
    const int64_t n = h->n_hits;
    const int32_t ne = h->n_events;
    if (h->mem == HT_HOST) {
        CU(ctx->sx.ensure(std::max<int64_t>(n, 1), &ctx->gen));
        CU(ctx->sy.ensure(std::max<int64_t>(n, 1), &ctx->gen));
        CU(ctx->soffs.ensure(ne + 1, &ctx->gen));
        if (n) {
            CU(cudaMemcpyAsync(ctx->sx.p, h->x, n * sizeof(float), cudaMemcpyHostToDevice, s));
            CU(cudaMemcpyAsync(ctx->sy.p, h->y, n * sizeof(float), cudaMemcpyHostToDevice, s));
        }
        CU(cudaMemcpyAsync(ctx->soffs.p, h->event_offsets, (ne + 1) * sizeof(int32_t), cudaMemcpyHostToDevice, s));
        const int8_t* lay = nullptr;
        if (h->layer && n) {
            CU(ctx->slayer.ensure(n, &ctx->gen));
            CU(cudaMemcpyAsync(ctx->slayer.p, h->layer, n, cudaMemcpyHostToDevice, s));
            lay = ctx->slayer.p;
        }
        ctx->cx = ctx->sx.p;
        ctx->cy = ctx->sy.p;
        ctx->coffs = ctx->soffs.p;
        ctx->clayer = lay;
        if (n) CU(launch_validate(ctx->cx, ctx->cy, lay, n, ctx->coffs, ne, ctx->n_layers, ctx->d_err, s));
    } else {
        ctx->cx = h->x;
        ctx->cy = h->y;
        ctx->coffs = h->event_offsets;
        ctx->clayer = h->layer;
        CU(launch_validate(h->x, h->y, h->layer, n, h->event_offsets, ne, ctx->n_layers, ctx->d_err, s));
    }
    ctx->c_hits = n;
    ctx->c_events = ne;
    return HT_OK;
}

// Decide whether the staged batch associates through the angular index
// (point voting, layer ids present, at most 32 layers) and size its buffers;
// called before any capture.
int ensure_index(ht_ctx* ctx) {
    ctx->use_index = ctx->assoc_index && ctx->vote_mode == HT_VOTE_POINT && ctx->clayer && ctx->n_layers >= 1 &&
                     ctx->n_layers <= 32 && ctx->c_hits > 0 && ctx->c_events > 0;
    if (!ctx->use_index) return HT_OK;
    const int64_t nb = (int64_t)ctx->c_events * ctx->n_layers;
    CU(ctx->ibcount.ensure(nb, &ctx->gen));
    CU(ctx->ibcursor.ensure(nb, &ctx->gen));
    CU(ctx->ibstart.ensure(nb + 1, &ctx->gen));
    CU(ctx->ir2min.ensure(nb, &ctx->gen));
    CU(ctx->ir2max.ensure(nb, &ctx->gen));
    CU(ctx->itheta.ensure(ctx->c_hits, &ctx->gen));
    CU(ctx->ihid.ensure(ctx->c_hits, &ctx->gen));
    CU(ctx->itab.ensure(nb * 257, &ctx->gen));
    return HT_OK;
}

int build_index(ht_ctx* ctx, cudaStream_t s) {
    IndexParams ip{};
    ip.x = ctx->cx;
    ip.y = ctx->cy;
    ip.layer = ctx->clayer;
    ip.offs = ctx->coffs;
    ip.n_events = ctx->c_events;
    ip.nl = ctx->n_layers;
    ip.bcount = ctx->ibcount.p;
    ip.bstart = ctx->ibstart.p;
    ip.bcursor = ctx->ibcursor.p;
    ip.r2min = ctx->ir2min.p;
    ip.r2max = ctx->ir2max.p;
    ip.theta = ctx->itheta.p;
    ip.hid = ctx->ihid.p;
    ip.tab = ctx->itab.p;
    ip.scratch = ctx->scratch.p;
    CU(launch_index_build(ip, s));
    return HT_OK;
}

int ensure_wave_buffers(ht_ctx* ctx, int32_t wave_events) {
    const int64_t ncols = (int64_t)wave_events * ctx->cols_per_event;
    CU(ctx->acc.ensure(std::max<int64_t>(1, (int64_t)wave_events * ctx->cells), &ctx->gen));
    CU(ctx->mask.ensure(std::max<int64_t>(1, ncols * ctx->nkw), &ctx->gen));
    CU(ctx->wpre.ensure(std::max<int64_t>(1, ncols * ctx->nkw), &ctx->gen));
    CU(ctx->npk.ensure(std::max<int64_t>(1, ncols), &ctx->gen));
    CU(ctx->colbase.ensure(std::max<int64_t>(1, ncols + 1), &ctx->gen));
    CU(ctx->order.ensure(std::max<int32_t>(1, wave_events), &ctx->gen));
    CU(ctx->scratch.ensure(2 * kScanBlocks, &ctx->gen));
    return HT_OK;
}

VoteParams vote_params(ht_ctx* ctx, int32_t event0, int32_t ne, bool persistent) {
    VoteParams p{};
    p.x = ctx->cx;
    p.y = ctx->cy;
    p.offs = ctx->coffs;
    p.n_hits = ctx->c_hits;
    p.event0 = event0;
    p.n_events = ne;
    p.order = persistent ? ctx->order.p : nullptr;
    p.queue = persistent ? ctx->d_queue : nullptr;
    p.item0 = 0;
    p.tiles_phi = (ctx->grid.n_phi + ctx->r_tile_phi - 1) / ctx->r_tile_phi;
    p.tiles_d = (ctx->grid.n_d0 + ctx->r_tile_d - 1) / ctx->r_tile_d;
    p.tile_d = ctx->r_tile_d;
    p.n_items = ne * p.tiles_phi * p.tiles_d;
    p.acc = ctx->acc.p;
    p.cells = ctx->cells;
    p.cphi = ctx->d_cphi;
    p.sphi = ctx->d_sphi;
    p.dtab = ctx->d_dtab;
    p.ecos = ctx->d_ecos;
    p.esin = ctx->d_esin;
    p.edtab = ctx->d_edtab;
    p.K = ctx->K;
    p.stats = ctx->count_stages ? ctx->d_stats : nullptr;
    p.err = ctx->d_err;
    p.narrow = ctx->r_narrow;
    return p;
}

// Vote records per hit of the batch: one record per vote tile of its event.
int64_t rec_per_hit(const ht_ctx* ctx) {
    const int64_t tiles = (int64_t)((ctx->grid.n_phi + ctx->r_tile_phi - 1) / ctx->r_tile_phi) *
                          ((ctx->grid.n_d0 + ctx->r_tile_d - 1) / ctx->r_tile_d);
    return tiles * ctx->r_tile_phi * ctx->r_tile_d;
}

// Vote events [event0, event0 + ne) of the staged batch into acc[0..ne)
// (and, with ctx->use_rec, their records).
int run_vote(ht_ctx* ctx, int32_t event0, int32_t ne, bool persistent, cudaStream_t s) {
    if (ne <= 0) return HT_OK;
    VoteParams p = vote_params(ctx, event0, ne, persistent);
    int variant = ctx->r_variant, per_sm = ctx->r_blocks_per_sm, smem = ctx->r_smem;
    if (ctx->use_rec && ctx->vote_mode == HT_VOTE_POINT) {
        p.rec = ctx->rec.p;
        p.rbits = ctx->rbits.p;
        p.rec_bytes = ctx->r_tile_phi * ctx->r_tile_d;
        variant = ctx->r_rec_variant;
        per_sm = ctx->r_rec_blocks_per_sm;
    }
    // staged hit blocks: bulk copies need 16-byte-aligned x and y
    if (ctx->r_stage && (variant == 1 || variant == 3) && ((uintptr_t)ctx->cx & 15) == 0 &&
        ((uintptr_t)ctx->cy & 15) == 0) {
        variant = variant == 1 ? 6 : 7;
        per_sm = variant == 6 ? ctx->r_stage_blocks_per_sm : ctx->r_stage_rec_blocks_per_sm;
        smem = ctx->r_stage_smem;
    }
    if (ctx->vote_mode == HT_VOTE_LINE) {
        if (persistent) CU(launch_order(ctx->coffs, event0, ne, ctx->c_hits, ctx->order.p, s));
        CU(cudaMemsetAsync(ctx->acc.p, 0, (size_t)ne * ctx->cells * sizeof(uint32_t), s));
        CU(launch_vote_line(p, (double)ctx->grid.d0_min, (double)ctx->grid.d0_max, s));
        return HT_OK;
    }
    if (persistent) {
        CU(launch_order(ctx->coffs, event0, ne, ctx->c_hits, ctx->order.p, s));
        CU(cudaMemsetAsync(ctx->d_queue, 0, sizeof(int32_t), s));
        const int grid = std::min<int64_t>(p.n_items, (int64_t)ctx->sms * per_sm);
        CU(launch_vote(ctx->r_tile_phi, p, grid, ctx->r_threads, smem, s, variant));
    } else {
        CU(launch_vote(ctx->r_tile_phi, p, p.n_items, ctx->r_threads, smem, s, variant));
    }
    return HT_OK;
}

PeakParams peak_params(ht_ctx* ctx, int32_t event0, int32_t ne, uint32_t thr, ht_peak* peaks, int64_t cap,
                       int32_t window) {
    PeakParams p{};
    p.acc = ctx->acc.p;
    p.cells = ctx->cells;
    p.n_events = ne;
    p.event0 = event0;
    p.thr = thr;
    p.nphi = ctx->grid.n_phi;
    p.nd = ctx->pnd;
    p.nk = ctx->pnk;
    p.nkw = ctx->nkw;
    p.line = ctx->vote_mode == HT_VOTE_LINE ? 1 : 0;
    p.mask = ctx->mask.p;
    p.wpre = ctx->wpre.p;
    p.npk = ctx->npk.p;
    p.colbase = ctx->colbase.p;
    p.peaks = peaks;
    p.peak_cap = cap;
    p.window = window;
    p.paircnt = ctx->paircnt.p;
    p.extra_pairs = ctx->d_scal + 4;
    return p;
}

// detect + scan of per-column peak counts; colbase starts at d_scal[0] (running
// peak total), which is advanced to include this wave's peaks.
int run_detect_scan(ht_ctx* ctx, const PeakParams& pp, cudaStream_t s) {
    CU(launch_detect(pp, s));
    CU(cudaMemcpyAsync(ctx->d_scal + 2, ctx->d_scal + 0, sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
    ScanRange r{};
    r.in = ctx->npk.p;
    r.out = ctx->colbase.p;
    r.lo = 0;
    r.hi = (int64_t)pp.n_events * ctx->cols_per_event;
    r.cap = r.hi;
    r.base_dev = ctx->d_scal + 2;
    r.total = ctx->d_scal + 0;
    r.write_end = 0;
    CU(launch_scan(r, ctx->scratch.p, s));
    return HT_OK;
}

// Association of events [event0, event0 + ne) (their peaks numbered from the
// column bases): the item-layout fields, a zeroed work counter, a grid of
// resident blocks.
// pass: 0 point association, 1 range counting, 2 range writing
int launch_assoc_ctx(ht_ctx* ctx, AssocParams& a, int32_t event0, int32_t ne, const int32_t* order, int pass,
                     cudaStream_t s) {
    a.x = ctx->cx;
    a.y = ctx->cy;
    a.offs = ctx->coffs;
    a.n_hits = ctx->c_hits;
    a.event0 = event0;
    a.n_events = ne;
    a.mask = ctx->mask.p;
    a.wpre = ctx->wpre.p;
    a.npk = ctx->npk.p;
    a.colbase = ctx->colbase.p;
    a.band = ctx->a_band ? 1 : 0;
    a.wd = ctx->a_tile_d;
    a.cap = ctx->a_cap;
    a.warp_bytes = ctx->a_warp_bytes;
    a.order = order;
    a.queue = ctx->d_aqueue;
    a.cphi = ctx->d_cphi;
    a.sphi = ctx->d_sphi;
    a.dtab = ctx->d_dtab;
    a.ecos = ctx->d_ecos;
    a.esin = ctx->d_esin;
    a.edtab = ctx->d_edtab;
    a.K = ctx->Kp;
    a.stats = ctx->count_stages ? ctx->d_stats : nullptr;
    if (ctx->vote_mode == HT_VOTE_LINE) {
        a.line_nd = ctx->grid.n_d0;
        a.line_d0min = (double)ctx->grid.d0_min;
        a.line_d0max = (double)ctx->grid.d0_max;
    }
    if (pass == 0 && ctx->use_rec) {
        a.rec = ctx->rec.p;
        a.rbits = ctx->rbits.p;
        a.rec_bytes = ctx->r_tile_phi * ctx->r_tile_d;
        a.rtiles_phi = (ctx->grid.n_phi + ctx->r_tile_phi - 1) / ctx->r_tile_phi;
        a.rtiles_d = (ctx->grid.n_d0 + ctx->r_tile_d - 1) / ctx->r_tile_d;
        a.rtile_d = ctx->r_tile_d;
        a.cap = ctx->rc_cap;
        a.warp_bytes = ctx->rc_warp_bytes;
        const int64_t items = (int64_t)ne * a.rtiles_phi * a.rtiles_d;
        const int warps = ctx->rc_threads / 32;
        const int grid = (int)std::max<int64_t>(
            1, std::min<int64_t>((items + warps - 1) / warps, (int64_t)ctx->sms * ctx->rc_blocks_per_sm));
        CU(cudaMemsetAsync(ctx->d_aqueue, 0, sizeof(unsigned long long), s));
        CU(launch_assoc_rec(a, ctx->r_tile_phi, ctx->rc_threads, grid, s));
        return HT_OK;
    }
    const int64_t items = (int64_t)ne * ((ctx->grid.n_phi + ctx->a_tile_phi - 1) / ctx->a_tile_phi) *
                          ((ctx->pnd + ctx->a_tile_d - 1) / ctx->a_tile_d);
    const int warps = ctx->a_threads / 32;
    const int grid = (int)std::max<int64_t>(
        1, std::min<int64_t>((items + warps - 1) / warps, (int64_t)ctx->sms * ctx->a_blocks_per_sm));
    CU(cudaMemsetAsync(ctx->d_aqueue, 0, sizeof(unsigned long long), s));
    if (pass == 0)
        CU(launch_assoc(a, ctx->a_tile_phi, ctx->a_threads, grid, s));
    else
        CU(launch_assoc_range(a, pass == 1, ctx->a_threads, grid, s));
    return HT_OK;
}

// pair offsets for this wave's peaks [d_scal[2], d_scal[0]) clamped to cap, and association
int mark(ht_ctx* ctx, int wi, int which, cudaStream_t s);

int run_pairs_assoc(ht_ctx* ctx, int32_t event0, int32_t ne, const int32_t* order, int64_t peak_cap,
                    int64_t* peak_offsets, int32_t* hit_idx, int64_t pair_cap, int32_t window, int wave_timed,
                    cudaStream_t s) {
    const bool range = ctx->vote_mode != HT_VOTE_POINT;
    if (range) {
        // row lengths by a counting pass (window sums over-count range votes;
        // line votes run along d0, across the window sums' kappa axis)
        AssocParams c{};
        c.peak_offsets = peak_offsets;
        c.peak_cap = peak_cap;
        c.window = window;
        c.paircnt = ctx->paircnt.p;
        c.extra_pairs = ctx->d_scal + 4;
        const int st = launch_assoc_ctx(ctx, c, event0, ne, order, 1, s);
        if (st) return st;
    }
    CU(cudaMemcpyAsync(ctx->d_scal + 3, ctx->d_scal + 1, sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
    ScanRange r{};
    r.in = ctx->paircnt.p;
    r.out = peak_offsets;
    r.lo_dev = ctx->d_scal + 2;
    r.hi_dev = ctx->d_scal + 0;
    r.cap = peak_cap;
    r.base_dev = ctx->d_scal + 3;
    r.total = ctx->d_scal + 1;
    r.write_end = 1;
    CU(launch_scan(r, ctx->scratch.p, s));
    AssocParams a{};
    a.peak_offsets = peak_offsets;
    a.peak_cap = peak_cap;
    a.hit_idx = hit_idx;
    a.pair_cap = pair_cap;
    a.window = window;
    if (wave_timed >= 0) {
        const int st = mark(ctx, wave_timed, 4, s);
        if (st) return st;
    }
    if (!range && ctx->use_index && !ctx->use_rec) {
        AssocIndexParams q{};
        q.a = a;
        q.a.x = ctx->cx;
        q.a.y = ctx->cy;
        q.a.offs = ctx->coffs;
        q.a.n_hits = ctx->c_hits;
        q.a.cphi = ctx->d_cphi;
        q.a.sphi = ctx->d_sphi;
        q.a.dtab = ctx->d_dtab;
        q.a.K = ctx->K;
        q.a.stats = ctx->count_stages ? ctx->d_stats : nullptr;
        q.peaks = ctx->cur_peaks;
        q.lo_dev = ctx->d_scal + 2;
        q.hi_dev = ctx->d_scal + 0;
        q.theta = ctx->itheta.p;
        q.hid = ctx->ihid.p;
        q.tab = ctx->itab.p;
        q.bstart = ctx->ibstart.p;
        q.r2min = ctx->ir2min.p;
        q.r2max = ctx->ir2max.p;
        q.nl = ctx->n_layers;
        q.kmin = ctx->grid.kappa_min;
        q.dk = (float)(((double)ctx->grid.kappa_max - (double)ctx->grid.kappa_min) / (double)ctx->grid.n_kappa);
        q.err = ctx->d_err;
        CU(launch_assoc_index(q, s));
        return HT_OK;
    }
    return launch_assoc_ctx(ctx, a, event0, ne, order, range ? 2 : 0, s);
}

// The legacy default stream cannot be captured into a graph; a caller's NULL
// stream is replaced by a context-owned blocking stream, which the legacy
// stream synchronises with implicitly (both directions).
int resolve_stream(ht_ctx* ctx, void* stream, cudaStream_t* out) {
    if (stream) {
        *out = (cudaStream_t)stream;
        return HT_OK;
    }
    if (!ctx->own_stream) CU(cudaStreamCreateWithFlags(&ctx->own_stream, cudaStreamDefault));
    *out = ctx->own_stream;
    return HT_OK;
}

int32_t events_per_wave(ht_ctx* ctx, int32_t n_events) {
    const int64_t per = ctx->cells * 4;
    int64_t w = ctx->budget / std::max<int64_t>(per, 1);
    if (w < 1) return 0;
    return (int32_t)std::min<int64_t>(w, std::max<int32_t>(n_events, 1));
}

// Device work of ht_process for the staged batch (graph-capturable).
// Records one of wave wi's phase events (external, so it also works inside a graph).
int mark(ht_ctx* ctx, int wi, int which, cudaStream_t s) {
    if (!ctx->timing || (size_t)(5 * wi + which) >= ctx->tev.size()) return HT_OK;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    CU(cudaStreamIsCapturing(s, &cs));
    if (cs == cudaStreamCaptureStatusActive)
        CU(cudaEventRecordWithFlags(ctx->tev[5 * wi + which], s, cudaEventRecordExternal));
    else
        CU(cudaEventRecord(ctx->tev[5 * wi + which], s));
    return HT_OK;
}

// Phase events for n waves (created before any capture).
int ensure_timing_events(ht_ctx* ctx, int n) {
    while ((int)ctx->tev.size() < 5 * std::max(n, 1)) {
        cudaEvent_t e = nullptr;
        CU(cudaEventCreate(&e));
        ctx->tev.push_back(e);
    }
    return HT_OK;
}

// The waves of the staged batch: at most `step` events each and, when the
// association reads vote records, at most rec_budget bytes of records each.
// The events' sizes are needed only when the whole batch's records exceed the
// budget; device offsets are then read back once (synchronously).  An event
// whose records alone exceed the budget turns records off for the call.  The
// record buffers are sized for the largest wave.
int plan_waves(ht_ctx* ctx, const ht_hits* hits, int32_t step, cudaStream_t s) {
    std::vector<int32_t>& w = ctx->wave_start;
    w.clear();
    const int32_t ne = ctx->c_events;
    step = std::max<int32_t>(step, 1);
    ctx->use_rec = ctx->r_rec && ctx->vote_mode == HT_VOTE_POINT && ctx->c_hits > 0 && ne > 0;
    const int64_t rph = ctx->use_rec ? rec_per_hit(ctx) : 0;
    const int64_t hits_fit = rph > 0 ? ctx->rec_budget / rph : 0;  // hits whose records fit the budget
    int64_t max_hits = ctx->c_hits;
    int32_t max_ne = std::min(step, ne);
    const bool by_size = ctx->use_rec && ctx->c_hits > hits_fit;
    if (by_size) {
        const int32_t* o = nullptr;
        if (hits && hits->mem == HT_HOST) {
            o = hits->event_offsets;
        } else {
            ctx->h_offs.resize((size_t)ne + 1);
            CU(cudaMemcpyAsync(ctx->h_offs.data(), ctx->coffs, ((size_t)ne + 1) * sizeof(int32_t),
                               cudaMemcpyDeviceToHost, s));
            CU(cudaStreamSynchronize(s));
            o = ctx->h_offs.data();
            if (o[0] != 0 || (int64_t)o[ne] != ctx->c_hits)
                return fail(ctx, HT_ERR_INVALID_ARG, "event_offsets must start at 0 and end at n_hits");
            for (int32_t e = 0; e < ne; ++e)
                if (o[e] > o[e + 1]) return fail(ctx, HT_ERR_INVALID_ARG, "event_offsets decrease at event %d", e);
        }
        max_hits = 0;
        max_ne = 0;
        for (int32_t e = 0; e < ne;) {
            const int32_t e0 = e;
            int64_t h = 0;
            while (e < ne && e - e0 < step) {
                const int64_t he = (int64_t)o[e + 1] - o[e];
                if (e > e0 && h + he > hits_fit) break;
                h += he;
                ++e;
            }
            if (h > hits_fit) {  // one event alone exceeds the budget
                ctx->use_rec = false;
                break;
            }
            w.push_back(e0);
            max_hits = std::max(max_hits, h);
            max_ne = std::max(max_ne, e - e0);
        }
    }
    if (!by_size || !ctx->use_rec) {
        w.clear();
        for (int32_t e = 0; e < ne; e += step) w.push_back(e);
        max_hits = ctx->c_hits;
        max_ne = std::min(step, ne);
    }
    w.push_back(ne);
    if (ctx->use_rec) {
        const int64_t tiles = rph / ((int64_t)ctx->r_tile_phi * ctx->r_tile_d);
        CU(ctx->rec.ensure((size_t)std::max<int64_t>(1, max_hits * rph), &ctx->gen, false));
        CU(ctx->rbits.ensure((size_t)std::max<int64_t>(1, ((max_hits >> 5) + max_ne + 1) * tiles), &ctx->gen));
    }
    return HT_OK;
}

int process_device(ht_ctx* ctx, uint32_t thr, int32_t window, ht_peak* peaks, int64_t peak_cap,
                   int64_t* peak_offsets, int32_t* hit_idx, int64_t pair_cap, cudaStream_t s) {
    CU(cudaMemsetAsync(ctx->d_scal, 0, 8 * sizeof(int64_t), s));
    const bool plain = ctx->mode == HT_MODE_PLAIN;
    // kernels per wave: [order] vote, detect, scan x3, emit, scan x3, assoc
    ctx->launches = 1;  // finalize
    int st = HT_OK;
    ctx->cur_peaks = peaks;
    if (ctx->use_index && !ctx->use_rec) {  // count, scan x3, scatter, sort
        if ((st = build_index(ctx, s))) return st;
        ctx->launches += 6;
    }
    const std::vector<int32_t>& waves = ctx->wave_start;
    const int nwaves = waves.empty() ? 0 : (int)waves.size() - 1;
    ctx->tev_waves = ctx->timing ? std::min<int>(nwaves, (int)ctx->tev.size() / 5) : 0;
    for (int wi = 0; wi < nwaves; ++wi) {
        const int32_t e0 = waves[wi];
        const int32_t ne = waves[wi + 1] - e0;
        if ((st = mark(ctx, wi, 0, s))) return st;
        st = run_vote(ctx, e0, ne, !plain, s);
        if (st) return st;
        if ((st = mark(ctx, wi, 1, s))) return st;
        // range voting counts rows in the association (window sums over-count)
        PeakParams pp = peak_params(ctx, e0, ne, thr, peaks, peak_cap, ctx->vote_mode != HT_VOTE_POINT ? -1 : window);
        st = run_detect_scan(ctx, pp, s);
        if (st) return st;
        CU(launch_emit(pp, s));
        st = run_pairs_assoc(ctx, e0, ne, plain ? nullptr : ctx->order.p, peak_cap, peak_offsets, hit_idx, pair_cap,
                             window, wi, s);
        if (st) return st;
        if ((st = mark(ctx, wi, 2, s))) return st;
        if (ctx->wave_marks) {  // running totals after this wave, then its event (host copies follow it)
            CU(launch_publish(ctx->d_scal, ctx->d_h_wave + 2 * wi, s));
            CU(cudaEventRecord(ctx->wave_ev[wi], s));
        }
        ctx->launches += (plain ? 1 : 2) + 1 + 3 + 1 + 3 + 1 + (ctx->vote_mode != HT_VOTE_POINT ? 1 : 0) +
                         (ctx->wave_marks ? 1 : 0);
    }
    if (nwaves > 0 && (st = mark(ctx, nwaves - 1, 3, s))) return st;
    if (ctx->c_events == 0 && peak_offsets && peak_cap >= 0)
        CU(cudaMemsetAsync(peak_offsets, 0, sizeof(int64_t), s));
    CU(launch_finalize(ctx->d_scal, s));
    return HT_OK;
}

int read_err(ht_ctx* ctx) {
    int32_t err = 0;
    CU(cudaMemcpy(&err, ctx->d_err, sizeof(int32_t), cudaMemcpyDeviceToHost));
    if (err & 16) {
        CU(cudaMemset(ctx->d_err, 0, sizeof(int32_t)));
        return fail(ctx, HT_ERR_TIMEOUT, "internal: a hit-block copy into shared memory did not complete");
    }
    if (err & 8) {
        CU(cudaMemset(ctx->d_err, 0, sizeof(int32_t)));
        return fail(ctx, HT_ERR_CUDA, "internal: an association row through the angular index came out with "
                                      "another length than its window sum");
    }
    if (err) {
        CU(cudaMemset(ctx->d_err, 0, sizeof(int32_t)));
        return fail(ctx, HT_ERR_INVALID_ARG, "invalid hits in batch:%s%s%s", (err & 1) ? " non-finite or |coordinate|>1e4" : "",
                    (err & 2) ? " layer id out of range" : "", (err & 4) ? " bad event offsets" : "");
    }
    return HT_OK;
}

}  // namespace

extern "C" {

const char* ht_strerror(int status) {
    switch (status) {
        case HT_OK: return "ok";
        case HT_ERR_INVALID_ARG: return "invalid argument";
        case HT_ERR_OOM: return "out of memory";
        case HT_ERR_OVERFLOW: return "output capacity exceeded";
        case HT_ERR_CUDA: return "CUDA error";
        case HT_ERR_TIMEOUT: return "device wait timed out";
        case HT_ERR_BUDGET: return "accumulator memory budget exceeded";
        case HT_ERR_STATE: return "call out of order";
    }
    return "unknown status";
}

const char* ht_last_error(ht_ctx* ctx) { return ctx ? ctx->last_error.c_str() : "no context"; }

int ht_create(const ht_geometry* geometry, const ht_grid* grid, ht_ctx** out) {
    ht_ctx* ctx = nullptr;
    int dev_probe = 0;
    if (!out || !grid) return HT_ERR_INVALID_ARG;
    *out = nullptr;
    if (!grid_ok(*grid)) return HT_ERR_INVALID_ARG;
    if (geometry && (geometry->n_layers < 0 || geometry->n_layers > 127 || (geometry->n_layers > 0 && !geometry->layer_r)))
        return HT_ERR_INVALID_ARG;
    if (cudaGetDevice(&dev_probe) != cudaSuccess) {
        cudaGetLastError();
        return HT_ERR_CUDA;
    }
    ctx = new ht_ctx();
    ctx->grid = *grid;
    ctx->n_layers = geometry ? geometry->n_layers : 0;
    ctx->device = dev_probe;
    if (cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, ctx->device) != cudaSuccess) {
        delete ctx;
        return HT_ERR_CUDA;
    }
    build_tables(*grid, ctx->h_cphi, ctx->h_sphi, ctx->h_d0);
    ctx->K = make_consts(*grid, ctx->h_d0);
    ctx->cells = (int64_t)grid->n_phi * grid->n_d0 * grid->n_kappa;
    ctx->cols_per_event = (int64_t)grid->n_phi * grid->n_d0;
    ctx->nkw = (grid->n_kappa + 31) / 32;
    ctx->pnd = grid->n_d0;
    ctx->pnk = grid->n_kappa;
    ctx->Kp = ctx->K;
    std::vector<float4> dt(grid->n_d0);
    for (int j = 0; j < grid->n_d0; ++j) {
        const float d = ctx->h_d0[j];
        // (d0, 2 d0, d0^2, d0 * S2): the last is the kappa-scaled d0 of stage 1
        dt[j] = make_float4(d, d + d, d * d, (float)((double)d * (double)ctx->K.S2));
    }
    build_edges(*grid, ctx->h_ecos, ctx->h_esin, ctx->h_de);
    std::vector<float4> dte(grid->n_d0 + 1);
    for (int n = 0; n <= grid->n_d0; ++n) {
        const float d = ctx->h_de[n];
        dte[n] = make_float4(d, d + d, d * d, (float)((double)d * (double)ctx->K.S2));
    }
    int st = HT_OK;
    auto bad = [&](cudaError_t e) {
        if (e == cudaSuccess) return false;
        st = fail(ctx, e == cudaErrorMemoryAllocation ? HT_ERR_OOM : HT_ERR_CUDA, "ht_create: %s", cudaGetErrorString(e));
        return true;
    };
    if (bad(cudaMalloc(&ctx->d_cphi, grid->n_phi * sizeof(float))) ||
        bad(cudaMalloc(&ctx->d_sphi, grid->n_phi * sizeof(float))) ||
        bad(cudaMalloc(&ctx->d_dtab, grid->n_d0 * sizeof(float4))) ||
        bad(cudaMalloc(&ctx->d_ecos, grid->n_phi * sizeof(float))) ||
        bad(cudaMalloc(&ctx->d_esin, grid->n_phi * sizeof(float))) ||
        bad(cudaMalloc(&ctx->d_edtab, (grid->n_d0 + 1) * sizeof(float4))) ||
        bad(cudaMalloc(&ctx->d_scal, 8 * sizeof(int64_t))) || bad(cudaMalloc(&ctx->d_err, sizeof(int32_t))) ||
        bad(cudaMalloc(&ctx->d_queue, 16)) || bad(cudaMalloc(&ctx->d_stats, 4 * sizeof(unsigned long long))) ||
        bad(cudaMallocHost(&ctx->h_pinned, 8 * sizeof(int64_t))) ||
        bad(cudaMemcpy(ctx->d_cphi, ctx->h_cphi.data(), grid->n_phi * sizeof(float), cudaMemcpyHostToDevice)) ||
        bad(cudaMemcpy(ctx->d_sphi, ctx->h_sphi.data(), grid->n_phi * sizeof(float), cudaMemcpyHostToDevice)) ||
        bad(cudaMemcpy(ctx->d_dtab, dt.data(), grid->n_d0 * sizeof(float4), cudaMemcpyHostToDevice)) ||
        bad(cudaMemcpy(ctx->d_ecos, ctx->h_ecos.data(), grid->n_phi * sizeof(float), cudaMemcpyHostToDevice)) ||
        bad(cudaMemcpy(ctx->d_esin, ctx->h_esin.data(), grid->n_phi * sizeof(float), cudaMemcpyHostToDevice)) ||
        bad(cudaMemcpy(ctx->d_edtab, dte.data(), (grid->n_d0 + 1) * sizeof(float4), cudaMemcpyHostToDevice)) ||
        bad(cudaMemset(ctx->d_err, 0, sizeof(int32_t))) || bad(cudaMemset(ctx->d_stats, 0, 4 * sizeof(unsigned long long))) ||
        bad(cudaMemset(ctx->d_scal, 0, 8 * sizeof(int64_t)))) {
        ht_destroy(ctx);
        return st;
    }
    ctx->d_aqueue = reinterpret_cast<unsigned long long*>(reinterpret_cast<char*>(ctx->d_queue) + 8);
    st = resolve_tiles(ctx);
    if (st) {
        ht_destroy(ctx);
        return st;
    }
    *out = ctx;
    return HT_OK;
}

int ht_destroy(ht_ctx* ctx) {
    if (!ctx) return HT_ERR_INVALID_ARG;
    cudaDeviceSynchronize();
    if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
    for (auto& e : ctx->tev)
        if (e) cudaEventDestroy(e);
    for (void* p : {(void*)ctx->d_ecos, (void*)ctx->d_esin, (void*)ctx->d_edtab})
        if (p) cudaFree(p);
    for (void* p : {(void*)ctx->d_cphi, (void*)ctx->d_sphi, (void*)ctx->d_dtab, (void*)ctx->d_scal, (void*)ctx->d_err,
                    (void*)ctx->d_queue, (void*)ctx->d_stats})
        if (p) cudaFree(p);
    if (ctx->h_pinned) cudaFreeHost(ctx->h_pinned);
    if (ctx->own_stream) cudaStreamDestroy(ctx->own_stream);
    if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
    for (cudaEvent_t ev : ctx->wave_ev) cudaEventDestroy(ev);
    if (ctx->h_wave) cudaFreeHost(ctx->h_wave);
    ctx->rec.release();
    ctx->rbits.release();
    ctx->sx.release();
    ctx->sy.release();
    ctx->slayer.release();
    ctx->soffs.release();
    ctx->acc.release();
    ctx->mask.release();
    ctx->wpre.release();
    ctx->npk.release();
    ctx->colbase.release();
    ctx->order.release();
    ctx->paircnt.release();
    ctx->peaks.release();
    ctx->peakoff.release();
    ctx->hitidx.release();
    ctx->fits.release();
    ctx->mstate.release();
    ctx->ibcount.release();
    ctx->ibcursor.release();
    ctx->ihid.release();
    ctx->itab.release();
    ctx->ibstart.release();
    ctx->ir2min.release();
    ctx->ir2max.release();
    ctx->itheta.release();
    ctx->mkept.release();
    ctx->vacc.release();
    ctx->vrow.release();
    ctx->vbase.release();
    ctx->vscal.release();
    ctx->vout.release();
    ctx->scratch.release();
    delete ctx;
    return HT_OK;
}

int ht_set_option(ht_ctx* ctx, int32_t key, int64_t value) {
    if (!ctx) return HT_ERR_INVALID_ARG;
    switch (key) {
        case HT_OPT_MODE:
            if (value != HT_MODE_BATCHED && value != HT_MODE_PLAIN) return fail(ctx, HT_ERR_INVALID_ARG, "bad mode");
            ctx->mode = (int)value;
            break;
        case HT_OPT_TILE_PHI:
            if (value != 0 && value != 1 && value != 2 && value != 4 && value != 8)
                return fail(ctx, HT_ERR_INVALID_ARG, "tile_phi must be 0, 1, 2, 4 or 8");
            ctx->tile_phi = (int)value;
            break;
        case HT_OPT_TILE_D0:
            if (value < 0 || value > ctx->grid.n_d0) return fail(ctx, HT_ERR_INVALID_ARG, "tile_d0 out of range");
            ctx->tile_d = (int)value;
            break;
        case HT_OPT_THREADS:
            if (value != 0 && value != 128 && value != 256)
                return fail(ctx, HT_ERR_INVALID_ARG, "threads must be 0, 128 or 256");
            ctx->threads = (int)value;
            break;
        case HT_OPT_ACC_BUDGET:
            if (value < 0) return fail(ctx, HT_ERR_INVALID_ARG, "budget < 0");
            ctx->budget = value ? value : kDefaultBudget;
            break;
        case HT_OPT_COUNT_STAGES: ctx->count_stages = value != 0; break;
        case HT_OPT_USE_GRAPH: ctx->use_graph = value != 0; break;
        case HT_OPT_PRUNE:
            if (value < 0 || value > 3) return fail(ctx, HT_ERR_INVALID_ARG, "prune must be 0..3");
            ctx->prune = (int)value;
            break;
        case HT_OPT_ATILE_PHI:
            if (value != 0 && value != 1 && value != 2 && value != 4 && value != 8)
                return fail(ctx, HT_ERR_INVALID_ARG, "association tile_phi must be 0, 1, 2, 4 or 8");
            ctx->atile_phi = (int)value;
            break;
        case HT_OPT_ATILE_D0:
            if (value < 0 || value > ctx->grid.n_d0) return fail(ctx, HT_ERR_INVALID_ARG, "association tile_d0 out of range");
            ctx->atile_d = (int)value;
            break;
        case HT_OPT_ASSOC_CURSORS:
            if (value < 0 || value > 65536 || (value % 32) != 0)
                return fail(ctx, HT_ERR_INVALID_ARG, "association cursors must be 0 or a multiple of 32 up to 65536");
            ctx->acap = (int)value;
            break;
        case HT_OPT_HOST_CHUNKS:
            if (value < 1 || value > 64) return fail(ctx, HT_ERR_INVALID_ARG, "host chunks must be in [1, 64]");
            ctx->host_chunks = (int)value;
            break;
        case HT_OPT_ASSOC_INDEX:
            if (value != 0 && value != 1) return fail(ctx, HT_ERR_INVALID_ARG, "assoc index must be 0 or 1");
            ctx->assoc_index = (int)value;
            ctx->gvalid = false;
            break;
        case HT_OPT_RECORDS:
            if (value != 0 && value != 1) return fail(ctx, HT_ERR_INVALID_ARG, "records must be 0 or 1");
            ctx->records = (int)value;
            break;
        case HT_OPT_VOTE_ITEMS:
            if (value != 0 && value != 1) return fail(ctx, HT_ERR_INVALID_ARG, "vote items must be 0 or 1");
            ctx->vote_items = (int)value;
            break;
        case HT_OPT_HIT_STAGING:
            if (value != 0 && value != 1) return fail(ctx, HT_ERR_INVALID_ARG, "hit staging must be 0 or 1");
            ctx->hit_staging = (int)value;
            break;
        case HT_OPT_HOST_COPY:
            if (value < 0 || value > 4096) return fail(ctx, HT_ERR_INVALID_ARG, "host copy must be in [0, 4096]");
            ctx->host_copy = (int)value;
            break;
        case HT_OPT_BAND_SPLIT:
            if (value < -1 || value > 256) return fail(ctx, HT_ERR_INVALID_ARG, "band split must be in [-1, 256]");
            ctx->band_split = (int)value;
            break;
        case HT_OPT_RECORD_BUDGET:
            if (value < 0) return fail(ctx, HT_ERR_INVALID_ARG, "record budget < 0");
            ctx->rec_budget = value ? value : kDefaultRecBudget;
            break;
        case HT_OPT_VOTE_MODE: {
            if (value != HT_VOTE_POINT && value != HT_VOTE_RANGE && value != HT_VOTE_LINE)
                return fail(ctx, HT_ERR_INVALID_ARG, "vote mode must be HT_VOTE_POINT, HT_VOTE_RANGE or HT_VOTE_LINE");
            if (value == HT_VOTE_LINE && ctx->grid.n_kappa != 1)
                return fail(ctx, HT_ERR_INVALID_ARG, "line voting needs a grid with n_kappa = 1");
            const bool line = value == HT_VOTE_LINE;
            const int pnd = line ? 1 : ctx->grid.n_d0, pnk = line ? ctx->grid.n_d0 : ctx->grid.n_kappa;
            ctx->vote_mode = (int)value;
            ctx->pnd = pnd;
            ctx->pnk = pnk;
            ctx->nkw = (pnk + 31) / 32;
            ctx->cols_per_event = (int64_t)ctx->grid.n_phi * pnd;
            ctx->Kp = ctx->K;
            ctx->Kp.nd = pnd;
            ctx->Kp.nk = pnk;
            ctx->have_votes = ctx->have_peaks = ctx->have_results = false;
            ++ctx->gen;
            break;
        }
        case HT_OPT_PHASE_TIMING:
            if (value) {
                const int st = ensure_timing_events(ctx, 1);
                if (st) return st;
            }
            ctx->timing = value != 0;
            break;
        default: return fail(ctx, HT_ERR_INVALID_ARG, "unknown option %d", key);
    }
    ctx->gvalid = false;
    if (key == HT_OPT_TILE_PHI || key == HT_OPT_TILE_D0 || key == HT_OPT_THREADS || key == HT_OPT_ATILE_PHI ||
        key == HT_OPT_ATILE_D0 || key == HT_OPT_PRUNE || key == HT_OPT_VOTE_MODE || key == HT_OPT_ASSOC_CURSORS ||
        key == HT_OPT_RECORDS || key == HT_OPT_VOTE_ITEMS || key == HT_OPT_HIT_STAGING || key == HT_OPT_BAND_SPLIT) {
        int st = resolve_tiles(ctx);
        if (st) return st;
    }
    return HT_OK;
}

int ht_get_option(ht_ctx* ctx, int32_t key, int64_t* value) {
    if (!ctx || !value) return HT_ERR_INVALID_ARG;
    switch (key) {
        case HT_OPT_MODE: *value = ctx->mode; break;
        case HT_OPT_TILE_PHI: *value = ctx->r_tile_phi; break;
        case HT_OPT_TILE_D0: *value = ctx->r_tile_d; break;
        case HT_OPT_THREADS: *value = ctx->r_threads; break;
        case HT_OPT_ACC_BUDGET: *value = ctx->budget; break;
        case HT_OPT_COUNT_STAGES: *value = ctx->count_stages; break;
        case HT_OPT_USE_GRAPH: *value = ctx->use_graph; break;
        case HT_OPT_PHASE_TIMING: *value = ctx->timing; break;
        case HT_OPT_ATILE_PHI: *value = ctx->a_tile_phi; break;
        case HT_OPT_PRUNE: *value = (ctx->r_band ? 1 : 0) | (ctx->a_band ? 2 : 0); break;
        case HT_OPT_ATILE_D0: *value = ctx->a_tile_d; break;
        case HT_OPT_VOTE_MODE: *value = ctx->vote_mode; break;
        case HT_OPT_ASSOC_CURSORS: *value = ctx->r_rec ? ctx->rc_cap : ctx->a_cap; break;
        case HT_OPT_HOST_CHUNKS: *value = ctx->host_chunks; break;
        case HT_OPT_ASSOC_INDEX: *value = ctx->assoc_index; break;
        case HT_OPT_LAUNCHES: *value = ctx->launches; break;
        case HT_OPT_RECORDS: *value = ctx->r_rec ? 1 : 0; break;
        case HT_OPT_VOTE_ITEMS: *value = ctx->vote_items; break;
        case HT_OPT_HIT_STAGING: *value = ctx->r_stage ? 1 : 0; break;
        case HT_OPT_BAND_SPLIT: *value = ctx->r_narrow; break;
        case HT_OPT_HOST_COPY: *value = ctx->host_copy; break;
        case HT_OPT_RECORD_BUDGET: *value = ctx->rec_budget; break;
        case HT_OPT_WAVES: *value = ctx->wave_start.empty() ? 0 : (int64_t)ctx->wave_start.size() - 1; break;
        default: return fail(ctx, HT_ERR_INVALID_ARG, "unknown option %d", key);
    }
    return HT_OK;
}

int ht_vote(ht_ctx* ctx, const ht_hits* hits, void* stream) {
    if (!ctx) return HT_ERR_INVALID_ARG;
    cudaStream_t s = nullptr;
    if (int st0 = resolve_stream(ctx, stream, &s)) return st0;
    if (hits && (int64_t)hits->n_events * ctx->cells * 4 > ctx->budget)
        return fail(ctx, HT_ERR_BUDGET, "%d accumulators of %lld B exceed the budget of %lld B", hits->n_events,
                    (long long)(ctx->cells * 4), (long long)ctx->budget);
    int st = stage_hits(ctx, hits, s);
    if (st) return st;
    ctx->stream = s;
    ctx->have_votes = ctx->have_peaks = ctx->have_results = false;
    ctx->use_rec = false;  // the separate calls bin again in ht_associate
    st = ensure_wave_buffers(ctx, ctx->c_events);
    if (st) return st;
    const bool plain = ctx->mode == HT_MODE_PLAIN;
    if (plain) {
        for (int32_t e = 0; e < ctx->c_events; ++e) {
            VoteParams p = vote_params(ctx, e, 1, false);
            p.acc = ctx->acc.p + (int64_t)e * ctx->cells;
            CU(launch_vote(ctx->r_tile_phi, p, p.n_items, ctx->r_threads, ctx->r_smem, s, ctx->r_variant));
        }
    } else {
        st = run_vote(ctx, 0, ctx->c_events, true, s);
        if (st) return st;
    }
    ctx->c_event0 = 0;
    ctx->c_wave_events = ctx->c_events;
    ctx->have_votes = true;
    return HT_OK;
}

int ht_peaks(ht_ctx* ctx, uint32_t threshold, ht_peak* out, int64_t cap, int64_t* n_out) {
    if (!ctx || !n_out || cap < 0 || (cap > 0 && !out)) return HT_ERR_INVALID_ARG;
    if (!ctx->have_votes) return fail(ctx, HT_ERR_STATE, "ht_peaks needs a preceding ht_vote");
    cudaStream_t s = ctx->stream;
    int st = read_err(ctx);
    if (st) return st;
    CU(cudaMemsetAsync(ctx->d_scal, 0, 8 * sizeof(int64_t), s));
    PeakParams pp = peak_params(ctx, 0, ctx->c_events, threshold, nullptr, 0, -1);
    st = run_detect_scan(ctx, pp, s);
    if (st) return st;
    CU(cudaMemcpyAsync(ctx->h_pinned, ctx->d_scal, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    const int64_t total = ctx->h_pinned[0];
    CU(ctx->peaks.ensure(std::max<int64_t>(total, 1), &ctx->gen));
    pp.peaks = ctx->peaks.p;
    pp.peak_cap = total;
    CU(launch_emit(pp, s));
    const int64_t ncopy = std::min(total, cap);
    if (ncopy > 0) CU(cudaMemcpyAsync(out, ctx->peaks.p, ncopy * sizeof(ht_peak), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    *n_out = total;
    ctx->n_peaks_held = total;
    ctx->last_threshold = threshold;
    ctx->have_peaks = true;
    if (total > cap) return fail(ctx, HT_ERR_OVERFLOW, "%lld peaks, cap %lld", (long long)total, (long long)cap);
    return HT_OK;
}

int ht_associate(ht_ctx* ctx, int32_t window, int64_t* peak_offsets, int32_t* hit_idx, int64_t cap, int64_t* n_pairs) {
    if (!ctx || !n_pairs || !peak_offsets || cap < 0 || (cap > 0 && !hit_idx) || window < 0 || window > 15)
        return HT_ERR_INVALID_ARG;
    if (!ctx->have_peaks) return fail(ctx, HT_ERR_STATE, "ht_associate needs a preceding ht_peaks");
    cudaStream_t s = ctx->stream;
    const int64_t np = ctx->n_peaks_held;
    CU(ctx->paircnt.ensure(std::max<int64_t>(np, 1), &ctx->gen));
    CU(ctx->peakoff.ensure(np + 1, &ctx->gen));
    // per-peak pair counts from the accumulators, then their scan
    CU(cudaMemsetAsync(ctx->d_scal, 0, 8 * sizeof(int64_t), s));
    ctx->h_pinned[0] = np;
    CU(cudaMemcpyAsync(ctx->d_scal + 0, ctx->h_pinned, sizeof(int64_t), cudaMemcpyHostToDevice, s));
    if (ctx->vote_mode != HT_VOTE_POINT) {
        AssocParams c{};
        c.peak_offsets = ctx->peakoff.p;
        c.peak_cap = np;
        c.window = window;
        c.paircnt = ctx->paircnt.p;
        c.extra_pairs = ctx->d_scal + 4;
        const int st = launch_assoc_ctx(ctx, c, 0, ctx->c_events, nullptr, 1, s);
        if (st) return st;
    } else {
        PeakParams pp = peak_params(ctx, 0, ctx->c_events, ctx->last_threshold, ctx->peaks.p, np, window);
        CU(launch_paircount(pp, ctx->d_scal + 2, ctx->d_scal + 0, s));
    }
    CU(cudaMemcpyAsync(ctx->d_scal + 3, ctx->d_scal + 1, sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
    ScanRange r{};
    r.in = ctx->paircnt.p;
    r.out = ctx->peakoff.p;
    r.lo_dev = ctx->d_scal + 2;
    r.hi_dev = ctx->d_scal + 0;
    r.cap = np;
    r.base_dev = ctx->d_scal + 3;
    r.total = ctx->d_scal + 1;
    r.write_end = 1;
    CU(launch_scan(r, ctx->scratch.p, s));
    CU(cudaMemcpyAsync(ctx->h_pinned + 1, ctx->d_scal + 1, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    const int64_t total = ctx->h_pinned[1];
    CU(ctx->hitidx.ensure(std::max<int64_t>(total, 1), &ctx->gen));
    AssocParams a{};
    a.peak_offsets = ctx->peakoff.p;
    a.peak_cap = np;
    a.hit_idx = ctx->hitidx.p;
    a.pair_cap = total;
    a.window = window;
    const int st = launch_assoc_ctx(ctx, a, 0, ctx->c_events, nullptr, ctx->vote_mode != HT_VOTE_POINT ? 2 : 0, s);
    if (st) return st;
    CU(cudaMemcpyAsync(peak_offsets, ctx->peakoff.p, (np + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    const int64_t ncopy = std::min(total, cap);
    if (ncopy > 0) CU(cudaMemcpyAsync(hit_idx, ctx->hitidx.p, ncopy * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    *n_pairs = total;
    if (total > cap) return fail(ctx, HT_ERR_OVERFLOW, "%lld pairs, cap %lld", (long long)total, (long long)cap);
    return HT_OK;
}

// The device address of a page-locked host result array, for copies by
// host_copy_kernel; nullptr for pageable memory (copied by the copy engine).
static unsigned char* locked_addr(const void* p) {
    if (!p) return nullptr;
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost && a.devicePointer ? static_cast<unsigned char*>(a.devicePointer) : nullptr;
}

// bytes [off, off + bytes) of a device result array into the host array `dst`
// (device address `dst_dev` when page-locked and kernel copies are on)
static int copy_out(ht_ctx* ctx, void* dst, unsigned char* dst_dev, const void* src, size_t off, size_t bytes,
                    cudaStream_t s) {
    if (bytes == 0) return HT_OK;
    const unsigned char* from = static_cast<const unsigned char*>(src) + off;
    if (dst_dev)
        CU(launch_host_copy(dst_dev + off, from, bytes, ctx->host_copy, s));
    else
        CU(cudaMemcpyAsync(static_cast<unsigned char*>(dst) + off, from, bytes, cudaMemcpyDeviceToHost, s));
    ++ctx->launches;
    return HT_OK;
}

int ht_process(ht_ctx* ctx, const ht_hits* hits, uint32_t threshold, int32_t window, const ht_results* res,
               void* stream) {
    if (!ctx || !res || window < 0 || window > 15) return HT_ERR_INVALID_ARG;
    if (res->peak_cap < 0 || res->pair_cap < 0 || !res->counts || !res->peak_offsets ||
        (res->peak_cap > 0 && !res->peaks) || (res->pair_cap > 0 && !res->hit_idx) ||
        (res->mem != HT_HOST && res->mem != HT_DEVICE))
        return fail(ctx, HT_ERR_INVALID_ARG, "bad ht_results");
    cudaStream_t s = nullptr;
    if (int st0 = resolve_stream(ctx, stream, &s)) return st0;
    int st = stage_hits(ctx, hits, s);
    if (st) return st;
    ctx->stream = s;
    ctx->have_votes = ctx->have_peaks = ctx->have_results = false;
    const int32_t epw = events_per_wave(ctx, ctx->c_events);
    if (epw < 1)
        return fail(ctx, HT_ERR_BUDGET, "one accumulator (%lld B) exceeds the budget", (long long)(ctx->cells * 4));
    st = ensure_wave_buffers(ctx, ctx->mode == HT_MODE_PLAIN ? 1 : epw);
    if (st) return st;
    const int64_t pcap = res->peak_cap, qcap = res->pair_cap;
    CU(ctx->paircnt.ensure(std::max<int64_t>(pcap, 1), &ctx->gen));
    st = ensure_index(ctx);
    if (st) return st;
    ht_peak* peaks = res->peaks;
    int64_t* poff = res->peak_offsets;
    int32_t* hidx = res->hit_idx;
    if (res->mem == HT_HOST) {
        CU(ctx->peaks.ensure(std::max<int64_t>(pcap, 1), &ctx->gen));
        CU(ctx->peakoff.ensure(pcap + 1, &ctx->gen));
        CU(ctx->hitidx.ensure(std::max<int64_t>(qcap, 1), &ctx->gen));
        peaks = ctx->peaks.p;
        poff = ctx->peakoff.p;
        hidx = ctx->hitidx.p;
    }
    // host results in batched mode: at least host_chunks waves, each copied
    // to the host on the copy stream while the following waves compute
    const bool pipe = res->mem == HT_HOST && ctx->mode == HT_MODE_BATCHED && ctx->host_chunks > 1 &&
                      ctx->c_events > 1;
    int32_t step = epw;
    if (pipe) step = std::min<int32_t>(epw, (ctx->c_events + ctx->host_chunks - 1) / ctx->host_chunks);
    st = plan_waves(ctx, hits, ctx->mode == HT_MODE_PLAIN ? 1 : step, s);
    if (st) return st;
    const int32_t nwaves = (int32_t)ctx->wave_start.size() - 1;
    if (ctx->timing) {
        st = ensure_timing_events(ctx, nwaves);
        if (st) return st;
    }
    ctx->wave_marks = pipe;
    if (pipe) {
        while ((int32_t)ctx->wave_ev.size() < nwaves) {
            cudaEvent_t ev = nullptr;
            CU(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
            ctx->wave_ev.push_back(ev);
        }
        if (ctx->h_wave_n < nwaves) {
            if (ctx->h_wave) cudaFreeHost(ctx->h_wave);
            ctx->h_wave = nullptr;
            ctx->d_h_wave = nullptr;
            ctx->h_wave_n = 0;
            CU(cudaHostAlloc(reinterpret_cast<void**>(&ctx->h_wave), 2 * sizeof(int64_t) * (size_t)nwaves,
                             cudaHostAllocMapped));
            CU(cudaHostGetDevicePointer(reinterpret_cast<void**>(&ctx->d_h_wave), ctx->h_wave, 0));
            ctx->h_wave_n = nwaves;
        }
        if (!ctx->copy_stream) CU(cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking));
    }
    // the wave-by-wave copies wait on events recorded by direct launches (a
    // few dozen launches per batch), so that path does not replay the graph
    const bool graph = ctx->use_graph && ctx->mode == HT_MODE_BATCHED && !pipe;
    if (graph) {
        GraphKey key{};
        key.ptrs[0] = ctx->cx;
        key.ptrs[1] = ctx->cy;
        key.ptrs[2] = ctx->coffs;
        key.ptrs[3] = peaks;
        key.ptrs[4] = poff;
        key.ptrs[5] = hidx;
        key.ptrs[6] = s;
        key.ptrs[7] = ctx->use_index ? ctx->clayer : nullptr;
        key.vals[0] = ctx->c_hits;
        key.vals[1] = ctx->c_events;
        key.vals[2] = threshold;
        key.vals[3] = window;
        key.vals[4] = pcap;
        key.vals[5] = qcap;
        key.vals[6] = step;
        key.vals[7] = ctx->gen;
        key.vals[8] = ctx->r_tile_phi * 100000 + ctx->r_tile_d;
        key.vals[9] = ctx->r_threads;
        key.vals[10] = ctx->count_stages * 2 + ctx->timing;
        key.vals[11] = ((int64_t)ctx->a_tile_phi << 40) | ((int64_t)ctx->a_tile_d << 20) | ((int64_t)ctx->a_cap << 2) |
                       (ctx->r_band ? 2 : 0) | (ctx->a_band ? 1 : 0) | ((int64_t)ctx->vote_mode << 60);
        key.vals[12] = (ctx->use_rec ? 1 : 0) | ((int64_t)ctx->rc_cap << 1) | ((int64_t)ctx->r_variant << 40) |
                       ((int64_t)ctx->r_stage << 48);
        if (!ctx->gvalid || !(key == ctx->gkey) || ctx->gwaves != ctx->wave_start) {
            if (ctx->gexec) {
                cudaGraphExecDestroy(ctx->gexec);
                ctx->gexec = nullptr;
            }
            ctx->gvalid = false;
            cudaGraph_t g = nullptr;
            CU(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
            st = process_device(ctx, threshold, window, peaks, pcap, poff, hidx, qcap, s);
            cudaError_t ce = cudaStreamEndCapture(s, &g);
            if (st) {
                if (g) cudaGraphDestroy(g);
                return st;
            }
            CU(ce);
            cudaError_t ie = cudaGraphInstantiate(&ctx->gexec, g, 0);
            cudaGraphDestroy(g);
            CU(ie);
            ctx->gkey = key;
            ctx->gwaves = ctx->wave_start;
            ctx->gvalid = true;
        }
        CU(cudaGraphLaunch(ctx->gexec, s));
    } else {
        st = process_device(ctx, threshold, window, peaks, pcap, poff, hidx, qcap, s);
        if (st) return st;
    }
    ctx->have_results = true;
    // counts = {peak total, pair total + pairs of peaks beyond the cap}
    if (res->mem == HT_DEVICE) {
        CU(cudaMemcpyAsync(res->counts, ctx->d_scal + 6, 2 * sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
        ctx->pending_check = true;
        ctx->pending_copy = *res;
        return HT_OK;
    }
    CU(cudaMemcpyAsync(ctx->h_pinned, ctx->d_scal + 6, 2 * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    unsigned char* dk_peaks = ctx->host_copy ? locked_addr(res->peaks) : nullptr;
    unsigned char* dk_poff = ctx->host_copy ? locked_addr(res->peak_offsets) : nullptr;
    unsigned char* dk_hidx = ctx->host_copy ? locked_addr(res->hit_idx) : nullptr;
    // stored peaks / pairs already on the host (wave by wave)
    int64_t p_done = 0, q_done = 0;
    if (pipe) {
        cudaStream_t cs = ctx->copy_stream;
        for (int32_t w = 0; w < nwaves; ++w) {
            CU(cudaEventSynchronize(ctx->wave_ev[w]));
            const int64_t p_cur = std::min(ctx->h_wave[2 * w], pcap), q_cur = std::min(ctx->h_wave[2 * w + 1], qcap);
            CU(cudaStreamWaitEvent(cs, ctx->wave_ev[w], 0));
            if (p_cur > p_done) {
                st = copy_out(ctx, res->peaks, dk_peaks, peaks, p_done * sizeof(ht_peak),
                              (p_cur - p_done) * sizeof(ht_peak), cs);
                if (!st)
                    st = copy_out(ctx, res->peak_offsets, dk_poff, poff, p_done * sizeof(int64_t),
                                  (p_cur - p_done) * sizeof(int64_t), cs);
                if (st) return st;
                p_done = p_cur;
            }
            if (q_cur > q_done) {
                st = copy_out(ctx, res->hit_idx, dk_hidx, hidx, q_done * sizeof(int32_t),
                              (q_cur - q_done) * sizeof(int32_t), cs);
                if (st) return st;
                q_done = q_cur;
            }
        }
    }
    CU(cudaStreamSynchronize(s));
    st = read_err(ctx);
    if (st) {
        if (pipe) cudaStreamSynchronize(ctx->copy_stream);
        return st;
    }
    const int64_t np = ctx->h_pinned[0], nq = ctx->h_pinned[1];
    res->counts[0] = np;
    res->counts[1] = nq;
    const int64_t cp = std::min(np, pcap), cq = std::min(nq, qcap);
    // the rest (everything, without the wave copies) and the final row end
    if (cp > p_done) st = copy_out(ctx, res->peaks, dk_peaks, peaks, p_done * sizeof(ht_peak),
                                   (cp - p_done) * sizeof(ht_peak), s);
    const int64_t o0 = std::min(p_done, cp);
    if (!st)
        st = copy_out(ctx, res->peak_offsets, dk_poff, poff, o0 * sizeof(int64_t), (cp + 1 - o0) * sizeof(int64_t), s);
    if (!st && cq > q_done)
        st = copy_out(ctx, res->hit_idx, dk_hidx, hidx, q_done * sizeof(int32_t), (cq - q_done) * sizeof(int32_t), s);
    if (st) {
        cudaStreamSynchronize(s);
        if (pipe) cudaStreamSynchronize(ctx->copy_stream);
        return st;
    }
    CU(cudaStreamSynchronize(s));
    if (pipe) CU(cudaStreamSynchronize(ctx->copy_stream));
    if (np > pcap || nq > qcap)
        return fail(ctx, HT_ERR_OVERFLOW, "%lld peaks (cap %lld), %lld pairs (cap %lld)", (long long)np,
                    (long long)pcap, (long long)nq, (long long)qcap);
    return HT_OK;
}

int ht_sync(ht_ctx* ctx) {
    if (!ctx) return HT_ERR_INVALID_ARG;
    CU(cudaStreamSynchronize(ctx->stream));
    if (ctx->timing && ctx->c_events > 0 && ctx->tev_waves > 0) {
        // vote, peaks + association and association summed over the waves;
        // the whole step from the first wave's start to the end
        float sum[4] = {0, 0, 0, 0}, ms = 0;
        const int nw = ctx->tev_waves;
        for (int w = 0; w < nw; ++w) {
            const cudaEvent_t* t = ctx->tev.data() + 5 * w;
            if (cudaEventElapsedTime(&ms, t[0], t[1]) == cudaSuccess) sum[0] += ms;
            if (cudaEventElapsedTime(&ms, t[1], t[2]) == cudaSuccess) sum[1] += ms;
            if (cudaEventElapsedTime(&ms, t[4], t[2]) == cudaSuccess) sum[3] += ms;
        }
        if (cudaEventElapsedTime(&ms, ctx->tev[0], ctx->tev[5 * (nw - 1) + 3]) == cudaSuccess) sum[2] = ms;
        cudaGetLastError();
        for (int i = 0; i < 4; ++i) ctx->phase_ms[i] = sum[i];
    }
    int st = read_err(ctx);
    if (st) return st;
    if (ctx->pending_check) {
        ctx->pending_check = false;
        CU(cudaMemcpy(ctx->h_pinned, ctx->d_scal + 6, 2 * sizeof(int64_t), cudaMemcpyDeviceToHost));
        if (ctx->h_pinned[0] > ctx->pending_copy.peak_cap || ctx->h_pinned[1] > ctx->pending_copy.pair_cap)
            return fail(ctx, HT_ERR_OVERFLOW, "%lld peaks (cap %lld), %lld pairs (cap %lld)",
                        (long long)ctx->h_pinned[0], (long long)ctx->pending_copy.peak_cap,
                        (long long)ctx->h_pinned[1], (long long)ctx->pending_copy.pair_cap);
    }
    return HT_OK;
}

int ht_get_accumulator(ht_ctx* ctx, int32_t event, uint32_t* out) {
    if (!ctx || !out) return HT_ERR_INVALID_ARG;
    if (!ctx->have_votes) return fail(ctx, HT_ERR_STATE, "no accumulators: call ht_vote first");
    if (event < 0 || event >= ctx->c_wave_events) return fail(ctx, HT_ERR_INVALID_ARG, "event %d out of range", event);
    CU(cudaStreamSynchronize(ctx->stream));
    CU(cudaMemcpy(out, ctx->acc.p + (int64_t)event * ctx->cells, ctx->cells * sizeof(uint32_t), cudaMemcpyDeviceToHost));
    return HT_OK;
}

int ht_get_tables(ht_ctx* ctx, float* cos_phi, float* sin_phi, float* d0) {
    if (!ctx) return HT_ERR_INVALID_ARG;
    if (cos_phi) std::memcpy(cos_phi, ctx->h_cphi.data(), ctx->h_cphi.size() * sizeof(float));
    if (sin_phi) std::memcpy(sin_phi, ctx->h_sphi.data(), ctx->h_sphi.size() * sizeof(float));
    if (d0) std::memcpy(d0, ctx->h_d0.data(), ctx->h_d0.size() * sizeof(float));
    return HT_OK;
}

int ht_fit(ht_ctx* ctx, const ht_results* res, ht_track* out, int64_t cap, void* stream) {
    if (!ctx || !res || cap < 0 || (cap > 0 && !out)) return HT_ERR_INVALID_ARG;
    if (res->mem != HT_HOST && res->mem != HT_DEVICE) return fail(ctx, HT_ERR_INVALID_ARG, "res.mem must be HT_HOST or HT_DEVICE");
    if (!ctx->have_results) return fail(ctx, HT_ERR_STATE, "ht_fit needs a preceding ht_process");
    cudaStream_t s = nullptr;
    if (int st0 = resolve_stream(ctx, stream, &s)) return st0;
    FitParams p{};
    p.x = ctx->cx;
    p.y = ctx->cy;
    p.peak_cap = res->peak_cap;
    p.pair_cap = res->pair_cap;
    p.cap = cap;
    p.kmin = (double)ctx->grid.kappa_min;
    p.kmax = (double)ctx->grid.kappa_max;
    p.nk = ctx->grid.n_kappa;
    if (res->mem == HT_DEVICE) {
        p.peaks = res->peaks;
        p.po = res->peak_offsets;
        p.hidx = res->hit_idx;
        p.n_peaks = res->counts;
        p.out = out;
        CU(launch_fit(p, s));
        return HT_OK;
    }
    // host results: the context still holds them on the device
    const int64_t n = std::min(std::min(res->counts[0], res->peak_cap), cap);
    if (n <= 0) return HT_OK;
    CU(ctx->fits.ensure(n, &ctx->gen));
    p.peaks = ctx->peaks.p;
    p.po = ctx->peakoff.p;
    p.hidx = ctx->hitidx.p;
    p.n_peaks = ctx->d_scal + 6;
    p.cap = n;
    p.out = ctx->fits.p;
    CU(launch_fit(p, s));
    CU(cudaMemcpyAsync(out, ctx->fits.p, n * sizeof(ht_track), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    return HT_OK;
}

int ht_merge(ht_ctx* ctx, const ht_results* res, const ht_track* fits, int32_t radius, int32_t* state,
             int64_t cap, int64_t* n_kept, void* stream) {
    if (!ctx || !res || !n_kept || cap < 0 || (cap > 0 && (!fits || !state))) return HT_ERR_INVALID_ARG;
    if (radius < 0 || radius > 64) return fail(ctx, HT_ERR_INVALID_ARG, "merge radius must be in [0, 64]");
    if (res->mem != HT_HOST && res->mem != HT_DEVICE) return fail(ctx, HT_ERR_INVALID_ARG, "res.mem must be HT_HOST or HT_DEVICE");
    if (!ctx->have_results) return fail(ctx, HT_ERR_STATE, "ht_merge needs a preceding ht_process");
    cudaStream_t s = nullptr;
    if (int st0 = resolve_stream(ctx, stream, &s)) return st0;
    CU(ctx->mkept.ensure(1, nullptr));
    CU(cudaMemsetAsync(ctx->mkept.p, 0, sizeof(unsigned long long), s));
    MergeParams p{};
    p.x = ctx->cx;
    p.y = ctx->cy;
    p.peak_cap = res->peak_cap;
    p.pair_cap = res->pair_cap;
    p.kept = ctx->mkept.p;
    p.n_phi = ctx->grid.n_phi;
    p.n_d0 = ctx->grid.n_d0;
    p.n_kappa = ctx->grid.n_kappa;
    p.radius = radius;
    if (res->mem == HT_DEVICE) {
        p.peaks = res->peaks;
        p.po = res->peak_offsets;
        p.hidx = res->hit_idx;
        p.n_peaks = res->counts;
        p.cap = cap;
        p.fits = fits;
        p.state = state;
        CU(launch_merge(p, s));
        // the counter is unsigned 64-bit and n_kept int64: same bytes for any count
        CU(cudaMemcpyAsync(n_kept, ctx->mkept.p, sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
        return HT_OK;
    }
    // host results: the context still holds them on the device
    const int64_t n = std::min(std::min(res->counts[0], res->peak_cap), cap);
    *n_kept = 0;
    if (n <= 0) return HT_OK;
    CU(ctx->fits.ensure(n, &ctx->gen));
    CU(ctx->mstate.ensure(n, nullptr));
    CU(cudaMemcpyAsync(ctx->fits.p, fits, n * sizeof(ht_track), cudaMemcpyHostToDevice, s));
    p.peaks = ctx->peaks.p;
    p.po = ctx->peakoff.p;
    p.hidx = ctx->hitidx.p;
    p.n_peaks = ctx->d_scal + 6;
    p.cap = n;
    p.fits = ctx->fits.p;
    p.state = ctx->mstate.p;
    CU(launch_merge(p, s));
    CU(cudaMemcpyAsync(state, ctx->mstate.p, n * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    CU(cudaMemcpyAsync(ctx->h_pinned + 2, ctx->mkept.p, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    *n_kept = ctx->h_pinned[2];
    return HT_OK;
}

int ht_vertices(ht_ctx* ctx, const ht_vgrid* vg, const ht_results* res, uint32_t threshold, ht_vertex* out,
                int64_t cap, int64_t* count, void* stream) {
    if (!ctx || !vg || !res || !count || cap < 0 || (cap > 0 && !out)) return HT_ERR_INVALID_ARG;
    if (vg->n_x < 1 || vg->n_y < 1 || vg->n_x > 65535 || vg->n_y > 65535 || !std::isfinite(vg->x_min) ||
        !std::isfinite(vg->x_max) || !std::isfinite(vg->y_min) || !std::isfinite(vg->y_max) ||
        !(vg->x_max > vg->x_min) || !(vg->y_max > vg->y_min))
        return fail(ctx, HT_ERR_INVALID_ARG, "bad vertex grid");
    if (res->mem != HT_HOST && res->mem != HT_DEVICE) return fail(ctx, HT_ERR_INVALID_ARG, "res.mem must be HT_HOST or HT_DEVICE");
    if (!ctx->have_results) return fail(ctx, HT_ERR_STATE, "ht_vertices needs a preceding ht_process");
    cudaStream_t s = nullptr;
    if (int st0 = resolve_stream(ctx, stream, &s)) return st0;
    const int64_t ne = ctx->c_events;
    const int64_t cells = ne * vg->n_x * vg->n_y, rows = ne * vg->n_x;
    CU(ctx->vacc.ensure(std::max<int64_t>(cells, 1), nullptr));
    CU(ctx->vrow.ensure(std::max<int64_t>(rows, 1), nullptr));
    CU(ctx->vbase.ensure(rows + 1, nullptr));
    CU(ctx->vscal.ensure(2, nullptr));
    CU(cudaMemsetAsync(ctx->vacc.p, 0, std::max<int64_t>(cells, 1) * sizeof(uint32_t), s));
    CU(cudaMemsetAsync(ctx->vscal.p, 0, 2 * sizeof(int64_t), s));
    VertexParams p{};
    const bool dev = res->mem == HT_DEVICE;
    p.peaks = dev ? res->peaks : ctx->peaks.p;
    p.n_peaks = dev ? res->counts : ctx->d_scal + 6;
    p.peak_cap = res->peak_cap;
    p.n_events = (int32_t)ne;
    p.cphi = ctx->d_cphi;
    p.sphi = ctx->d_sphi;
    p.d0 = ctx->d_dtab;
    p.nx = vg->n_x;
    p.ny = vg->n_y;
    p.xmin = (double)vg->x_min;
    p.xmax = (double)vg->x_max;
    p.ymin = (double)vg->y_min;
    p.ymax = (double)vg->y_max;
    p.acc = ctx->vacc.p;
    p.thr = threshold;
    p.rowcnt = ctx->vrow.p;
    p.rowbase = ctx->vbase.p;
    p.cap = cap;
    if (dev) {
        p.out = out;
    } else {
        CU(ctx->vout.ensure(std::max<int64_t>(cap, 1), nullptr));
        p.out = ctx->vout.p;
    }
    if (p.peak_cap > 0 && (dev || res->counts[0] > 0)) CU(launch_vertex_vote(p, s));
    CU(launch_vertex_rows(p, false, s));
    ScanRange r{};
    r.in = ctx->vrow.p;
    r.out = ctx->vbase.p;
    r.lo = 0;
    r.hi = rows;
    r.cap = rows;
    r.base_dev = ctx->vscal.p + 0;
    r.total = ctx->vscal.p + 1;
    r.write_end = 1;
    CU(launch_scan(r, ctx->scratch.p, s));
    CU(launch_vertex_rows(p, true, s));
    if (dev) {
        CU(cudaMemcpyAsync(count, ctx->vscal.p + 1, sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
        return HT_OK;
    }
    CU(cudaMemcpyAsync(ctx->h_pinned + 2, ctx->vscal.p + 1, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    const int64_t total = ctx->h_pinned[2];
    *count = total;
    const int64_t ncopy = std::min(total, cap);
    if (ncopy > 0) {
        CU(cudaMemcpyAsync(out, ctx->vout.p, ncopy * sizeof(ht_vertex), cudaMemcpyDeviceToHost, s));
        CU(cudaStreamSynchronize(s));
    }
    if (total > cap) return fail(ctx, HT_ERR_OVERFLOW, "%lld vertices, cap %lld", (long long)total, (long long)cap);
    return HT_OK;
}

int ht_phase_times(ht_ctx* ctx, float* ms) {
    if (!ctx || !ms) return HT_ERR_INVALID_ARG;
    if (!ctx->timing) return fail(ctx, HT_ERR_STATE, "HT_OPT_PHASE_TIMING is off");
    for (int i = 0; i < 4; ++i) ms[i] = ctx->phase_ms[i];
    return HT_OK;
}

int ht_filter_stats(ht_ctx* ctx, int64_t* out, int32_t reset) {
    if (!ctx || !out) return HT_ERR_INVALID_ARG;
    unsigned long long v[4];
    CU(cudaDeviceSynchronize());
    CU(cudaMemcpy(v, ctx->d_stats, sizeof v, cudaMemcpyDeviceToHost));
    out[0] = (int64_t)v[0];
    out[1] = (int64_t)v[1];
    out[2] = (int64_t)v[2];
    if (reset) CU(cudaMemset(ctx->d_stats, 0, sizeof v));
    return HT_OK;
}

int ht_autotune(ht_ctx* ctx, const ht_hits* hits, void* stream) {
    if (!ctx) return HT_ERR_INVALID_ARG;
    cudaStream_t s = nullptr;
    if (int st0 = resolve_stream(ctx, stream, &s)) return st0;
    const int64_t budget_ev = ctx->budget / std::max<int64_t>(ctx->cells * 4, 1);
    if (hits && (int64_t)hits->n_events > budget_ev)
        return fail(ctx, HT_ERR_BUDGET, "autotune sample exceeds the accumulator budget");
    int st = stage_hits(ctx, hits, s);
    if (st) return st;
    ctx->stream = s;
    st = ensure_wave_buffers(ctx, ctx->c_events);
    if (st) return st;
    const int nk = ctx->grid.n_kappa, nd = ctx->grid.n_d0;
    const int save_p = ctx->tile_phi, save_d = ctx->tile_d, save_t = ctx->threads;
    std::vector<int> tds;
    for (int td : {nd, 128, 64, 32, 16, 8})
        if (td <= nd && std::find(tds.begin(), tds.end(), td) == tds.end()) tds.push_back(td);
    // With records, the tile also decides the association's items and record
    // size: time the whole step (vote, peaks, association; threshold 9,
    // window 1, the batch workload's reading) over the tiles that support
    // records, and keep the fastest.
    if (ctx->records && ctx->vote_mode == HT_VOTE_POINT && (ctx->prune & 1) && ctx->K.band_ok && nk <= 255) {
        DBuf<ht_peak> pk;
        DBuf<int64_t> po;
        DBuf<int32_t> hi;
        const int64_t pcap = std::min<int64_t>(ctx->cells * ctx->c_events / 8 + 1024, 1LL << 27);
        const int64_t qcap = std::min<int64_t>(pcap * 64, 1LL << 31);
        float rbest = 1e30f;
        int rp = 0, rd = 0, rt = 0, ri = ctx->vote_items;
        const int save_items = ctx->vote_items;
        if (pk.ensure(pcap, nullptr) == cudaSuccess && po.ensure(pcap + 1, nullptr) == cudaSuccess &&
            hi.ensure(qcap, nullptr) == cudaSuccess && ctx->paircnt.ensure(pcap, &ctx->gen) == cudaSuccess) {
            const bool timing = ctx->timing;
            const int32_t epw = events_per_wave(ctx, ctx->c_events);
            ctx->wave_marks = false;
            ctx->timing = true;
            for (int tp : {1, 2, 4, 8}) {
                if (tp > ctx->grid.n_phi) continue;
                for (int td : tds) {
                    if (!assoc_rec_supported(tp, td, nk)) continue;
                    const int smem = vote_smem_bytes(tp, td, nk, 256, 3);
                    if (smem > 200 * 1024) continue;
                    for (int cfg = 0; cfg < 4; ++cfg) {
                        const int thr = (cfg & 1) ? 256 : 128, items = cfg >> 1;
                        ctx->tile_phi = tp;
                        ctx->tile_d = td;
                        ctx->threads = thr;
                        ctx->vote_items = items;
                        if (resolve_tiles(ctx) || !ctx->r_rec) continue;
                        if (plan_waves(ctx, hits, ctx->mode == HT_MODE_PLAIN ? 1 : epw, s) || ensure_timing_events(ctx, (int)ctx->wave_start.size() - 1))
                            continue;
                        if (process_device(ctx, 9, 1, pk.p, pcap, po.p, hi.p, qcap, s)) continue;  // warm
                        float ms = 1e30f;
                        bool ok = true;
                        for (int rep = 0; rep < 3 && ok; ++rep) {
                            if (process_device(ctx, 9, 1, pk.p, pcap, po.p, hi.p, qcap, s)) {
                                ok = false;
                                break;
                            }
                            CU(cudaStreamSynchronize(s));
                            float m1 = 0;
                            const int nw = ctx->tev_waves;
                            if (nw < 1 ||
                                cudaEventElapsedTime(&m1, ctx->tev[0], ctx->tev[5 * (nw - 1) + 3]) != cudaSuccess) {
                                cudaGetLastError();
                                ok = false;
                                break;
                            }
                            ms = std::min(ms, m1);
                        }
                        if (!ok) continue;
                        if (ms < rbest) {
                            rbest = ms;
                            rp = tp;
                            rd = td;
                            rt = thr;
                            ri = items;
                        }
                    }
                }
            }
            ctx->timing = timing;
        }
        pk.release();
        po.release();
        hi.release();
        ctx->vote_items = save_items;
        if (rp) {
            ctx->tile_phi = rp;
            ctx->tile_d = rd;
            ctx->threads = rt;
            ctx->vote_items = ri;
            ctx->gvalid = false;
            ctx->have_votes = ctx->have_peaks = ctx->have_results = false;
            return resolve_tiles(ctx);
        }
    }
    cudaEvent_t e0, e1;
    CU(cudaEventCreate(&e0));
    CU(cudaEventCreate(&e1));
    float best = 1e30f;
    int bp = 0, bd = 0, bt = 0;
    ctx->use_rec = false;
    for (int tp : {1, 2, 4, 8}) {
        if (tp > ctx->grid.n_phi) continue;
        for (int td : tds) {
            const int smem = vote_smem_bytes(tp, td, nk, 256, ctx->r_variant);
            if (smem > 200 * 1024 || smem < 8 * 1024) continue;
            for (int thr : {128, 256}) {
                ctx->tile_phi = tp;
                ctx->tile_d = td;
                ctx->threads = thr;
                if (resolve_tiles(ctx)) continue;
                run_vote(ctx, 0, ctx->c_events, true, s);  // warm
                CU(cudaEventRecord(e0, s));
                for (int r = 0; r < 2; ++r) run_vote(ctx, 0, ctx->c_events, true, s);
                CU(cudaEventRecord(e1, s));
                CU(cudaEventSynchronize(e1));
                float ms = 0;
                CU(cudaEventElapsedTime(&ms, e0, e1));
                if (ms < best) {
                    best = ms;
                    bp = tp;
                    bd = td;
                    bt = thr;
                }
            }
        }
    }
    if (bp == 0) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        ctx->tile_phi = save_p;
        ctx->tile_d = save_d;
        ctx->threads = save_t;
        resolve_tiles(ctx);
        return fail(ctx, HT_ERR_INVALID_ARG, "no tile shape fits");
    }
    ctx->tile_phi = bp;
    ctx->tile_d = bd;
    ctx->threads = bt;
    st = resolve_tiles(ctx);
    if (st) return st;
    // association tile, timed on the peaks + association phase of one wave
    // (threshold 9, window 1: the batch workload's reading)
    {
        DBuf<ht_peak> pk;
        DBuf<int64_t> po;
        DBuf<int32_t> hi;
        const int64_t pcap = std::min<int64_t>(ctx->cells * ctx->c_events / 8 + 1024, 1LL << 27);
        const int64_t qcap = std::min<int64_t>(pcap * 64, 1LL << 31);
        if (pk.ensure(pcap, nullptr) == cudaSuccess && po.ensure(pcap + 1, nullptr) == cudaSuccess &&
            hi.ensure(qcap, nullptr) == cudaSuccess && ctx->paircnt.ensure(pcap, &ctx->gen) == cudaSuccess) {
            const int save_ap = ctx->atile_phi, save_ad = ctx->atile_d;
            float abest = 1e30f;
            int ap_best = 0, ad_best = 0;
            const int32_t epw = events_per_wave(ctx, ctx->c_events);
            ctx->wave_marks = false;  // no host copies here
            if (ensure_index(ctx)) ctx->use_index = false;
            for (int ap : {1, 2, 4, 8}) {
                if (ap > ctx->grid.n_phi) continue;
                for (int ad : {nd, 32, 16, 8}) {
                    if (ad > nd) continue;
                    ctx->atile_phi = ap;
                    ctx->atile_d = ad;
                    if (resolve_tiles(ctx)) continue;
                    if (ctx->a_tile_d != ad) continue;  // did not fit
                    const bool timing = ctx->timing;
                    if (ensure_timing_events(ctx, 1)) continue;
                    ctx->timing = true;
                    if (plan_waves(ctx, hits, ctx->mode == HT_MODE_PLAIN ? 1 : epw, s)) continue;
                    ctx->use_rec = false;  // this loop times the binning association
                    process_device(ctx, 9, 1, pk.p, pcap, po.p, hi.p, qcap, s);  // warm
                    process_device(ctx, 9, 1, pk.p, pcap, po.p, hi.p, qcap, s);
                    CU(cudaStreamSynchronize(s));
                    ctx->timing = timing;
                    float ms = 0;
                    if (cudaEventElapsedTime(&ms, ctx->tev[1], ctx->tev[2]) != cudaSuccess) {
                        cudaGetLastError();
                        continue;
                    }
                    if (ms < abest) {
                        abest = ms;
                        ap_best = ap;
                        ad_best = ad;
                    }
                }
            }
            ctx->atile_phi = ap_best ? ap_best : save_ap;
            ctx->atile_d = ap_best ? ad_best : save_ad;
        }
        pk.release();
        po.release();
        hi.release();
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->gvalid = false;
    ctx->have_votes = ctx->have_peaks = ctx->have_results = false;
    return resolve_tiles(ctx);
}

// Accuracy of rcp.approx.ftz.f32 over `count` consecutive float bit patterns
// starting at first_bits: out[0] = max |rcp(x) x - 1| * 2^40, out[1] = count.
int ht_check_rcp(uint32_t first_bits, uint32_t count, uint64_t* out) {
    ht_ctx* ctx = nullptr;
    if (!out) return HT_ERR_INVALID_ARG;
    unsigned long long* d = nullptr;
    CU(cudaMalloc(&d, 2 * sizeof(unsigned long long)));
    CU(cudaMemset(d, 0, 2 * sizeof(unsigned long long)));
    CU(launch_rcp_check(first_bits, count, d, nullptr));
    CU(cudaMemcpy(out, d, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost));
    CU(cudaFree(d));
    return HT_OK;
}

int ht_microbench(int32_t kind, int64_t iters, double* rate) {
    ht_ctx* ctx = nullptr;
    if (!rate || kind < HT_MB_FP32 || kind > HT_MB_FP64 || iters < 1) return HT_ERR_INVALID_ARG;
    int dev = 0, sms = 0;
    CU(cudaGetDevice(&dev));
    CU(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    float* sink = nullptr;
    CU(cudaMalloc(&sink, sizeof(float) * (size_t)sms * 8));
    float ms = 0.f;
    double ops = 0.0;
    const cudaError_t e = run_microbench(kind, iters, sms, sink, &ms, &ops);
    cudaFree(sink);
    CU(e);
    *rate = ms > 0.f ? ops / (ms * 1e-3) : 0.0;
    return HT_OK;
}

}  // extern "C"
