// ht_internal.h — kernel launch interface shared by the host API and the kernels.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

#include "../../include/ht.h"
#include "ht_kbin.cuh"

namespace ht {

struct VoteParams {
    const float* x;
    const float* y;
    const int32_t* offs;   // batch event offsets (n_events_batch + 1)
    int64_t n_hits;
    int32_t event0;        // first batch event of this wave
    int32_t n_events;      // events in this wave
    const int32_t* order;  // wave-local event order (LPT) or nullptr
    int32_t* queue;        // persistent work counter (zeroed) or nullptr: one item per block
    int32_t item0;         // first item (non-persistent launches)
    int32_t n_items;       // items = n_events * tiles_phi * tiles_d
    int32_t tiles_phi, tiles_d, tile_d;
    uint32_t* acc;         // wave accumulators [n_events][cells]
    int64_t cells;
    const float* cphi;
    const float* sphi;
    const float4* dtab;    // (d0_j, 2 d0_j, d0_j^2, d0_j * S2)
    const float* ecos;     // range voting: cos/sin of the phi0 edges m 2pi/n_phi
    const float* esin;
    const float4* edtab;   // range voting: the n_d0 + 1 d0 edges, as dtab
    KConsts K;
    unsigned long long* stats;
    // vote records (band vote only; nullptr: none).  For every hit whose d0
    // band meets a tile, the bins of the tile's cells, one byte each (255: no
    // vote), `rec_bytes` = tile_phi * tile_d bytes per record, columns outer,
    // phi rows inner; record of (wave event e, tile t, hit h) at
    // ((hb - whb) * tiles + t * n_e + (h - hb)) * rec_bytes, whb the wave's
    // first hit.  rbits: one bit per (tile, hit) marking the hits that have a
    // record, words of event e from (((hb - whb) >> 5) + e) * tiles + t * ceil(n_e / 32).
    uint8_t* rec;
    uint32_t* rbits;
    int32_t rec_bytes;
    int32_t* err;          // staged hit loads: bit 16 when a block copy did not complete
    int32_t narrow;        // band vote: bands of at most this many columns walk their own band (0: none)
};

struct PeakParams {
    const uint32_t* acc;
    int64_t cells;
    int32_t n_events;       // wave events
    int32_t event0;         // batch index of the wave's first event
    uint32_t thr;
    int32_t nphi, nd, nk, nkw;
    uint32_t* mask;         // [cols][nkw] peak bits
    uint16_t* wpre;         // [cols][nkw] peaks in earlier words of the column
    int32_t* npk;           // [cols]
    int64_t* colbase;       // [cols] first peak id of the column (global, includes earlier waves)
    ht_peak* peaks;
    int64_t peak_cap;
    int32_t window;         // < 0: no pair counts
    int32_t* paircnt;       // [peak_cap]
    int64_t* extra_pairs;   // pairs of peaks beyond peak_cap (device scalar) or nullptr
    int32_t line;           // 1: line voting's [phi][1][d0] view, emitted as (phi, d0, 0)
};

struct AssocParams {
    const float* x;
    const float* y;
    const int32_t* offs;
    int64_t n_hits;
    int32_t event0, n_events;
    const uint32_t* mask;
    const uint16_t* wpre;
    const int32_t* npk;
    const int64_t* colbase;
    const int64_t* peak_offsets;
    int64_t peak_cap;
    int32_t* hit_idx;
    int64_t pair_cap;
    int32_t window;
    int32_t band;           // 1: evaluate only the d0 columns inside some lane's band
    int32_t wd;             // d0 columns per item (tile_phi * wd <= 32; tile_phi > 1 needs wd == n_d0)
    int32_t cap;            // row cursors per warp
    size_t warp_bytes;      // shared memory per warp
    const int32_t* order;   // wave-local event order (largest first) or nullptr
    unsigned long long* queue;  // work counter, zeroed before the launch
    const float* ecos;      // range association: phi0 edges and d0 edges
    const float* esin;
    const float4* edtab;
    int32_t* paircnt;       // range counting pass: row lengths of stored peaks
    int64_t* extra_pairs;   // range counting pass: pairs of peaks past the cap (device scalar)
    int32_t line_nd;        // line voting (K holds the [phi][1][d0] view): n_d0, 0 otherwise
    double line_d0min, line_d0max;
    const float* cphi;
    const float* sphi;
    const float4* dtab;
    KConsts K;
    unsigned long long* stats;
    // association over vote records (items are the vote's tiles)
    const uint8_t* rec;
    const uint32_t* rbits;
    int32_t rec_bytes;      // tile_phi * tile_d
    int32_t rtiles_phi, rtiles_d, rtile_d;
};

// Exclusive scan of int32 counts over [lo, hi) (clamped to cap) into int64
// outputs: out[i] = base + sum(in[lo..i)), out[hi] = total, *total = base + sum.
// lo/hi/base come from device scalars when the pointers are non-null.
struct ScanRange {
    const int32_t* in;
    int64_t* out;
    const int64_t* lo_dev;
    const int64_t* hi_dev;
    const int64_t* base_dev;
    int64_t lo, hi, base, cap;
    int64_t* total;        // device scalar or nullptr
    int32_t write_end;     // 1: also write out[hi] = total
};

constexpr int kScanBlocks = 304;
constexpr int kScanThreads = 1024;

// vote kernel variants: 0 full sweep, 1 d0-band compaction (hull of queued
// hits), 2 range voting, 3 = 1 writing vote records, 4 d0 bands as
// (hit, column) items, 5 = 4 writing vote records, 6 = 1 and 7 = 3 with the
// hits staged into shared memory by bulk copies
int vote_smem_bytes(int tile_phi, int tile_d, int nk, int threads, int variant);
cudaError_t vote_prepare(int tile_phi, int nk, int smem_bytes, int variant);
cudaError_t vote_occupancy(int tile_phi, int nk, int threads, int smem, int* blocks, int variant);
cudaError_t launch_finalize(int64_t* scal, cudaStream_t s);
cudaError_t launch_publish(const int64_t* scal, int64_t* host, cudaStream_t s);
// dst: device address of page-locked host memory
cudaError_t launch_host_copy(void* dst, const void* src, size_t bytes, int blocks, cudaStream_t s);
cudaError_t launch_vote(int tile_phi, const VoteParams& p, int grid, int threads, int smem, cudaStream_t s,
                        int variant);
cudaError_t launch_validate(const float* x, const float* y, const int8_t* layer, int64_t n_hits,
                            const int32_t* offs, int32_t n_events, int32_t n_layers, int32_t* err,
                            cudaStream_t s);
cudaError_t launch_order(const int32_t* offs, int32_t event0, int32_t n_events, int64_t n_hits,
                         int32_t* order, cudaStream_t s);
cudaError_t launch_detect(const PeakParams& p, cudaStream_t s);
cudaError_t launch_emit(const PeakParams& p, cudaStream_t s);
cudaError_t launch_paircount(const PeakParams& p, const int64_t* lo_dev, const int64_t* hi_dev,
                             cudaStream_t s);
cudaError_t launch_scan(const ScanRange& r, int64_t* scratch /* 2 * kScanBlocks */, cudaStream_t s);
size_t assoc_warp_smem(int rows, int wd, int nk, int cap);
cudaError_t assoc_prepare(int tile_phi, int nk, int smem, bool band, int threads, int* blocks_per_sm);
cudaError_t launch_assoc(const AssocParams& p, int tile_phi, int threads, int grid, cudaStream_t s);
size_t assoc_range_warp_smem(int wd, int nk, int cap);
cudaError_t assoc_range_prepare(int nk, int smem, int threads, int* blocks_per_sm, bool line = false);
cudaError_t launch_vote_line(const VoteParams& p, double d0min, double d0max, cudaStream_t s);
cudaError_t launch_assoc_range(const AssocParams& p, bool count, int threads, int grid, cudaStream_t s);
// association over vote records (ht_assoc_rec.cu): one warp per vote tile of
// an event, lanes own the tile's cells
bool assoc_rec_supported(int tile_phi, int tile_d, int nk);
size_t assoc_rec_warp_smem(int tile_phi, int tile_d, int nk, int cap);
cudaError_t assoc_rec_prepare(int tile_phi, int tile_d, int nk, int smem, int threads, int* blocks_per_sm);
cudaError_t launch_assoc_rec(const AssocParams& p, int tile_phi, int threads, int grid, cudaStream_t s);
// circle fit of the stored candidates' rows (ht_fit.cu)
struct FitParams {
    const float* x;
    const float* y;
    const ht_peak* peaks;
    const int64_t* po;       // CSR offsets [peak_cap + 1]
    const int32_t* hidx;
    const int64_t* n_peaks;  // device scalar: the true peak count
    int64_t peak_cap, pair_cap, cap;
    ht_track* out;
    double kmin, kmax;
    int32_t nk;
};
cudaError_t launch_fit(const FitParams& p, cudaStream_t s);
// association through a per-(event, layer) angular index (ht_assoc_index.cu)
struct IndexParams {
    const float* x;
    const float* y;
    const int8_t* layer;
    const int32_t* offs;
    int32_t n_events, nl;
    int32_t* bcount;      // [n_events * nl]
    int64_t* bstart;      // [n_events * nl + 1]
    int32_t* bcursor;     // [n_events * nl]
    uint32_t* r2min;      // [n_events * nl] float bits
    uint32_t* r2max;
    float* theta;         // [n_hits] bucket order, sorted by angle within a bucket
    int32_t* hid;         // [n_hits]
    int32_t* tab;         // [n_events * nl][257] coarse angle table (positions within the bucket)
    int64_t* scratch;     // scan scratch
};
cudaError_t launch_index_build(const IndexParams& p, cudaStream_t s);
struct AssocIndexParams {
    AssocParams a;            // hits, offsets, rows, caps, window, tables, K, stats
    const ht_peak* peaks;
    const int64_t* lo_dev;    // the wave's peaks: [*lo_dev, min(*hi_dev, peak_cap))
    const int64_t* hi_dev;
    const float* theta;
    const int32_t* hid;
    const int32_t* tab;
    const int64_t* bstart;
    const uint32_t* r2min;
    const uint32_t* r2max;
    int32_t nl;
    float kmin, dk;           // kappa range start and bin width (float)
    int32_t* err;             // bit 8: a row came out with another length
};
cudaError_t launch_assoc_index(const AssocIndexParams& p, cudaStream_t s);
// duplicate and mirror merging of fitted candidates (ht_merge.cu)
struct MergeParams {
    const float* x;
    const float* y;
    const ht_peak* peaks;     // sorted by (event, linear index)
    const int64_t* po;
    const int32_t* hidx;
    const int64_t* n_peaks;   // device scalar: the true peak count
    int64_t peak_cap, pair_cap, cap;
    const ht_track* fits;
    int32_t* state;
    unsigned long long* kept; // device counter, zeroed by the caller
    int32_t n_phi, n_d0, n_kappa, radius;
};
cudaError_t launch_merge(const MergeParams& p, cudaStream_t s);
// second Hough transform for displaced vertices (ht_vertex.cu)
struct VertexParams {
    const ht_peak* peaks;
    const int64_t* n_peaks;   // device scalar: the true peak count
    int64_t peak_cap;
    int32_t n_events;
    const float* cphi;
    const float* sphi;
    const float4* d0;         // the first grid's d0 table (x = d0_j)
    int32_t nx, ny;
    double xmin, xmax, ymin, ymax;
    uint32_t* acc;            // [n_events][nx][ny]
    uint32_t thr;
    int32_t* rowcnt;          // [n_events * nx] vertices per x row
    const int64_t* rowbase;   // [n_events * nx] first output slot of each row
    ht_vertex* out;
    int64_t cap;
};
cudaError_t launch_vertex_vote(const VertexParams& p, cudaStream_t s);
cudaError_t launch_vertex_rows(const VertexParams& p, bool emit, cudaStream_t s);
cudaError_t launch_rcp_check(uint32_t first_bits, uint32_t count, unsigned long long* out, cudaStream_t s);
// throughput microbenchmarks (ht_microbench.cu): kind 0 FP32 mul/add, 1 shared reductions, 2 FP32 IEEE
// division, 3 binary64 mul/add
cudaError_t run_microbench(int kind, int64_t iters, int sms, float* sink, float* ms, double* ops);

}  // namespace ht
