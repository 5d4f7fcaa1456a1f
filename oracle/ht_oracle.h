/*
 * CPU oracle for the Hough-transform track finder — TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded C statement of what the GPU library computes,
 * used by the tests, the smoke check and the CPU-baseline leg of the bench to
 * judge the CUDA path.  It shares no code, header, table or constant with the
 * library (include/ht.h, paper_1311_2769_gb300/csrc) and neither links the
 * other.  Nothing on the product path may call it.
 *
 * Method (Lujan et al., "GPU Enhancement of the Trigger to Extend Physics Reach
 * at the LHC", Section 3): every parameter instance starts with zero votes;
 * each hit adds one vote to every instance that contains it; local maxima of
 * the vote array are track candidates.  The instances are the cells of a
 * (phi0, d0, kappa) perigee-helix grid — the curved, displaced 3-parameter
 * model Section 3 calls for — whose two 2-parameter special cases (d0 = 0:
 * curved tracks through the origin; kappa = 0: straight displaced tracks) are
 * the models the paper's own implementation used.
 *
 * Precision: the curvature bin of a (hit, phi0, d0) column is defined by one
 * fixed sequence of IEEE-754 binary64 operations on the float32 hit
 * coordinates and float32 bin-centre tables (see ht_oracle.c); compile with
 * -ffp-contract=off so no FMA is formed.
 */
#ifndef HT_ORACLE_H
#define HT_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int32_t n_phi, n_d0, n_kappa;
    float d0_min, d0_max, kappa_min, kappa_max;
} hto_grid;

typedef struct {
    int32_t event, i_phi, i_d0, i_kappa;
    uint32_t votes;
} hto_peak;

/* Bin-centre tables: cos/sin of phi_i = (i + 1/2) 2pi / n_phi and
 * d0_j = d0_min + (j + 1/2)(d0_max - d0_min)/n_d0, each rounded to float once. */
void hto_tables(const hto_grid *g, float *cos_phi, float *sin_phi, float *d0);

/* Curvature bin of hit (x, y) in column (i, j) by the binary64 definition;
 * -1 when the hit casts no vote in that column. */
int32_t hto_kbin(const hto_grid *g, float x, float y, int32_t i, int32_t j);

/* Same, but with the column's table values given directly. */
int32_t hto_kbin_at(const hto_grid *g, float x, float y, float c, float s, float d);

/* The binary64 value w = (kappa - kappa_min) * n_kappa / (kappa_max - kappa_min)
 * for (hit, column), or NaN when den <= 0 (used by the filter-bound tests). */
double hto_w64(const hto_grid *g, float x, float y, float c, float s, float d);

/* hto_kbin_at for n independent cells (plain loop; used by tests). */
void hto_kbin_cells(const hto_grid *g, int64_t n, const float *x, const float *y, const float *c,
                    const float *s, const float *d, int32_t *out);

/* Plain float32 op-order bin coordinate w (IEEE division, no contraction),
 * NaN when den <= 0, and its bin (-1 when out of range): the form whose
 * disagreement with hto_kbin is reported as the flip fraction. */
float hto_w32(const hto_grid *g, float x, float y, float c, float s, float d);
int32_t hto_kbin_fp32(const hto_grid *g, float x, float y, float c, float s, float d);

/* Vote every event: acc is [n_events][n_phi][n_d0][n_kappa] uint32, zeroed here. */
void hto_vote(const hto_grid *g, const float *x, const float *y,
              const int32_t *event_offsets, int32_t n_events, uint32_t *acc);

/* One (phi, d0) column of one event: out[n_kappa], zeroed here. */
void hto_vote_column(const hto_grid *g, const float *x, const float *y, int64_t n_hits,
                     int32_t i, int32_t j, uint32_t *out);

/* Local maxima at or above threshold, ascending (event, linear index).
 * Returns the number of peaks found (may exceed cap; only cap are written). */
int64_t hto_peaks(const hto_grid *g, const uint32_t *acc, int32_t n_events,
                  uint32_t threshold, hto_peak *out, int64_t cap);

/* Is cell (i, j, k) of one event's accumulator a peak? */
int32_t hto_is_peak(const hto_grid *g, const uint32_t *acc1, uint32_t threshold,
                    int32_t i, int32_t j, int32_t k);

/* Hit-to-candidate association (CSR).  peak_offsets has n_peaks + 1 entries;
 * hit_idx receives global hit indices, ascending within each peak.  Returns
 * the number of pairs (may exceed cap; only cap are written). */
int64_t hto_associate(const hto_grid *g, const float *x, const float *y,
                      const int32_t *event_offsets, const hto_peak *peaks, int64_t n_peaks,
                      int32_t window, int64_t *peak_offsets, int32_t *hit_idx, int64_t cap);

/* Flip metric over all (hit, column) pairs of the given events:
 * out[0] = binary64 votes, out[1] = float32 votes, out[2] = columns whose
 * bins differ (a vote in one form and none, or another bin, in the other). */
void hto_flip_count(const hto_grid *g, const float *x, const float *y,
                    const int32_t *event_offsets, int32_t n_events, int64_t *out);

/* Whole path per event (vote, peaks, associate) on n_threads host threads,
 * one event at a time per thread (largest first from a shared counter),
 * results reduced to counts:
 * out[0] = votes cast, out[1] = peaks, out[2] = pairs.  Used to time the
 * oracle as a CPU baseline. */
void hto_run_events(const hto_grid *g, const float *x, const float *y,
                    const int32_t *event_offsets, int32_t n_events,
                    uint32_t threshold, int32_t window, int32_t n_threads, int64_t *out);

/* ---- range voting ----------------------------------------------------------
 * A hit votes, in cell (i, j), for every kappa bin from the lowest to the
 * highest bin of its curve at the cell's four corners (phi0 edges
 * m 2pi/n_phi, periodic; d0 edges d0_min + n (d0_max - d0_min)/n_d0), clipped
 * to [0, n_kappa); no vote if a corner has den <= 0. */
#define HTO_UNDEF (-2)

/* Edge tables: cos_e/sin_e[n_phi], d_e[n_d0 + 1]. */
void hto_edges(const hto_grid *g, float *cos_e, float *sin_e, float *d_e);

/* Corner code: HTO_UNDEF (den <= 0), -1 (below), n_kappa (above) or the bin. */
int32_t hto_code_at(const hto_grid *g, float x, float y, float c, float s, float d);
void hto_code_cells(const hto_grid *g, int64_t n, const float *x, const float *y, const float *c,
                    const float *s, const float *d, int32_t *out);

/* Bins [*lo, *hi] of hit (x, y) in cell (i, j); returns 0 when none. */
int32_t hto_range(const hto_grid *g, float x, float y, int32_t i, int32_t j, int32_t *lo, int32_t *hi);

/* Range vote of every event (acc as for hto_vote). */
void hto_vote_range(const hto_grid *g, const float *x, const float *y,
                    const int32_t *event_offsets, int32_t n_events, uint32_t *acc);

/* Range association: hit h joins peak (i, j, k) when its bins in column
 * (i, j) reach within `window` of k.  CSR as hto_associate. */
int64_t hto_associate_range(const hto_grid *g, const float *x, const float *y,
                            const int32_t *event_offsets, const hto_peak *peaks, int64_t n_peaks,
                            int32_t window, int64_t *peak_offsets, int32_t *hit_idx, int64_t cap);

/* ---- circle fit ----------------------------------------------------------
 * Algebraic least-squares circle through a candidate's hits (binary64, sums
 * in row order, Cramer's rule), as perigee parameters with the turning sign
 * of the peak's kappa bin centre.  status 1 fitted, 0 not (< 3 hits, singular
 * system, R^2 <= 0, centre at the origin). */
typedef struct {
    int32_t status, n_hits;
    double cos_phi0, sin_phi0, d0, kappa, chi2;
} hto_track;

void hto_fit_row(const hto_grid *g, const float *x, const float *y, const int32_t *idx, int64_t n,
                 int32_t i_kappa, hto_track *out);
void hto_fit(const hto_grid *g, const float *x, const float *y, const hto_peak *peaks, int64_t n_peaks,
             const int64_t *peak_offsets, const int32_t *hit_idx, hto_track *out);

/* ---- second Hough transform: displaced vertices --------------------------
 * Every candidate votes along its line y cos(phi_i) - x sin(phi_i) = d0_j in
 * an (x, y) grid, walking the less steep axis (binary64); vertices are the
 * 2-D local maxima at or above a threshold (linear-order tie rule,
 * 8-neighbourhood, no wrap). */
typedef struct {
    int32_t n_x, n_y;
    float x_min, x_max, y_min, y_max;
} hto_vgrid;

typedef struct {
    int32_t event, i_x, i_y;
    uint32_t votes;
} hto_vertex;

/* acc is [n_events][n_x][n_y] uint32, zeroed here; peaks of events outside
 * [0, n_events) are ignored. */
void hto_vertex_vote(const hto_grid *g, const hto_vgrid *v, const hto_peak *peaks, int64_t n_peaks,
                     int32_t n_events, uint32_t *acc);
int64_t hto_vertex_peaks(const hto_vgrid *v, const uint32_t *acc, int32_t n_events, uint32_t threshold,
                         hto_vertex *out, int64_t cap);

/* ---- straight displaced tracks (kappa = 0) --------------------------------
 * On a grid with n_kappa = 1, each hit votes in every phi0 row for the d0 bin
 * of q = y cos phi0 - x sin phi0 (binary64); it joins peak (i, j, 0) when its
 * d0 bin in row i lies within `window` of j. */
int32_t hto_line_bin(const hto_grid *g, float x, float y, int32_t i);
void hto_vote_line(const hto_grid *g, const float *x, const float *y, const int32_t *event_offsets,
                   int32_t n_events, uint32_t *acc);
int64_t hto_associate_line(const hto_grid *g, const float *x, const float *y, const int32_t *event_offsets,
                           const hto_peak *peaks, int64_t n_peaks, int32_t window, int64_t *peak_offsets,
                           int32_t *hit_idx, int64_t cap);

/* ---- duplicate and mirror merging ----------------------------------------
 * After the fit: UNFITTED (status != 1); BACKWARD (the row's hits do not lie
 * ahead of the perigee: the binary64 sum of x cos phi0 + y sin phi0 is not
 * > 0); DUPLICATE when a better (more votes, then smaller index) forward
 * fitted candidate of the same event lies within `radius` cells in each of
 * phi0 (periodic), d0, kappa; else KEPT.  Returns the number kept. */
#define HTO_MERGE_KEPT 1
#define HTO_MERGE_DUPLICATE 0
#define HTO_MERGE_BACKWARD (-1)
#define HTO_MERGE_UNFITTED (-2)
int64_t hto_merge(const hto_grid *g, const float *x, const float *y, const hto_peak *peaks, int64_t n_peaks,
                  const int64_t *peak_offsets, const int32_t *hit_idx, const hto_track *fits,
                  int32_t radius, int32_t *state);

#ifdef __cplusplus
}
#endif
#endif
