/*
 * CPU oracle for the Hough-transform track finder — TEST INFRASTRUCTURE ONLY.
 * Only tests/, the smoke check and the bench's CPU-baseline leg use it; it
 * shares nothing with the GPU library.  Build with
 *   gcc -O2 -ffp-contract=off -fno-fast-math -fPIC -shared -pthread
 * (-ffp-contract=off matters: gcc on aarch64 would otherwise fuse a*b+c).
 *
 * Paper: Lujan et al., "GPU Enhancement of the Trigger to Extend Physics Reach
 * at the LHC" (arXiv:1311.2769).  Section 3 defines the Hough transform used
 * here: zero votes everywhere, one vote per (datum, containing instance),
 * local maxima = features, then hits are attached to the features found.
 */
#include "ht_oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

static const double kPi = 3.14159265358979323846;

/* Bin centres (Section 3: the parameter space is a grid of feature
 * instances; each instance is represented by its cell centre). */
void hto_tables(const hto_grid *g, float *cos_phi, float *sin_phi, float *d0)
{
    for (int32_t i = 0; i < g->n_phi; ++i) {
        double phi = ((double)i + 0.5) * (2.0 * kPi / (double)g->n_phi);
        cos_phi[i] = (float)cos(phi);
        sin_phi[i] = (float)sin(phi);
    }
    for (int32_t j = 0; j < g->n_d0; ++j) {
        double w = ((double)g->d0_max - (double)g->d0_min) / (double)g->n_d0;
        d0[j] = (float)((double)g->d0_min + ((double)j + 0.5) * w);
    }
}

/*
 * Track model (Section 3 asks for curved, displaced tracks, i.e. three
 * parameters): the circle with perigee d0 n, n = (-sin phi0, cos phi0),
 * tangent t = (cos phi0, sin phi0) and signed curvature kappa.  Requiring the
 * hit h to lie on it gives
 *     kappa = 2 (q - d0) / (r^2 + d0^2 - 2 d0 q),   q = h . n = y cos phi0 - x sin phi0,
 * whose denominator is |h - P|^2.  The bin coordinate is
 *     w = (kappa - kappa_min) * n_kappa / (kappa_max - kappa_min),
 * and the hit votes into bin floor(w) when den > 0 and 0 <= w < n_kappa.
 * Every operation below is one binary64 IEEE operation in this order.
 */
double hto_w64(const hto_grid *g, float xf, float yf, float cf, float sf, float df)
{
    double x = xf, y = yf, c = cf, s = sf, d = df;
    double q = (y * c) - (x * s);
    double a = q - d;
    double den = (((x * x) + (y * y)) + (d * d)) - ((2.0 * d) * q);
    if (!(den > 0.0))
        return NAN;
    double kappa = (2.0 * a) / den;
    double scale = (double)g->n_kappa / ((double)g->kappa_max - (double)g->kappa_min);
    return (kappa - (double)g->kappa_min) * scale;
}

int32_t hto_kbin_at(const hto_grid *g, float x, float y, float c, float s, float d)
{
    double w = hto_w64(g, x, y, c, s, d);
    if (!(w >= 0.0 && w < (double)g->n_kappa))
        return -1;
    return (int32_t)w;
}

void hto_kbin_cells(const hto_grid *g, int64_t n, const float *x, const float *y, const float *c,
                    const float *s, const float *d, int32_t *out)
{
    for (int64_t t = 0; t < n; ++t)
        out[t] = hto_kbin_at(g, x[t], y[t], c[t], s[t], d[t]);
}

/* Bin centre tables are rebuilt per call: slow and plain on purpose. */
int32_t hto_kbin(const hto_grid *g, float x, float y, int32_t i, int32_t j)
{
    double phi = ((double)i + 0.5) * (2.0 * kPi / (double)g->n_phi);
    double w = ((double)g->d0_max - (double)g->d0_min) / (double)g->n_d0;
    float d = (float)((double)g->d0_min + ((double)j + 0.5) * w);
    return hto_kbin_at(g, x, y, (float)cos(phi), (float)sin(phi), d);
}

/* The same formula with float32 operations in a fixed order (IEEE division,
 * no contraction).  Not part of the method's definition: it is the form whose
 * bins are compared against the binary64 ones to report the flip fraction.
 * Returns the float32 bin coordinate w, or NaN when den <= 0. */
float hto_w32(const hto_grid *g, float x, float y, float c, float s, float d)
{
    double scale = (double)g->n_kappa / ((double)g->kappa_max - (double)g->kappa_min);
    float S2 = (float)(2.0 * scale);
    float H = (float)(-(double)g->kappa_min * scale);
    float r2 = (x * x) + (y * y);
    float q = (y * c) - (x * s);
    float a = q - d;
    float n = a * S2;
    float den = (r2 + (d * d)) - ((d + d) * q);
    if (!(den > 0.0f))
        return NAN;
    float v = n / den;
    return v + H;
}

int32_t hto_kbin_fp32(const hto_grid *g, float x, float y, float c, float s, float d)
{
    float wv = hto_w32(g, x, y, c, s, d);
    if (!(wv >= 0.0f && wv < (float)g->n_kappa))
        return -1;
    return (int32_t)wv;
}

/* Section 3 voting: every hit adds one vote to each instance containing it. */
static void vote_event(const hto_grid *g, const float *cphi, const float *sphi, const float *d0,
                       const float *x, const float *y, int64_t n_hits, uint32_t *acc1)
{
    const int64_t nd = g->n_d0, nk = g->n_kappa;
    memset(acc1, 0, sizeof(uint32_t) * (size_t)g->n_phi * (size_t)nd * (size_t)nk);
    for (int64_t h = 0; h < n_hits; ++h)
        for (int32_t i = 0; i < g->n_phi; ++i)
            for (int32_t j = 0; j < g->n_d0; ++j) {
                int32_t k = hto_kbin_at(g, x[h], y[h], cphi[i], sphi[i], d0[j]);
                if (k >= 0)
                    acc1[((int64_t)i * nd + j) * nk + k] += 1u;
            }
}

static void tables_alloc(const hto_grid *g, float **c, float **s, float **d)
{
    *c = (float *)malloc(sizeof(float) * (size_t)g->n_phi);
    *s = (float *)malloc(sizeof(float) * (size_t)g->n_phi);
    *d = (float *)malloc(sizeof(float) * (size_t)g->n_d0);
    hto_tables(g, *c, *s, *d);
}

void hto_vote(const hto_grid *g, const float *x, const float *y,
              const int32_t *event_offsets, int32_t n_events, uint32_t *acc)
{
    float *c, *s, *d;
    tables_alloc(g, &c, &s, &d);
    const int64_t cells = (int64_t)g->n_phi * g->n_d0 * g->n_kappa;
    for (int32_t e = 0; e < n_events; ++e) {
        int64_t lo = event_offsets[e], hi = event_offsets[e + 1];
        vote_event(g, c, s, d, x + lo, y + lo, hi - lo, acc + (int64_t)e * cells);
    }
    free(c); free(s); free(d);
}

void hto_vote_column(const hto_grid *g, const float *x, const float *y, int64_t n_hits,
                     int32_t i, int32_t j, uint32_t *out)
{
    float *c, *s, *d;
    tables_alloc(g, &c, &s, &d);
    memset(out, 0, sizeof(uint32_t) * (size_t)g->n_kappa);
    for (int64_t h = 0; h < n_hits; ++h) {
        int32_t k = hto_kbin_at(g, x[h], y[h], c[i], s[i], d[j]);
        if (k >= 0)
            out[k] += 1u;
    }
    free(c); free(s); free(d);
}

/*
 * Section 3: "local maxima in the parameter space".  A cell at or above the
 * threshold is a peak when it is strictly greater than every neighbour that
 * precedes it in linear (phi, d0, kappa) order and at least as large as every
 * neighbour that follows it.  Neighbours are the distinct cells other than
 * itself at offsets {-1, 0, 1}^3; phi0 is periodic, d0 and kappa are not.
 */
int32_t hto_is_peak(const hto_grid *g, const uint32_t *acc1, uint32_t threshold,
                    int32_t i, int32_t j, int32_t k)
{
    const int64_t nd = g->n_d0, nk = g->n_kappa;
    const int64_t self = ((int64_t)i * nd + j) * nk + k;
    const uint32_t v = acc1[self];
    if (v < threshold)
        return 0;
    for (int di = -1; di <= 1; ++di)
        for (int dj = -1; dj <= 1; ++dj)
            for (int dk = -1; dk <= 1; ++dk) {
                int32_t ii = ((i + di) % g->n_phi + g->n_phi) % g->n_phi;
                int32_t jj = j + dj, kk = k + dk;
                if (jj < 0 || jj >= g->n_d0 || kk < 0 || kk >= g->n_kappa)
                    continue;
                int64_t other = ((int64_t)ii * nd + jj) * nk + kk;
                if (other == self)
                    continue;
                uint32_t u = acc1[other];
                if (other < self ? !(v > u) : !(v >= u))
                    return 0;
            }
    return 1;
}

int64_t hto_peaks(const hto_grid *g, const uint32_t *acc, int32_t n_events,
                  uint32_t threshold, hto_peak *out, int64_t cap)
{
    const int64_t cells = (int64_t)g->n_phi * g->n_d0 * g->n_kappa;
    int64_t n = 0;
    for (int32_t e = 0; e < n_events; ++e) {
        const uint32_t *a1 = acc + (int64_t)e * cells;
        for (int32_t i = 0; i < g->n_phi; ++i)
            for (int32_t j = 0; j < g->n_d0; ++j)
                for (int32_t k = 0; k < g->n_kappa; ++k)
                    if (hto_is_peak(g, a1, threshold, i, j, k)) {
                        if (n < cap) {
                            hto_peak p = {e, i, j, k, a1[((int64_t)i * g->n_d0 + j) * g->n_kappa + k]};
                            out[n] = p;
                        }
                        ++n;
                    }
    }
    return n;
}

/*
 * Hits of a candidate (Section 3: the maxima become reconstructed tracks,
 * which a confirmation fit then uses): hit h of the peak's event belongs to
 * peak (i, j, k) when it votes in column (i, j) and its bin lies within
 * `window` bins of k.
 */
int64_t hto_associate(const hto_grid *g, const float *x, const float *y,
                      const int32_t *event_offsets, const hto_peak *peaks, int64_t n_peaks,
                      int32_t window, int64_t *peak_offsets, int32_t *hit_idx, int64_t cap)
{
    float *c, *s, *d;
    tables_alloc(g, &c, &s, &d);
    int64_t n = 0;
    peak_offsets[0] = 0;
    for (int64_t p = 0; p < n_peaks; ++p) {
        const hto_peak *pk = &peaks[p];
        int64_t lo = event_offsets[pk->event], hi = event_offsets[pk->event + 1];
        for (int64_t h = lo; h < hi; ++h) {
            int32_t kb = hto_kbin_at(g, x[h], y[h], c[pk->i_phi], s[pk->i_phi], d[pk->i_d0]);
            if (kb >= 0 && abs(kb - pk->i_kappa) <= window) {
                if (n < cap)
                    hit_idx[n] = (int32_t)h;
                ++n;
            }
        }
        peak_offsets[p + 1] = n;
    }
    free(c); free(s); free(d);
    return n;
}

void hto_flip_count(const hto_grid *g, const float *x, const float *y,
                    const int32_t *event_offsets, int32_t n_events, int64_t *out)
{
    float *c, *s, *d;
    tables_alloc(g, &c, &s, &d);
    int64_t v64 = 0, v32 = 0, diff = 0;
    for (int64_t h = event_offsets[0]; h < event_offsets[n_events]; ++h)
        for (int32_t i = 0; i < g->n_phi; ++i)
            for (int32_t j = 0; j < g->n_d0; ++j) {
                int32_t k64 = hto_kbin_at(g, x[h], y[h], c[i], s[i], d[j]);
                int32_t k32 = hto_kbin_fp32(g, x[h], y[h], c[i], s[i], d[j]);
                v64 += k64 >= 0;
                v32 += k32 >= 0;
                diff += k64 != k32;
            }
    out[0] = v64; out[1] = v32; out[2] = diff;
    free(c); free(s); free(d);
}

/* ---- event-parallel harness (timing only; the per-event work is the plain code above) ---- */

typedef struct {
    const hto_grid *g;
    const float *x, *y;
    const int32_t *offs;
    const int32_t *order;   /* events in the order they are handed out */
    int32_t n_events;
    int32_t *next;          /* shared position in `order` */
    uint32_t threshold;
    int32_t window;
    int64_t votes, peaks, pairs;
} run_arg;

static void *run_worker(void *p)
{
    run_arg *a = (run_arg *)p;
    const hto_grid *g = a->g;
    const int64_t cells = (int64_t)g->n_phi * g->n_d0 * g->n_kappa;
    uint32_t *acc1 = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)cells);
    int64_t pcap = 1 << 16;
    hto_peak *pk = (hto_peak *)malloc(sizeof(hto_peak) * (size_t)pcap);
    for (;;) {
        int32_t t = __atomic_fetch_add(a->next, 1, __ATOMIC_RELAXED);
        if (t >= a->n_events)
            break;
        int32_t e = a->order[t];
        int64_t lo = a->offs[e], hi = a->offs[e + 1];
        int32_t offs1[2] = {0, (int32_t)(hi - lo)};
        hto_vote(g, a->x + lo, a->y + lo, offs1, 1, acc1);
        for (int64_t c = 0; c < cells; ++c)
            a->votes += acc1[c];
        int64_t np = hto_peaks(g, acc1, 1, a->threshold, pk, pcap);
        if (np > pcap) {
            pcap = np;
            pk = (hto_peak *)realloc(pk, sizeof(hto_peak) * (size_t)pcap);
            np = hto_peaks(g, acc1, 1, a->threshold, pk, pcap);
        }
        a->peaks += np;
        int64_t *po = (int64_t *)malloc(sizeof(int64_t) * (size_t)(np + 1));
        a->pairs += hto_associate(g, a->x + lo, a->y + lo, offs1, pk, np, a->window, po, NULL, 0);
        free(po);
    }
    free(pk);
    free(acc1);
    return NULL;
}

/* Events are handed out one at a time from a shared counter, largest event
 * first (ties by index), so the threads finish together; the per-event work
 * is the plain single-threaded code above. */
void hto_run_events(const hto_grid *g, const float *x, const float *y,
                    const int32_t *event_offsets, int32_t n_events,
                    uint32_t threshold, int32_t window, int32_t n_threads, int64_t *out)
{
    if (n_threads < 1)
        n_threads = 1;
    int32_t *order = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n_events > 0 ? n_events : 1));
    for (int32_t e = 0; e < n_events; ++e) {
        /* insertion by size, descending (plain; n_events is small) */
        int32_t t = e;
        int64_t n = (int64_t)event_offsets[e + 1] - event_offsets[e];
        while (t > 0) {
            int32_t o = order[t - 1];
            int64_t no = (int64_t)event_offsets[o + 1] - event_offsets[o];
            if (no >= n)
                break;
            order[t] = o;
            --t;
        }
        order[t] = e;
    }
    int32_t next = 0;
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)n_threads);
    run_arg *args = (run_arg *)calloc((size_t)n_threads, sizeof(run_arg));
    for (int32_t t = 0; t < n_threads; ++t) {
        run_arg a = {g, x, y, event_offsets, order, n_events, &next, threshold, window, 0, 0, 0};
        args[t] = a;
        pthread_create(&th[t], NULL, run_worker, &args[t]);
    }
    out[0] = out[1] = out[2] = 0;
    for (int32_t t = 0; t < n_threads; ++t) {
        pthread_join(th[t], NULL);
        out[0] += args[t].votes;
        out[1] += args[t].peaks;
        out[2] += args[t].pairs;
    }
    free(args);
    free(th);
    free(order);
}

/* ---- range voting (the first extension beyond the point vote) -------------
 *
 * Section 3 lets a hit vote for every instance containing it.  With point
 * sampling, an instance (cell) contains the hit when the hit's curve passes
 * through the cell's centre column; range voting instead takes every kappa
 * bin the curve crosses over the whole (phi0, d0) cell.  Reading used here:
 * the curve's kappa is evaluated, by the binary64 definition above, at the
 * cell's four corners (phi0 edges m 2pi/n_phi, periodic; d0 edges
 * d0_min + n (d0_max - d0_min)/n_d0), and the hit votes for every bin from
 * the lowest to the highest corner bin, clipped to [0, n_kappa).  A corner
 * whose denominator is not positive (the hit is that corner's perigee point)
 * leaves the cell without a vote.
 */

/* Edge tables: cos/sin of m 2pi/n_phi for m = 0..n_phi-1 and the n_d0 + 1
 * d0 edges, each rounded to float once. */
void hto_edges(const hto_grid *g, float *cos_e, float *sin_e, float *d_e)
{
    for (int32_t m = 0; m < g->n_phi; ++m) {
        double phi = (double)m * (2.0 * kPi / (double)g->n_phi);
        cos_e[m] = (float)cos(phi);
        sin_e[m] = (float)sin(phi);
    }
    for (int32_t n = 0; n <= g->n_d0; ++n) {
        double w = ((double)g->d0_max - (double)g->d0_min) / (double)g->n_d0;
        d_e[n] = (float)((double)g->d0_min + (double)n * w);
    }
}

/* Corner code: HTO_UNDEF when den <= 0, -1 below the kappa range, n_kappa
 * above it, else the bin. */
int32_t hto_code_at(const hto_grid *g, float x, float y, float c, float s, float d)
{
    double w = hto_w64(g, x, y, c, s, d);
    if (isnan(w))
        return HTO_UNDEF;
    if (w < 0.0)
        return -1;
    if (w >= (double)g->n_kappa)
        return g->n_kappa;
    return (int32_t)w;
}

void hto_code_cells(const hto_grid *g, int64_t n, const float *x, const float *y, const float *c,
                    const float *s, const float *d, int32_t *out)
{
    for (int64_t t = 0; t < n; ++t)
        out[t] = hto_code_at(g, x[t], y[t], c[t], s[t], d[t]);
}

/* Bins [*lo, *hi] (clipped) that hit (x, y) votes for in cell (i, j); returns
 * 0 when it votes for none. */
static int range_cell(const hto_grid *g, const float *ce, const float *se, const float *de,
                      float x, float y, int32_t i, int32_t j, int32_t *lo, int32_t *hi)
{
    int32_t i1 = (i + 1) % g->n_phi;
    int32_t code[4];
    code[0] = hto_code_at(g, x, y, ce[i], se[i], de[j]);
    code[1] = hto_code_at(g, x, y, ce[i1], se[i1], de[j]);
    code[2] = hto_code_at(g, x, y, ce[i], se[i], de[j + 1]);
    code[3] = hto_code_at(g, x, y, ce[i1], se[i1], de[j + 1]);
    int32_t a = code[0], b = code[0];
    for (int t = 0; t < 4; ++t) {
        if (code[t] == HTO_UNDEF)
            return 0;
        if (code[t] < a) a = code[t];
        if (code[t] > b) b = code[t];
    }
    if (b < 0 || a >= g->n_kappa)
        return 0;
    *lo = a < 0 ? 0 : a;
    *hi = b >= g->n_kappa ? g->n_kappa - 1 : b;
    return 1;
}

int32_t hto_range(const hto_grid *g, float x, float y, int32_t i, int32_t j, int32_t *lo, int32_t *hi)
{
    float *ce = (float *)malloc(sizeof(float) * (size_t)g->n_phi);
    float *se = (float *)malloc(sizeof(float) * (size_t)g->n_phi);
    float *de = (float *)malloc(sizeof(float) * (size_t)(g->n_d0 + 1));
    hto_edges(g, ce, se, de);
    int32_t ok = range_cell(g, ce, se, de, x, y, i, j, lo, hi);
    free(ce); free(se); free(de);
    return ok;
}

void hto_vote_range(const hto_grid *g, const float *x, const float *y,
                    const int32_t *event_offsets, int32_t n_events, uint32_t *acc)
{
    float *ce = (float *)malloc(sizeof(float) * (size_t)g->n_phi);
    float *se = (float *)malloc(sizeof(float) * (size_t)g->n_phi);
    float *de = (float *)malloc(sizeof(float) * (size_t)(g->n_d0 + 1));
    hto_edges(g, ce, se, de);
    const int64_t nd = g->n_d0, nk = g->n_kappa;
    const int64_t cells = (int64_t)g->n_phi * nd * nk;
    for (int32_t e = 0; e < n_events; ++e) {
        uint32_t *a1 = acc + (int64_t)e * cells;
        memset(a1, 0, sizeof(uint32_t) * (size_t)cells);
        for (int64_t h = event_offsets[e]; h < event_offsets[e + 1]; ++h)
            for (int32_t i = 0; i < g->n_phi; ++i)
                for (int32_t j = 0; j < g->n_d0; ++j) {
                    int32_t lo, hi;
                    if (!range_cell(g, ce, se, de, x[h], y[h], i, j, &lo, &hi))
                        continue;
                    for (int32_t k = lo; k <= hi; ++k)
                        a1[((int64_t)i * nd + j) * nk + k] += 1u;
                }
    }
    free(ce); free(se); free(de);
}

/* Range association: hit h belongs to peak (i, j, k) when its bins in
 * column (i, j) reach within `window` of k. */
int64_t hto_associate_range(const hto_grid *g, const float *x, const float *y,
                            const int32_t *event_offsets, const hto_peak *peaks, int64_t n_peaks,
                            int32_t window, int64_t *peak_offsets, int32_t *hit_idx, int64_t cap)
{
    float *ce = (float *)malloc(sizeof(float) * (size_t)g->n_phi);
    float *se = (float *)malloc(sizeof(float) * (size_t)g->n_phi);
    float *de = (float *)malloc(sizeof(float) * (size_t)(g->n_d0 + 1));
    hto_edges(g, ce, se, de);
    int64_t n = 0;
    peak_offsets[0] = 0;
    for (int64_t p = 0; p < n_peaks; ++p) {
        const hto_peak *pk = &peaks[p];
        for (int64_t h = event_offsets[pk->event]; h < event_offsets[pk->event + 1]; ++h) {
            int32_t lo, hi;
            if (!range_cell(g, ce, se, de, x[h], y[h], pk->i_phi, pk->i_d0, &lo, &hi))
                continue;
            if (lo <= pk->i_kappa + window && hi >= pk->i_kappa - window) {
                if (n < cap)
                    hit_idx[n] = (int32_t)h;
                ++n;
            }
        }
        peak_offsets[p + 1] = n;
    }
    free(ce); free(se); free(de);
    return n;
}

/* ---- circle fit of a candidate's hits (the second extension) -------------
 *
 * Section 3: the HT candidates seed a confirmation fit.  Reading used here:
 * the algebraic (Kasa) least-squares circle through the candidate's
 * associated hits, x^2 + y^2 + D x + E y + F = 0 minimising the sum of the
 * squared left-hand sides, solved from its 3 x 3 normal equations by
 * Cramer's rule; sums run over the row's hits in ascending order, every
 * operation one binary64 IEEE operation in the order written.  The circle
 * becomes perigee parameters with the turning sign s of the peak's kappa bin
 * centre (s = +1 when that centre is >= 0): kappa = s / R, unit normal
 * n = s C / |C|, d0 = s (|C| - R), phi0 from n = (-sin phi0, cos phi0); the
 * outputs are cos phi0, sin phi0, d0, kappa and the geometric chi^2 =
 * sum (|h - C| - R)^2.  status: 1 fitted, 0 fewer than three hits or a
 * singular system or R^2 <= 0 or C = 0.
 */
void hto_fit_row(const hto_grid *g, const float *x, const float *y, const int32_t *idx, int64_t n,
                 int32_t i_kappa, hto_track *out)
{
    memset(out, 0, sizeof(*out));
    out->n_hits = (int32_t)n;
    if (n < 3)
        return;
    double sx = 0.0, sy = 0.0, sxx = 0.0, sxy = 0.0, syy = 0.0, sz = 0.0, sxz = 0.0, syz = 0.0;
    for (int64_t t = 0; t < n; ++t) {
        double a = x[idx[t]], b = y[idx[t]];
        double z = (a * a) + (b * b);
        sx = sx + a;
        sy = sy + b;
        sxx = sxx + (a * a);
        sxy = sxy + (a * b);
        syy = syy + (b * b);
        sz = sz + z;
        sxz = sxz + (a * z);
        syz = syz + (b * z);
    }
    double nn = (double)n;
    /* M (D E F)^T = -(sxz, syz, sz)^T, M = [[sxx sxy sx] [sxy syy sy] [sx sy n]] */
    double c00 = (syy * nn) - (sy * sy);
    double c01 = (sxy * nn) - (sy * sx);
    double c02 = (sxy * sy) - (syy * sx);
    double det = ((sxx * c00) - (sxy * c01)) + (sx * c02);
    if (!(det != 0.0))
        return;
    double r0 = -sxz, r1 = -syz, r2 = -sz;
    /* Cramer: replace one column by r */
    double dD = ((r0 * c00) - (sxy * ((r1 * nn) - (sy * r2)))) + (sx * ((r1 * sy) - (syy * r2)));
    double dE = ((sxx * ((r1 * nn) - (sy * r2))) - (r0 * c01)) + (sx * ((sxy * r2) - (r1 * sx)));
    double dF = ((sxx * ((syy * r2) - (r1 * sy))) - (sxy * ((sxy * r2) - (r1 * sx)))) + (r0 * c02);
    double D = dD / det, E = dE / det, F = dF / det;
    double cx = -0.5 * D, cy = -0.5 * E;
    double R2 = ((cx * cx) + (cy * cy)) - F;
    double rho = sqrt((cx * cx) + (cy * cy));
    if (!(R2 > 0.0) || !(rho > 0.0))
        return;
    double R = sqrt(R2);
    double kc = (double)g->kappa_min + (((double)i_kappa + 0.5) * (((double)g->kappa_max - (double)g->kappa_min) / (double)g->n_kappa));
    double s = kc >= 0.0 ? 1.0 : -1.0;
    double nx = (s * cx) / rho, ny = (s * cy) / rho;
    double chi2 = 0.0;
    for (int64_t t = 0; t < n; ++t) {
        double a = (double)x[idx[t]] - cx, b = (double)y[idx[t]] - cy;
        double r = sqrt((a * a) + (b * b)) - R;
        chi2 = chi2 + (r * r);
    }
    out->status = 1;
    out->cos_phi0 = ny;
    out->sin_phi0 = -nx;
    out->d0 = s * (rho - R);
    out->kappa = s / R;
    out->chi2 = chi2;
}

void hto_fit(const hto_grid *g, const float *x, const float *y, const hto_peak *peaks, int64_t n_peaks,
             const int64_t *peak_offsets, const int32_t *hit_idx, hto_track *out)
{
    for (int64_t p = 0; p < n_peaks; ++p)
        hto_fit_row(g, x, y, hit_idx + peak_offsets[p], peak_offsets[p + 1] - peak_offsets[p],
                    peaks[p].i_kappa, &out[p]);
}

/* ---- second Hough transform: displaced vertices (the third extension) -----
 *
 * Section "Displaced vertex identification": tracks from a common vertex
 * (xv, yv) satisfy d0 = yv cos phi0 - xv sin phi0, a sinusoid in the first
 * transform's (phi0, d0) space, and a second Hough transform of the first
 * one's maxima finds them.  Reading used here: every candidate (peak) votes,
 * with its cell's centre tables (cos phi_i, sin phi_i, d0_j as floats), for
 * the cells of an (x, y) vertex grid that its line y c - x s = d crosses,
 * walking the axis along which the line is less steep: when |c| >= |s|, for
 * each x bin centre X the y of the line (d + X s) / c, else for each y bin
 * centre Y the x of the line (Y c - d) / s; one vote per bin of the walked
 * axis whose other coordinate falls inside the grid.  Every operation is one
 * binary64 IEEE operation in the order written.  Vertices are the local
 * maxima of each event's (x, y) accumulator at or above a threshold, by the
 * first transform's rule: strictly above the neighbours preceding in linear
 * (x, y) order, at least the ones following, 8-neighbourhood, no wrap.
 */
static void vgrid_centres(const hto_vgrid *v, double *xc, double *yc)
{
    double wx = ((double)v->x_max - (double)v->x_min) / (double)v->n_x;
    double wy = ((double)v->y_max - (double)v->y_min) / (double)v->n_y;
    for (int32_t a = 0; a < v->n_x; ++a)
        xc[a] = (double)v->x_min + (((double)a + 0.5) * wx);
    for (int32_t b = 0; b < v->n_y; ++b)
        yc[b] = (double)v->y_min + (((double)b + 0.5) * wy);
}

static int32_t vbin(double u, float lo, float hi, int32_t n)
{
    double t = (u - (double)lo) * ((double)n / ((double)hi - (double)lo));
    if (!(t >= 0.0 && t < (double)n))
        return -1;
    return (int32_t)t;
}

void hto_vertex_vote(const hto_grid *g, const hto_vgrid *v, const hto_peak *peaks, int64_t n_peaks,
                     int32_t n_events, uint32_t *acc)
{
    float *c, *s, *d;
    tables_alloc(g, &c, &s, &d);
    double *xc = (double *)malloc(sizeof(double) * (size_t)v->n_x);
    double *yc = (double *)malloc(sizeof(double) * (size_t)v->n_y);
    vgrid_centres(v, xc, yc);
    const int64_t cells = (int64_t)v->n_x * v->n_y;
    memset(acc, 0, sizeof(uint32_t) * (size_t)(cells * n_events));
    for (int64_t p = 0; p < n_peaks; ++p) {
        const hto_peak *pk = &peaks[p];
        if (pk->event < 0 || pk->event >= n_events)
            continue;
        uint32_t *a1 = acc + (int64_t)pk->event * cells;
        double cc = c[pk->i_phi], ss = s[pk->i_phi], dd = d[pk->i_d0];
        if (fabs(cc) >= fabs(ss)) {
            for (int32_t a = 0; a < v->n_x; ++a) {
                int32_t b = vbin((dd + (xc[a] * ss)) / cc, v->y_min, v->y_max, v->n_y);
                if (b >= 0)
                    a1[(int64_t)a * v->n_y + b] += 1u;
            }
        } else {
            for (int32_t b = 0; b < v->n_y; ++b) {
                int32_t a = vbin(((yc[b] * cc) - dd) / ss, v->x_min, v->x_max, v->n_x);
                if (a >= 0)
                    a1[(int64_t)a * v->n_y + b] += 1u;
            }
        }
    }
    free(xc); free(yc); free(c); free(s); free(d);
}

int64_t hto_vertex_peaks(const hto_vgrid *v, const uint32_t *acc, int32_t n_events, uint32_t threshold,
                         hto_vertex *out, int64_t cap)
{
    const int64_t cells = (int64_t)v->n_x * v->n_y;
    int64_t n = 0;
    for (int32_t e = 0; e < n_events; ++e) {
        const uint32_t *a1 = acc + (int64_t)e * cells;
        for (int32_t a = 0; a < v->n_x; ++a)
            for (int32_t b = 0; b < v->n_y; ++b) {
                const int64_t self = (int64_t)a * v->n_y + b;
                const uint32_t val = a1[self];
                if (val < threshold)
                    continue;
                int ok = 1;
                for (int da = -1; da <= 1 && ok; ++da)
                    for (int db = -1; db <= 1; ++db) {
                        int32_t aa = a + da, bb = b + db;
                        if ((da == 0 && db == 0) || aa < 0 || aa >= v->n_x || bb < 0 || bb >= v->n_y)
                            continue;
                        const int64_t other = (int64_t)aa * v->n_y + bb;
                        const uint32_t u = a1[other];
                        if (other < self ? !(val > u) : !(val >= u)) {
                            ok = 0;
                            break;
                        }
                    }
                if (ok) {
                    if (n < cap) {
                        hto_vertex t = {e, a, b, val};
                        out[n] = t;
                    }
                    ++n;
                }
            }
    }
    return n;
}

/* ---- straight displaced tracks (the paper's kappa = 0 model) --------------
 *
 * Section 3's implementation of the paper used two-parameter models; the
 * straight displaced one is the line through the perigee d0 n with
 * direction t, so a hit (x, y) lies on it when d0 = q = y cos phi0 - x sin phi0.
 * Line voting: on a grid with a single kappa bin, each hit votes, for every
 * phi0 row, in the d0 bin of q: floor((q - d0_min) n_d0 / (d0_max - d0_min))
 * when that lies in [0, n_d0) (binary64, in this order: the two products of
 * float values are exact, so q is rounded once).  It joins peak (i, j, 0)
 * when its d0 bin in row i lies within `window` of j.
 */
static int32_t line_bin(const hto_grid *g, float xf, float yf, float cf, float sf)
{
    double q = ((double)yf * (double)cf) - ((double)xf * (double)sf);
    double t = (q - (double)g->d0_min) * ((double)g->n_d0 / ((double)g->d0_max - (double)g->d0_min));
    if (!(t >= 0.0 && t < (double)g->n_d0))
        return -1;
    return (int32_t)t;
}

int32_t hto_line_bin(const hto_grid *g, float x, float y, int32_t i)
{
    double phi = ((double)i + 0.5) * (2.0 * kPi / (double)g->n_phi);
    return line_bin(g, x, y, (float)cos(phi), (float)sin(phi));
}

void hto_vote_line(const hto_grid *g, const float *x, const float *y, const int32_t *event_offsets,
                   int32_t n_events, uint32_t *acc)
{
    float *c, *s, *d;
    tables_alloc(g, &c, &s, &d);
    const int64_t cells = (int64_t)g->n_phi * g->n_d0;
    for (int32_t e = 0; e < n_events; ++e) {
        uint32_t *a1 = acc + (int64_t)e * cells;
        memset(a1, 0, sizeof(uint32_t) * (size_t)cells);
        for (int64_t h = event_offsets[e]; h < event_offsets[e + 1]; ++h)
            for (int32_t i = 0; i < g->n_phi; ++i) {
                int32_t j = line_bin(g, x[h], y[h], c[i], s[i]);
                if (j >= 0)
                    a1[(int64_t)i * g->n_d0 + j] += 1u;
            }
    }
    free(c); free(s); free(d);
}

int64_t hto_associate_line(const hto_grid *g, const float *x, const float *y, const int32_t *event_offsets,
                           const hto_peak *peaks, int64_t n_peaks, int32_t window, int64_t *peak_offsets,
                           int32_t *hit_idx, int64_t cap)
{
    float *c, *s, *d;
    tables_alloc(g, &c, &s, &d);
    int64_t n = 0;
    peak_offsets[0] = 0;
    for (int64_t p = 0; p < n_peaks; ++p) {
        const hto_peak *pk = &peaks[p];
        for (int64_t h = event_offsets[pk->event]; h < event_offsets[pk->event + 1]; ++h) {
            int32_t j = line_bin(g, x[h], y[h], c[pk->i_phi], s[pk->i_phi]);
            if (j >= 0 && abs(j - pk->i_d0) <= window) {
                if (n < cap)
                    hit_idx[n] = (int32_t)h;
                ++n;
            }
        }
        peak_offsets[p + 1] = n;
    }
    free(c); free(s); free(d);
    return n;
}

/* ---- duplicate and mirror merging of fitted candidates (second extension) --
 *
 * Section 3 hands the transform's candidates to a confirmation step.  Every
 * track leaves two kinds of extra candidates: the mirror cell (phi0 + pi,
 * -d0, -kappa), the same circle travelled the other way, and nearby cells
 * that its hits also fill above threshold.  Reading used here, applied after
 * the circle fit:
 *  1. A candidate whose fit has status != 1 is UNFITTED.
 *  2. A track leaves its perigee P = d0 n moving along t = (cos phi0,
 *     sin phi0), so its hits lie ahead of P: (h - P).t > 0, and since
 *     P.t = 0 this is h.t.  A fitted candidate is BACKWARD (the mirror of a
 *     forward one) unless the sum over its row's hits, in row order, of
 *     x cos phi0 + y sin phi0 (each term fl(fl(x c) + fl(y s)), summed in
 *     binary64) is > 0.
 *  3. A forward fitted candidate is a DUPLICATE when another forward fitted
 *     candidate of the same event lies within `radius` cells of it in each
 *     of phi0 (periodic), d0 and kappa and is better: more votes, or as many
 *     and a smaller index.  Otherwise it is KEPT.
 * Written as the definition: every pair of the event's candidates is
 * compared (peaks must be grouped by event).  Returns the number kept.
 */
static int32_t phi_distance(int32_t a, int32_t b, int32_t n_phi)
{
    int32_t d = abs(a - b);
    return d < n_phi - d ? d : n_phi - d;
}

int64_t hto_merge(const hto_grid *g, const float *x, const float *y, const hto_peak *peaks, int64_t n_peaks,
                  const int64_t *peak_offsets, const int32_t *hit_idx, const hto_track *fits,
                  int32_t radius, int32_t *state)
{
    for (int64_t p = 0; p < n_peaks; ++p) {
        const hto_track *f = &fits[p];
        if (f->status != 1) {
            state[p] = HTO_MERGE_UNFITTED;
            continue;
        }
        double t = 0.0;
        for (int64_t q = peak_offsets[p]; q < peak_offsets[p + 1]; ++q) {
            int32_t h = hit_idx[q];
            t = t + (((double)x[h] * f->cos_phi0) + ((double)y[h] * f->sin_phi0));
        }
        state[p] = t > 0.0 ? HTO_MERGE_KEPT : HTO_MERGE_BACKWARD;
    }
    int64_t kept = 0;
    int64_t lo = 0, hi = 0; /* [lo, hi): the candidates of p's event (peaks are grouped by event) */
    for (int64_t p = 0; p < n_peaks; ++p) {
        if (p == hi) {
            lo = p;
            for (hi = p; hi < n_peaks && peaks[hi].event == peaks[p].event; ++hi)
                ;
        }
        if (state[p] != HTO_MERGE_KEPT && state[p] != HTO_MERGE_DUPLICATE)
            continue;
        const hto_peak *a = &peaks[p];
        int dup = 0;
        for (int64_t q = lo; q < hi && !dup; ++q) {
            const hto_peak *b = &peaks[q];
            if (q == p)
                continue;
            if (state[q] != HTO_MERGE_KEPT && state[q] != HTO_MERGE_DUPLICATE)
                continue;
            if (phi_distance(a->i_phi, b->i_phi, g->n_phi) > radius || abs(a->i_d0 - b->i_d0) > radius ||
                abs(a->i_kappa - b->i_kappa) > radius)
                continue;
            if (b->votes > a->votes || (b->votes == a->votes && q < p))
                dup = 1;
        }
        state[p] = dup ? HTO_MERGE_DUPLICATE : HTO_MERGE_KEPT;
        kept += !dup;
    }
    return kept;
}
