// ht_kbin.cuh — the curvature bin of a (hit, phi0_i, d0_j) column on the GPU.
//
// Definition (Section 3 track model, curved and displaced): with
//   q = y c - x s, a = q - d, den = (x^2 + y^2 + d^2) - 2 d q,
//   kappa = 2 a / den, w = (kappa - kappa_min) * n_kappa / (kappa_max - kappa_min),
// the hit votes into bin floor(w) when den > 0 and 0 <= w < n_kappa.  The bin
// is *defined* by binary64 IEEE operations in exactly this order on the float32
// hit (x, y) and float32 tables (c, s, d).  GB300 runs binary64 at a tiny
// fraction of its float32 rate, so the bin is reached in three stages, each of
// which either decides the binary64 bin with a proof or hands on:
//
//   1. float32 estimate with an a-priori error bound tau (fast path, every cell);
//   2. double-float ("float-float") evaluation with a much smaller bound
//      (cells whose stage-1 interval [w - tau, w + tau] straddles a bin edge,
//      or whose denominator is too small for the stage-1 bound);
//   3. the binary64 definition itself, op for op (cells stage 2 cannot decide:
//      hits within a fraction of a millimetre of the perigee point, or w within
//      ~1e-9 of a bin edge).
//
// Notation for the bounds: u = 2^-24 (float32 unit roundoff), e_r = 2^-22 (a
// bound on the relative error of rcp.approx.ftz.f32, checked by a GPU test),
// R1 = r + dabs with r = |h| and dabs = max_j |d0_j|, V = the largest |v| of a
// cell that still matters (v = w - H, H = -kappa_min * scale).  Every bound
// below carries a factor-2 safety margin over the first-order analysis.
#pragma once
#include <cstdint>

namespace ht {

// Grid constants shared by every kernel that bins a cell (filled on the host).
struct KConsts {
    int nphi, nd, nk;
    // stage 1 (float32 estimate)
    float S2;       // float(2 * scale), scale = n_kappa / (kappa_max - kappa_min)
    float H;        // float(-kappa_min * scale)
    float T0;       // constant part of tau
    float cG1, cG2; // tau = T0 + (cG1 R1^2 + cG2 P1) * |rcp(den)|, P1 = 4.02 r + 2.02 dabs
    float cD1, cD2; // den_min = max(cD1 R1^2, cD2 P1): below it the bound is not used
    float wlo, whi; // w outside (wlo, whi) = (-m, n_kappa + m) is out of range for sure
    float dabs;
    // stage 2 (double-float)
    float S2hi, S2lo, Hhi, Hlo; // 2*scale and H as float pairs (hi + lo)
    float T0b;                  // constant part of tau2
    float cGb1, cGb2;           // tau2 = T0b + (cGb1 R1^2 + cGb2 R1) * rcp(den)
    float cDb;                  // den_min2 = cDb * R1^2
    // stage 3 (binary64 definition)
    double kmin, scale;
    // d0 band of a (hit, phi row): kappa window widened by two bins each side
    int band_ok;           // 0: kappa range does not straddle 0 or d0 columns too narrow: no bands
    float bA2, bB2, biA, biB, bdfirst, bidd;
};

__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// The d0 columns [jlo, jhi] of the tile [j0, j0 + nj) where hit (x, y) can vote
// in the row with table values (c, s), as a superset: with u = d0 - q and
// p^2 = r^2 - q^2 the curvature is -2u / (u^2 + p^2); it lies in [A, B)
// (A < 0 < B, the kappa range widened by two bins) outside the forbidden
// intervals (a1, a2) (kappa < A) and [b1, b2] (kappa >= B), whose ends are
// roots of A u^2 + 2u + A p^2 = 0 and B u^2 + 2u + B p^2 = 0.  The hull of
// the allowed u in the tile is widened by one column below and two above.
// Returns jhi < jlo when the tile holds no allowed column.
__device__ __forceinline__ void d0_band(float r2, float q, float dlo, float dhi, int j0, int nj, const KConsts& K,
                                        int& jlo, int& jhi) {
    const float BIG = 1e30f;
    const float p2 = fmaxf(fmaf(-q, q, r2), 0.0f);
    const float DA = fmaf(-K.bA2, p2, 1.0f);
    const float DB = fmaf(-K.bB2, p2, 1.0f);
    // approximate square roots and reciprocals (relative errors of a few
    // ulps): a root off by eps moves kappa by |dkappa/du| eps, far below the
    // two bins the window is widened by, and the u bounds stay well inside
    // the one-column margin (the host keeps bands off for narrower columns)
    const float sA = DA > 0.0f ? DA * rsqrtf(DA) : 0.0f;
    const float sB = DB > 0.0f ? DB * rsqrtf(DB) : 0.0f;
    const float a1 = DA > 0.0f ? ((K.bA2 * p2) * K.biA) * rcp_approx(1.0f + sA) : BIG;
    const float a2 = DA > 0.0f ? (1.0f + sA) * K.biA : BIG;
    const float b2 = DB > 0.0f ? ((-(K.bB2 * p2)) * K.biB) * rcp_approx(1.0f + sB) : -BIG;
    const float b1 = DB > 0.0f ? (-(1.0f + sB)) * K.biB : -BIG;
    const float ulo = dlo - q, uhi = dhi - q;
    const float lo = ulo < b1 ? ulo
                              : ((ulo <= a1) & (uhi > b2) ? fmaxf(ulo, b2) : (uhi >= a2 ? fmaxf(ulo, a2) : BIG));
    const float hi = uhi >= a2 ? uhi
                               : ((uhi > b2) & (ulo <= a1) ? fminf(uhi, a1) : (ulo < b1 ? fminf(uhi, b1) : -BIG));
    if (!(lo <= hi)) {
        jlo = j0 + nj;
        jhi = j0 - 1;
        return;
    }
    const float jl = floorf(((lo + q) - K.bdfirst) * K.bidd) - 1.0f;
    const float jh = floorf(((hi + q) - K.bdfirst) * K.bidd) + 2.0f;
    jlo = (int)fminf(fmaxf(jl, (float)j0), (float)(j0 + nj));
    jhi = (int)fminf(fmaxf(jh, (float)(j0 - 1)), (float)(j0 + nj - 1));
}

// ---- stage 1 -------------------------------------------------------------
// Inputs hoisted out of the cell loop:
//   per hit      r2 = fl(fma(x, x, fl(y*y))), G = cG1 R1^2 + cG2 P1, dmin
//   per (hit,i)  q  = fl(fma(y, c, -fl(x*s)))            |q - q*|   <= 2.01 u r
//   per (hit,j)  Rj = fl(r2 + fl(d*d))                    |Rj - R*|  <= 3.02 u r^2 + 2.01 u d^2
// Per cell:
//   a   = fl(q - d)                                       |a - a*|   <= u (3.02 r + 1.01 |d|)
//   (the kernels fold S2 in: a' = fl(fl(q S2) - fl(d S2)), |a' - S2 a*| <= S2 u (4.02 r + 2.02 |d|))
//   den = fl(fma(-2d, q, Rj))                             |den-den*| <= E = 4.03 u R1^2
//   w   = fl(fma(fl(a * rcp(den)), S2, H))
// With den > den_min >= 64 E the relative error of den is <= 1/64, and for a
// cell whose w lies in (-m, n_kappa + m) (so |v| <= V):
//   |w - w*| <= (e_r + 3u) V + u(|H| + 2 (n_kappa + m)) + u     (constant: T0)
//             + (64/63) E V / den + 1.01 S2 u (4.02 r + 2.02 |d|) / den   (per-hit: G)
// and w* (the exact real value) is within ~1e-11 bins of the binary64 w.
// A cell whose w lies outside (-m, n_kappa + m) is out of range in binary64
// too: m is chosen on the host so that m (1 - e_v) exceeds e_v (n_kappa + |H|) + 0.3, where
// e_v <= e_r + 4u + 1/63 bounds the relative error of v and 0.3 bounds the
// absolute part (den >= den_min also caps the a-error term at 0.28 bins).
// Stage 1 as the tile kernels evaluate it, with the kappa scale folded into
// the operands: qs = fl(q * S2) per (hit, row) and ds = fl(d * S2) from the
// table, a' = fl(qs - ds), w = fl(fma(a', rcp(den), H)).  Relative to the
// unfolded form the a-error becomes S2 u (4.02 r + 2.02 |d|) (P1 below) and
// the product t disappears; the bound keeps the same shape.
// stage1_fast: the certified bin candidate; decided iff flo == fhi, then kb
// is the bin (a vote iff kb < n_kappa).  The den > den_min test is implicit
// (G >= 0.55 den_min makes tau > 1/2 below it).
struct S1 {
    float flo, fhi, w, den;
    unsigned kb;
};

__device__ __forceinline__ S1 stage1_fast(float qs, float q, float4 dt, float Rj, float G, float H, float T0) {
    S1 o;
    const float a = qs - dt.w;
    o.den = fmaf(-dt.y, q, Rj);
    const float rc = rcp_approx(o.den);
    o.w = fmaf(a, rc, H);
    const float tau = fmaf(G, fabsf(rc), T0);
    o.flo = __fadd_rd(o.w - tau, 12582912.0f);
    o.fhi = __fadd_rd(o.w + tau, 12582912.0f);
    o.kb = __float_as_uint(o.flo) - 0x4B400000u;
    return o;
}

// For a cell stage1_fast did not decide: does it need stage 2?  Not when
// den > den_min (the bound holds) and w lies outside (-m, n_kappa + m),
// which proves it out of range.
__device__ __forceinline__ bool stage1_pending(const S1& o, float dmin, float wlo, float whi) {
    return !(o.den > dmin) || ((o.w > wlo) & (o.w < whi));
}

// ---- stage 2: double-float ---------------------------------------------
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
    p = __fmul_rn(a, b);
    e = fmaf(a, b, -p);
}

// Exact products and error-free sums give q, a and den with absolute errors
// <= 8 u^2 r, 8 u^2 (r + |d|) and 24 u^2 R1^2; the quotient a/den is formed
// as q1 + q2 (q1 = a_hi rcp(den_hi), q2 = remainder * rcp) with relative
// error <= 2^-40; v = (q1 + q2) * (S2hi + S2lo) and w = v + (Hhi + Hlo) add
// ~2^-44 V.  With den >= den_min2 = cDb R1^2 (relative den error <= 2^-20):
//   |w_dd - w64| <= T0b + (cGb1 R1^2 + cGb2 R1) / den = tau2,
// and w outside (-2, n_kappa + 2) is out of range for sure.
// Returns k >= 0, -1, or -2 (undecided: use binary64).
__device__ __forceinline__ int cell_dd(float x, float y, float c, float s, float d, float R1,
                                       const KConsts& K) {
    float p1, e1, p2, e2;
    two_prod(y, c, p1, e1);
    two_prod(x, s, p2, e2);
    float s1, t1;
    two_sum(p1, -p2, s1, t1);
    float qh, ql;
    two_sum(s1, __fadd_rn(t1, __fsub_rn(e1, e2)), qh, ql);
    float s2, t2;
    two_sum(qh, -d, s2, t2);
    float ah, al;
    two_sum(s2, __fadd_rn(t2, ql), ah, al);
    float xx, exx, yy, eyy, dd, edd;
    two_prod(x, x, xx, exx);
    two_prod(y, y, yy, eyy);
    two_prod(d, d, dd, edd);
    const float d2 = __fadd_rn(d, d);
    float mh, me;
    two_prod(d2, qh, mh, me);
    me = fmaf(d2, ql, me);
    float s3, t3, s4, t4, s5, t5;
    two_sum(xx, yy, s3, t3);
    two_sum(s3, dd, s4, t4);
    two_sum(s4, -mh, s5, t5);
    const float low = __fadd_rn(__fadd_rn(__fadd_rn(exx, eyy), __fsub_rn(edd, me)),
                                __fadd_rn(__fadd_rn(t3, t4), t5));
    float denh, denl;
    two_sum(s5, low, denh, denl);
    if (!(denh > K.cDb * R1 * R1)) return -2;
    const float rc = rcp_approx(denh);
    const float q1 = __fmul_rn(ah, rc);
    float pp, pe;
    two_prod(q1, denh, pp, pe);
    const float rem = fmaf(-q1, denl, __fadd_rn(__fsub_rn(__fsub_rn(ah, pp), pe), al));
    const float q2 = __fmul_rn(rem, rc);
    float vh, ve;
    two_prod(q1, K.S2hi, vh, ve);
    ve = fmaf(q1, K.S2lo, ve);
    ve = fmaf(q2, K.S2hi, ve);
    float s6, t6;
    two_sum(vh, K.Hhi, s6, t6);
    float wh, wl;
    two_sum(s6, __fadd_rn(__fadd_rn(t6, ve), K.Hlo), wh, wl);
    if (!(wh > -2.0f && wh < (float)K.nk + 2.0f)) return -1;
    const float tau2 = fmaf(fmaf(K.cGb1 * R1, R1, K.cGb2 * R1), rc, K.T0b);
    // floor of wh + wl: wh may round up onto an integer while wl < 0
    float kf = floorf(wh);
    float a0, b0, a1, b1;
    two_sum(wh, -kf, a0, b0);
    float dist_lo = __fadd_rn(a0, __fadd_rn(b0, wl));
    two_sum(__fadd_rn(kf, 1.0f), -wh, a1, b1);
    float dist_hi = __fadd_rn(a1, __fsub_rn(b1, wl));
    if (dist_lo < 0.0f) {
        kf = __fsub_rn(kf, 1.0f);
        dist_hi = -dist_lo;
        dist_lo = __fadd_rn(dist_lo, 1.0f);
    }
    if (dist_lo > tau2 && dist_hi > tau2) {
        const int k = (int)kf;
        return (k >= 0 && k < K.nk) ? k : -1;
    }
    return -2;
}

// ---- stage 3: the binary64 definition, op for op ------------------------
__device__ __forceinline__ int cell_f64(float xf, float yf, float cf, float sf, float df,
                                        const KConsts& K) {
    const double x = xf, y = yf, c = cf, s = sf, d = df;
    const double q = __dsub_rn(__dmul_rn(y, c), __dmul_rn(x, s));
    const double a = __dsub_rn(q, d);
    const double den = __dsub_rn(__dadd_rn(__dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y)), __dmul_rn(d, d)),
                                 __dmul_rn(__dmul_rn(2.0, d), q));
    if (!(den > 0.0)) return -1;
    const double kappa = __ddiv_rn(__dmul_rn(2.0, a), den);
    const double w = __dmul_rn(__dsub_rn(kappa, K.kmin), K.scale);
    if (!(w >= 0.0 && w < (double)K.nk)) return -1;
    return (int)w;
}

// Stages 2 and 3, kept out of line so the hot loop stays small.
// stats (optional): [0] cells (counted by callers), [1] stage-2 decisions, [2] stage-3 decisions.
static __device__ __noinline__ int cell_slow(float x, float y, float c, float s, float d, float R1,
                                      const KConsts& K, unsigned long long* stats) {
    int k = cell_dd(x, y, c, s, d, R1, K);
    if (k != -2) {
        if (stats) atomicAdd(&stats[1], 1ull);
        return k;
    }
    if (stats) atomicAdd(&stats[2], 1ull);
    return cell_f64(x, y, c, s, d, K);
}

// Per-hit quantities of stage 1.
struct HitFast {
    float r2, R1, G, dmin;
};

__device__ __forceinline__ HitFast hit_fast(float x, float y, const KConsts& K) {
    HitFast h;
    h.r2 = fmaf(x, x, __fmul_rn(y, y));
    const float r = sqrtf(h.r2);
    h.R1 = r + K.dabs;
    const float P1 = fmaf(4.02f, r, 2.02f * K.dabs);
    const float R1s = h.R1 * h.R1;
    h.dmin = fmaxf(K.cD1 * R1s, K.cD2 * P1);
    // G >= 0.55 dmin: a cell with den <= dmin (or den <= 0, via |rcp|) gets
    // tau > 1/2, so stage 1 can never certify it
    h.G = fmaxf(fmaf(K.cG1, R1s, K.cG2 * P1), 0.55f * h.dmin);
    return h;
}

__device__ __forceinline__ float q_of(float x, float y, float c, float s) {
    return fmaf(y, c, -__fmul_rn(x, s));
}


// ---- corner codes (range voting) -----------------------------------------
// A range vote bins the curve at a cell's four corners.  A corner's code is
// kCodeUndef when its denominator is not positive (binary64), -1 below the
// kappa range, n_kappa above it, else the bin; kCodeUndecided marks a stage
// that could not decide.
constexpr int kCodeUndef = -2, kCodeUndecided = -3;

__device__ __forceinline__ int clamp_code(int v, int nk) { return v < 0 ? -1 : (v > nk ? nk : v); }

// Stage 1 for a corner: decided when den > den_min (so the bound holds) and
// both ends of [w - tau, w + tau] give the same code; far outside the kappa
// range that holds even when an end lies near an integer.
__device__ __forceinline__ int code_stage1(const S1& o, float dmin, int nk) {
    const int a = clamp_code((int)o.kb, nk);
    const int b = clamp_code((int)(__float_as_uint(o.fhi) - 0x4B400000u), nk);
    return (o.den > dmin && a == b) ? a : kCodeUndecided;
}

// Stage 2 for a corner (the double-float evaluation of cell_dd).
__device__ __forceinline__ int code_dd(float x, float y, float c, float s, float d, float R1, const KConsts& K) {
    float p1, e1, p2, e2;
    two_prod(y, c, p1, e1);
    two_prod(x, s, p2, e2);
    float s1, t1;
    two_sum(p1, -p2, s1, t1);
    float qh, ql;
    two_sum(s1, __fadd_rn(t1, __fsub_rn(e1, e2)), qh, ql);
    float s2, t2;
    two_sum(qh, -d, s2, t2);
    float ah, al;
    two_sum(s2, __fadd_rn(t2, ql), ah, al);
    float xx, exx, yy, eyy, dd, edd;
    two_prod(x, x, xx, exx);
    two_prod(y, y, yy, eyy);
    two_prod(d, d, dd, edd);
    const float d2 = __fadd_rn(d, d);
    float mh, me;
    two_prod(d2, qh, mh, me);
    me = fmaf(d2, ql, me);
    float s3, t3, s4, t4, s5, t5;
    two_sum(xx, yy, s3, t3);
    two_sum(s3, dd, s4, t4);
    two_sum(s4, -mh, s5, t5);
    const float low = __fadd_rn(__fadd_rn(__fadd_rn(exx, eyy), __fsub_rn(edd, me)),
                                __fadd_rn(__fadd_rn(t3, t4), t5));
    float denh, denl;
    two_sum(s5, low, denh, denl);
    if (!(denh > K.cDb * R1 * R1)) return kCodeUndecided;
    const float rc = rcp_approx(denh);
    const float q1 = __fmul_rn(ah, rc);
    float pp, pe;
    two_prod(q1, denh, pp, pe);
    const float rem = fmaf(-q1, denl, __fadd_rn(__fsub_rn(__fsub_rn(ah, pp), pe), al));
    const float q2 = __fmul_rn(rem, rc);
    float vh, ve;
    two_prod(q1, K.S2hi, vh, ve);
    ve = fmaf(q1, K.S2lo, ve);
    ve = fmaf(q2, K.S2hi, ve);
    float s6, t6;
    two_sum(vh, K.Hhi, s6, t6);
    float wh, wl;
    two_sum(s6, __fadd_rn(__fadd_rn(t6, ve), K.Hlo), wh, wl);
    // |w - (wh + wl)| is far below one bin: two bins out is out for sure
    if (!(wh > -2.0f)) return -1;
    if (!(wh < (float)K.nk + 2.0f)) return K.nk;
    const float tau2 = fmaf(fmaf(K.cGb1 * R1, R1, K.cGb2 * R1), rc, K.T0b);
    float kf = floorf(wh);
    float a0, b0, a1, b1;
    two_sum(wh, -kf, a0, b0);
    float dist_lo = __fadd_rn(a0, __fadd_rn(b0, wl));
    two_sum(__fadd_rn(kf, 1.0f), -wh, a1, b1);
    float dist_hi = __fadd_rn(a1, __fsub_rn(b1, wl));
    if (dist_lo < 0.0f) {
        kf = __fsub_rn(kf, 1.0f);
        dist_hi = -dist_lo;
        dist_lo = __fadd_rn(dist_lo, 1.0f);
    }
    const int kc = clamp_code((int)kf, K.nk);
    if (dist_lo <= tau2 && clamp_code((int)kf - 1, K.nk) != kc) return kCodeUndecided;
    if (dist_hi <= tau2 && clamp_code((int)kf + 1, K.nk) != kc) return kCodeUndecided;
    return kc;
}

// Stage 3 for a corner: the binary64 definition.
__device__ __forceinline__ int code_f64(float xf, float yf, float cf, float sf, float df, const KConsts& K) {
    const double x = xf, y = yf, c = cf, s = sf, d = df;
    const double q = __dsub_rn(__dmul_rn(y, c), __dmul_rn(x, s));
    const double a = __dsub_rn(q, d);
    const double den = __dsub_rn(__dadd_rn(__dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y)), __dmul_rn(d, d)),
                                 __dmul_rn(__dmul_rn(2.0, d), q));
    if (!(den > 0.0)) return kCodeUndef;
    const double kappa = __ddiv_rn(__dmul_rn(2.0, a), den);
    const double w = __dmul_rn(__dsub_rn(kappa, K.kmin), K.scale);
    if (w < 0.0) return -1;
    if (w >= (double)K.nk) return K.nk;
    return (int)w;
}

static __device__ __noinline__ int code_slow(float x, float y, float c, float s, float d, float R1,
                                             const KConsts& K, unsigned long long* stats) {
    const int k = code_dd(x, y, c, s, d, R1, K);
    if (k != kCodeUndecided) {
        if (stats) atomicAdd(&stats[1], 1ull);
        return k;
    }
    if (stats) atomicAdd(&stats[2], 1ull);
    return code_f64(x, y, c, s, d, K);
}

}  // namespace ht
