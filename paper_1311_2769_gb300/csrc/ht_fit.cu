// ht_fit.cu — circle fit of each candidate's associated hits.
//
// Section 3 hands the HT candidates to a confirmation fit.  This is the
// algebraic (Kasa) least-squares circle through each candidate's CSR row,
// x^2 + y^2 + D x + E y + F = 0 minimising the summed squared left-hand
// sides, solved from its 3 x 3 normal equations by Cramer's rule, then
// returned as perigee parameters with the turning sign of the peak's kappa
// bin centre.  One thread fits one candidate, summing over the row's hits in
// ascending order with one IEEE binary64 operation per step (intrinsics, so
// no contraction), which makes every output reproducible bit for bit.
#include <cuda_runtime.h>

#include <cstdint>

#include "ht_internal.h"

namespace ht {
namespace {

__device__ void fit_row(const FitParams& p, int64_t c) {
    ht_track t{};
    const int64_t lo = p.po[c], hi = p.po[c + 1];
    const int64_t n = hi - lo;
    t.n_hits = (int32_t)n;
    if (hi > p.pair_cap) {  // the row lost hits to the output cap
        t.status = -1;
        p.out[c] = t;
        return;
    }
    if (n < 3) {
        p.out[c] = t;
        return;
    }
    double sx = 0.0, sy = 0.0, sxx = 0.0, sxy = 0.0, syy = 0.0, sz = 0.0, sxz = 0.0, syz = 0.0;
    for (int64_t k = lo; k < hi; ++k) {
        const int32_t h = p.hidx[k];
        const double a = (double)p.x[h], b = (double)p.y[h];
        const double aa = __dmul_rn(a, a), bb = __dmul_rn(b, b);
        const double z = __dadd_rn(aa, bb);
        sx = __dadd_rn(sx, a);
        sy = __dadd_rn(sy, b);
        sxx = __dadd_rn(sxx, aa);
        sxy = __dadd_rn(sxy, __dmul_rn(a, b));
        syy = __dadd_rn(syy, bb);
        sz = __dadd_rn(sz, z);
        sxz = __dadd_rn(sxz, __dmul_rn(a, z));
        syz = __dadd_rn(syz, __dmul_rn(b, z));
    }
    const double nn = (double)n;
    const double c00 = __dsub_rn(__dmul_rn(syy, nn), __dmul_rn(sy, sy));
    const double c01 = __dsub_rn(__dmul_rn(sxy, nn), __dmul_rn(sy, sx));
    const double c02 = __dsub_rn(__dmul_rn(sxy, sy), __dmul_rn(syy, sx));
    const double det = __dadd_rn(__dsub_rn(__dmul_rn(sxx, c00), __dmul_rn(sxy, c01)), __dmul_rn(sx, c02));
    if (!(det != 0.0)) {
        p.out[c] = t;
        return;
    }
    const double r0 = -sxz, r1 = -syz, r2 = -sz;
    const double m12 = __dsub_rn(__dmul_rn(r1, nn), __dmul_rn(sy, r2));   // r1 n - sy r2
    const double m13 = __dsub_rn(__dmul_rn(r1, sy), __dmul_rn(syy, r2));  // r1 sy - syy r2
    const double m22 = __dsub_rn(__dmul_rn(sxy, r2), __dmul_rn(r1, sx));  // sxy r2 - r1 sx
    const double dD = __dadd_rn(__dsub_rn(__dmul_rn(r0, c00), __dmul_rn(sxy, m12)), __dmul_rn(sx, m13));
    const double dE = __dadd_rn(__dsub_rn(__dmul_rn(sxx, m12), __dmul_rn(r0, c01)), __dmul_rn(sx, m22));
    const double dF = __dadd_rn(__dsub_rn(__dmul_rn(sxx, __dsub_rn(__dmul_rn(syy, r2), __dmul_rn(r1, sy))),
                                          __dmul_rn(sxy, m22)),
                                __dmul_rn(r0, c02));
    const double D = __ddiv_rn(dD, det), E = __ddiv_rn(dE, det), F = __ddiv_rn(dF, det);
    const double cx = __dmul_rn(-0.5, D), cy = __dmul_rn(-0.5, E);
    const double cc = __dadd_rn(__dmul_rn(cx, cx), __dmul_rn(cy, cy));
    const double R2 = __dsub_rn(cc, F);
    const double rho = __dsqrt_rn(cc);
    if (!(R2 > 0.0) || !(rho > 0.0)) {
        p.out[c] = t;
        return;
    }
    const double R = __dsqrt_rn(R2);
    const double kc = __dadd_rn(p.kmin, __dmul_rn(__dadd_rn((double)p.peaks[c].i_kappa, 0.5),
                                                  __ddiv_rn(__dsub_rn(p.kmax, p.kmin), (double)p.nk)));
    const double s = kc >= 0.0 ? 1.0 : -1.0;
    const double nx = __ddiv_rn(__dmul_rn(s, cx), rho), ny = __ddiv_rn(__dmul_rn(s, cy), rho);
    double chi2 = 0.0;
    for (int64_t k = lo; k < hi; ++k) {
        const int32_t h = p.hidx[k];
        const double a = __dsub_rn((double)p.x[h], cx), b = __dsub_rn((double)p.y[h], cy);
        const double r = __dsub_rn(__dsqrt_rn(__dadd_rn(__dmul_rn(a, a), __dmul_rn(b, b))), R);
        chi2 = __dadd_rn(chi2, __dmul_rn(r, r));
    }
    t.status = 1;
    t.cos_phi0 = ny;
    t.sin_phi0 = -nx;
    t.d0 = __dmul_rn(s, __dsub_rn(rho, R));
    t.kappa = __ddiv_rn(s, R);
    t.chi2 = chi2;
    p.out[c] = t;
}

__global__ void fit_kernel(const FitParams p) {
    int64_t n = *p.n_peaks;
    if (n > p.peak_cap) n = p.peak_cap;
    if (n > p.cap) n = p.cap;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n; c += stride) fit_row(p, c);
}

}  // namespace

cudaError_t launch_fit(const FitParams& p, cudaStream_t s) {
    if (p.cap <= 0 || p.peak_cap <= 0) return cudaSuccess;
    const int64_t want = (std::min(p.cap, p.peak_cap) + 255) / 256;
    const int grid = (int)(want < 152 * 16 ? (want > 0 ? want : 1) : 152 * 16);
    fit_kernel<<<grid, 256, 0, s>>>(p);
    return cudaGetLastError();
}

}  // namespace ht
