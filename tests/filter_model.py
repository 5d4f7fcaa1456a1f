"""numpy float32 model of the GPU's staged curvature-bin evaluation.

Restates, for testing only, the float32 arithmetic of the library's stage 1
(float32 estimate with an error bound) and stage 2 (double-float), and the
host-side constants of their bounds, so that the bounds can be checked
against the binary64 oracle on millions of cells without a GPU.  The
reciprocal approximation is modelled as the exact reciprocal scaled by
(1 + rcp_err); the GPU test of the approximation checks |rcp_err| <= 2^-22.
fma(a, b, c) is modelled as a binary64 product (exact for float32 inputs)
plus c, rounded to float32.
"""

import math

import numpy as np

F = np.float32
U = 2.0 ** -24
ER = 2.0 ** -22


def fma(a, b, c):
    return (np.asarray(a, np.float64) * np.asarray(b, np.float64) + np.asarray(c, np.float64)).astype(F)


def consts(grid, d0):
    nk = int(grid.n_kappa)
    kmin, kmax = float(F(grid.kappa_min)), float(F(grid.kappa_max))
    scale = nk / (kmax - kmin)
    Hd = -kmin * scale
    dabs = float(np.max(np.abs(np.asarray(d0, np.float64))))
    V0 = max(abs(Hd), abs(nk - Hd))
    ev = ER + 4 * U + 1 / 63
    m = math.ceil(2 * (ev * (nk + abs(Hd)) + 0.3) / (1 - ev)) + 1
    Vmax = V0 + m
    S2 = float(F(2 * scale))
    K = dict(nk=nk, S2=F(2 * scale), H=F(Hd), dabs=F(dabs), wlo=F(-m), whi=F(nk + m),
             T0=F(2 * ((ER + 3 * U) * Vmax + U * (abs(Hd) + 2 * (nk + m)) + U)),
             cG1=F(2 * (64 / 63) * 4.03 * U * Vmax * (1 + ER) * (1 + ER + 4 * U)),
             cG2=F(2 * 1.01 * S2 * U * (1 + ER)),
             cD1=F(64 * 4.03 * U), cD2=F(3.6 * 1.01 * S2 * U * (1 + ER)))
    V2 = V0 + 2
    K.update(S2hi=F(2 * scale), H_hi=F(Hd))
    K.update(S2lo=F(2 * scale - float(K["S2hi"])), H_lo=F(Hd - float(K["H_hi"])),
             T0b=F(2.0 ** -34 * (V2 + nk + abs(Hd))), cGb1=F(64 * U * U * V2), cGb2=F(20 * U * U * S2),
             cDb=F(2.0 ** -23))
    return K


def stage1(x, y, c, s, d, K, rcp_err=0.0):
    """Returns k >= 0, -1 (no vote) or -2 (undecided), elementwise."""
    x, y, c, s, d = (np.asarray(v, F) for v in (x, y, c, s, d))
    with np.errstate(all="ignore"):
        yy = y * y
        r2 = fma(x, x, yy)
        r = np.sqrt(r2)
        R1 = r + K["dabs"]
        P1 = fma(F(4.02), r, F(2.02) * K["dabs"])
        R1s = R1 * R1
        dmin = np.maximum(K["cD1"] * R1s, K["cD2"] * P1)
        # G >= 0.55 dmin: a cell with den <= dmin gets tau > 1/2 and is never certified
        G = np.maximum(fma(K["cG1"], R1s, K["cG2"] * P1), F(0.55) * dmin)
        q = fma(y, c, -(x * s))
        qs = q * K["S2"]                                   # per (hit, row)
        ds = (d.astype(np.float64) * np.float64(K["S2"])).astype(F)  # table: d * S2 rounded once
        Rj = r2 + d * d
        a = qs - ds
        den = fma(-(d + d), q, Rj)
        rc = (1.0 / den.astype(np.float64) * (1.0 + rcp_err)).astype(F)
        w = fma(a, rc, K["H"])
        tau = fma(G, np.abs(rc), K["T0"])
        lo, hi = w - tau, w + tau
        flo, fhi = np.floor(lo), np.floor(hi)
        denok = den > dmin
        same = (flo == fhi) & np.isfinite(lo) & (np.abs(lo) < 2 ** 22)
        # the implicit den test: a certified cell always has den > dmin
        assert not np.any(same & ~denok), "certified a cell below den_min"
        k = np.where(same, flo, 0).astype(np.int64)
        out = np.full(x.shape, -2, np.int64)
        out[same] = np.where((k[same] >= 0) & (k[same] < K["nk"]), k[same], -1)
        # uncertified cells go to stage 2 unless den > den_min and w lies outside
        # (-m, n_kappa + m), which proves them out of range
        far = ~same & denok & ~((w > K["wlo"]) & (w < K["whi"]))
        out[far] = -1
    return out


def _two_sum(a, b):
    s = a + b
    bb = s - a
    return s, (a - (s - bb)) + (b - bb)


def _two_prod(a, b):
    p = a * b
    return p, fma(a, b, -p)


def stage2(x, y, c, s, d, K, rcp_err=0.0):
    x, y, c, s, d = (np.asarray(v, F) for v in (x, y, c, s, d))
    with np.errstate(all="ignore"):
        r = np.sqrt(fma(x, x, y * y))
        R1 = r + K["dabs"]
        p1, e1 = _two_prod(y, c)
        p2, e2 = _two_prod(x, s)
        s1, t1 = _two_sum(p1, -p2)
        qh, ql = _two_sum(s1, t1 + (e1 - e2))
        s2, t2 = _two_sum(qh, -d)
        ah, al = _two_sum(s2, t2 + ql)
        xx, exx = _two_prod(x, x)
        yy, eyy = _two_prod(y, y)
        dd, edd = _two_prod(d, d)
        d2 = d + d
        mh, me = _two_prod(d2, qh)
        me = fma(d2, ql, me)
        s3, t3 = _two_sum(xx, yy)
        s4, t4 = _two_sum(s3, dd)
        s5, t5 = _two_sum(s4, -mh)
        low = ((exx + eyy) + (edd - me)) + ((t3 + t4) + t5)
        denh, denl = _two_sum(s5, low)
        ok = denh > K["cDb"] * R1 * R1
        rc = (1.0 / denh.astype(np.float64) * (1.0 + rcp_err)).astype(F)
        q1 = ah * rc
        pp, pe = _two_prod(q1, denh)
        rem = fma(-q1, denl, ((ah - pp) - pe) + al)
        q2 = rem * rc
        vh, ve = _two_prod(q1, K["S2hi"])
        ve = fma(q1, K["S2lo"], ve)
        ve = fma(q2, K["S2hi"], ve)
        s6, t6 = _two_sum(vh, K["H_hi"])
        wh, wl = _two_sum(s6, (t6 + ve) + K["H_lo"])
        inwin = (wh > F(-2)) & (wh < F(K["nk"] + 2))
        tau2 = fma(fma(K["cGb1"] * R1, R1, K["cGb2"] * R1), rc, K["T0b"])
        kf = np.floor(wh)
        a0, b0 = _two_sum(wh, -kf)
        dist_lo = a0 + (b0 + wl)
        a1, b1 = _two_sum(kf + F(1), -wh)
        dist_hi = a1 + (b1 - wl)
        neg = dist_lo < 0
        kf = np.where(neg, kf - F(1), kf)
        dist_hi = np.where(neg, -dist_lo, dist_hi)
        dist_lo = np.where(neg, dist_lo + F(1), dist_lo)
        cert = ok & inwin & (dist_lo > tau2) & (dist_hi > tau2)
        out = np.full(x.shape, -2, np.int64)
        kk = np.where(cert, kf, 0).astype(np.int64)
        out[cert] = np.where((kk[cert] >= 0) & (kk[cert] < K["nk"]), kk[cert], -1)
        out[ok & ~inwin] = -1
    return out


# ---- d0 band of a (hit, phi row): a superset of the columns where it can vote

def band_consts(grid, d0):
    """Constants of the band computation (the library's make_consts restated)."""
    nk = int(grid.n_kappa)
    kmin, kmax = float(F(grid.kappa_min)), float(F(grid.kappa_max))
    dk = (kmax - kmin) / nk
    A = kmin - 2 * dk           # widened by two bins each side
    B = kmax + 2 * dk
    d0 = np.asarray(d0, np.float64)
    return dict(A2=F(A * A), B2=F(B * B), iA=F(1.0 / abs(A)), iB=F(1.0 / B), dfirst=F(d0[0]),
                idd=F(grid.n_d0 / (float(F(grid.d0_max)) - float(F(grid.d0_min)))), big=F(1e30))


def band(x, y, c, s, j0, nj, d0, C, tilt=(0, 0, 0, 0)):
    """[jlo, jhi] (inclusive, clipped to the tile [j0, j0 + nj)) in float32; jhi < jlo if empty.

    The kernels take the square roots and the reciprocals approximately (a
    few ulps); `tilt` = signs (-1, 0, +1) by which sqrt(DA), sqrt(DB), a1 and
    b2 are pushed by a relative 2^-20, beyond those errors, so that a test can
    hold the band to the superset property in the adversarial directions."""
    x, y, c, s = (np.asarray(v, F) for v in (x, y, c, s))
    e = [F(1.0 + t * 2.0 ** -20) for t in tilt]
    with np.errstate(all="ignore"):
        r2 = fma(x, x, y * y)
        q = fma(y, c, -(x * s))
        p2 = np.maximum(fma(-q, q, r2), F(0))
        DA = fma(-C["A2"], p2, F(1))
        DB = fma(-C["B2"], p2, F(1))
        sA = np.sqrt(np.maximum(DA, F(0))) * e[0]
        sB = np.sqrt(np.maximum(DB, F(0))) * e[1]
        # forbidden (a1, a2) where kappa < A, [b1, b2] where kappa > B (empty when D <= 0)
        a1 = np.where(DA > 0, (C["A2"] * p2) * C["iA"] / (F(1) + sA) * e[2], C["big"])
        a2 = np.where(DA > 0, (F(1) + sA) * C["iA"], C["big"])
        b2 = np.where(DB > 0, -(C["B2"] * p2) * C["iB"] / (F(1) + sB) * e[3], -C["big"])
        b1 = np.where(DB > 0, -(F(1) + sB) * C["iB"], -C["big"])
        ulo = F(d0[j0]) - q
        uhi = F(d0[j0 + nj - 1]) - q
        lo = np.where(ulo < b1, ulo, np.where((ulo <= a1) & (uhi > b2), np.maximum(ulo, b2),
                                             np.where(uhi >= a2, np.maximum(ulo, a2), C["big"])))
        hi = np.where(uhi >= a2, uhi, np.where((uhi > b2) & (ulo <= a1), np.minimum(uhi, a1),
                                              np.where(ulo < b1, np.minimum(uhi, b1), -C["big"])))
        jl = np.floor((lo + q - C["dfirst"]) * C["idd"]) - 1
        jh = np.floor((hi + q - C["dfirst"]) * C["idd"]) + 2
        jlo = np.clip(jl, j0, j0 + nj).astype(np.int64)
        jhi = np.clip(jh, j0 - 1, j0 + nj - 1).astype(np.int64)
        empty = ~(lo <= hi)
        jlo = np.where(empty, j0 + nj, jlo)
        jhi = np.where(empty, j0 - 1, jhi)
    return jlo, jhi
