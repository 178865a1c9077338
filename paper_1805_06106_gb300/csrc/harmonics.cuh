// Solid harmonics used by every expansion kernel.
//
// R_n^m (regular) and S_n^m (irregular), defined for all |m| <= n by
//   sum_{n,m} lambda^n mu^m R_n^m(x) = exp(lambda (z + mu w/2 - conj(w)/(2 mu))),  w = x + i y,
//   S_n^m(x) = (n-|m|)! |x|^{-n-1} P_n^|m|(cos theta) e^{i m phi}  (no Condon-Shortley phase),
// with R_n^{-m} = (-1)^m conj R_n^m and S_n^{-m} = (-1)^m conj S_n^m.  They carry the
// paper's harmonics up to constant factors (|x|^n Y_n^m and |x|^{-n-1} Y_n^m of
// eq. spherical-harmonics) and satisfy, for |a| < |b|,
//   1/|a - b| = sum R_n^m(a) conj S_n^m(b)                          (eqn sph-harm)
//   R_n^m(a + b) = sum_{k,l} R_k^l(a) R_{n-k}^{m-l}(b)
//   conj S_n^m(X + y) = sum_{k,l} (-1)^k R_k^l(y) conj S_{n+k}^{m+l}(X),  |y| < |X|
//   (dx - i dy) R_n^m = R_{n-1}^{m-1}, (dx + i dy) R_n^m = -R_{n-1}^{m+1}, dz R_n^m = R_{n-1}^m
//   (dx - i dy) S_n^m = S_{n+1}^{m-1}, (dx + i dy) S_n^m = -S_{n+1}^{m+1}, dz S_n^m = -S_{n+1}^m.
// Both follow three-term recurrences with integer coefficients:
//   R_0^0 = 1, R_m^m = w R_{m-1}^{m-1} / (2m),
//   (n+m)(n-m) R_n^m = (2n-1) z R_{n-1}^m - |x|^2 R_{n-2}^m;
//   S_0^0 = 1/|x|, S_m^m = (2m-1) w S_{m-1}^{m-1} / |x|^2,
//   S_n^m = ((2n-1) z S_{n-1}^m - (n+m-1)(n-m-1) S_{n-2}^m) / |x|^2.
// Coefficients with m >= 0 are stored at tri(n, m) = n(n+1)/2 + m as double2 (re, im).
#pragma once

#include "qbx_internal.cuh"

namespace qbx {

__device__ __forceinline__ double2 cmul(double2 a, double2 b)
{
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }

// value at (n, m) for any m from a table holding m >= 0: X_n^{-m} = (-1)^m conj X_n^m
__device__ __forceinline__ double2 sym_get(const double2 *tab, int n, int m)
{
    if (m >= 0) return tab[tri(n, m)];
    double2 v = tab[tri(n, -m)];
    return (m & 1) ? make_double2(-v.x, v.y) : make_double2(v.x, -v.y);
}

// Regular harmonics R_n^m(x), 0 <= m <= n <= p, into tab (tri layout).
__device__ inline void regular_table(int p, double x, double y, double z, double2 *tab)
{
    double r2 = x * x + y * y + z * z;
    double2 w = make_double2(x, y);
    double2 diag = make_double2(1.0, 0.0);
    for (int m = 0; m <= p; ++m) {
        if (m > 0) diag = cscale(cmul(diag, w), 1.0 / (2.0 * m));
        double2 a2 = make_double2(0.0, 0.0), a1 = diag;
        tab[tri(m, m)] = diag;
        for (int n = m + 1; n <= p; ++n) {
            double inv = 1.0 / ((double)(n + m) * (double)(n - m));
            double2 v = make_double2(((2 * n - 1) * z * a1.x - r2 * a2.x) * inv, ((2 * n - 1) * z * a1.y - r2 * a2.y) * inv);
            tab[tri(n, m)] = v;
            a2 = a1;
            a1 = v;
        }
    }
}

// Irregular harmonics S_n^m(x), 0 <= m <= n <= p, into tab, each row n scaled by scale^n * s0.
__device__ inline void irregular_table(int p, double x, double y, double z, double scale, double s0, double2 *tab)
{
    double r2 = x * x + y * y + z * z;
    double ir2 = 1.0 / r2;
    double rinv = sqrt(ir2);
    double2 wr = make_double2(x * ir2, y * ir2);
    double zz = z * ir2;
    double2 diag = make_double2(rinv * s0, 0.0);
    for (int m = 0; m <= p; ++m) {
        if (m > 0) diag = cscale(cmul(diag, wr), (2.0 * m - 1.0) * scale);
        double2 a2 = make_double2(0.0, 0.0), a1 = diag;
        tab[tri(m, m)] = diag;
        double sn = scale, sn2 = scale * scale;
        for (int n = m + 1; n <= p; ++n) {
            double c1 = (2 * n - 1) * zz * sn, c2 = (double)(n + m - 1) * (double)(n - m - 1) * ir2 * sn2;
            double2 v = make_double2(c1 * a1.x - c2 * a2.x, c1 * a1.y - c2 * a2.y);
            tab[tri(n, m)] = v;
            a2 = a1;
            a1 = v;
        }
    }
}

// Warp-parallel tables: lane m fills columns m, m+32, ... (diagonal by repeated products).
// Row j of the regular table is scaled by scale^j.
__device__ inline void regular_table_warp(int p, double x, double y, double z, double scale, double2 *tab, int lane)
{
    double r2 = x * x + y * y + z * z;
    double2 w = make_double2(x * scale, y * scale);
    double zs = z * scale, r2s = r2 * scale * scale;
    for (int m = lane; m <= p; m += 32) {
        double2 diag = make_double2(1.0, 0.0);
        for (int j = 1; j <= m; ++j) diag = cscale(cmul(diag, w), 1.0 / (2.0 * j));
        double2 a2 = make_double2(0.0, 0.0), a1 = diag;
        tab[tri(m, m)] = diag;
        for (int n = m + 1; n <= p; ++n) {
            double inv = 1.0 / ((double)(n + m) * (double)(n - m));
            double2 v = make_double2(((2 * n - 1) * zs * a1.x - r2s * a2.x) * inv, ((2 * n - 1) * zs * a1.y - r2s * a2.y) * inv);
            tab[tri(n, m)] = v;
            a2 = a1;
            a1 = v;
        }
    }
}

// Row j of the irregular table scaled by scale^j * s0.
__device__ inline void irregular_table_warp(int p, double x, double y, double z, double scale, double s0, double2 *tab,
                                            int lane)
{
    double r2 = x * x + y * y + z * z;
    double ir2 = 1.0 / r2;
    double rinv = sqrt(ir2);
    double2 wr = make_double2(x * ir2 * scale, y * ir2 * scale);
    double zz = z * ir2 * scale, ir2s = ir2 * scale * scale;
    for (int m = lane; m <= p; m += 32) {
        double2 diag = make_double2(rinv * s0, 0.0);
        for (int j = 1; j <= m; ++j) diag = cscale(cmul(diag, wr), 2.0 * j - 1.0);
        double2 a2 = make_double2(0.0, 0.0), a1 = diag;
        tab[tri(m, m)] = diag;
        for (int n = m + 1; n <= p; ++n) {
            double c1 = (2 * n - 1) * zz, c2 = (double)(n + m - 1) * (double)(n - m - 1) * ir2s;
            double2 v = make_double2(c1 * a1.x - c2 * a2.x, c1 * a1.y - c2 * a2.y);
            tab[tri(n, m)] = v;
            a2 = a1;
            a1 = v;
        }
    }
}

}  // namespace qbx
