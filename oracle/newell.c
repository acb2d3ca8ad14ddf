/*
 * Oracle (test infrastructure only; only tests/, __graft_entry__.smoke() and
 * bench.py's CPU baseline may load it): plain CPU implementation of the
 * generalized Newell demagnetization tensor of Sec. 2 of the paper
 * (Eqs. Nxx, F, F2, F_2, Nxy, G, G2, G2_as_g; App. A and App. B).
 *
 * Three evaluations of the same quantity are exported:
 *   - the exact formula in _Float128 ("q"), the reference definition;
 *   - the exact formula in double ("d"), which cancels catastrophically at
 *     distant cells (the paper is silent on this);
 *   - a far-field evaluation in double: tensor-product (composite)
 *     Gauss-Legendre quadrature of the defining volume integral
 *        N_ab = -1/(4 pi |tau|) int_tau int_tau' d_a d_b (1/|r - r'|),
 *     written per axis over the trapezoidal density of the coordinate
 *     difference of the two boxes.  This is not in the paper; it is the
 *     reading this library takes for cells beyond a switch distance.
 * and the "reading" that combines the last two (exact double near, quadrature
 * far), which the GPU path implements independently.
 *
 * Units are arbitrary but common (nm in this project); the tensor is
 * dimensionless.  Build: see oracle/build.py (gcc -O2 -fopenmp, libm).
 */
#define __STDC_WANT_IEC_60559_TYPES_EXT__ 1
#define _GNU_SOURCE 1
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---- the exact formula, in double and in _Float128 ---------------------- */
#define REAL double
#define RSQRT sqrt
#define RASINH asinh
#define RATAN atan
#define RPI 3.14159265358979323846264338327950288
#define SFX _d
#include "newell_impl.h"
#undef REAL
#undef RSQRT
#undef RASINH
#undef RATAN
#undef RPI
#undef SFX

#define REAL _Float128
#define RSQRT sqrtf128
#define RASINH asinhf128
#define RATAN atanf128
#define RPI 3.141592653589793238462643383279502884197f128
#define SFX _q
#include "newell_impl.h"
#undef REAL
#undef RSQRT
#undef RASINH
#undef RATAN
#undef RPI
#undef SFX

/* ---- far-field quadrature (reading; not in the paper) -------------------- */

/* Gauss-Legendre nodes and weights on [-1, 1] by Newton's method on the
 * Legendre polynomial P_n (three-term recurrence). */
static void gauss_legendre(int n, double *x, double *w)
{
    for (int i = 0; i < n; ++i) {
        double z = cos(3.14159265358979323846 * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        /* recompute the derivative at the converged node */
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= n; ++k) {
            double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

#define GL_MAX 16

/* Nodes u and weights W for int du T(u) phi(u), where T is the density of
 * u = xi - xi' with xi uniform on [0, a] (target) and xi' on [0, b] (source),
 * unnormalised: T(u) = |[0,a] intersect [u, u+b]| = min(a, u+b) - max(0, u),
 * supported on [-b, a] and linear on each of its (up to) three pieces.
 * Each piece is cut into equal sub-pieces no wider than wcap (wcap <= 0: no
 * cut), and each sub-piece gets an n-point Gauss-Legendre rule.  Returns the
 * node count; u and W are allocated here (free both). */
static int trapezoid_rule(double a, double b, int n, double wcap, double **u_out, double **W_out,
                          double *widest)
{
    double gx[GL_MAX], gw[GL_MAX];
    gauss_legendre(n, gx, gw);
    double br[4] = {-b, fmin(0.0, a - b), fmax(0.0, a - b), a};
    int cuts[3], total = 0;
    for (int p = 0; p < 3; ++p) {
        double w = br[p + 1] - br[p];
        cuts[p] = w <= 0.0 ? 0 : (wcap > 0.0 ? (int)ceil(w / wcap) : 1);
        if (cuts[p] > 0 && w / cuts[p] > *widest) *widest = w / cuts[p];
        total += cuts[p] * n;
    }
    double *u = (double *)malloc((size_t)total * sizeof(double));
    double *W = (double *)malloc((size_t)total * sizeof(double));
    int m = 0;
    for (int p = 0; p < 3; ++p) {
        for (int c = 0; c < cuts[p]; ++c) {
            double lo = br[p] + (br[p + 1] - br[p]) * c / cuts[p];
            double hi = br[p] + (br[p + 1] - br[p]) * (c + 1) / cuts[p];
            double mid = 0.5 * (lo + hi), half = 0.5 * (hi - lo);
            for (int i = 0; i < n; ++i) {
                double uu = mid + half * gx[i];
                double T = fmin(a, uu + b) - fmax(0.0, uu);
                u[m] = uu;
                W[m] = half * gw[i] * T;
                ++m;
            }
        }
    }
    *u_out = u;
    *W_out = W;
    return m;
}

/* Quadrature of N_ab = -1/(4 pi |tau|) int du dv dw T_x T_y T_z H_ab(X+u, Y+v, Z+w),
 * H_ab(d) = (3 d_a d_b - delta_ab |d|^2) / |d|^5 (the Hessian of 1/|d|). */
static void quadrature_tensor(double X, double Y, double Z, const double t[3], const double s[3],
                              int n, double wcap, double out[6])
{
    double *ux, *wx, *uy, *wy, *uz, *wz, widest = 0.0;
    int mx = trapezoid_rule(t[0], s[0], n, wcap, &ux, &wx, &widest);
    int my = trapezoid_rule(t[1], s[1], n, wcap, &uy, &wy, &widest);
    int mz = trapezoid_rule(t[2], s[2], n, wcap, &uz, &wz, &widest);
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int i = 0; i < mx; ++i)
        for (int j = 0; j < my; ++j)
            for (int k = 0; k < mz; ++k) {
                double d0 = X + ux[i], d1 = Y + uy[j], d2 = Z + uz[k];
                double r2 = d0 * d0 + d1 * d1 + d2 * d2;
                double r = sqrt(r2);
                double w = wx[i] * wy[j] * wz[k] / (r2 * r2 * r);
                acc[0] += w * (3 * d0 * d0 - r2);
                acc[1] += w * (3 * d1 * d1 - r2);
                acc[2] += w * (3 * d2 * d2 - r2);
                acc[3] += w * (3 * d0 * d1);
                acc[4] += w * (3 * d0 * d2);
                acc[5] += w * (3 * d1 * d2);
            }
    free(ux); free(wx); free(uy); free(wy); free(uz); free(wz);
    double scale = -1.0 / (4.0 * 3.14159265358979323846 * t[0] * t[1] * t[2]);
    for (int c = 0; c < 6; ++c) out[c] = acc[c] * scale;
}

/* Distance from the origin to the box of possible differences r - r'
 * (target point minus source point): [X - s, X + t] per axis. */
static double min_separation(double X, double Y, double Z, const double t[3], const double s[3])
{
    double o[3] = {X, Y, Z}, d2 = 0.0;
    for (int k = 0; k < 3; ++k) {
        double lo = o[k] - s[k], hi = o[k] + t[k];
        double c = lo > 0.0 ? lo : (hi < 0.0 ? hi : 0.0);
        d2 += c * c;
    }
    return sqrt(d2);
}

/* The reading for distant cells (not in the paper).  With d = min_separation:
 *   d <  the largest in-plane edge: exact formula in double;
 *   otherwise: quadrature, every linear piece of the difference densities cut
 *   into sub-pieces no wider than d/2, and the node count per sub-piece taken
 *   from rho = d / (widest sub-piece) so that the quadrature error stays near
 *   1e-14 of the largest component (calibrated against the _Float128 formula). */
static int reading_nodes(double rho)
{
    if (rho >= 128.0) return 3;
    if (rho >= 32.0) return 4;
    if (rho >= 11.0) return 5;
    if (rho >= 5.5) return 6;
    if (rho >= 2.75) return 7;
    return 8;
}

static void reading_tensor(double X, double Y, double Z, const double t[3], const double s[3],
                           double out[6])
{
    double d = min_separation(X, Y, Z, t, s);
    double e = fmax(fmax(t[0], t[1]), fmax(s[0], s[1]));
    if (d < e) {
        gen_tensor_d(X, Y, Z, t, s, 0, out);
        return;
    }
    double wcap = 0.5 * d, widest = 0.0;
    for (int k = 0; k < 3; ++k) {
        double br[4] = {-s[k], fmin(0.0, t[k] - s[k]), fmax(0.0, t[k] - s[k]), t[k]};
        for (int p = 0; p < 3; ++p) {
            double w = br[p + 1] - br[p];
            if (w > 0.0) widest = fmax(widest, w / ceil(w / wcap));
        }
    }
    quadrature_tensor(X, Y, Z, t, s, reading_nodes(d / widest), wcap, out);
}

/* ---- exported entry points ---------------------------------------------- */

enum {
    ORACLE_EXACT_Q = 0,      /* exact, _Float128, 64-term form          */
    ORACLE_EXACT_Q_FULL = 1, /* exact, _Float128, 256/128-term form     */
    ORACLE_EXACT_D = 2,      /* exact, double, 64-term form             */
    ORACLE_FARFIELD_D = 3,   /* quadrature, double, n = ORACLE_N arg    */
    ORACLE_READING_D = 4     /* exact double near, quadrature far       */
};

/* One tensor evaluation.  t, s: target and source edge lengths; out[6] =
 * {xx, yy, zz, xy, xz, yz}.  For the "q" modes out_lo (may be NULL) receives
 * the _Float128 result minus its rounding to double.  nquad is used only by
 * ORACLE_FARFIELD_D. */
void oracle_tensor(int mode, double X, double Y, double Z, const double *t, const double *s,
                   int nquad, double *out, double *out_lo)
{
    if (mode == ORACLE_EXACT_Q || mode == ORACLE_EXACT_Q_FULL) {
        _Float128 tq[3] = {t[0], t[1], t[2]}, sq[3] = {s[0], s[1], s[2]}, oq[6];
        gen_tensor_q(X, Y, Z, tq, sq, mode == ORACLE_EXACT_Q_FULL, oq);
        for (int c = 0; c < 6; ++c) {
            out[c] = (double)oq[c];
            if (out_lo) out_lo[c] = (double)(oq[c] - (_Float128)out[c]);
        }
        return;
    }
    if (out_lo) memset(out_lo, 0, 6 * sizeof(double));
    if (mode == ORACLE_EXACT_D) {
        gen_tensor_d(X, Y, Z, t, s, 0, out);
        return;
    }
    if (mode == ORACLE_FARFIELD_D) {
        quadrature_tensor(X, Y, Z, t, s, nquad, 0.0, out);
        return;
    }
    /* ORACLE_READING_D */
    reading_tensor(X, Y, Z, t, s, out);
}

/* One layer pair of oracle_layer_kernels (full offsets): K[6][2ny-1][2nx-1]
 * for target layer i, source layer j. */
void oracle_pair_kernel(int mode, int nx, int ny, double dx, double dy, int L, const double *th, int i,
                        int j, double *K)
{
    double zi = 0.0, zj = 0.0;
    for (int l = 0; l < i; ++l) zi += th[l];
    for (int l = 0; l < j; ++l) zj += th[l];
    int PW = 2 * nx - 1, QH = 2 * ny - 1;
    long long total = (long long)QH * PW;
#pragma omp parallel for schedule(dynamic, 64)
    for (long long e = 0; e < total; ++e) {
        int pi = (int)(e % PW), qi = (int)(e / PW);
        double t[3] = {dx, dy, th[i]}, s[3] = {dx, dy, th[j]};
        double out[6];
        oracle_tensor(mode, (pi - (nx - 1)) * dx, (qi - (ny - 1)) * dy, zi - zj, t, s, 0, out, NULL);
        for (int c = 0; c < 6; ++c) K[((size_t)c * QH + qi) * PW + pi] = out[c];
    }
}

/* Derivative of N(target <- source) along (dtz, dsz, dZ) (target z-edge,
 * source z-edge, z-offset), by a central difference of the exact _Float128
 * formula with step h: truncation O(h^2), rounding ~1e-34 / h. */
void oracle_tensor_dt(double X, double Y, double Z, const double *t, const double *s, double dtz,
                      double dsz, double dZ, double h, double *out)
{
    _Float128 hq = h, op[6], om[6];
    _Float128 tp[3] = {t[0], t[1], (_Float128)t[2] + hq * dtz};
    _Float128 sp[3] = {s[0], s[1], (_Float128)s[2] + hq * dsz};
    _Float128 tm[3] = {t[0], t[1], (_Float128)t[2] - hq * dtz};
    _Float128 sm[3] = {s[0], s[1], (_Float128)s[2] - hq * dsz};
    gen_tensor_q(X, Y, (_Float128)Z + hq * dZ, tp, sp, 0, op);
    gen_tensor_q(X, Y, (_Float128)Z - hq * dZ, tm, sm, 0, om);
    for (int c = 0; c < 6; ++c) out[c] = (double)((op[c] - om[c]) / (2 * hq));
}

/* d/dt_layer of the layer-pair kernels of oracle_layer_kernels (full offsets),
 * from oracle_tensor_dt: the target z-edge moves if i == layer, the source
 * z-edge if j == layer, the offset z_i - z_j by [i > layer] - [j > layer]. */
void oracle_layer_dkernels(int nx, int ny, double dx, double dy, int L, const double *th, int layer,
                           double h, double *K)
{
    double *z = (double *)malloc((size_t)(L + 1) * sizeof(double));
    z[0] = 0.0;
    for (int l = 0; l < L; ++l) z[l + 1] = z[l] + th[l];
    int PW = 2 * nx - 1, QH = 2 * ny - 1;
    long long total = (long long)L * L * QH * PW;
#pragma omp parallel for schedule(dynamic, 16)
    for (long long e = 0; e < total; ++e) {
        int pi = (int)(e % PW);
        long long r = e / PW;
        int qi = (int)(r % QH);
        r /= QH;
        int j = (int)(r % L);
        int i = (int)(r / L);
        double dtz = i == layer, dsz = j == layer, dZ = (double)(i > layer) - (double)(j > layer);
        double out[6] = {0, 0, 0, 0, 0, 0};
        if (dtz != 0 || dsz != 0 || dZ != 0) {
            double t[3] = {dx, dy, th[i]}, s[3] = {dx, dy, th[j]};
            oracle_tensor_dt((pi - (nx - 1)) * dx, (qi - (ny - 1)) * dy, z[i] - z[j], t, s, dtz, dsz,
                             dZ, h, out);
        }
        for (int c = 0; c < 6; ++c)
            K[((((size_t)i * L + j) * 6 + c) * QH + qi) * PW + pi] = out[c];
    }
    free(z);
}

/* f and g with a double-double split of the _Float128 value (hi + lo). */
void oracle_newell_fg_q(int which, double x, double y, double z, double *hi, double *lo)
{
    _Float128 v = which == 0 ? newell_f_q(x, y, z) : newell_g_q(x, y, z);
    *hi = (double)v;
    *lo = (double)(v - (_Float128)*hi);
}

double oracle_newell_fg_d(int which, double x, double y, double z)
{
    return which == 0 ? newell_f_d(x, y, z) : newell_g_d(x, y, z);
}

void oracle_gauss_legendre(int n, double *x, double *w) { gauss_legendre(n, x, w); }

/* Layer-pair convolution kernels of the non-equidistant grid (Sec. 3):
 * for target layer i and source layer j (bottom interfaces z[i], z[j],
 * thicknesses th[i], th[j]) and in-plane offsets p*dx, q*dy,
 *     K[i][j][c][q + qoff][p + poff] = N_c(i <- j)(p dx, q dy, z[i] - z[j])
 * with the target cell (dx, dy, th[i]) and the source cell (dx, dy, th[j]).
 * full=1: p in (-nx, nx), q in (-ny, ny), array [L][L][6][2ny-1][2nx-1].
 * full=0: p in [0, nx),  q in [0, ny),   array [L][L][6][ny][nx].
 * The layers are stacked contiguously from z = 0 (z[0] = 0). */
void oracle_layer_kernels(int mode, int nx, int ny, double dx, double dy, int L,
                          const double *th, int full, double *K)
{
    double *z = (double *)malloc((size_t)(L + 1) * sizeof(double));
    z[0] = 0.0;
    for (int l = 0; l < L; ++l) z[l + 1] = z[l] + th[l];
    int px0 = full ? -(nx - 1) : 0, qy0 = full ? -(ny - 1) : 0;
    int PW = full ? 2 * nx - 1 : nx, QH = full ? 2 * ny - 1 : ny;
    long long total = (long long)L * L * QH * PW;
#pragma omp parallel for schedule(dynamic, 64)
    for (long long e = 0; e < total; ++e) {
        int pi = (int)(e % PW);
        long long r = e / PW;
        int qi = (int)(r % QH);
        r /= QH;
        int j = (int)(r % L);
        int i = (int)(r / L);
        double t[3] = {dx, dy, th[i]}, s[3] = {dx, dy, th[j]};
        double out[6];
        oracle_tensor(mode, (px0 + pi) * dx, (qy0 + qi) * dy, z[i] - z[j], t, s, 0, out, NULL);
        for (int c = 0; c < 6; ++c)
            K[((((size_t)i * L + j) * 6 + c) * QH + qi) * PW + pi] = out[c];
    }
    free(z);
}
