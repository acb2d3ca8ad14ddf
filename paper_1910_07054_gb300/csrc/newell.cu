// Generalized Newell demagnetization tensor on the GPU (double precision) and
// the plan's Fourier-space layer tensor.
//
// Sec. 2 of the paper: for a target cuboid (tx, ty, tz) at offset (X, Y, Z)
// from a source cuboid (sx, sy, sz) (offset = target corner - source corner),
//   N_xx = 1/(4 pi tx ty tz) sum_{a,b,c} w_a w_b w_c f(X + a, Y + b, Z + c)
//   N_xy = 1/(4 pi tx ty tz) sum_{a,b,c} w_a w_b w_c g(X + a, Y + b, Z + c)
// with weights (+, -, -, +) on the four shifts of each axis.  The shift sets
// are Eq. Nxx times the splitting of F into F_1 and F_2 (App. A) and Eq. Nxy
// times the splitting of G into G_1 and G_2 (App. B), with F_2 -> f and
// G_2 -> g because the omitted terms cancel (end of Sec. 2.1 and 2.2).  The
// fourth term of Eq. Nxy is taken at Y + Delta y.  The other components follow
// by permuting the axes.
//
// Far from the source the closed form cancels catastrophically in double
// precision; there the same volume integral,
//   N_ab = -1/(4 pi |tau|) int_tau int_tau' d_a d_b (1/|r - r'|),
// is integrated by a composite Gauss-Legendre rule over the trapezoidal
// density of each coordinate difference (a reading not in the paper).
#include <cuda_bf16.h>

#include <cmath>
#include <cstdint>
#include <vector>

#include "fft.cuh"
#include "internal.h"
#include "layout.cuh"

namespace demag {

__constant__ double c_gl_x[kGLMax + 1][kGLMax];
__constant__ double c_gl_w[kGLMax + 1][kGLMax];
__constant__ float c_gl_xf[kGLMax + 1][kGLMax];  // the same rules rounded to float
__constant__ float c_gl_wf[kGLMax + 1][kGLMax];

// Gauss-Legendre nodes from the eigen-decomposition-free Newton iteration on
// P_n, seeded with Tricomi's asymptotic node estimate.
static void gauss_legendre_host(int n, double *x, double *w) {
    const double pi = 3.14159265358979323846;
    for (int k = 1; k <= n; ++k) {
        double th = pi * (4.0 * k - 1.0) / (4.0 * n + 2.0);
        double t = (1.0 - (n - 1.0) / (8.0 * n * n * n)) * std::cos(th);
        double dp = 1.0;
        for (int it = 0; it < 60; ++it) {
            double pm = 1.0, p = t;  // P_0, P_1
            for (int l = 2; l <= n; ++l) {
                double pn = ((2.0 * l - 1.0) * t * p - (l - 1.0) * pm) / l;
                pm = p;
                p = pn;
            }
            dp = n * (pm - t * p) / (1.0 - t * t);  // P_n'(t)
            double step = p / dp;
            t -= step;
            if (std::fabs(step) <= 1e-17) break;
        }
        double pm = 1.0, p = t;
        for (int l = 2; l <= n; ++l) {
            double pn = ((2.0 * l - 1.0) * t * p - (l - 1.0) * pm) / l;
            pm = p;
            p = pn;
        }
        dp = n * (pm - t * p) / (1.0 - t * t);
        x[k - 1] = t;
        w[k - 1] = 2.0 / ((1.0 - t * t) * dp * dp);
    }
}

demag_status upload_gauss_legendre() {
    static bool done[64] = {false};
    int dev = 0;
    DEMAG_CUDA(cudaGetDevice(&dev));
    if (dev < 64 && done[dev]) return DEMAG_OK;
    double hx[kGLMax + 1][kGLMax] = {}, hw[kGLMax + 1][kGLMax] = {};
    for (int n = 1; n <= kGLMax; ++n) gauss_legendre_host(n, hx[n], hw[n]);
    DEMAG_CUDA(cudaMemcpyToSymbol(c_gl_x, hx, sizeof(hx)));
    DEMAG_CUDA(cudaMemcpyToSymbol(c_gl_w, hw, sizeof(hw)));
    float fx[kGLMax + 1][kGLMax] = {}, fw[kGLMax + 1][kGLMax] = {};
    for (int n = 0; n <= kGLMax; ++n)
        for (int i = 0; i < kGLMax; ++i) {
            fx[n][i] = (float)hx[n][i];
            fw[n][i] = (float)hw[n][i];
        }
    DEMAG_CUDA(cudaMemcpyToSymbol(c_gl_xf, fx, sizeof(fx)));
    DEMAG_CUDA(cudaMemcpyToSymbol(c_gl_wf, fw, sizeof(fw)));
    if (dev < 64) done[dev] = true;
    return DEMAG_OK;
}

// ---- closed form (Sec. 2) ------------------------------------------------
//
// Written once for a scalar type S: double, or Dual (value and first
// derivative along one direction of the arguments) for d/dt of the tensor.

struct Dual {
    double v, d;
};
__device__ __forceinline__ Dual operator+(Dual a, Dual b) { return {a.v + b.v, a.d + b.d}; }
__device__ __forceinline__ Dual operator-(Dual a, Dual b) { return {a.v - b.v, a.d - b.d}; }
__device__ __forceinline__ Dual operator-(Dual a) { return {-a.v, -a.d}; }
__device__ __forceinline__ Dual operator*(Dual a, Dual b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }
__device__ __forceinline__ Dual operator*(double a, Dual b) { return {a * b.v, a * b.d}; }
__device__ __forceinline__ Dual operator/(Dual a, Dual b) {
    const double q = a.v / b.v;
    return {q, (a.d - q * b.d) / b.v};
}
__device__ __forceinline__ Dual operator/(Dual a, double b) { return {a.v / b, a.d / b}; }
__device__ __forceinline__ Dual &operator+=(Dual &a, Dual b) { a = a + b; return a; }
__device__ __forceinline__ Dual &operator-=(Dual &a, Dual b) { a = a - b; return a; }

__device__ __forceinline__ double val(double a) { return a; }
__device__ __forceinline__ double val(Dual a) { return a.v; }
__device__ __forceinline__ double s_sqrt(double a) { return sqrt(a); }
__device__ __forceinline__ Dual s_sqrt(Dual a) {
    const double r = sqrt(a.v);
    return {r, r > 0.0 ? a.d / (2.0 * r) : 0.0};
}
__device__ __forceinline__ double s_asinh(double a) { return asinh(a); }
__device__ __forceinline__ Dual s_asinh(Dual a) { return {asinh(a.v), a.d / sqrt(1.0 + a.v * a.v)}; }
__device__ __forceinline__ double s_atan(double a) { return atan(a); }
__device__ __forceinline__ Dual s_atan(Dual a) { return {atan(a.v), a.d / (1.0 + a.v * a.v)}; }
template <typename S> __device__ __forceinline__ S s_const(double c);
template <> __device__ __forceinline__ double s_const<double>(double c) { return c; }
template <> __device__ __forceinline__ Dual s_const<Dual>(double c) { return {c, 0.0}; }

// Newell f: d^2/dy^2 d^2/dz^2 f = 1/R.  Products with a vanishing prefactor
// are dropped (their limit, and that of their derivative, is zero).
template <typename S>
__device__ __noinline__ S newell_f(S x, S y, S z) {
    const S x2 = x * x, y2 = y * y, z2 = z * z;
    const S R = s_sqrt(x2 + y2 + z2);
    S v = (2.0 * x2 - y2 - z2) * R / 6.0;
    const S xz = x2 + z2, xy = x2 + y2;
    if (val(y) != 0.0 && val(xz) > 0.0) v += 0.5 * (y * (z2 - x2) * s_asinh(y / s_sqrt(xz)));
    if (val(z) != 0.0 && val(xy) > 0.0) v += 0.5 * (z * (y2 - x2) * s_asinh(z / s_sqrt(xy)));
    if (val(x) != 0.0 && val(y) != 0.0 && val(z) != 0.0) v -= x * y * z * s_atan(y * z / (x * R));
    return v;
}

// Newell g: d/dx d/dy d^2/dz^2 g = 1/R.
template <typename S>
__device__ __noinline__ S newell_g(S x, S y, S z) {
    const S x2 = x * x, y2 = y * y, z2 = z * z;
    const S R = s_sqrt(x2 + y2 + z2);
    S v = -(x * y * R) / 3.0;
    if (val(y) != 0.0) v += y * (3.0 * z2 - y2) * s_asinh(x / s_sqrt(y2 + z2)) / 6.0;
    if (val(x) != 0.0) v += x * (3.0 * z2 - x2) * s_asinh(y / s_sqrt(x2 + z2)) / 6.0;
    if (val(x) != 0.0 && val(y) != 0.0 && val(z) != 0.0) {
        v += x * y * z * s_asinh(z / s_sqrt(x2 + y2));
        v -= z2 * z * s_atan(x * y / (z * R)) / 6.0;
        v -= 0.5 * (z * y2 * s_atan(x * z / (y * R)));
        v -= 0.5 * (z * x2 * s_atan(y * z / (x * R)));
    }
    return v;
}

constexpr double kPi = 3.14159265358979323846;

// N_xx: x-face pairs (Eq. Nxx) x F split into F_1 (y) and F_2 (z) (App. A).
template <typename S>
__device__ __noinline__ S closed_nxx(S X, S Y, S Z, S tx, S ty, S tz, S sx, S sy, S sz) {
    const S zero = s_const<S>(0.0);
    const S sxa[4] = {zero, tx, -sx, tx - sx};
    const S sya[4] = {ty, zero, ty - sy, -sy};
    const S sza[4] = {tz, zero, tz - sz, -sz};
    S acc = zero;
#pragma unroll 1
    for (int a = 0; a < 4; ++a) {
        S ya = zero;
#pragma unroll 1
        for (int b = 0; b < 4; ++b) {
            S zb = zero;
#pragma unroll 1
            for (int c = 0; c < 4; ++c) {
                const S v = newell_f<S>(X + sxa[a], Y + sya[b], Z + sza[c]);
                if (c == 0 || c == 3) zb += v; else zb -= v;
            }
            if (b == 0 || b == 3) ya += zb; else ya -= zb;
        }
        if (a == 0 || a == 3) acc += ya; else acc -= ya;
    }
    return acc / (4.0 * kPi * (tx * ty * tz));
}

// N_xy: target/source face pairs of Eq. Nxy (fourth term at Y + Delta y) x G
// split over x and y (App. B) x G_1 over z.
template <typename S>
__device__ __noinline__ S closed_nxy(S X, S Y, S Z, S tx, S ty, S tz, S sx, S sy, S sz) {
    const S zero = s_const<S>(0.0);
    const S sxa[4] = {tx, zero, tx - sx, -sx};
    const S sya[4] = {zero, -sy, ty, ty - sy};
    const S sza[4] = {tz, zero, tz - sz, -sz};
    S acc = zero;
#pragma unroll 1
    for (int a = 0; a < 4; ++a) {
        S ya = zero;
#pragma unroll 1
        for (int b = 0; b < 4; ++b) {
            S zb = zero;
#pragma unroll 1
            for (int c = 0; c < 4; ++c) {
                const S v = newell_g<S>(X + sxa[a], Y + sya[b], Z + sza[c]);
                if (c == 0 || c == 3) zb += v; else zb -= v;
            }
            if (b == 0 || b == 3) ya += zb; else ya -= zb;
        }
        if (a == 0 || a == 3) acc += ya; else acc -= ya;
    }
    return acc / (4.0 * kPi * (tx * ty * tz));
}

// All six components: N_yy, N_zz from N_xx and N_xz, N_yz from N_xy by axis
// permutation (Sec. 2).  out = {xx, yy, zz, xy, xz, yz}.
template <typename S>
__device__ void closed_tensor(S X, S Y, S Z, const S t[3], const S s[3], S out[6]) {
    out[0] = closed_nxx<S>(X, Y, Z, t[0], t[1], t[2], s[0], s[1], s[2]);
    out[1] = closed_nxx<S>(Y, X, Z, t[1], t[0], t[2], s[1], s[0], s[2]);
    out[2] = closed_nxx<S>(Z, Y, X, t[2], t[1], t[0], s[2], s[1], s[0]);
    out[3] = closed_nxy<S>(X, Y, Z, t[0], t[1], t[2], s[0], s[1], s[2]);
    out[4] = closed_nxy<S>(X, Z, Y, t[0], t[2], t[1], s[0], s[2], s[1]);
    out[5] = closed_nxy<S>(Z, Y, X, t[2], t[1], t[0], s[2], s[1], s[0]);
}

// ---- far field: composite Gauss-Legendre quadrature -----------------------

// Difference density of one axis: u = xi - xi', xi on [0, a] (target),
// xi' on [0, b] (source); T(u) = min(a, u + b) - max(0, u) on [-b, a], linear on
// three pieces, each cut into `cuts` equal sub-pieces of n nodes.
constexpr int kAxisMax = 48;  // double quadrature: node arrays up to this count per axis

struct AxisRule {
    double a, b;
    double br[4];
    double len[3];  // sub-piece length of each piece
    int cuts[3];
    int count;  // total nodes
};

__device__ void axis_rule(AxisRule &r, double a, double b, double wcap, int n) {
    r.a = a;
    r.b = b;
    r.br[0] = -b;
    r.br[1] = fmin(0.0, a - b);
    r.br[2] = fmax(0.0, a - b);
    r.br[3] = a;
    r.count = 0;
    for (int p = 0; p < 3; ++p) {
        const double w = r.br[p + 1] - r.br[p];
        r.cuts[p] = w > 0.0 ? (int)ceil(w / wcap) : 0;
        r.len[p] = r.cuts[p] > 0 ? w / r.cuts[p] : 0.0;
        r.count += r.cuts[p] * n;
    }
}

__device__ __forceinline__ void axis_node(const AxisRule &r, int n, int k, double &u, double &W) {
    int p = 0;
    int per = r.cuts[0] * n;
    while (k >= per) {  // at most two steps
        k -= per;
        ++p;
        per = r.cuts[p] * n;
    }
    const int c = k / n, i = k - c * n;
    const double len = r.len[p];
    const double lo = r.br[p] + len * c;
    const double half = 0.5 * len;
    u = lo + half + half * c_gl_x[n][i];
    const double T = fmin(r.a, u + r.b) - fmax(0.0, u);
    W = half * c_gl_w[n][i] * T;
}

__device__ void quadrature_tensor(double X, double Y, double Z, const double t[3],
                                  const double s[3], int n, double wcap, double out[6]) {
    AxisRule rx, ry, rz;
    axis_rule(rx, t[0], s[0], wcap, n);
    axis_rule(ry, t[1], s[1], wcap, n);
    axis_rule(rz, t[2], s[2], wcap, n);
    double hxx = 0, hyy = 0, hzz = 0, hxy = 0, hxz = 0, hyz = 0;
    if (rx.count <= kAxisMax && ry.count <= kAxisMax && rz.count <= kAxisMax) {
        // each axis's nodes once (the same values the loops below compute per use)
        double xd[kAxisMax], xw[kAxisMax], yd[kAxisMax], yw[kAxisMax], zd[kAxisMax], zw[kAxisMax];
        for (int k = 0; k < rx.count; ++k) {
            double u;
            axis_node(rx, n, k, u, xw[k]);
            xd[k] = X + u;
        }
        for (int k = 0; k < ry.count; ++k) {
            double u;
            axis_node(ry, n, k, u, yw[k]);
            yd[k] = Y + u;
        }
        for (int k = 0; k < rz.count; ++k) {
            double u;
            axis_node(rz, n, k, u, zw[k]);
            zd[k] = Z + u;
        }
        for (int kx = 0; kx < rx.count; ++kx) {
            const double dxv = xd[kx], wx = xw[kx];
            for (int ky = 0; ky < ry.count; ++ky) {
                const double dyv = yd[ky];
                const double wxy = wx * yw[ky];
                for (int kz = 0; kz < rz.count; ++kz) {
                    const double dzv = zd[kz], wz = zw[kz];
                    const double r2 = dxv * dxv + dyv * dyv + dzv * dzv;
                    const double ir = 1.0 / sqrt(r2);
                    const double ir2 = ir * ir;
                    const double q = wxy * wz * ir * ir2 * ir2;  // weight / r^5
                    const double q3 = 3.0 * q;
                    hxx += q3 * dxv * dxv - q * r2;
                    hyy += q3 * dyv * dyv - q * r2;
                    hzz += q3 * dzv * dzv - q * r2;
                    hxy += q3 * dxv * dyv;
                    hxz += q3 * dxv * dzv;
                    hyz += q3 * dyv * dzv;
                }
            }
        }
    } else
    for (int kx = 0; kx < rx.count; ++kx) {
        double ux, wx;
        axis_node(rx, n, kx, ux, wx);
        const double dxv = X + ux;
        for (int ky = 0; ky < ry.count; ++ky) {
            double uy, wy;
            axis_node(ry, n, ky, uy, wy);
            const double dyv = Y + uy;
            const double wxy = wx * wy;
            for (int kz = 0; kz < rz.count; ++kz) {
                double uz, wz;
                axis_node(rz, n, kz, uz, wz);
                const double dzv = Z + uz;
                const double r2 = dxv * dxv + dyv * dyv + dzv * dzv;
                const double ir = 1.0 / sqrt(r2);
                const double ir2 = ir * ir;
                const double q = wxy * wz * ir * ir2 * ir2;  // weight / r^5
                const double q3 = 3.0 * q;
                hxx += q3 * dxv * dxv - q * r2;
                hyy += q3 * dyv * dyv - q * r2;
                hzz += q3 * dzv * dzv - q * r2;
                hxy += q3 * dxv * dyv;
                hxz += q3 * dxv * dzv;
                hyz += q3 * dyv * dzv;
            }
        }
    }
    const double sc = -1.0 / (4.0 * kPi * t[0] * t[1] * t[2]);
    out[0] = hxx * sc;
    out[1] = hyy * sc;
    out[2] = hzz * sc;
    out[3] = hxy * sc;
    out[4] = hxz * sc;
    out[5] = hyz * sc;
}

// Node count per sub-piece from rho = gap / widest sub-piece, calibrated so
// that the quadrature error stays near 1e-14 of the largest component.
__device__ __forceinline__ int far_nodes(double rho) {
    return rho >= 128.0 ? 3 : rho >= 32.0 ? 4 : rho >= 11.0 ? 5 : rho >= 5.5 ? 6 : rho >= 2.75 ? 7 : 8;
}

constexpr int kF32AxisMax = 64;

// The far-field quadrature of quadrature_tensor entirely in float (node
// counts, sub-pieces, nodes and sums): for float plans, whose stored tensor
// carries float rounding anyway, and because double arithmetic runs at a small
// fraction of the float rate.  Node counts for ~3e-8 of the largest component.
// Returns false (nothing written) if an axis needs more than kF32AxisMax nodes.
struct AxisRuleF {
    float a, b, br[4], len[3];
    int cuts[3], count;
};

__device__ __forceinline__ void axis_rule_f(AxisRuleF &r, float a, float b, float inv_wcap, int n) {
    r.a = a;
    r.b = b;
    r.br[0] = -b;
    r.br[1] = fminf(0.f, a - b);
    r.br[2] = fmaxf(0.f, a - b);
    r.br[3] = a;
    r.count = 0;
    for (int p = 0; p < 3; ++p) {
        const float w = r.br[p + 1] - r.br[p];
        r.cuts[p] = w > 0.f ? (int)ceilf(w * inv_wcap) : 0;
        r.len[p] = r.cuts[p] > 0 ? w / (float)r.cuts[p] : 0.f;
        r.count += r.cuts[p] * n;
    }
}

// All nodes of one axis: positions off + u and weights (Gauss-Legendre on each
// sub-piece times the difference density T(u)).
__device__ __forceinline__ void axis_nodes_f(const AxisRuleF &r, int n, float off, float *d, float *w) {
    int k = 0;
    for (int p = 0; p < 3; ++p)
        for (int c = 0; c < r.cuts[p]; ++c) {
            const float half = 0.5f * r.len[p];
            const float mid = r.br[p] + r.len[p] * (float)c + half;
            for (int i = 0; i < n; ++i, ++k) {
                const float u = mid + half * c_gl_xf[n][i];
                const float T = fminf(r.a, u + r.b) - fmaxf(0.f, u);
                d[k] = off + u;
                w[k] = half * c_gl_wf[n][i] * T;
            }
        }
}

// Nodes per sub-piece of the float quadrature from rho = gap / widest sub-piece
// (sub-pieces no wider than half the gap).
__device__ __forceinline__ int f32_nodes(const float tf[3], const float sf[3], float gapf, float inv_wcap) {
    float widest = 0.f;
    for (int k = 0; k < 3; ++k) {
        const float br0 = -sf[k], br1 = fminf(0.f, tf[k] - sf[k]), br2 = fmaxf(0.f, tf[k] - sf[k]), br3 = tf[k];
        const float ws[3] = {br1 - br0, br2 - br1, br3 - br2};
        for (int p = 0; p < 3; ++p)
            if (ws[p] > 0.f) widest = fmaxf(widest, ws[p] / ceilf(ws[p] * inv_wcap));
    }
    const float rho = gapf / widest;
    return rho >= 64.f ? 2 : rho >= 11.f ? 3 : rho >= 4.f ? 4 : rho >= 2.75f ? 5 : 6;
}

__device__ bool quadrature_tensor_f32(double Xd, double Yd, double Zd, const double t[3], const double s[3],
                                      double gap, double out[6]) {
    const float tf[3] = {(float)t[0], (float)t[1], (float)t[2]};
    const float sf[3] = {(float)s[0], (float)s[1], (float)s[2]};
    const float gapf = (float)gap, wcap = 0.5f * gapf, inv_wcap = 1.f / wcap;
    const int n = f32_nodes(tf, sf, gapf, inv_wcap);
    AxisRuleF rx, ry, rz;
    axis_rule_f(rx, tf[0], sf[0], inv_wcap, n);
    axis_rule_f(ry, tf[1], sf[1], inv_wcap, n);
    axis_rule_f(rz, tf[2], sf[2], inv_wcap, n);
    if (rx.count > kF32AxisMax || ry.count > kF32AxisMax || rz.count > kF32AxisMax) return false;
    float xd[kF32AxisMax], xw[kF32AxisMax], yd[kF32AxisMax], yw[kF32AxisMax], zd[kF32AxisMax], zw[kF32AxisMax];
    axis_nodes_f(rx, n, (float)Xd, xd, xw);
    axis_nodes_f(ry, n, (float)Yd, yd, yw);
    axis_nodes_f(rz, n, (float)Zd, zd, zw);
    float hxx = 0.f, hyy = 0.f, hzz = 0.f, hxy = 0.f, hxz = 0.f, hyz = 0.f;
    for (int kx = 0; kx < rx.count; ++kx) {
        const float dxv = xd[kx], wx = xw[kx];
        for (int ky = 0; ky < ry.count; ++ky) {
            const float dyv = yd[ky];
            const float wxy = wx * yw[ky];
            const float rxy = dxv * dxv + dyv * dyv;
            for (int kz = 0; kz < rz.count; ++kz) {
                const float dzv = zd[kz];
                const float r2 = rxy + dzv * dzv;
                const float ir = rsqrtf(r2);
                const float ir2 = ir * ir;
                const float q = wxy * zw[kz] * ir * ir2 * ir2;
                const float q3 = 3.f * q;
                hxx += q3 * dxv * dxv - q * r2;
                hyy += q3 * dyv * dyv - q * r2;
                hzz += q3 * dzv * dzv - q * r2;
                hxy += q3 * dxv * dyv;
                hxz += q3 * dxv * dzv;
                hyz += q3 * dyv * dzv;
            }
        }
    }
    const double sc = -1.0 / (4.0 * kPi * t[0] * t[1] * t[2]);
    out[0] = hxx * sc;
    out[1] = hyy * sc;
    out[2] = hzz * sc;
    out[3] = hxy * sc;
    out[4] = hxz * sc;
    out[5] = hyz * sc;
    return true;
}

// Distance between the two cuboids; true when it is below the larger in-plane
// edge (the closed form applies there, the quadrature beyond).
__device__ __forceinline__ bool near_pair(double X, double Y, double Z, const double t[3], const double s[3],
                                          double &gap) {
    const double o[3] = {X, Y, Z};
    double gap2 = 0.0;
    for (int k = 0; k < 3; ++k) {
        const double lo = o[k] - s[k], hi = o[k] + t[k];
        const double c = lo > 0.0 ? lo : (hi < 0.0 ? hi : 0.0);
        gap2 += c * c;
    }
    gap = sqrt(gap2);
    return gap < fmax(fmax(t[0], t[1]), fmax(s[0], s[1]));
}

// The evaluation used everywhere: closed form while the gap between the two
// cuboids is below the larger in-plane edge, quadrature (sub-pieces no wider
// than half the gap) beyond.  With skip_near, near offsets are left to the
// warp-parallel closed form of k_near_planes (returns false, nothing written).
__device__ bool tensor_eval(double X, double Y, double Z, const double t[3], const double s[3],
                            double out[6], bool far32 = false, bool skip_near = false) {
    double gap;
    if (near_pair(X, Y, Z, t, s, gap)) {
        if (skip_near) return false;
        closed_tensor<double>(X, Y, Z, t, s, out);
        return true;
    }
    if (far32 && quadrature_tensor_f32(X, Y, Z, t, s, gap, out)) return true;
    const double wcap = 0.5 * gap;
    double widest = 0.0;
    for (int k = 0; k < 3; ++k) {
        const double br0 = -s[k], br1 = fmin(0.0, t[k] - s[k]), br2 = fmax(0.0, t[k] - s[k]),
                     br3 = t[k];
        const double ws[3] = {br1 - br0, br2 - br1, br3 - br2};
        for (int p = 0; p < 3; ++p)
            if (ws[p] > 0.0) widest = fmax(widest, ws[p] / ceil(ws[p] / wcap));
    }
    quadrature_tensor(X, Y, Z, t, s, far_nodes(gap / widest), wcap, out);
    return true;
}

// ---- d/dt of the tensor ----------------------------------------------------
//
// Derivative of N(target <- source) along (dtz, dsz, dZ): target z-edge, source
// z-edge and z-offset (the in-plane quantities are fixed).  Near pairs: the
// closed form in Dual arithmetic.  Far pairs: differentiating the volume
// integral itself.  With I(a, b, Z) = int dw T(w; a, b) Phi(Z + w), T the
// z-difference density of edges a (target) and b (source) and Phi the in-plane
// integral of the Hessian of 1/r,
//   dI/da = int_{a-b}^{a} Phi,   dI/db = int_{-b}^{a-b} Phi,
//   dI/dZ = int_{max(0,a-b)}^{a} Phi - int_{-b}^{min(0,a-b)} Phi
// (dT/da, dT/db are indicators; dI/dZ by parts with dT/dw = +1, 0, -1 on the
// three pieces), and N = -I / (4 pi |tau|) adds -N dtz / tz.

// Plain composite Gauss-Legendre rule on [lo, hi], sub-pieces <= wcap.
struct IntervalRule {
    double lo, len;
    int cuts, count;
};

__device__ void interval_rule(IntervalRule &r, double lo, double hi, double wcap, int n) {
    r.lo = lo;
    const double w = hi - lo;
    r.cuts = w > 0.0 ? (int)ceil(w / wcap) : 0;
    r.len = r.cuts > 0 ? w / r.cuts : 0.0;
    r.count = r.cuts * n;
}

__device__ __forceinline__ void interval_node(const IntervalRule &r, int n, int k, double &u, double &W) {
    const int c = k / n, i = k - c * n;
    const double half = 0.5 * r.len;
    u = r.lo + r.len * c + half + half * c_gl_x[n][i];
    W = half * c_gl_w[n][i];
}

__device__ void quadrature_tensor_dt(double X, double Y, double Z, const double t[3],
                                     const double s[3], int n, double wcap, double dtz, double dsz,
                                     double dZ, double out[6], double dout[6]) {
    AxisRule rx, ry, rz;
    axis_rule(rx, t[0], s[0], wcap, n);
    axis_rule(ry, t[1], s[1], wcap, n);
    axis_rule(rz, t[2], s[2], wcap, n);
    const double a = t[2], b = s[2];
    // derivative intervals and their coefficients
    IntervalRule ir[4];
    double coef[4];
    interval_rule(ir[0], a - b, a, wcap, n);
    coef[0] = dtz;
    interval_rule(ir[1], -b, a - b, wcap, n);
    coef[1] = dsz;
    interval_rule(ir[2], fmax(0.0, a - b), a, wcap, n);
    coef[2] = dZ;
    interval_rule(ir[3], -b, fmin(0.0, a - b), wcap, n);
    coef[3] = -dZ;
    double h[6] = {0, 0, 0, 0, 0, 0}, dh[6] = {0, 0, 0, 0, 0, 0};
    for (int kx = 0; kx < rx.count; ++kx) {
        double ux, wx;
        axis_node(rx, n, kx, ux, wx);
        const double dxv = X + ux;
        for (int ky = 0; ky < ry.count; ++ky) {
            double uy, wy;
            axis_node(ry, n, ky, uy, wy);
            const double dyv = Y + uy;
            const double wxy = wx * wy;
            // value: trapezoid-weighted nodes; derivative: interval nodes
            for (int part = 0; part < 5; ++part) {
                if (part > 0 && coef[part - 1] == 0.0) continue;
                const int cnt = part == 0 ? rz.count : ir[part - 1].count;
                for (int kz = 0; kz < cnt; ++kz) {
                    double uz, wz;
                    if (part == 0)
                        axis_node(rz, n, kz, uz, wz);
                    else {
                        interval_node(ir[part - 1], n, kz, uz, wz);
                        wz *= coef[part - 1];
                    }
                    const double dzv = Z + uz;
                    const double r2 = dxv * dxv + dyv * dyv + dzv * dzv;
                    const double ir1 = 1.0 / sqrt(r2);
                    const double ir2 = ir1 * ir1;
                    const double q = wxy * wz * ir1 * ir2 * ir2;
                    const double q3 = 3.0 * q;
                    double *acc = part == 0 ? h : dh;
                    acc[0] += q3 * dxv * dxv - q * r2;
                    acc[1] += q3 * dyv * dyv - q * r2;
                    acc[2] += q3 * dzv * dzv - q * r2;
                    acc[3] += q3 * dxv * dyv;
                    acc[4] += q3 * dxv * dzv;
                    acc[5] += q3 * dyv * dzv;
                }
            }
        }
    }
    const double sc = -1.0 / (4.0 * kPi * t[0] * t[1] * t[2]);
    for (int c = 0; c < 6; ++c) {
        out[c] = h[c] * sc;
        dout[c] = dh[c] * sc - out[c] * dtz / t[2];
    }
}

// The derivative of quadrature_tensor_dt entirely in float, with the node
// counts of quadrature_tensor_f32, for float plans.  dN = sc (dI - I dtz / tz)
// is linear in the node weights, so the trapezoid-weighted z nodes of I (scaled
// by -dtz / tz) and the derivative-interval nodes of dI form one z list and one
// sum.  Returns false (nothing written) if an axis needs more than kF32AxisMax
// nodes or the z list more than 2 kF32AxisMax.
__device__ bool quadrature_tensor_dt_f32(double Xd, double Yd, double Zd, const double t[3], const double s[3],
                                         double gap, double dtz, double dsz, double dZ, double dout[6]) {
    const float tf[3] = {(float)t[0], (float)t[1], (float)t[2]};
    const float sf[3] = {(float)s[0], (float)s[1], (float)s[2]};
    const float gapf = (float)gap, wcap = 0.5f * gapf, inv_wcap = 1.f / wcap;
    const int n = f32_nodes(tf, sf, gapf, inv_wcap);
    AxisRuleF rx, ry, rz;
    axis_rule_f(rx, tf[0], sf[0], inv_wcap, n);
    axis_rule_f(ry, tf[1], sf[1], inv_wcap, n);
    if (rx.count > kF32AxisMax || ry.count > kF32AxisMax) return false;
    float xd[kF32AxisMax], xw[kF32AxisMax], yd[kF32AxisMax], yw[kF32AxisMax];
    float zd[2 * kF32AxisMax], zw[2 * kF32AxisMax];
    int nz = 0;
    const float a = tf[2], b = sf[2], Zf = (float)Zd;
    if (dtz != 0.0) {
        axis_rule_f(rz, a, b, inv_wcap, n);
        if (rz.count > kF32AxisMax) return false;
        axis_nodes_f(rz, n, Zf, zd, zw);
        const float f = (float)(-dtz / t[2]);
        for (int k = 0; k < rz.count; ++k) zw[k] *= f;
        nz = rz.count;
    }
    // dI/da, dI/db and dI/dZ as plain integrals of Phi over sub-intervals of [-b, a]
    const float lo[4] = {a - b, -b, fmaxf(0.f, a - b), -b};
    const float hi[4] = {a, a - b, a, fminf(0.f, a - b)};
    const float cf[4] = {(float)dtz, (float)dsz, (float)dZ, (float)-dZ};
    for (int iv = 0; iv < 4; ++iv) {
        const float w = hi[iv] - lo[iv];
        if (cf[iv] == 0.f || !(w > 0.f)) continue;
        const int cuts = (int)ceilf(w * inv_wcap);
        if (nz + cuts * n > 2 * kF32AxisMax) return false;
        const float len = w / (float)cuts, half = 0.5f * len;
        for (int c = 0; c < cuts; ++c) {
            const float mid = lo[iv] + len * (float)c + half;
            for (int i = 0; i < n; ++i, ++nz) {
                zd[nz] = Zf + mid + half * c_gl_xf[n][i];
                zw[nz] = half * c_gl_wf[n][i] * cf[iv];
            }
        }
    }
    axis_nodes_f(rx, n, (float)Xd, xd, xw);
    axis_nodes_f(ry, n, (float)Yd, yd, yw);
    float hxx = 0.f, hyy = 0.f, hzz = 0.f, hxy = 0.f, hxz = 0.f, hyz = 0.f;
    for (int kx = 0; kx < rx.count; ++kx) {
        const float dxv = xd[kx], wx = xw[kx];
        for (int ky = 0; ky < ry.count; ++ky) {
            const float dyv = yd[ky];
            const float wxy = wx * yw[ky];
            const float rxy = dxv * dxv + dyv * dyv;
            for (int kz = 0; kz < nz; ++kz) {
                const float dzv = zd[kz];
                const float r2 = rxy + dzv * dzv;
                const float ir = rsqrtf(r2);
                const float ir2 = ir * ir;
                const float q = wxy * zw[kz] * ir * ir2 * ir2;
                const float q3 = 3.f * q;
                hxx += q3 * dxv * dxv - q * r2;
                hyy += q3 * dyv * dyv - q * r2;
                hzz += q3 * dzv * dzv - q * r2;
                hxy += q3 * dxv * dyv;
                hxz += q3 * dxv * dzv;
                hyz += q3 * dyv * dzv;
            }
        }
    }
    const double sc = -1.0 / (4.0 * kPi * t[0] * t[1] * t[2]);
    dout[0] = hxx * sc;
    dout[1] = hyy * sc;
    dout[2] = hzz * sc;
    dout[3] = hxy * sc;
    dout[4] = hxz * sc;
    dout[5] = hyz * sc;
    return true;
}

// Value and derivative of the evaluation used everywhere (tensor_eval).  With
// far32, far offsets take quadrature_tensor_dt_f32 and only dout is written.
__device__ void tensor_eval_dt(double X, double Y, double Z, const double t[3], const double s[3],
                               double dtz, double dsz, double dZ, double out[6], double dout[6],
                               bool far32 = false) {
    const double o[3] = {X, Y, Z};
    double gap2 = 0.0;
    for (int k = 0; k < 3; ++k) {
        const double lo = o[k] - s[k], hi = o[k] + t[k];
        const double c = lo > 0.0 ? lo : (hi < 0.0 ? hi : 0.0);
        gap2 += c * c;
    }
    const double gap = sqrt(gap2);
    const double e = fmax(fmax(t[0], t[1]), fmax(s[0], s[1]));
    if (gap < e) {
        const Dual td[3] = {{t[0], 0.0}, {t[1], 0.0}, {t[2], dtz}};
        const Dual sd[3] = {{s[0], 0.0}, {s[1], 0.0}, {s[2], dsz}};
        Dual r[6];
        closed_tensor<Dual>(Dual{X, 0.0}, Dual{Y, 0.0}, Dual{Z, dZ}, td, sd, r);
        for (int c = 0; c < 6; ++c) {
            out[c] = r[c].v;
            dout[c] = r[c].d;
        }
        return;
    }
    if (far32 && quadrature_tensor_dt_f32(X, Y, Z, t, s, gap, dtz, dsz, dZ, dout)) return;
    const double wcap = 0.5 * gap;
    double widest = 0.0;
    for (int k = 0; k < 3; ++k) {
        const double br0 = -s[k], br1 = fmin(0.0, t[k] - s[k]), br2 = fmax(0.0, t[k] - s[k]),
                     br3 = t[k];
        const double ws[3] = {br1 - br0, br2 - br1, br3 - br2};
        for (int p = 0; p < 3; ++p)
            if (ws[p] > 0.0) widest = fmax(widest, ws[p] / ceil(ws[p] / wcap));
    }
    quadrature_tensor_dt(X, Y, Z, t, s, far_nodes(gap / widest), wcap, dtz, dsz, dZ, out, dout);
}

// ---- kernels ---------------------------------------------------------------

__global__ void k_tensor_points(int n, const double *__restrict__ geom, double *__restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double *g = geom + (size_t)i * 9;
    const double t[3] = {g[3], g[4], g[5]}, s[3] = {g[6], g[7], g[8]};
    double r[6];
    tensor_eval(g[0], g[1], g[2], t, s, r);
    for (int c = 0; c < 6; ++c) out[(size_t)i * 6 + c] = r[c];
}

cudaError_t launch_tensor_points(int n, const double *geom, double *out, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_tensor_points<<<(n + 127) / 128, 128, 0, st>>>(n, geom, out);
    return cudaGetLastError();
}

// Write N at offset (p, q) of a pair's three planes, with the parity of each
// component in X and Y (f even, g odd in x and y), at the up to four mirrored
// positions of the circulant grid.
template <typename C>
__device__ __forceinline__ C plane_val(double a, double b) {
    C v;
    v.x = a;
    v.y = b;
    return v;
}

template <typename C>
__device__ __forceinline__ void write_planes(C *base, int p, int q, int Px, int Py, const double N[6]) {
    for (int my = 0; my < 2; ++my) {
        if (my && q == 0) continue;
        const int yi = my ? Py - q : q;
        const double sgy = my ? -1.0 : 1.0;
        for (int mx = 0; mx < 2; ++mx) {
            if (mx && p == 0) continue;
            const int xi = mx ? Px - p : p;
            const double sgx = mx ? -1.0 : 1.0;
            const size_t o = (size_t)yi * Px + xi;
            base[o] = plane_val<C>(N[0], N[1]);
            base[(size_t)Px * Py + o] = plane_val<C>(N[2], sgx * sgy * N[3]);
            base[(size_t)2 * Px * Py + o] = plane_val<C>(sgx * N[4], sgy * N[5]);
        }
    }
}

// The closed form at the near offsets, one warp per (pair, p <= pm, q <= qm):
// the 6 x 64 signed Newell terms (closed_nxx / closed_nxy with their axis
// permutations) are spread over the lanes, 12 each, and summed by a warp
// reduction; offsets that are not near return (k_kernel_planes has them).
template <typename C>
__global__ void __launch_bounds__(32) k_near_planes(C *__restrict__ planes, int p0, int np,
                                                    const int *__restrict__ pair_i,
                                                    const int *__restrict__ pair_j, int nx, int ny, double dx,
                                                    double dy, int log2Px, int log2Py,
                                                    const double *__restrict__ z, const double *__restrict__ th,
                                                    int pm) {
    const int P = blockIdx.x, p = blockIdx.y % (pm + 1), q = blockIdx.y / (pm + 1);
    if (p >= nx || q >= ny) return;
    const int i = pair_i[p0 + P], j = pair_j[p0 + P];
    const double t[3] = {dx, dy, th[i]}, s[3] = {dx, dy, th[j]};
    const double o[3] = {p * dx, q * dy, z[i] - z[j]};
    double gap;
    if (!near_pair(o[0], o[1], o[2], t, s, gap)) return;
    // component -> axis order of its arguments (xx yy zz: closed_nxx; xy xz yz: closed_nxy)
    constexpr int kAx[6][3] = {{0, 1, 2}, {1, 0, 2}, {2, 1, 0}, {0, 1, 2}, {0, 2, 1}, {2, 1, 0}};
    const int lane = threadIdx.x;
    double N[6];
#pragma unroll 1
    for (int c = 0; c < 6; ++c) {
        const int A = kAx[c][0], Bx = kAx[c][1], Cz = kAx[c][2];
        const double X = o[A], Y = o[Bx], Z = o[Cz];
        const double TX = t[A], TY = t[Bx], TZ = t[Cz], SX = s[A], SY = s[Bx], SZ = s[Cz];
        double acc = 0.0;
#pragma unroll 1
        for (int h = 0; h < 2; ++h) {
            const int tt = lane + 32 * h, a = tt >> 4, b = (tt >> 2) & 3, cc = tt & 3;
            const double sgn = ((a == 0 || a == 3) ? 1.0 : -1.0) * ((b == 0 || b == 3) ? 1.0 : -1.0) *
                               ((cc == 0 || cc == 3) ? 1.0 : -1.0);
            const double sz = cc == 0 ? TZ : cc == 1 ? 0.0 : cc == 2 ? TZ - SZ : -SZ;
            double v;
            if (c < 3) {
                const double sx = a == 0 ? 0.0 : a == 1 ? TX : a == 2 ? -SX : TX - SX;
                const double sy = b == 0 ? TY : b == 1 ? 0.0 : b == 2 ? TY - SY : -SY;
                v = newell_f<double>(X + sx, Y + sy, Z + sz);
            } else {
                const double sx = a == 0 ? TX : a == 1 ? 0.0 : a == 2 ? TX - SX : -SX;
                const double sy = b == 0 ? 0.0 : b == 1 ? -SY : b == 2 ? TY : TY - SY;
                v = newell_g<double>(X + sx, Y + sy, Z + sz);
            }
            acc += sgn * v;
        }
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
        N[c] = acc / (4.0 * kPi * (TX * TY * TZ));
    }
    if (lane == 0) {
        const int Px = 1 << log2Px, Py = 1 << log2Py;
        write_planes(planes + (size_t)P * 3 * Px * Py, p, q, Px, Py, N);
    }
}

// One thread per (pair, q, p) with 0 <= p < nx, 0 <= q < ny: evaluate N(i <- j)
// at (p dx, q dy, z_i - z_j) and write it (write_planes); near offsets are
// k_near_planes'.
template <typename C>
__global__ void k_kernel_planes(C *__restrict__ planes, int p0, int np,
                                const int *__restrict__ pair_i, const int *__restrict__ pair_j,
                                int nx, int ny, double dx, double dy, int log2Px, int log2Py,
                                const double *__restrict__ z, const double *__restrict__ th,
                                int far32) {
    // blocks: pair fastest, then rows q (see plane_grid)
    const int cpr = (nx + blockDim.x - 1) / blockDim.x;
    const int P = blockIdx.x, q = blockIdx.y / cpr;
    const int p = (blockIdx.y - q * cpr) * blockDim.x + threadIdx.x;
    if (p >= nx) return;
    const int i = pair_i[p0 + P], j = pair_j[p0 + P];
    const double t[3] = {dx, dy, th[i]}, s[3] = {dx, dy, th[j]};
    double N[6];
    if (!tensor_eval(p * dx, q * dy, z[i] - z[j], t, s, N, far32 != 0, true)) return;
    write_planes(planes + (size_t)P * 3 * ((size_t)1 << (log2Px + log2Py)), p, q, 1 << log2Px, 1 << log2Py, N);
}

// geom[n][12]: X, Y, Z, tx, ty, tz, sx, sy, sz, dtz, dsz, dZ -> out[n][6], dout[n][6]
__global__ void k_tensor_points_dt(int n, const double *__restrict__ geom, double *__restrict__ out,
                                   double *__restrict__ dout) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double *g = geom + (size_t)i * 12;
    const double t[3] = {g[3], g[4], g[5]}, s[3] = {g[6], g[7], g[8]};
    double r[6], dr[6];
    tensor_eval_dt(g[0], g[1], g[2], t, s, g[9], g[10], g[11], r, dr);
    for (int c = 0; c < 6; ++c) {
        out[(size_t)i * 6 + c] = r[c];
        dout[(size_t)i * 6 + c] = dr[c];
    }
}

cudaError_t launch_tensor_points_dt(int n, const double *geom, double *out, double *dout,
                                    cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_tensor_points_dt<<<(n + 127) / 128, 128, 0, st>>>(n, geom, out, dout);
    return cudaGetLastError();
}

// d N(i <- j) / d t_layer for all L*L pairs (P = i*L + j) of [p0, p0 + np),
// written with the in-plane parity like k_kernel_planes.  Seeds: the target
// edge moves if i == layer, the source edge if j == layer, and the offset
// z_i - z_j by [i > layer] - [j > layer].  Float planes (float plans) take the
// far field in float.
template <typename C>
__global__ void k_dkernel_planes(C *__restrict__ planes, int p0, int np, int L, int layer,
                                 int nx, int ny, double dx, double dy, int log2Px, int log2Py,
                                 const double *__restrict__ z, const double *__restrict__ th) {
    const int cpr = (nx + blockDim.x - 1) / blockDim.x;  // blocks as in k_kernel_planes
    const int P = blockIdx.x, q = blockIdx.y / cpr;
    const int p = (blockIdx.y - q * cpr) * blockDim.x + threadIdx.x;
    if (p >= nx) return;
    const int i = (p0 + P) / L, j = (p0 + P) % L;
    const double dtz = i == layer ? 1.0 : 0.0, dsz = j == layer ? 1.0 : 0.0;
    const double dZ = (i > layer ? 1.0 : 0.0) - (j > layer ? 1.0 : 0.0);
    if (dtz == 0.0 && dsz == 0.0 && dZ == 0.0) return;  // planes are zeroed beforehand
    const double t[3] = {dx, dy, th[i]}, s[3] = {dx, dy, th[j]};
    double N[6], dN[6];
    tensor_eval_dt(p * dx, q * dy, z[i] - z[j], t, s, dtz, dsz, dZ, N, dN, sizeof(C) == sizeof(float2));
    const int Px = 1 << log2Px, Py = 1 << log2Py;
    write_planes(planes + (size_t)P * 3 * Px * Py, p, q, Px, Py, dN);
}

// Grid of the plane kernels: x = pair, y = (row q, chunk of 128 offsets p).  The
// pair index runs fastest, so the first blocks dispatched are the first rows of
// every pair: the near-field offsets (closed form in double) and the dense
// quadratures just beyond it, which take far longer than the rest, start first
// and on different SMs instead of queueing behind one another.
static dim3 plane_grid(int np, int nx, int ny, int bs) { return dim3(np, ny * ((nx + bs - 1) / bs)); }

cudaError_t launch_dkernel_planes(void *planes, bool f32, int p0, int np, int L, int layer, int nx, int ny,
                                  double dx, double dy, int log2Px, int log2Py, const double *z,
                                  const double *th, cudaStream_t st) {
    if (np <= 0) return cudaSuccess;
    if (f32)
        k_dkernel_planes<float2><<<plane_grid(np, nx, ny, 128), 128, 0, st>>>(
            (float2 *)planes, p0, np, L, layer, nx, ny, dx, dy, log2Px, log2Py, z, th);
    else
        k_dkernel_planes<double2><<<plane_grid(np, nx, ny, 128), 128, 0, st>>>(
            (double2 *)planes, p0, np, L, layer, nx, ny, dx, dy, log2Px, log2Py, z, th);
    return cudaGetLastError();
}

template <typename C>
static cudaError_t kernel_planes(C *planes, int p0, int np, const int *pair_i, const int *pair_j, int nx, int ny,
                                 double dx, double dy, int log2Px, int log2Py, const double *z, const double *th,
                                 cudaStream_t st, bool far32) {
    // near offsets: gap >= (p - 1) dx along x (and likewise y), so only
    // p <= ceil(e / dx), q <= ceil(e / dy) can be below e = max(dx, dy)
    const double e = dx > dy ? dx : dy;
    const int pm = (int)ceil(e / dx), qm = (int)ceil(e / dy);
    k_near_planes<C><<<dim3(np, (pm + 1) * (qm + 1)), 32, 0, st>>>(planes, p0, np, pair_i, pair_j, nx, ny, dx,
                                                                   dy, log2Px, log2Py, z, th, pm);
    cudaError_t e1 = cudaGetLastError();
    if (e1 != cudaSuccess) return e1;
    k_kernel_planes<C><<<plane_grid(np, nx, ny, 128), 128, 0, st>>>(planes, p0, np, pair_i, pair_j, nx, ny, dx,
                                                                   dy, log2Px, log2Py, z, th, far32 ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_kernel_planes(void *planes, bool f32, int p0, int np, const int *pair_i,
                                 const int *pair_j, int nx, int ny, double dx, double dy,
                                 int log2Px, int log2Py, const double *z, const double *th,
                                 cudaStream_t st, bool far32) {
    if (np <= 0) return cudaSuccess;
    return f32 ? kernel_planes((float2 *)planes, p0, np, pair_i, pair_j, nx, ny, dx, dy, log2Px, log2Py, z, th,
                               st, far32)
               : kernel_planes((double2 *)planes, p0, np, pair_i, pair_j, nx, ny, dx, dy, log2Px, log2Py, z, th,
                               st, far32);
}

// Row FFTs of [nrows][Px] complex double, rows_per_block rows per block.
// Row FFTs: each row is loaded in natural order and scattered to its
// bit-reversed positions; a padding slot after every 128 elements keeps the
// eight 16-byte writes of a quarter warp (bit-reversed positions 128 apart) in
// distinct banks.
constexpr int kRowPad = 7;

template <typename C>
__global__ void k_fft_rows_f64(C *__restrict__ data, long long nrows, int log2n, int rows_per_block,
                               const C *__restrict__ tw, int log2tw) {
    extern __shared__ __align__(16) unsigned char sm_rows_raw[];
    C *sm_rows = reinterpret_cast<C *>(sm_rows_raw);
    const int n = 1 << log2n;
    const int stride = n + (n >> kRowPad);
    const long long r0 = (long long)blockIdx.x * rows_per_block;
    const int nr = (int)min((long long)rows_per_block, nrows - r0);
    for (int e = threadIdx.x; e < nr * n; e += blockDim.x) {
        const int r = e >> log2n, x = e & (n - 1);
        sm_rows[r * stride + fft_pos<kRowPad>(bit_reverse(x, log2n))] = data[(size_t)(r0 + r) * n + x];
    }
    __syncthreads();
    fft_dit<false, C, kRowPad>(sm_rows, log2n, nr, stride, tw, log2tw);
    for (int e = threadIdx.x; e < nr * n; e += blockDim.x) {
        const int r = e >> log2n, x = e & (n - 1);
        data[(size_t)r0 * n + e] = sm_rows[r * stride + fft_pos<kRowPad>(x)];
    }
}

// Column FFTs of planes [nplanes][Py][Px]: a block takes `tile` adjacent columns.
template <typename C>
__global__ void k_fft_cols_f64(C *__restrict__ data, int log2Px, int log2Py, int tile, int tiles_per_plane,
                               const C *__restrict__ tw, int log2tw) {
    extern __shared__ __align__(16) unsigned char sm_cols_raw[];
    C *sm_cols = reinterpret_cast<C *>(sm_cols_raw);
    const int Px = 1 << log2Px, Py = 1 << log2Py;
    const int plane = blockIdx.x / tiles_per_plane;
    const int x0 = (blockIdx.x % tiles_per_plane) * tile;
    C *base = data + (size_t)plane * Px * Py + x0;
    const int stride = Py + 1;
    for (int e = threadIdx.x; e < tile * Py; e += blockDim.x) {
        const int y = e / tile, c = e - y * tile;
        sm_cols[c * stride + bit_reverse(y, log2Py)] = base[(size_t)y * Px + c];
    }
    __syncthreads();
    fft_dit<false>(sm_cols, log2Py, tile, stride, tw, log2tw);
    for (int e = threadIdx.x; e < tile * Py; e += blockDim.x) {
        const int y = e / tile, c = e - y * tile;
        base[(size_t)y * Px + c] = sm_cols[c * stride + y];
    }
}

template <typename C>
static cudaError_t fft2_planes(C *planes, int nplanes, int log2Px, int log2Py, const C *twx, int log2twx,
                               const C *twy, int log2twy, cudaStream_t st) {
    const int Px = 1 << log2Px, Py = 1 << log2Py;
    // 32 KB of shared memory per block: several blocks per SM hide the
    // global-memory latency of the load and store phases
    const int budget = (32 << 10) / (int)sizeof(C);
    const int rstride = Px + (Px >> kRowPad);
    int rpb = budget / rstride;
    if (rpb < 1) rpb = 1;
    const long long nrows = (long long)nplanes * Py;
    size_t smem = (size_t)rpb * rstride * sizeof(C);
    cudaError_t e = cudaFuncSetAttribute(k_fft_rows_f64<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_fft_rows_f64<C><<<(unsigned)((nrows + rpb - 1) / rpb), 256, smem, st>>>(planes, nrows, log2Px, rpb, twx,
                                                                               log2twx);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // columns: 64 KB blocks of up to 8 adjacent columns (128-byte row pieces in double)
    int tile = (64 << 10) / (int)sizeof(C) / (Py + 1);
    if (tile > 8) tile = 8;
    if (tile > Px) tile = Px;
    if (tile < 1) tile = 1;
    int t2 = 1;
    while (t2 * 2 <= tile) t2 *= 2;
    tile = t2;
    smem = (size_t)tile * (Py + 1) * sizeof(C);
    e = cudaFuncSetAttribute(k_fft_cols_f64<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    // only the columns kx <= Px/2 that k_extract reads: each packed plane holds two
    // components whose spectra are both real or both imaginary (their parities
    // in x and y), so no Hermitian partner at Px - kx is needed
    const int ntile = (Px / 2 + 1 + tile - 1) / tile;  // tile <= Px/2 or tile = Px: inside the plane
    k_fft_cols_f64<C><<<(unsigned)((long long)nplanes * ntile), 256, smem, st>>>(planes, log2Px, log2Py, tile,
                                                                                 ntile, twy, log2twy);
    return cudaGetLastError();
}

cudaError_t launch_fft2_planes(void *planes, bool f32, int nplanes, int log2Px, int log2Py, const void *twx,
                               int log2twx, const void *twy, int log2twy, cudaStream_t st) {
    return f32 ? fft2_planes((float2 *)planes, nplanes, log2Px, log2Py, (const float2 *)twx, log2twx,
                             (const float2 *)twy, log2twy, st)
               : fft2_planes((double2 *)planes, nplanes, log2Px, log2Py, (const double2 *)twx, log2twx,
                             (const double2 *)twy, log2twy, st);
}

// The BF16 split pair of a tensor value, as the bits of a float: v rounded to
// float, hi = bf16(v) in the upper half, lo = bf16(v - hi) in the lower half,
// both rounded to nearest even (the split the contraction applies to its
// other operand).
__device__ __forceinline__ float bf16_pair(double x) {
    const float v = (float)x;
    const __nv_bfloat16 hi = __float2bfloat16_rn(v);
    const __nv_bfloat16 lo = __float2bfloat16_rn(v - __bfloat162float(hi));
    const uint32_t w = ((uint32_t)__bfloat16_as_ushort(hi) << 16) | (uint32_t)__bfloat16_as_ushort(lo);
    return __uint_as_float(w);
}

// Quadrant kx <= Px/2, ky <= Py/2 of the transformed planes -> plan tensor,
// stored entry u holding ky = u_kyq(u) (layout.cuh).
// plane 0 = FFT(N_xx) + i FFT(N_yy), both real; plane 1 = FFT(N_zz) + i FFT(N_xy),
// both real; plane 2 = FFT(N_xz) + i FFT(N_yz) = i a - b with FFT(N_xz) = i a,
// FFT(N_yz) = i b.  Dense-product plans (umajor) write the blocked, prescaled
// layout of layout.cuh: pair (i, j) of the pair lists, times t_i / t_0, and in
// a diagonal block also its mirror (j, i) with xz and yz negated; the tensor
// is zeroed beforehand (padding layers).  umajor 2: the same with zz negated
// and each value as its BF16 split pair (bf16_pair).
template <typename T, typename C>
__global__ void k_extract(const C *__restrict__ planes, int p0, int np, int npairs,
                          int log2Px, int log2Py, int QyS, T *__restrict__ tensor, int umajor,
                          int natural, const int *__restrict__ pair_i, const int *__restrict__ pair_j,
                          const double *__restrict__ th, int L) {
    const int Px = 1 << log2Px, Py = 1 << log2Py;
    const int Kx = Px / 2 + 1, Qy = Py / 2 + 1;
    const long long total = (long long)np * Kx * Qy;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    const int u = (int)(idx % Qy);
    const int kx = (int)((idx / Qy) % Kx);
    const int P = (int)(idx / ((long long)Qy * Kx));
    const int kq = natural ? u : u_kyq(u, log2Py);
    const C *base = planes + (size_t)P * 3 * Px * Py + (size_t)kq * Px + kx;
    const double2 A = make_double2(base[0].x, base[0].y);
    const double2 Bp = make_double2(base[(size_t)Px * Py].x, base[(size_t)Px * Py].y);
    const double2 Cc = make_double2(base[(size_t)2 * Px * Py].x, base[(size_t)2 * Px * Py].y);
    const double sc = 1.0 / ((double)Px * (double)Py);
    if (umajor) {
        const int i = pair_i[p0 + P], j = pair_j[p0 + P], nb = ub_nb(L), rl = ub_row(L);
        const double f = sc * th[i] / th[0];
        // umajor 2 (BF16 split plans): zz negated (the -K_zz block of the
        // contraction) and every value stored as its BF16 split pair
        const double zs = umajor == 2 ? -1.0 : 1.0;
        const double v[6] = {A.x * f, A.y * f, zs * Bp.x * f, Bp.y * f, Cc.y * f, -Cc.x * f};
        T *o = tensor + ((size_t)kx * Qy + u) * (6 * (size_t)rl);
        const int I = i >> 3, J = j >> 3;
        const int e1 = ub_blk(I, J, nb) + ub_at(i & 7, j & 7, J);
        for (int c = 0; c < 6; ++c) o[(size_t)c * rl + e1] = umajor == 2 ? (T)bf16_pair(v[c]) : (T)v[c];
        if (I == J && i != j) {
            const int e2 = ub_blk(I, I, nb) + ub_at(j & 7, i & 7, I);
            for (int c = 0; c < 6; ++c) {
                const double w = c >= 4 ? -v[c] : v[c];
                o[(size_t)c * rl + e2] = umajor == 2 ? (T)bf16_pair(w) : (T)w;
            }
        }
        return;
    }
    const size_t cs = QyS;  // component stride
    T *o = tensor + ((size_t)kx * npairs + (p0 + P)) * 6 * QyS + u;
    o[0 * cs] = (T)(A.x * sc);
    o[1 * cs] = (T)(A.y * sc);
    o[2 * cs] = (T)(Bp.x * sc);
    o[3 * cs] = (T)(Bp.y * sc);
    o[4 * cs] = (T)(Cc.y * sc);
    o[5 * cs] = (T)(-Cc.x * sc);
}

cudaError_t launch_extract_tensor(const void *planes, bool f32, int p0, int np, int npairs, int log2Px,
                                  int log2Py, int QyS, void *tensor, bool fp64, cudaStream_t st,
                                  int umajor, int natural, const int *pair_i, const int *pair_j,
                                  const double *th, int L) {
    if (umajor && (fp64 || !pair_i || !pair_j || !th || L < 1)) return cudaErrorInvalidValue;
    const long long total = (long long)np * ((1 << log2Px) / 2 + 1) * ((1 << log2Py) / 2 + 1);
    const unsigned grid = (unsigned)((total + 255) / 256);
    if (f32) {
        if (fp64)
            k_extract<double, float2><<<grid, 256, 0, st>>>((const float2 *)planes, p0, np, npairs, log2Px, log2Py,
                                                            QyS, (double *)tensor, umajor, natural, pair_i,
                                                            pair_j, th, L);
        else
            k_extract<float, float2><<<grid, 256, 0, st>>>((const float2 *)planes, p0, np, npairs, log2Px, log2Py,
                                                           QyS, (float *)tensor, umajor, natural, pair_i,
                                                           pair_j, th, L);
    } else {
        if (fp64)
            k_extract<double, double2><<<grid, 256, 0, st>>>((const double2 *)planes, p0, np, npairs, log2Px,
                                                             log2Py, QyS, (double *)tensor, umajor, natural,
                                                             pair_i, pair_j, th, L);
        else
            k_extract<float, double2><<<grid, 256, 0, st>>>((const double2 *)planes, p0, np, npairs, log2Px,
                                                            log2Py, QyS, (float *)tensor, umajor, natural,
                                                            pair_i, pair_j, th, L);
    }
    return cudaGetLastError();
}

}  // namespace demag
