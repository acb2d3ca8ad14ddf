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
#include <cmath>
#include <vector>

#include "fft.cuh"
#include "internal.h"

namespace demag {

__constant__ double c_gl_x[kGLMax + 1][kGLMax];
__constant__ double c_gl_w[kGLMax + 1][kGLMax];

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
    if (dev < 64) done[dev] = true;
    return DEMAG_OK;
}

// ---- closed form (Sec. 2) ------------------------------------------------

// Newell f: d^2/dy^2 d^2/dz^2 f = 1/R.  Products with a vanishing prefactor
// are dropped (their limit is zero).
__device__ __noinline__ double newell_f(double x, double y, double z) {
    const double x2 = x * x, y2 = y * y, z2 = z * z;
    const double R = sqrt(x2 + y2 + z2);
    double v = (2.0 * x2 - y2 - z2) * R / 6.0;
    const double xz = x2 + z2, xy = x2 + y2;
    if (y != 0.0 && xz > 0.0) v += 0.5 * y * (z2 - x2) * asinh(y / sqrt(xz));
    if (z != 0.0 && xy > 0.0) v += 0.5 * z * (y2 - x2) * asinh(z / sqrt(xy));
    if (x != 0.0 && y != 0.0 && z != 0.0) v -= x * y * z * atan(y * z / (x * R));
    return v;
}

// Newell g: d/dx d/dy d^2/dz^2 g = 1/R.
__device__ __noinline__ double newell_g(double x, double y, double z) {
    const double x2 = x * x, y2 = y * y, z2 = z * z;
    const double R = sqrt(x2 + y2 + z2);
    double v = -x * y * R / 3.0;
    if (y != 0.0) v += y / 6.0 * (3.0 * z2 - y2) * asinh(x / sqrt(y2 + z2));
    if (x != 0.0) v += x / 6.0 * (3.0 * z2 - x2) * asinh(y / sqrt(x2 + z2));
    if (x != 0.0 && y != 0.0 && z != 0.0) {
        v += x * y * z * asinh(z / sqrt(x2 + y2));
        v -= z2 * z / 6.0 * atan(x * y / (z * R));
        v -= 0.5 * z * y2 * atan(x * z / (y * R));
        v -= 0.5 * z * x2 * atan(y * z / (x * R));
    }
    return v;
}

constexpr double kPi = 3.14159265358979323846;

// N_xx: x-face pairs (Eq. Nxx) x F split into F_1 (y) and F_2 (z) (App. A).
__device__ __noinline__ double closed_nxx(double X, double Y, double Z, double tx, double ty, double tz,
                             double sx, double sy, double sz) {
    const double sxa[4] = {0.0, tx, -sx, tx - sx};
    const double sya[4] = {ty, 0.0, ty - sy, -sy};
    const double sza[4] = {tz, 0.0, tz - sz, -sz};
    double acc = 0.0;
#pragma unroll 1
    for (int a = 0; a < 4; ++a) {
        double ya = 0.0;
#pragma unroll 1
        for (int b = 0; b < 4; ++b) {
            double zb = 0.0;
#pragma unroll 1
            for (int c = 0; c < 4; ++c) {
                const double v = newell_f(X + sxa[a], Y + sya[b], Z + sza[c]);
                zb += (c == 0 || c == 3) ? v : -v;
            }
            ya += (b == 0 || b == 3) ? zb : -zb;
        }
        acc += (a == 0 || a == 3) ? ya : -ya;
    }
    return acc / (4.0 * kPi * tx * ty * tz);
}

// N_xy: target/source face pairs of Eq. Nxy (fourth term at Y + Delta y) x G
// split over x and y (App. B) x G_1 over z.
__device__ __noinline__ double closed_nxy(double X, double Y, double Z, double tx, double ty, double tz,
                             double sx, double sy, double sz) {
    const double sxa[4] = {tx, 0.0, tx - sx, -sx};
    const double sya[4] = {0.0, -sy, ty, ty - sy};
    const double sza[4] = {tz, 0.0, tz - sz, -sz};
    double acc = 0.0;
#pragma unroll 1
    for (int a = 0; a < 4; ++a) {
        double ya = 0.0;
#pragma unroll 1
        for (int b = 0; b < 4; ++b) {
            double zb = 0.0;
#pragma unroll 1
            for (int c = 0; c < 4; ++c) {
                const double v = newell_g(X + sxa[a], Y + sya[b], Z + sza[c]);
                zb += (c == 0 || c == 3) ? v : -v;
            }
            ya += (b == 0 || b == 3) ? zb : -zb;
        }
        acc += (a == 0 || a == 3) ? ya : -ya;
    }
    return acc / (4.0 * kPi * tx * ty * tz);
}

// All six components: N_yy, N_zz from N_xx and N_xz, N_yz from N_xy by axis
// permutation (Sec. 2).  out = {xx, yy, zz, xy, xz, yz}.
__device__ void closed_tensor(double X, double Y, double Z, const double t[3], const double s[3],
                              double out[6]) {
    out[0] = closed_nxx(X, Y, Z, t[0], t[1], t[2], s[0], s[1], s[2]);
    out[1] = closed_nxx(Y, X, Z, t[1], t[0], t[2], s[1], s[0], s[2]);
    out[2] = closed_nxx(Z, Y, X, t[2], t[1], t[0], s[2], s[1], s[0]);
    out[3] = closed_nxy(X, Y, Z, t[0], t[1], t[2], s[0], s[1], s[2]);
    out[4] = closed_nxy(X, Z, Y, t[0], t[2], t[1], s[0], s[2], s[1]);
    out[5] = closed_nxy(Z, Y, X, t[2], t[1], t[0], s[2], s[1], s[0]);
}

// ---- far field: composite Gauss-Legendre quadrature -----------------------

// Difference density of one axis: u = xi - xi', xi on [0, a] (target),
// xi' on [0, b] (source); T(u) = min(a, u + b) - max(0, u) on [-b, a], linear on
// three pieces, each cut into `cuts` equal sub-pieces of n nodes.
struct AxisRule {
    double a, b;
    double br[4];
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
    const double len = (r.br[p + 1] - r.br[p]) / r.cuts[p];
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

// The evaluation used everywhere: closed form while the gap between the two
// cuboids is below the larger in-plane edge, quadrature (sub-pieces no wider
// than half the gap) beyond.
__device__ void tensor_eval(double X, double Y, double Z, const double t[3], const double s[3],
                            double out[6]) {
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
        closed_tensor(X, Y, Z, t, s, out);
        return;
    }
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

// One thread per (pair, q, p) with 0 <= p < nx, 0 <= q < ny: evaluate N(i <- j)
// at (p dx, q dy, z_i - z_j) and write it, with the parity of each component
// in X and Y (f even, g odd in x and y), at the up to four mirrored positions
// of the circulant grid.
__global__ void k_kernel_planes(double2 *__restrict__ planes, int p0, int np,
                                const int *__restrict__ pair_i, const int *__restrict__ pair_j,
                                int nx, int ny, double dx, double dy, int log2Px, int log2Py,
                                const double *__restrict__ z, const double *__restrict__ th) {
    const long long total = (long long)np * nx * ny;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    const int p = (int)(idx % nx);
    const int q = (int)((idx / nx) % ny);
    const int P = (int)(idx / ((long long)nx * ny));
    const int i = pair_i[p0 + P], j = pair_j[p0 + P];
    const double t[3] = {dx, dy, th[i]}, s[3] = {dx, dy, th[j]};
    double N[6];
    tensor_eval(p * dx, q * dy, z[i] - z[j], t, s, N);
    const int Px = 1 << log2Px, Py = 1 << log2Py;
    double2 *base = planes + (size_t)P * 3 * Px * Py;
    for (int my = 0; my < 2; ++my) {
        if (my && q == 0) continue;
        const int yi = my ? Py - q : q;
        const double sgy = my ? -1.0 : 1.0;
        for (int mx = 0; mx < 2; ++mx) {
            if (mx && p == 0) continue;
            const int xi = mx ? Px - p : p;
            const double sgx = mx ? -1.0 : 1.0;
            const size_t o = (size_t)yi * Px + xi;
            base[o] = make_double2(N[0], N[1]);
            base[(size_t)Px * Py + o] = make_double2(N[2], sgx * sgy * N[3]);
            base[(size_t)2 * Px * Py + o] = make_double2(sgx * N[4], sgy * N[5]);
        }
    }
}

cudaError_t launch_kernel_planes(double2 *planes, int p0, int np, const int *pair_i,
                                 const int *pair_j, int nx, int ny, double dx, double dy,
                                 int log2Px, int log2Py, const double *z, const double *th,
                                 cudaStream_t st) {
    const long long total = (long long)np * nx * ny;
    const int bs = 128;
    k_kernel_planes<<<(unsigned)((total + bs - 1) / bs), bs, 0, st>>>(
        planes, p0, np, pair_i, pair_j, nx, ny, dx, dy, log2Px, log2Py, z, th);
    return cudaGetLastError();
}

// Row FFTs of [nrows][Px] complex double, rows_per_block rows per block.
__global__ void k_fft_rows_f64(double2 *__restrict__ data, long long nrows, int log2n,
                               int rows_per_block, const double2 *__restrict__ tw, int log2tw) {
    extern __shared__ double2 sm_rows[];
    const int n = 1 << log2n;
    const long long r0 = (long long)blockIdx.x * rows_per_block;
    const int nr = (int)min((long long)rows_per_block, nrows - r0);
    for (int e = threadIdx.x; e < nr * n; e += blockDim.x) {
        const int r = e >> log2n, x = e & (n - 1);
        sm_rows[r * n + bit_reverse(x, log2n)] = data[(size_t)(r0 + r) * n + x];
    }
    __syncthreads();
    fft_dit<false>(sm_rows, log2n, nr, n, tw, log2tw);
    for (int e = threadIdx.x; e < nr * n; e += blockDim.x) data[(size_t)r0 * n + e] = sm_rows[e];
}

// Column FFTs of planes [nplanes][Py][Px]: a block takes `tile` adjacent columns.
__global__ void k_fft_cols_f64(double2 *__restrict__ data, int log2Px, int log2Py, int tile,
                               const double2 *__restrict__ tw, int log2tw) {
    extern __shared__ double2 sm_cols[];
    const int Px = 1 << log2Px, Py = 1 << log2Py;
    const int tiles_per_plane = Px / tile;
    const int plane = blockIdx.x / tiles_per_plane;
    const int x0 = (blockIdx.x % tiles_per_plane) * tile;
    double2 *base = data + (size_t)plane * Px * Py + x0;
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

cudaError_t launch_fft2_planes(double2 *planes, int nplanes, int log2Px, int log2Py,
                               const double2 *twx, int log2twx, const double2 *twy, int log2twy,
                               cudaStream_t st) {
    const int Px = 1 << log2Px, Py = 1 << log2Py;
    const int budget = 8192;  // complex doubles of shared memory per block (128 KB)
    int rpb = budget / Px;
    if (rpb < 1) rpb = 1;
    const long long nrows = (long long)nplanes * Py;
    size_t smem = (size_t)rpb * Px * sizeof(double2);
    cudaError_t e = cudaFuncSetAttribute(k_fft_rows_f64, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    k_fft_rows_f64<<<(unsigned)((nrows + rpb - 1) / rpb), 256, smem, st>>>(planes, nrows, log2Px, rpb,
                                                                         twx, log2twx);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    int tile = budget / (Py + 1);
    if (tile > Px) tile = Px;
    int t2 = 1;
    while (t2 * 2 <= tile) t2 *= 2;
    tile = t2;
    smem = (size_t)tile * (Py + 1) * sizeof(double2);
    e = cudaFuncSetAttribute(k_fft_cols_f64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_fft_cols_f64<<<(unsigned)((long long)nplanes * (Px / tile)), 256, smem, st>>>(
        planes, log2Px, log2Py, tile, twy, log2twy);
    return cudaGetLastError();
}

// Quadrant kx <= Px/2, ky <= Py/2 of the transformed planes -> plan tensor.
// plane 0 = FFT(N_xx) + i FFT(N_yy), both real; plane 1 = FFT(N_zz) + i FFT(N_xy),
// both real; plane 2 = FFT(N_xz) + i FFT(N_yz) = i a - b with FFT(N_xz) = i a,
// FFT(N_yz) = i b.
template <typename T>
__global__ void k_extract(const double2 *__restrict__ planes, int p0, int np, int npairs,
                          int log2Px, int log2Py, T *__restrict__ tensor) {
    const int Px = 1 << log2Px, Py = 1 << log2Py;
    const int Kx = Px / 2 + 1, Qy = Py / 2 + 1;
    const long long total = (long long)np * Kx * Qy;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    const int kq = (int)(idx % Qy);
    const int kx = (int)((idx / Qy) % Kx);
    const int P = (int)(idx / ((long long)Qy * Kx));
    const double2 *base = planes + (size_t)P * 3 * Px * Py + (size_t)kq * Px + kx;
    const double2 A = base[0], Bp = base[(size_t)Px * Py], C = base[(size_t)2 * Px * Py];
    const double sc = 1.0 / ((double)Px * (double)Py);
    T *o = tensor + ((size_t)kx * npairs + (p0 + P)) * 6 * Qy + kq;
    o[0 * Qy] = (T)(A.x * sc);
    o[1 * Qy] = (T)(A.y * sc);
    o[2 * Qy] = (T)(Bp.x * sc);
    o[3 * Qy] = (T)(Bp.y * sc);
    o[4 * Qy] = (T)(C.y * sc);
    o[5 * Qy] = (T)(-C.x * sc);
}

cudaError_t launch_extract_tensor(const double2 *planes, int p0, int np, int npairs, int log2Px,
                                  int log2Py, void *tensor, bool fp64, cudaStream_t st) {
    const long long total = (long long)np * ((1 << log2Px) / 2 + 1) * ((1 << log2Py) / 2 + 1);
    const unsigned grid = (unsigned)((total + 255) / 256);
    if (fp64)
        k_extract<double><<<grid, 256, 0, st>>>(planes, p0, np, npairs, log2Px, log2Py,
                                                (double *)tensor);
    else
        k_extract<float><<<grid, 256, 0, st>>>(planes, p0, np, npairs, log2Px, log2Py,
                                               (float *)tensor);
    return cudaGetLastError();
}

}  // namespace demag
