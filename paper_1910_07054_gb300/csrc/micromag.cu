// Micromagnetic relaxation of one layer of the stack (Sec. 4: the free layer
// of the MRAM cell is relaxed by a limited-memory BFGS energy minimisation for
// every applied field of an easy-axis hysteresis loop, with the other layers'
// magnetization pinned).
//
// Energy of the relaxed layer, in units of Ms V (tesla), V the cell volume:
//   e = sum_pairs c_d |m_j - m_i|^2             exchange, c_d = A mu0 / (Js d^2)
//     - sum_i (c_an / 2) m_z,i^2                 uniaxial anisotropy along z, c_an = 2 Ku mu0 / Js
//     - sum_i m_i . b_ext                        Zeeman
//     - sum_i m_i . (b_self,i / 2 + b_bias,i)    demag: the layer's own field and the pinned layers'
// with every field in tesla (mu0 H) and the demag fields from the library's own
// apply (Eq. FFT_v2) of the stack with only the relaxed layer (b_self) or with
// every layer but it (b_bias, once per call).  The effective field is
// b_eff = -de/dm = 2 sum_j c_d (m_j - m_i) + c_an m_z e_z + b_ext + b_self + b_bias.
//
// Minimisation: the unit vectors are m_i = v_i / |v_i| with v free, so the
// problem is unconstrained; de/dv_i = (g_i - (m_i . g_i) m_i) / |v_i| with
// g_i = -b_eff,i.  L-BFGS (two-loop recursion over the last `history` pairs,
// initial scaling s.y / y.y) with Armijo backtracking from a unit step (the
// first step, and any step after a reset, is scaled to 0.1 rad RMS per cell).
// It stops when the largest torque |m_i x b_eff,i| is below the tolerance, or
// when no step lowers the energy any further (its change is then below the
// rounding of the energy sum), or after max_iter iterations.
//
// The line search compares energies by their difference, not their values:
// every term is linear or quadratic in the Cartesian m, so its gradient -b_eff
// is linear in m and the trapezoid rule is exact,
//     e(m1) - e(m0) = -1/2 sum_i (b_eff(m0)_i + b_eff(m1)_i) . (m1_i - m0_i).
// Its rounding scales with |m1 - m0|, where that of two energy sums scales
// with |m|: with float demag fields (rounding ~1e-7 T per cell) the energy
// values stop resolving a step's decrease at torques of a few mT, the
// difference does not.
//
// The vectors of the minimiser (3 ny nx doubles) are small; the two-loop
// recursion runs in one block of 1024 threads so that it needs no host round
// trip.  The host reads two numbers per energy evaluation (energy, torque).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <string>

#include "fft.cuh"
#include "internal.h"

namespace demag {

constexpr double kMu0 = 4e-7 * 3.14159265358979323846;
constexpr int kRelaxThreads = 256;
constexpr int kLbfgsThreads = 1024;

// Block-wide sum (any blockDim multiple of 32, up to 1024); every thread gets it.
__device__ double block_sum(double v, double *red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    for (int k = 0; k < nw; ++k) s += red[k];
    return s;
}

// m = v / |v| in the mask (zero elsewhere) into the stack slice (plan type) and a double copy.
template <typename T>
__global__ void k_relax_set_m(const double *__restrict__ v, const unsigned char *__restrict__ mask, T *m_layer,
                              double *mlay, int N) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        double x = v[i], y = v[N + i], z = v[2 * N + i];
        const double n = sqrt(x * x + y * y + z * z);
        if (!mask[i] || n == 0.0) {
            x = y = z = 0.0;
        } else {
            x /= n;
            y /= n;
            z /= n;
        }
        mlay[i] = x;
        mlay[N + i] = y;
        mlay[2 * N + i] = z;
        m_layer[i] = (T)x;
        m_layer[N + i] = (T)y;
        m_layer[2 * N + i] = (T)z;
    }
}

// b_bias = mu0 H of the layer (H in A/m from the apply of the other layers).
template <typename T>
__global__ void k_relax_bias(const T *__restrict__ h_layer, double *b_bias, int n3) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += gridDim.x * blockDim.x)
        b_bias[i] = kMu0 * (double)h_layer[i];
}

struct RelaxCoef {
    double cx, cy;     // A mu0 / (Js dx^2), A mu0 / (Js dy^2)
    double can;        // 2 Ku mu0 / Js
    double bx, by, bz; // applied field (T)
};

// Effective field, energy and gradient in v of every cell of the layer.
// acc[0] += energy (units of Ms V), acc[1] = max torque (bits of a non-negative double).
template <typename T>
__global__ void __launch_bounds__(kRelaxThreads) k_relax_field(const double *__restrict__ mlay,
                                                               const double *__restrict__ v,
                                                               const T *__restrict__ h_self,
                                                               const double *__restrict__ b_bias,
                                                               const unsigned char *__restrict__ mask, int nx,
                                                               int ny, RelaxCoef k, double *__restrict__ g,
                                                               double *__restrict__ beff, double *acc) {
    __shared__ double red[kRelaxThreads / 32];
    const int N = nx * ny;
    double e = 0.0, tq = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        if (!mask[i]) {
            g[i] = g[N + i] = g[2 * N + i] = 0.0;
            beff[i] = beff[N + i] = beff[2 * N + i] = 0.0;
            continue;
        }
        const int x = i % nx, y = i / nx;
        const double mx = mlay[i], my = mlay[N + i], mz = mlay[2 * N + i];
        double bx = 0.0, by = 0.0, bz = 0.0;
        // exchange with the in-plane neighbours inside the mask; the pairs to the
        // right and above carry the pair energy (each pair once)
        const int nb[4] = {x + 1 < nx ? i + 1 : -1, x > 0 ? i - 1 : -1, y + 1 < ny ? i + nx : -1,
                           y > 0 ? i - nx : -1};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int j = nb[q];
            if (j < 0 || !mask[j]) continue;
            const double c = q < 2 ? k.cx : k.cy;
            const double dx = mlay[j] - mx, dy = mlay[N + j] - my, dz = mlay[2 * N + j] - mz;
            bx += 2.0 * c * dx;
            by += 2.0 * c * dy;
            bz += 2.0 * c * dz;
            if (q == 0 || q == 2) e += c * (dx * dx + dy * dy + dz * dz);
        }
        const double sx = kMu0 * (double)h_self[i], sy = kMu0 * (double)h_self[N + i],
                     sz = kMu0 * (double)h_self[2 * N + i];
        const double px = b_bias[i], py = b_bias[N + i], pz = b_bias[2 * N + i];
        bx += k.bx + sx + px;
        by += k.by + sy + py;
        bz += k.bz + sz + pz + k.can * mz;
        e += -0.5 * k.can * mz * mz - (mx * k.bx + my * k.by + mz * k.bz) -
             (mx * (0.5 * sx + px) + my * (0.5 * sy + py) + mz * (0.5 * sz + pz));
        const double cx = my * bz - mz * by, cy = mz * bx - mx * bz, cz = mx * by - my * bx;
        tq = fmax(tq, sqrt(cx * cx + cy * cy + cz * cz));
        // de/dm = -b; tangential part over |v|
        const double vn = sqrt(v[i] * v[i] + v[N + i] * v[N + i] + v[2 * N + i] * v[2 * N + i]);
        const double mb = mx * bx + my * by + mz * bz;
        g[i] = -(bx - mb * mx) / vn;
        g[N + i] = -(by - mb * my) / vn;
        g[2 * N + i] = -(bz - mb * mz) / vn;
        beff[i] = bx;
        beff[N + i] = by;
        beff[2 * N + i] = bz;
    }
    const double es = block_sum(e, red);
    __syncthreads();
    for (int o = 16; o > 0; o >>= 1) tq = fmax(tq, __shfl_xor_sync(0xffffffffu, tq, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = tq;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = fmax(t, red[w]);
        atomicAdd(&acc[0], es);
        atomicMax(reinterpret_cast<unsigned long long *>(&acc[1]), (unsigned long long)__double_as_longlong(t));
    }
}

// L-BFGS search direction d = -H g by the two-loop recursion over the stored
// pairs (slots (newest - k) mod hist, k < count; a pair with rho = 0 is
// skipped); out[0] = g.d, out[1] = d.d.  One block.
__global__ void __launch_bounds__(kLbfgsThreads) k_lbfgs_dir(const double *__restrict__ g, double *__restrict__ d,
                                                             const double *__restrict__ S,
                                                             const double *__restrict__ Y,
                                                             const double *__restrict__ rho, int hist, int count,
                                                             int newest, int n, double *out) {
    __shared__ double red[kLbfgsThreads / 32];
    __shared__ double alpha[32];
    for (int i = threadIdx.x; i < n; i += blockDim.x) d[i] = g[i];
    __syncthreads();
    for (int k = 0; k < count; ++k) {
        const int s = (newest - k + hist) % hist;
        const double *sv = S + (size_t)s * n, *yv = Y + (size_t)s * n;
        double p = 0.0;
        for (int i = threadIdx.x; i < n; i += blockDim.x) p += sv[i] * d[i];
        const double a = rho[s] * block_sum(p, red);
        if (threadIdx.x == 0) alpha[k] = a;
        for (int i = threadIdx.x; i < n; i += blockDim.x) d[i] -= a * yv[i];
        __syncthreads();
    }
    double gamma = 1.0;
    if (count > 0) {
        const double *sv = S + (size_t)newest * n, *yv = Y + (size_t)newest * n;
        double sy = 0.0, yy = 0.0;
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            sy += sv[i] * yv[i];
            yy += yv[i] * yv[i];
        }
        sy = block_sum(sy, red);
        yy = block_sum(yy, red);
        if (yy > 0.0 && sy > 0.0) gamma = sy / yy;
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) d[i] *= gamma;
    __syncthreads();
    for (int k = count - 1; k >= 0; --k) {
        const int s = (newest - k + hist) % hist;
        const double *sv = S + (size_t)s * n, *yv = Y + (size_t)s * n;
        double p = 0.0;
        for (int i = threadIdx.x; i < n; i += blockDim.x) p += yv[i] * d[i];
        const double b = rho[s] * block_sum(p, red);
        const double a = alpha[k];
        for (int i = threadIdx.x; i < n; i += blockDim.x) d[i] += (a - b) * sv[i];
        __syncthreads();
    }
    double gd = 0.0, dd = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        d[i] = -d[i];
        gd += g[i] * d[i];
        dd += d[i] * d[i];
    }
    gd = block_sum(gd, red);
    dd = block_sum(dd, red);
    if (threadIdx.x == 0) {
        out[0] = gd;
        out[1] = dd;
    }
}

// Store the pair s = v1 - v0, y = g1 - g0 in slot `slot`, rho = 1 / (y.s)
// (0 when y.s is not positive: the pair is skipped).  One block.
__global__ void __launch_bounds__(kLbfgsThreads) k_lbfgs_pair(const double *v1, const double *v0, const double *g1,
                                                              const double *g0, double *S, double *Y, double *rho,
                                                              int slot, int n) {
    __shared__ double red[kLbfgsThreads / 32];
    double *sv = S + (size_t)slot * n, *yv = Y + (size_t)slot * n;
    double p = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double s = v1[i] - v0[i], y = g1[i] - g0[i];
        sv[i] = s;
        yv[i] = y;
        p += s * y;
    }
    p = block_sum(p, red);
    if (threadIdx.x == 0) rho[slot] = p > 1e-300 ? 1.0 / p : 0.0;
}

// out = -1/2 sum_i (b0_i + b1_i) . (m1_i - m0_i): e(m1) - e(m0), exactly for
// an energy quadratic in m.  One block.
__global__ void __launch_bounds__(kLbfgsThreads) k_relax_delta(const double *m0, const double *b0,
                                                               const double *m1, const double *b1, int n,
                                                               double *out) {
    __shared__ double red[kLbfgsThreads / 32];
    double p = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) p += (b0[i] + b1[i]) * (m1[i] - m0[i]);
    p = block_sum(p, red);
    if (threadIdx.x == 0) *out = -0.5 * p;
}

// v1 = v0 + a d
__global__ void k_axpy(const double *v0, const double *d, double a, double *v1, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) v1[i] = v0[i] + a * d[i];
}

// Copy of the stack with layer `layer` zeroed (other) or with only that layer (self, from mlay).
template <typename T>
__global__ void k_relax_split(const T *m, T *other, T *self, int layer, int L, int n3) {
    const size_t total = (size_t)L * n3;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const bool in = (int)(i / n3) == layer;
        other[i] = in ? (T)0 : m[i];
        self[i] = (T)0;
    }
}

// Normalized v back into the caller's layer (plan type): m = v / |v| in the mask.
template <typename T>
__global__ void k_relax_out(const double *mlay, T *m_layer, int n3) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += gridDim.x * blockDim.x) m_layer[i] = (T)mlay[i];
}

// v = m (double) for the start
template <typename T>
__global__ void k_relax_in(const T *m_layer, const unsigned char *mask, double *v, int N) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        double x = mask[i] ? (double)m_layer[i] : 0.0, y = mask[i] ? (double)m_layer[N + i] : 0.0,
               z = mask[i] ? (double)m_layer[2 * N + i] : 0.0;
        if (mask[i] && x == 0.0 && y == 0.0 && z == 0.0) z = 1.0;  // a magnetic cell needs a direction
        v[i] = x;
        v[N + i] = y;
        v[2 * N + i] = z;
    }
}

}  // namespace demag

using namespace demag;

namespace {

struct RelaxWork {
    void *other = nullptr, *self = nullptr, *h = nullptr;  // stacks (plan type)
    double *v = nullptr, *vt = nullptr, *g = nullptr, *gt = nullptr, *d = nullptr, *mlay = nullptr,
           *mlt = nullptr, *be = nullptr, *bet = nullptr, *bias = nullptr, *S = nullptr, *Y = nullptr,
           *rho = nullptr, *acc = nullptr;
    double *h_acc = nullptr;  // pinned host copy of acc: energy, torque, g.d, d.d, energy change
    int hist = 0;
    ~RelaxWork() {
        cudaFree(other);
        cudaFree(self);
        cudaFree(h);
        cudaFree(v);
        cudaFree(vt);
        cudaFree(g);
        cudaFree(gt);
        cudaFree(d);
        cudaFree(mlay);
        cudaFree(mlt);
        cudaFree(be);
        cudaFree(bet);
        cudaFree(bias);
        cudaFree(S);
        cudaFree(Y);
        cudaFree(rho);
        cudaFree(acc);
        if (h_acc) cudaFreeHost(h_acc);
    }
};

}  // namespace

extern "C" demag_status demag_relax_layer(demag_plan_t plan, void *m, int layer, const unsigned char *mask,
                                          const demag_relax_params *prm, demag_relax_stats *stats, void *stream) {
    if (!plan || !m || !mask || !prm) return fail(DEMAG_EINVAL, "plan, m, mask or params is NULL");
    if (layer < 0 || layer >= plan->L) return fail(DEMAG_EINVAL, "layer out of range");
    if (plan->umajor || plan->method != 0)
        return fail(DEMAG_EUNSUPPORTED, "relaxation needs a DEMAG_PREC_FP64 or DEMAG_PREC_FP32 hybrid plan");
    if (!(prm->Js > 0 && std::isfinite(prm->Js)) || !(prm->A_ex >= 0 && std::isfinite(prm->A_ex)) ||
        !std::isfinite(prm->Ku) || !(prm->length_unit > 0 && std::isfinite(prm->length_unit)) ||
        !(prm->tol_torque > 0) || prm->max_iter < 0 || prm->history < 1 || prm->history > 32)
        return fail(DEMAG_EINVAL, "invalid relaxation parameters");
    for (int c = 0; c < 3; ++c)
        if (!std::isfinite(prm->b_ext[c])) return fail(DEMAG_EINVAL, "b_ext must be finite");
    const bool fp64 = plan->precision == DEMAG_PREC_FP64;
    const size_t real = fp64 ? 8 : 4;
    const int nx = plan->nx, ny = plan->ny, L = plan->L, N = nx * ny, n = 3 * N;
    cudaStream_t st = (cudaStream_t)stream;
    RelaxWork w;
    w.hist = prm->history;
    const size_t stack = (size_t)L * n * real;
    auto alloc = [&](void **p, size_t b) -> demag_status {
        cudaError_t e = cudaMalloc(p, b);
        if (e != cudaSuccess) {
            *p = nullptr;
            return cuda_fail(e, "cudaMalloc(relaxation workspace)");
        }
        return DEMAG_OK;
    };
#define RELAX_TRY(x)                            \
    do {                                        \
        demag_status s_ = (x);                  \
        if (s_ != DEMAG_OK) return s_;          \
    } while (0)
    RELAX_TRY(alloc(&w.other, stack));
    RELAX_TRY(alloc(&w.self, stack));
    RELAX_TRY(alloc(&w.h, stack));
    for (double **p : {&w.v, &w.vt, &w.g, &w.gt, &w.d, &w.mlay, &w.mlt, &w.be, &w.bet, &w.bias})
        RELAX_TRY(alloc((void **)p, (size_t)n * 8));
    RELAX_TRY(alloc((void **)&w.S, (size_t)w.hist * n * 8));
    RELAX_TRY(alloc((void **)&w.Y, (size_t)w.hist * n * 8));
    RELAX_TRY(alloc((void **)&w.rho, (size_t)w.hist * 8));
    RELAX_TRY(alloc((void **)&w.acc, 5 * 8));
    {
        cudaError_t e = cudaHostAlloc((void **)&w.h_acc, 5 * 8, cudaHostAllocDefault);
        if (e != cudaSuccess) {
            w.h_acc = nullptr;
            return cuda_fail(e, "cudaHostAlloc(relaxation scalars)");
        }
    }
#undef RELAX_TRY
    const double Ms = prm->Js / kMu0;
    const double dxm = plan->dx * prm->length_unit, dym = plan->dy * prm->length_unit;
    RelaxCoef k;
    k.cx = prm->A_ex * kMu0 / (prm->Js * dxm * dxm);
    k.cy = prm->A_ex * kMu0 / (prm->Js * dym * dym);
    k.can = 2.0 * prm->Ku * kMu0 / prm->Js;
    k.bx = prm->b_ext[0];
    k.by = prm->b_ext[1];
    k.bz = prm->b_ext[2];
    const unsigned gN = (unsigned)std::min((N + 255) / 256, 1024);
    const unsigned gS = (unsigned)std::min<size_t>(((size_t)L * n + 255) / 256, 4096);
    char *layer_of = (char *)m + (size_t)layer * n * real;
    cudaError_t e;
    // the pinned layers' field in the relaxed layer
    if (fp64) {
        k_relax_split<double><<<gS, 256, 0, st>>>((const double *)m, (double *)w.other, (double *)w.self, layer, L, n);
    } else {
        k_relax_split<float><<<gS, 256, 0, st>>>((const float *)m, (float *)w.other, (float *)w.self, layer, L, n);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "relaxation set-up");
    demag_status rc = demag_apply(plan, w.other, Ms, w.h, 1, stream);
    if (rc != DEMAG_OK) return rc;
    char *h_layer = (char *)w.h + (size_t)layer * n * real;
    char *self_layer = (char *)w.self + (size_t)layer * n * real;
    if (fp64) {
        k_relax_bias<double><<<gN, 256, 0, st>>>((const double *)h_layer, w.bias, n);
        k_relax_in<double><<<gN, 256, 0, st>>>((const double *)layer_of, mask, w.v, N);
    } else {
        k_relax_bias<float><<<gN, 256, 0, st>>>((const float *)h_layer, w.bias, n);
        k_relax_in<float><<<gN, 256, 0, st>>>((const float *)layer_of, mask, w.v, N);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "relaxation set-up");

    // energy (units of Ms V), max torque and gradient at v -> g; m and b_eff of
    // the point into mb, bb; with m0, b0 also the energy change from that point
    auto evaluate = [&](const double *v, double *g, double *mb, double *bb, const double *m0, const double *b0,
                        double &energy, double &torque, double &delta) -> demag_status {
        cudaError_t e2;
        if (fp64)
            k_relax_set_m<double><<<gN, 256, 0, st>>>(v, mask, (double *)self_layer, mb, N);
        else
            k_relax_set_m<float><<<gN, 256, 0, st>>>(v, mask, (float *)self_layer, mb, N);
        if ((e2 = cudaGetLastError()) != cudaSuccess) return cuda_fail(e2, "relaxation kernels");
        demag_status r = demag_apply(plan, w.self, Ms, w.h, 1, stream);
        if (r != DEMAG_OK) return r;
        if ((e2 = cudaMemsetAsync(w.acc, 0, 2 * 8, st)) != cudaSuccess) return cuda_fail(e2, "cudaMemsetAsync");
        if (fp64)
            k_relax_field<double><<<gN, kRelaxThreads, 0, st>>>(mb, v, (const double *)h_layer, w.bias, mask, nx, ny,
                                                                k, g, bb, w.acc);
        else
            k_relax_field<float><<<gN, kRelaxThreads, 0, st>>>(mb, v, (const float *)h_layer, w.bias, mask, nx, ny,
                                                               k, g, bb, w.acc);
        if (m0) k_relax_delta<<<1, kLbfgsThreads, 0, st>>>(m0, b0, mb, bb, n, w.acc + 4);
        if ((e2 = cudaGetLastError()) != cudaSuccess) return cuda_fail(e2, "relaxation kernels");
        if ((e2 = cudaMemcpyAsync(w.h_acc, w.acc, 2 * 8, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
            (m0 && (e2 = cudaMemcpyAsync(w.h_acc + 4, w.acc + 4, 8, cudaMemcpyDeviceToHost, st)) != cudaSuccess) ||
            (e2 = cudaStreamSynchronize(st)) != cudaSuccess)
            return cuda_fail(e2, "relaxation energy");
        energy = w.h_acc[0];
        torque = w.h_acc[1];
        delta = m0 ? w.h_acc[4] : 0.0;
        return DEMAG_OK;
    };

    double f = 0.0, tq = 0.0, df = 0.0;
    rc = evaluate(w.v, w.g, w.mlay, w.be, nullptr, nullptr, f, tq, df);
    if (rc != DEMAG_OK) return rc;
    int count = 0, newest = -1, it = 0, evals = 1;
    bool stalled = false;
    for (; it < prm->max_iter && tq >= prm->tol_torque; ++it) {
        k_lbfgs_dir<<<1, kLbfgsThreads, 0, st>>>(w.g, w.d, w.S, w.Y, w.rho, w.hist, count,
                                                 newest < 0 ? 0 : newest, n, w.acc + 2);
        if ((e = cudaGetLastError()) != cudaSuccess ||
            (e = cudaMemcpyAsync(w.h_acc + 2, w.acc + 2, 2 * 8, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
            (e = cudaStreamSynchronize(st)) != cudaSuccess)
            return cuda_fail(e, "L-BFGS direction");
        double gd = w.h_acc[2], dd = w.h_acc[3];
        bool fresh = count == 0;
        if (!(gd < 0.0)) {  // not a descent direction: start over from steepest descent
            count = 0;
            newest = -1;
            k_lbfgs_dir<<<1, kLbfgsThreads, 0, st>>>(w.g, w.d, w.S, w.Y, w.rho, w.hist, 0, 0, n, w.acc + 2);
            if ((e = cudaGetLastError()) != cudaSuccess ||
                (e = cudaMemcpyAsync(w.h_acc + 2, w.acc + 2, 2 * 8, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
                (e = cudaStreamSynchronize(st)) != cudaSuccess)
                return cuda_fail(e, "L-BFGS direction");
            gd = w.h_acc[2];
            dd = w.h_acc[3];
            fresh = true;
            if (!(gd < 0.0)) break;  // zero gradient
        }
        // unit step, or 0.1 rad RMS per magnetic cell for a fresh direction
        double a = 1.0;
        if (fresh) a = std::min(1.0, 0.1 / std::sqrt(std::max(dd / (double)N, 1e-300)));
        double ft = 0.0, tt = 0.0;
        bool ok = false;
        for (int bt = 0; bt < 40; ++bt) {
            k_axpy<<<gN, 256, 0, st>>>(w.v, w.d, a, w.vt, n);
            rc = evaluate(w.vt, w.gt, w.mlt, w.bet, w.mlay, w.be, ft, tt, df);
            ++evals;
            if (rc != DEMAG_OK) return rc;
            if (df <= 1e-4 * a * gd) {
                ok = true;
                break;
            }
            a *= 0.5;
        }
        if (!ok) {
            stalled = true;  // no step lowers the energy: converged to its rounding
            break;
        }
        newest = (newest + 1) % w.hist;
        k_lbfgs_pair<<<1, kLbfgsThreads, 0, st>>>(w.vt, w.v, w.gt, w.g, w.S, w.Y, w.rho, newest, n);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "L-BFGS update");
        count = std::min(count + 1, w.hist);
        std::swap(w.v, w.vt);
        std::swap(w.g, w.gt);
        std::swap(w.mlay, w.mlt);
        std::swap(w.be, w.bet);
        f = ft;
        tq = tt;
    }
    // the final state (m of the last accepted point) back into the caller's layer
    if (fp64)
        k_relax_out<double><<<gN, 256, 0, st>>>(w.mlay, (double *)layer_of, n);
    else
        k_relax_out<float><<<gN, 256, 0, st>>>(w.mlay, (float *)layer_of, n);
    if ((e = cudaGetLastError()) != cudaSuccess || (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return cuda_fail(e, "relaxation write-back");
    if (stats) {
        stats->iterations = it;
        stats->evaluations = evals;
        stats->energy = f * Ms * dxm * dym * plan->thickness[layer] * prm->length_unit;
        stats->max_torque = tq;
        stats->converged = tq < prm->tol_torque ? 1 : (stalled ? 2 : 0);
    }
    return DEMAG_OK;
}
