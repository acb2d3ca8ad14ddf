// The equidistant method of Sec. 3.1 (Eq. FFT_3D): when every layer has the
// same thickness dz, N(i <- j) depends on i - j alone, so the sum over the
// source layers at each in-plane frequency is itself a convolution along z and
// can be taken by a third, zero-padded FFT of length Pz >= 2 nz.
//
// The row and column transforms are those of the hybrid's split path; this
// file holds the step that replaces the layer contraction:
//
//   k_zconv    one warp per (kx, column position p) of the column spectrum
//              spec2[kx][p][B][L][3]: for each state the three components'
//              L values are zero-padded to Pz, transformed along z
//              (decimation in frequency, bit-reversed output), multiplied by
//              the real 3x3 tensor block of (kx, ky, kz), transformed back
//              (decimation in time, natural order) and written in place.
//   k_ztensor  plan set-up: the z-transform of the 2D-transformed kernels of
//              the offsets r = i - j.
//
// Tensor structure.  For cuboids of one size N(X, Y, -Z) = sx sy N(X, Y, Z)
// with sx, sy the component's parities in X and Y (the block is invariant
// under the full inversion d -> -d), so xx, yy, zz, xy are even in Z and xz,
// yz odd.  With the 2D transforms real (xx, yy, zz, xy) or imaginary (xz, yz:
// i c), the z-transform over r in (-nz, nz) is
//     even:  N2(0) + 2 sum_{r >= 1} N2(r) cos(2 pi kz r / Pz)
//     odd:   sum_{r >= 1} i c(r) (e^{-i th} - e^{i th}) = 2 sum_{r >= 1} c(r) sin(2 pi kz r / Pz)
// -- all six are real.  Only kz <= Pz / 2 is stored; kz > Pz / 2 negates xz and
// yz, and a mirrored y-frequency (ky > Py / 2) negates xy and yz, as in the
// hybrid.  1 / (Px Py Pz) is folded into the stored values.
#include <algorithm>

#include "fft.cuh"
#include "internal.h"
#include "layout.cuh"

namespace demag {

constexpr int kZWarps = 8;  // warps per block of k_zconv

template <typename T>
__global__ void k_ztensor(const double *__restrict__ src, T *__restrict__ dst, int Kx, int Qy, int QyS2, int L,
                          int log2Pz) {
    const int Pz = 1 << log2Pz, Qz = Pz / 2 + 1;
    const long long total = (long long)Kx * Qy * Qz;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int qz = (int)(idx % Qz);
        const long long t = idx / Qz;
        const int q = (int)(t % Qy), kx = (int)(t / Qy);
        double acc[6] = {0, 0, 0, 0, 0, 0};
        for (int r = 0; r < L; ++r) {
            const double *s = src + ((size_t)kx * L + r) * 6 * QyS2 + q;
            double sn, cs;
            sincospi(2.0 * (double)((long long)qz * r % Pz) / (double)Pz, &sn, &cs);
            const double we = r == 0 ? cs : 2.0 * cs;
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[c] += we * s[(size_t)c * QyS2];
#pragma unroll
            for (int c = 4; c < 6; ++c) acc[c] += 2.0 * sn * s[(size_t)c * QyS2];
        }
        T *o = dst + (size_t)idx * 6;
#pragma unroll
        for (int c = 0; c < 6; ++c) o[c] = (T)(acc[c] / (double)Pz);
    }
}

// Radix-2 transforms of the warp's three component rows x[c * Pz + i] in
// shared memory; tw[k] = exp(-2 pi i k / Pz), k < Pz / 2.
template <typename C>
__device__ __forceinline__ void warp_dif_forward(C *x, const C *tw, int log2Pz, int lane) {
    const int Pz = 1 << log2Pz, half = Pz / 2;
    for (int lh = log2Pz - 1; lh >= 0; --lh) {
        const int h = 1 << lh, ts = half >> lh;  // twiddle stride Pz / (2h)
        for (int k = lane; k < 3 * half; k += 32) {
            const int c = k / half, kk = k - c * half;
            const int j = kk & (h - 1), i0 = ((kk >> lh) << (lh + 1)) + j, i1 = i0 + h;
            C *xc = x + c * Pz;
            const C a = xc[i0], b = xc[i1], w = tw[j * ts];
            const C d = C{a.x - b.x, a.y - b.y};
            xc[i0] = C{a.x + b.x, a.y + b.y};
            xc[i1] = C{d.x * w.x - d.y * w.y, d.x * w.y + d.y * w.x};
        }
        __syncwarp();
    }
}

template <typename C>
__device__ __forceinline__ void warp_dit_inverse(C *x, const C *tw, int log2Pz, int lane) {
    const int Pz = 1 << log2Pz, half = Pz / 2;
    for (int lh = 0; lh < log2Pz; ++lh) {
        const int h = 1 << lh, ts = half >> lh;
        for (int k = lane; k < 3 * half; k += 32) {
            const int c = k / half, kk = k - c * half;
            const int j = kk & (h - 1), i0 = ((kk >> lh) << (lh + 1)) + j, i1 = i0 + h;
            C *xc = x + c * Pz;
            const C a = xc[i0], v = xc[i1], w = tw[j * ts];
            const C b = C{v.x * w.x + v.y * w.y, v.y * w.x - v.x * w.y};  // v * conj(w)
            xc[i0] = C{a.x + b.x, a.y + b.y};
            xc[i1] = C{a.x - b.x, a.y - b.y};
        }
        __syncwarp();
    }
}

template <typename T>
__global__ void __launch_bounds__(32 * kZWarps) k_zconv(typename cpx_of<T>::type *__restrict__ spec2,
                                                      const T *__restrict__ t3, const typename cpx_of<T>::type *twz,
                                                      int Kx, int log2Py, int L, int B, int log2Pz) {
    using C = typename cpx_of<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int Pz = 1 << log2Pz, half = Pz / 2, Qz = half + 1;
    const int Py = 1 << log2Py, Qy = Py / 2 + 1;
    C *tw = reinterpret_cast<C *>(smem_raw);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    C *x = tw + half + warp * 3 * Pz;
    for (int k = threadIdx.x; k < half; k += blockDim.x) tw[k] = twz[k];
    __syncthreads();
    const long long e = (long long)blockIdx.x * kZWarps + warp;
    if (e >= (long long)Kx * Py) return;
    const int kx = (int)(e >> log2Py), p = (int)(e & (Py - 1));
    const int ky = bitrev_n(p, log2Py);
    const int q = ky <= Py - ky ? ky : Py - ky;
    const T sy = ky > Py / 2 ? (T)-1 : (T)1;
    const T *tk = t3 + ((size_t)kx * Qy + q) * Qz * 6;
    const int planes = B * 3 * L;
    for (int b = 0; b < B; ++b) {
        C *row = spec2 + (size_t)e * planes + (size_t)b * 3 * L;
        for (int k = lane; k < 3 * Pz; k += 32) {
            const int c = k / Pz, l = k - c * Pz;
            if (l >= L) x[k] = C{0, 0};
        }
        for (int k = lane; k < 3 * L; k += 32) {
            const int l = k / 3, c = k - 3 * l;
            x[c * Pz + l] = row[k];
        }
        __syncwarp();
        warp_dif_forward(x, tw, log2Pz, lane);
        for (int j = lane; j < Pz; j += 32) {
            const int kz = bitrev_n(j, log2Pz);
            const int qz = kz <= Pz - kz ? kz : Pz - kz;
            const T sz = kz > half ? (T)-1 : (T)1;
            const T *n = tk + qz * 6;
            const T nxx = n[0], nyy = n[1], nzz = n[2], nxy = sy * n[3], nxz = sz * n[4], nyz = sy * sz * n[5];
            const C mx = x[j], my = x[Pz + j], mz = x[2 * Pz + j];
            x[j] = C{nxx * mx.x + nxy * my.x + nxz * mz.x, nxx * mx.y + nxy * my.y + nxz * mz.y};
            x[Pz + j] = C{nxy * mx.x + nyy * my.x + nyz * mz.x, nxy * mx.y + nyy * my.y + nyz * mz.y};
            x[2 * Pz + j] = C{nxz * mx.x + nyz * my.x + nzz * mz.x, nxz * mx.y + nyz * my.y + nzz * mz.y};
        }
        __syncwarp();
        warp_dit_inverse(x, tw, log2Pz, lane);
        for (int k = lane; k < 3 * L; k += 32) {
            const int l = k / 3, c = k - 3 * l;
            row[k] = x[c * Pz + l];
        }
        __syncwarp();
    }
}

size_t zconv_smem_bytes(int log2Pz, bool fp64) {
    const size_t cpx = fp64 ? 16 : 8;
    const size_t Pz = (size_t)1 << log2Pz;
    return (Pz / 2 + (size_t)kZWarps * 3 * Pz) * cpx;
}

cudaError_t launch_zconv(const ApplyArgs &a, bool fp64, cudaStream_t st) {
    const int Kx = (1 << a.log2Px) / 2 + 1, Py = 1 << a.log2Py;
    const size_t smem = zconv_smem_bytes(a.log2Pz, fp64);
    const long long entries = (long long)Kx * Py;
    const unsigned grid = (unsigned)((entries + kZWarps - 1) / kZWarps);
    cudaError_t e;
    if (fp64) {
        if ((e = cudaFuncSetAttribute(k_zconv<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
            cudaSuccess)
            return e;
        k_zconv<double><<<grid, 32 * kZWarps, smem, st>>>((double2 *)a.spec2, (const double *)a.tensor,
                                                          (const double2 *)a.twz, Kx, a.log2Py, a.L, a.B,
                                                          a.log2Pz);
    } else {
        if ((e = cudaFuncSetAttribute(k_zconv<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
            cudaSuccess)
            return e;
        k_zconv<float><<<grid, 32 * kZWarps, smem, st>>>((float2 *)a.spec2, (const float *)a.tensor,
                                                         (const float2 *)a.twz, Kx, a.log2Py, a.L, a.B, a.log2Pz);
    }
    return cudaGetLastError();
}

cudaError_t launch_ztensor(const double *src, void *dst, bool fp64, int log2Px, int log2Py, int QyS2, int L,
                           int log2Pz, cudaStream_t st) {
    const int Kx = (1 << log2Px) / 2 + 1, Qy = (1 << log2Py) / 2 + 1, Qz = (1 << log2Pz) / 2 + 1;
    const long long total = (long long)Kx * Qy * Qz;
    const unsigned grid = (unsigned)std::min<long long>((total + 255) / 256, 65535LL * 16);
    if (fp64)
        k_ztensor<double><<<grid, 256, 0, st>>>(src, (double *)dst, Kx, Qy, QyS2, L, log2Pz);
    else
        k_ztensor<float><<<grid, 256, 0, st>>>(src, (float *)dst, Kx, Qy, QyS2, L, log2Pz);
    return cudaGetLastError();
}

}  // namespace demag
