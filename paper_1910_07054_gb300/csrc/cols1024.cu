// Column transforms of the split path for Py = 1024 (257 <= ny <= 512), float:
// the y-transform of Eq. FFT_v2 on columns zero-padded from ny to 1024 values,
// as two 512-point radix-8 transforms per column (fft1024.cuh).
//
// Layouts are those of the generic column kernels: spec [plane][kx][ny] (the
// row transforms' output) and spec2 [kx][p][plane] with position p holding
// frequency ky = bitrev_10(p), so the contraction kernels are unchanged.
#include "fft1024.cuh"
#include "internal.h"

namespace demag {

namespace {

using namespace f1024;

__global__ void __launch_bounds__(kF10Threads, 2) k_columns_forward1024(const float2 *__restrict__ spec,
                                                                         float2 *__restrict__ spec2, int ny,
                                                                         int Kx, int planes,
                                                                         const float2 *__restrict__ tw, int sh) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *buf = reinterpret_cast<float2 *>(smem_raw);
    float2 *tws = buf + kF10Planes * kF10Plane;
    const int kx = blockIdx.y, g0 = blockIdx.x * kF10Planes;
    const int group = threadIdx.x >> 6, j = threadIdx.x & 63;
    const int g = g0 + group;
    f10_load_table(tws, tw, sh);
    // column values x[j + 64 r] (zero beyond ny and for planes past the end)
    float2 v[2][8];
    const float2 *src = spec + ((size_t)(g < planes ? g : 0) * Kx + kx) * ny;
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const int n = j + 64 * r;
        v[0][r] = (g < planes && n < ny) ? src[n] : float2{0.f, 0.f};
    }
    __syncthreads();  // twiddle table
#pragma unroll
    for (int r = 0; r < 8; ++r) v[1][r] = c_mul(v[0][r], f10_w<false>(tws, j + 64 * r));
    float2 *a = buf + group * kF10Plane, *b = a + kF10Col;
    const F10Bases bs(j);
    f10_transform<false>(v, a, b, bs, j, group, tws);
    // X[2k] = A[k], X[2k + 1] = B[k], k = j + 64 r: back to the columns (the
    // positions just read), then out through a transposed store
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        a[bs.bx(r)] = v[0][r];
        b[bs.bx(r)] = v[1][r];
    }
    __syncthreads();
    const int ng = min(kF10Planes, planes - g0);
    float2 *out = spec2 + (size_t)kx * 1024 * planes + g0;
    if ((planes & 1) == 0) {
        // planes in pairs, one 16-byte store each (planes even: ng is even and
        // the stores 16-byte aligned)
        constexpr int kP = kF10Planes / 2;
        for (int e = threadIdx.x; e < 1024 * kP; e += kF10Threads) {
            const int ky = e / kP, gg = 2 * (e % kP);
            if (gg >= ng) continue;
            const int p = (int)(__brev((unsigned)ky) >> 22);
            const float2 *src = buf + gg * kF10Plane + (ky & 1) * kF10Col + f10_pad(ky >> 1);
            const float2 x0 = src[0], x1 = src[kF10Plane];
            *reinterpret_cast<float4 *>(out + (size_t)p * planes + gg) = make_float4(x0.x, x0.y, x1.x, x1.y);
        }
        return;
    }
    for (int e = threadIdx.x; e < 1024 * kF10Planes; e += kF10Threads) {
        const int ky = e >> 3, gg = e & (kF10Planes - 1);
        if (gg >= ng) continue;
        const int p = (int)(__brev((unsigned)ky) >> 22);
        out[(size_t)p * planes + gg] = buf[gg * kF10Plane + (ky & 1) * kF10Col + f10_pad(ky >> 1)];
    }
}

__global__ void __launch_bounds__(kF10Threads, 2) k_columns_inverse1024(const float2 *__restrict__ spec2,
                                                                         float2 *__restrict__ spec, int ny,
                                                                         int Kx, int planes,
                                                                         const float2 *__restrict__ tw, int sh) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *buf = reinterpret_cast<float2 *>(smem_raw);
    float2 *tws = buf + kF10Planes * kF10Plane;
    const int kx = blockIdx.y, g0 = blockIdx.x * kF10Planes;
    const int group = threadIdx.x >> 6, j = threadIdx.x & 63;
    const int g = g0 + group;
    const int ng = min(kF10Planes, planes - g0);
    f10_load_table<true>(tws, tw, sh);  // W_64 slots permuted (fft1024.cuh)
    // Y[ky] from row p = bitrev(ky): even frequencies to column a, odd to b
    // (8 loads in flight per thread before their stores)
    const float2 *in = spec2 + (size_t)kx * 1024 * planes + g0;
    if ((planes & 1) == 0) {
        // planes in pairs, one 16-byte load each (planes even: 16-byte aligned);
        // all 8 loads of a thread in flight before their stores
        constexpr int kP = kF10Planes / 2;
        float4 t[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int e = q * kF10Threads + threadIdx.x;
            const int ky = e / kP, gg = 2 * (e % kP);
            const int p = (int)(__brev((unsigned)ky) >> 22);
            const float2 *src = in + (size_t)p * planes + gg;
            t[q] = gg + 1 < ng ? *reinterpret_cast<const float4 *>(src)
                   : gg < ng   ? make_float4(src->x, src->y, 0.f, 0.f)
                               : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int e = q * kF10Threads + threadIdx.x;
            const int ky = e / kP, gg = 2 * (e % kP);
            float2 *dst = buf + gg * kF10Plane + (ky & 1) * kF10Col + f10_pad(ky >> 1);
            dst[0] = make_float2(t[q].x, t[q].y);
            dst[kF10Plane] = make_float2(t[q].z, t[q].w);
        }
    } else {
        for (int base = 0; base < 1024 * kF10Planes; base += 8 * kF10Threads) {
            float2 t[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int e = base + q * kF10Threads + threadIdx.x;
                const int ky = e >> 3, gg = e & (kF10Planes - 1);
                const int p = (int)(__brev((unsigned)ky) >> 22);
                t[q] = gg < ng ? in[(size_t)p * planes + gg] : float2{0.f, 0.f};
            }
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int e = base + q * kF10Threads + threadIdx.x;
                const int ky = e >> 3, gg = e & (kF10Planes - 1);
                buf[gg * kF10Plane + (ky & 1) * kF10Col + f10_pad(ky >> 1)] = t[q];
            }
        }
    }
    __syncthreads();
    float2 *a = buf + group * kF10Plane, *b = a + kF10Col;
    const F10Bases bs(j);
    float2 v[2][8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        v[0][r] = a[bs.bx(r)];
        v[1][r] = b[bs.bx(r)];
    }
    f10_sync(group);  // pass 1 stores over positions other threads read
    f10_transform<true, true>(v, a, b, bs, j, group, tws);
    // y[n] = a[n] + W_1024^-n b[n], n = j + 64 r < ny
    if (g < planes) {
        float2 *dst = spec + ((size_t)g * Kx + kx) * ny;
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const int n = j + 64 * r;
            if (n < ny) dst[n] = c_add(v[0][r], c_mul(v[1][r], f10_w<true>(tws, n)));
        }
    }
}

}  // namespace

bool cols1024_supported(int log2Py, int ny, bool fp64) { return !fp64 && log2Py == 10 && ny <= 512; }

cudaError_t launch_cols1024(bool inverse, const void *src, void *dst, int ny, int Kx, int planes, const void *tw,
                            int log2tw, cudaStream_t st) {
    if (log2tw < 10) return cudaErrorInvalidValue;
    auto kern = inverse ? k_columns_inverse1024 : k_columns_forward1024;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kF10Smem);
    if (e != cudaSuccess) return e;
    // plane groups fastest: the blocks that share the 128-byte lines of one
    // spectrum2 row (8 planes each) run together and meet in L2
    const dim3 grid((planes + kF10Planes - 1) / kF10Planes, Kx);
    kern<<<grid, kF10Threads, kF10Smem, st>>>((const float2 *)src, (float2 *)dst, ny, Kx, planes,
                                              (const float2 *)tw, log2tw - 10);
    return cudaGetLastError();
}

}  // namespace demag
