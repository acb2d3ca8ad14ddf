// Row transforms for Px = 1024 (257 <= nx <= 512), float: the x-transform of
// Eq. FFT_v2 on rows zero-padded from nx to 1024 values, as two 512-point
// radix-8 transforms per sequence (fft1024.cuh).
//
// As in the generic row kernels, two real rows a, b of one plane travel as one
// complex sequence z = a + i b, and the layouts are m, H [plane][y][x] and
// spec [plane][kx][y] (kx = 0..512, the half spectrum, written transposed).
//   forward  Z = DFT_1024(z);  A[k] = (Z[k] + conj Z[-k]) / 2,
//            B[k] = (Z[k] - conj Z[-k]) / (2 i)
//   inverse  Z[k] = A[k] + i B[k],  Z[-k] = conj A[k] + i conj B[k] (the DC and
//            Nyquist bins of a real row are real);  a + i b = IDFT_1024(Z),
//            cropped to x < nx and scaled
// A block holds 8 row pairs (16 rows of one plane), one 64-thread group each.
#include "fft1024.cuh"
#include "internal.h"

namespace demag {

namespace {

using namespace f1024;

// Item e of the forward transform's untangling phase (ny even) -> x-frequency
// kx; its row pair is e mod 8.  Each 8 lanes take the 8 row pairs of one kx (one 128-byte run of
// the spectrum), and a half-warp's two kx are two apart (kx, kx + 2 of a group
// of four), so that their padded column slots differ by one and the 16 lanes'
// shared-memory accesses (plane stride 1150, even) meet 16 bank pairs instead
// of 8.  Items 4096..4103 give kx = 512.  (The inverse transform's placing
// stores have the same 2-way pattern; the same mapping there measured slower,
// 2.20 -> 2.24 ms at 512 x 512 x 64 x 16, and is not used.)
static_assert(kF10Planes == 8, "r10_kx maps 8 row pairs per kx");
__device__ __forceinline__ int r10_kx(int e) {
    const int s = (e >> 3) & 3;
    return 4 * (e >> 5) + (((s & 1) << 1) | (s >> 1));
}

constexpr int kR10Rows = 2 * kF10Planes;  // rows per block

__global__ void __launch_bounds__(kF10Threads, 2) k_rows_forward1024(const float *__restrict__ m,
                                                                      float2 *__restrict__ spec, int nx, int ny,
                                                                      const float2 *__restrict__ tw, int sh,
                                                                      const float *__restrict__ layer_scale,
                                                                      int L) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *buf = reinterpret_cast<float2 *>(smem_raw);
    float2 *tws = buf + kF10Planes * kF10Plane;
    const int plane = blockIdx.y, y0 = blockIdx.x * kR10Rows;
    const int group = threadIdx.x >> 6, j = threadIdx.x & 63;
    const float in_scale = layer_scale ? layer_scale[(plane / 3) % L] : 1.f;
    f10_load_table(tws, tw, sh);
    const int ya = y0 + 2 * group, yb = ya + 1;
    const float *ra = m + ((size_t)plane * ny + (ya < ny ? ya : 0)) * nx;
    const float *rb = m + ((size_t)plane * ny + (yb < ny ? yb : 0)) * nx;
    float2 v[2][8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const int x = j + 64 * r;
        const float va = (ya < ny && x < nx) ? ra[x] : 0.f;
        const float vb = (yb < ny && x < nx) ? rb[x] : 0.f;
        v[0][r] = float2{in_scale * va, in_scale * vb};
    }
    __syncthreads();  // twiddle table
#pragma unroll
    for (int r = 0; r < 8; ++r) v[1][r] = c_mul(v[0][r], f10_w<false>(tws, j + 64 * r));
    float2 *a = buf + group * kF10Plane, *b = a + kF10Col;
    const F10Bases bs(j);
    f10_transform<false>(v, a, b, bs, j, group, tws);
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        a[bs.bx(r)] = v[0][r];  // Z[2k], k = j + 64 r
        b[bs.bx(r)] = v[1][r];  // Z[2k + 1]
    }
    __syncthreads();
    float2 *sp = spec + (size_t)plane * 513 * ny;
    if ((ny & 1) == 0) {
        // untangle and store transposed, one item per (kx, row pair q): rows a
        // and b of the pair are adjacent in the spectrum, so both leave in one
        // 16-byte store (ny even) from one pair of reads
        for (int e = threadIdx.x; e < 513 * kF10Planes; e += kF10Threads) {
            const int kx = r10_kx(e), q = e % kF10Planes;
            const int ya = y0 + 2 * q;
            if (ya >= ny) continue;
            const float2 *zp = buf + q * kF10Plane;
            const int mk = (1024 - kx) & 1023;
            const float2 z1 = zp[(kx & 1) * kF10Col + f10_pad(kx >> 1)];
            const float2 z2 = zp[(mk & 1) * kF10Col + f10_pad(mk >> 1)];
            *reinterpret_cast<float4 *>(sp + (size_t)kx * ny + ya) =
                make_float4(0.5f * (z1.x + z2.x), 0.5f * (z1.y - z2.y), 0.5f * (z1.y + z2.y), 0.5f * (z2.x - z1.x));
        }
        return;
    }
    // odd ny: lane (kx, row r of the block)
    for (int e = threadIdx.x; e < 513 * kR10Rows; e += kF10Threads) {
        const int kx = e >> 4, r = e & (kR10Rows - 1);
        const int y = y0 + r;
        if (y >= ny) continue;
        const float2 *zp = buf + (r >> 1) * kF10Plane;
        const int mk = (1024 - kx) & 1023;
        const float2 z1 = zp[(kx & 1) * kF10Col + f10_pad(kx >> 1)];
        const float2 z2 = zp[(mk & 1) * kF10Col + f10_pad(mk >> 1)];
        const float2 o = (r & 1) == 0 ? float2{0.5f * (z1.x + z2.x), 0.5f * (z1.y - z2.y)}
                                      : float2{0.5f * (z1.y + z2.y), 0.5f * (z2.x - z1.x)};
        sp[(size_t)kx * ny + y] = o;
    }
}

__global__ void __launch_bounds__(kF10Threads, 2) k_rows_inverse1024(const float2 *__restrict__ spec,
                                                                      float *__restrict__ H, int nx, int ny,
                                                                      const float2 *__restrict__ tw, int sh,
                                                                      float out_scale,
                                                                      const float *__restrict__ layer_scale,
                                                                      int L) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2 *buf = reinterpret_cast<float2 *>(smem_raw);
    float2 *tws = buf + kF10Planes * kF10Plane;
    const int plane = blockIdx.y, y0 = blockIdx.x * kR10Rows;
    const int group = threadIdx.x >> 6, j = threadIdx.x & 63;
    const float scale = out_scale * (layer_scale ? layer_scale[(plane / 3) % L] : 1.f);
    f10_load_table(tws, tw, sh);
    // A (even rows of the block) and B (odd rows) of one kx give Z[kx] and
    // Z[1024 - kx]; all loads of a thread are issued before any is placed.
    const float2 *sp = spec + (size_t)plane * 513 * ny;
    if ((ny & 1) == 0) {
        // one item per (kx, row pair q): A and B in one 16-byte load (rows a, b
        // adjacent, ny even); the item places Z[kx] and Z[1024 - kx]
        constexpr int kItP = (513 * kF10Planes + kF10Threads - 1) / kF10Threads;  // 9
        float4 t4[kItP];
#pragma unroll
        for (int q = 0; q < kItP; ++q) {
            const int e = q * kF10Threads + threadIdx.x;
            const int kx = e / kF10Planes, ya = y0 + 2 * (e % kF10Planes);
            t4[q] = (e < 513 * kF10Planes && ya < ny)
                        ? *reinterpret_cast<const float4 *>(sp + (size_t)kx * ny + ya)
                        : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int q = 0; q < kItP; ++q) {
            const int e = q * kF10Threads + threadIdx.x;
            if (e >= 513 * kF10Planes) continue;
            const int kx = e / kF10Planes, pq = e % kF10Planes;
            const float2 A = make_float2(t4[q].x, t4[q].y), B = make_float2(t4[q].z, t4[q].w);
            float2 *zp = buf + pq * kF10Plane + (kx & 1) * kF10Col;  // 1024 - kx has the parity of kx
            if (kx == 0 || kx == 512) {
                zp[f10_pad(kx >> 1)] = float2{A.x, B.x};  // A, B real at DC and Nyquist
            } else {
                zp[f10_pad(kx >> 1)] = float2{A.x - B.y, A.y + B.x};
                zp[f10_pad((1024 - kx) >> 1)] = float2{A.x + B.y, B.x - A.y};
            }
        }
    } else {
        // odd ny: one item per (kx, row r); A and B meet in lanes 2q, 2q + 1, the
        // even lane places Z[kx], the odd one Z[1024 - kx] (the loops run the
        // same trip count in every thread: whole warps shuffle)
        constexpr int kIt = (513 * kR10Rows + kF10Threads - 1) / kF10Threads;  // 17
        float2 t[kIt];
#pragma unroll
        for (int q = 0; q < kIt; ++q) {
            const int e = q * kF10Threads + threadIdx.x;
            const int kx = e >> 4, r = e & (kR10Rows - 1);
            t[q] = (e < 513 * kR10Rows && y0 + r < ny) ? sp[(size_t)kx * ny + y0 + r] : float2{0.f, 0.f};
        }
#pragma unroll
        for (int q = 0; q < kIt; ++q) {
            const int e = q * kF10Threads + threadIdx.x;
            const int kx = e >> 4, r = e & (kR10Rows - 1);
            const float2 mine = t[q];
            const float2 other = float2{__shfl_xor_sync(0xffffffffu, mine.x, 1), __shfl_xor_sync(0xffffffffu, mine.y, 1)};
            if (e >= 513 * kR10Rows) continue;
            float2 A = (r & 1) ? other : mine, B = (r & 1) ? mine : other;
            float2 *zp = buf + (r >> 1) * kF10Plane + (kx & 1) * kF10Col;  // 1024 - kx has the parity of kx
            if (kx == 0 || kx == 512) {
                A.y = 0.f;
                B.y = 0.f;
                if ((r & 1) == 0) zp[f10_pad(kx >> 1)] = float2{A.x, B.x};
            } else if ((r & 1) == 0) {
                zp[f10_pad(kx >> 1)] = float2{A.x - B.y, A.y + B.x};
            } else {
                zp[f10_pad((1024 - kx) >> 1)] = float2{A.x + B.y, B.x - A.y};
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
    f10_transform<true>(v, a, b, bs, j, group, tws);
    // z[x] = e[x] + W_1024^-x o[x]: Re z -> row ya, Im z -> row yb
    const int ya = y0 + 2 * group, yb = ya + 1;
    float *ha = H + ((size_t)plane * ny + ya) * nx, *hb = ha + nx;
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const int x = j + 64 * r;
        if (x >= nx) continue;
        const float2 z = c_add(v[0][r], c_mul(v[1][r], f10_w<true>(tws, x)));
        if (ya < ny) ha[x] = scale * z.x;
        if (yb < ny) hb[x] = scale * z.y;
    }
}

}  // namespace

bool rows1024_supported(int log2Px, int nx, bool fp64) { return !fp64 && log2Px == 10 && nx <= 512; }

cudaError_t launch_rows1024(bool inverse, const void *src, void *dst, int nx, int ny, int planes, const void *tw,
                            int log2tw, float out_scale, const void *layer_scale, int L, cudaStream_t st) {
    if (log2tw < 10) return cudaErrorInvalidValue;
    const dim3 grid((ny + kR10Rows - 1) / kR10Rows, planes);
    cudaError_t e;
    if (!inverse) {
        if ((e = cudaFuncSetAttribute(k_rows_forward1024, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)kF10Smem)) != cudaSuccess)
            return e;
        k_rows_forward1024<<<grid, kF10Threads, kF10Smem, st>>>((const float *)src, (float2 *)dst, nx, ny,
                                                                 (const float2 *)tw, log2tw - 10,
                                                                 (const float *)layer_scale, L);
    } else {
        if ((e = cudaFuncSetAttribute(k_rows_inverse1024, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)kF10Smem)) != cudaSuccess)
            return e;
        k_rows_inverse1024<<<grid, kF10Threads, kF10Smem, st>>>((const float2 *)src, (float *)dst, nx, ny,
                                                                 (const float2 *)tw, log2tw - 10, out_scale,
                                                                 (const float *)layer_scale, L);
    }
    return cudaGetLastError();
}

}  // namespace demag
