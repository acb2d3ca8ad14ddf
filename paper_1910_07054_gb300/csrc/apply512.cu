// The hybrid field (Sec. 3, Eq. FFT_v2) for padded transforms of 512 points
// (grids with 128 < nx, ny <= 256), with the register-resident radix-8
// Stockham FFT of fft8.cuh.
//
// Same three steps as apply.cu (row R2C -> column FFT + layer contraction +
// inverse column FFT -> inverse row C2R), but every 512-point transform takes
// three radix-8 passes by a 64-thread group, the first pass reads global
// memory directly (the zero half of the padded input is never loaded) and the
// last inverse pass writes global memory directly (only the first half of the
// outputs is kept).  The spectra are in natural order, so the plan tensor of
// this path stores the folded y-frequency q = min(ky, Py - ky) at index q.
//
// Shared memory holds columns of 512 values with one padding slot per 8
// (index p + p / 8), which makes the radix-8 stores of the first pass
// conflict-free.
#include "fft8.cuh"
#include "internal.h"

namespace demag {

constexpr int kN8 = 512;
constexpr int kCol8 = kN8 + kN8 / 8;  // padded column length
constexpr int kGroup = 64;            // threads per transform

__device__ __forceinline__ int pad8i(int p) { return p + (p >> 3); }

__device__ __forceinline__ void group_sync(int group) {
    asm volatile("bar.sync %0, %1;" ::"r"(group + 1), "r"(kGroup) : "memory");
}

// Passes 2 and 3 of a forward or inverse transform held in shared memory
// (input written by pass 1 at its destinations).  For INV with to_global, the
// caller takes pass 3's outputs from `v` instead (positions j + 64 r).
template <bool INV, typename C>
__device__ __forceinline__ void passes23(C *col, int j, const C *__restrict__ tw, int group,
                                        C (&v)[8], bool store_last) {
    // pass 2: Ns = 8
#pragma unroll
    for (int r = 0; r < 8; ++r) v[r] = col[pad8i(j + 64 * r)];
    group_sync(group);
    twiddle8<INV>(v, tw, j & 7, 8);
    dft8<INV>(v);
#pragma unroll
    for (int r = 0; r < 8; ++r) col[pad8i(dest8(j, 8, r))] = v[r];
    group_sync(group);
    // pass 3: Ns = 64, destinations j + 64 r (the positions just read)
#pragma unroll
    for (int r = 0; r < 8; ++r) v[r] = col[pad8i(j + 64 * r)];
    twiddle8<INV>(v, tw, j, 64);
    dft8<INV>(v);
    if (store_last) {
#pragma unroll
        for (int r = 0; r < 8; ++r) col[pad8i(j + 64 * r)] = v[r];
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_rows_forward8(const T *__restrict__ m,
                                                      typename cpx_of<T>::type *__restrict__ spec,
                                                      int nx, int ny,
                                                      const typename cpx_of<T>::type *__restrict__ tw,
                                                      const T *__restrict__ layer_scale, int L) {
    using C = typename cpx_of<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *buf = reinterpret_cast<C *>(smem_raw);  // 8 row pairs x kCol8
    const int Kx = kN8 / 2 + 1;
    const int plane = blockIdx.y, y0 = blockIdx.x * 16;
    const int group = threadIdx.x >> 6, j = threadIdx.x & 63;
    const T *mp = m + (size_t)plane * ny * nx;
    const T sc = layer_scale ? layer_scale[(plane / 3) % L] : (T)1;
    // pass 1 (Ns = 1) straight from global memory: pairs group and group + 4,
    // z = row_a + i row_b, x = j + 64 r, zero for x >= nx (all r >= 4)
    C v[2][8];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int q = group + 4 * h, ya = y0 + 2 * q, yb = ya + 1;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int x = j + 64 * r;
            T a = 0, bv = 0;
            if (x < nx) {
                if (ya < ny) a = mp[(size_t)ya * nx + x];
                if (yb < ny) bv = mp[(size_t)yb * nx + x];
            }
            v[h][r] = C{sc * a, sc * bv};
        }
#pragma unroll
        for (int r = 4; r < 8; ++r) v[h][r] = C{0, 0};
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        dft8<false>(v[h]);
        C *col = buf + (group + 4 * h) * kCol8;
#pragma unroll
        for (int r = 0; r < 8; ++r) col[pad8i(8 * j + r)] = v[h][r];
    }
    group_sync(group);
#pragma unroll
    for (int h = 0; h < 2; ++h) passes23<false>(buf + (group + 4 * h) * kCol8, j, tw, group, v[h], true);
    __syncthreads();
    // A[k] = (Z[k] + conj Z[-k]) / 2,  B[k] = (Z[k] - conj Z[-k]) / (2i)
    C *sp = spec + (size_t)plane * Kx * ny;
    for (int e = threadIdx.x; e < Kx * 16; e += 256) {
        const int kx = e >> 4, r = e & 15;
        const int y = y0 + r;
        if (y >= ny) continue;
        const C *zb = buf + (r >> 1) * kCol8;
        const C z1 = zb[pad8i(kx)], z2 = zb[pad8i((kN8 - kx) & (kN8 - 1))];
        C o;
        if ((r & 1) == 0)
            o = C{(T)0.5 * (z1.x + z2.x), (T)0.5 * (z1.y - z2.y)};
        else
            o = C{(T)0.5 * (z1.y + z2.y), (T)0.5 * (z2.x - z1.x)};
        sp[(size_t)kx * ny + y] = o;
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_rows_inverse8(const typename cpx_of<T>::type *__restrict__ spec,
                                                      T *__restrict__ H, int nx, int ny,
                                                      const typename cpx_of<T>::type *__restrict__ tw,
                                                      T out_scale, const T *__restrict__ layer_scale,
                                                      int L) {
    using C = typename cpx_of<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *buf = reinterpret_cast<C *>(smem_raw);
    const int half = kN8 / 2, Kx = half + 1;
    const int plane = blockIdx.y, y0 = blockIdx.x * 16;
    const int group = threadIdx.x >> 6, j = threadIdx.x & 63;
    const C *sp = spec + (size_t)plane * Kx * ny;
    const T scale = out_scale * (layer_scale ? layer_scale[(plane / 3) % L] : (T)1);
    // Z[kx] = A + iB, Z[512 - kx] = conj(A) + i conj(B); DC and Nyquist real
    const int total = Kx * 8;
    for (int base = threadIdx.x; base < total; base += 256 * 4) {
        C A[4], Bv[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int e = base + k * 256;
            const int kx = e >> 3, q = e & 7;
            const int ya = y0 + 2 * q, yb = ya + 1;
            A[k] = C{0, 0};
            Bv[k] = C{0, 0};
            if (e < total) {
                if (ya < ny) A[k] = sp[(size_t)kx * ny + ya];
                if (yb < ny) Bv[k] = sp[(size_t)kx * ny + yb];
            }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int e = base + k * 256;
            if (e >= total) continue;
            const int kx = e >> 3, q = e & 7;
            C a = A[k], bv = Bv[k];
            if (kx == 0 || kx == half) {
                a.y = 0;
                bv.y = 0;
            }
            C *zb = buf + q * kCol8;
            zb[pad8i(kx)] = C{a.x - bv.y, a.y + bv.x};
            if (kx != 0 && kx != half) zb[pad8i(kN8 - kx)] = C{a.x + bv.y, bv.x - a.y};
        }
    }
    __syncthreads();
    C v[2][8];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const C *col = buf + (group + 4 * h) * kCol8;
#pragma unroll
        for (int r = 0; r < 8; ++r) v[h][r] = col[pad8i(j + 64 * r)];
    }
    group_sync(group);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        dft8<true>(v[h]);
        C *col = buf + (group + 4 * h) * kCol8;
#pragma unroll
        for (int r = 0; r < 8; ++r) col[pad8i(8 * j + r)] = v[h][r];
    }
    group_sync(group);
    T *hp = H + (size_t)plane * ny * nx;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        passes23<true>(buf + (group + 4 * h) * kCol8, j, tw, group, v[h], false);
        const int q = group + 4 * h, ya = y0 + 2 * q, yb = ya + 1;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int x = j + 64 * r;
            if (x >= nx) continue;
            if (ya < ny) hp[(size_t)ya * nx + x] = scale * v[h][r].x;
            if (yb < ny) hp[(size_t)yb * nx + x] = scale * v[h][r].y;
        }
    }
}

// Pair index of (a <= b) in the row-by-row numbering.
__device__ __forceinline__ int pair_index8(int a, int b, int L) {
    return a * L - (a * (a - 1)) / 2 + (b - a);
}

template <typename C, typename T>
__device__ __forceinline__ void block_apply8(C &ox, C &oy, C &oz, T kxx, T kyy, T kzz, T kxy, T kxz,
                                             T kyz, C mx, C my, C mz) {
    ox.x += kxx * mx.x + kxy * my.x - kxz * mz.y;
    ox.y += kxx * mx.y + kxy * my.y + kxz * mz.x;
    oy.x += kxy * mx.x + kyy * my.x - kyz * mz.y;
    oy.y += kxy * mx.y + kyy * my.y + kyz * mz.x;
    oz.x += -kxz * mx.y - kyz * my.y + kzz * mz.x;
    oz.y += kxz * mx.x + kyz * my.x + kzz * mz.y;
}

// Prefetch of [p, p + bytes) into L2 by bulk requests (p, bytes multiples of 16).
__device__ __forceinline__ void prefetch_l2_8(const void *p, size_t bytes) {
    const char *c = static_cast<const char *>(p);
    for (size_t off = 0; off < bytes; off += 65536) {
        const unsigned n = (unsigned)((bytes - off) < 65536 ? (bytes - off) : 65536);
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(c + off), "r"(n) : "memory");
    }
}

template <typename T, bool FULL>
__global__ void __launch_bounds__(256, 2) k_columns_fused8(typename cpx_of<T>::type *__restrict__ spec,
                                                          const T *__restrict__ tensor,
                                                          const T *__restrict__ ratio, int Kx, int ny,
                                                          int L, int npairs, int QyS, int TU,
                                                          const typename cpx_of<T>::type *__restrict__ tw) {
    using C = typename cpx_of<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *buf = reinterpret_cast<C *>(smem_raw);  // 3L columns x kCol8
    constexpr int Qy = kN8 / 2 + 1;  // Py = 512; Kx = Px / 2 + 1 for any Px
    const int kx = blockIdx.x, b = blockIdx.y;
    const int ncol = 3 * L;
    const int group = threadIdx.x >> 6, j = threadIdx.x & 63;
    const T *tk = tensor + (size_t)kx * npairs * 6 * QyS;
    if (threadIdx.x == 0) prefetch_l2_8(tk, (size_t)npairs * 6 * QyS * sizeof(T));
    C *sp = spec + (size_t)b * ncol * Kx * ny + (size_t)kx * ny;

    // forward pass 1 from global memory: the group's columns c = group + 4 t;
    // y = j + 64 r, zero for y >= ny (all r >= 4)
    for (int c0 = group; c0 < ncol; c0 += 8) {
        C v[2][8];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int c = c0 + 4 * h;
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int y = j + 64 * r;
                v[h][r] = (c < ncol && y < ny) ? sp[(size_t)c * Kx * ny + y] : C{0, 0};
            }
#pragma unroll
            for (int r = 4; r < 8; ++r) v[h][r] = C{0, 0};
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int c = c0 + 4 * h;
            if (c >= ncol) break;
            dft8<false>(v[h]);
            C *col = buf + c * kCol8;
#pragma unroll
            for (int r = 0; r < 8; ++r) col[pad8i(8 * j + r)] = v[h][r];
        }
    }
    group_sync(group);
    for (int c = group; c < ncol; c += 4) {
        C v[8];
        passes23<false>(buf + c * kCol8, j, tw, group, v, true);
    }
    __syncthreads();

    // contraction: items (folded frequency q, target layer i), TU q per pass;
    // q holds ky = q (sign +1 for xy, yz) and ky = 512 - q (sign -1)
    const int items = TU * L;
    for (int q0 = 0; q0 < Qy; q0 += TU) {
        const int it = threadIdx.x;
        const int i = it / TU, q = q0 + (it - i * TU);
        const bool active = it < items && q < Qy;
        C a1x{0, 0}, a1y{0, 0}, a1z{0, 0}, a2x{0, 0}, a2y{0, 0}, a2z{0, 0};
        const int p1 = pad8i(q), p2 = pad8i((kN8 - q) & (kN8 - 1));
        const bool two = q != 0 && q != kN8 / 2;
        if (active) {
#pragma unroll 4
            for (int jj = 0; jj < L; ++jj) {
                int P;
                T rr, sx;
                if (FULL) {
                    P = i * L + jj;
                    rr = (T)1;
                    sx = (T)1;
                } else {
                    const bool up = i <= jj;
                    P = up ? pair_index8(i, jj, L) : pair_index8(jj, i, L);
                    rr = up ? (T)1 : ratio[i * L + jj];  // t_j / t_i for the reversed pair
                    sx = up ? rr : -rr;                  // xz and yz change sign reversed
                }
                const T *tp = tk + (size_t)P * 6 * QyS + q;
                const T kxx = rr * tp[0], kyy = rr * tp[QyS], kzz = rr * tp[2 * QyS];
                const T kxy = rr * tp[3 * QyS], kxz = sx * tp[4 * QyS], kyz = sx * tp[5 * QyS];
                const C *mj = buf + 3 * jj * kCol8;
                block_apply8(a1x, a1y, a1z, kxx, kyy, kzz, kxy, kxz, kyz, mj[p1], mj[kCol8 + p1],
                             mj[2 * kCol8 + p1]);
                if (two)
                    block_apply8(a2x, a2y, a2z, kxx, kyy, kzz, -kxy, kxz, -kyz, mj[p2], mj[kCol8 + p2],
                                 mj[2 * kCol8 + p2]);
            }
        }
        __syncthreads();
        if (active) {
            C *mi = buf + 3 * i * kCol8;
            mi[p1] = a1x;
            mi[kCol8 + p1] = a1y;
            mi[2 * kCol8 + p1] = a1z;
            if (two) {
                mi[p2] = a2x;
                mi[kCol8 + p2] = a2y;
                mi[2 * kCol8 + p2] = a2z;
            }
        }
        __syncthreads();
    }

    // inverse: pass 1 in shared memory, passes 2 and 3, outputs y = j + 64 r
    for (int c0 = group; c0 < ncol; c0 += 8) {
        C v[2][8];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int c = c0 + 4 * h;
            if (c >= ncol) break;
            const C *col = buf + c * kCol8;
#pragma unroll
            for (int r = 0; r < 8; ++r) v[h][r] = col[pad8i(j + 64 * r)];
        }
        group_sync(group);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int c = c0 + 4 * h;
            if (c >= ncol) break;
            dft8<true>(v[h]);
            C *col = buf + c * kCol8;
#pragma unroll
            for (int r = 0; r < 8; ++r) col[pad8i(8 * j + r)] = v[h][r];
        }
        group_sync(group);
    }
    for (int c = group; c < ncol; c += 4) {
        C v[8];
        passes23<true>(buf + c * kCol8, j, tw, group, v, false);
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int y = j + 64 * r;
            if (y < ny) sp[(size_t)c * Kx * ny + y] = v[r];
        }
    }
}

bool cols512_supported(int log2Py, int L, bool fp64) {
    const size_t elem = fp64 ? sizeof(double2) : sizeof(float2);
    return log2Py == 9 && (size_t)3 * L * kCol8 * elem <= 220 * 1024;
}

template <typename T>
cudaError_t launch_rows512(const ApplyArgs &a, const void *m, void *H, bool forward, cudaStream_t st) {
    using C = typename cpx_of<T>::type;
    const size_t smem = (size_t)8 * kCol8 * sizeof(C);
    const dim3 grid((a.ny + 15) / 16, a.B * a.L * 3);
    cudaError_t e;
    if (forward) {
        if ((e = cudaFuncSetAttribute(k_rows_forward8<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem)) != cudaSuccess)
            return e;
        k_rows_forward8<T><<<grid, 256, smem, st>>>((const T *)m, (C *)a.spec, a.nx, a.ny,
                                                    (const C *)a.twx, (const T *)a.in_scale, a.L);
    } else {
        if ((e = cudaFuncSetAttribute(k_rows_inverse8<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem)) != cudaSuccess)
            return e;
        k_rows_inverse8<T><<<grid, 256, smem, st>>>((const C *)a.spec, (T *)H, a.nx, a.ny,
                                                    (const C *)a.twx, (T)(-a.Ms),
                                                    (const T *)a.out_scale, a.L);
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_cols512(const ApplyArgs &a, cudaStream_t st) {
    using C = typename cpx_of<T>::type;
    const size_t smem = (size_t)3 * a.L * kCol8 * sizeof(C);
    int TU = 1;
    while (2 * TU * a.L <= 256) TU *= 2;
    const int Kx = (1 << a.log2Px) / 2 + 1;
    const dim3 grid(Kx, a.B);
    cudaError_t e;
    if (a.full_pairs) {
        if ((e = cudaFuncSetAttribute(k_columns_fused8<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem)) != cudaSuccess ||
            (e = cudaFuncSetAttribute(k_columns_fused8<T, true>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                      (int)cudaSharedmemCarveoutMaxShared)) != cudaSuccess)
            return e;
        k_columns_fused8<T, true><<<grid, 256, smem, st>>>((C *)a.spec, (const T *)a.tensor,
                                                           (const T *)a.ratio, Kx, a.ny, a.L, a.npairs,
                                                           a.QyS, TU, (const C *)a.twy);
    } else {
        if ((e = cudaFuncSetAttribute(k_columns_fused8<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem)) != cudaSuccess ||
            (e = cudaFuncSetAttribute(k_columns_fused8<T, false>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                      (int)cudaSharedmemCarveoutMaxShared)) != cudaSuccess)
            return e;
        k_columns_fused8<T, false><<<grid, 256, smem, st>>>((C *)a.spec, (const T *)a.tensor,
                                                            (const T *)a.ratio, Kx, a.ny, a.L, a.npairs,
                                                            a.QyS, TU, (const C *)a.twy);
    }
    return cudaGetLastError();
}

template cudaError_t launch_rows512<float>(const ApplyArgs &, const void *, void *, bool, cudaStream_t);
template cudaError_t launch_rows512<double>(const ApplyArgs &, const void *, void *, bool, cudaStream_t);
template cudaError_t launch_cols512<float>(const ApplyArgs &, cudaStream_t);
template cudaError_t launch_cols512<double>(const ApplyArgs &, cudaStream_t);

}  // namespace demag
