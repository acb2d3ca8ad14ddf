// The hybrid demagnetization field (Sec. 3, Eq. FFT_v2) on the GPU.
//
//   H_i = -Ms F_y^-1 F_x^-1 sum_j [ F_x F_y (N_ij) F_x F_y (m_j) ]
//
// computed by three kernels per batch of states:
//   k_rows_forward  real-to-complex FFT along x of every row of m (zero-padded
//                   to Px), two real rows packed into one complex transform,
//                   decimation in frequency; the Px/2 + 1 bins of each row are
//                   written transposed, spec[plane][kx][y] (plane = (b, layer,
//                   component)).
//   k_columns_fused one block per (kx, state): the ny rows of all 3L planes are
//                   zero-padded to Py and transformed along y (decimation in
//                   frequency, bit-reversed result), contracted over the source
//                   layers at every ky with the symmetric 3x3 tensor blocks,
//                   transformed back (decimation in time, natural order) and
//                   the first ny rows written back in place.  The block's slice
//                   of the tensor is prefetched into L2 by one bulk request at
//                   the start, so its HBM stream overlaps the forward FFT.
//   k_rows_inverse  complex-to-real inverse FFT along x, cropped to nx and
//                   scaled by -Ms (the 1/(Px Py) of the inverse DFT is folded
//                   into the stored tensor).
// Float rows of Px = 512 and 1024 use the radix-8 kernels of apply512.cu and
// rows1024.cu instead of k_rows_forward / k_rows_inverse.
#include "fft.cuh"
#include "internal.h"
#include "layout.cuh"
#include "nvtx.cuh"

namespace demag {

// ---- row transforms ---------------------------------------------------------

constexpr int kRowThreads = 256;
constexpr int kRowPairsMax = 8;
constexpr size_t kRowSmemBudget = 96 * 1024;
constexpr int kLoadBatch = 8;  // independent global loads issued per thread before use

// Rows per block = 2 * npair, npair <= kRowPairsMax rows of Px + 1 complex
// values within kRowSmemBudget.
template <typename T>
static int row_pairs(int log2Px) {
    const size_t per = ((size_t)(1 << log2Px) + 1) * sizeof(typename cpx_of<T>::type);
    size_t n = kRowSmemBudget / per;
    if (n < 1) n = 1;
    if (n > (size_t)kRowPairsMax) n = kRowPairsMax;
    return (int)n;
}

template <typename T>
__global__ void __launch_bounds__(kRowThreads) k_rows_forward(const T *__restrict__ m,
                                                             typename cpx_of<T>::type *__restrict__ spec,
                                                             int nx, int ny, int log2Px, int npair,
                                                             const typename cpx_of<T>::type *__restrict__ tw,
                                                             int log2tw, const T *__restrict__ layer_scale,
                                                             int L) {
    using C = typename cpx_of<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *buf = reinterpret_cast<C *>(smem_raw);
    const int Px = 1 << log2Px, Kx = Px / 2 + 1, stride = Px + 1;
    const int plane = blockIdx.y;
    const int y0 = blockIdx.x * 2 * npair;
    const T *mp = m + (size_t)plane * ny * nx;
    const T in_scale = layer_scale ? layer_scale[(plane / 3) % L] : (T)1;
    // two rows -> one complex sequence z = row_a + i row_b, zero beyond nx
    const int total = npair * Px;
    for (int base = threadIdx.x; base < total; base += kRowThreads * kLoadBatch) {
        T va[kLoadBatch], vb[kLoadBatch];
#pragma unroll
        for (int k = 0; k < kLoadBatch; ++k) {
            const int e = base + k * kRowThreads;
            const int r = e >> log2Px, x = e & (Px - 1);
            const int ya = y0 + 2 * r, yb = ya + 1;
            va[k] = 0;
            vb[k] = 0;
            if (e < total && x < nx) {
                if (ya < ny) va[k] = mp[(size_t)ya * nx + x];
                if (yb < ny) vb[k] = mp[(size_t)yb * nx + x];
            }
        }
#pragma unroll
        for (int k = 0; k < kLoadBatch; ++k) {
            const int e = base + k * kRowThreads;
            if (e < total) buf[(e >> log2Px) * stride + (e & (Px - 1))] = C{in_scale * va[k], in_scale * vb[k]};
        }
    }
    __syncthreads();
    fft_dif<false>(buf, log2Px, npair, stride, tw, log2tw);  // Z[k] at position bitrev(k)
    // A[k] = (Z[k] + conj Z[-k]) / 2,  B[k] = (Z[k] - conj Z[-k]) / (2i)
    C *sp = spec + (size_t)plane * Kx * ny;
    const int rows = 2 * npair;
    for (int e = threadIdx.x; e < Kx * rows; e += kRowThreads) {
        const int kx = e / rows, r = e - kx * rows;
        const int y = y0 + r;
        if (y >= ny) continue;
        const C *zb = buf + (r >> 1) * stride;
        const C z1 = zb[bit_reverse(kx, log2Px)];
        const C z2 = zb[bit_reverse((Px - kx) & (Px - 1), log2Px)];
        C o;
        if ((r & 1) == 0)
            o = C{(T)0.5 * (z1.x + z2.x), (T)0.5 * (z1.y - z2.y)};
        else
            o = C{(T)0.5 * (z1.y + z2.y), (T)0.5 * (z2.x - z1.x)};
        sp[(size_t)kx * ny + y] = o;
    }
}

template <typename T>
__global__ void __launch_bounds__(kRowThreads) k_rows_inverse(const typename cpx_of<T>::type *__restrict__ spec,
                                                             T *__restrict__ H, int nx, int ny, int log2Px,
                                                             int npair,
                                                             const typename cpx_of<T>::type *__restrict__ tw,
                                                             int log2tw, T out_scale,
                                                             const T *__restrict__ layer_scale, int L) {
    using C = typename cpx_of<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *buf = reinterpret_cast<C *>(smem_raw);
    const int Px = 1 << log2Px, half = Px / 2, Kx = half + 1, stride = Px + 1;
    const int plane = blockIdx.y;
    const T scale = out_scale * (layer_scale ? layer_scale[(plane / 3) % L] : (T)1);
    const int y0 = blockIdx.x * 2 * npair;
    const C *sp = spec + (size_t)plane * Kx * ny;
    // Z[k] = A[k] + i B[k] on the full circle from the Hermitian halves:
    // Z[kx] = A + iB, Z[Px - kx] = conj(A) + i conj(B); the DC and Nyquist
    // bins of a real row are real.  Stored bit-reversed for the DIT transform.
    const int total = Kx * npair;
    for (int base = threadIdx.x; base < total; base += kRowThreads * kLoadBatch) {
        C A[kLoadBatch], Bv[kLoadBatch];
#pragma unroll
        for (int k = 0; k < kLoadBatch; ++k) {
            const int e = base + k * kRowThreads;
            const int kx = e / npair, r = e - kx * npair;
            const int ya = y0 + 2 * r, yb = ya + 1;
            A[k] = C{0, 0};
            Bv[k] = C{0, 0};
            if (e < total) {
                if (ya < ny) A[k] = sp[(size_t)kx * ny + ya];
                if (yb < ny) Bv[k] = sp[(size_t)kx * ny + yb];
            }
        }
#pragma unroll
        for (int k = 0; k < kLoadBatch; ++k) {
            const int e = base + k * kRowThreads;
            if (e >= total) continue;
            const int kx = e / npair, r = e - kx * npair;
            C a = A[k], bv = Bv[k];
            if (kx == 0 || kx == half) {
                a.y = 0;
                bv.y = 0;
            }
            C *zb = buf + r * stride;
            zb[bit_reverse(kx, log2Px)] = C{a.x - bv.y, a.y + bv.x};
            if (kx != 0 && kx != half) zb[bit_reverse(Px - kx, log2Px)] = C{a.x + bv.y, bv.x - a.y};
        }
    }
    __syncthreads();
    fft_dit<true>(buf, log2Px, npair, stride, tw, log2tw);  // natural order
    T *hp = H + (size_t)plane * ny * nx;
    const int rows = 2 * npair;
    for (int e = threadIdx.x; e < rows * nx; e += kRowThreads) {
        const int r = e / nx, x = e - r * nx;
        const int y = y0 + r;
        if (y >= ny) continue;
        const C z = buf[(r >> 1) * stride + x];
        hp[(size_t)y * nx + x] = scale * ((r & 1) ? z.y : z.x);
    }
}

// ---- fused column FFT + layer contraction ----------------------------------

// Stored pair index of (a <= b): pairs numbered row by row.
__device__ __forceinline__ int pair_index(int a, int b, int L) { return a * L - (a * (a - 1)) / 2 + (b - a); }

// out += K * in for the symmetric block K with real xx, yy, zz, xy and
// imaginary xz = i kxz, yz = i kyz.
template <typename C, typename T>
__device__ __forceinline__ void block_apply(C &ox, C &oy, C &oz, T kxx, T kyy, T kzz, T kxy, T kxz,
                                            T kyz, C mx, C my, C mz) {
    ox.x += kxx * mx.x + kxy * my.x - kxz * mz.y;
    ox.y += kxx * mx.y + kxy * my.y + kxz * mz.x;
    oy.x += kxy * mx.x + kyy * my.x - kyz * mz.y;
    oy.y += kxy * mx.y + kyy * my.y + kyz * mz.x;
    oz.x += -kxz * mx.y - kyz * my.y + kzz * mz.x;
    oz.y += kxz * mx.x + kyz * my.x + kzz * mz.y;
}

constexpr int kColThreads = 256;

// Bulk prefetch of [p, p + bytes) into L2 (p and bytes multiples of 16).
__device__ __forceinline__ void prefetch_l2(const void *p, size_t bytes) {
    const char *c = static_cast<const char *>(p);
    for (size_t off = 0; off < bytes; off += 65536) {
        const unsigned n = (unsigned)((bytes - off) < 65536 ? (bytes - off) : 65536);
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(c + off), "r"(n) : "memory");
    }
}

template <typename T>
__global__ void __launch_bounds__(kColThreads, 2) k_columns_fused(typename cpx_of<T>::type *__restrict__ spec,
                                                                  const T *__restrict__ tensor,
                                                                  const T *__restrict__ ratio, int ny,
                                                                  int L, int log2Px, int log2Py,
                                                                  int npairs, int QyS, int TU,
                                                                  int full_pairs,
                                                                  const typename cpx_of<T>::type *__restrict__ tw,
                                                                  int log2tw) {
    using C = typename cpx_of<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *buf = reinterpret_cast<C *>(smem_raw);
    const int Py = 1 << log2Py, Qy = Py / 2 + 1, stride = Py + 1;
    const int Kx = (1 << log2Px) / 2 + 1;
    const int kx = blockIdx.x, b = blockIdx.y;
    const int ncol = 3 * L;
    const T *tk = tensor + (size_t)kx * npairs * 6 * QyS;
    if (threadIdx.x == 0) prefetch_l2(tk, (size_t)npairs * 6 * QyS * sizeof(T));

    C *sp = spec + (size_t)b * ncol * Kx * ny + (size_t)kx * ny;
    const int total = ncol * Py;
    for (int base = threadIdx.x; base < total; base += kColThreads * kLoadBatch) {
        C v[kLoadBatch];
#pragma unroll
        for (int k = 0; k < kLoadBatch; ++k) {
            const int e = base + k * kColThreads;
            const int col = e >> log2Py, y = e & (Py - 1);
            v[k] = C{0, 0};
            if (e < total && y < ny) v[k] = sp[(size_t)col * Kx * ny + y];
        }
#pragma unroll
        for (int k = 0; k < kLoadBatch; ++k) {
            const int e = base + k * kColThreads;
            if (e < total) buf[(e >> log2Py) * stride + (e & (Py - 1))] = v[k];
        }
    }
    __syncthreads();
    fft_dif<false>(buf, log2Py, ncol, stride, tw, log2tw);  // ky at position bitrev(ky)

    // contraction: items (stored entry u, target layer i), TU entries per pass
    const int items = TU * L;
    for (int u0 = 0; u0 < Qy; u0 += TU) {
        const int it = threadIdx.x;
        const int i = it / TU, u = u0 + (it - i * TU);
        const bool active = it < items && u < Qy;
        C a1x{0, 0}, a1y{0, 0}, a1z{0, 0}, a2x{0, 0}, a2y{0, 0}, a2z{0, 0};
        int p1 = 0, p2 = 0;
        if (active) {
            u_positions(u, log2Py, p1, p2);
            const int ky1 = bit_reverse(p1, log2Py);
            const T s1 = ky1 > Py / 2 ? (T)-1 : (T)1;  // xy and yz are odd in ky
            const T s2 = -s1;                          // partner at Py - ky1
#pragma unroll 4
            for (int j = 0; j < L; ++j) {
                const bool up = full_pairs || i <= j;
                const int P = full_pairs ? i * L + j : (up ? pair_index(i, j, L) : pair_index(j, i, L));
                const T r = up ? (T)1 : ratio[i * L + j];  // t_j / t_i for the reversed pair
                const T *tp = tk + (size_t)P * 6 * QyS + u;
                const T kxx = r * tp[0], kyy = r * tp[QyS], kzz = r * tp[2 * QyS];
                const T kxy = r * tp[3 * QyS];
                const T kxz = (up ? r : -r) * tp[4 * QyS], kyz = (up ? r : -r) * tp[5 * QyS];
                const C *mj = buf + 3 * j * stride;
                block_apply(a1x, a1y, a1z, kxx, kyy, kzz, s1 * kxy, kxz, s1 * kyz, mj[p1],
                            mj[stride + p1], mj[2 * stride + p1]);
                if (p2 != p1)
                    block_apply(a2x, a2y, a2z, kxx, kyy, kzz, s2 * kxy, kxz, s2 * kyz, mj[p2],
                                mj[stride + p2], mj[2 * stride + p2]);
            }
        }
        __syncthreads();  // every item of this pass has read its inputs
        if (active) {
            C *mi = buf + 3 * i * stride;
            mi[p1] = a1x;
            mi[stride + p1] = a1y;
            mi[2 * stride + p1] = a1z;
            if (p2 != p1) {
                mi[p2] = a2x;
                mi[stride + p2] = a2y;
                mi[2 * stride + p2] = a2z;
            }
        }
        __syncthreads();
    }
    fft_dit<true>(buf, log2Py, ncol, stride, tw, log2tw);  // natural order
    for (int e = threadIdx.x; e < ncol * ny; e += kColThreads) {
        const int col = e / ny, y = e - col * ny;
        sp[(size_t)col * Kx * ny + y] = buf[col * stride + y];
    }
}

int fused_max_layers(bool fp64, int log2Py) {
    const size_t elem = fp64 ? sizeof(double2) : sizeof(float2);
    const size_t col = ((size_t)(1 << log2Py) + 1) * elem;
    const size_t budget = 220 * 1024;
    const int byL = (int)(budget / (3 * col));
    return byL < 256 ? byL : 256;
}

// Entries of the stored y-frequency order per contraction pass: the largest
// power of two with TU * L <= kColThreads.
static int contraction_tile(int L) {
    int t = 1;
    while (2 * t * L <= kColThreads) t *= 2;
    return t;
}

template <typename T>
static cudaError_t launch_fused(const ApplyArgs &a, cudaStream_t st) {
    using C = typename cpx_of<T>::type;
    const int Py = 1 << a.log2Py;
    const int Kx = (1 << a.log2Px) / 2 + 1;
    const size_t smem = (size_t)3 * a.L * (Py + 1) * sizeof(C);
    cudaError_t e = cudaFuncSetAttribute(k_columns_fused<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_columns_fused<T>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    dim3 grid(Kx, a.B);
    k_columns_fused<T><<<grid, kColThreads, smem, st>>>((C *)a.spec, (const T *)a.tensor,
                                                         (const T *)a.ratio, a.ny, a.L, a.log2Px,
                                                         a.log2Py, a.npairs, a.QyS,
                                                         contraction_tile(a.L), a.full_pairs,
                                                         (const C *)a.twy, a.log2twy);
    return cudaGetLastError();
}

// Row transforms of the a.B states of a (forward: m -> a.spec; inverse:
// a.spec -> H, cropped and scaled by -Ms).
template <typename T>
static cudaError_t rows_stage(const ApplyArgs &a, const T *m, T *H, bool forward, cudaStream_t st) {
    using C = typename cpx_of<T>::type;
    const int Px = 1 << a.log2Px;
    const int planes = a.planes ? a.planes : a.B * a.L * 3;
    const int npair = row_pairs<T>(a.log2Px);
    const int chunks = (a.ny + 2 * npair - 1) / (2 * npair);
    const size_t smem_rows = (size_t)npair * (Px + 1) * sizeof(C);
    cudaError_t e;
    if (a.log2Px == 9) return launch_rows512<T>(a, m, H, forward, st);
    if (rows1024_supported(a.log2Px, a.nx, sizeof(T) == 8))
        return forward ? launch_rows1024(false, m, a.spec, a.nx, a.ny, planes, a.twx, a.log2twx, 0.f, a.in_scale,
                                         a.L, st)
                       : launch_rows1024(true, a.spec, H, a.nx, a.ny, planes, a.twx, a.log2twx, (float)(-a.Ms),
                                         a.out_scale, a.L, st);
    dim3 grid_rows(chunks, planes);
    if (forward) {
        e = cudaFuncSetAttribute(k_rows_forward<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_rows);
        if (e != cudaSuccess) return e;
        k_rows_forward<T><<<grid_rows, kRowThreads, smem_rows, st>>>(m, (C *)a.spec, a.nx, a.ny, a.log2Px, npair,
                                                                     (const C *)a.twx, a.log2twx,
                                                                     (const T *)a.in_scale, a.L);
    } else {
        e = cudaFuncSetAttribute(k_rows_inverse<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_rows);
        if (e != cudaSuccess) return e;
        k_rows_inverse<T><<<grid_rows, kRowThreads, smem_rows, st>>>((const C *)a.spec, H, a.nx, a.ny, a.log2Px,
                                                                     npair, (const C *)a.twx, a.log2twx, (T)(-a.Ms),
                                                                     (const T *)a.out_scale, a.L);
    }
    return cudaGetLastError();
}

template <typename T>
static cudaError_t columns_stage(const ApplyArgs &a, cudaStream_t st) {
    return a.split ? launch_split_columns(a, sizeof(T) == 8, st)
                   : (a.natural ? launch_cols512<T>(a, st) : launch_fused<T>(a, st));
}

template <typename T>
static cudaError_t apply_impl(const ApplyArgs &a, const T *m, T *H, cudaStream_t st,
                              cudaEvent_t *ev) {
    cudaError_t e;
    if (ev && (e = cudaEventRecord(ev[0], st)) != cudaSuccess) return e;
    {
        NvtxRange r("demag rows forward");
        if ((e = rows_stage<T>(a, m, H, true, st)) != cudaSuccess) return e;
    }
    if (ev && (e = cudaEventRecord(ev[1], st)) != cudaSuccess) return e;
    {
        NvtxRange r("demag columns and layer sum");
        if ((e = columns_stage<T>(a, st)) != cudaSuccess) return e;
    }
    if (ev && (e = cudaEventRecord(ev[2], st)) != cudaSuccess) return e;
    {
        NvtxRange r("demag rows inverse");
        if ((e = rows_stage<T>(a, m, H, false, st)) != cudaSuccess) return e;
    }
    if (ev && (e = cudaEventRecord(ev[3], st)) != cudaSuccess) return e;
    return cudaSuccess;
}

cudaError_t launch_apply_stage(const ApplyArgs &a, int stage, const void *m, void *H, bool fp64, cudaStream_t st) {
    NvtxRange r(stage == 0 ? "demag rows forward" : stage == 1 ? "demag columns and layer sum" : "demag rows inverse");
    if (stage == 1) return fp64 ? columns_stage<double>(a, st) : columns_stage<float>(a, st);
    if (fp64) return rows_stage<double>(a, (const double *)m, (double *)H, stage == 0, st);
    return rows_stage<float>(a, (const float *)m, (float *)H, stage == 0, st);
}

cudaError_t launch_apply(const ApplyArgs &a, const void *m, void *H, bool fp64, cudaStream_t st,
                         cudaEvent_t *events) {
    if (fp64) return apply_impl<double>(a, (const double *)m, (double *)H, st, events);
    return apply_impl<float>(a, (const float *)m, (float *)H, st, events);
}

}  // namespace demag
