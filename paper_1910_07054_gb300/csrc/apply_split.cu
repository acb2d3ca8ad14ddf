// The hybrid field with the column transforms and the layer contraction in
// separate kernels, for stacks whose columns (3L planes x Py values, or B
// states of them) do not fit one block's shared memory.
//
//   k_columns_forward  per (kx, group of planes): the ny rows are zero-padded
//                      to Py and transformed along y (decimation in frequency);
//                      the bit-reversed spectrum is written as
//                      spec2[kx][p][plane], p the bit-reversed position, so that
//                      one frequency of all planes is contiguous.
//   k_contract         per (kx, tile of stored entries u): the two positions of
//                      each entry (ky and Py - ky) are staged in shared memory
//                      for all planes, H_k(b, i) = sum_j N_k(i <- j) m_k(b, j)
//                      is formed item by item (u, b, i), and the result is
//                      written back in place.
//   k_columns_inverse  per (kx, group of planes): spec2 -> inverse transform
//                      along y (decimation in time) -> spec[plane][kx][y < ny].
//
// For Py = 1024 the column transforms are those of cols1024.cu (two 512-point
// radix-8 transforms per zero-padded column, same layouts).  The row transforms
// are those of the fused path (apply.cu).
#include "fft.cuh"
#include "internal.h"
#include "layout.cuh"

namespace demag {

constexpr int kSplitThreads = 256;
constexpr int kSplitBatch = 8;

__device__ __forceinline__ int pair_index_s(int a, int b, int L) {
    return a * L - (a * (a - 1)) / 2 + (b - a);
}

template <typename C, typename T>
__device__ __forceinline__ void block_acc(C &ox, C &oy, C &oz, T kxx, T kyy, T kzz, T kxy, T kxz,
                                          T kyz, C mx, C my, C mz) {
    ox.x += kxx * mx.x + kxy * my.x - kxz * mz.y;
    ox.y += kxx * mx.y + kxy * my.y + kxz * mz.x;
    oy.x += kxy * mx.x + kyy * my.x - kyz * mz.y;
    oy.y += kxy * mx.y + kyy * my.y + kyz * mz.x;
    oz.x += -kxz * mx.y - kyz * my.y + kzz * mz.x;
    oz.y += kxz * mx.x + kyz * my.x + kzz * mz.y;
}

template <typename T>
__global__ void __launch_bounds__(kSplitThreads) k_columns_forward(
    const typename cpx_of<T>::type *__restrict__ spec, typename cpx_of<T>::type *__restrict__ spec2,
    int ny, int Kx, int planes, int G, int log2Py, const typename cpx_of<T>::type *__restrict__ tw,
    int log2tw) {
    using C = typename cpx_of<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *buf = reinterpret_cast<C *>(smem_raw);
    const int Py = 1 << log2Py, stride = Py + 1;
    const int kx = blockIdx.x, g0 = blockIdx.y * G;
    const int ng = min(G, planes - g0);
    const int total = ng * Py;
    for (int base = threadIdx.x; base < total; base += kSplitThreads * kSplitBatch) {
        C v[kSplitBatch];
#pragma unroll
        for (int k = 0; k < kSplitBatch; ++k) {
            const int e = base + k * kSplitThreads;
            const int g = e >> log2Py, y = e & (Py - 1);
            v[k] = C{0, 0};
            if (e < total && y < ny) v[k] = spec[((size_t)(g0 + g) * Kx + kx) * ny + y];
        }
#pragma unroll
        for (int k = 0; k < kSplitBatch; ++k) {
            const int e = base + k * kSplitThreads;
            if (e < total) buf[(e >> log2Py) * stride + (e & (Py - 1))] = v[k];
        }
    }
    __syncthreads();
    fft_dif<false>(buf, log2Py, ng, stride, tw, log2tw);
    C *out = spec2 + (size_t)kx * Py * planes + g0;
    for (int e = threadIdx.x; e < total; e += kSplitThreads) {
        const int p = e / ng, g = e - p * ng;
        out[(size_t)p * planes + g] = buf[g * stride + p];
    }
}

template <typename T>
__global__ void __launch_bounds__(kSplitThreads) k_columns_inverse(
    const typename cpx_of<T>::type *__restrict__ spec2, typename cpx_of<T>::type *__restrict__ spec,
    int ny, int Kx, int planes, int G, int log2Py, const typename cpx_of<T>::type *__restrict__ tw,
    int log2tw) {
    using C = typename cpx_of<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *buf = reinterpret_cast<C *>(smem_raw);
    const int Py = 1 << log2Py, stride = Py + 1;
    const int kx = blockIdx.x, g0 = blockIdx.y * G;
    const int ng = min(G, planes - g0);
    const int total = ng * Py;
    const C *in = spec2 + (size_t)kx * Py * planes + g0;
    for (int base = threadIdx.x; base < total; base += kSplitThreads * kSplitBatch) {
        C v[kSplitBatch];
#pragma unroll
        for (int k = 0; k < kSplitBatch; ++k) {
            const int e = base + k * kSplitThreads;
            const int p = e / ng, g = e - p * ng;
            v[k] = C{0, 0};
            if (e < total) v[k] = in[(size_t)p * planes + g];
        }
#pragma unroll
        for (int k = 0; k < kSplitBatch; ++k) {
            const int e = base + k * kSplitThreads;
            if (e < total) {
                const int p = e / ng, g = e - p * ng;
                buf[g * stride + p] = v[k];
            }
        }
    }
    __syncthreads();
    fft_dit<true>(buf, log2Py, ng, stride, tw, log2tw);
    for (int e = threadIdx.x; e < ng * ny; e += kSplitThreads) {
        const int g = e / ny, y = e - g * ny;
        spec[((size_t)(g0 + g) * Kx + kx) * ny + y] = buf[g * stride + y];
    }
}

// Layer contraction over stored entries [u0, u0 + TU) of one kx.  Shared
// memory holds, for each entry of the tile, the spectra of all planes at its
// two positions: stage[(uu * 2 + side) * planes + plane].
template <typename T>
__global__ void __launch_bounds__(kSplitThreads) k_contract(
    typename cpx_of<T>::type *__restrict__ spec2, const T *__restrict__ tensor,
    const T *__restrict__ ratio, int L, int B, int log2Py, int npairs, int QyS, int TU,
    int full_pairs) {
    using C = typename cpx_of<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *stage = reinterpret_cast<C *>(smem_raw);
    const int Py = 1 << log2Py, Qy = Py / 2 + 1;
    const int planes = B * 3 * L;
    const int kx = blockIdx.x, u0 = blockIdx.y * TU;
    const int nu = min(TU, Qy - u0);
    C *sk = spec2 + (size_t)kx * Py * planes;
    // stage the two positions of every entry (rows of `planes` contiguous values)
    const int rows = 2 * nu;
    for (int base = threadIdx.x; base < rows * planes; base += kSplitThreads * kSplitBatch) {
        C v[kSplitBatch];
#pragma unroll
        for (int k = 0; k < kSplitBatch; ++k) {
            const int e = base + k * kSplitThreads;
            v[k] = C{0, 0};
            if (e < rows * planes) {
                const int row = e / planes, g = e - row * planes;
                int p1, p2;
                u_positions(u0 + (row >> 1), log2Py, p1, p2);
                v[k] = sk[(size_t)((row & 1) ? p2 : p1) * planes + g];
            }
        }
#pragma unroll
        for (int k = 0; k < kSplitBatch; ++k) {
            const int e = base + k * kSplitThreads;
            if (e < rows * planes) stage[e] = v[k];
        }
    }
    __syncthreads();
    const T *tk = tensor + (size_t)kx * npairs * 6 * QyS;
    const int items = nu * B * L;
    // results stay in registers until every item has read its inputs
    constexpr int kMaxItems = 4;
    C res[kMaxItems][6];
#pragma unroll
    for (int q = 0; q < kMaxItems; ++q) {
        const int it = threadIdx.x + q * kSplitThreads;
        if (it >= items) break;
        const int uu = it % nu, rest = it / nu;
        const int b = rest % B, i = rest / B;
        const int u = u0 + uu;
        int p1, p2;
        u_positions(u, log2Py, p1, p2);
        const int ky1 = bit_reverse(p1, log2Py);
        const T s1 = ky1 > Py / 2 ? (T)-1 : (T)1;
        const T s2 = -s1;
        C a1x{0, 0}, a1y{0, 0}, a1z{0, 0}, a2x{0, 0}, a2y{0, 0}, a2z{0, 0};
        const C *m1 = stage + (size_t)(uu * 2) * planes + b * 3 * L;
        const C *m2 = m1 + planes;
        for (int j = 0; j < L; ++j) {
            bool up;
            int P;
            T r;
            if (full_pairs) {
                up = true;
                P = i * L + j;
                r = (T)1;
            } else {
                up = i <= j;
                P = up ? pair_index_s(i, j, L) : pair_index_s(j, i, L);
                r = up ? (T)1 : ratio[i * L + j];
            }
            const T *tp = tk + (size_t)P * 6 * QyS + u;
            const T kxx = r * tp[0], kyy = r * tp[QyS], kzz = r * tp[2 * QyS];
            const T kxy = r * tp[3 * QyS];
            const T kxz = (up ? r : -r) * tp[4 * QyS], kyz = (up ? r : -r) * tp[5 * QyS];
            block_acc(a1x, a1y, a1z, kxx, kyy, kzz, s1 * kxy, kxz, s1 * kyz, m1[3 * j], m1[3 * j + 1],
                      m1[3 * j + 2]);
            if (p2 != p1)
                block_acc(a2x, a2y, a2z, kxx, kyy, kzz, s2 * kxy, kxz, s2 * kyz, m2[3 * j],
                          m2[3 * j + 1], m2[3 * j + 2]);
        }
        res[q][0] = a1x;
        res[q][1] = a1y;
        res[q][2] = a1z;
        res[q][3] = a2x;
        res[q][4] = a2y;
        res[q][5] = a2z;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kMaxItems; ++q) {
        const int it = threadIdx.x + q * kSplitThreads;
        if (it >= items) break;
        const int uu = it % nu, rest = it / nu;
        const int b = rest % B, i = rest / B;
        C *o1 = stage + (size_t)(uu * 2) * planes + (b * L + i) * 3;
        C *o2 = o1 + planes;
        o1[0] = res[q][0];
        o1[1] = res[q][1];
        o1[2] = res[q][2];
        o2[0] = res[q][3];
        o2[1] = res[q][4];
        o2[2] = res[q][5];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < rows * planes; e += kSplitThreads) {
        const int row = e / planes, g = e - row * planes;
        int p1, p2;
        u_positions(u0 + (row >> 1), log2Py, p1, p2);
        if ((row & 1) && p2 == p1) continue;  // self-partnered entry: written once
        sk[(size_t)((row & 1) ? p2 : p1) * planes + g] = stage[e];
    }
}

// Tile of stored entries per contraction block: bounded by the staging size
// and by kMaxItems items per thread.
template <typename T>
static int split_tile(int L, int B, size_t smem_budget) {
    const size_t per_u = (size_t)2 * B * 3 * L * sizeof(typename cpx_of<T>::type);
    int tu = 64;
    while (tu > 1 && ((size_t)tu * per_u > smem_budget || (long long)tu * B * L > 4 * kSplitThreads))
        tu /= 2;
    return tu;
}

size_t split_workspace_bytes(int L, int B, int log2Px, int log2Py, bool fp64) {
    const size_t cpx = fp64 ? 16 : 8;
    return (size_t)((1 << log2Px) / 2 + 1) * (1 << log2Py) * B * 3 * L * cpx;
}

bool split_supported(int L, int B, bool fp64) {
    const size_t per_u = (size_t)2 * B * 3 * L * (fp64 ? 16 : 8);
    return per_u <= 200 * 1024 && (long long)B * L <= 4 * kSplitThreads;
}

template <typename T>
static cudaError_t split_columns(const ApplyArgs &a, cudaStream_t st, cudaEvent_t *ev) {
    using C = typename cpx_of<T>::type;
    const int Py = 1 << a.log2Py;
    const int Kx = a.kx_count ? a.kx_count : (1 << a.log2Px) / 2 + 1;
    const int planes = a.B * 3 * a.L;
    int G = 16;  // planes per column block: at most ~72 KB, so that 3 blocks share an SM
    while (G > 1 && (size_t)G * (Py + 1) * sizeof(C) > 72 * 1024) G /= 2;
    if (G > planes) G = planes;
    const size_t smem_col = (size_t)G * (Py + 1) * sizeof(C);
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_columns_forward<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem_col)) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(k_columns_inverse<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem_col)) != cudaSuccess)
        return e;
    dim3 gcol(Kx, (planes + G - 1) / G);
    const bool c1024 = cols1024_supported(a.log2Py, a.ny, sizeof(T) == 8);
    auto columns_inverse = [&]() -> cudaError_t {
        if (c1024) return launch_cols1024(true, a.spec2, a.spec, a.ny, Kx, planes, a.twy, a.log2twy, st);
        k_columns_inverse<T><<<gcol, kSplitThreads, smem_col, st>>>((const C *)a.spec2, (C *)a.spec, a.ny,
                                                                    Kx, planes, G, a.log2Py,
                                                                    (const C *)a.twy, a.log2twy);
        return cudaGetLastError();
    };
    cudaEvent_t *iev = a.inner_ev;
    if (iev && (e = cudaEventRecord(iev[0], st)) != cudaSuccess) return e;
    if (c1024) {
        e = launch_cols1024(false, a.spec, a.spec2, a.ny, Kx, planes, a.twy, a.log2twy, st);
    } else {
        k_columns_forward<T><<<gcol, kSplitThreads, smem_col, st>>>((const C *)a.spec, (C *)a.spec2, a.ny,
                                                                    Kx, planes, G, a.log2Py,
                                                                    (const C *)a.twy, a.log2twy);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return e;
    if (iev && (e = cudaEventRecord(iev[1], st)) != cudaSuccess) return e;
    if (a.contract_mode != 0) {
        e = a.contract_mode == 5   ? launch_zconv(a, sizeof(T) == 8, st)
            : a.contract_mode >= 3 ? launch_contract_tc5(a, a.contract_mode == 4, st)
                                   : launch_contract_gemm(a, a.contract_mode == 2, st);
        if (e != cudaSuccess) return e;
        if (iev && (e = cudaEventRecord(iev[2], st)) != cudaSuccess) return e;
        if ((e = columns_inverse()) != cudaSuccess) return e;
        if (iev && (e = cudaEventRecord(iev[3], st)) != cudaSuccess) return e;
        return cudaSuccess;
    }
    const int TU = split_tile<T>(a.L, a.B, 200 * 1024);
    const size_t smem_ct = (size_t)TU * 2 * planes * sizeof(C);
    if ((e = cudaFuncSetAttribute(k_contract<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem_ct)) != cudaSuccess)
        return e;
    const int Qy = Py / 2 + 1;
    dim3 gct(Kx, (Qy + TU - 1) / TU);
    k_contract<T><<<gct, kSplitThreads, smem_ct, st>>>((C *)a.spec2, (const T *)a.tensor,
                                                       (const T *)a.ratio, a.L, a.B, a.log2Py,
                                                       a.npairs, a.QyS, TU, a.full_pairs);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (iev && (e = cudaEventRecord(iev[2], st)) != cudaSuccess) return e;
    if ((e = columns_inverse()) != cudaSuccess) return e;
    if (iev && (e = cudaEventRecord(iev[3], st)) != cudaSuccess) return e;
    return cudaSuccess;
}

cudaError_t launch_split_columns(const ApplyArgs &a, bool fp64, cudaStream_t st) {
    if (fp64) return split_columns<double>(a, st, nullptr);
    return split_columns<float>(a, st, nullptr);
}

}  // namespace demag
