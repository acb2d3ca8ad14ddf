// The hybrid demagnetization field (Sec. 3, Eq. FFT_v2) on the GPU.
//
//   H_i = -Ms F_2^-1 F_1^-1 sum_j [ F_1 F_2 (N_ij) F_1 F_2 (m_j) ]
//
// computed by three kernels per batch of states:
//   k_rows_forward  real-to-complex FFT along x of every row of m (zero-padded
//                   to Px), two real rows packed into one complex transform;
//                   the nx/2+1.. Px/2+1 half spectrum is written transposed,
//                   spec[plane][kx][y] (plane = (b, layer, component)).
//   k_columns_fused per kx column and state: the ny rows of all 3L planes are
//                   zero-padded to Py and transformed along y (DIT), contracted
//                   over the source layers at every ky with the symmetric 3x3
//                   tensor blocks, transformed back (DIF) and the first ny rows
//                   written back in place.
//   k_rows_inverse  complex-to-real inverse FFT along x, cropped to nx and
//                   scaled by -Ms (the 1/(Px Py) of the inverse DFT is folded
//                   into the stored tensor).
#include "fft.cuh"
#include "internal.h"

namespace demag {

// ---- row transforms ---------------------------------------------------------

// Rows handled per block by the row kernels: 2 * npair, npair <= kRowPairsMax
// chosen so that npair rows of Px + 1 complex values fit kRowSmemBudget.
constexpr int kRowPairsMax = 8;
constexpr size_t kRowSmemBudget = 96 * 1024;

template <typename T>
static int row_pairs(int log2Px) {
    const size_t per = ((size_t)(1 << log2Px) + 1) * sizeof(typename cpx_of<T>::type);
    size_t n = kRowSmemBudget / per;
    if (n < 1) n = 1;
    if (n > (size_t)kRowPairsMax) n = kRowPairsMax;
    return (int)n;
}

template <typename T>
__global__ void __launch_bounds__(256) k_rows_forward(const T *__restrict__ m,
                                                      typename cpx_of<T>::type *__restrict__ spec,
                                                      int nx, int ny, int log2Px, int npair,
                                                      const typename cpx_of<T>::type *__restrict__ tw,
                                                      int log2tw) {
    using C = typename cpx_of<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *buf = reinterpret_cast<C *>(smem_raw);
    const int Px = 1 << log2Px, Kx = Px / 2 + 1, stride = Px + 1;
    const int plane = blockIdx.y;
    const int y0 = blockIdx.x * 2 * npair;
    const T *mp = m + (size_t)plane * ny * nx;
    // two rows -> one complex sequence z = row_a + i row_b, zero beyond nx
    for (int e = threadIdx.x; e < npair * Px; e += blockDim.x) {
        const int k = e >> log2Px, x = e & (Px - 1);
        const int ya = y0 + 2 * k, yb = ya + 1;
        T va = 0, vb = 0;
        if (x < nx) {
            if (ya < ny) va = mp[(size_t)ya * nx + x];
            if (yb < ny) vb = mp[(size_t)yb * nx + x];
        }
        buf[k * stride + bit_reverse(x, log2Px)] = C{va, vb};
    }
    __syncthreads();
    fft_dit<false>(buf, log2Px, npair, stride, tw, log2tw);
    // A[k] = (Z[k] + conj Z[-k]) / 2,  B[k] = (Z[k] - conj Z[-k]) / (2i)
    C *sp = spec + (size_t)plane * Kx * ny;
    const int rows = 2 * npair;
    for (int e = threadIdx.x; e < Kx * rows; e += blockDim.x) {
        const int kx = e / rows, r = e - kx * rows;
        const int y = y0 + r;
        if (y >= ny) continue;
        const C *zb = buf + (r >> 1) * stride;
        const C z1 = zb[kx], z2 = zb[(Px - kx) & (Px - 1)];
        C o;
        if ((r & 1) == 0)
            o = C{(T)0.5 * (z1.x + z2.x), (T)0.5 * (z1.y - z2.y)};
        else
            o = C{(T)0.5 * (z1.y + z2.y), (T)0.5 * (z2.x - z1.x)};
        sp[(size_t)kx * ny + y] = o;
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_rows_inverse(const typename cpx_of<T>::type *__restrict__ spec,
                                                      T *__restrict__ H, int nx, int ny, int log2Px,
                                                      int npair,
                                                      const typename cpx_of<T>::type *__restrict__ tw,
                                                      int log2tw, T scale) {
    using C = typename cpx_of<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *buf = reinterpret_cast<C *>(smem_raw);
    const int Px = 1 << log2Px, half = Px / 2, Kx = half + 1, stride = Px + 1;
    const int plane = blockIdx.y;
    const int y0 = blockIdx.x * 2 * npair;
    const C *sp = spec + (size_t)plane * Kx * ny;
    const int rows = 2 * npair;
    // Z[k] = A[k] + i B[k] on the full circle from the Hermitian halves:
    // Z[kx] = A + iB, Z[Px - kx] = conj(A) + i conj(B); the DC and Nyquist
    // bins of a real row are real.
    for (int e = threadIdx.x; e < Kx * npair; e += blockDim.x) {
        const int kx = e / npair, k = e - kx * npair;
        const int ya = y0 + 2 * k, yb = ya + 1;
        C A = C{0, 0}, Bv = C{0, 0};
        if (ya < ny) A = sp[(size_t)kx * ny + ya];
        if (yb < ny) Bv = sp[(size_t)kx * ny + yb];
        if (kx == 0 || kx == half) {
            A.y = 0;
            Bv.y = 0;
        }
        C *zb = buf + k * stride;
        zb[kx] = C{A.x - Bv.y, A.y + Bv.x};
        if (kx != 0 && kx != half) zb[Px - kx] = C{A.x + Bv.y, Bv.x - A.y};
    }
    __syncthreads();
    fft_dif<true>(buf, log2Px, npair, stride, tw, log2tw);
    T *hp = H + (size_t)plane * ny * nx;
    for (int e = threadIdx.x; e < rows * nx; e += blockDim.x) {
        const int r = e / nx, x = e - r * nx;
        const int y = y0 + r;
        if (y >= ny) continue;
        const C z = buf[(r >> 1) * stride + bit_reverse(x, log2Px)];
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

template <typename T, int LMAX, int NT>
__global__ void __launch_bounds__(NT) k_columns_fused(typename cpx_of<T>::type *__restrict__ spec,
                                                       const T *__restrict__ tensor,
                                                       const T *__restrict__ ratio, int ny, int L,
                                                       int log2Px, int log2Py, int npairs,
                                                       const typename cpx_of<T>::type *__restrict__ tw,
                                                       int log2tw) {
    using C = typename cpx_of<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *buf = reinterpret_cast<C *>(smem_raw);
    const int Py = 1 << log2Py, Qy = Py / 2 + 1, stride = Py + 1;
    const int Kx = (1 << log2Px) / 2 + 1;
    const int kx = blockIdx.x, b = blockIdx.y;
    const int ncol = 3 * L;
    C *sp = spec + (size_t)b * ncol * Kx * ny + (size_t)kx * ny;
    for (int e = threadIdx.x; e < ncol * Py; e += blockDim.x) {
        const int col = e >> log2Py, y = e & (Py - 1);
        C v = C{0, 0};
        if (y < ny) v = sp[(size_t)col * Kx * ny + y];
        buf[col * stride + bit_reverse(y, log2Py)] = v;
    }
    __syncthreads();
    fft_dit<false>(buf, log2Py, ncol, stride, tw, log2tw);

    const T *tk = tensor + (size_t)kx * npairs * 6 * Qy;
    for (int ky = threadIdx.x; ky < Py; ky += blockDim.x) {
        const bool mirror = ky > Py / 2;
        const int kq = mirror ? Py - ky : ky;
        const T sy = mirror ? (T)-1 : (T)1;  // xy and yz are odd in y
        C acc[3 * LMAX];
#pragma unroll
        for (int c = 0; c < 3 * LMAX; ++c) acc[c] = C{0, 0};
#pragma unroll
        for (int a = 0; a < LMAX; ++a) {
#pragma unroll
            for (int bb = a; bb < LMAX; ++bb) {
                if (a >= L || bb >= L) continue;
                const T *tp = tk + (size_t)pair_index(a, bb, L) * 6 * Qy + kq;
                const T kxx = tp[0], kyy = tp[Qy], kzz = tp[2 * Qy];
                const T kxy = sy * tp[3 * Qy], kxz = tp[4 * Qy], kyz = sy * tp[5 * Qy];
                // target a <- source bb
                const C mbx = buf[(3 * bb + 0) * stride + ky];
                const C mby = buf[(3 * bb + 1) * stride + ky];
                const C mbz = buf[(3 * bb + 2) * stride + ky];
                block_apply(acc[3 * a], acc[3 * a + 1], acc[3 * a + 2], kxx, kyy, kzz, kxy, kxz, kyz,
                            mbx, mby, mbz);
                if (bb != a) {
                    // target bb <- source a: (t_a / t_bb) times the block at -k,
                    // i.e. xz and yz change sign (reciprocity)
                    const T r = ratio[bb * L + a];
                    const C max_ = buf[(3 * a + 0) * stride + ky];
                    const C may = buf[(3 * a + 1) * stride + ky];
                    const C maz = buf[(3 * a + 2) * stride + ky];
                    block_apply(acc[3 * bb], acc[3 * bb + 1], acc[3 * bb + 2], r * kxx, r * kyy,
                                r * kzz, r * kxy, -r * kxz, -r * kyz, max_, may, maz);
                }
            }
        }
        // every thread owns its ky column entries: the inputs for this ky were
        // read above, so the results can replace them in place
#pragma unroll
        for (int c = 0; c < 3 * LMAX; ++c)
            if (c < 3 * L) buf[c * stride + ky] = acc[c];
    }
    __syncthreads();
    fft_dif<true>(buf, log2Py, ncol, stride, tw, log2tw);
    for (int e = threadIdx.x; e < ncol * ny; e += blockDim.x) {
        const int col = e / ny, y = e - col * ny;
        sp[(size_t)col * Kx * ny + y] = buf[col * stride + bit_reverse(y, log2Py)];
    }
}

int fused_max_layers(bool fp64, int log2Py) {
    const size_t elem = fp64 ? sizeof(double2) : sizeof(float2);
    const size_t col = ((size_t)(1 << log2Py) + 1) * elem;
    const size_t budget = 220 * 1024;
    int byL = (int)(budget / (3 * col));
    const int lmax = fp64 ? 8 : 16;
    return byL < lmax ? byL : lmax;
}

template <typename T, int LMAX, int NT>
static cudaError_t launch_fused(const ApplyArgs &a, cudaStream_t st) {
    using C = typename cpx_of<T>::type;
    const int Py = 1 << a.log2Py;
    const int Kx = (1 << a.log2Px) / 2 + 1;
    const size_t smem = (size_t)3 * a.L * (Py + 1) * sizeof(C);
    cudaError_t e = cudaFuncSetAttribute(k_columns_fused<T, LMAX, NT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid(Kx, a.B);
    k_columns_fused<T, LMAX, NT><<<grid, NT, smem, st>>>(
        (C *)a.spec, (const T *)a.tensor, (const T *)a.ratio, a.ny, a.L, a.log2Px, a.log2Py,
        a.npairs, (const C *)a.twy, a.log2twy);
    return cudaGetLastError();
}

template <typename T>
static cudaError_t apply_impl(const ApplyArgs &a, const T *m, T *H, cudaStream_t st,
                              cudaEvent_t *ev) {
    using C = typename cpx_of<T>::type;
    const int Px = 1 << a.log2Px;
    const int planes = a.B * a.L * 3;
    const int npair = row_pairs<T>(a.log2Px);
    const int chunks = (a.ny + 2 * npair - 1) / (2 * npair);
    const size_t smem_rows = (size_t)npair * (Px + 1) * sizeof(C);
    cudaError_t e;
    e = cudaFuncSetAttribute(k_rows_forward<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem_rows);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_rows_inverse<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem_rows);
    if (e != cudaSuccess) return e;
    dim3 grid_rows(chunks, planes);
    if (ev && (e = cudaEventRecord(ev[0], st)) != cudaSuccess) return e;
    k_rows_forward<T><<<grid_rows, 256, smem_rows, st>>>(m, (C *)a.spec, a.nx, a.ny, a.log2Px, npair,
                                                         (const C *)a.twx, a.log2twx);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (ev && (e = cudaEventRecord(ev[1], st)) != cudaSuccess) return e;
    if (a.L <= 4)
        e = launch_fused<T, 4, 512>(a, st);
    else if (a.L <= 8)
        e = launch_fused<T, 8, sizeof(T) == 8 ? 256 : 512>(a, st);
    else if constexpr (sizeof(T) == 4)
        e = launch_fused<T, 16, 256>(a, st);
    else
        e = cudaErrorInvalidValue;  // excluded by fused_max_layers
    if (e != cudaSuccess) return e;
    if (ev && (e = cudaEventRecord(ev[2], st)) != cudaSuccess) return e;
    k_rows_inverse<T><<<grid_rows, 256, smem_rows, st>>>((const C *)a.spec, H, a.nx, a.ny, a.log2Px,
                                                         npair, (const C *)a.twx, a.log2twx,
                                                         (T)(-a.Ms));
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (ev && (e = cudaEventRecord(ev[3], st)) != cudaSuccess) return e;
    return cudaSuccess;
}

cudaError_t launch_apply(const ApplyArgs &a, const void *m, void *H, bool fp64, cudaStream_t st,
                         cudaEvent_t *events) {
    if (fp64) return apply_impl<double>(a, (const double *)m, (double *)H, st, events);
    return apply_impl<float>(a, (const float *)m, (float *)H, st, events);
}

}  // namespace demag
