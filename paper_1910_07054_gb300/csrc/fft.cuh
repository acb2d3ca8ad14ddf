// Shared-memory radix-4/2 FFTs for the hybrid demagnetization kernels.
//
// Every routine transforms `ncols` independent columns of length n = 2^log2n
// that live in shared memory at buf + col * col_stride, cooperatively with all
// threads of the block, and ends with __syncthreads().  The caller must have
// synchronised after writing the input.
//
//   fft_dit<INV>: input in bit-reversed order, output in natural order.
//   fft_dif<INV>: input in natural order, output in bit-reversed order.
//
// INV = false computes X[k] = sum_x x[n] exp(-2 pi i k n / N); INV = true the
// same with +i (no 1/N scaling).  Two radix-2 stages are fused into one radix-4
// pass per shared-memory round trip; an odd log2n adds one radix-2 pass.
//
// Twiddles come from a table tw[k] = exp(-2 pi i k / Ntw), k < Ntw/2, with
// Ntw = 2^log2tw >= n, computed on the host in double precision.
#pragma once
#include <cuda_runtime.h>

template <typename T> struct cpx_of;
template <> struct cpx_of<float> { using type = float2; };
template <> struct cpx_of<double> { using type = double2; };

template <typename C> __device__ __forceinline__ C c_add(C a, C b) { return C{a.x + b.x, a.y + b.y}; }
template <typename C> __device__ __forceinline__ C c_sub(C a, C b) { return C{a.x - b.x, a.y - b.y}; }
template <typename C> __device__ __forceinline__ C c_mul(C a, C b) {
    return C{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
// multiply by -i (forward) or +i (inverse): the quarter-turn of a radix-4 butterfly
template <bool INV, typename C> __device__ __forceinline__ C c_quarter(C a) {
    return INV ? C{-a.y, a.x} : C{a.y, -a.x};
}
template <bool INV, typename C> __device__ __forceinline__ C twiddle(const C *__restrict__ tw, int k) {
    C w = tw[k];
    if (INV) w.y = -w.y;
    return w;
}

__device__ __forceinline__ int bit_reverse(int v, int log2n) {
    return (int)(__brev((unsigned)v) >> (32 - log2n));
}

// Position of element i of a column in shared memory: i itself, or with PAD > 0
// one slot of padding after every 2^PAD elements (spreads a bit-reversed
// scatter of 16-byte elements over the banks).
template <int PAD>
__device__ __forceinline__ int fft_pos(int i) {
    return PAD ? i + (i >> PAD) : i;
}

template <bool INV, typename C, int PAD = 0>
__device__ void fft_dit(C *buf, int log2n, int ncols, int col_stride, const C *__restrict__ tw,
                        int log2tw) {
    const int n = 1 << log2n;
    int s = 0;
    for (; s + 1 < log2n; s += 2) {
        // stages s and s+1: half-sizes h and 2h inside blocks of 4h
        const int h = 1 << s;
        const int lq = log2n - 2;  // log2 of butterflies per column
        const int total = ncols << lq;
        const int sh2 = log2tw - (s + 2);  // W_{4h}^j = tw[j << sh2]
        for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
            const int col = idx >> lq;
            const int bf = idx & ((1 << lq) - 1);
            const int j = bf & (h - 1);
            const int g = (bf >> s) << (s + 2);
            C *p = buf + col * col_stride;
            const int i0 = fft_pos<PAD>(g + j), i1 = fft_pos<PAD>(g + j + h), i2 = fft_pos<PAD>(g + j + 2 * h),
                      i3 = fft_pos<PAD>(g + j + 3 * h);
            C x0 = p[i0], x1 = p[i1], x2 = p[i2], x3 = p[i3];
            const C w1 = twiddle<INV>(tw, j << (sh2 + 1));  // W_{2h}^j
            const C w2 = twiddle<INV>(tw, j << sh2);        // W_{4h}^j
            C t1 = c_mul(w1, x1), t3 = c_mul(w1, x3);
            C a0 = c_add(x0, t1), a1 = c_sub(x0, t1);
            C a2 = c_add(x2, t3), a3 = c_sub(x2, t3);
            C u2 = c_mul(w2, a2);
            C u3 = c_quarter<INV>(c_mul(w2, a3));  // W_{4h}^{j+h} = W_{4h}^j * W_4
            p[i0] = c_add(a0, u2);
            p[i2] = c_sub(a0, u2);
            p[i1] = c_add(a1, u3);
            p[i3] = c_sub(a1, u3);
        }
        __syncthreads();
    }
    if (s < log2n) {  // last radix-2 stage, h = n/2
        const int h = 1 << s;
        const int total = ncols << s;
        const int sh = log2tw - (s + 1);
        for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
            const int col = idx >> s;
            const int j = idx & (h - 1);
            C *p = buf + col * col_stride;
            const int i0 = fft_pos<PAD>(j), i1 = fft_pos<PAD>(j + h);
            C t = c_mul(twiddle<INV>(tw, j << sh), p[i1]);
            C a = p[i0];
            p[i0] = c_add(a, t);
            p[i1] = c_sub(a, t);
        }
        __syncthreads();
    }
    (void)n;
}

template <bool INV, typename C>
__device__ void fft_dif(C *buf, int log2n, int ncols, int col_stride, const C *__restrict__ tw,
                        int log2tw) {
    int s = log2n - 1;  // stage index = log2 of the half-size
    if (log2n & 1) {    // first a radix-2 stage at h = n/2
        const int h = 1 << s;
        const int total = ncols << s;
        const int sh = log2tw - (s + 1);
        for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
            const int col = idx >> s;
            const int j = idx & (h - 1);
            C *p = buf + col * col_stride + j;
            C a = p[0], b = p[h];
            p[0] = c_add(a, b);
            p[h] = c_mul(c_sub(a, b), twiddle<INV>(tw, j << sh));
        }
        __syncthreads();
        --s;
    }
    for (; s >= 1; s -= 2) {
        // stages with half-sizes 2h and h, h = 2^(s-1), inside blocks of 4h
        const int h = 1 << (s - 1);
        const int lq = log2n - 2;
        const int total = ncols << lq;
        const int sh2 = log2tw - (s + 1);  // W_{4h}^j = tw[j << sh2]
        for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
            const int col = idx >> lq;
            const int bf = idx & ((1 << lq) - 1);
            const int j = bf & (h - 1);
            const int g = (bf >> (s - 1)) << (s + 1);
            C *p = buf + col * col_stride + g + j;
            C x0 = p[0], x1 = p[h], x2 = p[2 * h], x3 = p[3 * h];
            const C w2 = twiddle<INV>(tw, j << sh2);        // W_{4h}^j
            const C w1 = twiddle<INV>(tw, j << (sh2 + 1));  // W_{2h}^j
            C a0 = c_add(x0, x2);
            C a2 = c_mul(c_sub(x0, x2), w2);
            C a1 = c_add(x1, x3);
            C a3 = c_quarter<INV>(c_mul(c_sub(x1, x3), w2));  // times W_{4h}^{j+h}
            p[0] = c_add(a0, a1);
            p[h] = c_mul(c_sub(a0, a1), w1);
            p[2 * h] = c_add(a2, a3);
            p[3 * h] = c_mul(c_sub(a2, a3), w1);
        }
        __syncthreads();
    }
}
