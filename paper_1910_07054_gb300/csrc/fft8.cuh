// Register-resident radix-8 Stockham FFT for 512-point transforms.
//
// One transform of N = 512 = 8^3 points is carried out by a group of 64
// threads, one radix-8 butterfly per thread per pass, three passes
// (sub-transform lengths Ns = 1, 8, 64).  Pass with length Ns, butterfly j
// (0 <= j < 64), k = j mod Ns:
//   v[r] = x[j + 64 r]                  r = 0..7
//   v[r] *= W_{8 Ns}^{r k}              (W_M = exp(-+2 pi i / M))
//   v = DFT_8(v)
//   y[(j - k) 8 + k + Ns r] = v[r]
// which leaves the result in natural order (self-sorting, no bit reversal).
// The caller moves data between passes (registers <-> shared memory) and
// synchronises the group; the first pass may read global memory and the last
// may write it directly.
#pragma once
#include "fft.cuh"

namespace demag {

// exp(-+2 pi i m / 512) from the N/2-entry table of W_512^m (m < 256):
// W^(m + 256) = -W^m.
template <bool INV, typename C>
__device__ __forceinline__ C tw512(const C *__restrict__ tw, int m) {
    m &= 511;
    C w = tw[m & 255];
    if (m & 256) {
        w.x = -w.x;
        w.y = -w.y;
    }
    if (INV) w.y = -w.y;
    return w;
}

// In-place 8-point DFT (forward: exp(-2 pi i n k / 8); INV: +).
template <bool INV, typename C>
__device__ __forceinline__ void dft8(C (&v)[8]) {
    using T = decltype(v[0].x);
    const T h = (T)0.70710678118654752440;
    C a[4], b[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        a[r] = c_add(v[r], v[r + 4]);
        b[r] = c_sub(v[r], v[r + 4]);
    }
    // b[r] *= W_8^r
    {
        const C t1 = b[1];
        b[1] = INV ? C{h * (t1.x - t1.y), h * (t1.x + t1.y)} : C{h * (t1.x + t1.y), h * (t1.y - t1.x)};
        b[2] = c_quarter<INV>(b[2]);
        const C t3 = b[3];
        b[3] = INV ? C{-h * (t3.x + t3.y), h * (t3.x - t3.y)} : C{h * (t3.y - t3.x), -h * (t3.x + t3.y)};
    }
    // two 4-point DFTs: even outputs from a, odd outputs from b
    const C t0 = c_add(a[0], a[2]), t1 = c_sub(a[0], a[2]);
    const C t2 = c_add(a[1], a[3]), t3 = c_quarter<INV>(c_sub(a[1], a[3]));
    const C u0 = c_add(b[0], b[2]), u1 = c_sub(b[0], b[2]);
    const C u2 = c_add(b[1], b[3]), u3 = c_quarter<INV>(c_sub(b[1], b[3]));
    v[0] = c_add(t0, t2);
    v[4] = c_sub(t0, t2);
    v[2] = c_add(t1, t3);
    v[6] = c_sub(t1, t3);
    v[1] = c_add(u0, u2);
    v[5] = c_sub(u0, u2);
    v[3] = c_add(u1, u3);
    v[7] = c_sub(u1, u3);
}

// Twiddles of pass Ns for butterfly position k: v[r] *= W_{8 Ns}^{r k}
// = W_512^{r k 64 / Ns}.
template <bool INV, typename C>
__device__ __forceinline__ void twiddle8(C (&v)[8], const C *__restrict__ tw, int k, int Ns) {
    if (k == 0) return;
    const int step = k * (64 / Ns);
#pragma unroll
    for (int r = 1; r < 8; ++r) v[r] = c_mul(v[r], tw512<INV>(tw, r * step));
}

// Destination of output r of butterfly j in pass Ns.
__device__ __forceinline__ int dest8(int j, int Ns, int r) {
    const int k = j & (Ns - 1);
    return (j - k) * 8 + k + Ns * r;
}

}  // namespace demag
