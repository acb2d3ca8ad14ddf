// Storage order of the y-frequencies in the plan tensor and its row padding.
//
// After a decimation-in-frequency FFT of length Py = 2^n, position p of the
// shared-memory column holds frequency ky = bitrev_n(p).  The tensor is even or
// odd in ky, so one entry serves ky and Py - ky.  In bit-reversed positions the
// two partners of an "octave" block [2^m, 2^(m+1)) are p and 2^(m+1) - 1 - (p - 2^m):
// each block is its own mirror.  The stored index u enumerates one partner per
// pair, so that consecutive u map to consecutive positions:
//   u = 0           -> p1 = p2 = 0          (ky = 0)
//   u = 1           -> p1 = p2 = 1          (ky = Py/2)
//   u in [2^(m-1)+1, 2^m + 1), m = 1..n-1, r = u - 2^(m-1) - 1:
//                      p1 = 2^m + r,  p2 = 2^(m+1) - 1 - r
// giving Py/2 + 1 stored entries.  Entry u holds the tensor at
// kyq = min(ky1, Py - ky1), ky1 = bitrev_n(p1).
#pragma once
#include <cuda_runtime.h>

namespace demag {

__host__ __device__ inline int ilog2_floor(int v) {
    int l = 0;
    while ((2 << l) <= v) ++l;
    return l;
}

__host__ __device__ inline int bitrev_n(int v, int n) {
    int r = 0;
    for (int k = 0; k < n; ++k) r |= ((v >> k) & 1) << (n - 1 - k);
    return r;
}

__host__ __device__ inline void u_positions(int u, int n, int &p1, int &p2) {
    if (u < 2) {
        p1 = p2 = u;
        return;
    }
    const int m = ilog2_floor(u - 1) + 1;  // u - 1 in [2^(m-1), 2^m)
    const int r = u - (1 << (m - 1)) - 1;
    p1 = (1 << m) + r;
    p2 = (2 << m) - 1 - r;
}

// Folded y-frequency of stored entry u.
__host__ __device__ inline int u_kyq(int u, int n) {
    int p1, p2;
    u_positions(u, n, p1, p2);
    const int ky = bitrev_n(p1, n), Py = 1 << n;
    return ky <= Py - ky ? ky : Py - ky;
}

// Row length of the stored tensor: Py/2 + 1 entries padded so that every
// [kx][pair][component] row, and so every kx block, starts on 16 bytes.
__host__ __device__ inline int tensor_row(int log2Py, bool fp64) {
    const int Qy = (1 << log2Py) / 2 + 1;
    const int q = fp64 ? 2 : 4;
    return (Qy + q - 1) / q * q;
}

// The u-major tensor layout (dense-product plans) holds one (kx, u) block of
// 6 component rows, [component][pair]; each row is npairs padded to a multiple
// of 4, so rows and blocks start on 16-byte boundaries.
__host__ __device__ inline int umajor_row(int npairs) { return (npairs + 3) / 4 * 4; }
// Floats per (kx, u) block.
__host__ __device__ inline int umajor_block(int npairs) { return 6 * umajor_row(npairs); }

}  // namespace demag
