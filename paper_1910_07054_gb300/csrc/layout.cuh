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

// The u-major tensor layout (dense-product plans) holds one (kx, u) entry of
// 6 component rows.  A component row holds the layer matrix prescaled by the
// target thickness, M(i, j) = (t_i / t_0) N(i <- j), in 8 x 8 blocks of layers
// (R, C), R <= C, block row by block row; within a block the left halves
// (columns 0-3) of the 8 rows come first, then the right halves, each half-row
// 16 bytes, in a swizzled order (ub_at).  Off-diagonal blocks hold pairs i < j; a diagonal block holds both
// triangles, the lower one as M(i, j) = s_c M(j, i) with s_c = -1 for xz and
// yz, +1 otherwise (reciprocity, t_i N(i <- j) = t_j P N(j <- i) P with P =
// diag(1, 1, -1)).  Layers past L are zero.  For i > j in different blocks
// M(i, j) is s_c times element (j, i) of block (C, R).
__host__ __device__ inline int ub_nb(int L) { return (L + 7) / 8; }
// Floats per component row (a multiple of 64, so rows and blocks start on
// 256-byte boundaries) and per (kx, u) entry.
__host__ __device__ inline int ub_row(int L) { return ub_nb(L) * (ub_nb(L) + 1) / 2 * 64; }
__host__ __device__ inline int ub_entry(int L) { return 6 * ub_row(L); }
// First float of block (R, C), R <= C, in a component row.
__host__ __device__ inline int ub_blk(int R, int C, int nb) { return (R * nb - R * (R - 1) / 2 + (C - R)) * 64; }
// Float of element (a, b) (row a, column b) within block (R, C): half h = b / 4
// of row a is the 16-byte slot a ^ (C mod 4) ^ 4 h of half-block h.  The
// tensor-core contraction reads a block two ways, and both meet 32 different
// banks: 8 lanes reading rows 0..7 of one block, one half-row each (16-byte
// loads), and 32 lanes reading one value of columns 0..7 of four consecutive
// blocks (C = 4k .. 4k + 3) of a block row.  The slot is bits 4-6 of the byte
// offset in a 256-byte block, so a reader XORs it into the address.
__host__ __device__ inline int ub_at(int a, int b, int C) {
    const int h = b >> 2;
    return 32 * h + 4 * (a ^ (C & 3) ^ (4 * h)) + (b & 3);
}

}  // namespace demag
