// Two 512-point radix-8 transforms per zero-padded 1024-point sequence.
//
// A length-1024 sequence whose upper half is zero (a row or column of Eq.
// FFT_v2 zero-padded from n <= 512) has the transform
//   X[2k]     = DFT_512(x)[k]
//   X[2k + 1] = DFT_512(x[n] W_1024^n)[k]                  (W_M = exp(-2 pi i / M))
// and the inverse of a full spectrum Y, needed at n < 512 only (the crop), is
//   y[n] = IDFT_512(Y_even)[n] + W_1024^-n IDFT_512(Y_odd)[n]
// (no 1/N scaling).  Each 512-point transform is the register-resident radix-8
// Stockham of fft8.cuh: 64 threads, three passes through shared memory.  One
// group of 64 threads carries both transforms of one sequence (same positions,
// same twiddles), so one thread holds X[2k] and X[2k + 1], or both halves of
// y[n].  Used by the column (cols1024.cu) and row (rows1024.cu) kernels.
#pragma once
#include "fft8.cuh"

namespace demag {
namespace f1024 {


constexpr int kF10Planes = 8;                 // sequences per block (plane columns or row pairs)
constexpr int kF10Threads = 64 * kF10Planes;  // one 64-thread group per sequence
// A padded 512-point column has two layouts.  The exchange layout (the data
// before pass 1 and after pass 2, and in the transposed phases) holds index p
// at f10_pad(p) = p + p / 16 + 4 (p / 64) (571 slots); the pass-1 outputs use
// p + p / 16 (f10_padA).  The extra 4 slots per run of 64 make the pass-2
// stores (two groups of 8 lanes 64 indices apart in a half-warp) take the
// minimum two wavefronts, which p + p / 16 alone does not for both the pass-1
// and pass-2 stores.  The plane's second column starts 574 slots in and planes
// are 1150 slots apart (28 words mod 32), so that a warp of the transposed
// phases that move planes in pairs (8 consecutive frequencies x 4 plane pairs)
// also takes two wavefronts per access.  The transforms themselves stay within
// one plane.
constexpr int kF10Col = 574;
constexpr int kF10Plane = 2 * kF10Col + 2;
// Twiddle tables in shared memory: W_1024^k (k < 512), then W_64^m (m < 64),
// then W_512^j (j < 64) for conflict-free pass-2 and pass-3 lookups.
constexpr int kF10Tw = 512 + 64 + 64;
constexpr size_t kF10Smem = (size_t)kF10Planes * kF10Plane * sizeof(float2) + kF10Tw * sizeof(float2);

__device__ __forceinline__ int f10_pad(int p) { return p + (p >> 4) + 4 * (p >> 6); }
__device__ __forceinline__ int f10_padA(int p) { return p + (p >> 4); }
// Slot of W_64^m in its table when it is permuted (PERM): m with its low three
// bits flipped when bits 4 and 5 of m differ (an involution), so that the
// pass-2 lookups W_64^{r k mod 64}, k = j mod 8, of every r = 1..7 fall in
// distinct banks (in plain order r = 4 is 2-way).  The permutation costs a few
// integer instructions per lookup, which only the inverse column transform
// gains back (measured).
__device__ __forceinline__ int f10_w64_slot(int m) { return m ^ (7 * (((m >> 4) ^ (m >> 5)) & 1)); }

__device__ __forceinline__ void f10_sync(int group) {
    asm volatile("bar.sync %0, %1;" ::"r"(group + 1), "r"(64) : "memory");
}

// W_1024^m (m any integer) from the shared table of W_1024^k, k < 512.
template <bool INV>
__device__ __forceinline__ float2 f10_w(const float2 *tw, int m) {
    m &= 1023;
    float2 w = tw[m & 511];
    if (m & 512) {
        w.x = -w.x;
        w.y = -w.y;
    }
    if (INV) w.y = -w.y;
    return w;
}

// Access pattern bases of a thread j (positions of the three Stockham passes
// in the padded column; see fft8.cuh for the passes):
//   positions j + 64 r, pass-1 layout   -> bj + 68 r
//   positions j + 64 r, exchange layout -> bx(r) = bj + 72 r
//   pass-1 outputs 8 j + r (pass-1 layout)        -> b1 + r
//   pass-2 outputs 64 (j / 8) + j mod 8 + 8 r (exchange layout) -> b2 + 8 r + r / 2
struct F10Bases {
    int bj, b1, b2;
    __device__ explicit F10Bases(int j) : bj(j + (j >> 4)), b1(8 * j + (j >> 1)), b2(72 * (j >> 3) + (j & 7)) {}
    __device__ __forceinline__ int bx(int r) const { return bj + 72 * r; }
};

// Passes 1..3 of both 512-point transforms of a plane; v[0] and v[1] hold the
// pass-1 inputs (positions j + 64 r) on entry and the outputs (positions
// j + 64 r) on return.  a, b: the plane's two padded columns.
template <bool INV, bool PERM = false>
__device__ __forceinline__ void f10_transform(float2 (&v)[2][8], float2 *a, float2 *b, const F10Bases &bs, int j,
                                              int group, const float2 *tw) {
    float2 *col[2] = {a, b};
    // pass 1 (Ns = 1): no twiddles; outputs to 8 j + r
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        dft8<INV>(v[t]);
#pragma unroll
        for (int r = 0; r < 8; ++r) col[t][bs.b1 + r] = v[t][r];
    }
    f10_sync(group);
    // pass 2 (Ns = 8): twiddles W_64^{r k}, k = j mod 8
#pragma unroll
    for (int t = 0; t < 2; ++t)
#pragma unroll
        for (int r = 0; r < 8; ++r) v[t][r] = col[t][bs.bj + 68 * r];
    f10_sync(group);
    {
        // W_64^{rk} from the 64-entry table
        const int k = j & 7;
#pragma unroll
        for (int r = 1; r < 8; ++r) {
            float2 w = tw[512 + (PERM ? f10_w64_slot((r * k) & 63) : ((r * k) & 63))];
            if (INV) w.y = -w.y;
            v[0][r] = c_mul(v[0][r], w);
            v[1][r] = c_mul(v[1][r], w);
        }
    }
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        dft8<INV>(v[t]);
#pragma unroll
        for (int r = 0; r < 8; ++r) col[t][bs.b2 + 8 * r + (r >> 1)] = v[t][r];
    }
    f10_sync(group);
    // pass 3 (Ns = 64): twiddles W_512^{r j}; outputs to positions j + 64 r
#pragma unroll
    for (int t = 0; t < 2; ++t)
#pragma unroll
        for (int r = 0; r < 8; ++r) v[t][r] = col[t][bs.bx(r)];
    {
        // W_512^{rj}: one lookup of W_512^j (consecutive j, no conflict), the
        // other powers by products (within a few ulp of the table values)
        float2 w[8];
        w[1] = tw[576 + j];
        if (INV) w[1].y = -w[1].y;
        w[2] = c_mul(w[1], w[1]);
        w[3] = c_mul(w[2], w[1]);
        w[4] = c_mul(w[2], w[2]);
        w[5] = c_mul(w[4], w[1]);
        w[6] = c_mul(w[4], w[2]);
        w[7] = c_mul(w[6], w[1]);
#pragma unroll
        for (int r = 1; r < 8; ++r) {
            v[0][r] = c_mul(v[0][r], w[r]);
            v[1][r] = c_mul(v[1][r], w[r]);
        }
    }
    dft8<INV>(v[0]);
    dft8<INV>(v[1]);
}

// The three tables from the plan's table tw of W_{2^(10 + sh)}^k, k below half
// its period (W_1024^(m + 512) = -W_1024^m).
template <bool PERM = false>
__device__ __forceinline__ void f10_load_table(float2 *tws, const float2 *__restrict__ tw, int sh) {
    for (int k = threadIdx.x; k < kF10Tw; k += blockDim.x) {
        // exponent of W_1024 (< 1024) held by slot k
        const int m = k < 512 ? k : (k < 576 ? 16 * (PERM ? f10_w64_slot(k - 512) : k - 512) : 2 * (k - 576));
        float2 w = tw[(m & 511) << sh];
        if (m & 512) {
            w.x = -w.x;
            w.y = -w.y;
        }
        tws[k] = w;
    }
}

}  // namespace f1024
}  // namespace demag
