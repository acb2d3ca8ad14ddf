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
#include <algorithm>
#include <cstdint>

#include "fft8.cuh"
#include "internal.h"
#include "mbar.cuh"

namespace demag {

constexpr int kN8 = 512;
constexpr int kCol8 = kN8 + kN8 / 8;  // padded column length
constexpr int kGroup = 64;            // threads per transform

__device__ __forceinline__ int pad8i(int p) { return p + (p >> 3); }

__device__ __forceinline__ void group_sync(int group) {
    asm volatile("bar.sync %0, %1;" ::"r"(group + 1), "r"(kGroup) : "memory");
}

// Programmatic dependent launch: the kernels below are launched so that they
// may start while the previous kernel in the stream finishes.  Each waits for
// that kernel (and its memory) before reading anything it may have written,
// and lets its own successor be scheduled early.  Both are no-ops for a
// normal launch.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_release() { asm volatile("griddepcontrol.launch_dependents;" :::); }

// Launch with programmatic stream serialization (see pdl_wait).
template <typename... KArgs, typename... Args>
static cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
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

// Prefetch of [p, p + bytes) into L2 by bulk requests (p, bytes multiples of 16).
__device__ __forceinline__ void prefetch_l2_8(const void *p, size_t bytes) {
    const char *c = static_cast<const char *>(p);
    for (size_t off = 0; off < bytes; off += 65536) {
        const unsigned n = (unsigned)((bytes - off) < 65536 ? (bytes - off) : 65536);
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(c + off), "r"(n) : "memory");
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

// Same product as block_apply8, as one fused multiply-add chain per output.
template <typename C, typename T>
__device__ __forceinline__ void block_fma8(C &ox, C &oy, C &oz, T kxx, T kyy, T kzz, T kxy, T kxz, T kyz, C mx,
                                           C my, C mz) {
    ox.x = fma(kxx, mx.x, ox.x);
    ox.x = fma(kxy, my.x, ox.x);
    ox.x = fma(-kxz, mz.y, ox.x);
    ox.y = fma(kxx, mx.y, ox.y);
    ox.y = fma(kxy, my.y, ox.y);
    ox.y = fma(kxz, mz.x, ox.y);
    oy.x = fma(kxy, mx.x, oy.x);
    oy.x = fma(kyy, my.x, oy.x);
    oy.x = fma(-kyz, mz.y, oy.x);
    oy.y = fma(kxy, mx.y, oy.y);
    oy.y = fma(kyy, my.y, oy.y);
    oy.y = fma(kyz, mz.x, oy.y);
    oz.x = fma(-kxz, mx.y, oz.x);
    oz.x = fma(-kyz, my.y, oz.x);
    oz.x = fma(kzz, mz.x, oz.x);
    oz.y = fma(kxz, mx.x, oz.y);
    oz.y = fma(kyz, my.x, oz.y);
    oz.y = fma(kzz, mz.y, oz.y);
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

// ---------------------------------------------------------------------------
// Float columns for L <= 11 layers: the tensor streamed through shared memory.
//
// One block of 512 threads per (kx, state).  The 3L columns are transformed by
// eight 64-thread groups; in the contraction thread p owns the y-frequency
// position p (0 <= p < 512) in every column, so it reads and overwrites only
// its own entries and holds the field of all L target layers in registers.
// Each stored pair (i <= j) of the plan tensor then serves both directions,
// N(i<-j) m_j into layer i and, by reciprocity, (t_i / t_j) N'(j<-i) m_i into
// layer j (xz and yz change sign), so the tensor of one kx (6 reals per pair
// and folded frequency) is read exactly once.  It arrives in a ring of
// shared-memory stages, one pair per stage, by bulk copies that thread 0
// starts at block entry (overlapping the forward transforms) and re-arms as
// the stages drain.  Positions p > 256 take the stored entry q = 512 - p with
// xy and yz negated, done by negating m_y before and H_y after the sums.
//
// Columns have two layouts: the pass-1 outputs (stride-8 stores 8 j + r) at
// p + p / 16 (pad16), everything else (the transforms' inputs and the pass-2
// outputs, the contraction's positions) at p + p / 16 + 4 (p / 64) (padx16).
// The stride-1 accesses (j + 64 r), the pass-1 stores and the pass-2 stores
// (64 (j / 8) + j mod 8 + 8 r) then take the minimum two wavefronts for
// 8-byte elements, with constant offsets from per-thread bases.
// The pair loop runs over rows at run time and is unrolled only over the
// source layer, which keeps the code small enough for the instruction cache.
constexpr int kColR = 572;               // padded column length of the streamed kernel (padx16(511) = 570)
constexpr int kQyS8 = 260;               // stored frequencies per tensor row (257 padded to 16 B)
constexpr int kStage8 = 6 * kQyS8;       // floats per pair stage
constexpr int kRingBudget = 225 * 1024;  // dynamic shared memory of the streamed kernel

template <int L>
struct Ring8 {
    static constexpr int kCols = 3 * L;
    static constexpr int kColsPerGroup = (kCols + 7) / 8;
    static constexpr int kPairs = L * (L + 1) / 2;
    static constexpr int kFit = (kRingBudget - kCols * kColR * 8) / (kStage8 * 4);
    static constexpr int kStages = kPairs < kFit ? kPairs : kFit;  // pair slots of the ring
    static constexpr size_t kSmem = (size_t)kCols * kColR * 8 + (size_t)kStages * kStage8 * 4;
    // a row's pairs must all be resident at once (the row waits for all of them)
    static_assert(kStages >= L, "the ring must hold the longest pair row");
    // first stored pair of row i (pairs (i, j >= i), row by row)
    static __host__ __device__ constexpr int first(int i) { return i * L - (i * (i - 1)) / 2; }
};

__device__ __forceinline__ int pad16(int p) { return p + (p >> 4); }
// The exchange layout of the row kernels: p + p / 16 + 4 (p / 64).  Their data
// before pass 1 and after pass 2 (the untangling and placing steps) use it, the
// pass-1 outputs keep pad16; the 4 extra slots per run of 64 make the pass-2
// stores (two groups of 8 lanes 64 indices apart in a half-warp) take the
// minimum two wavefronts.
__device__ __forceinline__ int padx16(int p) { return p + (p >> 4) + 4 * (p >> 6); }

static __device__ unsigned g_wait_timeouts8;

// Twiddles of passes 2 (W_64^{r k}, k = j mod 8) and 3 (W_512^{r j}), r = 1..7.
template <bool INV, typename C>
__device__ __forceinline__ void load_twiddles8(C (&w2)[7], C (&w3)[7], const C *__restrict__ tw, int j) {
    const int k = j & 7;
#pragma unroll
    for (int r = 1; r < 8; ++r) {
        w2[r - 1] = tw512<INV>(tw, 8 * r * k);
        w3[r - 1] = tw512<INV>(tw, r * j);
    }
}

// Per-thread bases of the three access patterns (see the layout note above).
// XL (exchange layout, padx16) for the pass-2 stores and pass-3 accesses:
// j + 64 r -> bj + 72 r, pass-2 store -> b2x + 8 r + r / 2.
struct Bases8 {
    int b1;   // 8 j + r       -> b1 + r
    int bj;   // j + 64 r      -> bj + 68 r
    int b2;   // pass-2 store  -> b2 + 8 r + r / 2
    int b2x;  // the same in the exchange layout
    __device__ explicit Bases8(int j)
        : b1(8 * j + (j >> 1)), bj(j + (j >> 4)), b2(68 * (j >> 3) + (j & 7)), b2x(72 * (j >> 3) + (j & 7)) {}
};

// Pass 2 of the group's columns c = group + CSTEP u (column stride STRIDE),
// shared memory to shared memory.
template <bool INV, int CPG, int STRIDE, int CSTEP, typename C, bool XL = false>
__device__ __forceinline__ void ring8_pass2(C *cols, int group, int ncol, const Bases8 &bs, const C (&w2)[7],
                                            C (&v)[CPG][8]) {
#pragma unroll
    for (int u = 0; u < CPG; ++u) {
        const int c = group + CSTEP * u;
        if (c < ncol) {
            const C *col = cols + c * STRIDE + bs.bj;
#pragma unroll
            for (int r = 0; r < 8; ++r) v[u][r] = col[68 * r];
        }
    }
    group_sync(group);
#pragma unroll
    for (int u = 0; u < CPG; ++u) {
        const int c = group + CSTEP * u;
        if (c < ncol) {
#pragma unroll
            for (int r = 1; r < 8; ++r) v[u][r] = c_mul(v[u][r], w2[r - 1]);
            dft8<INV>(v[u]);
            C *col = cols + c * STRIDE + (XL ? bs.b2x : bs.b2);
#pragma unroll
            for (int r = 0; r < 8; ++r) col[8 * r + (r >> 1)] = v[u][r];
        }
    }
    group_sync(group);
}

// Pass 3 in place (positions j + 64 r), result left in v.
template <bool INV, int CPG, int STRIDE, int CSTEP, typename C, bool XL = false>
__device__ __forceinline__ void ring8_pass3(C *cols, int group, int ncol, const Bases8 &bs, const C (&w3)[7],
                                            C (&v)[CPG][8], bool store) {
#pragma unroll
    for (int u = 0; u < CPG; ++u) {
        const int c = group + CSTEP * u;
        if (c < ncol) {
            constexpr int kRun = XL ? 72 : 68;  // slots per run of 64 positions
            C *col = cols + c * STRIDE + bs.bj;
#pragma unroll
            for (int r = 0; r < 8; ++r) v[u][r] = col[kRun * r];
#pragma unroll
            for (int r = 1; r < 8; ++r) v[u][r] = c_mul(v[u][r], w3[r - 1]);
            dft8<INV>(v[u]);
            if (store) {
#pragma unroll
                for (int r = 0; r < 8; ++r) col[kRun * r] = v[u][r];
            }
        }
    }
}

// Thread 0: bulk copies of pairs [P, P_end) into their ring slots (pair P in
// slot P mod NS), each completing on its row's barrier.  A row announces its
// full byte count with its first pair, so its barrier completes only when all
// of its pairs have landed, whichever copies brought them.  Runs of pairs of
// one row with consecutive slots go in one copy.
template <int L>
__device__ __forceinline__ void ring8_issue(int P, int P_end, float *ring, const float *tk, uint64_t *full_row) {
    using R = Ring8<L>;
    while (P < P_end) {
        int k = 0;
        while (R::first(k + 1) <= P) ++k;
        if (P == R::first(k))
            mbar_arrive_expect_tx(&full_row[k], (unsigned)((L - k) * kStage8 * sizeof(float)));
        const int s = P % R::kStages;
        int n = R::first(k + 1) - P;                  // rest of the row
        if (n > P_end - P) n = P_end - P;             // not past the free slots
        if (n > R::kStages - s) n = R::kStages - s;   // not past the last slot
        bulk_copy_g2s(ring + s * kStage8, tk + (size_t)P * kStage8, (unsigned)(n * kStage8 * sizeof(float)),
                      &full_row[k]);
        P += n;
    }
}

template <int L>
__global__ void __launch_bounds__(544, 1) k_columns_ring8(float2 *__restrict__ spec,
                                                        const float *__restrict__ tensor,
                                                        const float *__restrict__ ratio, int Kx, int ny,
                                                        const float2 *__restrict__ tw) {
    using C = float2;
    using T = float;
    using R = Ring8<L>;
    constexpr int NC = R::kCols, CPG = R::kColsPerGroup, NP = R::kPairs, NS = R::kStages;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *cols = reinterpret_cast<C *>(smem_raw);                                      // NC x kColR
    T *ring = reinterpret_cast<T *>(smem_raw + (size_t)NC * kColR * sizeof(C));  // NS x kStage8
    __shared__ __align__(8) uint64_t full_row[L], empty_row[L];
    __shared__ T s_ratio[L * L];
    __shared__ int s_abort;
    const int tid = threadIdx.x, group = tid >> 6, j = tid & 63, lane = tid & 31;
    const int kx = blockIdx.x;
    const T *tk = tensor + (size_t)kx * NP * kStage8;
    C *sp = spec + ((size_t)blockIdx.y * NC * Kx + kx) * ny;
    bool ok = true;  // false once one of this thread's waits gave up

    if (tid == 0) {
#pragma unroll
        for (int r = 0; r < L; ++r) {
            mbar_init(&full_row[r], 1);
            mbar_init(&empty_row[r], 16);
        }
        mbar_init_fence();
        s_abort = 0;
    }
    if (tid < L * L) s_ratio[tid] = ratio[tid];
    __syncthreads();
    // warp 16 only copies the tensor: a bulk copy can hold its issuing thread
    // until the copy engine takes it, which must not stall a compute warp
    const bool producer = tid >= 512;
    if (producer && lane == 0) ring8_issue<L>(0, NS, ring, tk, full_row);
    // the plan tensor and ratios above do not depend on the previous kernel;
    // the spectrum does
    pdl_wait();
    pdl_release();

    const Bases8 bs(j);
    C w2[7], w3[7];
    C v[CPG][8];
    if (!producer) {
        // forward transforms: pass 1 from global memory (all loads issued first)
        load_twiddles8<false>(w2, w3, tw, j);
#pragma unroll
        for (int u = 0; u < CPG; ++u) {
            const int c = group + 8 * u;
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int y = j + 64 * r;
                v[u][r] = (c < NC && y < ny) ? sp[(size_t)c * Kx * ny + y] : C{0, 0};
            }
#pragma unroll
            for (int r = 4; r < 8; ++r) v[u][r] = C{0, 0};
        }
#pragma unroll
        for (int u = 0; u < CPG; ++u) {
            const int c = group + 8 * u;
            if (c < NC) {
                dft8<false>(v[u]);
                C *col = cols + c * kColR + bs.b1;
#pragma unroll
                for (int r = 0; r < 8; ++r) col[r] = v[u][r];
            }
        }
        group_sync(group);
        ring8_pass2<false, CPG, kColR, 8, C, true>(cols, group, NC, bs, w2, v);
        ring8_pass3<false, CPG, kColR, 8, C, true>(cols, group, NC, bs, w3, v, true);
    }
    __syncthreads();

    // contraction at position p = tid: m of every layer and the field of every
    // target in registers; pair rows i in order, each behind its copy barrier
    if (producer) {
        if (lane == 0) {
#pragma unroll
            for (int i = 1; i < L; ++i) {
                if (R::first(i - 1) + NS >= NP) break;
                // row i - 1 released: its slots take the next pairs
                if (ok && !mbar_wait(&empty_row[i - 1], 0, &g_wait_timeouts8)) ok = false;
                const int hi = R::first(i) + NS < NP ? R::first(i) + NS : NP;
                ring8_issue<L>(R::first(i - 1) + NS, hi, ring, tk, full_row);
            }
        }
    } else {
        const int p = tid;
        const int q = p <= kN8 / 2 ? p : kN8 - p;
        const bool mir = p > kN8 / 2;
        C *mp = cols + padx16(p);
        if (mir) {
#pragma unroll
            for (int l = 0; l < L; ++l) {
                const C t = mp[(3 * l + 1) * kColR];
                mp[(3 * l + 1) * kColR] = C{-t.x, -t.y};
            }
        }
        // m of layers >= KR stays in registers (m_j serves rows 0..j, so the
        // upper layers are reused most); lower layers are read when used
        constexpr int KR = L / 2;
        C acc[L][3], m[L][3];
#pragma unroll
        for (int l = 0; l < L; ++l)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                acc[l][c] = C{0, 0};
                if (l >= KR) m[l][c] = mp[(3 * l + c) * kColR];
            }
        const T *rq = ring + q;
#pragma unroll
        for (int i = 0; i < L; ++i) {
            if (ok && !mbar_wait(&full_row[i], 0, &g_wait_timeouts8)) ok = false;
            // acc[i] so far holds the reciprocal terms with sources scaled by
            // tau_j = t_j / t_0; dividing by tau_i gives sum_j (t_j / t_i) N' m_j
            if (i > 0) {
                const T inv_tau = s_ratio[i * L];  // t_0 / t_i
#pragma unroll
                for (int c = 0; c < 3; ++c) acc[i][c] = C{inv_tau * acc[i][c].x, inv_tau * acc[i][c].y};
            }
            C mi[3];  // the row's reciprocal source, scaled by tau_i
#pragma unroll
            for (int jj = i; jj < L; ++jj) {
                const int P = R::first(i) + jj - i;
                const T *kp = rq + (P % NS) * kStage8;
                const T kxx = kp[0], kyy = kp[kQyS8], kzz = kp[2 * kQyS8];
                const T kxy = kp[3 * kQyS8], kxz = kp[4 * kQyS8], kyz = kp[5 * kQyS8];
                C mj[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) mj[c] = jj >= KR ? m[jj][c] : mp[(3 * jj + c) * kColR];
                block_fma8(acc[i][0], acc[i][1], acc[i][2], kxx, kyy, kzz, kxy, kxz, kyz, mj[0], mj[1], mj[2]);
                if (jj == i) {
                    // m_i is no longer a direct source: scale it for the reciprocal terms
                    const T tau = s_ratio[i];  // t_i / t_0
#pragma unroll
                    for (int c = 0; c < 3; ++c) mi[c] = C{tau * mj[c].x, tau * mj[c].y};
                } else {
                    block_fma8(acc[jj][0], acc[jj][1], acc[jj][2], kxx, kyy, kzz, kxy, -kxz, -kyz, mi[0], mi[1],
                               mi[2]);
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty_row[i]);
            // target i is complete (its reciprocal terms came from rows < i)
            C *o = mp + 3 * i * kColR;
            o[0] = acc[i][0];
            o[kColR] = mir ? C{-acc[i][1].x, -acc[i][1].y} : acc[i][1];
            o[2 * kColR] = acc[i][2];
        }
    }
    if (!ok) s_abort = 1;
    __syncthreads();
    if (s_abort && tid == 512) {
        // a wait gave up: let the copies still in flight land (bounded) before exit
        for (int r = 0; r < L; ++r) mbar_wait(&full_row[r], 0, &g_wait_timeouts8);
    }
    if (producer) return;

    // inverse transforms: pass 1 in shared memory, pass 3 to global memory
    load_twiddles8<true>(w2, w3, tw, j);
#pragma unroll
    for (int u = 0; u < CPG; ++u) {
        const int c = group + 8 * u;
        if (c < NC) {
            const C *col = cols + c * kColR + bs.bj;
#pragma unroll
            for (int r = 0; r < 8; ++r) v[u][r] = col[72 * r];  // exchange layout
        }
    }
    group_sync(group);
#pragma unroll
    for (int u = 0; u < CPG; ++u) {
        const int c = group + 8 * u;
        if (c < NC) {
            dft8<true>(v[u]);
            C *col = cols + c * kColR + bs.b1;
#pragma unroll
            for (int r = 0; r < 8; ++r) col[r] = v[u][r];
        }
    }
    group_sync(group);
    ring8_pass2<true, CPG, kColR, 8, C, true>(cols, group, NC, bs, w2, v);
    ring8_pass3<true, CPG, kColR, 8, C, true>(cols, group, NC, bs, w3, v, false);
#pragma unroll
    for (int u = 0; u < CPG; ++u) {
        const int c = group + 8 * u;
        if (c < NC) {
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int y = j + 64 * r;
                if (y < ny) sp[(size_t)c * Kx * ny + y] = v[u][r];
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Row transforms for Px = 512: 16 rows of one plane per 256-thread block, the
// rows taken in pairs as one complex transform (z = row_a + i row_b), two
// pairs per 64-thread group.  The data enter pass 1 and leave pass 2 in the
// exchange layout (padx16; pass-1 outputs in pad16); the column stride of 574
// slots (padx16(511) = 570) makes the untangling step, where a warp reads 8
// columns at 4 frequencies, take at most 3 wavefronts per access.  Rows a and
// b of a pair are adjacent in the spectrum ([kx][y]), so both are moved with
// one 16-byte access (ny even).
constexpr int kColRow = 574;

// Two consecutive complex values as one 16-byte access (16-byte aligned).
__device__ __forceinline__ void store_pair(float2 *o, float2 a, float2 b) {
    *reinterpret_cast<float4 *>(o) = make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ void store_pair(double2 *o, double2 a, double2 b) {
    o[0] = a;
    o[1] = b;
}
__device__ __forceinline__ void load_pair(const float2 *p, float2 &a, float2 &b) {
    const float4 v = *reinterpret_cast<const float4 *>(p);
    a = make_float2(v.x, v.y);
    b = make_float2(v.z, v.w);
}
__device__ __forceinline__ void load_pair(const double2 *p, double2 &a, double2 &b) {
    a = p[0];
    b = p[1];
}

template <typename T>
__global__ void __launch_bounds__(256) k_rows_forward8(const T *__restrict__ m,
                                                      typename cpx_of<T>::type *__restrict__ spec,
                                                      int nx, int ny,
                                                      const typename cpx_of<T>::type *__restrict__ tw,
                                                      const T *__restrict__ layer_scale, int L) {
    using C = typename cpx_of<T>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C *buf = reinterpret_cast<C *>(smem_raw);  // 8 row pairs x kColRow
    constexpr int Kx = kN8 / 2 + 1;
    const int plane = blockIdx.y, y0 = blockIdx.x * 16;
    const int group = threadIdx.x >> 6, j = threadIdx.x & 63;
    const T *mp = m + (size_t)plane * ny * nx;
    pdl_wait();
    pdl_release();
    const T sc = layer_scale ? layer_scale[(plane / 3) % L] : (T)1;
    const Bases8 bs(j);
    // pass 1 straight from global memory (x = j + 64 r; zero for x >= nx and r >= 4)
    C v[2][8];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int q = group + 4 * h, ya = y0 + 2 * q, yb = ya + 1;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int x = j + 64 * r;
            T a = 0, b = 0;
            if (x < nx) {
                if (ya < ny) a = mp[(size_t)ya * nx + x];
                if (yb < ny) b = mp[(size_t)yb * nx + x];
            }
            v[h][r] = C{sc * a, sc * b};
        }
#pragma unroll
        for (int r = 4; r < 8; ++r) v[h][r] = C{0, 0};
    }
    C w2[7], w3[7];
    load_twiddles8<false>(w2, w3, tw, j);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        dft8<false>(v[h]);
        C *col = buf + (group + 4 * h) * kColRow + bs.b1;
#pragma unroll
        for (int r = 0; r < 8; ++r) col[r] = v[h][r];
    }
    group_sync(group);
    ring8_pass2<false, 2, kColRow, 4, C, true>(buf, group, 8, bs, w2, v);
    ring8_pass3<false, 2, kColRow, 4, C, true>(buf, group, 8, bs, w3, v, true);
    __syncthreads();
    // A[k] = (Z[k] + conj Z[-k]) / 2,  B[k] = (Z[k] - conj Z[-k]) / (2i): one
    // item per (kx, pair), rows a and b written together
    C *sp = spec + (size_t)plane * Kx * ny;
    const bool pairs16 = (ny & 1) == 0;
    for (int e = threadIdx.x; e < Kx * 8; e += 256) {
        const int kx = e >> 3, q = e & 7;
        const int ya = y0 + 2 * q;
        if (ya >= ny) continue;
        const C *zb = buf + q * kColRow;
        const C z1 = zb[padx16(kx)], z2 = zb[padx16((kN8 - kx) & (kN8 - 1))];
        const C a = C{(T)0.5 * (z1.x + z2.x), (T)0.5 * (z1.y - z2.y)};
        const C b = C{(T)0.5 * (z1.y + z2.y), (T)0.5 * (z2.x - z1.x)};
        C *o = sp + (size_t)kx * ny + ya;
        if (pairs16 && ya + 1 < ny) {
            store_pair(o, a, b);
        } else {
            o[0] = a;
            if (ya + 1 < ny) o[1] = b;
        }
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
    C *buf = reinterpret_cast<C *>(smem_raw);  // 8 row pairs x kColRow
    constexpr int half = kN8 / 2, Kx = half + 1;
    const int plane = blockIdx.y, y0 = blockIdx.x * 16;
    const int group = threadIdx.x >> 6, j = threadIdx.x & 63;
    const C *sp = spec + (size_t)plane * Kx * ny;
    pdl_wait();
    pdl_release();
    const T scale = out_scale * (layer_scale ? layer_scale[(plane / 3) % L] : (T)1);
    // thread (kx, q) reads rows a and b of pair q at kx (adjacent, one 16-byte
    // load) and writes Z[kx] = A + i B and Z[512 - kx] = conj(A) + i conj(B)
    // of the pair's column; DC and Nyquist are real in A and B
    const bool pairs16 = (ny & 1) == 0;
    constexpr int NIT = half * 8 / 256;  // items per thread for kx < 256
    const int qp = threadIdx.x & 7, ya = y0 + 2 * qp;
    C av[NIT], bv[NIT];
#pragma unroll
    for (int it = 0; it < NIT; ++it) {
        const int kx = (threadIdx.x >> 3) + 32 * it;
        const C *p = sp + (size_t)kx * ny + ya;
        av[it] = C{0, 0};
        bv[it] = C{0, 0};
        if (ya + 1 < ny && pairs16) {
            load_pair(p, av[it], bv[it]);
        } else if (ya < ny) {
            av[it] = p[0];
            if (ya + 1 < ny) bv[it] = p[1];
        }
    }
    C *zb = buf + qp * kColRow;
#pragma unroll
    for (int it = 0; it < NIT; ++it) {
        const int kx = (threadIdx.x >> 3) + 32 * it;
        C A = av[it], B = bv[it];
        if (kx == 0) {
            A.y = 0;
            B.y = 0;
            zb[padx16(0)] = C{A.x, B.x};
        } else {
            zb[padx16(kx)] = C{A.x - B.y, A.y + B.x};
            zb[padx16(kN8 - kx)] = C{A.x + B.y, B.x - A.y};
        }
    }
    if (threadIdx.x < 8) {
        const C *p = sp + (size_t)half * ny + ya;
        C A = C{0, 0}, B = C{0, 0};
        if (ya < ny) A = p[0];
        if (ya + 1 < ny) B = p[1];
        zb[padx16(half)] = C{A.x, B.x};  // A, B real at Nyquist
    }
    __syncthreads();
    // inverse transforms: pass 1 in shared memory, pass 3 straight to global
    const Bases8 bs(j);
    C w2[7], w3[7];
    load_twiddles8<true>(w2, w3, tw, j);
    C v[2][8];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const C *col = buf + (group + 4 * h) * kColRow + bs.bj;
#pragma unroll
        for (int q = 0; q < 8; ++q) v[h][q] = col[72 * q];  // exchange layout
    }
    group_sync(group);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        dft8<true>(v[h]);
        C *col = buf + (group + 4 * h) * kColRow + bs.b1;
#pragma unroll
        for (int q = 0; q < 8; ++q) col[q] = v[h][q];
    }
    group_sync(group);
    ring8_pass2<true, 2, kColRow, 4, C, true>(buf, group, 8, bs, w2, v);
    ring8_pass3<true, 2, kColRow, 4, C, true>(buf, group, 8, bs, w3, v, false);
    T *hp = H + (size_t)plane * ny * nx;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int q = group + 4 * h, ya = y0 + 2 * q, yb = ya + 1;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int x = j + 64 * k;
            if (x >= nx) continue;
            if (ya < ny) hp[(size_t)ya * nx + x] = scale * v[h][k].x;
            if (yb < ny) hp[(size_t)yb * nx + x] = scale * v[h][k].y;
        }
    }
}

template <int L>
static cudaError_t launch_ring8(const ApplyArgs &a, cudaStream_t st) {
    const size_t smem = Ring8<L>::kSmem;
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_columns_ring8<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
        cudaSuccess)
        return e;
    const int Kx = (1 << a.log2Px) / 2 + 1;
    return launch_pdl(k_columns_ring8<L>, dim3(Kx, a.B), dim3(544), smem, st, (float2 *)a.spec,
                      (const float *)a.tensor, (const float *)a.ratio, Kx, a.ny, (const float2 *)a.twy);
}

// The streamed kernel takes float plans with L <= 11 (its ring holds a full
// pair row), the pair-symmetric tensor with 260 stored frequencies per row and
// a 16-byte aligned tensor.
static bool ring8_supported(const ApplyArgs &a, bool fp64) {
    if (fp64 || a.full_pairs || a.L < 1 || a.L > 11 || a.QyS != kQyS8 || a.log2Py != 9) return false;
    return (reinterpret_cast<uintptr_t>(a.tensor) & 15) == 0;
}

static cudaError_t launch_ring8_any(const ApplyArgs &a, cudaStream_t st) {
    switch (a.L) {
    case 1: return launch_ring8<1>(a, st);
    case 2: return launch_ring8<2>(a, st);
    case 3: return launch_ring8<3>(a, st);
    case 4: return launch_ring8<4>(a, st);
    case 5: return launch_ring8<5>(a, st);
    case 6: return launch_ring8<6>(a, st);
    case 7: return launch_ring8<7>(a, st);
    case 8: return launch_ring8<8>(a, st);
    case 9: return launch_ring8<9>(a, st);
    case 10: return launch_ring8<10>(a, st);
    default: return launch_ring8<11>(a, st);
    }
}

// One thread waits on a barrier that no arrival or copy can complete, so the
// bounded wait must give up after `limit` cycles and count one timeout.
__global__ void k_selftest_wait(long long limit) {
    __shared__ __align__(8) uint64_t bar;
    mbar_init(&bar, 1);
    mbar_init_fence();
    mbar_wait(&bar, 0, &g_wait_timeouts8, limit);
}

cudaError_t launch_selftest_wait(long long limit, cudaStream_t st) {
    k_selftest_wait<<<1, 1, 0, st>>>(limit);
    return cudaGetLastError();
}

cudaError_t read_wait_timeouts(unsigned *dst, cudaStream_t st) {
    return cudaMemcpyFromSymbolAsync(dst, g_wait_timeouts8, sizeof(unsigned), 0, cudaMemcpyDeviceToHost, st);
}

bool cols512_supported(int log2Py, int L, bool fp64) {
    const size_t elem = fp64 ? sizeof(double2) : sizeof(float2);
    return log2Py == 9 && (size_t)3 * L * kCol8 * elem <= 220 * 1024;
}

template <typename T>
cudaError_t launch_rows512(const ApplyArgs &a, const void *m, void *H, bool forward, cudaStream_t st) {
    using C = typename cpx_of<T>::type;
    const size_t smem = (size_t)8 * kColRow * sizeof(C);
    const dim3 grid((a.ny + 15) / 16, a.planes ? a.planes : a.B * a.L * 3);
    cudaError_t e;
    if (forward) {
        if ((e = cudaFuncSetAttribute(k_rows_forward8<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem)) != cudaSuccess)
            return e;
        if ((e = launch_pdl(k_rows_forward8<T>, grid, dim3(256), smem, st, (const T *)m, (C *)a.spec, a.nx,
                            a.ny, (const C *)a.twx, (const T *)a.in_scale, a.L)) != cudaSuccess)
            return e;
    } else {
        if ((e = cudaFuncSetAttribute(k_rows_inverse8<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem)) != cudaSuccess)
            return e;
        if ((e = launch_pdl(k_rows_inverse8<T>, grid, dim3(256), smem, st, (const C *)a.spec, (T *)H, a.nx,
                            a.ny, (const C *)a.twx, (T)(-a.Ms), (const T *)a.out_scale, a.L)) != cudaSuccess)
            return e;
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_cols512(const ApplyArgs &a, cudaStream_t st) {
    using C = typename cpx_of<T>::type;
    if (ring8_supported(a, sizeof(T) == 8)) return launch_ring8_any(a, st);
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
