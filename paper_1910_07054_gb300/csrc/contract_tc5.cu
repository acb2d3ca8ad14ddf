// Layer contraction for batches of states on the fifth-generation tensor cores
// (tcgen05, accumulators in tensor memory), three split passes: TF32 operands
// (kind::tf32, K = 8 per MMA) or BF16 operands (kind::f16, K = 16 per MMA, half
// the MMAs for the same K; hi + lo carry 16 significant bits of each value).
//
// At one stored frequency entry (kx, u) the contraction of Eq. FFT_v2 for both
// of its y-frequencies (ky and Py - ky) and all B states is one real product
//     D (3L x 4B) = A (3L x 3L) * S (3L x 4B)
// with rows of A and D indexed by (output component c, target layer i), columns
// of A and rows of S by (source component c', source layer j), and the columns
// of S and D by (position q, real | imaginary, state b):
//   A = [[Kxx, Kxy, Kxz], [Kxy, Kyy, Kyz], [Kxz, Kyz, -Kzz]]   (L x L blocks)
//   S = [Mr_x; Mr_y; -Mi_z] in the real columns, [Mi_x; Mi_y; Mr_z] in the
//       imaginary ones,
// so that rows x and y of D are (Re H, Im H) and rows z are (Im H_z, -Re H_z).
// A is that of the stored frequency for both positions: at the mirrored one
// (where xy and yz change sign) m_y enters S negated and H_y leaves D negated.
// The kernel builds A with its rows prescaled by t_i / t_0, from the stored
// blocks of M(i, j) = (t_i / t_0) K(i <- j) (layout.cuh): a row of a block on
// or above the diagonal is 8 consecutive values, and below the diagonal M(i, j)
// = s_c M(j, i) is a column of the transposed block (s_c = -1 for xz and yz:
// reciprocity), so no value needs a per-element scale or selection; the
// epilogue multiplies row i of D by t_0 / t_i.  Products: a = a_hi + a_lo,
// s = s_hi + s_lo, D += a_lo s_hi + a_hi s_lo + a_hi s_hi in FP32.
//
// One persistent block per SM walks the entries.  A lives in tensor memory:
// each producer thread builds its own row of A (the thread's TMEM lane) for
// 8 columns of K and stores them with tcgen05.st, so A is never staged in
// shared memory; only S (N = 64 rows) passes through shared memory as the MMA's
// B operand.  Roles:
//   warp 21      loader: bulk copies of the entry's compact tensor and its two
//                state rows (one copy per state, to a bank-spreading stride)
//                into one of two input buffers, and L2 prefetch two entries
//                ahead;
//   warps 0-15   producers, chunk by chunk of K (16 TF32 or 32 BF16 columns),
//                2 stages: a warp of lane quarter q (warp mod 4) builds hi and
//                lo of the A rows in TMEM lanes 32 q + lane of one 128-row tile
//                t, its half h of the chunk's K columns, for one (t, h); warps
//                without such a block build S (hi and lo, K-major canonical
//                layout) in shared memory;
//   warp 20      MMA issue (one thread; M = 128 row tiles, N = 64) and the
//                tensor-memory allocation (512 columns: accumulators
//                double-buffered in 0..255, the A stages from 256);
//   warps 16-19  epilogue: accumulators to the state rows.
// Row r < 128 of A and D is lane r of tile 0; rows 128..3 Lp - 1 are the top
// lanes of tile 1 (lane r - 128 + lane0 of tile 1, lane0 a multiple of 32), so
// that the warps with two A blocks are in the upper lane quarters, away from
// the MMA warp's scheduler.  Lanes that hold no row hold whatever tensor memory
// held; they only feed accumulator rows that are never read.
#include <cuda_bf16.h>

#include <cstdint>

#include "internal.h"
#include "layout.cuh"
#include "tcgen05.cuh"

namespace demag {

namespace {

constexpr int kTcProd = 16;                          // producer warps
constexpr int kTcThreads = 32 * (kTcProd + 6);       // + 4 epilogue, MMA, loader warps
constexpr int kTcEpi = kTcProd, kTcMma = kTcProd + 4, kTcPre = kTcProd + 5;  // first warp of each role
constexpr int kTcN = 64;         // accumulator columns: 2 positions x (re, im) x 16 states
constexpr int kTcBp = 16;
// K columns per chunk (two MMA k-steps): 16 TF32 or 32 BF16 values, 64 bytes
// of each S row either way
template <bool BF> struct TcKC { static constexpr int value = BF ? 32 : 16; };
constexpr int kTcStages = 2;
constexpr int kTcCols = 512;     // tensor memory allocated
constexpr int kTcAcol = 256;     // first column of the A stages
constexpr int kTcAstage = 64;    // columns per A stage: 2 tiles x (16 hi + 16 lo)

__device__ unsigned g_tc_timeouts;

struct TcShape {
    int L, Lp, B, planes, R, T, nch, NB, seg;  // seg: padded float2 stride of one state's row segment
    size_t raw_bytes, rows_bytes, in_bytes, s_bytes, stage_bytes, off_stage, total;
};

__host__ __device__ inline size_t round256(size_t v) { return (v + 255) / 256 * 256; }

__host__ __device__ inline TcShape tc_shape(int L, int B, int npairs, int kc = 16) {
    TcShape s;
    s.L = L;
    s.Lp = (L + 7) / 8 * 8;
    s.B = B;
    s.planes = B * 3 * L;
    s.R = 3 * s.Lp;
    s.T = (s.R + 127) / 128;
    s.nch = (s.R + kc - 1) / kc;  // K = R padded to whole chunks (zero columns)
    s.NB = ub_entry(L);
    // a state's 3L complex values, padded so that consecutive states start 16
    // bytes apart modulo 128 (the 8 states a warp reads at once hit 8 bank groups)
    s.seg = 3 * L + ((2 - (3 * L) % 16) + 16) % 16;
    s.raw_bytes = round256((size_t)s.NB * 4 + 256);  // + a zero block for dropped blocks of compressed tensors
    s.rows_bytes = round256((size_t)2 * B * s.seg * 8);
    s.in_bytes = s.raw_bytes + s.rows_bytes;  // one input buffer (two of them): tensor blocks start on 256 bytes
    s.s_bytes = (size_t)kTcN * 64;  // N rows x 64 bytes of K
    s.stage_bytes = 2 * s.s_bytes;            // S hi, S lo
    s.off_stage = 2 * s.in_bytes;
    s.total = s.off_stage + kTcStages * s.stage_bytes;
    return s;
}

// (output component, source component) -> stored component (xx yy zz xy xz yz)
__device__ __forceinline__ int tc_comp(int co, int ci) {
    const int t = co * 3 + ci;
    return t == 0 ? 0 : t == 4 ? 1 : t == 8 ? 2 : (t == 1 || t == 3) ? 3 : (t == 2 || t == 6) ? 4 : 5;
}

// Round a finite float to TF32 (10 explicit mantissa bits), to nearest with
// ties away from zero: add half a unit of the last kept bit to the magnitude
// bits and clear the 13 dropped ones (a carry into the exponent is the correct
// result).  Two integer operations on the full-rate pipes.
__device__ __forceinline__ uint32_t tf32_round(uint32_t bits) { return (bits + 0x1000u) & 0xFFFFE000u; }

// v = hi + lo with hi the TF32 rounding of v and lo = v - hi exactly (|lo| <=
// 2^-11 |v|).  lo goes to the tensor core as it is: a TF32 operand is read from
// its upper 19 bits, so what reaches the product is lo truncated, within
// 2^-10 |lo| <= 2^-21 |v| of it.
__device__ __forceinline__ void split_tf32(float v, uint32_t &hi, uint32_t &lo) {
    hi = tf32_round(__float_as_uint(v));
    lo = __float_as_uint(v - __uint_as_float(hi));
}

// Split of one 32-bit operand word: TF32 takes one value per word, BF16 two
// (the lower K index in the low half).
template <bool BF> struct Split;
template <> struct Split<false> {
    static constexpr int kPerWord = 1;
    __device__ __forceinline__ static void word(const float *v, uint32_t &hi, uint32_t &lo) {
        split_tf32(v[0], hi, lo);
    }
};
template <> struct Split<true> {
    static constexpr int kPerWord = 2;
    // v = hi + lo + r with hi = bf16(v), lo = bf16(v - hi), both rounded to
    // nearest even (|r| <= 2^-18 |v|), two values at a time with the
    // hardware's paired conversion: six instructions for the pair
    __device__ __forceinline__ static void word(const float *v, uint32_t &hi, uint32_t &lo) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(v[0], v[1]);  // .x (low half) = v[0]
        const uint32_t hb = *reinterpret_cast<const uint32_t *>(&h);
        const __nv_bfloat162 l = __floats2bfloat162_rn(v[0] - __uint_as_float(hb << 16),
                                                       v[1] - __uint_as_float(hb & 0xFFFF0000u));
        hi = hb;
        lo = *reinterpret_cast<const uint32_t *>(&l);
    }
};

// One thread: the six MMAs of one 128-row tile and one chunk of K (two
// k-steps), A from tensor memory (hi in columns at..at+15, lo in at+16..at+31;
// each k-step's 8 columns hold 8 TF32 or 16 BF16 values), S hi and lo from
// shared memory (descriptors bh, bl; +16 in the start-address field is the
// second k-step, 256 bytes further):  D (+)= A_lo S_hi + A_hi S_lo + A_hi S_hi
// for k-steps 0 and 1.  `accumulate` false starts D over.
#define DEMAG_TC_MMA_CHUNK(KIND)                                                                         \
    asm volatile(                                                                                        \
        "{\n\t.reg .pred pa, pt;\n\t"                                                                    \
        "setp.ne.b32 pa, %9, 0;\n\t"                                                                     \
        "setp.eq.b32 pt, %9, %9;\n\t"                                                                    \
        "tcgen05.mma.cta_group::1.kind::" KIND " [%0], [%3], %5, %8, pa;\n\t"                            \
        "tcgen05.mma.cta_group::1.kind::" KIND " [%0], [%1], %6, %8, pt;\n\t"                            \
        "tcgen05.mma.cta_group::1.kind::" KIND " [%0], [%1], %5, %8, pt;\n\t"                            \
        "tcgen05.mma.cta_group::1.kind::" KIND " [%0], [%4], %7, %8, pt;\n\t"                            \
        "tcgen05.mma.cta_group::1.kind::" KIND " [%0], [%2], %10, %8, pt;\n\t"                           \
        "tcgen05.mma.cta_group::1.kind::" KIND " [%0], [%2], %7, %8, pt;\n\t}" ::"r"(dt),                \
        "r"(at), "r"(at + 8), "r"(at + 16), "r"(at + 24), "l"(bh), "l"(bl), "l"(bh + 16), "r"(idesc),   \
        "r"((unsigned)accumulate), "l"(bl + 16)                                                          \
        : "memory")

template <bool BF>
__device__ __forceinline__ void tc_mma_chunk(unsigned dt, unsigned at, uint64_t bh, uint64_t bl, uint32_t idesc,
                                             bool accumulate) {
    if (BF)
        DEMAG_TC_MMA_CHUNK("f16");
    else
        DEMAG_TC_MMA_CHUNK("tf32");
}
#undef DEMAG_TC_MMA_CHUNK

}  // namespace

// CMP: the plan's tensor is block-compressed (compress.cu): entry e holds its
// kept blocks only, bmask[e] tells which, bfirst[e] where they start.
// PK (with BF): the tensor holds each value as its BF16 split pair (hi in the
// upper half of the 32-bit slot, lo in the lower) and K_zz negated, so the
// producers only regroup halves into operand words and flip the signs of the
// reciprocal xz and yz blocks below the diagonal.
template <bool BF, bool CMP, bool PK>
__global__ void __launch_bounds__(kTcThreads, 1) k_contract_tc5(float2 *__restrict__ spec2,
                                                               const float *__restrict__ tensor_um,
                                                               const float *__restrict__ ratio, int L, int B,
                                                               int Kx, int log2Py, int npairs,
                                                               const unsigned long long *__restrict__ bmask,
                                                               const unsigned *__restrict__ bfirst) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t st_full[kTcStages], st_empty[kTcStages], d_full[2], d_empty[2];
    __shared__ __align__(8) uint64_t in_full[2], in_empty[2];  // the entry's tensor and state rows
    __shared__ unsigned tmem_slot;
    __shared__ __align__(16) float s_itau[64];
    __shared__ int s_bkept[2];       // compressed tensor: kept blocks of the entry in each input buffer
    __shared__ int s_boff[2][64];    // and the byte offset in a component row of block (I, J), -1 if dropped
    __shared__ int s_abort;
    constexpr int KC = TcKC<BF>::value;  // K columns per chunk
    constexpr int PW = Split<BF>::kPerWord;
    const TcShape sh = tc_shape(L, B, npairs, KC);
    const int Py = 1 << log2Py, Qy = Py / 2 + 1;
    const int nent = Kx * Qy;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int Lp = sh.Lp, planes = sh.planes, R = sh.R;
    const int lane0 = 128 - (R > 128 ? (R - 128 + 31) / 32 * 32 : 0);  // first TMEM lane of tile 1's rows
    bool ok = true;

    if (tid == 0) {
        for (int k = 0; k < kTcStages; ++k) {
            mbar_init(&st_full[k], kTcProd);
            mbar_init(&st_empty[k], 1);
        }
        for (int k = 0; k < 2; ++k) {
            mbar_init(&d_full[k], 1);
            mbar_init(&d_empty[k], 4);
            mbar_init(&in_full[k], 1);
            mbar_init(&in_empty[k], kTcProd);
        }
        mbar_init_fence();
        s_abort = 0;
    }
    if (tid < 64) s_itau[tid] = tid < L ? ratio[tid * L] : 0.f;  // t_0 / t_l
    if (CMP && tid < 128)  // the zero block at the end of each input buffer's tensor part
        reinterpret_cast<float *>(smem + (tid >> 6) * sh.in_bytes + sh.raw_bytes - 256)[tid & 63] = 0.f;
    if (warp == kTcMma) tc_alloc(&tmem_slot, kTcCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = tmem_slot;

    auto entry = [&](int lf, int &kx, int &u, int &p1, int &p2, int &npos, bool &mir0) {
        const int f = blockIdx.x + lf * gridDim.x;
        kx = f / Qy;
        u = f - kx * Qy;
        // positions of stored entry u (the order of u_positions, with bit intrinsics)
        if (u < 2) {
            p1 = p2 = u;
        } else {
            const int m = 32 - __clz(u - 1);  // u - 1 in [2^(m-1), 2^m)
            const int rr = u - (1 << (m - 1)) - 1;
            p1 = (1 << m) + rr;
            p2 = (2 << m) - 1 - rr;
        }
        npos = p2 != p1 ? 2 : 1;
        mir0 = (int)(__brev((unsigned)p1) >> (32 - log2Py)) > Py / 2;  // position 0 is the mirrored frequency
    };
    const int nlocal = blockIdx.x < nent ? (nent - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;

    if (warp == kTcPre) {
        // loader: entry lf into buffer lf mod 2 once the producers released
        // entry lf - 2 (lane 0 waits and announces the bytes; the per-state
        // copies are issued by all lanes, one each); L2 prefetch of entry lf + 2
        auto prefetch = [&](int lf) {
            if (lf >= nlocal) return;
            int kx, u, p1, p2, npos;
            bool mir0;
            entry(lf, kx, u, p1, p2, npos, mir0);
            if (CMP) {
                const size_t ent = (size_t)kx * Qy + u;
                const unsigned tb = 6u * 256u * (unsigned)__popcll(bmask[ent]);
                if (tb)
                    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(tensor_um + (size_t)bfirst[ent] * 64),
                                 "r"(tb) : "memory");
            } else {
                asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(tensor_um + ((size_t)kx * Qy + u) * sh.NB),
                             "r"((unsigned)sh.NB * 4) : "memory");
            }
            asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(spec2 + ((size_t)kx * Py + p1) * planes),
                         "r"((unsigned)planes * 8) : "memory");
            if (npos == 2)
                asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(
                                 spec2 + ((size_t)kx * Py + p2) * planes),
                             "r"((unsigned)planes * 8) : "memory");
        };
        if (lane == 0) {
            prefetch(0);
            prefetch(1);
        }
        const unsigned segb = (unsigned)(3 * L) * 8;  // one state's values (16-byte multiple)
        for (int lf = 0; lf < nlocal && ok; ++lf) {
            const int buf = lf & 1;
            if (lane == 0 && lf >= 2 && !mbar_wait(&in_empty[buf], ((lf >> 1) - 1) & 1, &g_tc_timeouts)) ok = false;
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) break;
            int kx, u, p1, p2, npos;
            bool mir0;
            entry(lf, kx, u, p1, p2, npos, mir0);
            unsigned char *in = smem + (size_t)buf * sh.in_bytes;
            unsigned tb = (unsigned)sh.NB * 4;
            const float *tsrc = tensor_um + ((size_t)kx * Qy + u) * sh.NB;
            if (CMP) {
                // the header (kept count, block offsets) is written by all lanes
                // before the arrival that publishes it
                const size_t ent = (size_t)kx * Qy + u;
                unsigned long long m = 0;
                unsigned f = 0;
                if (lane == 0) {
                    m = bmask[ent];
                    f = bfirst[ent];
                }
                m = __shfl_sync(0xffffffffu, m, 0);
                f = __shfl_sync(0xffffffffu, f, 0);
                const int nbk = ub_nb(L);
#pragma unroll
                for (int h2 = 0; h2 < 2; ++h2) {
                    const int idx = lane + 32 * h2, I = idx >> 3, J = idx & 7;
                    int bo = -1;
                    if (I < nbk && J < nbk) {
                        const int b = (I <= J ? ub_blk(I, J, nbk) : ub_blk(J, I, nbk)) >> 6;
                        if ((m >> b) & 1ull) bo = 256 * __popcll(m & ((1ull << b) - 1ull));
                    }
                    s_boff[buf][idx] = bo;
                }
                if (lane == 0) s_bkept[buf] = __popcll(m);
                tb = 6u * 256u * (unsigned)__popcll(m);
                tsrc = tensor_um + (size_t)f * 64;
                __syncwarp();
            }
            if (lane == 0) {
                mbar_arrive_expect_tx(&in_full[buf], tb + (unsigned)(npos * B) * segb);
                if (tb) bulk_copy_g2s(in, tsrc, tb, &in_full[buf]);
            }
            __syncwarp();
            for (int c = lane; c < npos * B; c += 32) {
                const int q = c >= B, b = c - q * B;
                const float2 *src = spec2 + ((size_t)kx * Py + (q ? p2 : p1)) * planes + (size_t)b * 3 * L;
                float2 *dst = reinterpret_cast<float2 *>(in + sh.raw_bytes) + ((size_t)q * B + b) * sh.seg;
                bulk_copy_g2s(dst, src, segb, &in_full[buf]);
            }
            if (lane == 0) prefetch(lf + 2);
        }
    } else if (warp < kTcProd) {
        // producers.  Warp (q = warp mod 4, wq = warp / 4): A block wq of lane
        // quarter q if that quarter has wq < nA(q) blocks (two K halves per
        // 128-row tile that has rows in the quarter), else S worker.
        const int q = warp & 3, wq = warp >> 2;
        auto nA = [&](int qq) {
            const bool t0 = 32 * qq < R;
            const bool t1 = 32 * qq + 32 > lane0 && 32 * qq < lane0 + (R - 128);
            return 2 * ((int)t0 + (int)t1);
        };
        const bool isA = wq < nA(q);
        int sidx = 0, nS = 0;
        for (int w = 0; w < kTcProd; ++w) {
            const bool s_w = (w >> 2) >= nA(w & 3);
            if (s_w && w < warp) ++sidx;
            nS += s_w;
        }
        const int nb = ub_nb(L), NR = ub_row(L);
        // All shared-memory operands below are byte offsets from smem (32-bit
        // shared-window addressing).
        // A block: row r of A (co, i), K columns 8 h .. 8 h + 7 of each chunk.
        // The row holds M(i, j) (the layer matrix prescaled by t_i / t_0; the
        // epilogue takes t_0 / t_i back out).  Lanes without a row (r >= 3 Lp)
        // read row 0 of component 0: finite values for accumulator rows that
        // are never read; rows L <= i < Lp read the zero padding.
        const int t = (wq >> 1) > 0 || 32 * q >= R, h = wq & 1;  // a quarter without tile-0 rows has tile 1 only
        const int r = t == 0 ? 32 * q + lane : 128 + 32 * q + lane - lane0;
        const int cor = r / Lp;
        const bool rin = isA && r < R;
        const int co = rin ? cor : 0, i = rin ? r - cor * Lp : 0;
        const int I = i >> 3, i8 = i & 7;  // the row's block row and its row in the block
        const unsigned ta_row = tmem + ((unsigned)(32 * q) << 16) + (unsigned)(kTcAcol + 32 * t + 8 * h);
        // per source component ci: byte offset of the stored component row, and
        // the sign of blocks on or above the diagonal (-1 for the -K_zz block of
        // A) and below it (there xz and yz also change sign: reciprocity)
        int offc[3], compc[3];
        float sup[3], slo[3];
#pragma unroll
        for (int ci = 0; ci < 3; ++ci) {
            const int comp = tc_comp(co, ci);
            const float zs = (!PK && co == 2 && ci == 2) ? -1.f : 1.f;  // a packed tensor holds -K_zz
            compc[ci] = comp;
            offc[ci] = comp * NR * 4;
            sup[ci] = zs;
            slo[ci] = comp >= 4 ? -zs : zs;
        }
        // S unit of this thread: (position pq, state b, core column k4)
        constexpr int KG = 4;  // core matrices (16 bytes of K) per S row and chunk
        // (lanes 8 g .. 8 g + 7 of a warp take states 0..7 or 8..15 of one core
        // column: a quarter-warp's 16-byte stores fill the 128 bytes of eight
        // core-matrix rows, one bank group each)
        const int sv = lane + 32 * sidx;
        const bool sact = !isA && sv < 2 * kTcBp * KG;
        const int k4 = (sv >> 3) & (KG - 1), sb = (sv & 7) | (((sv >> 5) & 1) << 3), spq = (sv >> 6) & 1;
        const int sn = 32 * spq + sb;  // real column of S; the imaginary one is sn + 16
        const int soff_r = (((sn >> 3) * KG + k4) * 32 + (sn & 7) * 4) * 4;
        const int soff_i = soff_r + 2 * KG * 32 * 4;  // 16 rows = two 8-row groups further
        const int srow = (int)sh.raw_bytes + (spq * B + sb) * sh.seg * 8;

        for (int lf = 0; lf < nlocal && ok; ++lf) {
            int kx, u, p1, p2, npos;
            bool mir0;
            entry(lf, kx, u, p1, p2, npos, mir0);
            const int buf = lf & 1;
            if (!mbar_wait(&in_full[buf], (lf >> 1) & 1, &g_tc_timeouts)) ok = false;
            const int inb = buf * (int)sh.in_bytes;  // this entry's input buffer
            if (CMP) {
                const int nk = s_bkept[buf];
#pragma unroll
                for (int ci = 0; ci < 3; ++ci) offc[ci] = compc[ci] * nk * 256;  // component rows of nk blocks
            }
            const bool slive = sact && spq < npos && sb < B;
            const float sy0 = ((spq == 0) == mir0) ? -1.f : 1.f;  // m_y negated at the mirrored position
            for (int ch = 0; ch < sh.nch && ok; ++ch) {
                const int gch = lf * sh.nch + ch, s = gch % kTcStages, use = gch / kTcStages;
                if (use >= 1 && !mbar_wait(&st_empty[s], (use - 1) & 1, &g_tc_timeouts)) ok = false;
                tc_fence_after();
                if (isA) {
                    // block h of the chunk: K columns KC/2 h .. KC/2 (h + 1) - 1,
                    // PW sub-blocks of 8 (each within one source component, as
                    // Lp is a multiple of 8)
                    uint32_t vb[8 * PW];  // the values' bits: floats, or BF16 split pairs (PK)
                    uint32_t nmask[PW];   // PK: sign bits to flip in the sub-block's words
#pragma unroll
                    for (int sbk = 0; sbk < PW; ++sbk) {
                        const int kc0 = ch * KC + 8 * PW * h + 8 * sbk;  // first K column of the sub-block
                        uint32_t *vs8 = vb + 8 * sbk;
                        nmask[sbk] = 0u;
                        if (kc0 < R) {
                            // the sub-block is layer block J of source component ci
                            const int ci = (kc0 >= Lp) + (kc0 >= 2 * Lp), J = (kc0 - ci * Lp) >> 3;
                            int off = inb + (ci == 0 ? offc[0] : (ci == 1 ? offc[1] : offc[2]));
                            float sg;
                            if (CMP) {
                                // the kept block's place, or the zero block that follows
                                // the raw buffer (a dropped block reads as zeros, without
                                // a branch of its own)
                                const int bo = s_boff[buf][8 * I + J];
                                off = bo >= 0 ? off + bo : inb + (int)sh.raw_bytes - 256;
                            }
                            if (I <= J) {
                                // row i8 of block (I, J): its two 16-byte halves, slot
                                // i8 ^ (J mod 4) of the first half-block and that slot
                                // ^ 4 of the second (layout.cuh; blocks start on 256
                                // bytes)
                                const unsigned a0 = (unsigned)(off + (CMP ? 0 : 4 * ub_blk(I, J, nb))) +
                                                    16u * (unsigned)(i8 ^ (J & 3));
                                const uint4 x0 = *reinterpret_cast<const uint4 *>(smem + a0);
                                const uint4 x1 = *reinterpret_cast<const uint4 *>(smem + (a0 ^ 0xC0u));
                                vs8[0] = x0.x, vs8[1] = x0.y, vs8[2] = x0.z, vs8[3] = x0.w;
                                vs8[4] = x1.x, vs8[5] = x1.y, vs8[6] = x1.z, vs8[7] = x1.w;
                                sg = ci == 0 ? sup[0] : (ci == 1 ? sup[1] : sup[2]);
                            } else {
                                // column i8 of block (J, I): M(i, 8 J + e) = s_c M(8 J + e, i).
                                // Row e's half holding it is slot e ^ (I mod 4) ^ 4 h of
                                // half-block h = i8 / 4 (layout.cuh): bits 4-6 of the byte
                                // offset, so one XOR per value
                                const int hh = i8 >> 2;
                                const unsigned a0 = ((unsigned)(off + (CMP ? 0 : 4 * ub_blk(J, I, nb)) + 128 * hh +
                                                                4 * (i8 & 3))) ^
                                                    (16u * (unsigned)((I & 3) ^ (4 * hh)));
#pragma unroll
                                for (int e = 0; e < 8; ++e)
                                    vs8[e] = *reinterpret_cast<const uint32_t *>(smem + (a0 ^ (16u * (unsigned)e)));
                                sg = ci == 0 ? slo[0] : (ci == 1 ? slo[1] : slo[2]);
                            }
                            if constexpr (PK) {
                                nmask[sbk] = sg < 0.f ? 0x80008000u : 0u;
                            } else {
#pragma unroll
                                for (int e = 0; e < 8; e += 2) {
                                    const float2 y = __fmul2_rn(
                                        make_float2(__uint_as_float(vs8[e]), __uint_as_float(vs8[e + 1])),
                                        make_float2(sg, sg));
                                    vs8[e] = __float_as_uint(y.x);
                                    vs8[e + 1] = __float_as_uint(y.y);
                                }
                            }
                        } else {
#pragma unroll
                            for (int e = 0; e < 8; ++e) vs8[e] = 0u;
                        }
                    }
                    uint32_t hi[8], lo[8];
                    if constexpr (PK) {
                        // the stored pairs (hi << 16 | lo) of two consecutive K
                        // columns give one hi word and one lo word (lower K index in
                        // the low half); a sign flips both halves of both
#pragma unroll
                        for (int w = 0; w < 8; ++w) {
                            const uint32_t m = nmask[w / 4];
                            hi[w] = __byte_perm(vb[2 * w], vb[2 * w + 1], 0x7632) ^ m;
                            lo[w] = __byte_perm(vb[2 * w], vb[2 * w + 1], 0x5410) ^ m;
                        }
                    } else {
                        float v[8 * PW];
#pragma unroll
                        for (int k = 0; k < 8 * PW; ++k) v[k] = __uint_as_float(vb[k]);
#pragma unroll
                        for (int w = 0; w < 8; ++w) Split<BF>::word(v + PW * w, hi[w], lo[w]);
                    }
                    const unsigned ta = ta_row + (unsigned)(s * kTcAstage);
                    tc_st8(ta, hi);
                    tc_st8(ta + 16, lo);
                    tc_wait_st();
                } else if (sact) {
                    // S unit: one (position, state) and 4 PW consecutive K columns
                    // (one source component, as Lp is a multiple of 8); the 4 PW
                    // complex values give 16 bytes of the core-matrix rows of both
                    // its columns of S: rows x, y take (Re, Im), rows z (-Im, Re)
                    constexpr int KU = 4 * PW;
                    const int kc = ch * KC + KU * k4;
                    float re[KU], im[KU];
#pragma unroll
                    for (int e = 0; e < KU; ++e) re[e] = im[e] = 0.f;
                    if (slive && kc < R) {
                        const int ci = (kc >= Lp) + (kc >= 2 * Lp), jb = kc - ci * Lp;
                        const bool z = ci == 2;
                        const float sre = z ? -1.f : (ci == 1 ? sy0 : 1.f);
                        const float sim = z ? 1.f : (ci == 1 ? sy0 : 1.f);
                        const int a = inb + srow + (jb * 3 + ci) * 8;
#pragma unroll
                        for (int e = 0; e < KU; ++e) {
                            if (jb + e < L) {
                                const float2 mv = *reinterpret_cast<const float2 *>(smem + a + 24 * e);
                                re[e] = sre * (z ? mv.y : mv.x);
                                im[e] = sim * (z ? mv.x : mv.y);
                            }
                        }
                    }
                    uint4 hr, lr, hm, lm;
                    Split<BF>::word(re + 0 * PW, hr.x, lr.x);
                    Split<BF>::word(re + 1 * PW, hr.y, lr.y);
                    Split<BF>::word(re + 2 * PW, hr.z, lr.z);
                    Split<BF>::word(re + 3 * PW, hr.w, lr.w);
                    Split<BF>::word(im + 0 * PW, hm.x, lm.x);
                    Split<BF>::word(im + 1 * PW, hm.y, lm.y);
                    Split<BF>::word(im + 2 * PW, hm.z, lm.z);
                    Split<BF>::word(im + 3 * PW, hm.w, lm.w);
                    unsigned char *st_hi = smem + sh.off_stage + s * sh.stage_bytes;
                    unsigned char *st_lo = st_hi + sh.s_bytes;
                    *reinterpret_cast<uint4 *>(st_hi + soff_r) = hr;
                    *reinterpret_cast<uint4 *>(st_lo + soff_r) = lr;
                    *reinterpret_cast<uint4 *>(st_hi + soff_i) = hm;
                    *reinterpret_cast<uint4 *>(st_lo + soff_i) = lm;
                }
                if (!isA) fence_proxy_async_smem();
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&st_full[s]);
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&in_empty[buf]);  // the entry's inputs are no longer read
        }
    } else if (warp == kTcMma) {
        // MMA issue
        if (lane == 0) {
            const uint32_t idesc = BF ? tc_idesc_bf16(128, kTcN) : tc_idesc_tf32(128, kTcN);
            constexpr unsigned LBO = 128, SBO = 4 * 128;  // K-adjacent cores; 8-row groups
            // S descriptors of each stage; one k-step (8 K columns = two core
            // matrices, 256 bytes) further is +16 in the start-address field
            uint64_t dhi[kTcStages], dlo[kTcStages];
#pragma unroll
            for (int k = 0; k < kTcStages; ++k) {
                const unsigned a = smem_addr(smem + sh.off_stage + k * sh.stage_bytes);
                dhi[k] = tc_smem_desc(a, LBO, SBO);
                dlo[k] = tc_smem_desc(a + (unsigned)sh.s_bytes, LBO, SBO);
            }
            for (int lf = 0; lf < nlocal && ok; ++lf) {
                const int db = lf & 1;
                if (lf >= 2 && !mbar_wait(&d_empty[db], ((lf >> 1) - 1) & 1, &g_tc_timeouts)) ok = false;
                tc_fence_after();
                for (int ch = 0; ch < sh.nch && ok; ++ch) {
                    const int gch = lf * sh.nch + ch, s = gch % kTcStages, use = gch / kTcStages;
                    if (!mbar_wait(&st_full[s], use & 1, &g_tc_timeouts)) ok = false;
                    tc_fence_after();
                    const uint64_t bh = s == 0 ? dhi[0] : (s == 1 ? dhi[1] : dhi[2]);
                    const uint64_t bl = s == 0 ? dlo[0] : (s == 1 ? dlo[1] : dlo[2]);
                    for (int t = 0; t < sh.T; ++t) {
                        const unsigned dt = tmem + (unsigned)((db * sh.T + t) * kTcN);
                        const unsigned at = tmem + (unsigned)(kTcAcol + s * kTcAstage + 32 * t);
                        tc_mma_chunk<BF>(dt, at, bh, bl, idesc, ch > 0);
                    }
                    tc_commit(&st_empty[s]);
                }
                tc_commit(&d_full[db]);
            }
        }
    } else {
        // epilogue: TMEM lane quarter ew = warp mod 4
        const int ew = warp - kTcEpi;
        for (int lf = 0; lf < nlocal && ok; ++lf) {
            const int db = lf & 1;
            if (!mbar_wait(&d_full[db], (lf >> 1) & 1, &g_tc_timeouts)) ok = false;
            tc_fence_after();
            int kx, u, p1, p2, npos;
            bool mir0;
            entry(lf, kx, u, p1, p2, npos, mir0);
            for (int t = 0; t < sh.T; ++t) {
                const int tl = 32 * ew + lane;  // TMEM lane
                const bool lane_row = t == 0 || tl >= lane0;
                const int rg = t == 0 ? tl : 128 + tl - lane0;
                const int cog = rg / Lp, ig = rg - cog * Lp;
                // one position (32 columns: 16 real, 16 imaginary) at a time
                for (int pq = 0; pq < 2; ++pq) {
                    uint32_t rr[32];
                    const unsigned ta = tmem + ((unsigned)(32 * ew) << 16) +
                                        (unsigned)((db * sh.T + t) * kTcN + 32 * pq);
                    tc_ld32(ta, rr);
                    tc_wait_ld();
                    if (t == sh.T - 1 && pq == 1) {
                        tc_fence_before();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(&d_empty[db]);
                    }
                    if (!lane_row || pq >= npos || rg >= R || ig >= L) continue;
                    const bool mir = (pq == 0) == mir0;
                    const float rs = s_itau[ig];  // the rows of A were prescaled by t_i / t_0
                    float2 *dst = spec2 + ((size_t)kx * Py + (pq ? p2 : p1)) * planes + ig * 3 + cog;
#pragma unroll
                    for (int b = 0; b < kTcBp; ++b) {
                        if (b >= B) break;
                        const float dre = rs * __uint_as_float(rr[b]), dim = rs * __uint_as_float(rr[16 + b]);
                        float2 hh;
                        if (cog == 2)
                            hh = make_float2(-dim, dre);
                        else if (cog == 1 && mir)
                            hh = make_float2(-dre, -dim);
                        else
                            hh = make_float2(dre, dim);
                        dst[(size_t)b * 3 * L] = hh;
                    }
                }
            }
        }
    }
    if (!ok) atomicExch(&s_abort, 1);
    tc_fence_before();
    __syncthreads();
    if (warp == kTcMma) {
        if (s_abort && lane == 0) {
            // a wait gave up: give the MMAs still in flight time to finish (bounded)
            for (int k = 0; k < 2; ++k) mbar_wait(&d_full[k], 0, &g_tc_timeouts, 1LL << 24);
        }
        __syncwarp();
        tc_fence_after();
        tc_dealloc(tmem, kTcCols);
    }
}

// The tensor-core path of the dense-product contraction: float plans, even
// L <= 64 (a state's 3L complex values are a 16-byte multiple for the bulk
// copies), B <= 16, whole block in shared memory.
bool tc5_supported(int L, int B, int npairs) {
    if (L < 2 || L > 64 || L % 2 != 0 || B < 1 || B > 16) return false;
    return tc_shape(L, B, npairs).total + 1024 <= 227 * 1024;  // 1 KB for the static shared memory
}

cudaError_t launch_contract_tc5(const ApplyArgs &a, bool bf16, cudaStream_t st) {
    const TcShape sh = tc_shape(a.L, a.B, a.npairs, bf16 ? TcKC<true>::value : TcKC<false>::value);
    const bool cmp = a.bmask != nullptr;
    if (a.packed && !bf16) return cudaErrorInvalidValue;  // BF16 split pairs feed the BF16 passes only
    auto kernel = a.packed ? (cmp ? k_contract_tc5<true, true, true> : k_contract_tc5<true, false, true>)
                  : bf16   ? (cmp ? k_contract_tc5<true, true, false> : k_contract_tc5<true, false, false>)
                           : (cmp ? k_contract_tc5<false, true, false> : k_contract_tc5<false, false, false>);
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh.total)) != cudaSuccess)
        return e;
    int dev = 0, nsm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const int Kx = a.kx_count ? a.kx_count : (1 << a.log2Px) / 2 + 1;
    const int nent = Kx * ((1 << a.log2Py) / 2 + 1);
    const int grid = nent < nsm ? nent : nsm;
    kernel<<<grid, kTcThreads, sh.total, st>>>((float2 *)a.spec2, (const float *)a.tensor, (const float *)a.ratio,
                                               a.L, a.B, Kx, a.log2Py, a.npairs, a.bmask, a.bfirst);
    return cudaGetLastError();
}

cudaError_t read_tc_timeouts(unsigned *dst, cudaStream_t st) {
    return cudaMemcpyFromSymbolAsync(dst, g_tc_timeouts, sizeof(unsigned), 0, cudaMemcpyDeviceToHost, st);
}

}  // namespace demag
