// Layer contraction for batches of states on the fifth-generation tensor cores
// (tcgen05, kind::tf32, accumulators in tensor memory), three TF32 passes.
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
// K_c(i <- j) is the stored pair (i <= j), or for i > j the stored (j, i)
// times t_j / t_i with xz and yz negated (reciprocity).  Products: a = a_hi +
// a_lo, s = s_hi + s_lo (TF32), D += a_lo s_hi + a_hi s_lo + a_hi s_hi in FP32.
//
// One persistent block per SM walks the entries.  Roles:
//   warp 21      loader: bulk copies of the entry's compact tensor and its two
//                state rows (one copy per state, to a bank-spreading stride)
//                into shared memory, and L2 prefetch two entries ahead;
//   warps 0-15   producers: build A and S, hi and lo, from those copies,
//                chunk by chunk of 16 columns of K (K-major canonical layout)
//                into a 3-stage ring;
//   warp 20      MMA issue (one thread; M = 128 row tiles, N = 64) and the
//                tensor-memory allocation;
//   warps 16-19  epilogue: accumulators (double-buffered in tensor memory) to
//                the state rows.
// Rows of the last 128-row tile beyond 3L read whatever shared memory follows
// (the MMA needs 128 rows); those accumulator rows are never read.
#include <cstdint>

#include "internal.h"
#include "layout.cuh"
#include "tcgen05.cuh"

namespace demag {

namespace {

constexpr int kTcProd = 16;                          // producer warps
constexpr int kTcThreads = 32 * (kTcProd + 6);       // + 4 epilogue, MMA, prefetch warps
constexpr int kTcEpi = kTcProd, kTcMma = kTcProd + 4, kTcPre = kTcProd + 5;  // first warp of each role
constexpr int kTcN = 64;         // accumulator columns: 2 positions x (re, im) x 16 states
constexpr int kTcBp = 16;
constexpr int kTcKC = 16;        // K columns per chunk (two MMA k-steps)
constexpr int kTcStages = 3;

__device__ unsigned g_tc_timeouts;

struct TcShape {
    int L, Lp, B, planes, R, T, nch, NB, seg;  // seg: padded float2 stride of one state's row segment
    size_t raw_bytes, rows_bytes, a_bytes, s_bytes, stage_bytes, off_rows, off_stage, total;
};

__host__ __device__ inline size_t round128(size_t v) { return (v + 127) / 128 * 128; }

__host__ __device__ inline TcShape tc_shape(int L, int B, int npairs) {
    TcShape s;
    s.L = L;
    s.Lp = (L + 7) / 8 * 8;
    s.B = B;
    s.planes = B * 3 * L;
    s.R = 3 * s.Lp;
    s.T = (s.R + 127) / 128;
    s.nch = (s.R + kTcKC - 1) / kTcKC;  // K = R padded to whole chunks (zero columns)
    s.NB = umajor_block(npairs);
    // a state's 3L complex values, padded so that consecutive states start 16
    // bytes apart modulo 128 (the 8 states a warp reads at once hit 8 bank groups)
    s.seg = 3 * L + ((2 - (3 * L) % 16) + 16) % 16;
    s.raw_bytes = round128((size_t)s.NB * 4);
    s.rows_bytes = round128((size_t)2 * B * s.seg * 8);
    s.a_bytes = (size_t)s.R * kTcKC * 4;
    s.s_bytes = (size_t)kTcN * kTcKC * 4;
    s.stage_bytes = round128(2 * s.a_bytes + 2 * s.s_bytes);
    s.off_rows = s.raw_bytes;
    s.off_stage = s.off_rows + s.rows_bytes;
    s.total = s.off_stage + kTcStages * s.stage_bytes;
    return s;
}

// (output component, source component) -> stored component (xx yy zz xy xz yz)
__device__ __forceinline__ int tc_comp(int co, int ci) {
    const int t = co * 3 + ci;
    return t == 0 ? 0 : t == 4 ? 1 : t == 8 ? 2 : (t == 1 || t == 3) ? 3 : (t == 2 || t == 6) ? 4 : 5;
}

__device__ __forceinline__ void split_tf32(float v, float &hi, float &lo) {
    uint32_t h, l;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(v));
    const float r = v - __uint_as_float(h);
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(l) : "f"(r));
    hi = __uint_as_float(h);
    lo = __uint_as_float(l);
}

}  // namespace

__global__ void __launch_bounds__(kTcThreads, 1) k_contract_tc5(float2 *__restrict__ spec2,
                                                               const float *__restrict__ tensor_um,
                                                               const float *__restrict__ ratio, int L, int B,
                                                               int log2Px, int log2Py, int npairs) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t st_full[kTcStages], st_empty[kTcStages], d_full[2], d_empty[2];
    __shared__ __align__(8) uint64_t in_full, in_empty;  // the entry's tensor and state rows in shared memory
    __shared__ unsigned tmem_slot;
    __shared__ __align__(16) float s_tau[64], s_itau[64];
    __shared__ int s_rb[64];  // index of pair (i, i) minus i: pair (i, j >= i) is s_rb[i] + j
    __shared__ int s_abort;
    const TcShape sh = tc_shape(L, B, npairs);
    const int Py = 1 << log2Py, Qy = Py / 2 + 1, Kx = (1 << log2Px) / 2 + 1;
    const int nent = Kx * Qy;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int Lp = sh.Lp, planes = sh.planes, R = sh.R;
    bool ok = true;

    if (tid == 0) {
        for (int k = 0; k < kTcStages; ++k) {
            mbar_init(&st_full[k], kTcProd);
            mbar_init(&st_empty[k], 1);
        }
        for (int k = 0; k < 2; ++k) {
            mbar_init(&d_full[k], 1);
            mbar_init(&d_empty[k], 4);
        }
        mbar_init(&in_full, 1);
        mbar_init(&in_empty, kTcProd);
        mbar_init_fence();
        s_abort = 0;
    }
    if (tid < 64) {
        s_tau[tid] = tid < L ? ratio[tid] : 0.f;       // t_l / t_0
        s_itau[tid] = tid < L ? ratio[tid * L] : 0.f;  // t_0 / t_l
        s_rb[tid] = tid * L - (tid * (tid - 1)) / 2 - tid;
    }
    if (warp == kTcMma) tc_alloc(&tmem_slot, 256);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = tmem_slot;

    auto entry = [&](int lf, int &kx, int &u, int &p1, int &p2, int &npos, bool &mir0) {
        const int f = blockIdx.x + lf * gridDim.x;
        kx = f / Qy;
        u = f - kx * Qy;
        u_positions(u, log2Py, p1, p2);
        npos = p2 != p1 ? 2 : 1;
        mir0 = bitrev_n(p1, log2Py) > Py / 2;  // position 0 is the mirrored frequency
    };
    const int nlocal = blockIdx.x < nent ? (nent - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;

    if (warp == kTcPre) {
        // loader: entry lf into shared memory once the producers released lf - 1;
        // L2 prefetch of entry lf + 2
        if (lane == 0) {
            auto prefetch = [&](int lf) {
                if (lf >= nlocal) return;
                int kx, u, p1, p2, npos;
                bool mir0;
                entry(lf, kx, u, p1, p2, npos, mir0);
                asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(tensor_um + ((size_t)kx * Qy + u) * sh.NB),
                             "r"((unsigned)sh.NB * 4) : "memory");
                asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(spec2 + ((size_t)kx * Py + p1) * planes),
                             "r"((unsigned)planes * 8) : "memory");
                if (npos == 2)
                    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(
                                     spec2 + ((size_t)kx * Py + p2) * planes),
                                 "r"((unsigned)planes * 8) : "memory");
            };
            prefetch(0);
            prefetch(1);
            const unsigned segb = (unsigned)(3 * L) * 8;  // one state's values (16-byte multiple)
            for (int lf = 0; lf < nlocal && ok; ++lf) {
                if (lf >= 1 && !mbar_wait(&in_empty, (lf - 1) & 1, &g_tc_timeouts)) ok = false;
                int kx, u, p1, p2, npos;
                bool mir0;
                entry(lf, kx, u, p1, p2, npos, mir0);
                mbar_arrive_expect_tx(&in_full, (unsigned)sh.NB * 4 + (unsigned)(npos * B) * segb);
                bulk_copy_g2s(smem, tensor_um + ((size_t)kx * Qy + u) * sh.NB, (unsigned)sh.NB * 4, &in_full);
                for (int q = 0; q < npos; ++q) {
                    const float2 *src = spec2 + ((size_t)kx * Py + (q ? p2 : p1)) * planes;
                    float2 *dst = reinterpret_cast<float2 *>(smem + sh.off_rows) + (size_t)q * B * sh.seg;
                    for (int b = 0; b < B; ++b)
                        bulk_copy_g2s(dst + (size_t)b * sh.seg, src + (size_t)b * 3 * L, segb, &in_full);
                }
                prefetch(lf + 2);
            }
        }
    } else if (warp < kTcProd) {
        // producers: a unit is 4 consecutive K columns of one row (16 bytes of one
        // core-matrix row); 8 consecutive units fill one core matrix, so each warp
        // store covers whole 128-byte core matrices.  A thread keeps its units (and
        // everything about them that does not depend on the chunk) for the whole run.
        constexpr int KG = kTcKC / 4;  // core matrices along K per chunk
        constexpr int NU = 4;          // at most 4 units per thread and chunk
        const int na = R * KG, ntot = na + kTcN * KG;
        const float *raw = reinterpret_cast<const float *>(smem);  // [6][NR]
        const float2 *rows = reinterpret_cast<const float2 *>(smem + sh.off_rows);
        const int NR = umajor_row(npairs);
        struct Unit {
            int off;      // float offset in the A or S buffer of a stage
            int row, k4;  // row (A: co * Lp + i; S: column n), core column
            int c0, c1, c2;  // A: stored component for source component x, y, z
            bool isA, live;
        };
        Unit un[NU];
#pragma unroll
        for (int k = 0; k < NU; ++k) {
            const int v = tid + k * 32 * kTcProd;
            Unit &x = un[k];
            x.live = v < ntot;
            x.isA = v < na;
            const int w = x.isA ? v : v - na;
            const int core = w >> 3, rr = w & 7;
            x.row = (core / KG) * 8 + rr;
            x.k4 = core % KG;
            x.off = core * 32 + rr * 4;
            const int co = (x.row >= Lp) + (x.row >= 2 * Lp);
            x.c0 = tc_comp(co, 0);
            x.c1 = tc_comp(co, 1);
            x.c2 = tc_comp(co, 2);
        }
        for (int lf = 0; lf < nlocal && ok; ++lf) {
            int kx, u, p1, p2, npos;
            bool mir0;
            entry(lf, kx, u, p1, p2, npos, mir0);
            if (!mbar_wait(&in_full, lf & 1, &g_tc_timeouts)) ok = false;
            for (int ch = 0; ch < sh.nch && ok; ++ch) {
                const int gch = lf * sh.nch + ch, s = gch % kTcStages, use = gch / kTcStages;
                if (use >= 1 && !mbar_wait(&st_empty[s], (use - 1) & 1, &g_tc_timeouts)) ok = false;
                float *a_hi = reinterpret_cast<float *>(smem + sh.off_stage + s * sh.stage_bytes);
                float *a_lo = a_hi + R * kTcKC, *s_hi = a_lo + R * kTcKC, *s_lo = s_hi + kTcN * kTcKC;
#pragma unroll
                for (int k = 0; k < NU; ++k) {
                    const Unit &x = un[k];
                    if (!x.live) continue;
                    const int kc = ch * kTcKC + 4 * x.k4;  // first K column of the unit
                    const int ci = (kc >= Lp) + (kc >= 2 * Lp), jb = kc - ci * Lp;
                    float val[4] = {0.f, 0.f, 0.f, 0.f};
                    if (kc < R) {
                        if (x.isA) {
                            const int co = (x.row >= Lp) + (x.row >= 2 * Lp), i = x.row - co * Lp;
                            const int comp = ci == 0 ? x.c0 : (ci == 1 ? x.c1 : x.c2);
                            const float zs = (co == 2 && ci == 2) ? -1.f : 1.f;
                            if (i < L) {
                                if (jb >= i) {
                                    // upper triangle: pairs (i, jb..jb+3) are consecutive
                                    const float *pb = raw + comp * NR + s_rb[i] + jb;
#pragma unroll
                                    for (int e = 0; e < 4; ++e)
                                        if (jb + e < L) val[e] = zs * pb[e];
                                } else {
                                    const float4 tj = *reinterpret_cast<const float4 *>(s_tau + jb);
                                    const float tjs[4] = {tj.x, tj.y, tj.z, tj.w};
                                    const float sc = zs * s_itau[i] * (comp >= 4 ? -1.f : 1.f);
#pragma unroll
                                    for (int e = 0; e < 4; ++e) {
                                        const int j = jb + e;
                                        if (j >= L) continue;
                                        val[e] = j < i ? sc * tjs[e] * raw[comp * NR + s_rb[j] + i]
                                                       : zs * raw[comp * NR + s_rb[i] + j];
                                    }
                                }
                            }
                        } else {
                            const int q = x.row >> 5, ri = (x.row >> 4) & 1, b = x.row & (kTcBp - 1);
                            if (q < npos && b < B) {
                                const bool neg_y = (ci == 1) && ((q == 0) == mir0);
                                const float2 *m = rows + ((size_t)q * B + b) * sh.seg + jb * 3 + ci;
#pragma unroll
                                for (int e = 0; e < 4; ++e) {
                                    if (jb + e >= L) continue;
                                    const float2 mv = m[3 * e];
                                    const float xv = ci < 2 ? (ri ? mv.y : mv.x) : (ri ? mv.x : -mv.y);
                                    val[e] = neg_y ? -xv : xv;
                                }
                            }
                        }
                    }
                    float4 h, l;
                    split_tf32(val[0], h.x, l.x);
                    split_tf32(val[1], h.y, l.y);
                    split_tf32(val[2], h.z, l.z);
                    split_tf32(val[3], h.w, l.w);
                    *reinterpret_cast<float4 *>((x.isA ? a_hi : s_hi) + x.off) = h;
                    *reinterpret_cast<float4 *>((x.isA ? a_lo : s_lo) + x.off) = l;
                }
                fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) mbar_arrive(&st_full[s]);
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&in_empty);  // the entry's inputs are no longer read
        }
    } else if (warp == kTcMma) {
        // MMA issue
        if (lane == 0) {
            const uint32_t idesc = tc_idesc_tf32(128, kTcN);
            constexpr unsigned LBO = 128, SBO = (kTcKC / 4) * 128;  // K-adjacent cores; 8-row groups
            for (int lf = 0; lf < nlocal && ok; ++lf) {
                const int db = lf & 1;
                if (lf >= 2 && !mbar_wait(&d_empty[db], ((lf >> 1) - 1) & 1, &g_tc_timeouts)) ok = false;
                tc_fence_after();
                for (int ch = 0; ch < sh.nch && ok; ++ch) {
                    const int gch = lf * sh.nch + ch, s = gch % kTcStages, use = gch / kTcStages;
                    if (!mbar_wait(&st_full[s], use & 1, &g_tc_timeouts)) ok = false;
                    tc_fence_after();
                    const unsigned stage = smem_addr(smem + sh.off_stage + s * sh.stage_bytes);
                    const unsigned a_hi = stage, a_lo = stage + (unsigned)sh.a_bytes;
                    const unsigned s_hi = a_lo + (unsigned)sh.a_bytes, s_lo = s_hi + (unsigned)sh.s_bytes;
                    for (int t = 0; t < sh.T; ++t) {
                        const unsigned dt = tmem + (unsigned)((db * sh.T + t) * kTcN);
                        const unsigned toff = (unsigned)t * 16 * SBO;  // 128 rows further
#pragma unroll
                        for (int ks = 0; ks < kTcKC / 8; ++ks) {
                            const unsigned ko = (unsigned)ks * 2 * LBO;  // 8 K columns further
                            tc_mma_tf32(dt, tc_smem_desc(a_lo + toff + ko, LBO, SBO),
                                        tc_smem_desc(s_hi + ko, LBO, SBO), idesc, ch > 0 || ks > 0);
                            tc_mma_tf32(dt, tc_smem_desc(a_hi + toff + ko, LBO, SBO),
                                        tc_smem_desc(s_lo + ko, LBO, SBO), idesc, true);
                            tc_mma_tf32(dt, tc_smem_desc(a_hi + toff + ko, LBO, SBO),
                                        tc_smem_desc(s_hi + ko, LBO, SBO), idesc, true);
                        }
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
                const int rg = t * 128 + 32 * ew + lane;
                const int co = rg / Lp, i = rg - co * Lp;
                // one position (32 columns: 16 real, 16 imaginary) at a time
                for (int q = 0; q < 2; ++q) {
                    uint32_t r[32];
                    const unsigned ta = tmem + ((unsigned)(32 * ew) << 16) +
                                        (unsigned)((db * sh.T + t) * kTcN + 32 * q);
                    tc_ld32(ta, r);
                    tc_wait_ld();
                    if (t == sh.T - 1 && q == 1) {
                        tc_fence_before();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(&d_empty[db]);
                    }
                    if (q >= npos || rg >= R || i >= L) continue;
                    const bool mir = (q == 0) == mir0;
                    float2 *dst = spec2 + ((size_t)kx * Py + (q ? p2 : p1)) * planes + i * 3 + co;
#pragma unroll
                    for (int b = 0; b < kTcBp; ++b) {
                        if (b >= B) break;
                        const float dre = __uint_as_float(r[b]), dim = __uint_as_float(r[16 + b]);
                        float2 h;
                        if (co == 2)
                            h = make_float2(-dim, dre);
                        else if (co == 1 && mir)
                            h = make_float2(-dre, -dim);
                        else
                            h = make_float2(dre, dim);
                        dst[(size_t)b * 3 * L] = h;
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
        tc_dealloc(tmem, 256);
    }
}

// The tensor-core path of the dense-product contraction: float plans, even
// L <= 64 (a state's 3L complex values are a 16-byte multiple for the bulk
// copies), B <= 16, whole block in shared memory.
bool tc5_supported(int L, int B, int npairs) {
    if (L < 2 || L > 64 || L % 2 != 0 || B < 1 || B > 16) return false;
    return tc_shape(L, B, npairs).total + 1024 <= 227 * 1024;  // 1 KB for the static shared memory
}

cudaError_t launch_contract_tc5(const ApplyArgs &a, cudaStream_t st) {
    const TcShape sh = tc_shape(a.L, a.B, a.npairs);
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_contract_tc5, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh.total)) !=
        cudaSuccess)
        return e;
    int dev = 0, nsm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    const int nent = ((1 << a.log2Px) / 2 + 1) * ((1 << a.log2Py) / 2 + 1);
    const int grid = nent < nsm ? nent : nsm;
    k_contract_tc5<<<grid, kTcThreads, sh.total, st>>>((float2 *)a.spec2, (const float *)a.tensor,
                                                       (const float *)a.ratio, a.L, a.B, a.log2Px, a.log2Py,
                                                       a.npairs);
    return cudaGetLastError();
}

unsigned take_tc_timeouts() {
    unsigned n = 0, zero = 0;
    if (cudaMemcpyFromSymbol(&n, g_tc_timeouts, sizeof(n)) != cudaSuccess) return ~0u;
    if (n != 0) cudaMemcpyToSymbol(g_tc_timeouts, &zero, sizeof(zero));
    return n;
}

}  // namespace demag
