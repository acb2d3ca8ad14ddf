// Layer contraction as small dense matrix products, for batches of states.
//
// At one frequency k the contraction of Eq. FFT_v2, H(b, i) = sum_j N_k(i <- j)
// m(b, j), with the symmetric blocks N = [[xx, xy, i xz], [xy, yy, i yz],
// [i xz, i yz, zz]] (xx, yy, zz, xy real, xz, yz imaginary coefficients) splits
// into 18 real products of L x L component matrices with L x B state matrices:
//   Hr_x = Kxx Mr_x + s Kxy Mr_y -   Kxz Mi_z     Hi_x = Kxx Mi_x + s Kxy Mi_y +   Kxz Mr_z
//   Hr_y = s Kxy Mr_x + Kyy Mr_y - s Kyz Mi_z     Hi_y = s Kxy Mi_x + Kyy Mi_y + s Kyz Mr_z
//   Hr_z = -Kxz Mi_x - s Kyz Mi_y + Kzz Mr_z      Hi_z = Kxz Mr_x + s Kyz Mr_y + Kzz Mi_z
// (s = -1 at the mirrored frequency Py - ky, where xy and yz change sign):
// exactly 36 L^2 B flops, nothing spent on zero blocks.
//
// One block per (kx, stored entry u): the compact tensor of the entry (pairs
// i <= j, [kx][u][pair][6], contiguous) is expanded into the six dense L x L
// matrices in shared memory (the lower triangle from reciprocity, t_i N(i<-j)
// = t_j N(j<-i)(-d)); the states at the entry's two positions are staged as
// 12 L x B matrices; the products run either on the tensor cores in three
// TF32 passes (a = a_hi + a_lo, b = b_hi + b_lo: a_hi b_hi + a_hi b_lo +
// a_lo b_hi, FP32 accumulation) or on the FP32 CUDA cores with the same data
// movement; the result is written back in place.
#include <cstdint>

#include "fft.cuh"
#include "internal.h"
#include "layout.cuh"

namespace demag {

constexpr int kGemmThreads = 256;

// Shared-memory row stride of the L x L and B x L operands: rows of 4 banks
// apart, so the 8 x 4 lane pattern of an m16n8k8 fragment hits 32 banks.
__host__ __device__ inline int gemm_stride(int Lp) { return Lp + 4; }

// Padded sizes: L to a multiple of 16 (MMA rows), B to a multiple of 8 (MMA columns).
__host__ __device__ inline int pad16(int v) { return (v + 15) / 16 * 16; }
__host__ __device__ inline int pad8(int v) { return (v + 7) / 8 * 8; }

// Operands (6 L x L matrices, 2 x 6 B x L matrices) and the output area
// (2 positions x 6 matrices x L x B).
size_t gemm_smem_bytes(int L, int B) {
    const int Lp = pad16(L), Bp = pad8(B), S = gemm_stride(Lp);
    return (size_t)(6 * Lp * S + 2 * 6 * Bp * S + 2 * 6 * Lp * Bp) * sizeof(float);
}

// The tensor-core variant keeps 2 x 8 accumulator tiles per warp: B <= 64.
bool gemm_supported(int L, int B) { return pad8(B) <= 64 && gemm_smem_bytes(L, B) <= 220 * 1024; }

__device__ __forceinline__ uint32_t to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Terms of the six output matrices: (component matrix, state matrix, sign
// flag).  Component 0..5 = xx, yy, zz, xy, xz, yz.  State matrix 0..5 =
// Mr_x, Mr_y, Mr_z, Mi_x, Mi_y, Mi_z.  Sign: +1 / -1, and "mirror" terms
// (xy, yz) are further multiplied by s.
struct Term {
    int comp, state;
    float sign;
};
__constant__ Term c_terms[6][3] = {
    {{0, 0, 1.f}, {3, 1, 1.f}, {4, 5, -1.f}},   // Hr_x
    {{0, 3, 1.f}, {3, 4, 1.f}, {4, 2, 1.f}},    // Hi_x
    {{3, 0, 1.f}, {1, 1, 1.f}, {5, 5, -1.f}},   // Hr_y
    {{3, 3, 1.f}, {1, 4, 1.f}, {5, 2, 1.f}},    // Hi_y
    {{4, 3, -1.f}, {5, 4, -1.f}, {2, 2, 1.f}},  // Hr_z
    {{4, 0, 1.f}, {5, 1, 1.f}, {2, 5, 1.f}},    // Hi_z
};

template <bool TC>
__global__ void __launch_bounds__(kGemmThreads, 1) k_contract_gemm(
    float2 *__restrict__ spec2, const float *__restrict__ tensor_um, const float *__restrict__ ratio,
    int L, int B, int log2Py, int npairs) {
    extern __shared__ __align__(16) float smem_f[];
    const int Lp = pad16(L), Bp = pad8(B), S = gemm_stride(Lp);
    float *Kd = smem_f;                  // [6][Lp][S]: K_c[i][j]
    float *Ms = smem_f + 6 * Lp * S;     // [2 positions][6][Bp][S]: M_s[b][j]
    const int Py = 1 << log2Py, Qy = Py / 2 + 1;
    const int planes = B * 3 * L;
    const int kx = blockIdx.x, u = blockIdx.y;
    int p1, p2;
    u_positions(u, log2Py, p1, p2);
    const int ky1 = bit_reverse(p1, log2Py);
    const float s_pos[2] = {ky1 > Py / 2 ? -1.f : 1.f, ky1 > Py / 2 ? 1.f : -1.f};
    const int npos = p2 != p1 ? 2 : 1;

    // zero the operands (padding rows and columns stay zero), then expand the
    // compact tensor
    for (int e = threadIdx.x; e < 6 * Lp * S + 2 * 6 * Bp * S; e += kGemmThreads) smem_f[e] = 0.f;
    __syncthreads();
    // compact tensor of the entry (blocked, layout.cuh), contiguous and 16-byte
    // aligned; all loads of a thread are issued before any is used
    const int nb = ub_nb(L), NR = ub_row(L), NB = 6 * NR;
    const float4 *tu4 = reinterpret_cast<const float4 *>(tensor_um + ((size_t)kx * Qy + u) * NB);
    const int n4 = NB / 4;
    constexpr int kBatch = 8;
    for (int base = threadIdx.x; base < n4; base += kGemmThreads * kBatch) {
        float4 v[kBatch];
#pragma unroll
        for (int k = 0; k < kBatch; ++k) {
            const int e4 = base + k * kGemmThreads;
            v[k] = e4 < n4 ? tu4[e4] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int k = 0; k < kBatch; ++k) {
            const int e4 = base + k * kGemmThreads;
            if (e4 >= n4) break;
            const float vals[4] = {v[k].x, v[k].y, v[k].z, v[k].w};
#pragma unroll
            for (int w = 0; w < 4; ++w) {
                const int e = 4 * e4 + w;
                const int c = e / NR, q = e - c * NR;  // [component][block][half-row slots]
                // block (R, C) of index q / 64: block rows of nb, nb - 1, ... blocks
                int R = 0, rem = q >> 6;
                while (rem >= nb - R) {
                    rem -= nb - R;
                    ++R;
                }
                // float f of block (R, C): half h = f / 32 of row
                // ((f / 4) mod 8) ^ (C mod 4) ^ 4 h (ub_at)
                const int f = q & 63, h = f >> 5;
                const int a = 8 * R + ((((f >> 2) & 7) ^ ((R + rem) & 3) ^ (4 * h))),
                          b = 8 * (R + rem) + 4 * h + (f & 3);
                if (a >= L || b >= L) continue;  // padding layers
                // value M(a, b) = (t_a / t_0) N(a <- b): target a <- source b
                Kd[(c * Lp + a) * S + b] = ratio[a * L] * vals[w];
                if (rem > 0)  // off-diagonal block: target b <- source a by reciprocity
                    Kd[(c * Lp + b) * S + a] = ratio[b * L] * (c >= 4 ? -1.f : 1.f) * vals[w];
            }
        }
    }
    // stage the states at the entry's positions: M[b][j] per (component, re/im)
    float2 *sk = spec2 + (size_t)kx * Py * planes;
    for (int pos = 0; pos < npos; ++pos) {
        const float2 *row = sk + (size_t)(pos ? p2 : p1) * planes;
        float *m = Ms + (size_t)pos * 6 * Bp * S;
        for (int base = threadIdx.x; base < planes; base += kGemmThreads * kBatch) {
            float2 v[kBatch];
#pragma unroll
            for (int k = 0; k < kBatch; ++k) {
                const int g = base + k * kGemmThreads;
                v[k] = g < planes ? row[g] : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int k = 0; k < kBatch; ++k) {
                const int g = base + k * kGemmThreads;
                if (g >= planes) break;
                const int b = g / (3 * L), rem = g - b * 3 * L, j = rem / 3, c = rem - j * 3;
                m[(c * Bp + b) * S + j] = v[k].x;        // Mr_c
                m[((3 + c) * Bp + b) * S + j] = v[k].y;  // Mi_c
            }
        }
    }
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int mtiles = Lp / 16, ntiles = Bp / 8;
    if (TC) {
        // unit = (output matrix, m-tile); a warp accumulates all n-tiles of both positions
        const int units = 6 * mtiles;
        const int gr = lane >> 2, gc = lane & 3;
        for (int unit = warp; unit < units; unit += kGemmThreads / 32) {
            const int o = unit / mtiles, mt = unit - o * mtiles;
            float acc[2][8][4];  // [position][n-tile <= 8][fragment]
#pragma unroll
            for (int q = 0; q < 2; ++q)
#pragma unroll
                for (int n = 0; n < 8; ++n)
#pragma unroll
                    for (int f = 0; f < 4; ++f) acc[q][n][f] = 0.f;
            for (int t = 0; t < 3; ++t) {
                const Term tm = c_terms[o][t];
                const bool mirror = tm.comp == 3 || tm.comp == 5;
                const float *A = Kd + (size_t)tm.comp * Lp * S + (mt * 16) * S;
                for (int k0 = 0; k0 < Lp; k0 += 8) {
                    const float a0 = A[gr * S + k0 + gc], a1 = A[(gr + 8) * S + k0 + gc];
                    const float a2 = A[gr * S + k0 + gc + 4], a3 = A[(gr + 8) * S + k0 + gc + 4];
#pragma unroll
                    for (int q = 0; q < 2; ++q) {
                        if (q >= npos) break;
                        const float sg = tm.sign * (mirror ? s_pos[q] : 1.f);
                        uint32_t ah[4], al[4];
                        const float av[4] = {sg * a0, sg * a1, sg * a2, sg * a3};
#pragma unroll
                        for (int f = 0; f < 4; ++f) {
                            ah[f] = to_tf32(av[f]);
                            al[f] = to_tf32(av[f] - __uint_as_float(ah[f]));
                        }
                        const float *Bm = Ms + ((size_t)q * 6 + tm.state) * Bp * S;
#pragma unroll
                        for (int n = 0; n < 8; ++n) {
                            if (n >= ntiles) break;
                            const float b0 = Bm[(n * 8 + gr) * S + k0 + gc];
                            const float b1 = Bm[(n * 8 + gr) * S + k0 + gc + 4];
                            uint32_t bh[2] = {to_tf32(b0), to_tf32(b1)};
                            uint32_t bl[2] = {to_tf32(b0 - __uint_as_float(bh[0])),
                                              to_tf32(b1 - __uint_as_float(bh[1]))};
                            mma_tf32(acc[q][n], al, bh);
                            mma_tf32(acc[q][n], ah, bl);
                            mma_tf32(acc[q][n], ah, bh);
                        }
                    }
                }
            }
            // results to the output area (spec2 is written after the final barrier)
            float *Out = smem_f + 6 * Lp * S + 2 * 6 * Bp * S;
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                if (q >= npos) break;
#pragma unroll
                for (int n = 0; n < 8; ++n) {
                    if (n >= ntiles) break;
#pragma unroll
                    for (int f = 0; f < 4; ++f) {
                        const int i = mt * 16 + gr + (f >= 2 ? 8 : 0);
                        const int b = n * 8 + 2 * gc + (f & 1);
                        Out[(((size_t)q * 6 + o) * Lp + i) * Bp + b] = acc[q][n][f];
                    }
                }
            }
        }
    } else {
        // CUDA cores: thread block of 4 rows x 4 states of one output matrix and position
        const int rb = Lp / 4, cb = Bp / 4;
        const int units = npos * 6 * rb * cb;
        float *Out = smem_f + 6 * Lp * S + 2 * 6 * Bp * S;
        for (int unit = threadIdx.x; unit < units; unit += kGemmThreads) {
            int r = unit;
            const int cbi = r % cb;
            r /= cb;
            const int rbi = r % rb;
            r /= rb;
            const int o = r % 6, q = r / 6;
            float acc[4][4] = {};
            for (int t = 0; t < 3; ++t) {
                const Term tm = c_terms[o][t];
                const bool mirror = tm.comp == 3 || tm.comp == 5;
                const float sg = tm.sign * (mirror ? s_pos[q] : 1.f);
                const float *A = Kd + (size_t)tm.comp * Lp * S + (rbi * 4) * S;
                const float *Bm = Ms + ((size_t)q * 6 + tm.state) * Bp * S + (cbi * 4) * S;
                for (int j = 0; j < Lp; ++j) {
                    float av[4], bv[4];
#pragma unroll
                    for (int x = 0; x < 4; ++x) {
                        av[x] = sg * A[x * S + j];
                        bv[x] = Bm[x * S + j];
                    }
#pragma unroll
                    for (int x = 0; x < 4; ++x)
#pragma unroll
                        for (int y = 0; y < 4; ++y) acc[x][y] = fmaf(av[x], bv[y], acc[x][y]);
                }
            }
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
                for (int y = 0; y < 4; ++y)
                    Out[(((size_t)q * 6 + o) * Lp + rbi * 4 + x) * Bp + cbi * 4 + y] = acc[x][y];
        }
    }
    __syncthreads();
    // results: Out[pos][o][i][b] -> spec2 at the entry's positions, (re, im) pairs
    const float *Out = smem_f + 6 * Lp * S + 2 * 6 * Bp * S;
    for (int e = threadIdx.x; e < npos * planes; e += kGemmThreads) {
        const int pos = e / planes, g = e - pos * planes;
        const int b = g / (3 * L), rem = g - b * 3 * L, i = rem / 3, c = rem - i * 3;
        const float re = Out[(((size_t)pos * 6 + 2 * c) * Lp + i) * Bp + b];
        const float im = Out[(((size_t)pos * 6 + 2 * c + 1) * Lp + i) * Bp + b];
        sk[(size_t)(pos ? p2 : p1) * planes + g] = make_float2(re, im);
    }
}

// ---------------------------------------------------------------------------
// Tensor-core contraction for B <= 16 (NT = Bp / 8 n-tiles), two blocks per SM.
//
// The compact tensor of the entry stays compact in shared memory: each
// m16n8k8 A fragment element (target i, source j) is M(i, j) t_0 / t_i, with
// M(i, j) read from its 8 x 8 block (layout.cuh), or for a block below the
// diagonal from element (j, i) of the transposed block with xz and yz negated
// (reciprocity), so the six dense L x L matrices are never formed.  Warp unit = (m-tile of 16 targets,
// position); it keeps the six outputs of its unit in registers and, per
// k-step, splits the 6 x NT state fragments once and each component's A
// fragment once, then issues the 18 products (3 TF32 passes each).
template <int NT>
__global__ void __launch_bounds__(kGemmThreads, 2) k_contract_tc(float2 *__restrict__ spec2,
                                                               const float *__restrict__ tensor_um,
                                                               const float *__restrict__ ratio, int L, int B,
                                                               int log2Py, int npairs) {
    extern __shared__ __align__(16) float smem_f[];
    const int Lp = pad16(L), Bp = 8 * NT, S = gemm_stride(Lp);
    const int nb = ub_nb(L), NR = ub_row(L), NB = 6 * NR;
    float *raw = smem_f;                     // [6][NR]: the entry's component rows
    float *Ms = smem_f + NB;                 // [2][6][Bp][S]: M_s[b][j]; later the output rows
    float *s_tau = Ms + 2 * 6 * Bp * S;      // [Lp]: t_l / t_0
    float *s_itau = s_tau + Lp;              // [Lp]: t_0 / t_l
    const int Py = 1 << log2Py, Qy = Py / 2 + 1;
    const int planes = B * 3 * L;
    const int kx = blockIdx.x, u = blockIdx.y;
    int p1, p2;
    u_positions(u, log2Py, p1, p2);
    const int ky1 = bit_reverse(p1, log2Py);
    const int npos = p2 != p1 ? 2 : 1;
    const int tid = threadIdx.x;

    // compact tensor (contiguous, 16-byte aligned)
    {
        const float4 *src = reinterpret_cast<const float4 *>(tensor_um + ((size_t)kx * Qy + u) * NB);
        float4 *dst = reinterpret_cast<float4 *>(raw);
        const int n4 = NB / 4;
        constexpr int kBatch = 13;
        for (int base = tid; base < n4; base += kGemmThreads * kBatch) {
            float4 v[kBatch];
#pragma unroll
            for (int k = 0; k < kBatch; ++k) {
                const int e = base + k * kGemmThreads;
                if (e < n4) v[k] = src[e];
            }
#pragma unroll
            for (int k = 0; k < kBatch; ++k) {
                const int e = base + k * kGemmThreads;
                if (e < n4) dst[e] = v[k];
            }
        }
    }
    if (tid < Lp) {
        s_tau[tid] = tid < L ? ratio[tid] : 0.f;           // t_l / t_0
        s_itau[tid] = tid < L ? ratio[tid * L] : 0.f;      // t_0 / t_l
    }
    if (Bp != B || Lp != L)
        for (int e = tid; e < 2 * 6 * Bp * S; e += kGemmThreads) Ms[e] = 0.f;
    __syncthreads();
    // states at the entry's positions: element (b, j, c) of a position row is
    // plane b * 3L + 3 j + c; thread r < 3L takes j = r / 3, c = r % 3 for every b
    float2 *sk = spec2 + (size_t)kx * Py * planes;
    if (tid < 3 * L) {
        const int j = tid / 3, c = tid - 3 * (tid / 3);
        for (int pos = 0; pos < npos; ++pos) {
            const float2 *row = sk + (size_t)(pos ? p2 : p1) * planes + tid;
            float *m = Ms + (size_t)pos * 6 * Bp * S;
            for (int b0 = 0; b0 < B; b0 += 16) {
                float2 v[16];
#pragma unroll
                for (int k = 0; k < 16; ++k)
                    if (b0 + k < B) v[k] = row[(size_t)(b0 + k) * 3 * L];
#pragma unroll
                for (int k = 0; k < 16; ++k) {
                    if (b0 + k >= B) break;
                    m[(c * Bp + b0 + k) * S + j] = v[k].x;        // Mr_c
                    m[((3 + c) * Bp + b0 + k) * S + j] = v[k].y;  // Mi_c
                }
            }
        }
    }
    __syncthreads();

    const int warp = tid >> 5, lane = tid & 31;
    const int gr = lane >> 2, gc = lane & 3;
    const int mtiles = Lp / 16;
    // a warp holds at most one unit's accumulators across the final barrier
    float acc[6][NT][4];
    int my_mt = -1, my_q = 0;
    for (int unit = warp; unit < mtiles * npos; unit += kGemmThreads / 32) {
        const int mt = unit % mtiles, q = unit / mtiles;
        // s = -1 at the mirrored frequency: xy and yz change sign
        const bool neg_mirror = ((q == 0) == (ky1 > Py / 2));
        const uint32_t smask = neg_mirror ? 0x80000000u : 0u;
#pragma unroll
        for (int o = 0; o < 6; ++o)
#pragma unroll
            for (int n = 0; n < NT; ++n)
#pragma unroll
                for (int f = 0; f < 4; ++f) acc[o][n][f] = 0.f;
        const float *Mq = Ms + (size_t)q * 6 * Bp * S;
        for (int k0 = 0; k0 < Lp; k0 += 8) {
            uint32_t bh[6][NT][2], bl[6][NT][2];
#pragma unroll
            for (int st = 0; st < 6; ++st)
#pragma unroll
                for (int n = 0; n < NT; ++n) {
                    const float *bp = Mq + ((size_t)st * Bp + n * 8 + gr) * S + k0 + gc;
                    const float b0 = bp[0], b1 = bp[4];
                    bh[st][n][0] = to_tf32(b0);
                    bh[st][n][1] = to_tf32(b1);
                    bl[st][n][0] = to_tf32(b0 - __uint_as_float(bh[st][n][0]));
                    bl[st][n][1] = to_tf32(b1 - __uint_as_float(bh[st][n][1]));
                }
            // fragment elements f: (row gr | gr + 8, column gc | gc + 4)
            int base[4];
            float scl[4];
            bool rev[4];
#pragma unroll
            for (int f = 0; f < 4; ++f) {
                const int i = mt * 16 + gr + ((f & 1) ? 8 : 0), jj = k0 + gc + ((f & 2) ? 4 : 0);
                const int I = i >> 3, J = jj >> 3;
                rev[f] = I > J;
                base[f] = (i < L && jj < L) ? (rev[f] ? ub_blk(J, I, nb) + ub_at(jj & 7, i & 7, I)
                                                      : ub_blk(I, J, nb) + ub_at(i & 7, jj & 7, J))
                                            : -1;
                scl[f] = s_itau[i];
            }
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                uint32_t ah[4], al[4];
#pragma unroll
                for (int f = 0; f < 4; ++f) {
                    float v = base[f] >= 0 ? raw[c * NR + base[f]] * scl[f] : 0.f;
                    if (c >= 4 && rev[f]) v = -v;
                    ah[f] = to_tf32(v);
                    al[f] = to_tf32(v - __uint_as_float(ah[f]));
                }
                // the component's terms: (output, state, sign mask)
                auto term = [&](int o, int st, uint32_t mask) {
                    uint32_t ahs[4], als[4];
#pragma unroll
                    for (int f = 0; f < 4; ++f) {
                        ahs[f] = ah[f] ^ mask;
                        als[f] = al[f] ^ mask;
                    }
#pragma unroll
                    for (int n = 0; n < NT; ++n) {
                        mma_tf32(acc[o][n], als, bh[st][n]);
                        mma_tf32(acc[o][n], ahs, bl[st][n]);
                        mma_tf32(acc[o][n], ahs, bh[st][n]);
                    }
                };
                constexpr uint32_t NEG = 0x80000000u;
                // states 0..5 = Mr_x, Mr_y, Mr_z, Mi_x, Mi_y, Mi_z; outputs 0..5 =
                // Hr_x, Hi_x, Hr_y, Hi_y, Hr_z, Hi_z
                if (c == 0) { term(0, 0, 0); term(1, 3, 0); }
                if (c == 1) { term(2, 1, 0); term(3, 4, 0); }
                if (c == 2) { term(4, 2, 0); term(5, 5, 0); }
                if (c == 3) { term(0, 1, smask); term(1, 4, smask); term(2, 0, smask); term(3, 3, smask); }
                if (c == 4) { term(0, 5, NEG); term(1, 2, 0); term(4, 3, NEG); term(5, 0, 0); }
                if (c == 5) { term(2, 5, NEG ^ smask); term(3, 2, smask); term(4, 4, NEG ^ smask); term(5, 1, smask); }
            }
        }
        my_mt = mt;
        my_q = q;
    }
    __syncthreads();  // every warp is done with Ms: it now takes the output rows
    if (my_mt >= 0) {
        float *out = Ms + (size_t)my_q * 2 * planes;  // [b][i][c] complex
#pragma unroll
        for (int o = 0; o < 6; ++o)
#pragma unroll
            for (int n = 0; n < NT; ++n)
#pragma unroll
                for (int f = 0; f < 4; ++f) {
                    const int i = my_mt * 16 + gr + (f >= 2 ? 8 : 0);
                    const int b = n * 8 + 2 * gc + (f & 1);
                    if (i < L && b < B) out[((b * L + i) * 3 + (o >> 1)) * 2 + (o & 1)] = acc[o][n][f];
                }
    }
    __syncthreads();
    for (int pos = 0; pos < npos; ++pos) {
        float2 *dst = sk + (size_t)(pos ? p2 : p1) * planes;
        if (planes % 2 == 0) {  // both ends 16-byte aligned
            const float4 *src = reinterpret_cast<const float4 *>(Ms + (size_t)pos * 2 * planes);
            for (int e = tid; e < planes / 2; e += kGemmThreads) reinterpret_cast<float4 *>(dst)[e] = src[e];
        } else {
            const float2 *src = reinterpret_cast<const float2 *>(Ms + (size_t)pos * 2 * planes);
            for (int e = tid; e < planes; e += kGemmThreads) dst[e] = src[e];
        }
    }
}

size_t tc_smem_bytes(int L, int npairs) {
    const int Lp = pad16(L), S = gemm_stride(Lp);
    return (size_t)(ub_entry(L) + 2 * 6 * 16 * S + 2 * Lp) * sizeof(float);
}

}  // namespace demag

namespace demag {

cudaError_t launch_contract_gemm(const ApplyArgs &a, bool tensor_cores, cudaStream_t st) {
    const int Py = 1 << a.log2Py, Qy = Py / 2 + 1, Kx = a.kx_count ? a.kx_count : (1 << a.log2Px) / 2 + 1;
    const size_t smem = gemm_smem_bytes(a.L, a.B);
    cudaError_t e;
    dim3 grid(Kx, Qy);
    if (tensor_cores && a.B <= 16) {
        const size_t sm = tc_smem_bytes(a.L, a.npairs);
        if (a.B <= 8) {
            if ((e = cudaFuncSetAttribute(k_contract_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)) !=
                cudaSuccess)
                return e;
            k_contract_tc<1><<<grid, kGemmThreads, sm, st>>>((float2 *)a.spec2, (const float *)a.tensor,
                                                             (const float *)a.ratio, a.L, a.B, a.log2Py,
                                                             a.npairs);
        } else {
            if ((e = cudaFuncSetAttribute(k_contract_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)) !=
                cudaSuccess)
                return e;
            k_contract_tc<2><<<grid, kGemmThreads, sm, st>>>((float2 *)a.spec2, (const float *)a.tensor,
                                                             (const float *)a.ratio, a.L, a.B, a.log2Py,
                                                             a.npairs);
        }
    } else if (tensor_cores) {
        if ((e = cudaFuncSetAttribute(k_contract_gemm<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem)) != cudaSuccess)
            return e;
        k_contract_gemm<true><<<grid, kGemmThreads, smem, st>>>((float2 *)a.spec2, (const float *)a.tensor,
                                                               (const float *)a.ratio, a.L, a.B, a.log2Py,
                                                               a.npairs);
    } else {
        if ((e = cudaFuncSetAttribute(k_contract_gemm<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem)) != cudaSuccess)
            return e;
        k_contract_gemm<false><<<grid, kGemmThreads, smem, st>>>((float2 *)a.spec2, (const float *)a.tensor,
                                                                (const float *)a.ratio, a.L, a.B, a.log2Py,
                                                                a.npairs);
    }
    return cudaGetLastError();
}

}  // namespace demag
