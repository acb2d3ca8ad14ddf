// Block-sparse compression of a dense-product plan's tensor (layout.cuh), of
// floats or of BF16 split pairs.
//
// In the in-plane Fourier domain the interaction of two layers decays roughly
// like exp(-|k| Z) with their distance Z (Sec. 3.2: the cost of the hybrid is
// the O(n_z^2) layer pairs), so at high in-plane frequencies most 8 x 8 layer
// blocks of distant layers hold values far below the field's float
// resolution.  compress_tensor drops, entry by entry, every block none of
// whose values exceeds tol times its component's largest value in the whole
// tensor, and stores the remaining blocks of an
// entry contiguously: [component][kept block, in block order][64 floats].  A
// 64-bit mask per entry (bit b: block b kept) and the entry's first block
// (units of 64 floats) let the contraction find block b of component c at
// first + (c * kept + rank(b)) with rank(b) the number of kept blocks before b.
#include <cstdint>
#include <vector>

#include "internal.h"
#include "layout.cuh"

namespace demag {

namespace {

// |value| of a stored slot: a float, or (packed) a BF16 split pair hi << 16 | lo
// standing for hi + lo.
__device__ __forceinline__ float slot_abs(float x, bool packed) {
    if (!packed) return fabsf(x);
    const uint32_t w = __float_as_uint(x);
    return fabsf(__uint_as_float(w & 0xFFFF0000u) + __uint_as_float(w << 16));
}

// Largest |value| of each component over the whole tensor, as float bits
// (non-negative floats order like their bit patterns).  Rows are (entry,
// component); the grid is a multiple of 6 blocks, so each block walks rows of
// one component and adds one atomic at the end.
constexpr int kMaxGrid = 6 * 202;

__global__ void k_component_max(const float *__restrict__ t, size_t nent, int row, bool packed,
                                unsigned *__restrict__ cmax) {
    __shared__ unsigned part[32];
    unsigned v = 0;
    for (size_t rr = blockIdx.x; rr < nent * 6; rr += gridDim.x) {
        const float *src = t + rr * (size_t)row;
        for (int i = threadIdx.x; i < row; i += blockDim.x) v = max(v, __float_as_uint(slot_abs(src[i], packed)));
    }
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) v = max(v, part[w]);
        if (v) atomicMax(&cmax[blockIdx.x % 6], v);
    }
}

// One warp per entry: the kept-block mask and count.  A block is kept when any
// of its 6 x 64 values exceeds tol times its component's maximum.
__global__ void k_block_mask(const float *__restrict__ t, size_t nent, int row, int nblk, bool packed,
                             const unsigned *__restrict__ cmax, float tol, unsigned long long *__restrict__ mask,
                             int *__restrict__ kept) {
    const size_t e = (size_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (e >= nent) return;
    float thr[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) thr[c] = tol * __uint_as_float(cmax[c]);
    const float *te = t + e * 6 * (size_t)row;
    unsigned long long m = 0;
    for (int b = 0; b < nblk; ++b) {
        bool keep = false;
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            const float *blk = te + (size_t)c * row + 64 * b;
            keep |= slot_abs(blk[lane], packed) > thr[c] || slot_abs(blk[lane + 32], packed) > thr[c];
        }
        if (__any_sync(0xffffffffu, keep)) m |= 1ull << b;
    }
    if (lane == 0) {
        mask[e] = m;
        kept[e] = __popcll(m);
    }
}

// One warp per entry: the kept blocks to their compact places.
__global__ void k_compact(const float *__restrict__ t, size_t nent, int row, int nblk,
                          const unsigned long long *__restrict__ mask, const unsigned *__restrict__ first,
                          float *__restrict__ out) {
    const size_t e = (size_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (e >= nent) return;
    const unsigned long long m = mask[e];
    const int kept = __popcll(m);
    const float *te = t + e * 6 * (size_t)row;
    float *oe = out + (size_t)first[e] * 64;
    int rank = 0;
    for (int b = 0; b < nblk; ++b) {
        if (!((m >> b) & 1)) continue;
        for (int c = 0; c < 6; ++c) {
            const float *src = te + (size_t)c * row + 64 * b;
            float *dst = oe + ((size_t)c * kept + rank) * 64;
            dst[lane] = src[lane];
            dst[lane + 32] = src[lane + 32];
        }
        ++rank;
    }
}

}  // namespace

cudaError_t compress_tensor(const float *tensor, size_t nent, int L, bool packed, double tol, float **out,
                            size_t *out_bytes, unsigned long long **mask, unsigned **first, cudaStream_t st) {
    *out = nullptr;
    *mask = nullptr;
    *first = nullptr;
    *out_bytes = 0;
    const int nb = ub_nb(L), row = ub_row(L), nblk = nb * (nb + 1) / 2;
    if (nblk > 64 || nent == 0 || nent > 0xFFFFFFFFull / (6ull * nblk)) return cudaErrorInvalidValue;
    unsigned *d_cmax = nullptr;
    int *d_kept = nullptr;
    unsigned long long *d_mask = nullptr;
    unsigned *d_first = nullptr;
    float *d_out = nullptr;
    cudaError_t e = cudaSuccess;
    auto fail = [&](cudaError_t err) {
        cudaFree(d_cmax);
        cudaFree(d_kept);
        cudaFree(d_mask);
        cudaFree(d_first);
        cudaFree(d_out);
        return err;
    };
    if ((e = cudaMalloc(&d_cmax, 6 * sizeof(unsigned))) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&d_kept, nent * sizeof(int))) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&d_mask, nent * sizeof(unsigned long long))) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&d_first, nent * sizeof(unsigned))) != cudaSuccess) return fail(e);
    if ((e = cudaMemsetAsync(d_cmax, 0, 6 * sizeof(unsigned), st)) != cudaSuccess) return fail(e);
    k_component_max<<<kMaxGrid, 256, 0, st>>>(tensor, nent, row, packed, d_cmax);
    const unsigned wgrid = (unsigned)((nent + 7) / 8);  // 8 warps per block
    k_block_mask<<<wgrid, 256, 0, st>>>(tensor, nent, row, nblk, packed, d_cmax, (float)tol, d_mask, d_kept);
    if ((e = cudaGetLastError()) != cudaSuccess) return fail(e);
    // first block of each entry: exclusive sum of 6 * kept, on the host
    std::vector<int> h_kept(nent);
    std::vector<unsigned> h_first(nent);
    if ((e = cudaMemcpyAsync(h_kept.data(), d_kept, nent * sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return fail(e);
    unsigned long long acc = 0;
    for (size_t i = 0; i < nent; ++i) {
        h_first[i] = (unsigned)acc;
        acc += 6ull * (unsigned)h_kept[i];
    }
    const size_t bytes = (size_t)acc * 64 * sizeof(float);
    if ((e = cudaMalloc(&d_out, bytes ? bytes : 64 * sizeof(float))) != cudaSuccess) return fail(e);
    if ((e = cudaMemcpyAsync(d_first, h_first.data(), nent * sizeof(unsigned), cudaMemcpyHostToDevice, st)) !=
        cudaSuccess)
        return fail(e);
    k_compact<<<wgrid, 256, 0, st>>>(tensor, nent, row, nblk, d_mask, d_first, d_out);
    if ((e = cudaGetLastError()) != cudaSuccess || (e = cudaStreamSynchronize(st)) != cudaSuccess) return fail(e);
    cudaFree(d_cmax);
    cudaFree(d_kept);
    *out = d_out;
    *out_bytes = bytes;
    *mask = d_mask;
    *first = d_first;
    return cudaSuccess;
}

}  // namespace demag
