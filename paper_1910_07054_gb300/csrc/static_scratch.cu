// demag_apply_static: the demag_apply kernels with their spectrum workspace,
// twiddle tables and reciprocity ratios placed in a fixed, file-scope device
// array instead of memory from cudaMalloc.
//
// Who needs it: callers that must not allocate device memory while they run,
// for example code inside a host framework whose own allocator has reserved the
// GPU's memory (a cudaMalloc there can fail or fragment the framework's pool),
// or a time-critical loop that cannot afford the device-wide synchronisation a
// cudaMalloc/cudaFree may imply.  Such a caller prepares the Fourier tensor once
// (for example with demag_plan_create + demag_plan_tensor into memory it owns,
// at a point where allocation is allowed) and then only passes device pointers.
//
// Limits and sharing: the array holds kStaticScratchBytes (32 MiB) on every GPU
// that loads this library, for the life of the process.  Every call on a device
// reuses the same array; the kernels overwrite all of it that they read, so
// nothing needs clearing, but two calls whose GPU work overlaps (different
// streams, or different host threads) race on it.
#include <cmath>
#include <cstdint>
#include <string>
#include <vector>

#include "internal.h"
#include "layout.cuh"

namespace demag {

constexpr size_t kStaticScratchBytes = 32u << 20;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// Device address of g_static_scratch for each device (host code only sees a
// host-side stand-in under that name, never a usable device address).
static void *g_scratch_addr[64] = {};

static demag_status scratch_address(void **out) {
    int dev = 0;
    DEMAG_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(DEMAG_EUNSUPPORTED, "device index above 63");
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(static scratch)");
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return DEMAG_OK;
}

static size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

template <typename C>
static void host_twiddles(int log2n, std::vector<C> &tw) {
    const int N = 1 << log2n;
    tw.assign(N / 2, C{});
    const double pi = 3.14159265358979323846;
    for (int k = 0; k < N / 2; ++k) {
        const double ang = 2.0 * pi * (double)k / (double)N;
        tw[k].x = std::cos(ang);
        tw[k].y = -std::sin(ang);
    }
}

static int log2_ceil_min4(int v) {
    int l = 0;
    while ((1 << l) < v) ++l;
    return l < 2 ? 2 : l;
}

}  // namespace demag

using namespace demag;

extern "C" demag_status demag_apply_static(const void *tensor, const double *thickness, int nx,
                                           int ny, int L, int precision, const void *m, double Ms,
                                           void *H, int B, void *stream) {
    if (!tensor || !thickness || !m || !H) return fail(DEMAG_EINVAL, "a pointer argument is NULL");
    if (m == H) return fail(DEMAG_EINVAL, "H must not alias m");
    if (reinterpret_cast<uintptr_t>(tensor) % 16 != 0)
        return fail(DEMAG_EINVAL, "tensor must be 16-byte aligned");
    if (nx < 1 || ny < 1 || L < 1 || B < 1) return fail(DEMAG_EINVAL, "nx, ny, L and B must be >= 1");
    if (nx > 2048 || ny > 2048 || L > 256) return fail(DEMAG_EUNSUPPORTED, "size above the library limits");
    if (precision != DEMAG_PREC_FP64 && precision != DEMAG_PREC_FP32)
        return fail(DEMAG_EINVAL, "unknown precision");
    if (!std::isfinite(Ms)) return fail(DEMAG_EINVAL, "Ms must be finite");
    for (int l = 0; l < L; ++l)
        if (!(std::isfinite(thickness[l]) && thickness[l] > 0))
            return fail(DEMAG_EINVAL, "thickness[" + std::to_string(l) + "] must be finite and > 0");
    if ((long long)B * L * 3 > 65535) return fail(DEMAG_EUNSUPPORTED, "B * L * 3 must be <= 65535");
    const bool fp64 = precision == DEMAG_PREC_FP64;
    const int log2Px = log2_ceil_min4(2 * nx), log2Py = log2_ceil_min4(2 * ny);
    if (L > fused_max_layers(fp64, log2Py))
        return fail(DEMAG_EUNSUPPORTED, "layer count above the fused contraction limit for this grid");
    const size_t real = fp64 ? 8 : 4, cpx = 2 * real;
    const int Kx = (1 << log2Px) / 2 + 1;
    const size_t spec = align256((size_t)B * L * 3 * Kx * ny * cpx);
    const size_t twx = align256((size_t)(1 << log2Px) / 2 * cpx);
    const size_t twy = align256((size_t)(1 << log2Py) / 2 * cpx);
    const size_t rat = align256((size_t)L * L * real);
    const size_t need = spec + twx + twy + rat;
    if (need > kStaticScratchBytes)
        return fail(DEMAG_EUNSUPPORTED, "demag_apply_static needs " + std::to_string(need) +
                                            " bytes of scratch; the fixed array holds " +
                                            std::to_string(kStaticScratchBytes));
    void *base = nullptr;
    demag_status rc = scratch_address(&base);
    if (rc != DEMAG_OK) return rc;
    unsigned char *b = (unsigned char *)base;
    cudaStream_t st = (cudaStream_t)stream;

    // twiddles and t_j / t_i, copied from the host into the fixed array
    std::vector<double> r64((size_t)L * L);
    for (int i = 0; i < L; ++i)
        for (int j = 0; j < L; ++j) r64[(size_t)i * L + j] = thickness[j] / thickness[i];
    std::vector<double2> tx64, ty64;
    host_twiddles(log2Px, tx64);
    host_twiddles(log2Py, ty64);
    if (fp64) {
        DEMAG_CUDA(cudaMemcpyAsync(b + spec, tx64.data(), tx64.size() * 16, cudaMemcpyHostToDevice, st));
        DEMAG_CUDA(cudaMemcpyAsync(b + spec + twx, ty64.data(), ty64.size() * 16, cudaMemcpyHostToDevice, st));
        DEMAG_CUDA(cudaMemcpyAsync(b + spec + twx + twy, r64.data(), r64.size() * 8, cudaMemcpyHostToDevice, st));
    } else {
        std::vector<float2> tx32(tx64.size()), ty32(ty64.size());
        std::vector<float> r32(r64.begin(), r64.end());
        for (size_t k = 0; k < tx64.size(); ++k) tx32[k] = make_float2((float)tx64[k].x, (float)tx64[k].y);
        for (size_t k = 0; k < ty64.size(); ++k) ty32[k] = make_float2((float)ty64[k].x, (float)ty64[k].y);
        DEMAG_CUDA(cudaMemcpyAsync(b + spec, tx32.data(), tx32.size() * 8, cudaMemcpyHostToDevice, st));
        DEMAG_CUDA(cudaMemcpyAsync(b + spec + twx, ty32.data(), ty32.size() * 8, cudaMemcpyHostToDevice, st));
        DEMAG_CUDA(cudaMemcpyAsync(b + spec + twx + twy, r32.data(), r32.size() * 4, cudaMemcpyHostToDevice, st));
    }

    ApplyArgs a;
    a.nx = nx;
    a.ny = ny;
    a.L = L;
    a.B = B;
    a.log2Px = log2Px;
    a.log2Py = log2Py;
    a.npairs = L * (L + 1) / 2;
    a.QyS = tensor_row(log2Py, fp64);
    a.natural = cols512_supported(log2Py, L, fp64) ? 1 : 0;
    a.tensor = tensor;
    a.ratio = b + spec + twx + twy;
    a.twx = b + spec;
    a.twy = b + spec + twx;
    a.log2twx = log2Px;
    a.log2twy = log2Py;
    a.spec = b;
    a.Ms = Ms;
    cudaError_t e = launch_apply(a, m, H, fp64, st);
    if (e != cudaSuccess) return cuda_fail(e, "demag_apply_static kernels");
    return DEMAG_OK;
}
