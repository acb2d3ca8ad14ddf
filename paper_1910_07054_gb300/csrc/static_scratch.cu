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
// reuses the same array; the kernels overwrite all of it that they read (the
// small tables are recomputed on the device by every call), so nothing needs
// clearing, but two calls whose GPU work overlaps (different streams, or
// different host threads) race on it.  The call makes no host-to-device copy.
#include <atomic>
#include <cmath>
#include <cstdint>
#include <string>

#include "fft.cuh"
#include "internal.h"
#include "layout.cuh"

namespace demag {

constexpr size_t kStaticScratchBytes = 32u << 20;
constexpr int kStaticMaxLayers = 256;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// Device address of g_static_scratch for each device (host code only sees a
// host-side stand-in under that name, never a usable device address).  Looked
// up once per device; concurrent first calls store the same value.  A
// cudaDeviceReset unloads the module, so the entry of that device is cleared
// whenever a call on it fails, and the next call looks the address up again.
static std::atomic<void *> g_scratch_addr[64];

static demag_status scratch_address(int dev, void **out) {
    void *p = g_scratch_addr[dev].load(std::memory_order_acquire);
    if (!p) {
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(static scratch)");
        g_scratch_addr[dev].store(p, std::memory_order_release);
    }
    *out = p;
    return DEMAG_OK;
}

static size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

static int log2_ceil_min4(int v) {
    int l = 0;
    while ((1 << l) < v) ++l;
    return l < 2 ? 2 : l;
}

// The layer thicknesses travel as a kernel parameter (no host copy).
struct StaticThickness {
    double t[kStaticMaxLayers];
};

// Twiddles exp(-2 pi i k / N) for Px and Py and the reciprocity ratios
// t_j / t_i, written into the fixed array by the device itself.
template <typename T>
__global__ void k_static_tables(typename cpx_of<T>::type *twx, int log2Px, typename cpx_of<T>::type *twy,
                                int log2Py, T *ratio, int L, StaticThickness th) {
    const int nx2 = (1 << log2Px) / 2, ny2 = (1 << log2Py) / 2;
    const int total = nx2 + ny2 + L * L;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < total; k += gridDim.x * blockDim.x) {
        if (k < nx2 + ny2) {
            const bool x = k < nx2;
            const int q = x ? k : k - nx2;
            double s, c;
            sincospi(2.0 * (double)q / (double)(1 << (x ? log2Px : log2Py)), &s, &c);
            typename cpx_of<T>::type w;
            w.x = (T)c;
            w.y = (T)(-s);
            (x ? twx : twy)[q] = w;
        } else {
            const int r = k - nx2 - ny2, i = r / L, j = r % L;
            ratio[r] = (T)(th.t[j] / th.t[i]);
        }
    }
}

}  // namespace demag

using namespace demag;

extern "C" demag_status demag_apply_static(const void *tensor, size_t tensor_bytes, const double *thickness,
                                           int nx, int ny, int L, int precision, const void *m, double Ms,
                                           void *H, int B, void *stream) {
    if (!tensor || !thickness || !m || !H) return fail(DEMAG_EINVAL, "a pointer argument is NULL");
    if (m == H) return fail(DEMAG_EINVAL, "H must not alias m");
    if (reinterpret_cast<uintptr_t>(tensor) % 16 != 0)
        return fail(DEMAG_EINVAL, "tensor must be 16-byte aligned");
    if (nx < 1 || ny < 1 || L < 1 || B < 1) return fail(DEMAG_EINVAL, "nx, ny, L and B must be >= 1");
    if (nx > 2048 || ny > 2048 || L > kStaticMaxLayers)
        return fail(DEMAG_EUNSUPPORTED, "size above the library limits");
    if (precision != DEMAG_PREC_FP64 && precision != DEMAG_PREC_FP32)
        return fail(DEMAG_EINVAL, "unknown precision");
    if (!std::isfinite(Ms)) return fail(DEMAG_EINVAL, "Ms must be finite");
    StaticThickness th;
    for (int l = 0; l < L; ++l) {
        if (!(std::isfinite(thickness[l]) && thickness[l] > 0))
            return fail(DEMAG_EINVAL, "thickness[" + std::to_string(l) + "] must be finite and > 0");
        th.t[l] = thickness[l];
    }
    if ((long long)B * L * 3 > 65535) return fail(DEMAG_EUNSUPPORTED, "B * L * 3 must be <= 65535");
    const bool fp64 = precision == DEMAG_PREC_FP64;
    const int log2Px = log2_ceil_min4(2 * nx), log2Py = log2_ceil_min4(2 * ny);
    if (L > fused_max_layers(fp64, log2Py))
        return fail(DEMAG_EUNSUPPORTED, "layer count above the fused contraction limit for this grid");
    const size_t real = fp64 ? 8 : 4, cpx = 2 * real;
    const int Kx = (1 << log2Px) / 2 + 1;
    const int npairs = L * (L + 1) / 2, QyS = tensor_row(log2Py, fp64);
    const size_t spec = align256((size_t)B * L * 3 * Kx * ny * cpx);
    const size_t twx = align256((size_t)(1 << log2Px) / 2 * cpx);
    const size_t twy = align256((size_t)(1 << log2Py) / 2 * cpx);
    const size_t rat = align256((size_t)L * L * real);
    const size_t need = spec + twx + twy + rat;
    if (need > kStaticScratchBytes)
        return fail(DEMAG_EUNSUPPORTED, "demag_apply_static needs " + std::to_string(need) +
                                            " bytes of scratch; the fixed array holds " +
                                            std::to_string(kStaticScratchBytes));
    const size_t want = (size_t)Kx * npairs * 6 * QyS * real;
    if (tensor_bytes != want)
        return fail(DEMAG_EINVAL, "tensor holds " + std::to_string(tensor_bytes) + " bytes; a plan of this grid, "
                                  "layer count and precision stores " + std::to_string(want));
    int dev = 0;
    DEMAG_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(DEMAG_EUNSUPPORTED, "device index above 63");
    void *base = nullptr;
    demag_status rc = scratch_address(dev, &base);
    if (rc != DEMAG_OK) return rc;
    unsigned char *b = (unsigned char *)base;
    cudaStream_t st = (cudaStream_t)stream;

    // twiddles and t_j / t_i, computed on the device into the fixed array
    const int ntab = (1 << log2Px) / 2 + (1 << log2Py) / 2 + L * L;
    const int tgrid = (ntab + 255) / 256 < 64 ? (ntab + 255) / 256 : 64;
    if (fp64)
        k_static_tables<double><<<tgrid, 256, 0, st>>>((double2 *)(b + spec), log2Px, (double2 *)(b + spec + twx),
                                                       log2Py, (double *)(b + spec + twx + twy), L, th);
    else
        k_static_tables<float><<<tgrid, 256, 0, st>>>((float2 *)(b + spec), log2Px, (float2 *)(b + spec + twx),
                                                      log2Py, (float *)(b + spec + twx + twy), L, th);
    cudaError_t e = cudaGetLastError();

    ApplyArgs a;
    a.nx = nx;
    a.ny = ny;
    a.L = L;
    a.B = B;
    a.log2Px = log2Px;
    a.log2Py = log2Py;
    a.npairs = npairs;
    a.QyS = QyS;
    a.natural = cols512_supported(log2Py, L, fp64) ? 1 : 0;
    a.tensor = tensor;
    a.ratio = b + spec + twx + twy;
    a.twx = b + spec;
    a.twy = b + spec + twx;
    a.log2twx = log2Px;
    a.log2twy = log2Py;
    a.spec = b;
    a.Ms = Ms;
    if (e == cudaSuccess) e = launch_apply(a, m, H, fp64, st);
    if (e != cudaSuccess) {
        g_scratch_addr[dev].store(nullptr, std::memory_order_release);
        return cuda_fail(e, "demag_apply_static kernels");
    }
    return DEMAG_OK;
}
