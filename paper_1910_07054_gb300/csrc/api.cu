// C ABI of libdemag: plan lifecycle, argument checks and error reporting.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <new>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "internal.h"
#include "nvtx.cuh"
#include "mbar.cuh"
#include "layout.cuh"

namespace demag {

static thread_local std::string g_last_error;

demag_status fail(demag_status st, const std::string &msg) {
    g_last_error = msg;
    return st;
}

demag_status cuda_fail(cudaError_t err, const char *what) {
    std::string m = std::string(what) + ": " + cudaGetErrorName(err) + " (" + cudaGetErrorString(err) + ")";
    g_last_error = m;
    return err == cudaErrorMemoryAllocation ? DEMAG_ENOMEM : DEMAG_ECUDA;
}

static int ilog2_ceil(int v) {
    int l = 0;
    while ((1 << l) < v) ++l;
    return l;
}

// exp(-2 pi i k / N) for k < N/2, N = 2^log2n
template <typename C>
static std::vector<C> twiddles(int log2n) {
    const int N = 1 << log2n;
    std::vector<C> tw(N / 2 > 0 ? N / 2 : 1);
    const double pi = 3.14159265358979323846;
    for (int k = 0; k < N / 2; ++k) {
        const double ang = 2.0 * pi * (double)k / (double)N;
        tw[k].x = std::cos(ang);
        tw[k].y = -std::sin(ang);
    }
    if (N / 2 == 0) tw[0] = C{1, 0};
    return tw;
}

static void free_plan(demag_plan *p) {
    if (!p) return;
    cudaFree(p->d_tensor);
    cudaFree(p->d_ratio);
    cudaFree(p->d_twx);
    cudaFree(p->d_twy);
    cudaFree(p->d_spec);
    cudaFree(p->d_stage_m);
    cudaFree(p->d_stage_H);
    cudaFree(p->d_stage2_m);
    cudaFree(p->d_stage2_H);
    cudaFree(p->d_spec2);
    cudaFree(p->d_tscale);
    cudaFree(p->d_dtensor);
    cudaFree(p->d_dH);
    cudaFree(p->d_dot);
    cudaFree(p->d_twz);
    cudaFree(p->d_bmask);
    cudaFree(p->d_bfirst);
    if (p->h_timeouts) cudaFreeHost(p->h_timeouts);
    for (auto &set : p->pipe_ev)
        for (cudaEvent_t ev : set)
            if (ev) cudaEventDestroy(ev);
    if (p->copy_st) cudaStreamDestroy(p->copy_st);
    if (p->copy_st2) cudaStreamDestroy(p->copy_st2);
    delete p;
}

// ---- bounded-wait timeouts ------------------------------------------------
// The kernels that stream the tensor with asynchronous copies count every
// bounded wait that gave up in two device counters that only grow.  The host
// remembers, per device, how much of each count it has already reported; a
// synchronising entry point (or demag_wait_timeouts) reports the rest.
static std::mutex g_timeout_mu;
static unsigned g_timeouts_seen[64][2];

// Counts new since the last report on this device; updates the record.
static unsigned long long take_new_timeouts(int dev, const unsigned *now) {
    if (dev < 0 || dev >= 64) return 0;
    std::lock_guard<std::mutex> lock(g_timeout_mu);
    unsigned long long n = 0;
    for (int k = 0; k < 2; ++k)
        if (now[k] > g_timeouts_seen[dev][k]) {
            n += now[k] - g_timeouts_seen[dev][k];
            g_timeouts_seen[dev][k] = now[k];
        }
    return n;
}

// Enqueues on `st` the copies of both counters into the plan's pinned words.
static cudaError_t enqueue_timeout_read(demag_plan *p, cudaStream_t st) {
    cudaError_t e = read_wait_timeouts(&p->h_timeouts[0], st);
    if (e == cudaSuccess) e = read_tc_timeouts(&p->h_timeouts[1], st);
    return e;
}

// After `st` was synchronised behind enqueue_timeout_read: DEMAG_ECUDA if a
// bounded wait gave up since the counts were last reported.
static demag_status timeout_status(demag_plan *p, const char *where) {
    const unsigned long long n = take_new_timeouts(p->device, p->h_timeouts);
    if (n == 0) return DEMAG_OK;
    return fail(DEMAG_ECUDA, std::string(where) + ": " + std::to_string(n) +
                                 " bounded device wait(s) gave up (an asynchronous tensor copy did not "
                                 "complete within the limit); the result is invalid");
}

// Device allocation that records the failure.
// Host-side fault injection (demag_debug_fail_alloc): allocations left before
// one is refused; negative = off.
static int g_alloc_fail_after = -1;

static demag_status dalloc(void **ptr, size_t bytes, const char *what) {
    if (g_alloc_fail_after >= 0 && g_alloc_fail_after-- == 0) {
        *ptr = nullptr;
        return fail(DEMAG_ENOMEM, std::string("cudaMalloc(") + what + "): refused by demag_debug_fail_alloc");
    }
    cudaError_t e = cudaMalloc(ptr, bytes);
    if (e != cudaSuccess) {
        *ptr = nullptr;
        cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? DEMAG_ENOMEM : DEMAG_ECUDA,
                    std::string("cudaMalloc(") + what + ", " + std::to_string(bytes) + " bytes): " +
                        cudaGetErrorString(e));
    }
    return DEMAG_OK;
}

#define DEMAG_TRY(expr)                       \
    do {                                      \
        demag_status s_ = (expr);             \
        if (s_ != DEMAG_OK) return s_;        \
    } while (0)

// Builds the plan tensor (layer < 0: pairs i <= j of N) or the derivative
// tensor d N / d t_layer (all L*L pairs) into dst; with zoffsets, the
// 2D-transformed kernels of the pairs (r, 0), r = 0..L-1, in double and
// natural folded-ky order [Kx][L][6][QyS of double] (equidistant plans).
static demag_status build_tensor(demag_plan *p, cudaStream_t st, int layer, void *dst, bool zoffsets = false) {
    const int L = p->L;
    std::vector<int> pi, pj;
    if (zoffsets) {
        for (int r = 0; r < L; ++r) {
            pi.push_back(r);
            pj.push_back(0);
        }
    } else {
        for (int i = 0; i < L; ++i)
            for (int j = i; j < L; ++j) {
                pi.push_back(i);
                pj.push_back(j);
            }
    }
    const int npairs = zoffsets ? L : (layer < 0 ? p->npairs : L * L);
    // the layout of dense-product plans: 1 floats, 2 BF16 split pairs
    const int blocked = !zoffsets && layer < 0 ? (p->umajor ? (p->packed ? 2 : 1) : 0) : 0;
    std::vector<double> z(L + 1, 0.0);
    for (int l = 0; l < L; ++l) z[l + 1] = z[l] + p->thickness[l];

    const int Px = 1 << p->log2Px, Py = 1 << p->log2Py;
    // Float plans take the values (evaluated in double) through float planes
    // and float 2D FFTs: the transform's rounding (~1e-7 of the spectrum) is
    // that of the float tensor they store.  Double plans and the z-offset
    // kernels of the equidistant method stay in double.
    const bool f32 = p->precision != DEMAG_PREC_FP64 && !zoffsets;
    const size_t cpx = f32 ? sizeof(float2) : sizeof(double2);
    const size_t plane_bytes = (size_t)3 * Px * Py * cpx;
    // pairs per chunk: bounded workspace (~4 GB)
    int chunk = 1;
    {
        size_t budget = (size_t)4 << 30;
        size_t c = budget / plane_bytes;
        if (c < 1) c = 1;
        if (c > (size_t)npairs) c = npairs;
        chunk = (int)c;
    }
    int *d_pi = nullptr, *d_pj = nullptr;
    double *d_z = nullptr, *d_th = nullptr;
    void *planes = nullptr, *twx = nullptr, *twy = nullptr;
    demag_status rc = DEMAG_OK;
    auto cleanup = [&]() {
        cudaFree(d_pi);
        cudaFree(d_pj);
        cudaFree(d_z);
        cudaFree(d_th);
        cudaFree(planes);
        cudaFree(twx);
        cudaFree(twy);
    };
    do {
        if ((rc = dalloc((void **)&d_pi, pi.size() * sizeof(int), "pair list")) != DEMAG_OK) break;
        if ((rc = dalloc((void **)&d_pj, pj.size() * sizeof(int), "pair list")) != DEMAG_OK) break;
        if ((rc = dalloc((void **)&d_z, z.size() * sizeof(double), "interfaces")) != DEMAG_OK) break;
        if ((rc = dalloc((void **)&d_th, L * sizeof(double), "thicknesses")) != DEMAG_OK) break;
        if ((rc = dalloc(&planes, plane_bytes * chunk, "tensor planes")) != DEMAG_OK) break;
        auto htwx = twiddles<double2>(p->log2Px), htwy = twiddles<double2>(p->log2Py);
        std::vector<float2> ftwx(htwx.size()), ftwy(htwy.size());
        for (size_t k = 0; k < htwx.size(); ++k) ftwx[k] = make_float2((float)htwx[k].x, (float)htwx[k].y);
        for (size_t k = 0; k < htwy.size(); ++k) ftwy[k] = make_float2((float)htwy[k].x, (float)htwy[k].y);
        const void *stwx = f32 ? (const void *)ftwx.data() : (const void *)htwx.data();
        const void *stwy = f32 ? (const void *)ftwy.data() : (const void *)htwy.data();
        if ((rc = dalloc(&twx, htwx.size() * cpx, "twiddles")) != DEMAG_OK) break;
        if ((rc = dalloc(&twy, htwy.size() * cpx, "twiddles")) != DEMAG_OK) break;
        cudaError_t e;
        if ((e = cudaMemcpyAsync(d_pi, pi.data(), pi.size() * sizeof(int), cudaMemcpyHostToDevice, st)) ||
            (e = cudaMemcpyAsync(d_pj, pj.data(), pj.size() * sizeof(int), cudaMemcpyHostToDevice, st)) ||
            (e = cudaMemcpyAsync(d_z, z.data(), z.size() * sizeof(double), cudaMemcpyHostToDevice, st)) ||
            (e = cudaMemcpyAsync(d_th, p->thickness.data(), L * sizeof(double), cudaMemcpyHostToDevice, st)) ||
            (e = cudaMemcpyAsync(twx, stwx, htwx.size() * cpx, cudaMemcpyHostToDevice, st)) ||
            (e = cudaMemcpyAsync(twy, stwy, htwy.size() * cpx, cudaMemcpyHostToDevice, st))) {
            rc = cuda_fail(e, "cudaMemcpyAsync(tensor set-up)");
            break;
        }
        // the blocked layout writes only the layers that exist: zero the rest
        if (blocked && (e = cudaMemsetAsync(dst, 0, p->tensor_bytes, st)) != cudaSuccess) {
            rc = cuda_fail(e, "cudaMemsetAsync(tensor)");
            break;
        }
        for (int p0 = 0; p0 < npairs && rc == DEMAG_OK; p0 += chunk) {
            const int np = std::min(chunk, npairs - p0);
            if ((e = cudaMemsetAsync(planes, 0, plane_bytes * np, st)) != cudaSuccess) {
                rc = cuda_fail(e, "cudaMemsetAsync(tensor planes)");
                break;
            }
            e = layer < 0 ? launch_kernel_planes(planes, f32, p0, np, d_pi, d_pj, p->nx, p->ny, p->dx, p->dy,
                                                 p->log2Px, p->log2Py, d_z, d_th, st,
                                                 p->precision != DEMAG_PREC_FP64)
                          : launch_dkernel_planes(planes, f32, p0, np, L, layer, p->nx, p->ny, p->dx, p->dy,
                                                  p->log2Px, p->log2Py, d_z, d_th, st);
            if (e != cudaSuccess) {
                rc = cuda_fail(e, "tensor evaluation kernel");
                break;
            }
            if ((e = launch_fft2_planes(planes, f32, 3 * np, p->log2Px, p->log2Py, twx, p->log2Px, twy,
                                        p->log2Py, st)) != cudaSuccess) {
                rc = cuda_fail(e, "tensor FFT kernels");
                break;
            }
            if ((e = launch_extract_tensor(planes, f32, p0, np, npairs, p->log2Px, p->log2Py,
                                           zoffsets ? tensor_row(p->log2Py, true) : p->QyS, dst,
                                           zoffsets || p->precision == DEMAG_PREC_FP64, st, blocked,
                                           zoffsets ? 1 : p->natural, d_pi, d_pj, d_th, L)) != cudaSuccess) {
                rc = cuda_fail(e, "tensor extraction kernel");
                break;
            }
        }
        if (rc != DEMAG_OK) break;
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) rc = cuda_fail(e, "tensor build");
    } while (0);
    cleanup();
    return rc;
}

// sum_i a[i] * b[i] accumulated in double into *out (zeroed beforehand)
template <typename T>
__global__ void k_dot(const T *__restrict__ a, const T *__restrict__ b, size_t n, double *out) {
    double acc = 0.0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        acc += (double)a[i] * (double)b[i];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    __shared__ double part[32];
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        acc = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (threadIdx.x == 0) atomicAdd(out, acc);
    }
}

static demag_status ensure_dtensor(demag_plan *p, int layer, cudaStream_t st) {
    if (p->dlayer == layer) return DEMAG_OK;
    const size_t real = p->precision == DEMAG_PREC_FP64 ? 8 : 4;
    const size_t bytes = (size_t)p->Kx * p->L * p->L * 6 * p->QyS * real;
    if (!p->d_dtensor) {
        DEMAG_TRY(dalloc(&p->d_dtensor, bytes, "derivative tensor"));
    }
    DEMAG_CUDA(cudaMemsetAsync(p->d_dtensor, 0, bytes, st));
    p->dlayer = -1;
    DEMAG_TRY(build_tensor(p, st, layer, p->d_dtensor));
    p->dlayer = layer;
    return DEMAG_OK;
}

// Tensor of an equidistant plan (Eq. FFT_3D): the 2D-transformed kernels of
// the z-offsets r = 0..L-1 (pairs (r, 0) of the stack), extracted in double and
// natural folded-ky order, then transformed along z by k_ztensor.
static demag_status build_tensor3d(demag_plan *p, cudaStream_t st) {
    const int L = p->L;
    const int QyS2 = tensor_row(p->log2Py, true);
    const size_t tmp_bytes = (size_t)p->Kx * L * 6 * QyS2 * sizeof(double);
    void *tmp = nullptr;
    DEMAG_TRY(dalloc(&tmp, tmp_bytes, "offset kernel spectra"));
    demag_status rc = build_tensor(p, st, -1, tmp, true);
    if (rc == DEMAG_OK) {
        cudaError_t e = launch_ztensor((const double *)tmp, p->d_tensor, p->precision == DEMAG_PREC_FP64, p->log2Px,
                                       p->log2Py, QyS2, L, p->log2Pz, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = cuda_fail(e, "z-transform of the offset kernels");
    }
    cudaFree(tmp);
    return rc;
}

}  // namespace demag

using namespace demag;

extern "C" {

const char *demag_status_string(demag_status s) {
    switch (s) {
        case DEMAG_OK: return "DEMAG_OK";
        case DEMAG_EINVAL: return "DEMAG_EINVAL";
        case DEMAG_ENOMEM: return "DEMAG_ENOMEM";
        case DEMAG_ECUDA: return "DEMAG_ECUDA";
        case DEMAG_EUNSUPPORTED: return "DEMAG_EUNSUPPORTED";
    }
    return "DEMAG_UNKNOWN";
}

const char *demag_last_error(void) { return g_last_error.c_str(); }

demag_status demag_debug_fail_alloc(int after) {
    g_alloc_fail_after = after < 0 ? -1 : after;
    return DEMAG_OK;
}

demag_status demag_selftest_bounded_wait(long long limit_cycles, void *stream) {
    if (limit_cycles < 1 || limit_cycles > kWaitLimitCycles)
        return fail(DEMAG_EINVAL, "limit_cycles must be in [1, 2^31]");
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = launch_selftest_wait(limit_cycles, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "bounded-wait self test");
    return DEMAG_OK;
}

demag_status demag_wait_timeouts(unsigned long long *count) {
    if (!count) return fail(DEMAG_EINVAL, "count is NULL");
    int dev = 0;
    DEMAG_CUDA(cudaGetDevice(&dev));
    DEMAG_CUDA(cudaDeviceSynchronize());
    unsigned now[2] = {0, 0};
    DEMAG_CUDA(read_wait_timeouts(&now[0], 0));
    DEMAG_CUDA(read_tc_timeouts(&now[1], 0));
    DEMAG_CUDA(cudaStreamSynchronize(0));
    *count = take_new_timeouts(dev, now);
    return DEMAG_OK;
}

}  // extern "C"

// Plan creation of both methods: 0 the hybrid of Eq. FFT_v2 (any thicknesses),
// 1 the equidistant 3D FFT of Eq. FFT_3D (all thicknesses equal).
static demag_status plan_create_impl(demag_plan_t *plan, int nx, int ny, double dx, double dy,
                                     const double *thickness, int L, int precision, int max_batch,
                                     void *stream, int method) {
    NvtxRange nvtx_range("demag plan build");
    g_last_error.clear();
    if (!plan) return fail(DEMAG_EINVAL, "plan pointer is NULL");
    if (!thickness) return fail(DEMAG_EINVAL, "thickness pointer is NULL");
    if (nx < 1 || ny < 1) return fail(DEMAG_EINVAL, "nx and ny must be >= 1");
    if (nx > 2048 || ny > 2048) return fail(DEMAG_EUNSUPPORTED, "nx and ny must be <= 2048");
    if (L < 1) return fail(DEMAG_EINVAL, "L must be >= 1");
    if (L > 256) return fail(DEMAG_EUNSUPPORTED, "L must be <= 256");
    if (!(std::isfinite(dx) && dx > 0 && std::isfinite(dy) && dy > 0))
        return fail(DEMAG_EINVAL, "dx and dy must be finite and > 0");
    for (int l = 0; l < L; ++l)
        if (!(std::isfinite(thickness[l]) && thickness[l] > 0))
            return fail(DEMAG_EINVAL, "thickness[" + std::to_string(l) + "] must be finite and > 0");
    if (precision != DEMAG_PREC_FP64 && precision != DEMAG_PREC_FP32 &&
        precision != DEMAG_PREC_SPLIT_TF32 && precision != DEMAG_PREC_SPLIT_BF16)
        return fail(DEMAG_EINVAL, "unknown precision");
    if (max_batch < 1) return fail(DEMAG_EINVAL, "max_batch must be >= 1");
    if ((long long)max_batch * L * 3 > 65535)
        return fail(DEMAG_EUNSUPPORTED, "max_batch * L * 3 must be <= 65535");

    demag_plan *p = new (std::nothrow) demag_plan();
    if (!p) return fail(DEMAG_ENOMEM, "host allocation of the plan");
    p->nx = nx;
    p->ny = ny;
    p->L = L;
    p->dx = dx;
    p->dy = dy;
    p->precision = precision;
    p->max_batch = max_batch;
    p->thickness.assign(thickness, thickness + L);
    p->log2Px = ilog2_ceil(2 * nx);
    p->log2Py = ilog2_ceil(2 * ny);
    if (p->log2Px < 2) p->log2Px = 2;
    if (p->log2Py < 2) p->log2Py = 2;
    p->Kx = (1 << p->log2Px) / 2 + 1;
    p->Qy = (1 << p->log2Py) / 2 + 1;
    p->QyS = tensor_row(p->log2Py, precision == DEMAG_PREC_FP64);
    p->npairs = L * (L + 1) / 2;
    const bool fp64 = precision == DEMAG_PREC_FP64;
    if (method == 1) {
        if (precision != DEMAG_PREC_FP64 && precision != DEMAG_PREC_FP32) {
            delete p;
            return fail(DEMAG_EUNSUPPORTED, "equidistant plans take DEMAG_PREC_FP64 or DEMAG_PREC_FP32");
        }
        p->method = 1;
        p->split = 1;
        p->contract_mode = 5;
        p->npairs = L;  // z-offsets r = 0..L-1
        p->log2Pz = ilog2_ceil(2 * L);
        if (p->log2Pz < 1) p->log2Pz = 1;
        if (zconv_smem_bytes(p->log2Pz, fp64) > 220 * 1024) {
            delete p;
            return fail(DEMAG_EUNSUPPORTED, "nz above the z-convolution kernel's shared memory");
        }
    } else if (precision == DEMAG_PREC_SPLIT_TF32 || precision == DEMAG_PREC_SPLIT_BF16) {
        // split path, dense-product contraction on the tensor cores
        if (!gemm_supported(L, max_batch)) {
            delete p;
            return fail(DEMAG_EUNSUPPORTED, "layer count x batch above the dense-product contraction limit");
        }
        p->split = 1;
        p->umajor = 1;
        // tcgen05 products where they hold the plan, else the warp-level TF32 MMAs
        p->contract_mode = tc5_supported(L, max_batch, p->npairs)
                               ? (precision == DEMAG_PREC_SPLIT_BF16 ? 4 : 3)
                               : 2;
        // BF16 plans on the tcgen05 kernel store every value pre-split
        p->packed = p->contract_mode == 4 ? 1 : 0;
    } else {
        p->split = L > fused_max_layers(fp64, p->log2Py) ? 1 : 0;
        p->natural = !p->split && cols512_supported(p->log2Py, L, fp64) ? 1 : 0;
        if (p->split && !split_supported(L, max_batch, fp64)) {
            delete p;
            return fail(DEMAG_EUNSUPPORTED, "layer count x batch above the contraction kernels' limits");
        }
    }
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaGetDevice(&p->device);
    if (e != cudaSuccess) {
        delete p;
        return cuda_fail(e, "cudaGetDevice");
    }
    demag_status rc = upload_gauss_legendre();
    const size_t real = fp64 ? sizeof(double) : sizeof(float);
    const size_t cpx = 2 * real;
    p->tensor_bytes = p->method == 1 ? (size_t)p->Kx * p->Qy * ((1 << p->log2Pz) / 2 + 1) * 6 * real
                      : p->umajor    ? (size_t)p->Kx * p->Qy * ub_entry(L) * real
                                     : (size_t)p->Kx * p->npairs * 6 * p->QyS * real;
    p->field_bytes_per_state = (size_t)L * 3 * ny * nx * real;
    if (rc == DEMAG_OK) rc = dalloc(&p->d_tensor, p->tensor_bytes, "tensor");
    if (rc == DEMAG_OK && (e = cudaMemset(p->d_tensor, 0, p->tensor_bytes)) != cudaSuccess)
        rc = cuda_fail(e, "cudaMemset(tensor)");
    if (rc == DEMAG_OK) rc = dalloc(&p->d_ratio, (size_t)L * L * real, "ratios");
    if (rc == DEMAG_OK) rc = dalloc(&p->d_twx, (size_t)(1 << p->log2Px) / 2 * cpx, "twiddles");
    if (rc == DEMAG_OK) rc = dalloc(&p->d_twy, (size_t)(1 << p->log2Py) / 2 * cpx, "twiddles");
    if (rc == DEMAG_OK)
        rc = dalloc(&p->d_spec, (size_t)max_batch * L * 3 * p->Kx * ny * cpx, "spectrum workspace");
    if (rc == DEMAG_OK && p->split)
        rc = dalloc(&p->d_spec2, split_workspace_bytes(L, max_batch, p->log2Px, p->log2Py, fp64),
                    "column workspace");
    if (rc == DEMAG_OK) rc = dalloc(&p->d_tscale, (size_t)2 * L * real, "layer scales");
    if (rc == DEMAG_OK && (e = cudaHostAlloc((void **)&p->h_timeouts, 2 * sizeof(unsigned), cudaHostAllocDefault)) !=
                              cudaSuccess) {
        p->h_timeouts = nullptr;
        rc = cuda_fail(e, "cudaHostAlloc(timeout counters)");
    }
    if (rc == DEMAG_OK) {
        // t_j / t_i for target i, source j (reciprocity of the stored pairs)
        std::vector<double> r64((size_t)L * L);
        for (int i = 0; i < L; ++i)
            for (int j = 0; j < L; ++j) r64[(size_t)i * L + j] = thickness[j] / thickness[i];
        auto tx64 = twiddles<double2>(p->log2Px), ty64 = twiddles<double2>(p->log2Py);
        std::vector<double> sc64(2 * L);
        for (int l = 0; l < L; ++l) {
            sc64[l] = thickness[l];            // t_l
            sc64[L + l] = 1.0 / thickness[l];  // 1 / t_l
        }
        if (fp64) {
            if ((e = cudaMemcpy(p->d_tscale, sc64.data(), sc64.size() * 8, cudaMemcpyHostToDevice)) ||
                (e = cudaMemcpy(p->d_ratio, r64.data(), r64.size() * 8, cudaMemcpyHostToDevice)) ||
                (e = cudaMemcpy(p->d_twx, tx64.data(), tx64.size() * 16, cudaMemcpyHostToDevice)) ||
                (e = cudaMemcpy(p->d_twy, ty64.data(), ty64.size() * 16, cudaMemcpyHostToDevice)))
                rc = cuda_fail(e, "cudaMemcpy(plan constants)");
        } else {
            std::vector<float> r32(r64.begin(), r64.end());
            std::vector<float2> tx32(tx64.size()), ty32(ty64.size());
            for (size_t k = 0; k < tx64.size(); ++k) tx32[k] = make_float2((float)tx64[k].x, (float)tx64[k].y);
            for (size_t k = 0; k < ty64.size(); ++k) ty32[k] = make_float2((float)ty64[k].x, (float)ty64[k].y);
            std::vector<float> sc32(sc64.begin(), sc64.end());
            if ((e = cudaMemcpy(p->d_tscale, sc32.data(), sc32.size() * 4, cudaMemcpyHostToDevice)) ||
                (e = cudaMemcpy(p->d_ratio, r32.data(), r32.size() * 4, cudaMemcpyHostToDevice)) ||
                (e = cudaMemcpy(p->d_twx, tx32.data(), tx32.size() * 8, cudaMemcpyHostToDevice)) ||
                (e = cudaMemcpy(p->d_twy, ty32.data(), ty32.size() * 8, cudaMemcpyHostToDevice)))
                rc = cuda_fail(e, "cudaMemcpy(plan constants)");
        }
    }
    if (rc == DEMAG_OK && p->method == 1) {
        rc = dalloc(&p->d_twz, (size_t)(1 << p->log2Pz) / 2 * cpx, "z twiddles");
        if (rc == DEMAG_OK) {
            auto tz64 = twiddles<double2>(p->log2Pz);
            if (fp64) {
                e = cudaMemcpy(p->d_twz, tz64.data(), tz64.size() * 16, cudaMemcpyHostToDevice);
            } else {
                std::vector<float2> tz32(tz64.size());
                for (size_t k = 0; k < tz64.size(); ++k) tz32[k] = make_float2((float)tz64[k].x, (float)tz64[k].y);
                e = cudaMemcpy(p->d_twz, tz32.data(), tz32.size() * 8, cudaMemcpyHostToDevice);
            }
            if (e != cudaSuccess) rc = cuda_fail(e, "cudaMemcpy(z twiddles)");
        }
    }
    if (rc == DEMAG_OK) rc = p->method == 1 ? build_tensor3d(p, st) : build_tensor(p, st, -1, p->d_tensor);
    if (rc != DEMAG_OK) {
        free_plan(p);
        return rc;
    }
    *plan = p;
    return DEMAG_OK;
}

extern "C" {

demag_status demag_plan_create(demag_plan_t *plan, int nx, int ny, double dx, double dy,
                               const double *thickness, int L, int precision, int max_batch,
                               void *stream) {
    return plan_create_impl(plan, nx, ny, dx, dy, thickness, L, precision, max_batch, stream, 0);
}

demag_status demag_plan_create_equidistant(demag_plan_t *plan, int nx, int ny, int nz, double dx, double dy,
                                           double dz, int precision, int max_batch, void *stream) {
    if (nz < 1) return fail(DEMAG_EINVAL, "nz must be >= 1");
    if (nz > 256) return fail(DEMAG_EUNSUPPORTED, "nz must be <= 256");
    if (!(std::isfinite(dz) && dz > 0)) return fail(DEMAG_EINVAL, "dz must be finite and > 0");
    std::vector<double> th((size_t)nz, dz);
    return plan_create_impl(plan, nx, ny, dx, dy, th.data(), nz, precision, max_batch, stream, 1);
}

static demag_status check_apply(demag_plan_t plan, const void *m, double Ms, const void *H, int B) {
    if (!plan) return fail(DEMAG_EINVAL, "plan is NULL");
    if (!m || !H) return fail(DEMAG_EINVAL, "m or H is NULL");
    if (m == H) return fail(DEMAG_EINVAL, "H must not alias m");
    if (B < 1 || B > plan->max_batch) return fail(DEMAG_EINVAL, "B must be in [1, max_batch]");
    if (!std::isfinite(Ms)) return fail(DEMAG_EINVAL, "Ms must be finite");
    if (plan->slab_k1 >= 0)
        return fail(DEMAG_EUNSUPPORTED, "the plan keeps one kx slab of its tensor: it runs demag_columns_slab only");
    return DEMAG_OK;
}

static ApplyArgs apply_args(demag_plan_t plan, double Ms, int B) {
    ApplyArgs a;
    a.nx = plan->nx;
    a.ny = plan->ny;
    a.L = plan->L;
    a.B = B;
    a.log2Px = plan->log2Px;
    a.log2Py = plan->log2Py;
    a.npairs = plan->npairs;
    a.QyS = plan->QyS;
    a.tensor = plan->d_tensor;
    a.ratio = plan->d_ratio;
    a.twx = plan->d_twx;
    a.twy = plan->d_twy;
    a.log2twx = plan->log2Px;
    a.log2twy = plan->log2Py;
    a.spec = plan->d_spec;
    a.spec2 = plan->d_spec2;
    a.split = plan->split;
    a.contract_mode = plan->contract_mode;
    a.natural = plan->natural;
    a.bmask = plan->d_bmask;
    a.bfirst = plan->d_bfirst;
    a.packed = plan->packed;
    a.twz = plan->d_twz;
    a.log2Pz = plan->log2Pz;
    a.Ms = Ms;
    return a;
}

demag_status demag_apply(demag_plan_t plan, const void *m, double Ms, void *H, int B, void *stream) {
    demag_status rc = check_apply(plan, m, Ms, H, B);
    if (rc != DEMAG_OK) return rc;
    cudaError_t e = launch_apply(apply_args(plan, Ms, B), m, H, plan->precision == DEMAG_PREC_FP64,
                                 (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "demag_apply kernels");
    return DEMAG_OK;
}

demag_status demag_apply_timed(demag_plan_t plan, const void *m, double Ms, void *H, int B,
                               void *stream, float *stage_ms, int nstage) {
    demag_status rc = check_apply(plan, m, Ms, H, B);
    if (rc != DEMAG_OK) return rc;
    if (!stage_ms || nstage < kApplyStages) return fail(DEMAG_EINVAL, "stage_ms must hold 3 values");
    const bool inner = nstage >= kApplyStages + 3 && plan->split;
    const int nev = kApplyStages + 1 + (inner ? 4 : 0);
    cudaEvent_t ev[kApplyStages + 5] = {};
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    int made = 0;
    for (; made < nev; ++made)
        if ((e = cudaEventCreate(&ev[made])) != cudaSuccess) break;
    ApplyArgs a = apply_args(plan, Ms, B);
    if (inner) a.inner_ev = ev + kApplyStages + 1;
    if (e == cudaSuccess) e = launch_apply(a, m, H, plan->precision == DEMAG_PREC_FP64, st, ev);
    if (e == cudaSuccess) e = enqueue_timeout_read(plan, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    for (int k = 0; e == cudaSuccess && k < kApplyStages; ++k)
        e = cudaEventElapsedTime(&stage_ms[k], ev[k], ev[k + 1]);
    for (int k = 0; e == cudaSuccess && inner && k < 3; ++k)
        e = cudaEventElapsedTime(&stage_ms[kApplyStages + k], ev[kApplyStages + 1 + k],
                                 ev[kApplyStages + 2 + k]);
    for (int k = kApplyStages; k < nstage && !inner; ++k) stage_ms[k] = 0.0f;
    for (int k = 0; k < made; ++k) cudaEventDestroy(ev[k]);
    if (e != cudaSuccess) return cuda_fail(e, "demag_apply_timed");
    return timeout_status(plan, "demag_apply_timed");
}

// demag_apply_host for page-locked buffers and a batch of states: the batch is
// cut into up to four chunks of whole states; chunk c's input copy (on the
// plan's input copy stream) overlaps the row transforms of chunk c - 1, the
// columns and layer sum run on the whole batch, and chunk c's output copy (on
// the output copy stream) overlaps the inverse row transforms of chunk c + 1.  With async the call alternates
// between two staging sets and returns without waiting: the next call's input
// copies then overlap this call's columns and layer sum, and this call's output
// copies the next call's work.
static demag_status apply_host_pipelined(demag_plan_t plan, const void *m_host, double Ms, void *H_host, int B,
                                         cudaStream_t st, bool async) {
    const size_t full = plan->field_bytes_per_state * (size_t)plan->max_batch;
    int set = 0;
    if (async) set = plan->stage_set ^= 1;
    void *&stm = set ? plan->d_stage2_m : plan->d_stage_m;
    void *&sth = set ? plan->d_stage2_H : plan->d_stage_H;
    if (!stm) DEMAG_TRY(dalloc(&stm, full, "host staging"));
    if (!sth) DEMAG_TRY(dalloc(&sth, full, "host staging"));
    if (!plan->copy_st) DEMAG_CUDA(cudaStreamCreateWithFlags(&plan->copy_st, cudaStreamNonBlocking));
    if (!plan->copy_st2) DEMAG_CUDA(cudaStreamCreateWithFlags(&plan->copy_st2, cudaStreamNonBlocking));
    for (cudaEvent_t &ev : plan->pipe_ev[set])
        if (!ev) DEMAG_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    const bool fp64 = plan->precision == DEMAG_PREC_FP64;
    const size_t per_state = plan->field_bytes_per_state;
    const size_t spec_state = (size_t)plan->L * 3 * plan->Kx * plan->ny * (fp64 ? 16 : 8);
    const int nch = B < 4 ? B : 4;
    int b0s[5];
    for (int c = 0; c <= nch; ++c) b0s[c] = (int)((long long)B * c / nch);
    cudaStream_t cs = plan->copy_st, cs2 = plan->copy_st2;  // input, output copies
    cudaEvent_t *ev = plan->pipe_ev[set];
    const char *mh = (const char *)m_host;
    char *hh = (char *)H_host, *sm = (char *)stm, *sh = (char *)sth;
    if (!async) {
        // the staging buffers are free once earlier work on st is done
        DEMAG_CUDA(cudaEventRecord(ev[0], st));
        DEMAG_CUDA(cudaStreamWaitEvent(cs, ev[0], 0));
    } else {
        // this set's input buffer is free once its previous row transforms read it
        DEMAG_CUDA(cudaStreamWaitEvent(cs, ev[9], 0));
    }
    for (int c = 0; c < nch; ++c) {
        const size_t off = (size_t)b0s[c] * per_state, n = (size_t)(b0s[c + 1] - b0s[c]) * per_state;
        DEMAG_CUDA(cudaMemcpyAsync(sm + off, mh + off, n, cudaMemcpyHostToDevice, cs));
        DEMAG_CUDA(cudaEventRecord(ev[1 + c], cs));
    }
    const ApplyArgs a = apply_args(plan, Ms, B);
    auto chunk = [&](int c) {
        ApplyArgs ac = a;
        ac.B = b0s[c + 1] - b0s[c];
        ac.spec = (char *)a.spec + (size_t)b0s[c] * spec_state;
        return ac;
    };
    cudaError_t e = cudaSuccess;
    for (int c = 0; c < nch && e == cudaSuccess; ++c) {
        if ((e = cudaStreamWaitEvent(st, ev[1 + c], 0)) == cudaSuccess)
            e = launch_apply_stage(chunk(c), 0, sm + (size_t)b0s[c] * per_state, nullptr, fp64, st);
    }
    if (e == cudaSuccess) e = cudaEventRecord(ev[9], st);
    if (e == cudaSuccess) e = launch_apply_stage(a, 1, nullptr, nullptr, fp64, st);
    // this set's output buffer is free once its previous output copies are done
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ev[10], 0);
    for (int c = 0; c < nch && e == cudaSuccess; ++c) {
        const size_t off = (size_t)b0s[c] * per_state, n = (size_t)(b0s[c + 1] - b0s[c]) * per_state;
        if ((e = launch_apply_stage(chunk(c), 2, nullptr, sh + off, fp64, st)) != cudaSuccess) break;
        if ((e = cudaEventRecord(ev[5 + c], st)) != cudaSuccess) break;
        if ((e = cudaStreamWaitEvent(cs2, ev[5 + c], 0)) != cudaSuccess) break;
        e = cudaMemcpyAsync(hh + off, sh + off, n, cudaMemcpyDeviceToHost, cs2);
    }
    if (e == cudaSuccess) e = cudaEventRecord(ev[10], cs2);
    if (e == cudaSuccess && !async) e = cudaStreamWaitEvent(st, ev[10], 0);
    if (e != cudaSuccess) {
        cudaStreamSynchronize(cs);
        cudaStreamSynchronize(cs2);
        return cuda_fail(e, "demag_apply_host pipelined batch");
    }
    if (async) return DEMAG_OK;
    DEMAG_CUDA(enqueue_timeout_read(plan, st));
    DEMAG_CUDA(cudaStreamSynchronize(st));
    return timeout_status(plan, "demag_apply_host");
}

demag_status demag_apply_host_async(demag_plan_t plan, const void *m_host, double Ms, void *H_host, int B,
                                    void *stream) {
    demag_status rc = check_apply(plan, m_host, Ms, H_host, B);
    if (rc != DEMAG_OK) return rc;
    cudaPointerAttributes am, ah;
    const bool pinned = cudaPointerGetAttributes(&am, m_host) == cudaSuccess && am.type == cudaMemoryTypeHost &&
                        cudaPointerGetAttributes(&ah, H_host) == cudaSuccess && ah.type == cudaMemoryTypeHost;
    cudaGetLastError();
    if (!pinned) return fail(DEMAG_EINVAL, "demag_apply_host_async needs page-locked m and H");
    return apply_host_pipelined(plan, m_host, Ms, H_host, B, (cudaStream_t)stream, true);
}

demag_status demag_apply_host_wait(demag_plan_t plan, void *stream) {
    if (!plan) return fail(DEMAG_EINVAL, "plan is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    if (plan->copy_st) DEMAG_CUDA(cudaStreamSynchronize(plan->copy_st));
    if (plan->copy_st2) DEMAG_CUDA(cudaStreamSynchronize(plan->copy_st2));
    DEMAG_CUDA(enqueue_timeout_read(plan, st));
    DEMAG_CUDA(cudaStreamSynchronize(st));
    return timeout_status(plan, "demag_apply_host_wait");
}

demag_status demag_apply_host(demag_plan_t plan, const void *m_host, double Ms, void *H_host, int B,
                              void *stream) {
    demag_status rc = check_apply(plan, m_host, Ms, H_host, B);
    if (rc != DEMAG_OK) return rc;
    const size_t bytes = plan->field_bytes_per_state * (size_t)B;
    cudaStream_t st = (cudaStream_t)stream;
    cudaPointerAttributes am, ah;
    const bool pinned = cudaPointerGetAttributes(&am, m_host) == cudaSuccess && am.type == cudaMemoryTypeHost &&
                        cudaPointerGetAttributes(&ah, H_host) == cudaSuccess && ah.type == cudaMemoryTypeHost;
    cudaGetLastError();  // attribute queries of unregistered memory may leave an error
    // a batch in page-locked buffers: copies pipelined with the row transforms
    if (pinned && B >= 2) return apply_host_pipelined(plan, m_host, Ms, H_host, B, st, false);
    // one state in pinned (device-mapped) buffers: the kernels read m and write
    // H in host memory directly, so the transfers overlap the row transforms
    if (pinned && am.devicePointer && ah.devicePointer) {
        cudaError_t e = launch_apply(apply_args(plan, Ms, B), am.devicePointer, ah.devicePointer,
                                     plan->precision == DEMAG_PREC_FP64, st);
        if (e != cudaSuccess) return cuda_fail(e, "demag_apply_host kernels");
        DEMAG_CUDA(enqueue_timeout_read(plan, st));
        DEMAG_CUDA(cudaStreamSynchronize(st));
        return timeout_status(plan, "demag_apply_host");
    }
    if (!plan->d_stage_m) {
        const size_t full = plan->field_bytes_per_state * (size_t)plan->max_batch;
        DEMAG_TRY(dalloc(&plan->d_stage_m, full, "host staging"));
        DEMAG_TRY(dalloc(&plan->d_stage_H, full, "host staging"));
    }
    DEMAG_CUDA(cudaMemcpyAsync(plan->d_stage_m, m_host, bytes, cudaMemcpyHostToDevice, st));
    cudaError_t e = launch_apply(apply_args(plan, Ms, B), plan->d_stage_m, plan->d_stage_H,
                                 plan->precision == DEMAG_PREC_FP64, st);
    if (e != cudaSuccess) return cuda_fail(e, "demag_apply_host kernels");
    DEMAG_CUDA(cudaMemcpyAsync(H_host, plan->d_stage_H, bytes, cudaMemcpyDeviceToHost, st));
    DEMAG_CUDA(enqueue_timeout_read(plan, st));
    DEMAG_CUDA(cudaStreamSynchronize(st));
    return timeout_status(plan, "demag_apply_host");
}

demag_status demag_plan_set_path(demag_plan_t plan, int path) {
    if (!plan) return fail(DEMAG_EINVAL, "plan is NULL");
    if (plan->method == 1) {
        if (path != 0 && path != 8) return fail(DEMAG_EUNSUPPORTED, "equidistant plans run path 8 only");
        return DEMAG_OK;
    }
    const bool fp64 = plan->precision == DEMAG_PREC_FP64;
    if (plan->umajor) {
        const bool tc5 = tc5_supported(plan->L, plan->max_batch, plan->npairs);
        if (path == 0) path = !tc5 ? 4 : (plan->precision == DEMAG_PREC_SPLIT_BF16 ? 7 : 6);
        if (plan->packed && path != 7)
            return fail(DEMAG_EUNSUPPORTED, "a DEMAG_PREC_SPLIT_BF16 plan on the tcgen05 kernel runs path 7 only");
        if (plan->d_bmask && path != 6 && path != 7)
            return fail(DEMAG_EUNSUPPORTED, "a compressed tensor is read by paths 6 and 7 only");
        if (path != 3 && path != 4 && path != 6 && path != 7)
            return fail(DEMAG_EUNSUPPORTED, "split-precision plans run path 3, 4, 6 or 7");
        if ((path == 6 || path == 7) && !tc5)
            return fail(DEMAG_EUNSUPPORTED, "paths 6 and 7 need an even L <= 64 and max_batch <= 16");
        plan->contract_mode = path == 3 ? 1 : (path == 4 ? 2 : (path == 6 ? 3 : 4));
        return DEMAG_OK;
    }
    if (path == 3 || path == 4 || path == 6 || path == 7)
        return fail(DEMAG_EUNSUPPORTED, "paths 3, 4, 6 and 7 need a split-precision plan");
    if (plan->natural) {
        if (path != 0 && path != 1 && path != 5)
            return fail(DEMAG_EUNSUPPORTED, "plans on the 512-point fused kernel run path 5 only");
        return DEMAG_OK;
    }
    if (path == 0) path = plan->L > fused_max_layers(fp64, plan->log2Py) ? 2 : 1;
    if (path == 1) {
        if (plan->L > fused_max_layers(fp64, plan->log2Py))
            return fail(DEMAG_EUNSUPPORTED, "the fused kernel cannot hold this stack's columns");
        plan->split = 0;
        return DEMAG_OK;
    }
    if (path != 2) return fail(DEMAG_EINVAL, "path must be 0, 1 or 2");
    if (!split_supported(plan->L, plan->max_batch, fp64))
        return fail(DEMAG_EUNSUPPORTED, "layer count x batch above the split kernels' limits");
    if (!plan->d_spec2)
        DEMAG_TRY(dalloc(&plan->d_spec2,
                         split_workspace_bytes(plan->L, plan->max_batch, plan->log2Px, plan->log2Py, fp64),
                         "column workspace"));
    plan->split = 1;
    return DEMAG_OK;
}

demag_status demag_apply_adjoint(demag_plan_t plan, const void *gH, double Ms, void *gm, int B,
                                 void *stream) {
    demag_status rc = check_apply(plan, gH, Ms, gm, B);
    if (rc != DEMAG_OK) return rc;
    ApplyArgs a = apply_args(plan, Ms, B);
    const size_t real = plan->precision == DEMAG_PREC_FP64 ? 8 : 4;
    a.in_scale = (const char *)plan->d_tscale + plan->L * real;  // 1 / t_j on the sources
    a.out_scale = plan->d_tscale;                               // t_i on the targets
    cudaError_t e = launch_apply(a, gH, gm, plan->precision == DEMAG_PREC_FP64, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "demag_apply_adjoint kernels");
    return DEMAG_OK;
}

demag_status demag_apply_dthickness(demag_plan_t plan, const void *m, double Ms, void *dH, int B,
                                    int layer, void *stream) {
    demag_status rc = check_apply(plan, m, Ms, dH, B);
    if (rc != DEMAG_OK) return rc;
    if (layer < 0 || layer >= plan->L) return fail(DEMAG_EINVAL, "layer out of range");
    if (plan->umajor)
        return fail(DEMAG_EUNSUPPORTED, "thickness derivatives need a DEMAG_PREC_FP64 or DEMAG_PREC_FP32 plan");
    if (plan->method == 1)
        return fail(DEMAG_EUNSUPPORTED, "thickness derivatives need a plan of demag_plan_create");
    cudaStream_t st = (cudaStream_t)stream;
    DEMAG_TRY(ensure_dtensor(plan, layer, st));
    ApplyArgs a = apply_args(plan, Ms, B);
    a.tensor = plan->d_dtensor;
    a.npairs = plan->L * plan->L;
    a.full_pairs = 1;
    cudaError_t e = launch_apply(a, m, dH, plan->precision == DEMAG_PREC_FP64, st);
    if (e != cudaSuccess) return cuda_fail(e, "demag_apply_dthickness kernels");
    return DEMAG_OK;
}

demag_status demag_thickness_grad(demag_plan_t plan, const void *m, const void *gH, double Ms, int B,
                                  int layer, double *out, void *stream) {
    if (!out) return fail(DEMAG_EINVAL, "out is NULL");
    if (!gH) return fail(DEMAG_EINVAL, "gH is NULL");
    if (!plan) return fail(DEMAG_EINVAL, "plan is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    if (!plan->d_dH) DEMAG_TRY(dalloc(&plan->d_dH, plan->field_bytes_per_state * plan->max_batch, "dH/dt"));
    if (!plan->d_dot) DEMAG_TRY(dalloc((void **)&plan->d_dot, sizeof(double), "reduction"));
    DEMAG_TRY(demag_apply_dthickness(plan, m, Ms, plan->d_dH, B, layer, stream));
    DEMAG_CUDA(cudaMemsetAsync(plan->d_dot, 0, sizeof(double), st));
    const size_t n = plan->field_bytes_per_state / (plan->precision == DEMAG_PREC_FP64 ? 8 : 4) * B;
    const unsigned grid = (unsigned)std::min<size_t>((n + 255) / 256, 1024);
    if (plan->precision == DEMAG_PREC_FP64)
        k_dot<double><<<grid, 256, 0, st>>>((const double *)gH, (const double *)plan->d_dH, n, plan->d_dot);
    else
        k_dot<float><<<grid, 256, 0, st>>>((const float *)gH, (const float *)plan->d_dH, n, plan->d_dot);
    DEMAG_CUDA(cudaGetLastError());
    DEMAG_CUDA(cudaMemcpyAsync(out, plan->d_dot, sizeof(double), cudaMemcpyDeviceToHost, st));
    DEMAG_CUDA(enqueue_timeout_read(plan, st));
    DEMAG_CUDA(cudaStreamSynchronize(st));
    return timeout_status(plan, "demag_thickness_grad");
}

demag_status demag_tensor_points_dt(int n, const double *geom, double *out, double *dout,
                                    void *stream) {
    if (n < 0) return fail(DEMAG_EINVAL, "n must be >= 0");
    if (n > 0 && (!geom || !out || !dout)) return fail(DEMAG_EINVAL, "geom, out or dout is NULL");
    DEMAG_TRY(upload_gauss_legendre());
    cudaError_t e = launch_tensor_points_dt(n, geom, out, dout, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "tensor derivative points kernel");
    return DEMAG_OK;
}

demag_status demag_plan_compress(demag_plan_t plan, double tol, size_t *stored_bytes) {
    if (!plan) return fail(DEMAG_EINVAL, "plan is NULL");
    if (!(tol >= 0.0) || !(tol < 1.0)) return fail(DEMAG_EINVAL, "tol must be in [0, 1)");
    if (!plan->umajor || plan->method != 0 || (plan->contract_mode != 3 && plan->contract_mode != 4))
        return fail(DEMAG_EUNSUPPORTED, "compression needs a split-precision plan on path 6 or 7");
    if (plan->d_bmask) return fail(DEMAG_EUNSUPPORTED, "the plan's tensor is already compressed");
    if (plan->slab_k1 >= 0) return fail(DEMAG_EUNSUPPORTED, "the plan keeps one kx slab of its tensor");
    DEMAG_CUDA(cudaDeviceSynchronize());  // no apply may be reading the tensor
    float *out = nullptr;
    size_t bytes = 0;
    unsigned long long *mask = nullptr;
    unsigned *first = nullptr;
    const size_t nent = (size_t)plan->Kx * plan->Qy;
    cudaError_t e = compress_tensor((const float *)plan->d_tensor, nent, plan->L, plan->packed != 0, tol, &out, &bytes,
                                    &mask, &first, 0);
    if (e != cudaSuccess) return cuda_fail(e, "tensor compression");
    cudaFree(plan->d_tensor);
    plan->d_tensor = out;
    plan->tensor_bytes = bytes;
    plan->d_bmask = mask;
    plan->d_bfirst = first;
    plan->compress_tol = tol;
    if (stored_bytes) *stored_bytes = bytes;
    return DEMAG_OK;
}

// Bytes of the stored tensor per x-frequency (every layout is kx-major).
static size_t tensor_kx_bytes(const demag_plan *p) {
    const size_t real = p->precision == DEMAG_PREC_FP64 ? 8 : 4;
    return p->umajor ? (size_t)p->Qy * ub_entry(p->L) * real : (size_t)p->npairs * 6 * p->QyS * real;
}

demag_status demag_plan_keep_slab(demag_plan_t plan, int k0, int k1) {
    if (!plan) return fail(DEMAG_EINVAL, "plan is NULL");
    if (plan->method != 0 || !plan->split)
        return fail(DEMAG_EUNSUPPORTED, "slabs need a hybrid plan on the split path (paths 2, 3, 4, 6, 7)");
    if (plan->d_bmask) return fail(DEMAG_EUNSUPPORTED, "the plan's tensor is compressed");
    if (plan->slab_k1 >= 0) return fail(DEMAG_EUNSUPPORTED, "the plan already keeps a slab");
    if (k0 < 0 || k1 <= k0 || k1 > plan->Kx)
        return fail(DEMAG_EINVAL, "need 0 <= k0 < k1 <= Px / 2 + 1 = " + std::to_string(plan->Kx));
    DEMAG_CUDA(cudaDeviceSynchronize());  // no apply may be reading the tensor
    const size_t kb = tensor_kx_bytes(plan), bytes = (size_t)(k1 - k0) * kb;
    void *slab = nullptr;
    DEMAG_TRY(dalloc(&slab, bytes, "tensor slab"));
    cudaError_t e = cudaMemcpy(slab, (const char *)plan->d_tensor + (size_t)k0 * kb, bytes, cudaMemcpyDeviceToDevice);
    if (e != cudaSuccess) {
        cudaFree(slab);
        return cuda_fail(e, "tensor slab copy");
    }
    cudaFree(plan->d_tensor);
    plan->d_tensor = slab;
    plan->tensor_bytes = bytes;
    plan->slab_k0 = k0;
    plan->slab_k1 = k1;
    // the row spectrum workspace serves demag_apply only; the column
    // workspace shrinks to the slab where a smaller one can be had (else the
    // plan keeps the full one, which holds any slab)
    cudaFree(plan->d_spec);
    plan->d_spec = nullptr;
    const bool fp64 = plan->precision == DEMAG_PREC_FP64;
    const size_t w2 = split_workspace_bytes(plan->L, plan->max_batch, plan->log2Px, plan->log2Py, fp64) /
                      plan->Kx * (k1 - k0);
    void *ws = nullptr;
    if (dalloc(&ws, w2, "column workspace of the slab") == DEMAG_OK) {
        cudaFree(plan->d_spec2);
        plan->d_spec2 = ws;
    }
    return DEMAG_OK;
}

static demag_status check_planes(demag_plan_t plan, const void *a, const void *b, int p0, int p1) {
    if (!plan) return fail(DEMAG_EINVAL, "plan is NULL");
    if (!a || !b) return fail(DEMAG_EINVAL, "a field or spectrum pointer is NULL");
    const int P = plan->max_batch * plan->L * 3;
    if (p0 < 0 || p1 <= p0 || p1 > P)
        return fail(DEMAG_EINVAL, "need 0 <= p0 < p1 <= max_batch * L * 3 = " + std::to_string(P));
    return DEMAG_OK;
}

demag_status demag_rows_forward(demag_plan_t plan, const void *m, int p0, int p1, void *spec, void *stream) {
    DEMAG_TRY(check_planes(plan, m, spec, p0, p1));
    const bool fp64 = plan->precision == DEMAG_PREC_FP64;
    const size_t real = fp64 ? 8 : 4;
    ApplyArgs a = apply_args(plan, 0.0, plan->max_batch);
    a.spec = spec;
    a.planes = p1 - p0;
    const char *mp = (const char *)m + (size_t)p0 * plan->nx * plan->ny * real;
    cudaError_t e = launch_apply_stage(a, 0, mp, nullptr, fp64, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "row transform kernels");
    return DEMAG_OK;
}

demag_status demag_rows_inverse(demag_plan_t plan, const void *spec, int p0, int p1, double Ms, void *H,
                                void *stream) {
    DEMAG_TRY(check_planes(plan, spec, H, p0, p1));
    if (!std::isfinite(Ms)) return fail(DEMAG_EINVAL, "Ms must be finite");
    const bool fp64 = plan->precision == DEMAG_PREC_FP64;
    const size_t real = fp64 ? 8 : 4;
    ApplyArgs a = apply_args(plan, Ms, plan->max_batch);
    a.spec = const_cast<void *>(spec);
    a.planes = p1 - p0;
    char *hp = (char *)H + (size_t)p0 * plan->nx * plan->ny * real;
    cudaError_t e = launch_apply_stage(a, 2, nullptr, hp, fp64, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "row transform kernels");
    return DEMAG_OK;
}

demag_status demag_columns_slab(demag_plan_t plan, void *spec, int k0, int k1, int B, void *stream) {
    if (!plan) return fail(DEMAG_EINVAL, "plan is NULL");
    if (!spec) return fail(DEMAG_EINVAL, "spec is NULL");
    if (plan->method != 0 || !plan->split)
        return fail(DEMAG_EUNSUPPORTED, "slabs need a hybrid plan on the split path (paths 2, 3, 4, 6, 7)");
    if (plan->d_bmask) return fail(DEMAG_EUNSUPPORTED, "the plan's tensor is compressed");
    if (B < 1 || B > plan->max_batch) return fail(DEMAG_EINVAL, "B must be in [1, max_batch]");
    const int s0 = plan->slab_k1 >= 0 ? plan->slab_k0 : 0, s1 = plan->slab_k1 >= 0 ? plan->slab_k1 : plan->Kx;
    if (k0 < s0 || k1 <= k0 || k1 > s1)
        return fail(DEMAG_EINVAL, "need " + std::to_string(s0) + " <= k0 < k1 <= " + std::to_string(s1) +
                                      " (the x-frequencies of the plan's tensor)");
    ApplyArgs a = apply_args(plan, 0.0, B);
    a.spec = spec;
    a.kx_count = k1 - k0;
    a.tensor = (const char *)plan->d_tensor + (size_t)(k0 - s0) * tensor_kx_bytes(plan);
    cudaError_t e = launch_apply_stage(a, 1, nullptr, nullptr, plan->precision == DEMAG_PREC_FP64,
                                       (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "column and contraction kernels");
    return DEMAG_OK;
}

demag_status demag_plan_info(demag_plan_t plan, long long *out) {
    if (!plan || !out) return fail(DEMAG_EINVAL, "plan or out is NULL");
    out[0] = plan->nx;
    out[1] = plan->ny;
    out[2] = plan->L;
    out[3] = 1LL << plan->log2Px;
    out[4] = 1LL << plan->log2Py;
    out[5] = plan->precision;
    out[6] = plan->max_batch;
    out[7] = plan->npairs;
    out[8] = plan->method == 1 ? (1 << plan->log2Pz) / 2 + 1 : plan->QyS;
    static const int umajor_path[5] = {3, 3, 4, 6, 7};
    out[9] = plan->method == 1 ? 8
           : plan->umajor      ? umajor_path[plan->contract_mode]
                          : (plan->split ? 2 : (plan->natural ? 5 : 1));
    return DEMAG_OK;
}

demag_status demag_plan_tensor(demag_plan_t plan, void *out, size_t bytes, void *stream) {
    if (!plan || !out) return fail(DEMAG_EINVAL, "plan or out is NULL");
    if (plan->d_bmask) return fail(DEMAG_EUNSUPPORTED, "the plan's tensor is compressed (demag_plan_compress)");
    if (bytes != plan->tensor_bytes)
        return fail(DEMAG_EINVAL, "out must hold exactly " + std::to_string(plan->tensor_bytes) + " bytes");
    DEMAG_CUDA(cudaMemcpyAsync(out, plan->d_tensor, bytes, cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    return DEMAG_OK;
}

demag_status demag_tensor_points(int n, const double *geom, double *out, void *stream) {
    if (n < 0) return fail(DEMAG_EINVAL, "n must be >= 0");
    if (n > 0 && (!geom || !out)) return fail(DEMAG_EINVAL, "geom or out is NULL");
    DEMAG_TRY(upload_gauss_legendre());
    cudaError_t e = launch_tensor_points(n, geom, out, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "tensor points kernel");
    return DEMAG_OK;
}

demag_status demag_destroy(demag_plan_t plan) {
    if (!plan) return DEMAG_OK;
    cudaError_t e = cudaDeviceSynchronize();
    free_plan(plan);
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize in demag_destroy");
    return DEMAG_OK;
}

}  // extern "C"
