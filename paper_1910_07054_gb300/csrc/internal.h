// Internal interfaces between the translation units of libdemag.
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <string>
#include <vector>

#include "../../include/demag.h"

namespace demag {

// Records a failure message for demag_last_error() and returns the status.
demag_status fail(demag_status st, const std::string &msg);
demag_status cuda_fail(cudaError_t err, const char *what);

#define DEMAG_CUDA(call)                                                   \
    do {                                                                   \
        cudaError_t e_ = (call);                                           \
        if (e_ != cudaSuccess) return ::demag::cuda_fail(e_, #call);       \
    } while (0)

// Gauss-Legendre rules for n = 1..kGLMax, uploaded to constant memory once.
constexpr int kGLMax = 8;
demag_status upload_gauss_legendre();

// Layer geometry on the device for the tensor builder.
struct StackDev {
    const double *z;   // [L+1] interface heights, z[0] = 0
    const double *th;  // [L] thicknesses
};

// Evaluate n tensors at geom[n][9] (X,Y,Z,tx,ty,tz,sx,sy,sz) -> out[n][6].
cudaError_t launch_tensor_points(int n, const double *geom, double *out, cudaStream_t st);

// Fill the padded real-space kernels of pairs [p0, p0 + np) into three complex
// planes per pair ([np][3][Py][Px], x fastest; float2 if f32, else double2),
// zeroed beforehand: plane 0 = N_xx + i N_yy, plane 1 = N_zz + i N_xy, plane 2 =
// N_xz + i N_yz; every value is evaluated in double.  far32: far-field
// quadrature with float node sums (float plans).
cudaError_t launch_kernel_planes(void *planes, bool f32, int p0, int np, const int *pair_i,
                                 const int *pair_j, int nx, int ny, double dx, double dy,
                                 int log2Px, int log2Py, const double *z, const double *th,
                                 cudaStream_t st, bool far32 = false);

// Tensor and its derivative along (dtz, dsz, dZ) at geom[n][12]
// (X,Y,Z,tx,ty,tz,sx,sy,sz,dtz,dsz,dZ) -> out[n][6], dout[n][6].
cudaError_t launch_tensor_points_dt(int n, const double *geom, double *out, double *dout,
                                    cudaStream_t st);

// d N(i <- j)/d t_layer of all L*L pairs P = i*L + j in [p0, p0 + np), as
// three complex planes per pair like launch_kernel_planes (zeroed beforehand).
cudaError_t launch_dkernel_planes(void *planes, bool f32, int p0, int np, int L, int layer, int nx, int ny,
                                  double dx, double dy, int log2Px, int log2Py, const double *z,
                                  const double *th, cudaStream_t st);

// In-place 2D FFT (forward) of nplanes planes [Py][Px] of float2 (f32, with
// float twiddle tables) or double2.
cudaError_t launch_fft2_planes(void *planes, bool f32, int nplanes, int log2Px, int log2Py, const void *twx,
                               int log2twx, const void *twy, int log2twy, cudaStream_t st);

// Extract the stored quadrant of pairs [p0, p0+np) from transformed planes into
// the plan tensor, scaled by 1/(Px Py), y-frequencies in the stored order of
// layout.cuh: [Kx][npairs][6][QyS] (umajor = 0) or [Kx][Qy][npairs][6]
// (umajor = 1, float only).
// umajor: the blocked layout of dense-product plans (layout.cuh), which needs
// the pair lists (target i <= source j), the thicknesses and L.
cudaError_t launch_extract_tensor(const void *planes, bool f32, int p0, int np, int npairs,
                                  int log2Px, int log2Py, int QyS, void *tensor, bool fp64,
                                  cudaStream_t st, int umajor = 0, int natural = 0,
                                  const int *pair_i = nullptr, const int *pair_j = nullptr,
                                  const double *th = nullptr, int L = 0);

// ---- apply ---------------------------------------------------------------
struct ApplyArgs {
    int nx, ny, L, B;
    int log2Px, log2Py;
    int npairs, QyS;
    const void *tensor;   // [Kx][npairs][6][QyS]
    const void *ratio;    // [L][L]: t_j / t_i (plan real type)
    const void *twx;      // twiddles for Px (complex of the plan type)
    const void *twy;      // twiddles for Py
    int log2twx, log2twy;
    void *spec;           // [B][L][3][Kx][ny] complex workspace
    void *spec2 = nullptr;  // split path: [Kx][Py][B][L][3] complex workspace
    int split = 0;        // 1: column transforms and contraction in separate kernels
    int full_pairs = 0;   // 1: tensor holds all L*L pairs (no reciprocity)
    int contract_mode = 0;  // split path: 0 per-item kernel, 1 dense products on FP32
                            // cores, 2 dense products on tensor cores (warp-level 3xTF32), 3 on
                            // the tcgen05 tensor cores (3xTF32, TMEM accumulators), 4 the same
                            // with 3xBF16, 5 the z-convolution of the equidistant method
    int natural = 0;      // 512-point column kernel, tensor in natural folded-ky order
    const unsigned long long *bmask = nullptr;  // block-compressed tensor: kept blocks per entry
    const unsigned *bfirst = nullptr;           // and the entry's first block (units of 64 floats)
    cudaEvent_t *inner_ev = nullptr;  // split path, optional [4]: before and after its 3 kernels
    const void *in_scale = nullptr;   // optional [L]: m of layer l scaled on input
    const void *out_scale = nullptr;  // optional [L]: H of layer l scaled on output
    const void *twz = nullptr;        // equidistant plans: twiddles for Pz
    int log2Pz = 0;                   // equidistant plans: padded z size
    int packed = 0;                   // tensor of BF16 split pairs, zz negated (contraction mode 4 only)
    int planes = 0;                   // row transforms: planes to transform (0: B * L * 3)
    int kx_count = 0;                 // split path: x-frequencies in spec, spec2 and tensor (0: all)
    double Ms;
};

// Dense-product contraction (contract_gemm.cu), float tensors in the u-major layout.
size_t gemm_smem_bytes(int L, int B);
bool gemm_supported(int L, int B);
cudaError_t launch_contract_gemm(const ApplyArgs &a, bool tensor_cores, cudaStream_t st);

// 512-point transforms with the radix-8 engine (apply512.cu).
bool cols512_supported(int log2Py, int L, bool fp64);
template <typename T>
cudaError_t launch_rows512(const ApplyArgs &a, const void *m, void *H, bool forward, cudaStream_t st);
template <typename T>
cudaError_t launch_cols512(const ApplyArgs &a, cudaStream_t st);
// Bounded waits of the streamed column kernel that gave up: the device
// counter only grows; this enqueues a copy of its value to *dst on `st`.
cudaError_t read_wait_timeouts(unsigned *dst, cudaStream_t st);
// One block whose single bounded wait cannot complete (gives up after `limit` cycles).
cudaError_t launch_selftest_wait(long long limit, cudaStream_t st);

// Dense-product contraction on the tcgen05 tensor cores (contract_tc5.cu).
// Column transforms of the split path for Py = 1024 (two 512-point radix-8
// transforms per column; cols1024.cu).
bool cols1024_supported(int log2Py, int ny, bool fp64);
cudaError_t launch_cols1024(bool inverse, const void *src, void *dst, int ny, int Kx, int planes, const void *tw,
                            int log2tw, cudaStream_t st);
// Row transforms for Px = 1024 (two 512-point radix-8 transforms per row pair;
// rows1024.cu).
bool rows1024_supported(int log2Px, int nx, bool fp64);
cudaError_t launch_rows1024(bool inverse, const void *src, void *dst, int nx, int ny, int planes, const void *tw,
                            int log2tw, float out_scale, const void *layer_scale, int L, cudaStream_t st);
bool tc5_supported(int L, int B, int npairs);
// bf16: three BF16 passes (kind::f16) instead of three TF32 passes.
cudaError_t launch_contract_tc5(const ApplyArgs &a, bool bf16, cudaStream_t st);
// The same count for the tcgen05 contraction kernel.
cudaError_t read_tc_timeouts(unsigned *dst, cudaStream_t st);
// Block-sparse copy of a dense-product tensor (compress.cu): nent entries of the
// blocked layout for L layers; blocks whose values are all below tol times their
// component's maximum are dropped.  On success *out (device, *out_bytes bytes),
// *mask and *first (device, nent each) are new allocations owned by the caller.
// packed: the slots hold BF16 split pairs (their value is hi + lo).
cudaError_t compress_tensor(const float *tensor, size_t nent, int L, bool packed, double tol, float **out,
                            size_t *out_bytes, unsigned long long **mask, unsigned **first, cudaStream_t st);

// Equidistant method of Eq. FFT_3D (fft3d.cu): the z-convolution that
// replaces the layer contraction (contract_mode 5), and the z-transform of the
// 2D-transformed offset kernels src [Kx][L][6][QyS2] (double, natural folded
// ky) into the tensor [Kx][Py/2+1][Pz/2+1][6].
size_t zconv_smem_bytes(int log2Pz, bool fp64);
cudaError_t launch_zconv(const ApplyArgs &a, bool fp64, cudaStream_t st);
cudaError_t launch_ztensor(const double *src, void *dst, bool fp64, int log2Px, int log2Py, int QyS2, int L,
                           int log2Pz, cudaStream_t st);

// Split path (apply_split.cu).
size_t split_workspace_bytes(int L, int B, int log2Px, int log2Py, bool fp64);
bool split_supported(int L, int B, bool fp64);
cudaError_t launch_split_columns(const ApplyArgs &a, bool fp64, cudaStream_t st);

// Largest layer count the fused column kernel handles for a precision.
int fused_max_layers(bool fp64, int log2Py);
// events (optional, may be null): [0] before the first kernel, [k] after kernel k.
constexpr int kApplyStages = 3;
cudaError_t launch_apply(const ApplyArgs &a, const void *m, void *H, bool fp64, cudaStream_t st,
                         cudaEvent_t *events = nullptr);
// One of the three stages of launch_apply: 0 forward rows (m -> a.spec), 1 the
// columns with the layer sum (a.spec in place), 2 inverse rows (a.spec -> H);
// the row stages work on the a.B states at m / H / a.spec as given.
cudaError_t launch_apply_stage(const ApplyArgs &a, int stage, const void *m, void *H, bool fp64, cudaStream_t st);

}  // namespace demag

struct demag_plan {
    int nx, ny, L, precision, max_batch;
    double dx, dy;
    int log2Px, log2Py, Kx, Qy, QyS, npairs;
    std::vector<double> thickness;
    void *d_tensor = nullptr;     // [Kx][npairs][6][QyS]
    void *d_ratio = nullptr;      // [L][L]
    void *d_twx = nullptr, *d_twy = nullptr;
    void *d_spec = nullptr;       // [max_batch][L][3][Kx][ny] complex
    void *d_spec2 = nullptr;      // split path workspace
    int split = 0;                // 1: split path
    int contract_mode = 0;        // split path contraction (see ApplyArgs)
    int umajor = 0;               // blocked tensor layout [Kx][Qy][6][blocks] (dense-product plans)
    int packed = 0;               // blocked layout of BF16 split pairs, zz negated (DEMAG_PREC_SPLIT_BF16 on path 7)
    unsigned long long *d_bmask = nullptr;  // after demag_plan_compress: kept blocks per entry
    unsigned *d_bfirst = nullptr;           // and each entry's first block
    double compress_tol = -1.0;             // < 0: not compressed
    int slab_k0 = 0, slab_k1 = -1;          // after demag_plan_keep_slab: the x-frequencies kept (k1 < 0: all)
    int natural = 0;              // fused 512-point column kernel, natural folded-ky tensor
    int method = 0;               // 0 hybrid (Eq. FFT_v2), 1 equidistant 3D FFT (Eq. FFT_3D)
    int log2Pz = 0;               // equidistant plans: padded z size
    void *d_twz = nullptr;        // equidistant plans: twiddles for Pz
    void *d_tscale = nullptr;     // [2L]: t_l, then 1 / t_l (plan real type)
    void *d_dtensor = nullptr;    // d N / d t_dlayer, all L*L pairs, [Kx][L*L][6][QyS]
    int dlayer = -1;              // layer of d_dtensor (-1: none)
    void *d_dH = nullptr;         // [max_batch] fields of d H / d t
    double *d_dot = nullptr;      // reduction scratch
    void *d_stage_m = nullptr;    // staging for demag_apply_host
    void *d_stage_H = nullptr;
    unsigned *h_timeouts = nullptr;  // pinned host copy of the two bounded-wait counters
    cudaStream_t copy_st = nullptr;  // demag_apply_host: input copies of a pipelined batch
    cudaStream_t copy_st2 = nullptr; // and its output copies
    // events of the two staging sets: start, 4 inputs, 4 outputs, m staging free,
    // H staging free
    cudaEvent_t pipe_ev[2][11] = {};
    void *d_stage2_m = nullptr;      // second staging set (demag_apply_host_async)
    void *d_stage2_H = nullptr;
    int stage_set = 0;               // set of the last demag_apply_host_async
    size_t tensor_bytes = 0, field_bytes_per_state = 0;
    int device = 0;
};
