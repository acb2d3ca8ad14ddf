// Surrogate network for the layer-thickness optimisation of Sec. 4: a small
// multilayer perceptron mapping the L layer thicknesses of a stack to the
// mean demagnetization field of one layer (the free layer).  Weights are kept
// in bfloat16 for compute (a float master copy for the optimiser), all sums
// accumulate in float.
//
//   x (in) -> h1 = tanh(W1 x + b1) -> h2 = tanh(W2 h1 + b2)
//          -> h3 = tanh(W3 h2 + b3) -> y = W4 h3 + b4 (out)
//
// Parameter vector (float master or bf16 copy), in this order:
//   W1 [H][I], b1 [H], W2 [H][H], b2 [H], W3 [H][H], b3 [H], W4 [O][H], b4 [O]
// with I inputs, H hidden units, O outputs (row-major, W[out][in]).
//
// One block per tile of kMlpTile samples; thread j of a layer owns hidden
// unit j.  Activations of the tile live in shared memory.
#include <cuda_bf16.h>

#include "internal.h"

namespace demag {

constexpr int kMlpTile = 32;
constexpr int kMlpThreads = 64;
constexpr int kMlpMaxH = 64, kMlpMaxI = 32, kMlpMaxO = 8;

struct MlpDims {
    int I, H, O;
    int oW1, ob1, oW2, ob2, oW3, ob3, oW4, ob4, P;
};

__host__ __device__ inline MlpDims mlp_dims(int I, int H, int O) {
    MlpDims d;
    d.I = I;
    d.H = H;
    d.O = O;
    d.oW1 = 0;
    d.ob1 = d.oW1 + H * I;
    d.oW2 = d.ob1 + H;
    d.ob2 = d.oW2 + H * H;
    d.oW3 = d.ob2 + H;
    d.ob3 = d.oW3 + H * H;
    d.oW4 = d.ob3 + H;
    d.ob4 = d.oW4 + O * H;
    d.P = d.ob4 + O;
    return d;
}

__device__ __forceinline__ float bf(const __nv_bfloat16 *w, int k) { return __bfloat162float(w[k]); }

// Loads the bf16 parameters into shared memory as float.
__device__ void load_params(const __nv_bfloat16 *__restrict__ w, float *ws, int P) {
    for (int k = threadIdx.x; k < P; k += blockDim.x) ws[k] = bf(w, k);
}

// Dense layer for the tile: out[s][j] = act(sum_k W[j][k] in[s][k] + b[j]).
__device__ void dense_tile(const float *W, const float *b, const float *in, int nin, float *out,
                           int nout, int ns, bool act) {
    for (int j = threadIdx.x; j < nout; j += blockDim.x) {
        const float *wj = W + j * nin;
        for (int s = 0; s < ns; ++s) {
            float acc = b[j];
            const float *xs = in + s * nin;
            for (int k = 0; k < nin; ++k) acc = fmaf(wj[k], xs[k], acc);
            out[s * nout + j] = act ? tanhf(acc) : acc;
        }
    }
}

}  // namespace demag

namespace demag {

// Shared-memory layout of a tile: params | x [T][I] | h1, h2, h3 [T][H] |
// g4 [T][O] | d3, d2, d1 [T][H]
__host__ __device__ inline size_t mlp_smem_floats(const MlpDims &d, bool backward) {
    size_t n = (size_t)d.P + kMlpTile * d.I + 3 * kMlpTile * d.H + kMlpTile * d.O;
    if (backward) n += 3 * kMlpTile * d.H;
    return n;
}

__device__ void mlp_forward_tile(const MlpDims &d, const float *ws, const float *xin, float *h1,
                                 float *h2, float *h3, float *yo, int ns) {
    dense_tile(ws + d.oW1, ws + d.ob1, xin, d.I, h1, d.H, ns, true);
    __syncthreads();
    dense_tile(ws + d.oW2, ws + d.ob2, h1, d.H, h2, d.H, ns, true);
    __syncthreads();
    dense_tile(ws + d.oW3, ws + d.ob3, h2, d.H, h3, d.H, ns, true);
    __syncthreads();
    dense_tile(ws + d.oW4, ws + d.ob4, h3, d.H, yo, d.O, ns, false);
    __syncthreads();
}

__global__ void __launch_bounds__(kMlpThreads) k_mlp_forward(const __nv_bfloat16 *__restrict__ w,
                                                            const float *__restrict__ x,
                                                            float *__restrict__ y, int N, int I,
                                                            int H, int O) {
    extern __shared__ float sm[];
    const MlpDims d = mlp_dims(I, H, O);
    float *ws = sm, *xin = ws + d.P, *h1 = xin + kMlpTile * I, *h2 = h1 + kMlpTile * H;
    float *h3 = h2 + kMlpTile * H, *yo = h3 + kMlpTile * H;
    const int s0 = blockIdx.x * kMlpTile, ns = min(kMlpTile, N - s0);
    load_params(w, ws, d.P);
    for (int e = threadIdx.x; e < ns * I; e += blockDim.x) xin[e] = x[(size_t)s0 * I + e];
    __syncthreads();
    mlp_forward_tile(d, ws, xin, h1, h2, h3, yo, ns);
    for (int e = threadIdx.x; e < ns * O; e += blockDim.x) y[(size_t)s0 * O + e] = yo[e];
}

// d_prev[s][k] = (sum_j W[j][k] d[s][j]) * (1 - a_prev[s][k]^2)  (tanh'),
// or without the factor for the input gradient (a_prev == nullptr).
__device__ void back_tile(const float *W, const float *dcur, int ncur, const float *a_prev,
                          float *dprev, int nprev, int ns) {
    for (int k = threadIdx.x; k < nprev; k += blockDim.x) {
        for (int s = 0; s < ns; ++s) {
            float acc = 0.f;
            for (int j = 0; j < ncur; ++j) acc = fmaf(W[j * nprev + k], dcur[s * ncur + j], acc);
            if (a_prev) {
                const float a = a_prev[s * nprev + k];
                acc *= 1.f - a * a;
            }
            dprev[s * nprev + k] = acc;
        }
    }
}

// gW[j][k] += sum_s d[s][j] a[s][k];  gb[j] += sum_s d[s][j]
__device__ void grad_tile(const float *dcur, int ncur, const float *a, int nin, float *gW, float *gb,
                          int ns) {
    for (int e = threadIdx.x; e < ncur * (nin + 1); e += blockDim.x) {
        const int j = e / (nin + 1), k = e - j * (nin + 1);
        float acc = 0.f;
        if (k < nin) {
            for (int s = 0; s < ns; ++s) acc = fmaf(dcur[s * ncur + j], a[s * nin + k], acc);
            atomicAdd(&gW[j * nin + k], acc);
        } else {
            for (int s = 0; s < ns; ++s) acc += dcur[s * ncur + j];
            atomicAdd(&gb[j], acc);
        }
    }
}

__global__ void __launch_bounds__(kMlpThreads) k_mlp_backward(const __nv_bfloat16 *__restrict__ w,
                                                             const float *__restrict__ x,
                                                             const float *__restrict__ gy,
                                                             float *__restrict__ gw,
                                                             float *__restrict__ gx, int N, int I,
                                                             int H, int O) {
    extern __shared__ float sm[];
    const MlpDims d = mlp_dims(I, H, O);
    float *ws = sm, *xin = ws + d.P, *h1 = xin + kMlpTile * I, *h2 = h1 + kMlpTile * H;
    float *h3 = h2 + kMlpTile * H, *g4 = h3 + kMlpTile * H, *d3 = g4 + kMlpTile * O;
    float *d2 = d3 + kMlpTile * H, *d1 = d2 + kMlpTile * H;
    const int s0 = blockIdx.x * kMlpTile, ns = min(kMlpTile, N - s0);
    load_params(w, ws, d.P);
    for (int e = threadIdx.x; e < ns * I; e += blockDim.x) xin[e] = x[(size_t)s0 * I + e];
    __syncthreads();
    // forward (the output area of the forward pass is g4, overwritten below)
    mlp_forward_tile(d, ws, xin, h1, h2, h3, g4, ns);
    for (int e = threadIdx.x; e < ns * O; e += blockDim.x) g4[e] = gy[(size_t)s0 * O + e];
    __syncthreads();
    back_tile(ws + d.oW4, g4, O, h3, d3, H, ns);
    __syncthreads();
    back_tile(ws + d.oW3, d3, H, h2, d2, H, ns);
    __syncthreads();
    back_tile(ws + d.oW2, d2, H, h1, d1, H, ns);
    __syncthreads();
    if (gw) {
        grad_tile(g4, O, h3, H, gw + d.oW4, gw + d.ob4, ns);
        grad_tile(d3, H, h2, H, gw + d.oW3, gw + d.ob3, ns);
        grad_tile(d2, H, h1, H, gw + d.oW2, gw + d.ob2, ns);
        grad_tile(d1, H, xin, I, gw + d.oW1, gw + d.ob1, ns);
    }
    if (gx) {
        __syncthreads();
        // input gradient: gx[s][k] = sum_j W1[j][k] d1[s][j]; d3 is free now
        back_tile(ws + d.oW1, d1, H, nullptr, d3, I, ns);
        __syncthreads();
        for (int e = threadIdx.x; e < ns * I; e += blockDim.x) gx[(size_t)s0 * I + e] = d3[e];
    }
}

// Mean squared error over N samples x O outputs: loss += sum (y - t)^2 / N,
// gy = 2 (y - t) / N.
__global__ void k_mlp_mse(const float *__restrict__ y, const float *__restrict__ t,
                          float *__restrict__ gy, double *loss, int n, float inv_n) {
    double acc = 0.0;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        const float r = y[e] - t[e];
        gy[e] = 2.f * r * inv_n;
        acc += (double)r * r * inv_n;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, acc);
}

// Adam on the float master weights; refreshes the bf16 copy and clears g.
__global__ void k_mlp_adam(float *__restrict__ w, __nv_bfloat16 *__restrict__ wb,
                           float *__restrict__ g, float *__restrict__ m1, float *__restrict__ m2,
                           int P, float lr, float b1, float b2, float eps, float c1, float c2) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= P) return;
    const float gk = g[k];
    const float a = b1 * m1[k] + (1.f - b1) * gk;
    const float v = b2 * m2[k] + (1.f - b2) * gk * gk;
    m1[k] = a;
    m2[k] = v;
    const float wk = w[k] - lr * (a / c1) / (sqrtf(v / c2) + eps);
    w[k] = wk;
    wb[k] = __float2bfloat16_rn(wk);
    g[k] = 0.f;
}

// out[b][c] = mean over the ny x nx cells of H[b][layer][c] (double sums).
template <typename T>
__global__ void k_layer_mean(const T *__restrict__ H, int L, int cells, int layer, double *out) {
    const int b = blockIdx.y, c = blockIdx.z;
    const T *p = H + (((size_t)b * L + layer) * 3 + c) * cells;
    double acc = 0.0;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < cells; e += gridDim.x * blockDim.x)
        acc += (double)p[e];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(&out[b * 3 + c], acc / cells);
}

}  // namespace demag

using namespace demag;

static demag_status mlp_check(int I, int H, int O) {
    if (I < 1 || H < 1 || O < 1) return fail(DEMAG_EINVAL, "layer widths must be >= 1");
    if (I > kMlpMaxI || H > kMlpMaxH || O > kMlpMaxO)
        return fail(DEMAG_EUNSUPPORTED, "layer widths above 32 inputs, 64 hidden, 8 outputs");
    return DEMAG_OK;
}

extern "C" {

int demag_mlp_param_count(int I, int H, int O) { return mlp_dims(I, H, O).P; }

demag_status demag_mlp_forward(const void *w_bf16, const float *x, float *y, int N, int I, int H,
                               int O, void *stream) {
    demag_status rc = mlp_check(I, H, O);
    if (rc != DEMAG_OK) return rc;
    if (N < 0) return fail(DEMAG_EINVAL, "N must be >= 0");
    if (N == 0) return DEMAG_OK;
    if (!w_bf16 || !x || !y) return fail(DEMAG_EINVAL, "a pointer argument is NULL");
    const MlpDims d = mlp_dims(I, H, O);
    const size_t smem = mlp_smem_floats(d, false) * sizeof(float);
    DEMAG_CUDA(cudaFuncSetAttribute(k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_mlp_forward<<<(N + kMlpTile - 1) / kMlpTile, kMlpThreads, smem, (cudaStream_t)stream>>>(
        (const __nv_bfloat16 *)w_bf16, x, y, N, I, H, O);
    DEMAG_CUDA(cudaGetLastError());
    return DEMAG_OK;
}

demag_status demag_mlp_backward(const void *w_bf16, const float *x, const float *gy, float *gw,
                                float *gx, int N, int I, int H, int O, void *stream) {
    demag_status rc = mlp_check(I, H, O);
    if (rc != DEMAG_OK) return rc;
    if (N < 0) return fail(DEMAG_EINVAL, "N must be >= 0");
    if (N == 0) return DEMAG_OK;
    if (!w_bf16 || !x || !gy || (!gw && !gx)) return fail(DEMAG_EINVAL, "a pointer argument is NULL");
    const MlpDims d = mlp_dims(I, H, O);
    const size_t smem = mlp_smem_floats(d, true) * sizeof(float);
    DEMAG_CUDA(cudaFuncSetAttribute(k_mlp_backward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_mlp_backward<<<(N + kMlpTile - 1) / kMlpTile, kMlpThreads, smem, (cudaStream_t)stream>>>(
        (const __nv_bfloat16 *)w_bf16, x, gy, gw, gx, N, I, H, O);
    DEMAG_CUDA(cudaGetLastError());
    return DEMAG_OK;
}

demag_status demag_mlp_mse(const float *y, const float *target, float *gy, double *loss, int N, int O,
                           void *stream) {
    if (N < 1 || O < 1) return fail(DEMAG_EINVAL, "N and O must be >= 1");
    if (!y || !target || !gy || !loss) return fail(DEMAG_EINVAL, "a pointer argument is NULL");
    const int n = N * O;
    const int grid = (n + 255) / 256 < 256 ? (n + 255) / 256 : 256;
    k_mlp_mse<<<grid, 256, 0, (cudaStream_t)stream>>>(y, target, gy, loss, n, 1.f / (float)N);
    DEMAG_CUDA(cudaGetLastError());
    return DEMAG_OK;
}

demag_status demag_mlp_adam(float *w, void *w_bf16, float *g, float *m1, float *m2, int P, float lr,
                            float beta1, float beta2, float eps, int step, void *stream) {
    if (P < 1 || step < 1) return fail(DEMAG_EINVAL, "P and step must be >= 1");
    if (!w || !w_bf16 || !g || !m1 || !m2) return fail(DEMAG_EINVAL, "a pointer argument is NULL");
    const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
    k_mlp_adam<<<(P + 255) / 256, 256, 0, (cudaStream_t)stream>>>(w, (__nv_bfloat16 *)w_bf16, g, m1, m2, P,
                                                                 lr, beta1, beta2, eps, c1, c2);
    DEMAG_CUDA(cudaGetLastError());
    return DEMAG_OK;
}

demag_status demag_layer_mean(const void *H, int precision, int B, int L, int ny, int nx, int layer,
                              double *out, void *stream) {
    if (!H || !out) return fail(DEMAG_EINVAL, "a pointer argument is NULL");
    if (B < 1 || L < 1 || ny < 1 || nx < 1 || layer < 0 || layer >= L)
        return fail(DEMAG_EINVAL, "bad sizes or layer");
    cudaStream_t st = (cudaStream_t)stream;
    DEMAG_CUDA(cudaMemsetAsync(out, 0, (size_t)B * 3 * sizeof(double), st));
    const int cells = nx * ny;
    dim3 grid((cells + 255) / 256 < 64 ? (cells + 255) / 256 : 64, B, 3);
    if (precision == DEMAG_PREC_FP64)
        k_layer_mean<double><<<grid, 256, 0, st>>>((const double *)H, L, cells, layer, out);
    else
        k_layer_mean<float><<<grid, 256, 0, st>>>((const float *)H, L, cells, layer, out);
    DEMAG_CUDA(cudaGetLastError());
    return DEMAG_OK;
}

}  // extern "C"
