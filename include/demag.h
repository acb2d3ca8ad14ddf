/*
 * demag.h - C ABI of the GB300 (sm_103a) hybrid demagnetization-field library.
 *
 * The library computes the demagnetization field of a stack of magnetic layers
 * that share a regular nx x ny in-plane grid of cells dx x dy but have
 * individual thicknesses t[0..L-1] (the "non-equidistant" case of Sec. 3 of
 * Heistracher et al., "Hybrid FFT algorithm for fast demagnetization field
 * calculations on non-equidistant magnetic layers"):
 *
 *     H_i = -Ms * sum_j N(i <- j) m_j                       (Sec. 3, Eq. Hi_discrete)
 *
 * evaluated as in Eq. FFT_v2: zero-padded 2D FFTs of every layer's
 * magnetization in x and y, an explicit sum over the source layers j at every
 * in-plane frequency with 3x3 generalized-Newell tensor blocks, and an inverse
 * 2D FFT cropped to the grid.  N(i <- j) is the generalized Newell tensor of
 * Sec. 2 (Eqs. Nxx and Nxy, App. A and B) between a target cell of thickness
 * t[i] and a source cell of thickness t[j], normalised by the target volume.
 *
 * Conventions shared by every entry point:
 *   - Layers are stacked contiguously from z = 0 upward; layer 0 is the bottom.
 *     A non-magnetic layer (spacer) is a layer whose m is zero.
 *   - Arrays of vectors are [B][L][3][ny][nx], x fastest, component order
 *     (x, y, z), dense, in the plan's real type (double for DEMAG_PREC_FP64,
 *     float otherwise).  m is dimensionless (unit vectors or zero), Ms and H
 *     in A/m.  Lengths (dx, dy, thickness) in any common unit (the tensor is
 *     dimensionless); nm by convention.
 *   - Device pointers are CUDA device memory of the device that was current
 *     when the plan was created.  "stream" is a cudaStream_t passed as void*
 *     (NULL = the legacy default stream).  Work is ordered on that stream; no
 *     entry point synchronises unless it says so.
 *   - The caller owns every buffer it passes; the plan owns its own device
 *     memory (tensor, workspaces) and frees it in demag_destroy.
 *   - Every entry point returns a demag_status and never aborts.  On failure
 *     demag_last_error() returns a message for the calling host thread.
 *   - A plan may be used by one host thread at a time; applies on different
 *     streams with the same plan share its workspace and must not overlap.
 */
#ifndef DEMAG_H
#define DEMAG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    DEMAG_OK = 0,
    DEMAG_EINVAL = 1,        /* an argument is invalid (size, pointer, value)  */
    DEMAG_ENOMEM = 2,        /* a device or host allocation failed            */
    DEMAG_ECUDA = 3,         /* a CUDA runtime call or kernel launch failed   */
    DEMAG_EUNSUPPORTED = 4   /* valid but outside this build's limits         */
} demag_status;

typedef enum {
    DEMAG_PREC_FP64 = 0,       /* FFTs and layer contraction in double          */
    DEMAG_PREC_FP32 = 1,       /* FFTs and layer contraction in float           */
    DEMAG_PREC_SPLIT_TF32 = 2, /* float FFTs; the contraction as dense products
                                  on the tensor cores in three TF32 passes
                                  (a_hi b_hi + a_hi b_lo + a_lo b_hi, float
                                  accumulation), for batches of states; each
                                  product within 2^-21 of exact              */
    DEMAG_PREC_SPLIT_BF16 = 3  /* the same with three BF16 passes (hi and lo
                                  each 8 significant bits): half the tensor-
                                  core instructions of SPLIT_TF32, each product
                                  within about 3 * 2^-18 of exact (field about
                                  2e-6 relative L2 from the double oracle)   */
} demag_precision;

typedef struct demag_plan *demag_plan_t;

/* Human-readable name of a status code (static string). */
const char *demag_status_string(demag_status status);

/* Detail of the last failure on the calling host thread ("" if none). */
const char *demag_last_error(void);

/*
 * demag_wait_timeouts - count of bounded device waits that gave up.
 *
 * Not a step of the paper's method: a health check of the kernels that stream
 * the plan tensor through shared memory with asynchronous bulk copies.  Each
 * of their waits on a copy is bounded (about one second); a wait that runs out
 * is counted on the device and the kernel completes without hanging, but the
 * field it wrote is then invalid.  This call synchronises the current device
 * and stores in *count the timeouts on that device not yet reported, by this
 * call or by a synchronising entry point (demag_apply_host, demag_apply_timed,
 * demag_thickness_grad: those return DEMAG_ECUDA when they find any).  The
 * asynchronous entry points (demag_apply, demag_apply_adjoint,
 * demag_apply_dthickness, demag_apply_static) cannot report a timeout in
 * their status; poll this call after them.  Returns DEMAG_EINVAL for a NULL
 * count, DEMAG_ECUDA if the counters cannot be read.  A non-zero count means
 * some apply since the previous report produced an invalid field.
 */
demag_status demag_wait_timeouts(unsigned long long *count);

/*
 * demag_selftest_bounded_wait - exercise the bounded-wait path on the GPU.
 *
 * Not a step of the paper's method: a test of the mechanism above.  Launches
 * one thread that waits on a shared-memory barrier which nothing can
 * complete; the wait gives up after limit_cycles SM clock cycles (1 to 2^31)
 * and counts one timeout, which the next demag_wait_timeouts() reports.  The
 * kernel then returns normally: nothing hangs or faults.  Synchronises
 * `stream`.  DEMAG_EINVAL for a limit out of range, DEMAG_ECUDA on a CUDA
 * error.
 */
demag_status demag_selftest_bounded_wait(long long limit_cycles, void *stream);

/*
 * demag_debug_fail_alloc - host-side fault injection for tests.
 *
 * Not a step of the paper's method.  After `after` further device allocations
 * by the library, the next one is refused as if cudaMalloc had run out of
 * memory (the call that needed it returns DEMAG_ENOMEM and frees what it had
 * allocated); the injection then switches itself off.  after < 0 switches it
 * off at once.  Process-wide, not thread-safe; always returns DEMAG_OK.
 */
demag_status demag_debug_fail_alloc(int after);

/*
 * demag_plan_create - build the Fourier-space layer tensor of a layer stack.
 *
 * Sec. 2 (generalized Newell tensor) and Sec. 3 (Eq. FFT_v2).  For every pair
 * of layers (target i, source j) and every in-plane offset (p dx, q dy),
 * |p| < nx, |q| < ny, the six components of N(i <- j) are evaluated in double
 * precision on the GPU, zero-padded onto the circulant grid (the next powers
 * of two >= 2nx and >= 2ny), transformed by a double-precision 2D FFT and
 * stored in the plan's real type.  Far cells, where the closed form loses its
 * digits to cancellation, use a quadrature of the same volume integral.
 *
 *   plan       out: the new plan (unchanged on failure)
 *   nx, ny     in-plane cells, 1 <= nx, ny <= 2048
 *   dx, dy     in-plane cell edges, > 0 and finite
 *   thickness  HOST array of L layer thicknesses, each > 0 and finite
 *   L          number of layers, 1 <= L <= 256
 *   precision  a demag_precision value; DEMAG_PREC_SPLIT_TF32 and
 *              DEMAG_PREC_SPLIT_BF16 need (6 L^2 + 12 L B + 12 L B) floats (L padded to 16, B to 8)
 *              within 220 KB of shared memory, and its tensor is stored in
 *              the blocked layout of demag_plan_tensor
 *   max_batch  largest batch B later passed to demag_apply, >= 1
 *   stream     stream for the set-up work; the call synchronises this stream
 *              before it returns
 *
 * Errors: DEMAG_EINVAL (bad argument), DEMAG_EUNSUPPORTED (limits, or a layer
 * count the precision's contraction kernels do not cover), DEMAG_ENOMEM,
 * DEMAG_ECUDA.
 */
demag_status demag_plan_create(demag_plan_t *plan, int nx, int ny, double dx, double dy,
                               const double *thickness, int L, int precision, int max_batch,
                               void *stream);

/*
 * demag_plan_create_equidistant - plan of the equidistant 3D-FFT method.
 *
 * Sec. 3.1, Eq. FFT_3D: when all nz layers have one thickness dz, N(i <- j)
 * depends on i - j alone and the sum over the source layers is a convolution
 * along z, taken by a third zero-padded FFT of length Pz (the next power of
 * two >= 2 nz) instead of the explicit per-frequency sum of Eq. FFT_v2.  The
 * plan holds the tensor of the 2nz - 1 z-offsets transformed in x, y and z:
 * six real values per (kx, ky, kz) with kx <= Px/2, ky <= Py/2, kz <= Pz/2
 * (the others follow from the parities of the components), built in double
 * like demag_plan_create's.  demag_apply, demag_apply_host, demag_apply_timed
 * and demag_apply_adjoint take the plan unchanged (the same [B][nz][3][ny][nx]
 * arrays; with equal thicknesses the operator is symmetric); the thickness
 * derivatives do not (DEMAG_EUNSUPPORTED).  demag_plan_info reports path 8,
 * the offset count nz in place of the stored pairs and the stored row
 * length Pz/2 + 1 of kz in place of QyS; demag_plan_tensor copies the tensor,
 * layout [kx][ky][kz][component] (float or double, components as in
 * demag_plan_tensor, divided by Px Py Pz).
 *
 *   nx, ny, dx, dy   as for demag_plan_create
 *   nz               number of layers, 1 <= nz <= 256
 *   dz               the common layer thickness, > 0 and finite
 *   precision        DEMAG_PREC_FP64 or DEMAG_PREC_FP32 (else
 *                    DEMAG_EUNSUPPORTED)
 *   max_batch, stream  as for demag_plan_create
 */
demag_status demag_plan_create_equidistant(demag_plan_t *plan, int nx, int ny, int nz, double dx, double dy,
                                           double dz, int precision, int max_batch, void *stream);

/*
 * demag_apply - demagnetization field of B magnetization states.
 *
 * Eq. FFT_v2 read right to left: forward real-to-complex FFT along x of every
 * row, FFT along y, H_k(i) = sum_j N_k(i <- j) m_k(j) at every frequency k,
 * inverse FFT along y, inverse complex-to-real FFT along x cropped to the
 * grid, scaled by -Ms (Eq. Hi_discrete).
 *
 *   m      DEVICE, [B][L][3][ny][nx] of the plan's real type, read only
 *   Ms     saturation magnetization (A/m), finite
 *   H      DEVICE, same shape and type as m, written (must not alias m)
 *   B      1 <= B <= max_batch of the plan
 *   stream stream to order the work on (asynchronous)
 *
 * The status reports argument and launch errors only; a bounded device wait
 * that gave up during the kernels (see demag_wait_timeouts) is reported by
 * demag_wait_timeouts or by the next synchronising entry point.
 */
demag_status demag_apply(demag_plan_t plan, const void *m, double Ms, void *H, int B,
                         void *stream);

/*
 * demag_plan_set_path - choose how the column transforms and the layer
 * contraction run.
 *
 *   path 1: one fused kernel per kx column (the whole column of 3L planes of a
 *           state in shared memory); possible while 3 * L * (Py + 1) complex
 *           values fit 220 KB.
 *   path 2: column FFT, contraction and inverse column FFT as three kernels
 *           through a [Kx][Py][B][L][3] complex workspace (allocated here on
 *           first use).
 *   path 3: (split-precision plans) column kernels of path 2 with the
 *           contraction as dense L x L by L x B products on the FP32 cores.
 *   path 4: (split-precision plans) the same products on the tensor
 *           cores in three TF32 passes (warp-level m16n8k8 TF32 MMAs, two
 *           blocks per SM).
 *   path 5: (reported, not selectable otherwise) the fused column kernel with
 *           the radix-8 512-point transforms, chosen by demag_plan_create
 *           when Py = 512 and the columns fit; its tensor is stored in
 *           natural folded-ky order, so such a plan runs path 5 only.
 *   path 6: (split-precision plans with even L <= 64 and max_batch <= 16;
 *           the default of DEMAG_PREC_SPLIT_TF32 plans) the same products on
 *           the tcgen05 tensor cores: 3xTF32, the tensor operand built in
 *           tensor memory, accumulators in tensor memory, one persistent
 *           block per SM.
 *   path 7: (the same plans; the default of DEMAG_PREC_SPLIT_BF16 plans) path
 *           6 with 3xBF16 operands (kind::f16, K = 16 per instruction).  A
 *           DEMAG_PREC_SPLIT_BF16 plan that takes path 7 at creation stores
 *           its tensor already split (see demag_plan_tensor) and runs path 7
 *           only (DEMAG_EUNSUPPORTED for 3, 4 and 6); a DEMAG_PREC_SPLIT_TF32
 *           plan on path 7 splits its float tensor in the kernel, with the
 *           same operands and the same field, bit for bit.
 *   path 0: the default choice of demag_plan_create (5 or 1 when it fits,
 *           else 2; for split-precision plans 6 (TF32) or 7 (BF16) when it
 *           holds the plan, else 4).
 * All paths compute the same field (Eq. FFT_v2); this entry point exists to
 * test and time them against each other.  Errors: DEMAG_EINVAL, DEMAG_ENOMEM,
 * DEMAG_EUNSUPPORTED (the path cannot hold this plan).
 */
demag_status demag_plan_set_path(demag_plan_t plan, int path);

/*
 * demag_apply_adjoint - vector-Jacobian product of demag_apply in m.
 *
 * demag_apply is linear, H = A m with A_ij = -Ms N(i <- j) (Eq. Hi_discrete),
 * so the gradient of a loss with respect to m is A^T gH.  The transposed
 * blocks follow from the target-volume normalisation of the tensor (Sec. 3):
 * t_i N(i <- j)(d) = t_j N(j <- i)(-d) with symmetric blocks, hence
 * A^T = D_t A D_t^-1, D_t = diag(layer thickness).  The kernels of
 * demag_apply run with the source layers scaled by 1/t_j and the target
 * layers by t_i.
 *
 *   gH     DEVICE, [B][L][3][ny][nx], upstream gradient dLoss/dH
 *   gm     DEVICE, same shape, written: dLoss/dm (must not alias gH)
 *   other arguments as in demag_apply
 */
demag_status demag_apply_adjoint(demag_plan_t plan, const void *gH, double Ms, void *gm, int B,
                                 void *stream);

/*
 * demag_apply_dthickness - derivative of the field with respect to one layer
 * thickness, dH/dt_layer = -Ms sum_j dN(i <- j)/dt_layer m_j.
 *
 * t_layer enters N(i <- j) through the target edge (i == layer), the source
 * edge (j == layer) and the offset z_i - z_j of every pair with exactly one
 * layer above it.  The derivative tensor of all L*L pairs is evaluated in
 * double precision on the GPU (Dual-number closed form of Sec. 2 near the
 * source, the derivative of the far-field volume integral beyond), transformed
 * like the plan tensor, kept in the plan for the last layer asked for (the
 * first call for a layer builds it and synchronises `stream`), and applied
 * with the kernels of demag_apply.
 *
 *   m      DEVICE, [B][L][3][ny][nx], read only
 *   dH     DEVICE, same shape, written (must not alias m)
 *   layer  0 <= layer < L (0 = bottom layer)
 */
demag_status demag_apply_dthickness(demag_plan_t plan, const void *m, double Ms, void *dH, int B,
                                    int layer, void *stream);

/*
 * demag_thickness_grad - dLoss/dt_layer = sum over all cells and states of
 * gH . dH/dt_layer (see demag_apply_dthickness), accumulated in double.
 *
 *   m, gH  DEVICE, [B][L][3][ny][nx]
 *   out    HOST, one double, written
 * Synchronises `stream`; reports bounded-wait timeouts like demag_apply_host.
 */
demag_status demag_thickness_grad(demag_plan_t plan, const void *m, const void *gH, double Ms, int B,
                                  int layer, double *out, void *stream);

/*
 * demag_apply_host - demag_apply on HOST buffers (end-to-end call).
 *
 * With pinned (page-locked) m and H and B >= 2, the batch is copied through
 * the plan's device staging buffers (allocated on first use) in up to four
 * chunks of whole states on a copy stream of the plan, each chunk's input copy
 * overlapping the row transforms of the chunk before it and each output copy
 * the inverse row transforms of the chunk after it.  With one state in
 * pinned, device-mapped buffers the kernels read m from and write H to host
 * memory directly over the host link.  Other host memory is copied through
 * the staging buffers before and after demag_apply.  Every way the call
 * synchronises the stream before it returns and the field is identical.  Returns DEMAG_ECUDA (message in
 * demag_last_error) if a bounded device wait on this device gave up since the
 * timeouts were last reported (see demag_wait_timeouts): the field is then
 * invalid.
 *
 *   m, H   HOST, [B][L][3][ny][nx] of the plan's real type
 *   other arguments as in demag_apply
 */
demag_status demag_apply_host(demag_plan_t plan, const void *m_host, double Ms, void *H_host,
                              int B, void *stream);

/*
 * demag_apply_host_async - demag_apply_host for a stream of batches.
 *
 * The pipelined path of demag_apply_host (page-locked m and H only, else
 * DEMAG_EINVAL), without the synchronisation: the call alternates between two
 * staging sets of the plan (the second allocated on first use) and returns once
 * the copies and kernels are enqueued, so that consecutive calls overlap one
 * batch's input copies and the previous batch's output copies with the
 * kernels.  m_host must stay unchanged and H_host unread until
 * demag_apply_host_wait returns; at most two calls may be outstanding per set
 * of host buffers the caller alternates (a call reuses the staging set of the
 * call two before).  Bounded-wait timeouts are reported by
 * demag_apply_host_wait.
 */
demag_status demag_apply_host_async(demag_plan_t plan, const void *m_host, double Ms, void *H_host,
                                    int B, void *stream);

/*
 * demag_apply_host_wait - wait for every demag_apply_host_async call on the
 * plan (its copy stream) and for `stream`; DEMAG_ECUDA if a bounded device wait
 * gave up meanwhile (see demag_wait_timeouts).
 */
demag_status demag_apply_host_wait(demag_plan_t plan, void *stream);

/*
 * demag_apply_timed - demag_apply with per-kernel device timing.
 *
 * Runs exactly the kernels of demag_apply on the device buffers m and H, with
 * CUDA events recorded on `stream` before the first kernel and after each
 * kernel, then synchronises the stream and writes the elapsed times:
 *   stage_ms (HOST, nstage values, nstage >= 3):
 *     [0] forward row transforms, [1] column transforms + layer contraction,
 *     [2] inverse row transforms (milliseconds, CUDA event resolution);
 *     with nstage >= 6 on a plan running the split path (2, 3, 4) also
 *     [3] forward column transforms, [4] layer contraction, [5] inverse
 *     column transforms (the parts of [1]); zero otherwise.
 * Other arguments as in demag_apply.  Reports bounded-wait timeouts like
 * demag_apply_host.
 */
demag_status demag_apply_timed(demag_plan_t plan, const void *m, double Ms, void *H, int B,
                               void *stream, float *stage_ms, int nstage);

/*
 * demag_plan_info - sizes of a plan.
 *
 * out (HOST, 10 values): {nx, ny, L, Px, Py, precision, max_batch,
 *                         number of stored layer pairs, stored row length QyS,
 *                         column path: 1 fused, 2 split, 3/4/6/7
 *                         split-precision variants, 5 fused 512-point}
 * Px, Py are the padded FFT sizes; the stored tensor holds the layer pairs
 * i <= j (the rest follow from reciprocity, t_i N(i<-j)(d) = t_j N(j<-i)(-d)).
 */
demag_status demag_plan_info(demag_plan_t plan, long long *out);

/*
 * demag_plan_compress - drop the negligible layer blocks of a split-precision
 * plan's tensor (a block-sparse compressed tensor).
 *
 * Sec. 3.2: the hybrid's cost grows with the layer pairs, whose tensor the
 * contraction streams once per apply.  In the in-plane Fourier domain the
 * coupling of two layers decays like exp(-|k| Z) with their distance Z, so
 * at high frequencies the 8 x 8 blocks of distant layers hold values far
 * below float resolution.  This call keeps, entry by entry, only the blocks
 * with a value of at least tol times the largest value of its component in
 * the whole tensor, and stores them contiguously with a 64-bit block mask and
 * an offset per entry; the contraction then neither reads nor multiplies the
 * dropped blocks' values (they count as zero).
 *
 *   plan          a DEMAG_PREC_SPLIT_TF32 or DEMAG_PREC_SPLIT_BF16 plan on
 *                 path 6 or 7 (even L <= 64, max_batch <= 16)
 *   tol           0 <= tol < 1; 0 keeps every block that holds a nonzero
 *   stored_bytes  out (may be NULL): bytes of the compressed tensor
 *
 * The call synchronises the device and replaces the plan's tensor.  After it
 * the plan runs paths 6 and 7 only, and demag_plan_tensor refuses.  Errors:
 * DEMAG_EINVAL (NULL plan, tol outside [0, 1)), DEMAG_EUNSUPPORTED (another
 * precision or path, or already compressed), DEMAG_ENOMEM / DEMAG_ECUDA
 * (the plan keeps its uncompressed tensor).
 */
demag_status demag_plan_compress(demag_plan_t plan, double tol, size_t *stored_bytes);

/*
 * Frequency-sharded apply: the three steps of Eq. FFT_v2 as separate calls, so
 * that several processes (one GPU each) can share one apply.  The row
 * transforms (x) work plane by plane, a plane being one (state, layer,
 * component) of m, plane index p = (b * L + l) * 3 + c; the column transforms
 * (y), the sum over source layers and the inverse column transforms work kx
 * by kx over every plane.  A rank transforms the rows of its planes, an
 * all-to-all (the caller's: NCCL, gloo, copies) gives each rank every plane
 * at its own x-frequencies, each rank runs its slab with only that slab of the
 * tensor, a second all-to-all returns the slabs, and each rank runs the
 * inverse row transforms of its planes.  The result is that of demag_apply,
 * bit for bit: every column, entry and row is computed by the same kernels.
 * Sec. 3.1 defines the steps; the split among ranks is this library's.
 *
 * The row spectrum of a plane is Kx = Px / 2 + 1 x-frequencies of ny complex
 * values each (frequency-major: [kx][y]); complex values are two reals of the
 * plan's type (float, or double for DEMAG_PREC_FP64), interleaved.  Every
 * pointer is DEVICE memory on the plan's device, owned by the caller; the calls
 * are asynchronous on `stream` (NULL: the legacy default stream) and report
 * bounded-wait timeouts like demag_apply.
 */

/*
 * demag_plan_keep_slab - keep only the x-frequencies k0 <= kx < k1 of the
 * plan's tensor, freeing the rest, and shrink its column workspace to them
 * (where the smaller workspace can be allocated; else the full one stays).
 *
 *   plan     a hybrid plan on the split path (DEMAG_PREC_SPLIT_TF32 or
 *            DEMAG_PREC_SPLIT_BF16 plans, or another plan after
 *            demag_plan_set_path(plan, 2)); not compressed
 *   k0, k1   0 <= k0 < k1 <= Px / 2 + 1
 *
 * Synchronises the device.  Afterwards the plan runs demag_columns_slab on
 * sub-ranges of [k0, k1) and the row calls below; demag_apply and every call
 * built on it return DEMAG_EUNSUPPORTED, and demag_plan_tensor copies out the
 * slab.  Errors: DEMAG_EINVAL (NULL plan, range), DEMAG_EUNSUPPORTED (another
 * path or method, a compressed tensor, already a slab), DEMAG_ENOMEM /
 * DEMAG_ECUDA (the slab's copy could not be made: the plan is unchanged).
 */
demag_status demag_plan_keep_slab(demag_plan_t plan, int k0, int k1);

/*
 * demag_rows_forward - forward row transforms (x) of planes p0 <= p < p1.
 *
 *   m     the batch's magnetisation [B][L][3][ny][nx] (the layout of
 *         demag_apply); planes p0 .. p1 - 1 are read
 *   spec  out: [p1 - p0][Kx][ny] complex, the planes' row spectra
 *   0 <= p0 < p1 <= max_batch * L * 3
 *
 * Errors: DEMAG_EINVAL (NULL pointer, plane range), DEMAG_ECUDA.
 */
demag_status demag_rows_forward(demag_plan_t plan, const void *m, int p0, int p1, void *spec, void *stream);

/*
 * demag_columns_slab - column transforms, layer sum (Eq. FFT_v2) and inverse
 * column transforms of every plane at the x-frequencies k0 <= kx < k1, in place.
 *
 *   spec  in/out: [B * L * 3][k1 - k0][ny] complex, the row spectra of all
 *         planes of a batch of B states at those x-frequencies
 *   k0, k1  within the plan's tensor (all of [0, Px / 2 + 1), or the range
 *           kept by demag_plan_keep_slab)
 *   B     states, 1 <= B <= max_batch
 *
 * Uses the plan's column workspace: calls on one plan must not overlap on the
 * GPU.  Errors: DEMAG_EINVAL (NULL pointer, range, B), DEMAG_EUNSUPPORTED (a
 * plan off the split path, equidistant or compressed), DEMAG_ECUDA.
 */
demag_status demag_columns_slab(demag_plan_t plan, void *spec, int k0, int k1, int B, void *stream);

/*
 * demag_rows_inverse - inverse row transforms of planes p0 <= p < p1, cropped
 * to nx and scaled by -Ms (the stored tensor carries the 1 / (Px Py) of the
 * inverse transforms): the field H = -Ms N * m of Eq. FFT_v2.
 *
 *   spec  [p1 - p0][Kx][ny] complex, the planes' row spectra after the column
 *         steps (read only)
 *   H     out: the batch's field [B][L][3][ny][nx]; planes p0 .. p1 - 1 are
 *         written
 *
 * Errors: DEMAG_EINVAL (NULL pointer, plane range, Ms not finite), DEMAG_ECUDA.
 */
demag_status demag_rows_inverse(demag_plan_t plan, const void *spec, int p0, int p1, double Ms, void *H,
                                void *stream);

/*
 * demag_plan_tensor - copy of the stored Fourier-space tensor.
 *
 * out DEVICE, (Px/2+1) * npairs * 6 * QyS values of the plan's real type,
 * layout [kx][pair][component][u] (split-precision plans:
 * (Px/2+1) * (Py/2+1) * NB floats, layout [kx][u][component][block][row][col]
 * with nb = ceil(L/8) layer blocks and NB = 6 * 64 * nb (nb + 1) / 2: each
 * component row holds the 8 x 8 blocks (R <= C) of M(i, j) = (t_i / t_0)
 * N(i <- j), block row by block row, element (i mod 8, j mod 8) of block
 * (R, C) = (i / 8, j / 8) at float 32 h + 4 (a XOR (C mod 4) XOR 4 h) + (b mod
 * 4) of the block, a = i mod 8, b = j mod 8, h = b / 4 (the block's left
 * half-rows, then its right half-rows, in an order that spreads the
 * contraction's row and column reads over the shared-memory banks); a
 * diagonal block holds both triangles, M(i, j) for i > j
 * being M(j, i) with the xz and yz components negated; layers past L zero;
 * a DEMAG_PREC_SPLIT_BF16 plan on path 7 holds in each 32-bit slot, in place
 * of the float v, its BF16 split pair hi << 16 | lo, hi = bf16(v), lo = bf16(v
 * - hi), both rounded to nearest even, with v = -M(i, j) for the zz
 * component)
 * with pair (i <= j) numbered row by row
 * (i = 0: j = 0..L-1, then i = 1: j = 1..L-1, ...) and components
 * {Re N_xx, Re N_yy, Re N_zz, Re N_xy, Im N_xz, Im N_yz} of the 2D DFT of
 * N(i <- j) on the padded grid, divided by Px*Py.  Entry u < Py/2 + 1 holds
 * the y-frequency ky(u) = min(k, Py - k), k = bitrev(p1(u)) over log2(Py)
 * bits, where p1(0) = 0, p1(1) = 1 and, for u in [2^(m-1)+1, 2^m+1),
 * p1(u) = 2^m + u - 2^(m-1) - 1: the order in which a decimation-in-frequency
 * column transform leaves the spectrum; plans whose columns run the
 * 512-point radix-8 kernel (Py = 512, fused) hold entry u at ky(u) = u
 * instead.  Entries u >= Py/2 + 1 (padding up
 * to QyS, a multiple of 16 bytes) are zero.  bytes is the size of out.
 * Asynchronous on stream.
 */
demag_status demag_plan_tensor(demag_plan_t plan, void *out, size_t bytes, void *stream);

/*
 * demag_tensor_points - the generalized Newell tensor at arbitrary geometries.
 *
 * Sec. 2, Eqs. Nxx and Nxy with App. A/B (closed form, double precision) for
 * near pairs of cuboids, and a composite Gauss-Legendre quadrature of the
 * defining volume integral (Eq. demag_tensor) for pairs further apart than the
 * larger in-plane edge.  This is the evaluation the plan builder uses.
 *
 *   n      number of points, >= 0
 *   geom   DEVICE double [n][9]: X, Y, Z (target corner minus source corner),
 *          target edges tx, ty, tz, source edges sx, sy, sz (all edges > 0)
 *   out    DEVICE double [n][6]: N_xx, N_yy, N_zz, N_xy, N_xz, N_yz of
 *          N(target <- source), normalised by the target volume
 */
demag_status demag_tensor_points(int n, const double *geom, double *out, void *stream);

/*
 * demag_apply_static - demag_apply for callers that cannot allocate device
 * memory.  The paper has no counterpart: this is a deployment variant of the
 * same kernels.
 *
 * Some callers must not call cudaMalloc while they run: code embedded in a
 * host framework whose allocator has reserved the GPU's memory (a cudaMalloc
 * there can fail or fragment that pool), or a time-critical loop that cannot
 * take the device-wide synchronisation an allocation may cause.  This entry
 * point allocates nothing.  The caller passes the Fourier tensor (prepared
 * earlier, e.g. by demag_plan_create + demag_plan_tensor into memory the caller
 * owns), the layer thicknesses, m and H; the spectrum workspace, twiddle tables
 * and reciprocity ratios live in one fixed 32 MiB device array inside the
 * library (held on every GPU that loads the library until the process exits).
 *
 *   tensor     DEVICE, 16-byte aligned, layout and values exactly as written
 *              by demag_plan_tensor for a plan of the same nx, ny, thickness,
 *              precision (any max_batch)
 *   tensor_bytes  size of tensor in bytes: must equal the size
 *              demag_plan_tensor writes for such a plan
 *              ((Px/2+1) * npairs * 6 * QyS values), else DEMAG_EINVAL
 *   thickness  HOST, L layer thicknesses (same as for that plan)
 *   nx, ny, L, precision   as for demag_plan_create (DEMAG_PREC_FP64 or
 *              DEMAG_PREC_FP32)
 *   m, Ms, H, B, stream    as for demag_apply (no max_batch: the scratch size
 *              is the limit)
 *
 * Scratch needed: B*L*3*(Px/2+1)*ny complex values of the precision plus the
 * twiddle tables and an L*L ratio table; a request above 32 MiB returns
 * DEMAG_EUNSUPPORTED with the required size in demag_last_error().
 * The first call on a device looks up the array's device address (a one-time
 * set-up per device, repeated after a call on that device fails); make that
 * first call before any stream capture.  All calls on a device share the
 * array: calls whose GPU work overlaps (other streams, other host threads)
 * race on it; calls ordered on one stream do not.  Every call recomputes the
 * small tables on the device and overwrites the workspace it reads, so
 * nothing in the array needs clearing between calls.  The call copies nothing
 * from host memory; the thicknesses travel as a kernel argument.
 */
demag_status demag_apply_static(const void *tensor, size_t tensor_bytes, const double *thickness,
                                int nx, int ny, int L, int precision, const void *m, double Ms, void *H,
                                int B, void *stream);

/*
 * demag_tensor_points_dt - the tensor of demag_tensor_points and its
 * derivative along (dtz, dsz, dZ): the target z-edge, the source z-edge and
 * the z-offset move at these rates.
 *
 *   geom   DEVICE double [n][12]: X, Y, Z, tx, ty, tz, sx, sy, sz, dtz, dsz, dZ
 *   out    DEVICE double [n][6]: the tensor
 *   dout   DEVICE double [n][6]: its derivative
 */
demag_status demag_tensor_points_dt(int n, const double *geom, double *out, double *dout,
                                    void *stream);

/*
 * Surrogate network for the thickness optimisation of Sec. 4 (the paper runs
 * Newton on one layer thickness to zero the mean z-field of the free layer;
 * the surrogate proposes those steps and the solver accepts or rejects them).
 *
 * A multilayer perceptron with I inputs, three tanh hidden layers of H units
 * and O linear outputs (I <= 32, H <= 64, O <= 8):
 *   h1 = tanh(W1 x + b1), h2 = tanh(W2 h1 + b2), h3 = tanh(W3 h2 + b3),
 *   y = W4 h3 + b4.
 * Parameters form one vector of demag_mlp_param_count(I, H, O) values:
 *   W1 [H][I], b1 [H], W2 [H][H], b2 [H], W3 [H][H], b3 [H], W4 [O][H], b4 [O]
 * (row-major W[out][in]).  Compute reads them as bfloat16 (w_bf16, DEVICE,
 * 16-bit values) and accumulates in float; the optimiser keeps a float master
 * copy.  x: DEVICE float [N][I]; y, gy: DEVICE float [N][O].
 */
int demag_mlp_param_count(int I, int H, int O);

/* y = network(x) for N samples. */
demag_status demag_mlp_forward(const void *w_bf16, const float *x, float *y, int N, int I, int H,
                               int O, void *stream);

/*
 * Back-propagation of gy = dLoss/dy through the network at x:
 *   gw (DEVICE float [P], may be NULL): dLoss/dparameters ADDED to gw;
 *   gx (DEVICE float [N][I], may be NULL): dLoss/dx written.
 */
demag_status demag_mlp_backward(const void *w_bf16, const float *x, const float *gy, float *gw,
                                float *gx, int N, int I, int H, int O, void *stream);

/* Mean squared error: *loss (DEVICE double) += sum (y - target)^2 / N;
 * gy = 2 (y - target) / N. */
demag_status demag_mlp_mse(const float *y, const float *target, float *gy, double *loss, int N, int O,
                           void *stream);

/* One Adam step on the float master weights w (DEVICE float [P]) with moments
 * m1, m2 and gradient g; refreshes w_bf16 (round to nearest even) and sets g
 * to zero.  step >= 1 is the bias-correction count. */
demag_status demag_mlp_adam(float *w, void *w_bf16, float *g, float *m1, float *m2, int P, float lr,
                            float beta1, float beta2, float eps, int step, void *stream);

/* out (DEVICE double [B][3]) = mean over the ny x nx cells of layer `layer` of
 * the field H ([B][L][3][ny][nx], float or double by precision): the mean
 * free-layer field the surrogate learns (Sec. 4's objective). */
demag_status demag_layer_mean(const void *H, int precision, int B, int L, int ny, int nx, int layer,
                              double *out, void *stream);

/*
 * Micromagnetic relaxation of one layer (Sec. 4: the free layer of the MRAM
 * cell is relaxed by a limited-memory BFGS energy minimisation at every
 * applied field of an easy-axis hysteresis loop, the other layers pinned).
 *
 * Energy of the relaxed layer (SI units, V the cell volume, fields in tesla):
 *   exchange    A V sum over in-plane neighbour pairs inside the mask of
 *               |m_j - m_i|^2 / d^2 (free surfaces at the mask's edge)
 *   anisotropy  -Ku V sum_i m_z,i^2 (uniaxial, easy axis z)
 *   Zeeman      -(Js / mu0) V sum_i m_i . b_ext
 *   demag       -(Js / mu0) V sum_i m_i . (b_self,i / 2 + b_bias,i), b_self the
 *               field of the layer's own magnetization and b_bias that of the
 *               other layers, both from demag_apply with Ms = Js / mu0 (one
 *               saturation magnetization for every magnetic layer).
 * The unit vectors are parametrized as m = v / |v|; L-BFGS with the given
 * history and Armijo backtracking; stop when max_i |m_i x b_eff,i| <
 * tol_torque (tesla), when no step lowers the energy (converged to the
 * rounding of its sum), or after max_iter iterations.
 */
typedef struct {
    double Js;           /* mu0 Ms (T), > 0 */
    double A_ex;         /* exchange constant (J/m), >= 0 */
    double Ku;           /* uniaxial anisotropy along z (J/m^3) */
    double b_ext[3];     /* applied field mu0 H (T) */
    double length_unit;  /* metres per length unit of the plan (1e-9 for nm) */
    double tol_torque;   /* stopping torque (T), > 0 */
    int max_iter;        /* >= 0 */
    int history;         /* L-BFGS pairs kept, 1..32 */
} demag_relax_params;

typedef struct {
    int iterations;      /* L-BFGS iterations taken */
    int evaluations;     /* energy and field evaluations (one demag_apply each) */
    int converged;       /* 1 torque below tolerance, 2 energy at its rounding, 0 max_iter */
    double energy;       /* energy of the relaxed layer (J) */
    double max_torque;   /* max_i |m_i x b_eff,i| (T) at the end */
} demag_relax_stats;

/*
 * demag_relax_layer - relax layer `layer` of m in place.
 *
 *   plan    a DEMAG_PREC_FP64 or DEMAG_PREC_FP32 plan of demag_plan_create
 *           (max_batch >= 1; one state)
 *   m       DEVICE, [L][3][ny][nx] of the plan's real type: the other layers
 *           are read (pinned), layer `layer` is read as the start and
 *           overwritten by the relaxed unit vectors (zero outside the mask)
 *   mask    DEVICE, [ny][nx] bytes: nonzero for magnetic cells of the layer
 *   params  HOST, see demag_relax_params
 *   stats   HOST, may be NULL
 * Allocates its workspace (about 2 + 2 history vectors of 3 nx ny doubles and
 * three stacks) for the call and synchronises `stream`.  Errors: DEMAG_EINVAL
 * (arguments), DEMAG_EUNSUPPORTED (split-precision or equidistant plan),
 * DEMAG_ENOMEM, DEMAG_ECUDA.
 */
demag_status demag_relax_layer(demag_plan_t plan, void *m, int layer, const unsigned char *mask,
                               const demag_relax_params *params, demag_relax_stats *stats, void *stream);

/* demag_destroy - free a plan (NULL is accepted).  Synchronises the device. */
demag_status demag_destroy(demag_plan_t plan);

#ifdef __cplusplus
}
#endif

#endif /* DEMAG_H */
