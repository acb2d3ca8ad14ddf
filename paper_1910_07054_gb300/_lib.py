"""ctypes binding of libdemag (``include/demag.h``): argument marshalling only.

Every function here has the name of the C entry point it calls and does no
arithmetic of the method: it checks tensor shapes, dtypes and devices, passes
raw pointers and the current CUDA stream, and raises ``DemagError`` on a
non-zero status.  The library is built in-tree by ``build.py`` and loaded from
``_build/libdemag.so``; if it cannot be built or loaded, every call raises.
"""
import ctypes
import os

from . import build as _build

DEMAG_OK, DEMAG_EINVAL, DEMAG_ENOMEM, DEMAG_ECUDA, DEMAG_EUNSUPPORTED = range(5)
PREC_FP64, PREC_FP32, PREC_SPLIT_TF32, PREC_SPLIT_BF16 = 0, 1, 2, 3

_lib = None


class RelaxParams(ctypes.Structure):
    """demag_relax_params of include/demag.h."""
    _fields_ = [("Js", ctypes.c_double), ("A_ex", ctypes.c_double), ("Ku", ctypes.c_double),
                ("b_ext", ctypes.c_double * 3), ("length_unit", ctypes.c_double), ("tol_torque", ctypes.c_double),
                ("max_iter", ctypes.c_int), ("history", ctypes.c_int)]


class RelaxStats(ctypes.Structure):
    """demag_relax_stats of include/demag.h."""
    _fields_ = [("iterations", ctypes.c_int), ("evaluations", ctypes.c_int), ("converged", ctypes.c_int),
                ("energy", ctypes.c_double), ("max_torque", ctypes.c_double)]


class DemagError(RuntimeError):
    def __init__(self, status, where, detail):
        self.status = status
        super().__init__("%s failed: %s (%s)" % (where, _status_name(status), detail))


def _status_name(s):
    return {0: "DEMAG_OK", 1: "DEMAG_EINVAL", 2: "DEMAG_ENOMEM", 3: "DEMAG_ECUDA",
            4: "DEMAG_EUNSUPPORTED"}.get(s, "status %d" % s)


def library_path():
    return _build.LIB


def lib():
    """Load (building first if needed) libdemag.so; raises if that is impossible."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build()
    if not os.path.exists(path):
        raise RuntimeError("libdemag.so is missing at %s" % path)
    L = ctypes.CDLL(path)
    vp, i, d, dp = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.POINTER(ctypes.c_double)
    L.demag_status_string.argtypes = [i]
    L.demag_status_string.restype = ctypes.c_char_p
    L.demag_last_error.argtypes = []
    L.demag_last_error.restype = ctypes.c_char_p
    L.demag_plan_create.argtypes = [ctypes.POINTER(vp), i, i, d, d, dp, i, i, i, vp]
    L.demag_plan_create.restype = i
    L.demag_plan_create_equidistant.argtypes = [ctypes.POINTER(vp), i, i, i, d, d, d, i, i, vp]
    L.demag_plan_create_equidistant.restype = i
    L.demag_apply.argtypes = [vp, vp, d, vp, i, vp]
    L.demag_apply.restype = i
    L.demag_apply_timed.argtypes = [vp, vp, d, vp, i, vp, ctypes.POINTER(ctypes.c_float), i]
    L.demag_apply_timed.restype = i
    L.demag_apply_host.argtypes = [vp, vp, d, vp, i, vp]
    L.demag_apply_host.restype = i
    L.demag_apply_host_async.argtypes = [vp, vp, d, vp, i, vp]
    L.demag_apply_host_async.restype = i
    L.demag_apply_host_wait.argtypes = [vp, vp]
    L.demag_apply_host_wait.restype = i
    L.demag_plan_info.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong)]
    L.demag_plan_info.restype = i
    L.demag_plan_tensor.argtypes = [vp, vp, ctypes.c_size_t, vp]
    L.demag_plan_tensor.restype = i
    L.demag_plan_compress.argtypes = [vp, d, ctypes.POINTER(ctypes.c_size_t)]
    L.demag_plan_compress.restype = i
    L.demag_plan_keep_slab.argtypes = [vp, i, i]
    L.demag_plan_keep_slab.restype = i
    L.demag_rows_forward.argtypes = [vp, vp, i, i, vp, vp]
    L.demag_rows_forward.restype = i
    L.demag_columns_slab.argtypes = [vp, vp, i, i, i, vp]
    L.demag_columns_slab.restype = i
    L.demag_rows_inverse.argtypes = [vp, vp, i, i, d, vp, vp]
    L.demag_rows_inverse.restype = i
    L.demag_tensor_points.argtypes = [i, vp, vp, vp]
    L.demag_tensor_points.restype = i
    L.demag_plan_set_path.argtypes = [vp, i]
    L.demag_plan_set_path.restype = i
    L.demag_apply_adjoint.argtypes = [vp, vp, d, vp, i, vp]
    L.demag_apply_adjoint.restype = i
    L.demag_apply_dthickness.argtypes = [vp, vp, d, vp, i, i, vp]
    L.demag_apply_dthickness.restype = i
    L.demag_thickness_grad.argtypes = [vp, vp, vp, d, i, i, dp, vp]
    L.demag_thickness_grad.restype = i
    L.demag_tensor_points_dt.argtypes = [i, vp, vp, vp, vp]
    L.demag_tensor_points_dt.restype = i
    L.demag_apply_static.argtypes = [vp, ctypes.c_size_t, dp, i, i, i, i, vp, d, vp, i, vp]
    L.demag_apply_static.restype = i
    f = ctypes.c_float
    L.demag_mlp_param_count.argtypes = [i, i, i]
    L.demag_mlp_param_count.restype = i
    L.demag_mlp_forward.argtypes = [vp, vp, vp, i, i, i, i, vp]
    L.demag_mlp_forward.restype = i
    L.demag_mlp_backward.argtypes = [vp, vp, vp, vp, vp, i, i, i, i, vp]
    L.demag_mlp_backward.restype = i
    L.demag_mlp_mse.argtypes = [vp, vp, vp, vp, i, i, vp]
    L.demag_mlp_mse.restype = i
    L.demag_mlp_adam.argtypes = [vp, vp, vp, vp, vp, i, f, f, f, f, i, vp]
    L.demag_mlp_adam.restype = i
    L.demag_layer_mean.argtypes = [vp, i, i, i, i, i, i, vp, vp]
    L.demag_layer_mean.restype = i
    L.demag_relax_layer.argtypes = [vp, vp, i, vp, ctypes.POINTER(RelaxParams), ctypes.POINTER(RelaxStats), vp]
    L.demag_relax_layer.restype = i
    L.demag_destroy.argtypes = [vp]
    L.demag_destroy.restype = i
    L.demag_wait_timeouts.argtypes = [ctypes.POINTER(ctypes.c_ulonglong)]
    L.demag_wait_timeouts.restype = i
    L.demag_selftest_bounded_wait.argtypes = [ctypes.c_longlong, vp]
    L.demag_selftest_bounded_wait.restype = i
    L.demag_debug_fail_alloc.argtypes = [i]
    L.demag_debug_fail_alloc.restype = i
    _lib = L
    return L


def _check(status, where):
    if status != DEMAG_OK:
        detail = lib().demag_last_error().decode(errors="replace")
        raise DemagError(status, where, detail)


def _stream(stream):
    """cudaStream_t of a torch stream (or the current stream) as void*."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def demag_status_string(status):
    return lib().demag_status_string(int(status)).decode()


def demag_last_error():
    return lib().demag_last_error().decode(errors="replace")


def demag_plan_create(nx, ny, dx, dy, thickness, precision=PREC_FP32, max_batch=1, stream=None):
    """Returns an opaque plan handle (int).  thickness: sequence of L floats."""
    th = (ctypes.c_double * len(thickness))(*[float(t) for t in thickness])
    handle = ctypes.c_void_p()
    _check(lib().demag_plan_create(ctypes.byref(handle), int(nx), int(ny), float(dx), float(dy), th,
                                   len(thickness), int(precision), int(max_batch), _stream(stream)),
           "demag_plan_create")
    return handle.value


def demag_plan_create_equidistant(nx, ny, nz, dx, dy, dz, precision=PREC_FP32, max_batch=1, stream=None):
    """Plan of the equidistant 3D-FFT method (nz layers of thickness dz)."""
    handle = ctypes.c_void_p()
    _check(lib().demag_plan_create_equidistant(ctypes.byref(handle), int(nx), int(ny), int(nz), float(dx), float(dy),
                                               float(dz), int(precision), int(max_batch), _stream(stream)),
           "demag_plan_create_equidistant")
    return handle.value


def demag_plan_info(plan):
    out = (ctypes.c_longlong * 10)()
    _check(lib().demag_plan_info(ctypes.c_void_p(plan), out), "demag_plan_info")
    keys = ("nx", "ny", "L", "Px", "Py", "precision", "max_batch", "npairs", "QyS", "path")
    return dict(zip(keys, [int(v) for v in out]))


def _field_check(t, info, name, device=True):
    import torch
    want = torch.float64 if info["precision"] == PREC_FP64 else torch.float32  # split-TF32: float
    if t.dtype != want:
        raise TypeError("%s must be %s for this plan, got %s" % (name, want, t.dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if device and not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor" % name)
    if not device and t.is_cuda:
        raise ValueError("%s must be a host tensor" % name)
    shape = tuple(t.shape)
    tail = (info["L"], 3, info["ny"], info["nx"])
    if shape[-4:] != tail or len(shape) not in (4, 5):
        raise ValueError("%s must have shape [B, %d, 3, %d, %d] or [%d, 3, %d, %d], got %s"
                         % (name, tail[0], tail[2], tail[3], tail[0], tail[2], tail[3], shape))
    return 1 if len(shape) == 4 else shape[0]


def demag_apply(plan, m, Ms, H, stream=None, info=None):
    """H <- demag field of m (device tensors of the plan's dtype, [B, L, 3, ny, nx])."""
    info = info or demag_plan_info(plan)
    B = _field_check(m, info, "m")
    if _field_check(H, info, "H") != B or H.shape != m.shape:
        raise ValueError("H must have the shape of m")
    _check(lib().demag_apply(ctypes.c_void_p(plan), ctypes.c_void_p(m.data_ptr()), float(Ms),
                             ctypes.c_void_p(H.data_ptr()), int(B), _stream(stream)), "demag_apply")
    return H


def demag_plan_set_path(plan, path):
    """0: the plan's default; 1: fused column kernel, 2: split column kernels;
    split-precision plans: 3 (FP32 cores), 4 (warp-level TF32 MMAs), 6 (tcgen05,
    3xTF32), 7 (tcgen05, 3xBF16); 6 or 7 is the default of DEMAG_PREC_SPLIT_TF32
    or DEMAG_PREC_SPLIT_BF16 plans where it holds the plan.  See
    demag_plan_set_path in demag.h."""
    _check(lib().demag_plan_set_path(ctypes.c_void_p(plan), int(path)), "demag_plan_set_path")


def demag_apply_adjoint(plan, gH, Ms, gm, stream=None, info=None):
    """gm <- A^T gH, the vector-Jacobian product of demag_apply in m."""
    info = info or demag_plan_info(plan)
    B = _field_check(gH, info, "gH")
    if _field_check(gm, info, "gm") != B or gm.shape != gH.shape:
        raise ValueError("gm must have the shape of gH")
    _check(lib().demag_apply_adjoint(ctypes.c_void_p(plan), ctypes.c_void_p(gH.data_ptr()), float(Ms),
                                     ctypes.c_void_p(gm.data_ptr()), int(B), _stream(stream)),
           "demag_apply_adjoint")
    return gm


def demag_apply_dthickness(plan, m, Ms, dH, layer, stream=None, info=None):
    """dH <- dH/dt_layer for the states m."""
    info = info or demag_plan_info(plan)
    B = _field_check(m, info, "m")
    if _field_check(dH, info, "dH") != B or dH.shape != m.shape:
        raise ValueError("dH must have the shape of m")
    _check(lib().demag_apply_dthickness(ctypes.c_void_p(plan), ctypes.c_void_p(m.data_ptr()), float(Ms),
                                        ctypes.c_void_p(dH.data_ptr()), int(B), int(layer),
                                        _stream(stream)), "demag_apply_dthickness")
    return dH


def demag_thickness_grad(plan, m, gH, Ms, layer, stream=None, info=None):
    """sum(gH * dH/dt_layer) as a float (synchronises)."""
    info = info or demag_plan_info(plan)
    B = _field_check(m, info, "m")
    if _field_check(gH, info, "gH") != B or gH.shape != m.shape:
        raise ValueError("gH must have the shape of m")
    out = ctypes.c_double()
    _check(lib().demag_thickness_grad(ctypes.c_void_p(plan), ctypes.c_void_p(m.data_ptr()),
                                      ctypes.c_void_p(gH.data_ptr()), float(Ms), int(B), int(layer),
                                      ctypes.byref(out), _stream(stream)), "demag_thickness_grad")
    return out.value


def demag_tensor_points_dt(geom, out, dout, stream=None):
    """geom: CUDA float64 [n, 12]; out, dout: CUDA float64 [n, 6]."""
    import torch
    for t in (geom, out, dout):
        if t.dtype != torch.float64 or not t.is_cuda:
            raise TypeError("geom, out and dout must be CUDA float64 tensors")
    if geom.shape[-1] != 12 or out.shape[-1] != 6 or dout.shape != out.shape or geom.shape[0] != out.shape[0]:
        raise ValueError("geom must be [n, 12], out and dout [n, 6]")
    _check(lib().demag_tensor_points_dt(int(geom.shape[0]), ctypes.c_void_p(geom.data_ptr()),
                                        ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(dout.data_ptr()),
                                        _stream(stream)), "demag_tensor_points_dt")
    return out, dout


def demag_apply_timed(plan, m, Ms, H, stream=None, info=None):
    """demag_apply with per-kernel event times (ms): [rows fwd, columns, rows inv,
    and for split plans: column fwd, contraction, column inv (else 0)]."""
    info = info or demag_plan_info(plan)
    B = _field_check(m, info, "m")
    if _field_check(H, info, "H") != B or H.shape != m.shape:
        raise ValueError("H must have the shape of m")
    ms = (ctypes.c_float * 6)()
    _check(lib().demag_apply_timed(ctypes.c_void_p(plan), ctypes.c_void_p(m.data_ptr()), float(Ms),
                                   ctypes.c_void_p(H.data_ptr()), int(B), _stream(stream), ms, 6),
           "demag_apply_timed")
    return [float(v) for v in ms]


def demag_apply_host(plan, m, Ms, H, stream=None, info=None):
    """demag_apply on host tensors (pinned for full copy speed); synchronises."""
    info = info or demag_plan_info(plan)
    B = _field_check(m, info, "m", device=False)
    if _field_check(H, info, "H", device=False) != B or H.shape != m.shape:
        raise ValueError("H must have the shape of m")
    _check(lib().demag_apply_host(ctypes.c_void_p(plan), ctypes.c_void_p(m.data_ptr()), float(Ms),
                                  ctypes.c_void_p(H.data_ptr()), int(B), _stream(stream)),
           "demag_apply_host")
    return H


def demag_apply_host_async(plan, m, Ms, H, stream=None, info=None):
    """Enqueue demag_apply_host on page-locked host tensors without waiting;
    H is valid after demag_apply_host_wait."""
    info = info or demag_plan_info(plan)
    B = _field_check(m, info, "m", device=False)
    if _field_check(H, info, "H", device=False) != B or H.shape != m.shape:
        raise ValueError("H must have the shape of m")
    _check(lib().demag_apply_host_async(ctypes.c_void_p(plan), ctypes.c_void_p(m.data_ptr()), float(Ms),
                                        ctypes.c_void_p(H.data_ptr()), int(B), _stream(stream)),
           "demag_apply_host_async")
    return H


def demag_apply_host_wait(plan, stream=None):
    """Wait for every demag_apply_host_async of the plan."""
    _check(lib().demag_apply_host_wait(ctypes.c_void_p(plan), _stream(stream)), "demag_apply_host_wait")


def demag_plan_tensor(plan, out, stream=None):
    _check(lib().demag_plan_tensor(ctypes.c_void_p(plan), ctypes.c_void_p(out.data_ptr()),
                                   out.numel() * out.element_size(), _stream(stream)),
           "demag_plan_tensor")
    return out


def demag_plan_compress(plan, tol):
    """Drop the tensor blocks below tol of their component's maximum
    (demag_plan_compress in demag.h); returns the compressed tensor's bytes."""
    n = ctypes.c_size_t(0)
    _check(lib().demag_plan_compress(ctypes.c_void_p(plan), float(tol), ctypes.byref(n)), "demag_plan_compress")
    return int(n.value)


def demag_plan_keep_slab(plan, k0, k1):
    """Keep only the x-frequencies k0 <= kx < k1 of the plan's tensor
    (demag_plan_keep_slab in demag.h)."""
    _check(lib().demag_plan_keep_slab(ctypes.c_void_p(plan), int(k0), int(k1)), "demag_plan_keep_slab")


def _spectrum_check(t, info, shape, name):
    import torch
    want = torch.complex128 if info["precision"] == PREC_FP64 else torch.complex64
    if t.dtype != want or not t.is_cuda or not t.is_contiguous():
        raise TypeError("%s must be a contiguous CUDA %s tensor" % (name, want))
    if tuple(t.shape) != tuple(shape):
        raise ValueError("%s must have shape %s, got %s" % (name, tuple(shape), tuple(t.shape)))


def _planes_check(t, info, p1, name):
    B = _field_check(t, info, name)
    if p1 > B * info["L"] * 3:
        raise ValueError("plane range beyond the %d planes of %s" % (B * info["L"] * 3, name))


def demag_rows_forward(plan, m, p0, p1, spec, stream=None, info=None):
    """spec [p1 - p0, Kx, ny] (complex) <- row spectra of planes p0..p1-1 of m."""
    info = info or demag_plan_info(plan)
    _planes_check(m, info, p1, "m")
    _spectrum_check(spec, info, (p1 - p0, info["Px"] // 2 + 1, info["ny"]), "spec")
    _check(lib().demag_rows_forward(ctypes.c_void_p(plan), ctypes.c_void_p(m.data_ptr()), int(p0), int(p1),
                                    ctypes.c_void_p(spec.data_ptr()), _stream(stream)), "demag_rows_forward")
    return spec


def demag_columns_slab(plan, spec, k0, k1, B, stream=None, info=None):
    """Column steps of every plane of B states at k0 <= kx < k1, in place on
    spec [B * L * 3, k1 - k0, ny] (complex)."""
    info = info or demag_plan_info(plan)
    _spectrum_check(spec, info, (B * info["L"] * 3, k1 - k0, info["ny"]), "spec")
    _check(lib().demag_columns_slab(ctypes.c_void_p(plan), ctypes.c_void_p(spec.data_ptr()), int(k0), int(k1),
                                    int(B), _stream(stream)), "demag_columns_slab")
    return spec


def demag_rows_inverse(plan, spec, p0, p1, Ms, H, stream=None, info=None):
    """Planes p0..p1-1 of H <- inverse row transforms of spec [p1 - p0, Kx, ny]."""
    info = info or demag_plan_info(plan)
    _planes_check(H, info, p1, "H")
    _spectrum_check(spec, info, (p1 - p0, info["Px"] // 2 + 1, info["ny"]), "spec")
    _check(lib().demag_rows_inverse(ctypes.c_void_p(plan), ctypes.c_void_p(spec.data_ptr()), int(p0), int(p1),
                                    float(Ms), ctypes.c_void_p(H.data_ptr()), _stream(stream)),
           "demag_rows_inverse")
    return H


def demag_tensor_points(geom, out, stream=None):
    """geom: CUDA float64 [n, 9]; out: CUDA float64 [n, 6]."""
    import torch
    if geom.dtype != torch.float64 or out.dtype != torch.float64 or not geom.is_cuda or not out.is_cuda:
        raise TypeError("geom and out must be CUDA float64 tensors")
    if geom.shape[-1] != 9 or out.shape[-1] != 6 or geom.shape[0] != out.shape[0]:
        raise ValueError("geom must be [n, 9] and out [n, 6]")
    _check(lib().demag_tensor_points(int(geom.shape[0]), ctypes.c_void_p(geom.data_ptr()),
                                     ctypes.c_void_p(out.data_ptr()), _stream(stream)),
           "demag_tensor_points")
    return out


def demag_apply_static(tensor, thickness, nx, ny, precision, m, Ms, H, stream=None):
    """demag_apply without device allocation: tensor is the device copy written by
    demag_plan_tensor; the library's fixed scratch array holds the workspace."""
    import torch
    info = {"L": len(thickness), "nx": nx, "ny": ny, "precision": precision}
    want = torch.float64 if precision == PREC_FP64 else torch.float32
    if tensor.dtype != want or not tensor.is_cuda or not tensor.is_contiguous():
        raise TypeError("tensor must be a contiguous CUDA %s tensor for this precision" % want)
    B = _field_check(m, info, "m")
    if _field_check(H, info, "H") != B or H.shape != m.shape:
        raise ValueError("H must have the shape of m")
    th = (ctypes.c_double * len(thickness))(*[float(t) for t in thickness])
    _check(lib().demag_apply_static(ctypes.c_void_p(tensor.data_ptr()), tensor.numel() * tensor.element_size(),
                                    th, int(nx), int(ny), len(thickness), int(precision),
                                    ctypes.c_void_p(m.data_ptr()), float(Ms), ctypes.c_void_p(H.data_ptr()),
                                    int(B), _stream(stream)),
           "demag_apply_static")
    return H


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def demag_mlp_param_count(I, H, O):
    return int(lib().demag_mlp_param_count(int(I), int(H), int(O)))


def demag_mlp_forward(w_bf16, x, y, I, H, O, stream=None):
    """y[N, O] = network(x[N, I]); w_bf16: CUDA bfloat16 [P]."""
    _check(lib().demag_mlp_forward(_ptr(w_bf16), _ptr(x), _ptr(y), int(x.shape[0]), int(I), int(H), int(O),
                                   _stream(stream)), "demag_mlp_forward")
    return y


def demag_mlp_backward(w_bf16, x, gy, gw, gx, I, H, O, stream=None):
    """gw += dLoss/dparameters (if not None); gx = dLoss/dx (if not None)."""
    _check(lib().demag_mlp_backward(_ptr(w_bf16), _ptr(x), _ptr(gy), _ptr(gw), _ptr(gx), int(x.shape[0]),
                                    int(I), int(H), int(O), _stream(stream)), "demag_mlp_backward")


def demag_mlp_mse(y, target, gy, loss, stream=None):
    """loss (CUDA float64 [1]) += mean squared error; gy = its gradient in y."""
    _check(lib().demag_mlp_mse(_ptr(y), _ptr(target), _ptr(gy), _ptr(loss), int(y.shape[0]), int(y.shape[1]),
                               _stream(stream)), "demag_mlp_mse")


def demag_mlp_adam(w, w_bf16, g, m1, m2, lr, beta1, beta2, eps, step, stream=None):
    _check(lib().demag_mlp_adam(_ptr(w), _ptr(w_bf16), _ptr(g), _ptr(m1), _ptr(m2), int(w.numel()), float(lr),
                                float(beta1), float(beta2), float(eps), int(step), _stream(stream)),
           "demag_mlp_adam")


def demag_layer_mean(H, precision, layer, out, stream=None):
    """out (CUDA float64 [B, 3]) = mean over the cells of layer `layer` of H [B, L, 3, ny, nx]."""
    B, L, _, ny, nx = H.shape
    _check(lib().demag_layer_mean(_ptr(H), int(precision), int(B), int(L), int(ny), int(nx), int(layer),
                                  _ptr(out), _stream(stream)), "demag_layer_mean")
    return out


def demag_wait_timeouts():
    """Bounded device waits that gave up since the previous call (synchronises the device)."""
    n = ctypes.c_ulonglong(0)
    _check(lib().demag_wait_timeouts(ctypes.byref(n)), "demag_wait_timeouts")
    return int(n.value)


def demag_selftest_bounded_wait(limit_cycles, stream=None):
    """Run one bounded wait that cannot complete (it gives up after limit_cycles)."""
    _check(lib().demag_selftest_bounded_wait(int(limit_cycles), _stream(stream)), "demag_selftest_bounded_wait")


def demag_debug_fail_alloc(after):
    """Refuse the library's device allocation after the next `after` ones (host-side injection)."""
    _check(lib().demag_debug_fail_alloc(int(after)), "demag_debug_fail_alloc")


def demag_relax_layer(plan, m, layer, mask, Js, A_ex, Ku, b_ext, length_unit=1e-9, tol_torque=1e-5,
                      max_iter=2000, history=10, stream=None, info=None):
    """Relax layer `layer` of m ([L, 3, ny, nx] or [1, L, 3, ny, nx], CUDA, the plan's
    dtype) in place: L-BFGS minimisation of exchange + uniaxial anisotropy (z) +
    Zeeman + demag energy, the other layers pinned.  mask: CUDA uint8 [ny, nx].
    Returns the stats as a dict."""
    import torch
    info = info or demag_plan_info(plan)
    if _field_check(m, info, "m") != 1:
        raise ValueError("m must hold one state")
    if mask.dtype != torch.uint8 or not mask.is_cuda or tuple(mask.shape) != (info["ny"], info["nx"]) \
            or not mask.is_contiguous():
        raise ValueError("mask must be a contiguous CUDA uint8 tensor [ny, nx]")
    prm = RelaxParams(float(Js), float(A_ex), float(Ku), (ctypes.c_double * 3)(*[float(b) for b in b_ext]),
                      float(length_unit), float(tol_torque), int(max_iter), int(history))
    st = RelaxStats()
    _check(lib().demag_relax_layer(ctypes.c_void_p(plan), ctypes.c_void_p(m.data_ptr()), int(layer),
                                   ctypes.c_void_p(mask.data_ptr()), ctypes.byref(prm), ctypes.byref(st),
                                   _stream(stream)), "demag_relax_layer")
    return {"iterations": st.iterations, "evaluations": st.evaluations, "converged": st.converged,
            "energy": st.energy, "max_torque": st.max_torque}


def demag_destroy(plan):
    if plan:
        _check(lib().demag_destroy(ctypes.c_void_p(plan)), "demag_destroy")


class Plan:
    """Owning wrapper of a demag plan handle."""

    def __init__(self, nx, ny, dx, dy, thickness, precision=PREC_FP32, max_batch=1, stream=None):
        self.handle = demag_plan_create(nx, ny, dx, dy, thickness, precision, max_batch, stream)
        self.info = demag_plan_info(self.handle)
        self.slab = None

    @property
    def dtype(self):
        import torch
        return torch.float64 if self.info["precision"] == PREC_FP64 else torch.float32

    def apply(self, m, Ms, H=None, stream=None):
        import torch
        if H is None:
            H = torch.empty_like(m)
        return demag_apply(self.handle, m, Ms, H, stream, self.info)

    @classmethod
    def equidistant(cls, nx, ny, nz, dx, dy, dz, precision=PREC_FP32, max_batch=1, stream=None):
        """Plan of the equidistant 3D-FFT method (Eq. FFT_3D): nz layers of one
        thickness dz; applied like any plan."""
        self = cls.__new__(cls)
        self.handle = demag_plan_create_equidistant(nx, ny, nz, dx, dy, dz, precision, max_batch, stream)
        self.info = demag_plan_info(self.handle)
        self.slab = None
        return self

    def compress(self, tol):
        """Block-compress the plan's tensor (split-precision plans on path 6
        or 7); returns the stored bytes."""
        n = demag_plan_compress(self.handle, tol)
        self.info = demag_plan_info(self.handle)
        return n

    def keep_slab(self, k0, k1):
        """Keep only the x-frequencies k0 <= kx < k1 of the tensor; the plan
        then runs the sharded steps only (demag_plan_keep_slab)."""
        demag_plan_keep_slab(self.handle, k0, k1)
        self.slab = (int(k0), int(k1))

    def close(self):
        if self.handle:
            demag_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
