"""Easy-axis hysteresis of one layer of a stack (Sec. 4: the free layer of the
MRAM cell, the two SAFM layers pinned, an applied field along z stepped over
the loop and the free layer relaxed by L-BFGS at every step).

Every relaxation runs in the library (demag_relax_layer: the energy terms and
the minimiser in CUDA/C++, the demag field by the library's apply); this module
only sets up the stack and steps the field.
"""
import numpy as np

from . import _lib as dm
from . import inputs

# CoFe values used in Sec. 4 for the switching simulation
JS_COFE = 1.75      # T (mu0 Ms)
A_COFE = 1.5e-11    # J/m
KU_COFE = 2.09e6    # J/m^3, easy axis +z
SAFM_T_OPT = 3.44   # nm: the optimised middle-layer thickness printed in Sec. 4


def mram_stack(t_middle=SAFM_T_OPT, n=64, diameter=60.0):
    """The Sec. 4 stack [5, 1, t, 1, 3] nm on n x n cells over the 60 nm disk:
    layer 1 pinned +z, layer 3 pinned -z, layers 2 and 4 spacers, layer 5 the
    free layer, starting along +z.  Returns (dx, thickness, m [5, 3, n, n],
    mask [n, n] bool, free layer index)."""
    dx, th, m = inputs.safm_stack(t_middle, n, diameter)
    mask = inputs.disk_mask(n, n)
    m[4, 2][mask] = 1.0
    return dx, th, m, mask, 4


def field_steps(b_max, steps):
    """Applied field magnitudes from +b_max down to -b_max (steps + 1 values)."""
    return np.linspace(b_max, -b_max, steps + 1)


def hysteresis(plan, m, layer, mask, b_values, Js=JS_COFE, A_ex=A_COFE, Ku=KU_COFE, tilt_deg=0.0,
               tol_torque=1e-4, max_iter=5000, stop_after_switch=None, length_unit=1e-9):
    """Relax layer `layer` of m (CUDA tensor [L, 3, ny, nx] of the plan's dtype,
    updated in place) at every applied field b (tesla) of b_values, applied at
    tilt_deg from z in the x-z plane.  Returns a list of (b, mean m_z over the
    mask, iterations, converged).  With stop_after_switch = k the sweep ends k
    steps after the mean m_z first changed sign."""
    import torch
    mk = torch.as_tensor(np.asarray(mask, dtype=np.uint8)).cuda()
    w = mk.double()
    info = plan.info
    out, start_sign, switched_at = [], None, None
    ps, pc = np.sin(np.radians(tilt_deg)), np.cos(np.radians(tilt_deg))
    for k, b in enumerate(b_values):
        st = dm.demag_relax_layer(plan.handle, m, layer, mk, Js, A_ex, Ku, (b * ps, 0.0, b * pc),
                                  length_unit=length_unit, tol_torque=tol_torque, max_iter=max_iter, info=info)
        mz = float((m[layer, 2].double() * w).sum() / w.sum())
        out.append((float(b), mz, st["iterations"], st["converged"]))
        if start_sign is None:
            start_sign = np.sign(mz)
        elif switched_at is None and np.sign(mz) != start_sign:
            switched_at = k
        if stop_after_switch is not None and switched_at is not None and k >= switched_at + stop_after_switch:
            break
    return out


def switching_field(loop):
    """|b| of the first step of the loop at which the mean m_z has changed sign
    (None if it never does)."""
    s0 = np.sign(loop[0][1])
    for b, mz, _, _ in loop:
        if np.sign(mz) != s0:
            return abs(b)
    return None
