"""The C-ABI library builds, loads and exports every symbol include/demag.h
declares; argument checks answer with status codes before any GPU work (these
calls run without a GPU)."""
import ctypes
import os
import re

import pytest

import paper_1910_07054_gb300 as dm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    with open(os.path.join(ROOT, "include", "demag.h")) as fh:
        text = fh.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(demag_[a-z_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    lib = dm.lib()
    syms = _declared_symbols()
    assert "demag_plan_create" in syms and "demag_apply" in syms and "demag_destroy" in syms
    for s in syms:
        assert hasattr(lib, s), s


def test_library_is_in_tree():
    path = os.path.realpath(dm.library_path())
    assert path.startswith(os.path.realpath(ROOT))
    assert os.path.exists(path)


def _create(nx=4, ny=4, dx=2.0, dy=2.0, th=(1.0,), prec=0, mb=1, plan=True):
    lib = dm.lib()
    h = ctypes.c_void_p()
    arr = (ctypes.c_double * max(1, len(th)))(*th) if th is not None else None
    return lib.demag_plan_create(ctypes.byref(h) if plan else None, nx, ny, dx, dy, arr,
                                 len(th) if th is not None else 0, prec, mb, None)


@pytest.mark.parametrize("kw,status", [
    (dict(nx=0), 1), (dict(ny=-3), 1), (dict(dx=0.0), 1), (dict(dy=float("nan")), 1),
    (dict(dx=float("inf")), 1), (dict(th=(1.0, -0.5)), 1), (dict(th=(1.0, float("nan"))), 1),
    (dict(th=()), 1), (dict(prec=7), 1), (dict(mb=0), 1), (dict(plan=False), 1),
    (dict(th=None), 1), (dict(nx=4096), 4), (dict(th=(1.0,) * 300), 4),
])
def test_plan_create_rejects_bad_arguments(kw, status):
    assert _create(**kw) == status
    assert dm.demag_last_error() != ""


def test_other_entry_points_reject_null_and_bad_sizes():
    lib = dm.lib()
    assert lib.demag_apply(None, None, 1.0, None, 1, None) == 1
    assert lib.demag_apply_host(None, None, 1.0, None, 1, None) == 1
    assert lib.demag_apply_timed(None, None, 1.0, None, 1, None, None, 3) == 1
    assert lib.demag_apply_static(None, 0, None, 4, 4, 1, 1, None, 1.0, None, 1, None) == 1
    assert lib.demag_tensor_points(-1, None, None, None) == 1
    assert lib.demag_tensor_points(5, None, None, None) == 1
    assert lib.demag_plan_info(None, None) == 1
    assert lib.demag_plan_tensor(None, None, 0, None) == 1
    assert lib.demag_plan_compress(None, 1e-8, None) == 1
    assert lib.demag_plan_keep_slab(None, 0, 1) == 1
    assert lib.demag_rows_forward(None, None, 0, 1, None, None) == 1
    assert lib.demag_rows_inverse(None, None, 0, 1, 1.0, None, None) == 1
    assert lib.demag_columns_slab(None, None, 0, 1, 1, None) == 1
    assert lib.demag_destroy(None) == 0


@pytest.mark.parametrize("args,status", [
    ((4, 4, 0, 2.0, 2.0, 1.0, 1, 1), 1),            # nz < 1
    ((4, 4, 3, 2.0, 2.0, 0.0, 1, 1), 1),            # dz <= 0
    ((4, 4, 3, 2.0, 2.0, float("nan"), 1, 1), 1),   # dz not finite
    ((0, 4, 3, 2.0, 2.0, 1.0, 1, 1), 1),            # nx < 1
    ((4, 4, 3, 2.0, 2.0, 1.0, 2, 1), 4),            # split precision: not for the 3D method
    ((4, 4, 300, 2.0, 2.0, 1.0, 1, 1), 4),          # nz above 256
    ((4, 4, 3, 2.0, 2.0, 1.0, 1, 0), 1),            # max_batch < 1
])
def test_equidistant_plan_rejects_bad_arguments(args, status):
    h = ctypes.c_void_p()
    assert dm.lib().demag_plan_create_equidistant(ctypes.byref(h), *args, None) == status
    assert dm.demag_last_error() != ""


def test_status_strings():
    names = [dm.demag_status_string(s) for s in range(5)]
    assert names == ["DEMAG_OK", "DEMAG_EINVAL", "DEMAG_ENOMEM", "DEMAG_ECUDA", "DEMAG_EUNSUPPORTED"]
