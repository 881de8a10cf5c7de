"""The C ABI library loads without a GPU and exports every entry point of include/bos.h."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "bos.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(bos_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for need in ("bos_create", "bos_destroy", "bos_set_grid", "bos_set_geometry", "bos_render",
                 "bos_render_reference", "bos_backward", "bos_loss_l2", "bos_status", "bos_error_string"):
        assert need in names


def test_library_exports_every_declared_symbol():
    from paper_2509_14442_gb300 import bos

    L = bos.lib()
    for name in declared_symbols():
        assert hasattr(L, name), name
        assert name in bos.SIGNATURES, f"{name} has no binding"


def test_status_strings():
    from paper_2509_14442_gb300 import bos

    L = bos.lib()
    for s in range(9):
        assert L.bos_error_string(s).decode()
    assert L.bos_error_string(99).decode() == "unknown status"


def test_null_arguments_are_rejected_without_touching_the_gpu():
    import ctypes as C

    from paper_2509_14442_gb300 import bos

    L = bos.lib()
    assert L.bos_create(None, 0, 0) == bos.BOS_ERR_INVALID_ARG
    assert L.bos_set_grid(None, None, None, None) == bos.BOS_ERR_INVALID_ARG
    assert L.bos_render(None, None, None, None, 0, None) == bos.BOS_ERR_INVALID_ARG
    assert L.bos_backward(None, None, None, None) == bos.BOS_ERR_INVALID_ARG
    assert L.bos_loss_l2(None, None, 0, None, None, None) == bos.BOS_ERR_INVALID_ARG
    assert b"NULL" in L.bos_last_error() or b"bad argument" in L.bos_last_error()
    assert L.bos_probe_fma(3, 1, None, None, None) == bos.BOS_ERR_INVALID_ARG
    assert L.bos_probe_fma(0, 0, None, None, None) == bos.BOS_ERR_INVALID_ARG
    assert L.bos_probe_read_l1(None, 65536, 1, None, None, None) == bos.BOS_ERR_INVALID_ARG
    assert L.bos_destroy(None) == bos.BOS_OK


def test_no_device_fails_loudly():
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2509_14442_gb300 import bos

    with pytest.raises(bos.BosError):
        bos.bos_create(0, 0)


def _noalloc_args(bos, scene, prec=None):
    """Descriptors of a scene and stand-in device pointers: the calls below must refuse
    before any pointer is used or any CUDA call is made."""
    p = prec if prec is not None else bos.BOS_PREC_FP32_COMP
    return [bos.grid_desc(scene.grid, p), 16, bos.camera_desc(scene.camera), bos.wall_desc(scene.wall),
            bos.light_desc(scene.light), 32, bos.integ_desc(scene.integ), 64, None, None]


def _call_noalloc(bos, args):
    import ctypes as C

    g, T, cam, wall, light, pat, integ, I, D, st = args
    return bos.lib().bos_render_noalloc(C.byref(g), T, C.byref(cam), C.byref(wall), C.byref(light), pat,
                                        C.byref(integ), I, D, st)


def test_noalloc_checks_descriptors_like_set_geometry_without_touching_the_gpu():
    """The allocation-free render applies the same descriptor checks as bos_set_grid and
    bos_set_geometry: an unbounded fixed step count, a non-unit viewing direction, a
    non-unit wall axis and a malformed projector camera are refused with
    BOS_ERR_INVALID_ARG before anything reaches the device."""
    from paper_2509_14442_gb300 import bos, scenes

    sc = scenes.blob_cube(n=8, width=8, height=8, steps=4)
    a = _noalloc_args(bos, sc)
    a[6].fixed_steps = 1 << 25
    assert _call_noalloc(bos, a) == bos.BOS_ERR_INVALID_ARG
    assert b"fixed_steps" in bos.lib().bos_last_error()
    a = _noalloc_args(bos, sc)
    a[2].fwd[0] += 0.5                                  # not a unit vector
    assert _call_noalloc(bos, a) == bos.BOS_ERR_INVALID_ARG
    assert b"camera" in bos.lib().bos_last_error()
    a = _noalloc_args(bos, sc)
    a[3].eu[0] *= 2.0
    assert _call_noalloc(bos, a) == bos.BOS_ERR_INVALID_ARG
    assert b"wall" in bos.lib().bos_last_error()
    room = scenes.room((16, 16, 12), 16, 16, 1, 7, field=False)
    a = _noalloc_args(bos, room)
    a[4].proj.fx = -1.0                                  # projector camera of light mode 1
    assert _call_noalloc(bos, a) == bos.BOS_ERR_INVALID_ARG
    assert b"projector" in bos.lib().bos_last_error()
    a = _noalloc_args(bos, sc)
    a[6].max_step_vox, a[6].fixed_steps = 1e9, 0
    assert _call_noalloc(bos, a) == bos.BOS_ERR_INVALID_ARG


def test_tile_count_is_capped_below_int_max():
    """Images whose warp tiles would overflow the 32-bit tile index are refused."""
    from paper_2509_14442_gb300 import bos, scenes

    sc = scenes.blob_cube(n=8, width=8, height=8, steps=4)
    a = _noalloc_args(bos, sc)
    a[2].width, a[2].height, a[2].spp = 1 << 19, 1 << 19, 1      # 2^33 tiles of 8 x 4 pixels
    assert _call_noalloc(bos, a) == bos.BOS_ERR_INVALID_ARG
    assert b"warp tiles" in bos.lib().bos_last_error()


def test_checked_build_exports_every_symbol_and_says_so():
    """The checked build (BOS_CHECKED=1) is the same ABI with bounds checks compiled in."""
    import ctypes

    from paper_2509_14442_gb300 import _build, bos

    path = _build.build(checked=True)
    Lc = ctypes.CDLL(path)
    for name in declared_symbols():
        assert hasattr(Lc, name), name
    Lc.bos_checked_build.restype = ctypes.c_int
    assert Lc.bos_checked_build() == 1
    assert bos.lib().bos_checked_build() == (1 if bos.checked() else 0)
    if not bos.checked():
        assert bos.lib().bos_debug_store_bound(None, 0) == bos.BOS_ERR_UNIMPLEMENTED
