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
