"""C-ABI boundary checks that need no GPU: the library builds for sm_103a, loads, exports every
function include/ica.h declares, and its host-only entry points behave as documented."""
import ctypes as C
import os
import re

import pytest

from conftest import ROOT


@pytest.fixture(scope="module")
def lib():
    from paper_2408_17118_gb300.build import build_library
    from paper_2408_17118_gb300 import _lib

    build_library()
    return _lib.load()


def header_functions():
    src = open(os.path.join(ROOT, "include", "ica.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ica_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    names = header_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name


def test_binding_covers_the_header(lib):
    from paper_2408_17118_gb300 import _lib

    assert sorted(_lib.SIGNATURES) == header_functions()


def test_default_opts_and_status_strings(lib):
    from paper_2408_17118_gb300 import _lib

    o = _lib.ica_opts()
    lib.ica_default_opts(C.byref(o))
    assert o.precision == _lib.ICA_BF16 and o.refine_topk == 4 and o.refine_iters == 10
    assert o.stage_persistent == 1
    assert o.stage_tol == 1e-4 and o.refine_tol == 1e-6 and o.fp32_tol_floor == 1e-6 and not o.B0
    for st in range(8):
        assert lib.ica_status_string(st) not in (None, b"unknown status")
    assert lib.ica_status_string(99) == b"unknown status"


def test_workspace_bytes(lib):
    from paper_2408_17118_gb300 import _lib

    o = _lib.ica_opts()
    lib.ica_default_opts(C.byref(o))
    small = lib.ica_workspace_bytes(8, 10_000, 64, C.byref(o))
    big = lib.ica_workspace_bytes(256, 1_000_000, 8192, C.byref(o))
    assert 0 < small < big
    # BF16 adds the BF16 copy of X~: 2 bytes per reduced sample
    o.precision = _lib.ICA_FP32
    assert lib.ica_workspace_bytes(256, 1_000_000, 8192, C.byref(o)) < big
    o.precision = _lib.ICA_PLAIN_FP32  # plain form stores Z: M x T floats
    assert lib.ica_workspace_bytes(64, 200_000, 1024, C.byref(o)) > 1024 * 200_000 * 4
    for bad in [(0, 100, 4), (257, 1000, 4), (8, 0, 4), (8, 100, 0), (8, 100, 70000)]:
        assert lib.ica_workspace_bytes(*bad, None) == 0


def test_argument_errors_without_a_device(lib):
    assert lib.ica_create(None, 0) == 1  # ICA_ERR_ARG
    assert lib.ica_set_stream(None, None) == 1
    assert lib.ica_destroy(None) == 0


def test_create_without_gpu_reports_cuda_error(lib):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = C.c_void_p()
    assert lib.ica_create(C.byref(h), 0) == 2  # ICA_ERR_CUDA
    assert not h.value
