"""Host-side checks of libnufft3d that need no GPU: the shared library loads,
exports every function that include/nufft3d.h declares, validates arguments
and reports workspace sizes."""
import os
import re

import numpy as np
import pytest

from paper_1605_05231_gb300 import binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"^\s*(?:int|const char\*|void)\s+(nufft3d_\w+)\s*\(", src, re.M))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(binding.LIB_PATH):
        from paper_1605_05231_gb300 import build as b

        b.build()
    return binding.load_library()


def test_every_declared_symbol_is_exported(lib):
    declared = _declared_functions()
    assert len(declared) >= 9
    for name in declared:
        assert hasattr(lib, name), name
    assert set(binding.EXPORTS) <= set(declared)


def test_error_strings(lib):
    for code in range(-6, 1):
        assert binding.error_string(code) not in ("", None)
    assert binding.error_string(-4) == "unsupported parameters"
    assert binding.error_string(123) == "unknown status"


def _ws(**kw):
    base = dict(n=32, dirs=np.eye(3), m=0, k=0, j=6, table_oversamp=1024)
    base.update(kw)
    return binding.workspace_bytes(**base)


def test_workspace_bytes_counts_grid_and_buffers(lib):
    b = _ws()
    K, N, D, M = 64, 32, 3, 64
    # forward grid + adjoint grid + FFT intermediates + line buffer + point sort
    expect = 2 * K ** 3 * 8 + N * N * K * 8 + N * K * K * 8 + D * M * 8 + D * M * 4
    assert expect <= b < expect + 200_000
    # a reduced-precision forward grid replaces the separate adjoint grid
    assert _ws(grid_dtype="bf16") == b - K ** 3 * 8 + K ** 3 * 4 + 4
    assert _ws(do_line_fft=False) == b - D * M * 8
    assert _ws(exact_coeffs=1) == b - 1025 * 6 * 8   # no table


@pytest.mark.parametrize("kw,status", [
    (dict(n=7), -1),                     # odd N
    (dict(n=4), -1),                     # too small
    (dict(n=1024), -1),                  # too large
    (dict(k=16), -1),                    # K < N
    (dict(j=5), -4),                     # odd J unsupported
    (dict(j=10), -1),
    (dict(table_oversamp=1000), -1),     # not a power of two
    (dict(m=63), -1),                    # odd M
    (dict(k=80), -4),                    # 80 = 16 * 5: not 2^a 3^b
    (dict(m=80), -4),
    (dict(grid_dtype=3), -1),
    (dict(exact_coeffs=2), -1),
    (dict(line_weight=np.array([1.0, np.nan, 1.0])), -1),
    (dict(dirs=np.array([[2.0, 0.0, 0.0]])), -1),   # |d| > 1
    (dict(dirs=np.array([[np.nan, 0.0, 0.0]])), -1),
    (dict(omega=np.full(64, 4.0)), -1),             # |omega| > pi
])
def test_argument_validation(lib, kw, status):
    with pytest.raises(binding.NufftError) as ei:
        _ws(**kw)
    assert ei.value.status == status


def test_null_arguments_rejected(lib):
    import ctypes

    assert lib.nufft3d_workspace_bytes(None, None) == -1
    assert lib.nufft3d_forward(None, None, None, None) == -1
    assert lib.nufft3d_adjoint(None, None, None, None) == -1
    assert lib.nufft3d_plan_destroy(None) == 0
    out = ctypes.c_void_p(1)
    assert lib.nufft3d_plan_create(ctypes.byref(out), None, None) == -1
    assert out.value is None
    assert lib.nufft3d_plan_info(None, None) == -1
    assert lib.nufft3d_plan_sync_status(None, None) == -1
    assert lib.nufft3d_adjoint_noalloc(None, None, None, None) == -1
    bout = ctypes.c_void_p(1)
    assert lib.nufft3d_batch_create(ctypes.byref(bout), None, 0, None) == -1
    assert bout.value is None
    assert lib.nufft3d_batch_forward_adjoint(None, None, None, None, None) == -1
    assert lib.nufft3d_batch_item(None, 0, None) == -1
    assert lib.nufft3d_batch_destroy(None) == 0
