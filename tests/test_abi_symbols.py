"""The C-ABI library builds for sm_103a, loads without a GPU, and exports
every entry point that include/masw.h declares."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "masw.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(masw_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2003_02256_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("masw_model_batch_create", "masw_model_batch_destroy", "masw_dispersion",
                     "masw_misfit", "masw_misfit_grad", "masw_strerror"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_strerror_needs_no_gpu(lib):
    lib.masw_strerror.restype = ctypes.c_char_p
    assert lib.masw_strerror(0) == b"ok"
    assert b"invalid" in lib.masw_strerror(1)
    assert lib.masw_strerror(999) == b"unknown error code"


def test_null_arguments_are_rejected_without_touching_the_gpu(lib):
    f = lib.masw_model_batch_create
    f.restype = ctypes.c_int
    assert f(None, None, None, None) == 1
    assert lib.masw_dispersion(None, None, None, None, 0) == 1
    assert lib.masw_misfit(None, None, 0, ctypes.c_double(1.0), None) == 1


def test_new_entry_points_reject_bad_arguments_without_the_gpu(lib):
    """Argument checks come before any CUDA call, so they answer on a machine
    without a GPU too."""
    p, i32 = ctypes.c_void_p, ctypes.c_int32
    assert lib.masw_dispersion_leaky(None, None, None, None, i32(0)) == 1
    assert lib.masw_dispersion_changes(None, i32(3), None, None, None, None, i32(0)) == 1
    assert lib.masw_mode_count(None, i32(1), None, None, None, None) == 1
    assert lib.masw_set_route(None, i32(0)) == 1
    assert lib.masw_server_set_route(None, i32(0)) == 1
    assert lib.masw_last_changes_linear(None, None) == 1
    assert lib.masw_test_fail_alloc(i32(-1)) == 0
    d = ctypes.c_double
    assert lib.masw_misfit_curves(None, None, i32(1), d(2.0), None, None, None, None) == 1
    assert lib.masw_server_profile(None, i32(1), None) == 1
    assert lib.masw_last_count_phases(None, None) == 1
    x = (d * 2)(1.0, 4.0)  # 4.0 is above 5 pi / 4
    out = [(d * 2)() for _ in range(4)]
    assert lib.masw_sincos_check(i32(2), x, *out, None) == 1
    assert lib.masw_sincos_check(i32(1), x, None, out[1], out[2], out[3], None) == 1


def test_no_cpu_fallback_without_a_gpu():
    """The product path has no CPU fallback: on a machine without a GPU the
    binding's batch creation fails with the CUDA error instead of computing
    anything on the host."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2003_02256_gb300 import masw, workloads as W

    m, g = W.uniform_batch(n_models=2, n_layers=3, n_lambda=5)
    with pytest.raises(masw.MaswError, match="masw_model_batch_create"):
        masw.Batch(m, g)
