"""Host-only checks of the C ABI: the library builds/loads and exports every
declared entry point; argument validation that runs before any CUDA call."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rf.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2511_12894_gb300 import build, load_library
    build.build()
    return load_library()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:[\w\s\*]+?)\b(rf_\w+)\s*\(", text, flags=re.M)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 14
    for name in names:
        assert hasattr(lib, name), name
    import paper_2511_12894_gb300 as p
    assert sorted(p.EXPORTED) == names


def test_version_and_error_string(lib):
    assert lib.rf_version() == 5
    assert isinstance(lib.rf_last_error(), bytes)


@pytest.mark.parametrize("field,value", [("n", 1000), ("n", 128), ("fs", -1.0), ("f_low", 0.0),
                                         ("f_high", 600.0), ("pn_order", 9), ("dtype", 7), ("df_high", -1.0)])
def test_create_rejects_bad_grid_without_touching_the_gpu(lib, field, value):
    from paper_2511_12894_gb300 import RF_EINVAL, rf_grid
    g = rf_grid(1 << 12, 1024.0, 40.0, 459.0, 53.0, 5.0, 2, 0)
    setattr(g, field, value)
    h = ctypes.c_void_p()
    st = lib.rf_create(ctypes.byref(g), ctypes.byref(h))
    assert st == RF_EINVAL
    assert h.value is None
    assert len(lib.rf_last_error()) > 0


def test_null_arguments_are_rejected(lib):
    from paper_2511_12894_gb300 import RF_EINVAL
    assert lib.rf_create(None, None) == RF_EINVAL
    assert lib.rf_kernels_info(None, None, None, None, None, None, None) == RF_EINVAL
    assert lib.rf_kernels_copy_taps(None, None, None) == RF_EINVAL
    lib.rf_destroy(None)
    lib.rf_kernels_free(None)


def test_null_context_and_handles_are_rejected_by_every_entry_point(lib):
    """Every call that takes a context or a kernel set refuses NULL with RF_EINVAL before any
    device work (host validation; no GPU needed)."""
    from paper_2511_12894_gb300 import RF_EINVAL
    i32 = ctypes.c_int32
    vp = ctypes.c_void_p
    cuts = (i32 * 1)(0)
    assert lib.rf_reserve(None, 4, None) == RF_EINVAL
    assert lib.rf_template_fd(None, None, None, None) == RF_EINVAL
    assert lib.rf_mf_reference(None, None, None, 1, None, None, None, None) == RF_EINVAL
    assert lib.rf_reference_filters(None, None, 1, None, None, None, None) == RF_EINVAL
    assert lib.rf_mf_filtered(None, None, 1, None, None, None) == RF_EINVAL
    assert lib.rf_build_ratio_kernels(None, None, None, 0, None, 1e-3, 1, 0, None, None) == RF_EINVAL
    assert lib.rf_kernels_grids(None, None) == RF_EINVAL
    assert lib.rf_kernels_prepare(None, None, 0, 0, None) == RF_EINVAL
    assert lib.rf_kernels_prepare_buckets(None, None, 1, cuts, cuts, cuts, None) == RF_EINVAL
    assert lib.rf_kernels_os_layout(None, None, None) == RF_EINVAL
    assert lib.rf_kernels_gemm_layout(None, None) == RF_EINVAL
    assert lib.rf_bank_structure(None, 4, 20.0, 7, 10.0, 500, None, None, None, None) == RF_EINVAL
    assert lib.rf_stream_winmax(None, None, 0, 0, None, None, 0, 0, None, None, None, None, None) == RF_EINVAL
    assert lib.rf_kernels_os_buckets(None, 1, None, None, None, None) == RF_EINVAL
    assert lib.rf_reconstruct(None, None, None, 0, 0, None, None) == RF_EINVAL
    assert lib.rf_reconstruct_winmax(None, None, None, 0, 0, 16, None, None, None) == RF_EINVAL
    zs = (vp * 1)(None)
    assert lib.rf_reconstruct_batched(None, 1, zs, zs, 0, 0, 16, None, None, None) == RF_EINVAL
    assert lib.rf_autotune(None, 1, zs, zs, 16, 0, 4, None, 0, None, None) == RF_EINVAL
    assert lib.rf_winmax(None, None, 1, 16, None, None, None) == RF_EINVAL
    assert lib.rf_device_status(None) == RF_EINVAL
    assert lib.rf_selftest_bounded_wait(None, None) == RF_EINVAL
    assert b"NULL" in lib.rf_last_error() or len(lib.rf_last_error()) > 0


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """No silent fallback: without the built library the binding raises instead of computing."""
    import paper_2511_12894_gb300 as p
    monkeypatch.setattr(p, "_lib", None)
    with pytest.raises(RuntimeError, match="not found"):
        p.load_library(str(tmp_path / "librf.so"))


def test_context_requires_a_cuda_device(lib, monkeypatch):
    """There is no CPU path: a context on a machine without a CUDA device raises."""
    import torch
    import paper_2511_12894_gb300 as p
    monkeypatch.setattr(torch.cuda, "is_available", lambda: False)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        p.RatioFilter(1 << 12, 1024.0, 40.0, 459.0, 7)


def test_product_package_never_imports_the_oracle():
    """The oracle is test infrastructure: importing the package (and its sharding helper) loads
    no module of it."""
    import subprocess
    import sys
    code = ("import sys; import paper_2511_12894_gb300, paper_2511_12894_gb300.shard; "
            "bad = [m for m in sys.modules if m == 'oracle' or m.startswith('oracle.')]; "
            "assert not bad, bad")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]


def test_binding_rejects_short_buffers_before_any_launch():
    """The library reads and writes through raw pointers and cannot see a buffer's size, so the
    binding checks every tensor against the element count the call touches (before it checks
    anything that needs a GPU)."""
    import torch
    import paper_2511_12894_gb300 as p
    with pytest.raises(ValueError, match="holds 100 elements; the call needs 4096"):
        p._dev(torch.zeros(100, dtype=torch.float32), torch.float32, "x", 4096)
    with pytest.raises(ValueError, match="z_out holds 8 elements; the call needs 16"):
        p._out(torch.zeros(8, dtype=torch.complex64), torch.complex64, 16, "z_out")
    # large enough: the next check (a CUDA device) is reached
    with pytest.raises(ValueError, match="must be a CUDA tensor"):
        p._dev(torch.zeros(4096, dtype=torch.float32), torch.float32, "x", 4096)
    with pytest.raises(ValueError, match="must be a CUDA tensor"):
        p._out(torch.zeros(16, dtype=torch.complex64), torch.complex64, 16, "z_out")
    with pytest.raises(TypeError, match="must be a torch tensor"):
        p._out([0.0] * 16, torch.complex64, 16, "z_out")
