"""The allocation-free reference matched filter (rf_mf_reference_noalloc).

Some callers cannot call cudaMalloc (a plug-in inside an application that owns all
device memory, a low-latency loop that must not synchronise on an allocation).  For
them the library offers one entry point that works from a static device workspace
and allocates nothing.  These tests call it through the C ABI and check it against
the regular rf_mf_reference on the same inputs, twice in a row (the workspace keeps
the previous call's contents, which must not leak into the next result), and once
against the FP64 oracle's matched filter.

The file sorts last so that a run stopping at the first failure has already run
every other test.
"""
import ctypes

import numpy as np
import pytest

import workload
from oracle import data

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 2e-6}


@pytest.fixture(scope="module")
def torch():
    import torch as t
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_12894_gb300 import build
    build.build()
    return t


def _grid(cfg):
    from paper_2511_12894_gb300 import RF_F32, RF_F64, rf_grid
    return rf_grid(cfg.n, cfg.fs, cfg.f_low, cfg.f_high, cfg.df_high, cfg.df_low_max, cfg.pn_order,
                   RF_F64 if cfg.dtype == "f64" else RF_F32)


def _templates(ts):
    from paper_2511_12894_gb300 import rf_template
    arr = (rf_template * len(ts))()
    for i, t in enumerate(ts):
        arr[i] = rf_template(t.m1, t.m2, t.tc, t.phic)
    return arr


@pytest.mark.parametrize("cfg_index,n", [(1, 1 << 16), (1, 1 << 12), (2, 1 << 16), (2, 1 << 10)])
def test_noalloc_matches_regular_matched_filter_twice(torch, cfg_index, n):
    from paper_2511_12894_gb300 import RatioFilter, load_library
    lib = load_library()
    cfg = workload.config(cfg_index, n_override=n, k_override=2)
    ref, nb = cfg.groups[0]
    rdt = torch.float64 if cfg.dtype == "f64" else torch.float32
    cdt = torch.complex128 if cfg.dtype == "f64" else torch.complex64
    ip = torch.tensor(workload.inv_psd(cfg), device="cuda")
    rf = RatioFilter.from_config(cfg)
    g = _grid(cfg)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    # two different inputs and templates, one call after the other
    for real, tmpl in [(0, ref), (1, nb[0])]:
        x = torch.tensor(data.strain(cfg, realisation=real), dtype=rdt, device="cuda")
        expect, sig_e = rf.mf_reference(x, ip, [tmpl])
        z = torch.full((n,), 7.0 + 7.0j, dtype=cdt, device="cuda")
        sig = torch.zeros(1, dtype=torch.float64, device="cuda")
        st = lib.rf_mf_reference_noalloc(ctypes.byref(g), ctypes.c_void_p(x.data_ptr()),
                                         ctypes.c_void_p(ip.data_ptr()), _templates([tmpl]),
                                         ctypes.c_void_p(z.data_ptr()), ctypes.c_void_p(sig.data_ptr()), stream)
        assert st == 0, lib.rf_last_error()
        torch.cuda.synchronize()
        a = z.cpu().numpy()
        b = expect[0].cpu().numpy()
        assert np.abs(a - b).max() <= TOL[cfg.dtype] * np.abs(b).max()
        assert abs(sig.item() / sig_e.item() - 1) < 1e-14
    rf.close()


@pytest.mark.parametrize("cfg_index", [1, 2])
def test_noalloc_matches_the_oracle(torch, cfg_index):
    """Its own twiddles (computed on the device, unlike the context's host tables) and its
    workspace layout, against the FP64 oracle's direct matched filter (Eqs. 2-3)."""
    from oracle import mf as omf
    from paper_2511_12894_gb300 import load_library
    lib = load_library()
    cfg = workload.config(cfg_index, n_override=1 << 12, k_override=2)
    ref = cfg.groups[0][0]
    rdt = torch.float64 if cfg.dtype == "f64" else torch.float32
    cdt = torch.complex128 if cfg.dtype == "f64" else torch.complex64
    xh = data.strain(cfg)
    iph = workload.inv_psd(cfg)
    x = torch.tensor(xh, dtype=rdt, device="cuda")
    ip = torch.tensor(iph, device="cuda")
    z = torch.empty(cfg.n, dtype=cdt, device="cuda")
    sig = torch.zeros(1, dtype=torch.float64, device="cuda")
    st = lib.rf_mf_reference_noalloc(ctypes.byref(_grid(cfg)), ctypes.c_void_p(x.data_ptr()),
                                     ctypes.c_void_p(ip.data_ptr()), _templates([ref]), ctypes.c_void_p(z.data_ptr()),
                                     ctypes.c_void_p(sig.data_ptr()),
                                     ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, lib.rf_last_error()
    torch.cuda.synchronize()
    zo, so = omf.matched_filter(np.asarray(xh, dtype=np.float64), iph, cfg.n, cfg.fs, cfg.f_low, cfg.f_high,
                                ref.m1, ref.m2, cfg.pn_order)
    assert np.abs(z.cpu().numpy() - zo).max() <= TOL[cfg.dtype] * np.abs(zo).max()
    assert abs(sig.item() / so - 1) < 1e-12


def test_noalloc_rejects_oversized_segment(torch):
    from paper_2511_12894_gb300 import RF_EINVAL, load_library
    lib = load_library()
    cfg = workload.config(2, n_override=1 << 17, k_override=2)
    g = _grid(cfg)
    x = torch.zeros(cfg.n, dtype=torch.float32, device="cuda")
    ip = torch.zeros(cfg.n // 2 + 1, dtype=torch.float64, device="cuda")
    z = torch.zeros(cfg.n, dtype=torch.complex64, device="cuda")
    st = lib.rf_mf_reference_noalloc(ctypes.byref(g), ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(ip.data_ptr()),
                                     _templates([cfg.groups[0][0]]), ctypes.c_void_p(z.data_ptr()), None,
                                     ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == RF_EINVAL
    assert b"static workspace" in lib.rf_last_error()


def test_noalloc_binding_wrapper(torch):
    from paper_2511_12894_gb300 import RatioFilter, mf_reference_noalloc
    cfg = workload.config(1, n_override=1 << 13, k_override=2)
    ref = cfg.groups[0][0]
    x = torch.tensor(data.strain(cfg), device="cuda")
    ip = torch.tensor(workload.inv_psd(cfg), device="cuda")
    z = torch.empty(cfg.n, dtype=torch.complex128, device="cuda")
    mf_reference_noalloc(_grid(cfg), x, ip, ref, z)
    rf = RatioFilter.from_config(cfg)
    e, _ = rf.mf_reference(x, ip, [ref])
    torch.cuda.synchronize()
    assert (z - e[0]).abs().max().item() <= 1e-12 * e.abs().max().item()
