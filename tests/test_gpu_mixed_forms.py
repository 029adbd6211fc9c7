"""Mixed forms within one reconstruction: a kernel-length bucket of the tensor-core form (or the
direct sum) next to overlap-save buckets (rf_kernels_prepare_forms), against the oracle's
direct sum (Eq. 8), for the single-reference and batched calls, the full series and the window
peaks; the tensor-core tile layouts the autotuner times; the autotuner's mixed candidates."""
from dataclasses import replace

import numpy as np
import pytest

import workload
from oracle import reconstruct

pytestmark = pytest.mark.gpu

TOL32 = 2e-6


@pytest.fixture(scope="module")
def torch():
    import torch as t
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_12894_gb300 import build
    build.build()
    return t


def _rf(n):
    from paper_2511_12894_gb300 import RatioFilter
    return RatioFilter.from_config(workload.config(2, n_override=n, k_override=1))


def _random_set(rng, n, lengths):
    lags = [int(v) for v in rng.integers(-n // 2 + 1, n // 2, len(lengths))]
    taps = [((rng.standard_normal(L) + 1j * rng.standard_normal(L)) / np.sqrt(max(L, 1))).astype(np.complex64)
            for L in lengths]
    return lags, taps


def _check_peaks(P, A, zs, W):
    for j, zh in enumerate(zs):
        if not np.any(zh):
            continue
        zmax = np.abs(zh).max()
        Po, Ao = reconstruct.window_peaks(zh, W)
        assert np.abs(np.sqrt(P[j]) - np.sqrt(Po)).max() <= TOL32 * zmax, j
        m2 = zh.real ** 2 + zh.imag ** 2
        for w in range(Po.shape[0]):
            seg = np.sort(m2[w * W:(w + 1) * W])
            bound = 4.0 * TOL32 * zmax * np.sqrt(seg[-1])
            if seg[-1] - seg[-2] > bound:
                assert A[j, w] == Ao[w], (j, w)
            else:
                assert m2[A[j, w]] >= seg[-1] - bound


@pytest.mark.parametrize("short_form,prec,nj,s", [("gemm", "bf16x6", 0, 0), ("gemm", "bf16x6", 16, 2),
                                                  ("gemm", "bf16x6", 40, 1), ("gemm", "3xtf32", 0, 0),
                                                  ("direct", "native", 0, 0)])
def test_mixed_buckets_single_reference(torch, short_form, prec, nj, s):
    n, W = 1 << 14, 1000
    rng = np.random.default_rng(31)
    lengths = [40, 3000, 255, 9000, 1, 600, 0, 2047, 128, 5000]
    lags, taps = _random_set(rng, n, lengths)
    rf = _rf(n)
    kern = rf.kernels_import(lags, lengths, np.concatenate(taps))
    kern.prepare_forms([0, 700, 4000], [short_form, "os", "os"], [prec, "native", "native"], [nj, 2048, 8192],
                       [s, 512, 2048])
    assert kern.bucket_forms() == [(short_form, prec), ("os", "native"), ("os", "native")]
    z = (rng.standard_normal(n) + 1j * rng.standard_normal(n)).astype(np.complex64)
    zt = torch.tensor(z, device="cuda")
    zs = [reconstruct.reconstruct_direct(z.astype(np.complex128), lags[j], taps[j].astype(np.complex128))
          for j in range(len(lengths))]
    out = rf.reconstruct(zt, kern, "auto").cpu().numpy()
    for j, zh in enumerate(zs):
        assert np.abs(out[j] - zh).max() <= TOL32 * max(np.abs(zh).max(), 1e-30), j
    P, A = rf.reconstruct_winmax(zt, kern, W, "auto")
    _check_peaks(P.cpu().numpy(), A.cpu().numpy(), zs, W)


def test_mixed_buckets_batched(torch):
    """Three references, each with a tensor-core bucket below 700 taps and overlap-save above,
    in one batched call (the overlap-save part persistent, the tensor-core buckets group by
    group), rows in place."""
    n, W = 1 << 14, 1024
    rng = np.random.default_rng(32)
    rf = _rf(n)
    kerns, zts, zss = [], [], []
    for lengths in ([300, 2000, 64], [5000], [10, 700, 699, 4000, 1]):
        lags, taps = _random_set(rng, n, lengths)
        k = rf.kernels_import(lags, lengths, np.concatenate(taps))
        k.prepare_forms([0, 700], ["gemm", "os"], ["bf16x6", "native"], [0, 4096], [0, 1024])
        z = (rng.standard_normal(n) + 1j * rng.standard_normal(n)).astype(np.complex64)
        kerns.append(k)
        zts.append(torch.tensor(z, device="cuda"))
        zss.append([reconstruct.reconstruct_direct(z.astype(np.complex128), lags[j], taps[j].astype(np.complex128))
                    for j in range(len(lengths))])
    P, A = rf.reconstruct_batched(zts, kerns, W, "auto")
    P, A = P.cpu().numpy(), A.cpu().numpy()
    row = 0
    for k, zs in zip(kerns, zss):
        _check_peaks(P[row:row + k.k], A[row:row + k.k], zs, W)
        row += k.k


def test_mixed_form_refusals(torch):
    from paper_2511_12894_gb300 import RFError
    n = 1 << 14
    rng = np.random.default_rng(33)
    lags, taps = _random_set(rng, n, [100, 200])
    rf = _rf(n)
    kern = rf.kernels_import(lags, [100, 200], np.concatenate(taps))
    with pytest.raises(RFError):   # a tensor-core bucket needs a split precision
        kern.prepare_forms([0, 150], ["gemm", "os"], ["native", "native"], [0, 1024], [0, 256])
    with pytest.raises(RFError):   # not one of the two tile layouts
        kern.prepare_forms([0, 150], ["gemm", "os"], ["bf16x6", "native"], [24, 1024], [3, 256])
    with pytest.raises(RFError):   # cuts must increase
        kern.prepare_forms([0, 0], ["direct", "os"], ["native", "native"], [0, 1024], [0, 256])


def test_autotune_times_tile_layouts_and_mixed_forms(torch):
    """Short kernels: the tuner times the tensor-core form in both tile layouts and a mixed
    candidate (tensor-core below a cut, overlap-save above), and AUTO then follows the winner."""
    n, W = 1 << 15, 2048
    rng = np.random.default_rng(34)
    lengths = [int(v) for v in rng.integers(20, 300, 24)] + [int(v) for v in rng.integers(1500, 3000, 8)]
    lags, taps = _random_set(rng, n, lengths)
    rf = _rf(n)
    kern = rf.kernels_import(lags, lengths, np.concatenate(taps))
    z = (rng.standard_normal(n) + 1j * rng.standard_normal(n)).astype(np.complex64)
    zt = torch.tensor(z, device="cuda")
    table = rf.autotune([zt], [kern], W, allow_split=True)
    gemm = [e for e in table if e["algo"] == "gemm" and not e["cut"]]
    assert {(e["block"], e["part"]) for e in gemm} == {(16, 2), (40, 1)}
    mixed = [e for e in table if e["algo"] == "gemm" and e["cut"]]
    assert mixed and all(e["block2"] and e["part2"] for e in mixed)
    assert all(e["ms"] > 0 for e in table)
    zs = [reconstruct.reconstruct_direct(z.astype(np.complex128), lags[j], taps[j].astype(np.complex128))
          for j in range(len(lengths))]
    P, A = rf.reconstruct_winmax(zt, kern, W, "auto")
    _check_peaks(P.cpu().numpy(), A.cpu().numpy(), zs, W)
