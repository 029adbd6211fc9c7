"""Two-phase overlap-save (bucket form RF_ALGO_OS_BINS): the partition sums of Eq. 7's block
form per bin over runs of output blocks, then the block transforms; against the FP64 oracle's
direct sum (Eq. 8) on full series, at sampled outputs and on window peaks, for single-reference
and batched calls, complex and real-form kernels, partition ratios 2 and 4, and kernels of more
partitions than one pass over the register window holds (40)."""
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


def _random_set(rng, n, lengths, real=False):
    lags = [int(v) for v in rng.integers(-n // 2 + 1, n // 2, len(lengths))]
    if real:
        taps = [(rng.standard_normal(L) / np.sqrt(max(L, 1))).astype(np.float32) for L in lengths]
    else:
        taps = [((rng.standard_normal(L) + 1j * rng.standard_normal(L)) / np.sqrt(max(L, 1))).astype(np.complex64)
                for L in lengths]
    return lags, taps


def _check_peaks(P, A, zs, W):
    for j, zh in enumerate(zs):
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


@pytest.mark.parametrize("B,Lp,real", [(4096, 2048, False), (4096, 1024, False), (8192, 4096, True),
                                       (16384, 4096, False)])
def test_two_phase_single_reference(torch, B, Lp, real):
    n, W = 1 << 15, 2000
    rng = np.random.default_rng(B + Lp + real)
    lengths = [1, 700, 2048, 5000, 9000, 13000, 3, 4096]
    lags, taps = _random_set(rng, n, lengths, real)
    rf = _rf(n)
    kern = rf.kernels_import(lags, lengths, np.concatenate(taps), real=real)
    kern.prepare_forms([0], ["os_bins"], ["native"], [B], [Lp])
    assert kern.bucket_forms() == [("os_bins", "native")]
    z = (rng.standard_normal(n) + 1j * rng.standard_normal(n)).astype(np.complex64)
    zt = torch.tensor(z, device="cuda")
    zs = [reconstruct.reconstruct_direct(z.astype(np.complex128), lags[j], taps[j].astype(np.complex128))
          for j in range(len(lengths))]
    out = rf.reconstruct(zt, kern, "auto").cpu().numpy()
    for j, zh in enumerate(zs):
        assert np.abs(out[j] - zh).max() <= TOL32 * np.abs(zh).max(), (j, np.abs(out[j] - zh).max() / np.abs(zh).max())
    P, A = rf.reconstruct_winmax(zt, kern, W, "auto")
    _check_peaks(P.cpu().numpy(), A.cpu().numpy(), zs, W)


@pytest.mark.parametrize("n,B,Lp,lengths", [
    # Q = 4: up to 59 partitions, two passes (the second adding to the buffer)
    (1 << 16, 4096, 1024, [60000, 49 * 1024, 48 * 1024, 30000, 47 * 1024 + 1, 40 * 1024, 40 * 1024 + 1,
                           32 * 1024 + 1]),
    # Q = 2: up to 44 partitions, two passes
    (1 << 17, 4096, 2048, [90000, 80 * 1024, 80 * 1024 + 1, 10000, 82 * 1024 + 1]),
    # 32768-point blocks on CTA pairs (parity-split spectra, the pair's block tail)
    (1 << 17, 32768, 16384, [90000, 5 * 16384, 5 * 16384 + 1, 10000, 16384, 1, 300]),
])
def test_two_phase_many_partitions(torch, n, B, Lp, lengths):
    """Kernels of more partitions than one phase-1 pass holds (several passes over the register
    window, the later ones adding to the buffer), and the pair layout, sampled outputs by the
    oracle's defining sum."""
    W = 2048
    rng = np.random.default_rng(60)
    lags, taps = _random_set(rng, n, lengths)
    rf = _rf(n)
    kern = rf.kernels_import(lags, lengths, np.concatenate(taps))
    kern.prepare_forms([0], ["os_bins"], ["native"], [B], [Lp])
    z = (rng.standard_normal(n) + 1j * rng.standard_normal(n)).astype(np.complex64)
    zt = torch.tensor(z, device="cuda")
    out = rf.reconstruct(zt, kern, "auto").cpu().numpy()
    P, A = rf.reconstruct_winmax(zt, kern, W, "auto")
    P, A = P.cpu().numpy(), A.cpu().numpy()
    zd = z.astype(np.complex128)
    for j in range(len(lengths)):
        c = taps[j].astype(np.complex128)
        idx = rng.choice(n, 192, replace=False)
        ref = reconstruct.reconstruct_at(zd, lags[j], c, idx)
        zmax = np.abs(out[j]).max()
        assert np.abs(out[j][idx] - ref).max() <= TOL32 * zmax, j
        # the reported peaks against the defining sum at their indices, and against the series
        wins = rng.choice(P.shape[1], 6, replace=False)
        vals = np.abs(reconstruct.reconstruct_at(zd, lags[j], c, A[j, wins].astype(np.int64)))
        assert np.abs(np.sqrt(P[j, wins]) - vals).max() <= TOL32 * zmax
        m2 = np.abs(out[j]) ** 2
        Pg, _ = reconstruct.window_peaks(out[j].astype(np.complex128), W)
        assert np.abs(np.sqrt(P[j]) - np.sqrt(Pg)).max() <= TOL32 * zmax


@pytest.mark.parametrize("n,B2,Lp2,long_lengths", [
    (1 << 15, 8192, 2048, (7000, 12000, 9000, 4000)),
    # the pair layout's two-phase bucket (32768-point blocks on CTA pairs)
    (1 << 16, 32768, 16384, (7000, 20000, 17000, 4000)),
])
def test_two_phase_batched_next_to_single_pass(torch, n, B2, Lp2, long_lengths):
    """Three references: single-pass overlap-save below 3000 taps, two-phase above, one batched
    call (the two-phase launches cover every reference's long kernels together)."""
    W = 1024
    rng = np.random.default_rng(33)
    rf = _rf(n)
    kerns, zts, zss = [], [], []
    a, b, c, d = long_lengths
    for lengths in ([300, a, b], [3000], [10, 2999, c, d, 1]):
        lags, taps = _random_set(rng, n, lengths)
        k = rf.kernels_import(lags, lengths, np.concatenate(taps))
        k.prepare_forms([0, 3000], ["os", "os_bins"], ["native", "native"], [4096, B2], [1024, Lp2])
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


def test_two_phase_layouts_refused(torch):
    from paper_2511_12894_gb300 import RFError
    n = 1 << 15
    rng = np.random.default_rng(34)
    lags, taps = _random_set(rng, n, [100, 5000])
    rf = _rf(n)
    kern = rf.kernels_import(lags, [100, 5000], np.concatenate(taps))
    with pytest.raises(RFError):   # block sizes 4096, 8192, 16384 (and 32768 on CTA pairs) only
        kern.prepare_forms([0], ["os_bins"], ["native"], [2048], [1024])
    with pytest.raises(RFError):   # partitions of B/2 or B/4
        kern.prepare_forms([0], ["os_bins"], ["native"], [8192], [1024])
    with pytest.raises(RFError):   # the pair layout with partitions of B/2 only
        kern.prepare_forms([0], ["os_bins"], ["native"], [32768], [8192])


@pytest.mark.parametrize("B2,Lp2", [(8192, 4096), (32768, 16384)])
def test_two_phase_waves_batched_and_graph(torch, B2, Lp2):
    """Three references x 12 long kernels: three waves of two-phase launches (two buffers, phase 2
    on the library's second stream beside the next wave's phase 1).  The batched call equals the
    per-reference calls row for row, and replays from a CUDA graph with the same result."""
    n, W = 1 << 15, 1024
    rng = np.random.default_rng(35)
    rf = _rf(n)
    kerns, zts = [], []
    for _ in range(3):
        lengths = [int(v) for v in rng.integers(3000, 20000, 12)]
        lags, taps = _random_set(rng, n, lengths)
        k = rf.kernels_import(lags, lengths, np.concatenate(taps))
        k.prepare_forms([0, 2000], ["os", "os_bins"], ["native", "native"], [4096, B2], [1024, Lp2])
        kerns.append(k)
        z = (rng.standard_normal(n) + 1j * rng.standard_normal(n)).astype(np.complex64)
        zts.append(torch.tensor(z, device="cuda"))
    P, A = rf.reconstruct_batched(zts, kerns, W, "auto")
    row = 0
    for g, k in enumerate(kerns):
        Pg, Ag = rf.reconstruct_winmax(zts[g], k, W, "auto")
        assert torch.equal(P[row:row + k.k], Pg) and torch.equal(A[row:row + k.k], Ag), g
        row += k.k
    P2, A2 = torch.zeros_like(P), torch.zeros_like(A)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        rf.reconstruct_batched(zts, kerns, W, "auto", max_out=P2, arg_out=A2)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    P2.zero_()
    A2.zero_()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        rf.reconstruct_batched(zts, kerns, W, "auto", max_out=P2, arg_out=A2)
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(P2, P) and torch.equal(A2, A)
