"""Ratio-filter SNR reconstruction on one GB300 (sm_103a).

Thin Python binding of the C ABI in ``include/rf.h`` (``librf.so``): argument
marshalling only.  Every step of the computation runs in the library's CUDA
kernels; PyTorch supplies device memory and streams.  There is no CPU
fallback: importing works without a GPU, but creating a context needs the
built library and a CUDA device, and fails loudly otherwise.

Names follow the paper (Murakami, Ghosh & Morisaki): ``mf_reference`` (Sec.
II.A), ``build_ratio_kernels`` (Sec. II.B-II.D), ``reconstruct`` and
``reconstruct_winmax`` (Eq. 8 and the per-window peak).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import Iterable, Optional, Sequence, Tuple

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librf.so")

RF_OK, RF_EINVAL, RF_ENOMEM, RF_ECUDA, RF_ETIMEOUT, RF_EUNSUPPORTED = 0, -1, -2, -3, -4, -5
RF_F64, RF_F32 = 0, 1
ALGOS = {"auto": 0, "direct": 1, "os": 2, "gemm": 3, "os_bins": 4}   # os_bins: a bucket form only
RF_TRUNC_RELATIVE = 1
RF_TRUNC_ANALYTIC = 2
RF_KERNEL_REAL = 4
PRECS = {"native": 0, "bf16": 1, "bf16x3": 2, "bf16x6": 3, "bf16x9": 4, "3xtf32": 5}

EXPORTED = (
    "rf_version", "rf_launch_count", "rf_last_error", "rf_create", "rf_destroy", "rf_reserve", "rf_template_fd",
    "rf_mf_reference", "rf_build_ratio_kernels", "rf_kernels_import", "rf_kernels_import_real",
    "rf_kernels_is_real", "rf_kernels_info", "rf_kernels_prepare",
    "rf_kernels_os_layout", "rf_kernels_prepare_buckets", "rf_kernels_prepare_forms", "rf_kernels_bucket_forms",
    "rf_kernels_os_buckets", "rf_kernels_grids",
    "rf_kernels_gemm_layout", "rf_bank_structure", "rf_stream_winmax",
    "rf_kernels_copy_taps", "rf_kernels_free", "rf_reconstruct", "rf_reconstruct_winmax", "rf_reconstruct_batched", "rf_winmax",
    "rf_mf_reference_noalloc", "rf_device_status", "rf_reference_filters", "rf_mf_filtered",
    "rf_selftest_bounded_wait", "rf_autotune",
)


class rf_tune_entry(ctypes.Structure):
    _fields_ = [("algo", ctypes.c_int32), ("block", ctypes.c_int32), ("part", ctypes.c_int32),
                ("prec", ctypes.c_int32), ("cut", ctypes.c_int32), ("block2", ctypes.c_int32),
                ("part2", ctypes.c_int32), ("algo2", ctypes.c_int32), ("cut3", ctypes.c_int32),
                ("block3", ctypes.c_int32), ("part3", ctypes.c_int32), ("algo3", ctypes.c_int32),
                ("ms", ctypes.c_float)]


class RFError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"rf status {status}: {msg}")
        self.status = status


class rf_template(ctypes.Structure):
    _fields_ = [("m1", ctypes.c_double), ("m2", ctypes.c_double), ("tc", ctypes.c_double),
                ("phic", ctypes.c_double)]


class rf_grid(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("fs", ctypes.c_double), ("f_low", ctypes.c_double),
                ("f_high", ctypes.c_double), ("df_high", ctypes.c_double), ("df_low_max", ctypes.c_double),
                ("pn_order", ctypes.c_int32), ("dtype", ctypes.c_int32)]


_lib = None


def load_library(path: Optional[str] = None) -> ctypes.CDLL:
    """Load librf.so (built by ``build.build()``); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"{p} not found: build it first (python -c 'import __graft_entry__ as g; g.build()')")
    lib = ctypes.CDLL(p)
    vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    P = ctypes.POINTER
    sig = {
        "rf_version": (i32, []),
        "rf_launch_count": (ctypes.c_uint64, []),
        "rf_last_error": (ctypes.c_char_p, []),
        "rf_create": (i32, [P(rf_grid), P(vp)]),
        "rf_destroy": (None, [vp]),
        "rf_reserve": (i32, [vp, i32, P(i64)]),
        "rf_template_fd": (i32, [vp, P(rf_template), vp, vp]),
        "rf_mf_reference": (i32, [vp, vp, vp, i32, P(rf_template), vp, vp, vp]),
        "rf_build_ratio_kernels": (i32, [vp, P(rf_template), P(rf_template), i32, vp, dbl, i32, i64, P(vp), vp]),
        "rf_kernels_grids": (i32, [vp, P(P(i64))]),
        "rf_kernels_import": (i32, [vp, i32, P(i32), P(i32), vp, P(vp)]),
        "rf_kernels_import_real": (i32, [vp, i32, P(i32), P(i32), vp, P(vp)]),
        "rf_kernels_is_real": (i32, [vp, P(i32)]),
        "rf_kernels_info": (i32, [vp, P(i32), P(P(i32)), P(P(i32)), P(P(i64)), P(P(dbl)), P(vp)]),
        "rf_kernels_copy_taps": (i32, [vp, vp, vp]),
        "rf_kernels_prepare": (i32, [vp, vp, i32, i32, vp]),
        "rf_kernels_os_layout": (i32, [vp, P(i32), P(i32)]),
        "rf_kernels_gemm_layout": (i32, [vp, P(i32)]),
        "rf_bank_structure": (i32, [vp, i32, dbl, i32, dbl, i32, P(i32), P(i32), P(i32), P(dbl)]),
        "rf_stream_winmax": (i32, [vp, vp, i64, i32, vp, vp, i64, i64, vp, vp, vp, vp, vp]),
        "rf_kernels_prepare_buckets": (i32, [vp, vp, i32, P(i32), P(i32), P(i32), vp]),
        "rf_kernels_os_buckets": (i32, [vp, i32, P(i32), P(i32), P(i32), P(i32)]),
        "rf_kernels_prepare_forms": (i32, [vp, vp, i32, P(i32), P(i32), P(i32), P(i32), P(i32), vp]),
        "rf_kernels_bucket_forms": (i32, [vp, i32, P(i32), P(i32), P(i32)]),
        "rf_kernels_free": (None, [vp]),
        "rf_reconstruct": (i32, [vp, vp, vp, i32, i32, vp, vp]),
        "rf_reconstruct_winmax": (i32, [vp, vp, vp, i32, i32, i64, vp, vp, vp]),
        "rf_winmax": (i32, [vp, vp, i32, i64, vp, vp, vp]),
        "rf_reconstruct_batched": (i32, [vp, i32, P(vp), P(vp), i32, i32, i64, vp, vp, vp]),
        "rf_mf_reference_noalloc": (i32, [P(rf_grid), vp, vp, P(rf_template), vp, vp, vp]),
        "rf_reference_filters": (i32, [vp, vp, i32, P(rf_template), vp, vp, vp]),
        "rf_mf_filtered": (i32, [vp, vp, i32, vp, vp, vp]),
        "rf_selftest_bounded_wait": (i32, [vp, vp]),
        "rf_autotune": (i32, [vp, i32, P(vp), P(vp), i64, i32, i32, P(rf_tune_entry), i32, P(i32), vp]),
        "rf_device_status": (i32, [vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def launch_count() -> int:
    """Kernels launched by the library so far in this process."""
    return int(load_library().rf_launch_count())


def _check(status: int) -> None:
    if status != RF_OK:
        msg = _lib.rf_last_error().decode(errors="replace") if _lib else ""
        raise RFError(status, msg)


def bank_structure(bank: Sequence, f_low: float, pn_order: int = 7, max_spread: float = 10.0,
                   max_size: int = 500):
    """Template-bank structuring (Sec. III.A) by the library, on the host: (sets, refs,
    durations) with sets lists of bank indices (depth first), refs the bank index of each
    set's reference and durations tau = -t(f_low) in seconds."""
    import numpy as np
    lib = load_library()
    n = len(bank)
    set_of = (ctypes.c_int32 * max(1, n))()
    refs = (ctypes.c_int32 * max(1, n))()
    ns = ctypes.c_int32(0)
    tau = (ctypes.c_double * max(1, n))()
    _check(lib.rf_bank_structure(_templates(bank), n, float(f_low), int(pn_order), float(max_spread), int(max_size),
                                 set_of, refs, ctypes.byref(ns), tau))
    sets = [[] for _ in range(ns.value)]
    for i in range(n):
        sets[set_of[i]].append(i)
    return sets, [refs[g] for g in range(ns.value)], np.array(tau[:n])


def _templates(ts: Sequence) -> ctypes.Array:
    arr = (rf_template * max(1, len(ts)))()
    for i, t in enumerate(ts):
        arr[i] = rf_template(float(t.m1), float(t.m2), float(getattr(t, "tc", 0.0)), float(getattr(t, "phic", 0.0)))
    return arr


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _need(t, count: int, name: str):
    """Raise unless ``t`` holds at least ``count`` elements: the library reads or writes that
    many through a raw pointer and cannot check the buffer's size itself."""
    if t.numel() < count:
        raise ValueError(f"{name} holds {t.numel()} elements; the call needs {count}")
    return t


def _dev(t, dtype, name, count: int = 0):
    """Contiguous, 16-byte-aligned CUDA tensor of the given dtype with at least ``count``
    elements (copied only if its layout needs it)."""
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch tensor")
    _need(t, count, name)
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must have dtype {dtype}, got {t.dtype}")
    if not t.is_contiguous() or t.data_ptr() % 16:
        t = t.contiguous().clone()
    return t


def _out(t, dtype, count: int, name: str):
    """A caller's output tensor, written in place (so never copied): CUDA, of the given dtype,
    contiguous, 16-byte aligned and holding at least ``count`` elements."""
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch tensor")
    _need(t, count, name)
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must have dtype {dtype}, got {t.dtype}")
    if not t.is_contiguous() or t.data_ptr() % 16:
        raise ValueError(f"{name} must be contiguous and 16-byte aligned (it is written in place)")
    return t


@dataclass
class Kernels:
    """A set of truncated ratio kernels held by the library (device taps)."""
    handle: ctypes.c_void_p
    ctx: "RatioFilter"
    k: int
    length: np.ndarray
    lag0: np.ndarray
    offset: np.ndarray
    df_low: np.ndarray
    grid: np.ndarray = None   # build grid of each kernel
    real: bool = False        # real-form taps (stored as real values)

    def taps(self):
        """Packed taps as a new CUDA tensor (sum(length) entries: complex, or real for a
        real-form set)."""
        import torch
        dt = self.ctx.rdtype if self.real else self.ctx.cdtype
        t = torch.empty(int(self.offset[-1]), dtype=dt, device="cuda")
        if t.numel():
            _check(_lib.rf_kernels_copy_taps(self.handle, ctypes.c_void_p(t.data_ptr()), _stream()))
        return t

    def prepare(self, block: int = 0, part: int = 0, stream=None) -> None:
        """Overlap-save preparation with block size ``block`` and partition length ``part``
        (0: defaults); synchronises."""
        _check(_lib.rf_kernels_prepare(self.ctx.handle, self.handle, int(block), int(part), _stream(stream)))

    def prepare_buckets(self, cuts: Sequence[int], blocks: Sequence[int], parts: Sequence[int], stream=None) -> None:
        """Overlap-save layout per kernel-length bucket: bucket b takes cuts[b] <= L < cuts[b+1]."""
        nb = len(cuts)
        arr = lambda v: (ctypes.c_int32 * nb)(*[int(x) for x in v])
        _check(_lib.rf_kernels_prepare_buckets(self.ctx.handle, self.handle, nb, arr(cuts), arr(blocks), arr(parts),
                                               _stream(stream)))

    def prepare_forms(self, cuts: Sequence[int], algos: Sequence[str], precs: Sequence[str],
                      blocks: Sequence[int], parts: Sequence[int], stream=None) -> None:
        """A form per kernel-length bucket: 'os' (blocks/parts = block size, partition length),
        'gemm' (precs = split precision, blocks/parts = tile layout or 0, 0) or 'direct'."""
        nb = len(cuts)
        arr = lambda v: (ctypes.c_int32 * nb)(*[int(x) for x in v])
        _check(_lib.rf_kernels_prepare_forms(self.ctx.handle, self.handle, nb, arr(cuts),
                                             arr([ALGOS[a] for a in algos]), arr([PRECS[p] for p in precs]),
                                             arr(blocks), arr(parts), _stream(stream)))

    def bucket_forms(self):
        """[(algo, prec), ...] of the bucketed preparation ([] if none)."""
        a, p = (ctypes.c_int32 * 8)(), (ctypes.c_int32 * 8)()
        nb = ctypes.c_int32(0)
        _check(_lib.rf_kernels_bucket_forms(self.handle, 8, a, p, ctypes.byref(nb)))
        an = {v: k for k, v in ALGOS.items()}
        pn = {v: k for k, v in PRECS.items()}
        return [(an[a[i]], pn[p[i]]) for i in range(nb.value)]

    def os_buckets(self):
        """[(cut, block, part), ...] of the overlap-save preparation ([] if none)."""
        c, b, p = (ctypes.c_int32 * 8)(), (ctypes.c_int32 * 8)(), (ctypes.c_int32 * 8)()
        nb = ctypes.c_int32(0)
        _check(_lib.rf_kernels_os_buckets(self.handle, 8, c, b, p, ctypes.byref(nb)))
        return [(c[i], b[i], p[i]) for i in range(nb.value)]

    def os_layout(self):
        """(block size, partition length) of the overlap-save preparation, (0, 0) if none."""
        b, p = ctypes.c_int32(0), ctypes.c_int32(0)
        _check(_lib.rf_kernels_os_layout(self.handle, ctypes.byref(b), ctypes.byref(p)))
        return b.value, p.value

    def gemm_layout(self):
        """Tensor-core layout of the last RF_ALGO_GEMM call: dict of prec, neighbours per group
        (nj), stacked output tiles (shifts), taps per K chunk (kc), chunks (nck) and padded
        length (lp); None when not prepared."""
        o = (ctypes.c_int32 * 6)()
        _check(_lib.rf_kernels_gemm_layout(self.handle, o))
        if o[1] == 0:
            return None
        pn = {v: k for k, v in PRECS.items()}
        return {"prec": pn[o[0]], "nj": o[1], "shifts": o[2], "kc": o[3], "nck": o[4], "lp": o[5]}

    def free(self) -> None:
        if self.handle:
            _lib.rf_kernels_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class RatioFilter:
    """One analysis grid on the current CUDA device (owns an ``rf_ctx``)."""

    def __init__(self, n: int, fs: float, f_low: float, f_high: float, pn_order: int, dtype: str = "f32",
                 df_high: float = 53.0, df_low_max: float = 5.0):
        import torch
        lib = load_library()
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required (there is no CPU fallback)")
        self.n = int(n)
        self.fs = float(fs)
        self.dtype = dtype
        self.rdtype = torch.float64 if dtype == "f64" else torch.float32
        self.cdtype = torch.complex128 if dtype == "f64" else torch.complex64
        g = rf_grid(self.n, self.fs, float(f_low), float(f_high), float(df_high), float(df_low_max), int(pn_order),
                    RF_F64 if dtype == "f64" else RF_F32)
        h = ctypes.c_void_p()
        _check(lib.rf_create(ctypes.byref(g), ctypes.byref(h)))
        self.handle = h

    @classmethod
    def from_config(cls, cfg) -> "RatioFilter":
        return cls(cfg.n, cfg.fs, cfg.f_low, cfg.f_high, cfg.pn_order, cfg.dtype, cfg.df_high, cfg.df_low_max)

    def close(self) -> None:
        if getattr(self, "handle", None):
            _lib.rf_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------ calls
    def reserve(self, k_max: int) -> int:
        b = ctypes.c_int64()
        _check(_lib.rf_reserve(self.handle, int(k_max), ctypes.byref(b)))
        return b.value

    def template_fd(self, tmpl, out=None, stream=None):
        import torch
        nf = self.n // 2 + 1
        out = _out(out, self.cdtype, nf, "out") if out is not None else \
            torch.empty(nf, dtype=self.cdtype, device="cuda")
        t = _templates([tmpl])
        _check(_lib.rf_template_fd(self.handle, t, ctypes.c_void_p(out.data_ptr()), _stream(stream)))
        return out

    def mf_reference(self, x, inv_psd, refs: Sequence, z_out=None, sigma_out=None, stream=None):
        """z_ref[nref, n] (complex) and N[nref] (float64) of each reference (Sec. II.A)."""
        import torch
        x = _dev(x, self.rdtype, "x", self.n)
        ip = _dev(inv_psd, torch.float64, "inv_psd", self.n // 2 + 1)
        nref = len(refs)
        z = _out(z_out, self.cdtype, nref * self.n, "z_out") if z_out is not None else \
            torch.empty((nref, self.n), dtype=self.cdtype, device="cuda")
        sg = _out(sigma_out, torch.float64, nref, "sigma_out") if sigma_out is not None else \
            torch.empty(nref, dtype=torch.float64, device="cuda")
        _check(_lib.rf_mf_reference(self.handle, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(ip.data_ptr()),
                                    nref, _templates(refs), ctypes.c_void_p(z.data_ptr()),
                                    ctypes.c_void_p(sg.data_ptr()), _stream(stream)))
        return z, sg

    def reference_filters(self, inv_psd, refs: Sequence, filt_out=None, sigma_out=None, stream=None):
        """Stored filters [nref, n/2+1] (complex) and N[nref] of each reference (Sec. II.A)."""
        import torch
        nf = self.n // 2 + 1
        ip = _dev(inv_psd, torch.float64, "inv_psd", nf)
        nref = len(refs)
        f = _out(filt_out, self.cdtype, nref * nf, "filt_out") if filt_out is not None else \
            torch.empty((nref, nf), dtype=self.cdtype, device="cuda")
        sg = _out(sigma_out, torch.float64, nref, "sigma_out") if sigma_out is not None else \
            torch.empty(nref, dtype=torch.float64, device="cuda")
        _check(_lib.rf_reference_filters(self.handle, ctypes.c_void_p(ip.data_ptr()), nref, _templates(refs),
                                         ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(sg.data_ptr()),
                                         _stream(stream)))
        return f, sg

    def mf_filtered(self, x, filt, z_out=None, stream=None):
        """z_ref[nref, n] from stored filters ``filt`` [nref, n/2+1]."""
        import torch
        x = _dev(x, self.rdtype, "x", self.n)
        filt = _dev(filt, self.cdtype, "filt", self.n // 2 + 1)
        f2 = filt.reshape(-1, self.n // 2 + 1)
        nref = f2.shape[0]
        z = _out(z_out, self.cdtype, nref * self.n, "z_out") if z_out is not None else \
            torch.empty((nref, self.n), dtype=self.cdtype, device="cuda")
        _check(_lib.rf_mf_filtered(self.handle, ctypes.c_void_p(x.data_ptr()), nref, ctypes.c_void_p(f2.data_ptr()),
                                   ctypes.c_void_p(z.data_ptr()), _stream(stream)))
        return z

    def _wrap_kernels(self, h: ctypes.c_void_p) -> Kernels:
        k = ctypes.c_int32()
        ln = ctypes.POINTER(ctypes.c_int32)()
        lg = ctypes.POINTER(ctypes.c_int32)()
        of = ctypes.POINTER(ctypes.c_int64)()
        dl = ctypes.POINTER(ctypes.c_double)()
        _check(_lib.rf_kernels_info(h, ctypes.byref(k), ctypes.byref(ln), ctypes.byref(lg), ctypes.byref(of),
                                    ctypes.byref(dl), None))
        kk = k.value
        arr = lambda p, m, dt: np.ctypeslib.as_array(p, shape=(m,)).astype(dt).copy() if m else np.zeros(m, dt)
        gp = ctypes.POINTER(ctypes.c_int64)()
        _check(_lib.rf_kernels_grids(h, ctypes.byref(gp)))
        real = ctypes.c_int32(0)
        _check(_lib.rf_kernels_is_real(h, ctypes.byref(real)))
        return Kernels(h, self, kk, arr(ln, kk, np.int64), arr(lg, kk, np.int64), arr(of, kk + 1, np.int64),
                       arr(dl, kk, np.float64), arr(gp, kk, np.int64), bool(real.value))

    def build_ratio_kernels(self, ref, nbrs: Sequence, inv_psd, threshold: float = 1e-3, relative: bool = True,
                            stream=None, n_build: int = 0, analytic: bool = False, real: bool = False) -> Kernels:
        """Truncated ratio kernels of ``nbrs`` against ``ref`` (Sec. II.B-II.D); synchronises.

        n_build: 0 on the data grid, a power of two for that build grid, -1 per neighbour.
        analytic: kept lags from the App. A expressions (threshold amplitude on |r| in 1/s, or
        relative to the kernel's peak) instead of the kernel's own magnitudes.
        real: the paper's real-kernel form, taps 2 Re rho."""
        import torch
        ip = _dev(inv_psd, torch.float64, "inv_psd", self.n // 2 + 1)
        h = ctypes.c_void_p()
        flags = (RF_TRUNC_RELATIVE if relative else 0) | (RF_TRUNC_ANALYTIC if analytic else 0) | \
            (RF_KERNEL_REAL if real else 0)
        _check(_lib.rf_build_ratio_kernels(self.handle, _templates([ref]), _templates(nbrs), len(nbrs),
                                           ctypes.c_void_p(ip.data_ptr()), float(threshold), flags,
                                           int(n_build), ctypes.byref(h), _stream(stream)))
        return self._wrap_kernels(h)

    def kernels_import(self, lag0: Iterable[int], length: Iterable[int], taps: np.ndarray,
                       real: bool = False) -> Kernels:
        """Kernels from host arrays (signed first lags, lengths, packed taps: complex, or real
        values for a real-form set)."""
        lag0 = np.ascontiguousarray(lag0, dtype=np.int32)
        length = np.ascontiguousarray(length, dtype=np.int32)
        if real:
            taps = np.ascontiguousarray(taps, dtype=np.float64 if self.dtype == "f64" else np.float32)
        else:
            taps = np.ascontiguousarray(taps, dtype=np.complex128 if self.dtype == "f64" else np.complex64)
        if taps.size < int(length.sum()):
            raise ValueError(f"taps holds {taps.size} values; the lengths need {int(length.sum())}")
        h = ctypes.c_void_p()
        P32 = ctypes.POINTER(ctypes.c_int32)
        fn = _lib.rf_kernels_import_real if real else _lib.rf_kernels_import
        _check(fn(self.handle, len(length), lag0.ctypes.data_as(P32), length.ctypes.data_as(P32),
                  ctypes.c_void_p(taps.ctypes.data), ctypes.byref(h)))
        return self._wrap_kernels(h)

    def reconstruct(self, z_ref, kern: Kernels, algo: str = "auto", out=None, stream=None, prec: str = "native"):
        """Neighbour SNR series [k, n] (Eq. 8)."""
        import torch
        z_ref = _dev(z_ref, self.cdtype, "z_ref", self.n)
        out = _out(out, self.cdtype, kern.k * self.n, "out") if out is not None else \
            torch.empty((kern.k, self.n), dtype=self.cdtype, device="cuda")
        _check(_lib.rf_reconstruct(self.handle, ctypes.c_void_p(z_ref.data_ptr()), kern.handle, ALGOS[algo],
                                   PRECS[prec], ctypes.c_void_p(out.data_ptr()), _stream(stream)))
        return out

    def device_status(self) -> None:
        """Raise if a bounded device-side wait of an earlier call ran out (synchronises)."""
        _check(_lib.rf_device_status(self.handle))

    def autotune(self, z_refs: Sequence, kerns: Sequence[Kernels], W: int, allow_split: bool = False,
                 max_os: int = 4, stream=None):
        """Time candidate forms for this batch and record the fastest in every kernel set.

        Returns the timed candidates, the winner first: dicts with algo, block, part, prec, ms."""
        G = len(z_refs)
        zs = [_dev(z, self.cdtype, "z_refs[g]", self.n) for z in z_refs]
        zp = (ctypes.c_void_p * G)(*[z.data_ptr() for z in zs])
        kp = (ctypes.c_void_p * G)(*[k.handle.value if isinstance(k.handle, ctypes.c_void_p) else k.handle
                                     for k in kerns])
        out = (rf_tune_entry * 64)()
        n = ctypes.c_int32(0)
        _check(_lib.rf_autotune(self.handle, G, zp, kp, int(W), 1 if allow_split else 0, int(max_os), out, 64,
                                ctypes.byref(n), _stream(stream)))
        names = {v: k for k, v in ALGOS.items()}
        pnames = {v: k for k, v in PRECS.items()}
        return [{"algo": names[e.algo], "block": e.block, "part": e.part, "prec": pnames[e.prec], "cut": e.cut,
                 "block2": e.block2, "part2": e.part2, "algo2": names[e.algo2] if e.cut else None,
                 "cut3": e.cut3, "block3": e.block3, "part3": e.part3, "algo3": names[e.algo3] if e.cut3 else None,
                 "ms": e.ms} for e in out[:n.value]]

    def selftest_bounded_wait(self, stream=None) -> None:
        """Exercise the timeout path: the next device_status() raises RF_ETIMEOUT."""
        _check(_lib.rf_selftest_bounded_wait(self.handle, _stream(stream)))

    def reconstruct_winmax(self, z_ref, kern: Kernels, W: int, algo: str = "auto", max_out=None, arg_out=None,
                           stream=None, prec: str = "native"):
        """Per-window max|z|^2 [k, nw] (float32) and its first index (int32)."""
        import torch
        z_ref = _dev(z_ref, self.cdtype, "z_ref", self.n)
        nw = -(-self.n // int(W))
        mo = _out(max_out, torch.float32, kern.k * nw, "max_out") if max_out is not None else \
            torch.empty((kern.k, nw), dtype=torch.float32, device="cuda")
        ao = _out(arg_out, torch.int32, kern.k * nw, "arg_out") if arg_out is not None else \
            torch.empty((kern.k, nw), dtype=torch.int32, device="cuda")
        _check(_lib.rf_reconstruct_winmax(self.handle, ctypes.c_void_p(z_ref.data_ptr()), kern.handle, ALGOS[algo],
                                          PRECS[prec], int(W), ctypes.c_void_p(mo.data_ptr()),
                                          ctypes.c_void_p(ao.data_ptr()), _stream(stream)))
        return mo, ao

    def reconstruct_batched(self, z_refs: Sequence, kerns: Sequence[Kernels], W: int, algo: str = "auto",
                            max_out=None, arg_out=None, stream=None, prec: str = "native"):
        """Fused window peaks of several references' neighbours in one persistent launch.

        z_refs: CUDA complex tensors of length n (one per reference); kerns: their kernel
        sets.  Returns ([sum k, nw] float32 peaks, int32 first indices), groups in order."""
        import torch
        G = len(z_refs)
        zs = [_dev(z, self.cdtype, "z_refs[g]", self.n) for z in z_refs]
        rows = sum(k.k for k in kerns)
        nw = -(-self.n // int(W))
        mo = _out(max_out, torch.float32, rows * nw, "max_out") if max_out is not None else \
            torch.empty((rows, nw), dtype=torch.float32, device="cuda")
        ao = _out(arg_out, torch.int32, rows * nw, "arg_out") if arg_out is not None else \
            torch.empty((rows, nw), dtype=torch.int32, device="cuda")
        zp = (ctypes.c_void_p * G)(*[z.data_ptr() for z in zs])
        kp = (ctypes.c_void_p * G)(*[k.handle.value if isinstance(k.handle, ctypes.c_void_p) else k.handle
                                     for k in kerns])
        _check(_lib.rf_reconstruct_batched(self.handle, G, zp, kp, ALGOS[algo], PRECS[prec], int(W),
                                           ctypes.c_void_p(mo.data_ptr()), ctypes.c_void_p(ao.data_ptr()),
                                           _stream(stream)))
        return mo, ao

    def stream_winmax(self, x, filt, kerns: Sequence[Kernels], W: int, guard: int, stream=None):
        """Window peaks over a host strain longer than one segment (segments overlapping by
        2 guard samples, each window from the segment whose interior holds it).  x: host
        real array (grid dtype); filt: the references' stored filters (reference_filters).
        Returns numpy (ref_max [G, nwt], ref_arg int64, nbr_max [sum k, nwt], nbr_arg int64)."""
        import numpy as np
        x = np.ascontiguousarray(x, dtype=np.float64 if self.dtype == "f64" else np.float32)
        G = len(kerns)
        fl = _dev(filt, self.cdtype, "filt", G * (self.n // 2 + 1))
        nwt = x.size // int(W)
        rows = sum(k.k for k in kerns)
        rm, ra = np.zeros((G, nwt), np.float32), np.zeros((G, nwt), np.int64)
        nm, na = np.zeros((max(rows, 1), nwt), np.float32), np.zeros((max(rows, 1), nwt), np.int64)
        kp = (ctypes.c_void_p * G)(*[k.handle.value if isinstance(k.handle, ctypes.c_void_p) else k.handle
                                     for k in kerns])
        p = lambda a: ctypes.c_void_p(a.ctypes.data)
        _check(_lib.rf_stream_winmax(self.handle, p(x), x.size, G, ctypes.c_void_p(fl.data_ptr()), kp, int(W),
                                     int(guard), p(rm), p(ra), p(nm), p(na), _stream(stream)))
        return rm, ra, nm[:rows], na[:rows]

    def winmax(self, z, W: int, max_out=None, arg_out=None, stream=None):
        """Window peaks of series already in memory, z[count, n]."""
        import torch
        z = _dev(z, self.cdtype, "z", self.n)
        z2 = z.reshape(-1, self.n)
        nw = -(-self.n // int(W))
        cnt = z2.shape[0] * nw
        mo = _out(max_out, torch.float32, cnt, "max_out") if max_out is not None else \
            torch.empty((z2.shape[0], nw), dtype=torch.float32, device="cuda")
        ao = _out(arg_out, torch.int32, cnt, "arg_out") if arg_out is not None else \
            torch.empty((z2.shape[0], nw), dtype=torch.int32, device="cuda")
        _check(_lib.rf_winmax(self.handle, ctypes.c_void_p(z2.data_ptr()), z2.shape[0], int(W),
                              ctypes.c_void_p(mo.data_ptr()), ctypes.c_void_p(ao.data_ptr()), _stream(stream)))
        return mo, ao


def mf_reference_noalloc(grid: rf_grid, x, inv_psd, ref, z_out, sigma_out=None, stream=None) -> None:
    """The reference matched filter for callers that cannot allocate device memory.

    Wraps ``rf_mf_reference_noalloc``: the library allocates nothing and uses a static
    device workspace (n <= 2^16).  All buffers are the caller's CUDA tensors; calls that
    overlap on the GPU race on the shared workspace.
    """
    import torch
    lib = load_library()
    cd = torch.complex128 if grid.dtype == RF_F64 else torch.complex64
    rd = torch.float64 if grid.dtype == RF_F64 else torch.float32
    x = _dev(x, rd, "x", grid.n)
    ip = _dev(inv_psd, torch.float64, "inv_psd", grid.n // 2 + 1)
    z_out = _out(z_out, cd, grid.n, "z_out")
    if sigma_out is not None:
        sigma_out = _out(sigma_out, torch.float64, 1, "sigma_out")
    sp = ctypes.c_void_p(sigma_out.data_ptr()) if sigma_out is not None else None
    _check(lib.rf_mf_reference_noalloc(ctypes.byref(grid), ctypes.c_void_p(x.data_ptr()),
                                       ctypes.c_void_p(ip.data_ptr()), _templates([ref]),
                                       ctypes.c_void_p(z_out.data_ptr()), sp, _stream(stream)))


__all__ = ["mf_reference_noalloc", "rf_grid", "rf_tune_entry", "RatioFilter", "Kernels", "RFError", "load_library", "launch_count", "EXPORTED", "LIB_PATH"]
