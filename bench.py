#!/usr/bin/env python3
"""Throughput of the ratio-filter hot path on one GB300 (template*samples/s).

One step = the whole online path for one data segment.  The default workload is the
long-duration batched configuration (fs 2048 Hz, f_low 5 Hz, 4096 s, n = 2^23, 128
references x 128 TaylorF2 3.5PN neighbours, kernels up to 3e5 taps on per-neighbour
build grids, autotuned overlap-save buckets, one persistent launch per bucket, the
whole step replayed from one CUDA graph); `--config 1..4` select the others:
    mf_filtered (data FFT, reference matched filters)   ->  z_ref of every reference
    winmax of z_ref                                      ->  reference peaks
    reconstruct (batched, all neighbours, fused peaks)   ->  neighbour peaks
Units per step: (G + sum K_g) * n template-samples.  Kernel building is offline
(its time is reported as `build_s`, outside the metric), and so is the stored
reference filter conj(h~_ref) / S_n / N_ref of each reference, which depends on
the template and the PSD only (`--mf onthefly` regenerates it in every step).

Also measured in the same run: the plain method (per-template full-length matched
filtering) on the same GPU in three arms, and the SNR error of our peaks against it;
the roofline of the dominant kernel; the e2e number through the public API with host
buffers; the FP64 oracle on the host cores (`cpu_baseline`).  `--impl reference`
times only the oracle.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workload  # noqa: E402

L2_BYTES = 129 * 1024 * 1024
GATE_THRESHOLD = 3e-5
FP32_LANES_PER_SM = 128
TF32_PER_BF16 = 1.1 / 2.25   # nominal dense TF32 : BF16 tensor rates of the part


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", type=int, default=5)
    ap.add_argument("--algo", default="auto", choices=["auto", "direct", "os", "gemm"])
    ap.add_argument("--prec", default=None, choices=["native", "bf16", "bf16x3", "bf16x6", "bf16x9", "3xtf32"],
                    help="arithmetic of the reconstruction (default: native; bf16x6 for --algo gemm)")
    ap.add_argument("--threshold", type=float, default=None)
    ap.add_argument("--bank", type=int, default=0,
                    help="reference groups from a structured synthetic bank of this many 1-3 Msun templates "
                         "(Sec. III.A: 10 s duration spread, at most 500 per set) on the batched workload's grid")
    ap.add_argument("--analytic", action="store_true",
                    help="truncate the kernels with the App. A expressions instead of their magnitudes")
    ap.add_argument("--stream", type=int, default=0,
                    help="also stream this many segment hops of data through rf_stream_winmax (guard from the "
                         "longest template and kernel extent) and report its rate under 'stream'")
    ap.add_argument("--real", action="store_true",
                    help="the paper's real-kernel form (taps 2 Re rho) instead of the complex one-sided kernel")
    ap.add_argument("--absolute", action="store_true",
                    help="absolute threshold (on |rho|; with --analytic a threshold amplitude on |r| in 1/s)")
    ap.add_argument("--block", type=int, default=0, help="overlap-save block size (0: library default)")
    ap.add_argument("--n-build", type=int, default=None,
                    help="kernel build grid: 0 the data grid, -1 per neighbour, or a power of two "
                         "(default: -1 for the 2^23-sample workload, else 0)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="skip the autotuner (with --algo auto: the cost-model overlap-save layout)")
    ap.add_argument("--mf", default="filtered", choices=["filtered", "onthefly"],
                    help="reference matched filter from stored filters, or template regenerated every step")
    ap.add_argument("--buckets", default="",
                    help="layout per kernel-length bucket, 'cut:block:part[:form],...' (first cut 0; form os "
                         "(default) or os_bins, the two-phase overlap-save); skips the autotuner")
    ap.add_argument("--part", type=int, default=0,
                    help="overlap-save partition length: block/2, /4 or /8 (0: library default)")
    ap.add_argument("--no-baseline", action="store_true", help="skip the cuFFT plain-method arm")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle cpu_baseline leg")
    ap.add_argument("--kernels", type=int, default=None, help="neighbours per group (default: the config's)")
    ap.add_argument("--groups", type=int, default=0,
                    help="keep only the first N reference groups (small cases for profiling; 0: all)")
    ap.add_argument("--no-graph", action="store_true", help="launch the step eagerly instead of one CUDA graph")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# --------------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"rf_bench_clocks_{os.getpid()}.csv")

    def __enter__(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        try:
            rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
        except Exception:
            return out
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                for nm, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
            except Exception:
                continue
        if sm:
            out.update(sm_mhz=statistics.median(sm), sm_max_mhz=max(mx), reasons=sorted(reasons), samples=len(sm))
        return out


# --------------------------------------------------------------------------- data

def make_strain_gpu(rf, cfg, torch, dev):
    """Noise (seeded draws) plus injections built with the library's own templates."""
    n, fs = cfg.n, cfg.fs
    xf = torch.tensor(workload.noise_spectrum(cfg), dtype=torch.complex128, device=dev)
    ip = torch.tensor(workload.inv_psd(cfg), dtype=torch.float64, device=dev)
    f = torch.arange(n // 2 + 1, dtype=torch.float64, device=dev) * (fs / n)
    band = ((f >= cfg.f_low) & (f <= cfg.f_high)).to(torch.float64)
    rf64 = None
    for inj in cfg.injections:
        ref, nb = cfg.groups[inj.group]
        t = ref if inj.template_index < 0 else nb[inj.template_index]
        tt = workload.Template(t.m1, t.m2, tc=inj.sample / fs)
        h = rf.template_fd(tt).to(torch.complex128)
        sig = torch.sqrt(4.0 * (fs / n) * torch.sum(h.abs() ** 2 * ip * band))
        xf = xf + (inj.snr / sig) * h * band
    x = torch.fft.irfft(xf, n) * fs
    return x.to(rf.rdtype).contiguous(), ip


# --------------------------------------------------------------------------- plain method (cuFFT)

def cufft_matched_filter_peaks(x, ip, templates_fd, cfg, torch, chunk=16):
    """Per-template full-length matched filter with cuFFT (the plain method) -> window peaks."""
    n, fs, W = cfg.n, cfg.fs, cfg.window
    nw = -(-n // W)
    xf = torch.fft.rfft(x.to(torch.float32)) / fs
    f = torch.arange(n // 2 + 1, device=x.device, dtype=torch.float64) * (fs / n)
    band = (f >= cfg.f_low) & (f <= cfg.f_high)
    ipb = torch.where(band, ip, torch.zeros_like(ip))
    sig = torch.sqrt(4.0 * (fs / n) * torch.sum(templates_fd[0].abs().double() ** 2 * ipb)).item()
    w = (4.0 * (fs / n) / sig * ipb).to(torch.float32)
    P = torch.empty((len(templates_fd), nw), dtype=torch.float32, device=x.device)
    A = torch.empty((len(templates_fd), nw), dtype=torch.int64, device=x.device)
    spec = torch.zeros((chunk, n), dtype=torch.complex64, device=x.device)
    for j0 in range(0, len(templates_fd), chunk):
        hs = templates_fd[j0:j0 + chunk]
        m = len(hs)
        spec[:m, : n // 2 + 1] = xf[None, :] * torch.conj(hs) * w[None, :]
        z = torch.fft.ifft(spec[:m]) * n
        mag = (z.real ** 2 + z.imag ** 2)
        pad = nw * W - n
        if pad:
            mag = torch.nn.functional.pad(mag, (0, pad), value=-1.0)
        mw = mag.view(m, nw, W)
        P[j0:j0 + m], a = mw.max(dim=2)
        A[j0:j0 + m] = a + torch.arange(nw, device=x.device)[None, :] * W
    return P, A


# --------------------------------------------------------------------------- oracle on the host

class OracleSample:
    """The FP64 oracle as it stands, on a bounded sample of the workload.

    Set-up (untimed, like the method's offline phase): the strain and the kernels of
    `n_nbrs` neighbours of the first reference, chosen at quantiles of their duration offset
    (which sets the kernel length, Sec. II.B), on the same build grid as the GPU arm.
    Timed once: the reference matched filter over the whole segment (data FFT, template,
    inverse FFT; Eqs. 2-3).  Timed per step: the direct reconstruction (Eq. 8) of those
    neighbours at `slice_len` output samples.  `value()` scales both to the step's units:
    G reference filters and sum_j L_j n multiply-adds of the neighbours, the latter by the
    workload's total taps over the sample's."""

    def __init__(self, cfg, n_nbrs: int, slice_len: int, n_build: int, thr: float, total_taps: float = None):
        from oracle import data as odata, mf as omf, ratio as oratio
        self.cfg = cfg
        ref, nb = cfg.groups[0]
        ip = workload.inv_psd(cfg)
        x = odata.strain(cfg)
        t0 = time.perf_counter()
        self.z_ref, _ = omf.matched_filter(x, ip, cfg.n, cfg.fs, cfg.f_low, cfg.f_high, ref.m1, ref.m2,
                                           cfg.pn_order)
        self.t_mf = time.perf_counter() - t0
        tau_ref = workload.newtonian_duration(ref, cfg.f_low)
        off = np.array([abs(workload.newtonian_duration(t, cfg.f_low) - tau_ref) for t in nb])
        order = np.argsort(off)
        sel = sorted({int(order[min(len(nb) - 1, int((q + 0.5) * len(nb) / n_nbrs))]) for q in range(n_nbrs)})
        self.pk = oratio.build_ratio_kernels(ref, [nb[j] for j in sel], cfg.n, cfg.fs, cfg.f_low, cfg.f_high,
                                             cfg.pn_order, ip, thr, n_build=n_build)
        self.idx = np.arange(slice_len, dtype=np.int64) * (cfg.n // slice_len)
        self.sample_taps = float(np.sum(self.pk.length))
        rows = sum(len(g[1]) for g in cfg.groups)
        # the workload's taps: the GPU arm's kernels when given, else the sample's mean length
        self.total_taps = float(total_taps) if total_taps else self.sample_taps / len(sel) * rows
        self.n_sel = len(sel)
        self.rows = rows

    def step(self) -> float:
        from oracle import reconstruct as orec
        t1 = time.perf_counter()
        for j in range(self.n_sel):
            orec.reconstruct_at(self.z_ref, *self.pk.kernel(j), self.idx)
        return time.perf_counter() - t1

    def value(self, t_rec: float) -> float:
        cfg = self.cfg
        G = len(cfg.groups)
        units = (G + self.rows) * cfg.n
        # reconstruction time per tap-output from the sample, times the workload's tap-outputs
        per_tap_out = t_rec / (self.sample_taps * len(self.idx))
        total = G * self.t_mf + per_tap_out * self.total_taps * cfg.n
        return units / total

    def describe(self, t_rec: float) -> str:
        return (f"reference MF over n={self.cfg.n} ({self.t_mf:.2f}s, timed once) + direct reconstruction of "
                f"{self.n_sel} neighbours (mean L={self.sample_taps / self.n_sel:.0f}) at {len(self.idx)} output "
                f"samples ({t_rec:.2f}s per step); scaled to {len(self.cfg.groups)} reference MFs and "
                f"{self.total_taps:.4g} taps x n; numpy single-threaded on {os.cpu_count()} host cores")


def cpu_baseline(cfg, n_build: int, thr: float, total_taps: float):
    """The oracle leg of the GPU arm's line (one timed step of OracleSample)."""
    o = OracleSample(cfg, n_nbrs=4, slice_len=1 << 11, n_build=n_build, thr=thr, total_taps=total_taps)
    t = o.step()
    return {"value": o.value(t), "unit": "template*samples/s", "cores": 1, "kind": "oracle", "sample": o.describe(t)}


def scipy_baseline(cfg, x, filt_row, kern, n_nbrs=8, budget_s=20.0):
    """The paper's own CPU route on the host cores (Sec. III: scipy FFTs and
    scipy.signal.oaconvolve, complex128): the reference matched filter with scipy.fft (the
    reference filter as stored, so template generation is not timed), then the time-domain
    convolution (Eq. 8, circular) of z_ref with a sample of the truncated kernels chosen at
    quantiles of their length; scaled to the step's units."""
    import scipy.fft as sfft
    import scipy.signal as ssig
    cores = os.cpu_count() or 1
    n = cfg.n
    xh = np.asarray(x, dtype=np.float64)
    fh = np.asarray(filt_row, dtype=np.complex128)
    t0 = time.perf_counter()
    X = sfft.rfft(xh, workers=cores)
    spec = np.zeros(n, dtype=np.complex128)
    spec[: n // 2 + 1] = X * fh
    z = sfft.ifft(spec, workers=cores) * n
    t_mf = time.perf_counter() - t0
    L = kern.length
    order = np.argsort(L)
    sel = sorted({int(order[min(len(L) - 1, int((q + 0.5) * len(L) / n_nbrs))]) for q in range(n_nbrs)})
    taps = kern.taps().cpu().numpy().astype(np.complex128)
    t1 = time.perf_counter()
    done = 0
    for j in sel:
        c = taps[kern.offset[j]:kern.offset[j + 1]]
        m0 = int(kern.lag0[j])
        # circular form: z_j[i] = sum_l c[l] z[(i - m0 - l) mod n], from a wrapped copy of z
        ext = np.concatenate([z[(np.arange(-(len(c) - 1), 0) - m0) % n], np.roll(z, m0)])
        ssig.oaconvolve(ext, c, mode="valid")
        done += 1
        if time.perf_counter() - t1 > budget_s:
            break
    t_rec = time.perf_counter() - t1
    K = len(L)
    units = (1 + K) * n
    per_nbr = t_rec / max(done, 1) * (float(np.mean(L)) / float(np.mean(L[sel[:done]])))
    return {"value": units / (t_mf + per_nbr * K), "unit": "template*samples/s", "cores": cores,
            "kind": "scipy.fft matched filter + scipy.signal.oaconvolve (complex128), the paper's CPU route",
            "sample": (f"reference MF {t_mf:.2f}s; {done} neighbours convolved in {t_rec:.2f}s, scaled by the "
                       f"mean kernel length to {K} neighbours")}


# --------------------------------------------------------------------------- ncu traffic

def ncu_traffic(kernel: str, layout: str = None):
    """DRAM bytes per launch of `kernel` from the committed ncu capture, or None when the
    kernel's sources (or its layout) changed since that capture, or no capture exists."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        recs = json.load(open(path))
        rec = recs.get(f"{kernel}@{layout}", recs[kernel])
        if layout is not None and rec.get("layout") != layout:
            return None
        m = hashlib.sha256()
        for f in rec["sources"]:
            m.update(open(os.path.join(ROOT, "paper_2511_12894_gb300", "csrc", f), "rb").read())
        return rec["traffic_bytes_per_launch"] if m.hexdigest() == rec["sha256"] else None
    except Exception:
        return None


def stream_rate(rf, cfg, x, filt, kerns, W: int, hops: int) -> dict:
    """Data longer than one segment through rf_stream_winmax: guard = the longest template's
    duration from f_low plus the largest kernel lag extent, in whole windows; the strain is the
    segment's host copy repeated over `hops` segment hops (a rate measurement, host buffers in
    and out, the per-segment copies included)."""
    tau = max(workload.newtonian_duration(t, cfg.f_low) for r, nb in cfg.groups for t in (r,) + tuple(nb))
    ext = max(int(np.max(np.maximum(np.abs(k.lag0), np.abs(k.lag0 + k.length)))) for k in kerns if k.k)
    guard = int(math.ceil((1.05 * tau * cfg.fs + ext) / W)) * W
    if 2 * guard >= cfg.n:
        return {"unavailable": f"guard {guard} samples does not fit a segment of {cfg.n}"}
    hop = cfg.n - 2 * guard
    total = hops * hop // W * W
    xh = np.resize(x.detach().cpu().numpy(), total)
    rf.stream_winmax(xh[: cfg.n], filt, kerns, W, guard)          # warm-up: staging buffers, plans
    t0 = time.perf_counter()
    rf.stream_winmax(xh, filt, kerns, W, guard)
    sec = time.perf_counter() - t0
    rows = sum(k.k for k in kerns)
    return {"value": (len(kerns) + rows) * total / sec, "unit": "template*samples/s", "seconds": sec,
            "data_s": total / cfg.fs, "segments": -(-total // hop), "guard_s": guard / cfg.fs,
            "hop_s": hop / cfg.fs, "what": "host strain -> per-segment matched filter, reference peaks and "
                                          "batched reconstruction -> host window peaks of the stream"}


def tune_groups(kerns, max_groups: int = 8):
    """Indices of at most `max_groups` reference groups spread over the batch's total kernel
    length per group (the quantiles of that distribution), for the autotuner."""
    G = len(kerns)
    if G <= max_groups:
        return list(range(G))
    tot = [int(np.sum(k.length)) for k in kerns]
    order = sorted(range(G), key=lambda g: (tot[g], g))
    return sorted({order[min(G - 1, int((q + 0.5) * G / max_groups))] for q in range(max_groups)})


def load_workload(args):
    """The configuration to run: one of the five workloads, or (--bank N) the batched
    workload's grid with the sets of a structured synthetic bank as its reference groups."""
    if not args.bank:
        cfg = workload.config(args.config, k_override=args.kernels)
        groups = getattr(args, "groups", 0)
        if groups and groups < len(cfg.groups):
            cfg = workload.with_groups(cfg, cfg.groups[:groups], cfg.name)
        return cfg
    from paper_2511_12894_gb300 import bank_structure
    base = workload.config(4)
    b = workload.synthetic_bank(args.bank, seed=2025)
    sets, refs, _ = bank_structure(b, base.f_low, base.pn_order, 10.0, 500)
    groups = [(b[r], tuple(b[i] for i in s if i != r)) for s, r in zip(sets, refs)]
    return workload.with_groups(base, groups, f"structured-bank-{args.bank}")


def workload_label(cfg, config: int, thr: float, trunc: str = "rel") -> str:
    """The workload name both arms print in config.workload."""
    G = len(cfg.groups)
    rows = sum(len(nb) for _, nb in cfg.groups)
    return (f"cfg{config}: {cfg.name}; n=2^{int(math.log2(cfg.n))} fs={cfg.fs:g} f_low={cfg.f_low:g}; "
            f"{G} ref + {rows} TaylorF2 nbrs; thr={thr:g} {trunc}; W={cfg.window}")


# --------------------------------------------------------------------------- main

def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return
    cfg = workload.config(args.config)
    thr = args.threshold if args.threshold is not None else GATE_THRESHOLD
    n_build = args.n_build if args.n_build is not None else (-1 if cfg.n > (1 << 20) else 0)
    o = OracleSample(cfg, n_nbrs=2, slice_len=1 << 10, n_build=n_build, thr=thr)
    vals, t = [], 0.0
    for s in range(args.warmup + args.steps):
        t = o.step()
        if s >= args.warmup:
            vals.append(o.value(t))
    v = statistics.median(vals) if vals else o.value(t)
    cb = {"value": v, "unit": "template*samples/s", "cores": 1, "kind": "oracle", "sample": o.describe(t)}
    line = {"impl": "reference", "metric": "template*samples/s", "value": v, "unit": "template*samples/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_label(cfg, args.config, thr), "parallelism": "host"},
            "cpu_baseline": cb,
            "e2e": {"value": v, "unit": "template*samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2511_12894_gb300 import RatioFilter, build, launch_count
    build.build()

    cfg = load_workload(args)
    # multi-reference workloads are sharded by whole groups across ranks, a single group by its
    # neighbours (every rank filtering the one reference); every rank builds the same strain
    # from the same seed, and the only exchange is the final gather of the window peaks
    from paper_2511_12894_gb300 import shard
    from dataclasses import replace as _replace
    all_groups = cfg.groups
    sharded = world > 1
    nb_sizes = [len(nb) for _, nb in all_groups]
    if sharded and len(all_groups) > 1:
        def est_lengths(ref, nb):
            t0 = workload.newtonian_duration(ref, cfg.f_low)
            return [max(512.0, abs(workload.newtonian_duration(t, cfg.f_low) - t0) * cfg.fs) for t in nb]
        costs = [shard.group_cost(cfg.n, est_lengths(r, nb)) for r, nb in all_groups]
        assign = shard.assign(costs, world)
        mine = assign[rank]
        cfg = _replace(cfg, groups=tuple(all_groups[g] for g in mine))
        ref_rows = [list(a) for a in assign]
        nb_rows = [shard.global_rows(nb_sizes, a) for a in assign]
        shard_mode = f"groups sharded over {world} ranks"
    elif sharded:
        ref0, nb0 = all_groups[0]
        runs = [shard.split_neighbours(len(nb0), world, r) for r in range(world)]
        cfg = _replace(cfg, groups=((ref0, tuple(nb0[j] for j in runs[rank])),))
        ref_rows = [[0]] + [[] for _ in range(world - 1)]   # rank 0 reports the reference
        nb_rows = [list(r) for r in runs]
        shard_mode = f"neighbours split over {world} ranks"
    else:
        shard_mode = "one GPU"
    units_total = sum(1 + len(nb) for _, nb in all_groups) * cfg.n
    full_cfg = load_workload(args)   # the whole workload, for its label
    # relative truncation threshold: the largest of 1e-3, 1e-4, 3e-5 whose window peaks stay
    # within 1e-4 of the loudest SNR against full matched filtering on this workload
    thr = args.threshold if args.threshold is not None else GATE_THRESHOLD
    refs = [g[0] for g in cfg.groups]
    G = len(refs)
    n, W = cfg.n, cfg.window
    rf = RatioFilter.from_config(cfg)
    x, ip = make_strain_gpu(rf, cfg, torch, dev)

    # ---------------- offline: ratio kernels (and their overlap-save spectra)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    n_build = args.n_build if args.n_build is not None else (-1 if cfg.n > (1 << 20) else 0)
    kerns = [rf.build_ratio_kernels(r, nb, ip, thr, relative=not args.absolute, n_build=n_build,
                                    analytic=args.analytic, real=args.real) for r, nb in cfg.groups]
    filt, sig = rf.reference_filters(ip, refs)
    tune, tune_s, tune_info, tuned_call = None, 0.0, None, None
    if args.buckets:
        spec = [b.split(":") for b in args.buckets.split(",")]
        for k in kerns:
            k.prepare_forms([int(b[0]) for b in spec], [b[3] if len(b) > 3 else "os" for b in spec],
                            ["native"] * len(spec), [int(b[1]) for b in spec], [int(b[2]) for b in spec])
        algo_used = "os"
    elif args.algo == "auto" and not args.no_autotune and args.block == 0 and args.part == 0:
        # the autotuner times candidate forms on a z_ref of this segment (offline, like the
        # kernels), on at most 8 groups spread over the batch's per-group kernel lengths; the
        # winning form and layout then apply to every group
        t1 = time.perf_counter()
        pick = tune_groups(kerns)
        zt = rf.mf_filtered(x, filt[pick] if len(pick) < G else filt)
        tune = rf.autotune([zt[q] for q in range(len(pick))], [kerns[g] for g in pick], W,
                           allow_split=cfg.dtype == "f32")
        del zt
        w = tune[0]
        bucketed = bool(w["cut"]) or w["algo"] in ("os", "os_bins")
        if len(pick) < G:
            if bucketed:
                if w["cut3"]:
                    forms = ([0, w["cut"], w["cut3"]], [w["algo"], w["algo2"], w["algo3"]],
                             [w["prec"], "native", "native"], [w["block"], w["block2"], w["block3"]],
                             [w["part"], w["part2"], w["part3"]])
                elif w["cut"]:
                    forms = ([0, w["cut"]], [w["algo"], w["algo2"]], [w["prec"], "native"], [w["block"], w["block2"]],
                             [w["part"], w["part2"]])
                else:
                    forms = ([0], [w["algo"]], [w["prec"]], [w["block"]], [w["part"]])
                for k in kerns:
                    k.prepare_forms(*forms)
            # groups outside the tuned subset resolve AUTO by default; name the form instead
            tuned_call = ("os", "native") if bucketed else (w["algo"], w["prec"])
        torch.cuda.synchronize()
        tune_s = time.perf_counter() - t1
        algo_used = "os" if bucketed else w["algo"]
        tune_info = {"groups_timed": len(pick), "of": G}
    else:
        algo_used = args.algo if args.algo != "auto" else ("os" if cfg.dtype == "f32" else "direct")
        if algo_used == "os":
            for k in kerns:
                k.prepare(args.block, args.part)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    L = np.concatenate([k.length for k in kerns]).astype(np.float64)
    rows = int(L.size)
    buckets = kerns[0].os_buckets() if algo_used == "os" else []   # [(cut, B, Lp), ...]
    forms = kerns[0].bucket_forms() if algo_used == "os" else []    # [(algo, prec), ...]
    layout = ",".join((f"{a}:" if a != "os" else "") + f"B={b},Lp={p}" + (f"@{c}" if c else "")
                      for (c, b, p), (a, _) in zip(buckets, forms))

    nw = -(-n // W)
    z = torch.empty((G, n), dtype=rf.cdtype, device=dev)
    Pn = torch.empty((rows, nw), dtype=torch.float32, device=dev)
    An = torch.empty((rows, nw), dtype=torch.int32, device=dev)
    Pr = torch.empty((G, nw), dtype=torch.float32, device=dev)
    Ar = torch.empty((G, nw), dtype=torch.int32, device=dev)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    if algo_used == "os":
        rf.reserve(rows)

    call_prec = args.prec or ("bf16x6" if args.algo == "gemm" else "native")
    call_algo = args.algo
    if tuned_call is not None:
        call_algo, call_prec = tuned_call
    prec = tune[0]["prec"] if tune else call_prec   # the precision the reconstruction runs at

    def recon():
        if G == 1:
            rf.reconstruct_winmax(z[0], kerns[0], W, call_algo, max_out=Pn, arg_out=An, prec=call_prec)
        else:
            rf.reconstruct_batched([z[g] for g in range(G)], kerns, W, call_algo, max_out=Pn, arg_out=An,
                                      prec=call_prec)

    def mf_step(xs):
        if args.mf == "filtered":
            rf.mf_filtered(xs, filt, z_out=z)
        else:
            rf.mf_reference(xs, ip, refs, z_out=z, sigma_out=sig)

    def step():
        mf_step(x)
        rf.winmax(z, W, max_out=Pr, arg_out=Ar)
        recon()

    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        for _ in range(args.warmup):
            step()
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    lc0 = launch_count()
    step()
    torch.cuda.synchronize()
    launches_per_step = launch_count() - lc0
    graph = None
    if not args.no_graph:
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            step()
        graph.replay()
        torch.cuda.synchronize()
    stream = torch.cuda.current_stream()

    # ---------------- timed region: K steps, L2 flushed between steps (outside the events)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for s in range(args.steps):
            flush.zero_()
            starts[s].record(stream)
            if graph is not None:
                graph.replay()
            else:
                step()
            ends[s].record(stream)
        torch.cuda.synchronize()
    step_ms = [a.elapsed_time(b) for a, b in zip(starts, ends)]
    total_ms = sum(step_ms)
    if world > 1:
        t = torch.tensor([total_ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = t.item()
    ms_per_step = total_ms / args.steps
    units_step = (G + rows) * n
    value = units_total * args.steps / (total_ms / 1e3)
    gathered = None
    if world > 1:
        # the one exchange: every rank's window peaks to rank 0, in the single-process row order
        import torch.distributed as dist
        nr = len(ref_rows[rank])
        total_nb = sum(nb_sizes)
        outs = [shard.gather_rows(t, rows_, tot, rank, world, dist)
                for t, rows_, tot in ((Pr[:nr], ref_rows, len(all_groups)), (Ar[:nr], ref_rows, len(all_groups)),
                                      (Pn, nb_rows, total_nb), (An, nb_rows, total_nb))]
        if rank == 0:
            gathered = {"reference_rows": int(outs[0].shape[0]), "neighbour_rows": int(outs[2].shape[0]),
                        "windows": int(outs[0].shape[1]), "how": "torch.distributed.gather to rank 0, "
                                                                 "after the timed region"}

    # ---------------- the dominant kernel alone (events on its stream), for the roofline: the
    # reconstruction's launches replayed from a graph of their own, so that the host work of an
    # eager call (argument checks, launch set-up) does not show as device time
    rec_graph = None
    if graph is not None:
        rec_graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(rec_graph):
            recon()
        rec_graph.replay()
        torch.cuda.synchronize()
    rec_ms = []
    for _ in range(max(3, args.steps // 2)):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        if rec_graph is not None:
            rec_graph.replay()
        else:
            recon()
        b.record(stream)
        b.synchronize()
        rec_ms.append(a.elapsed_time(b))
    rec_avg_ms = statistics.mean(rec_ms)

    # ---------------- the reference matched filter alone (its own graph), against HBM: per
    # step the data (one real segment) in, and per reference its stored filter (n/2 + 1
    # complex values) in and its series z_ref (n complex values) out
    mf_graph = None
    if graph is not None:
        mf_graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(mf_graph):
            mf_step(x)
        mf_graph.replay()
        torch.cuda.synchronize()
    mf_ms = []
    for _ in range(max(3, args.steps // 2)):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        if mf_graph is not None:
            mf_graph.replay()
        else:
            mf_step(x)
        b.record(stream)
        b.synchronize()
        mf_ms.append(a.elapsed_time(b))
    mf_avg_ms = statistics.mean(mf_ms)
    esz = 8 if cfg.dtype == "f32" else 16
    mf_bytes = esz / 2 * n + G * (esz * (n // 2 + 1) + esz * n) if args.mf == "filtered" else esz / 2 * n + G * esz * n
    hbm_peak = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("hbm_gbs", 6800.0)) \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else 6800.0
    mf_info = {"references": G, "kernel_ms": mf_avg_ms, "us_per_reference": mf_avg_ms * 1e3 / G,
               "alg_bytes": mf_bytes, "achieved_gbs": mf_bytes / (mf_avg_ms / 1e3) / 1e9,
               "frac_of_hbm": mf_bytes / (mf_avg_ms / 1e3) / 1e9 / hbm_peak,
               "transform": ("four-step, two passes" if cfg.dtype == "f32" and (1 << 18) <= n <= (1 << 24)
                             else "radix-16 passes"),
               "bytes_note": "data in once; per reference its filter in and z_ref out (the minimum)"
                             if args.mf == "filtered" else "data in once; per reference z_ref out"}

    # ---------------- e2e through the public API with host buffers
    x_host = torch.empty(n, dtype=rf.rdtype, pin_memory=True)
    x_host.copy_(x.cpu())
    P_host = torch.empty((G + rows, nw), dtype=torch.float32, pin_memory=True)
    A_host = torch.empty((G + rows, nw), dtype=torch.int32, pin_memory=True)
    x_dev = torch.empty_like(x)
    e_ms = []
    for s in range(args.warmup + max(3, args.steps // 2)):
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        x_dev.copy_(x_host, non_blocking=True)
        mf_step(x_dev)
        rf.winmax(z, W, max_out=Pr, arg_out=Ar)
        recon()
        P_host[:G].copy_(Pr, non_blocking=True)
        A_host[:G].copy_(Ar, non_blocking=True)
        P_host[G:].copy_(Pn, non_blocking=True)
        A_host[G:].copy_(An, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        if s >= args.warmup:
            e_ms.append(e0.elapsed_time(e1))
    e2e_ms = statistics.mean(e_ms)
    e2e = {"value": units_total / (e2e_ms / 1e3), "unit": "template*samples/s",
           "h2d_bytes_per_step": int(x_host.numel() * x_host.element_size()),
           "d2h_bytes_per_step": int(P_host.numel() * 4 + A_host.numel() * 4), "ms_per_step": e2e_ms,
           "path": f"pinned host x -> mf_{args.mf} -> winmax -> reconstruct (eager calls) -> pinned host peaks"}

    # ---------------- roofline of the dominant kernel (the neighbour reconstruction)
    if algo_used == "os":
        # per output block of H = B - Lp samples: one inverse B-point FFT (5 B log2 B) and
        # P_j = ceil(L_j / Lp) complex multiply-adds per bin (8 P_j B); the segment spectra
        # are shared by all neighbours of a reference
        cuts = np.array([c for c, _, _ in buckets])
        bi = np.searchsorted(cuts, L, side="right") - 1          # bucket of each kernel
        Bj = np.array([b for _, b, _ in buckets], dtype=np.float64)[bi]
        Lpj = np.array([p for _, _, p in buckets], dtype=np.float64)[bi]
        P = np.maximum(1, np.ceil(L / Lpj))
        flops = float(np.sum((5.0 * Bj * np.log2(Bj) + 8.0 * P * Bj) / (Bj - Lpj))) * n
    else:
        flops = 8.0 * float(L.sum()) * n
    props = torch.cuda.get_device_properties(dev)
    sm_max = 2070.0
    if algo_used == "gemm":
        # tensor-pipe work actually issued, from the layout the library chose: per super-tile of
        # S x 128 outputs and group of NJ neighbours, KC x NCK taps (LP + 128 (S - 1)) x 2 planes
        # x products, each 2 x 128 x (S x 2 NJ) flops per tap
        nprod = {"bf16": 1, "bf16x3": 3, "bf16x6": 6, "bf16x9": 9, "3xtf32": 3}[prec]
        mma_flops = 0.0
        for k in kerns:
            lay = k.gemm_layout()
            S, NJ = lay["shifts"], lay["nj"]
            groups = -(-k.k // NJ)
            mma_flops += (-(-n // (128 * S))) * groups * (lay["kc"] * lay["nck"]) * 2 * nprod * (2 * 128 * S * 2 * NJ)
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
            os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
        peak_tflops = float(peaks.get("bf16_tflops", 1900.0))
        if prec == "3xtf32":
            peak_tflops *= TF32_PER_BF16   # the TF32 pipe's own peak: measured BF16 x nominal ratio
        achieved = mma_flops / (rec_avg_ms / 1e3) / 1e12
        roofline = {"bound": "tensor", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                    "frac": achieved / peak_tflops, "traffic": ncu_traffic("k_gemm", prec) if args.config == 3 else None,
                    "kernel": f"reconstruct (tcgen05 Hankel GEMM, {prec}, one reference)",
                    "peak_note": ("measured cuBLAS bf16 burst (MEASURED_PEAKS.json)" if peaks else "fallback 1.9 PF/s") +
                                 (" x 1.1/2.25 nominal TF32:BF16" if prec == "3xtf32" else "") +
                                 "; achieved counts the MMA flops issued (split terms included)",
                    "algorithmic_tflops": flops / (rec_avg_ms / 1e3) / 1e12,
                    # the method's own work (8 L flops per template-sample) against what the pipe can
                    # deliver for it: the peak divided by the split products each flop needs
                    "algorithmic_frac": (flops / (rec_avg_ms / 1e3) / 1e12) / (peak_tflops / nprod),
                    "kernel_ms": rec_avg_ms, "share_of_step": rec_avg_ms / ms_per_step}
    else:
        peak_tflops = props.multi_processor_count * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
        achieved = flops / (rec_avg_ms / 1e3) / 1e12
        roofline = {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
                    "frac": achieved / peak_tflops,
                    # DRAM bytes of one reconstruction call from the committed capture of this
                    # workload and layout (null when the sources or the layout changed since)
                    "traffic": (ncu_traffic(f"reconstruct_cfg{args.config}", layout)
                                if (algo_used == "os" and not args.groups and not args.kernels and not args.bank
                                    and not args.real and not args.analytic and not args.absolute
                                    and args.threshold is None) else None),
                    "kernel": f"reconstruct ({algo_used}{', ' + layout if algo_used == 'os' else ''}, "
                              f"{'FP64' if cfg.dtype == 'f64' and algo_used == 'direct' else 'FP32'} CUDA cores, "
                              f"{'batched persistent' if G > 1 else 'one reference'})",
                    "peak_note": f"{props.multi_processor_count} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x {sm_max:.0f} MHz",
                    "kernel_ms": rec_avg_ms, "share_of_step": rec_avg_ms / ms_per_step}

    # ---------------- plain method on the same GPU, and the SNR error against it
    baseline = None
    err = None
    if not args.no_baseline:
        # the largest group's reference and up to 256 of its neighbours (the first group for
        # a single-group workload)
        gs = max(range(G), key=lambda g: (len(cfg.groups[g][1]), -g))
        row0 = sum(len(nb) for _, nb in cfg.groups[:gs])
        sub = [(gs, refs[gs], -1)] + [(gs, t, j) for j, t in enumerate(cfg.groups[gs][1])]
        sub = sub[:257]
        tmpl = [t for _, t, _ in sub]
        hs = torch.stack([rf.template_fd(t) for t in tmpl]).to(torch.complex64)

        def timed(fn, reps=3):
            fn()
            fn()
            torch.cuda.synchronize()
            ms, out = [], None
            for _ in range(reps):
                flush.zero_()
                torch.cuda.synchronize()
                b0 = torch.cuda.Event(enable_timing=True)
                b1 = torch.cuda.Event(enable_timing=True)
                b0.record(stream)
                out = fn()
                b1.record(stream)
                b1.synchronize()
                ms.append(b0.elapsed_time(b1))
            return statistics.median(ms), out

        # the minimum a stored-filter matched filter moves per template: its filter (n/2 + 1
        # complex64 values) in, its window peaks (8 B per window) out
        alg_bytes = 8.0 * (n // 2 + 1) + 8.0 * nw

        def arm(ms_sub, what):
            per_t = ms_sub / len(sub)
            return {"value": units_step / (per_t * (G + rows) / 1e3), "unit": "template*samples/s",
                    "ms_per_step": per_t * (G + rows), "us_per_template": per_t * 1e3,
                    "achieved_gbs": alg_bytes / (per_t / 1e3) / 1e9, "what": what}

        arms = {}
        t_cu, (Pf, Af) = timed(lambda: cufft_matched_filter_peaks(x, ip, hs, cfg, torch))
        arms["torch_cufft"] = arm(t_cu, "torch: product kernel, cuFFT C2C inverse (n), |z|^2 and window max as "
                                        "separate kernels, batched 16; stored template spectra")
        # the library's own fused path: stored per-template filters (the product formed inside the
        # first inverse-FFT pass), then the window peaks of the series
        filt_s, _ = rf.reference_filters(ip, tmpl)
        zs_s = torch.empty((len(sub), n), dtype=rf.cdtype, device=dev)
        Ps = torch.empty((len(sub), nw), dtype=torch.float32, device=dev)
        As = torch.empty((len(sub), nw), dtype=torch.int32, device=dev)
        t_lib, _ = timed(lambda: (rf.mf_filtered(x, filt_s, z_out=zs_s), rf.winmax(zs_s, W, max_out=Ps, arg_out=As)))
        arms["library_stored_filter"] = arm(t_lib, "rf_mf_filtered (data FFT, product in the first inverse pass) "
                                                   "+ rf_winmax; stored per-template filters")
        del filt_s
        # templates generated in every step (the paper's standard: generation + correlation)
        sig_s = torch.empty(len(sub), dtype=torch.float64, device=dev)
        t_otf, _ = timed(lambda: (rf.mf_reference(x, ip, tmpl, z_out=zs_s, sigma_out=sig_s),
                                  rf.winmax(zs_s, W, max_out=Ps, arg_out=As)))
        arms["library_on_the_fly"] = arm(t_otf, "rf_mf_reference (TaylorF2 template generated per step, FP64 "
                                                "phase) + rf_winmax: waveform generation + correlation")
        del zs_s
        fastest = max(arms, key=lambda a: arms[a]["value"])
        fits = 8.0 * (n // 2 + 1) * (G + rows) <= 0.8 * torch.cuda.get_device_properties(dev).total_memory
        # the stored-spectrum arms need every template's n/2 + 1 values in HBM; where they do not
        # fit, only the on-the-fly arm can run the whole bank from one GPU
        runnable = [a for a in arms if fits or a == "library_on_the_fly"]
        fastest_run = max(runnable, key=lambda a: arms[a]["value"])
        baseline = {**arms[fastest], "arm": fastest, "arms": arms, "templates_timed": len(sub),
                    "stored_filters_fit_in_hbm": bool(fits),
                    "speedup_vs_fastest": value / arms[fastest]["value"],
                    "fastest_whole_bank_arm": fastest_run,
                    "speedup_vs_fastest_whole_bank": value / arms[fastest_run]["value"]}
        ours_P = torch.cat([Pr[gs:gs + 1], Pn[row0:row0 + len(sub) - 1]]).double().sqrt()
        full_P = Pf.double().sqrt()
        err = {"peak_snr_max_abs_over_max": ((ours_P - full_P).abs().max() / full_P.max()).item()}
        jmax = int(torch.argmax(full_P.max(dim=1).values).item())
        wmax = int(torch.argmax(full_P[jmax]).item())
        err["loudest_peak_rel"] = (abs(ours_P[jmax, wmax] - full_P[jmax, wmax]) / full_P[jmax, wmax]).item()
        err["loudest_snr"] = full_P[jmax, wmax].item()
        err["templates"] = len(sub)

    cb = None
    sb = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cb = cpu_baseline(cfg, n_build, thr, float(L.sum()))
        if G == 1:
            try:
                sb = scipy_baseline(cfg, x.double().cpu().numpy(), filt[0].cpu().numpy(), kerns[0])
            except ImportError as e:   # scipy absent on the host
                sb = {"unavailable": str(e)}

    st = None
    if rank == 0 and args.stream > 0:
        st = stream_rate(rf, cfg, x, filt, kerns, W, args.stream)

    if rank == 0:
        line = {
            "metric": "template*samples/s", "value": value, "unit": "template*samples/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None,
            "dtype": "f32" if cfg.dtype == "f32" else "f64",
            "data": "synthetic",
            "config": {"workload": workload_label(full_cfg, full_cfg.index, thr,
                                                  ("abs" if args.absolute else "rel") +
                                                  (" analytic" if args.analytic else "") +
                                                  (" real-kernel" if args.real else "")),
                       "kernel_len": {"min": int(L.min()), "median": float(np.median(L)), "max": int(L.max()),
                                      "sum": int(L.sum())},
                       "l2": "flushed between steps (256 MB write outside the events)", "algo": algo_used, "mf": args.mf, "n_build": n_build,
                       "autotune": ({"seconds": tune_s, "timed": tune, **(tune_info or {})} if tune else None),
                       "prec": prec,
                       "graph": graph is not None,
                       "parallelism": shard_mode},
            "build_s": build_s, "gpu_launches": int(launches_per_step * args.steps),
            "roofline": roofline, "cpu_baseline": cb, "e2e": e2e, "matched_filter": mf_info, "plain_mf": baseline,
            "err_vs_full_mf": err,
            "scipy_oaconvolve": sb,
            "stream": st,
            "gathered": gathered,
            # what a search keeps per template between analyses (Sec. IV): the plain method a
            # template spectrum of n/2 + 1 complex values per neighbour, the ratio filter the
            # neighbour's truncated kernel (sum of the kernel lengths); the references' own
            # filters are common to both
            "storage": {"full_values": int(rows * (n // 2 + 1)), "ratio_kernel_values": int(L.sum()),
                        "ratio": float(rows * (n // 2 + 1) / max(1, int(L.sum())))},
            "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
