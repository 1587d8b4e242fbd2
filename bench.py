#!/usr/bin/env python
"""Throughput benchmark of the Fourier-domain light-pollution map.

One step = one call of the C-ABI map (row forward transform, column
transform with the PSF-spectrum product, row inverse transform and crop)
over a synthetic radiance map resident in HBM, with the PSF spectrum cached.
The L2 cache is flushed (256 MiB write) between timed steps, outside the
timed events.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
    python bench.py --impl reference ...   # the FP64 CPU oracle, host cores

Metric: output Mpix/s per PSF map = H * W * n_spectra * steps / time.
Multi-GPU (torchrun): every rank maps its own radiance map (independent
units, no data exchange); value = all ranks' pixels / max-over-ranks time.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "output Mpix/s per kernel map"
UNIT = "Mpix/s"
DEFAULT_WORKLOAD = "map4096_psf541"
FALLBACK_HBM_GBS = 6800.0
PASSES = ("p1_rows", "p2_cols", "p3_rows")
# the kernel headers; build.py contributes its generated-source templates
# and compiler flags (the rest of it is the compile driver)
KERNEL_SOURCES = ("paper_1907_02891_gb300/csrc/fft_core.cuh",
                  "paper_1907_02891_gb300/csrc/conv_kernels.cuh")
TUNED_PLANS = "paper_1907_02891_gb300/tuned_plans.json"
TC_SOURCES = ("paper_1907_02891_gb300/csrc/tc_kernels.cuh",)


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-cufft", action="store_true",
                    help="skip the torch.fft (cuFFT) comparator")
    ap.add_argument("--e2e-steps", type=int, default=100)
    ap.add_argument("--no-cpu-fft", action="store_true",
                    help="skip the host-core FFT comparator (scipy.fft, the paper's method on a CPU)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="target duration of the CPU-oracle sample")
    ap.add_argument("--prec", default="fp32", choices=["fp32", "split_bf16"],
                    help="column-pass precision: FP32 FFT stages, or the DFT stages as "
                         "split-BF16 (hi/lo) products on the tensor cores")
    ap.add_argument("--mode", default="map", choices=["map", "serve"],
                    help="map: the throughput line; serve: the request-scheduler run")
    ap.add_argument("--requests", type=int, default=2000)
    ap.add_argument("--load", type=float, default=0.7,
                    help="offered load as a fraction of the measured back-to-back capacity")
    ap.add_argument("--slots", type=int, default=4)
    ap.add_argument("--serve-log", default=None,
                    help="--mode serve: append one JSON line per request to this file")
    ap.add_argument("--forms", default="batched,split_bf16,same_pad,tiled,graph,serve",
                    help="forms measured beside the headline map (comma list; empty: none): "
                         "batched (8192^2, 16 PSFs), split_bf16 (16384^2, 801^2 PSF), "
                         "same_pad (4096^2 map in one tile at the SAME crop's padding), "
                         "tiled (17800 x 21000, 801^2 PSF, overlap-save tiles), "
                         "graph (loops of small maps as one CUDA-graph replay), "
                         "serve (Poisson requests at 130%% and at 70%% load)")
    ap.add_argument("--forms-serve-requests", type=int, default=2000)
    return ap.parse_args()


# ----------------------------------------------------------------------------
# byte model (algorithmic bytes per pass, complex64 intermediates)
# ----------------------------------------------------------------------------

def pass_bytes(H, W, ny, nx, n, s_k):
    nc = nx // 2 + 1
    t = 8 * H * nc
    return {
        "p1_rows": 4 * H * W + t,                          # read L, write T
        "p2_cols": t + n * (s_k * ny * nc + t),            # read T, K^, write U
        "p3_rows": n * (t + 4 * H * W),                    # read U, write B
    }


def max_over_ranks(x: float, device=None) -> float:
    """Largest value of x over the ranks of the default process group (the
    bench's timing rule: the job is as slow as its slowest rank)."""
    import torch
    import torch.distributed as td
    if not (td.is_available() and td.is_initialized()) or td.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    td.all_reduce(t, op=td.ReduceOp.MAX)
    return float(t.item())


def whole_job_mpix_s(px_per_rank_per_step: float, steps: int, world: int, max_ms: float) -> float:
    """Whole-job throughput: every rank maps its own map (weak scaling), so
    the job outputs world x the per-rank pixels in the slowest rank's time."""
    return px_per_rank_per_step * steps * world / (max_ms / 1e3) / 1e6


def kernel_source_sha(extra=(), lengths=()):
    """Fingerprint of the kernel sources and of the measured plans of the
    given FFT lengths (the plans of other lengths do not change them)."""
    from paper_1907_02891_gb300 import build as B
    h = hashlib.sha1()
    for p in KERNEL_SOURCES + tuple(extra):
        with open(os.path.join(ROOT, p), encoding="utf-8") as fh:
            for line in fh:  # whole-line comments and blank lines change no kernel
                t = line.strip()
                if t and not t.startswith(("//", "/*", "*")):
                    h.update(t.encode())
    for part in (B._SIZE_TU, B._REGISTRY_TU, " ".join(B.ARCH), " ".join(B.NVCC_FLAGS)):
        h.update(part.encode())
    try:
        with open(os.environ.get("LP_TUNE_CACHE") or os.path.join(ROOT, TUNED_PLANS)) as fh:
            tuned = json.load(fh)
    except (OSError, ValueError):
        tuned = {}
    for n in sorted(set(lengths)):
        e = tuned.get(str(n))
        if isinstance(e, dict):  # knobs only: notes and tuning metadata change no kernel
            e = {k: v for k, v in e.items() if k not in ("note", "tuned_on", "tuned_total_us", "tuned_map_us")}
        h.update(json.dumps(e, sort_keys=True).encode())
    return h.hexdigest()[:16]


def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as fh:
            v = float(json.load(fh)["hbm_gbs"])
        return v, "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def dram_traffic(kernel, workload, lengths):
    """ncu dram bytes per launch, if captured for the current kernel source
    (the tensor-core column pass, "p2_cols_tc", also fingerprints its own
    header)."""
    p = os.path.join(ROOT, "profiles", "dram_traffic.json")
    try:
        with open(p) as fh:
            rec = json.load(fh)[workload][kernel]
    except Exception:
        return None
    if rec.get("source_sha") != kernel_source_sha(TC_SOURCES if kernel.endswith("_tc") else (), lengths):
        return None
    return rec.get("dram_bytes_per_launch")


# ----------------------------------------------------------------------------
# clock sampling during the timed region
# ----------------------------------------------------------------------------

class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        with open(self.path) as fh:
            for line in fh:
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9 or not f[0].isdigit() or int(f[0]) != self.gpu:
                    continue
                try:
                    sm.append(float(f[1]))
                    mx.append(float(f[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, f[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "samples": len(sm), "reasons": sorted(reasons)}


# ----------------------------------------------------------------------------
# CPU oracle timing (baseline arm and reference arm)
# ----------------------------------------------------------------------------

def oracle_rate(L, K, seconds, seed):
    """Time the FP64 direct sum on seeded pixels for about `seconds`."""
    import oracle
    import synth
    H, W = L.shape
    ii, jj = synth.sample_pixels(H, W, 256, seed)
    t0 = time.perf_counter()
    oracle.conv_points_same(L, K, ii, jj)
    dt = max(time.perf_counter() - t0, 1e-6)
    n = int(min(2_000_000, max(256, 256 * seconds / dt)))
    ii, jj = synth.sample_pixels(H, W, n, seed + 1)
    t0 = time.perf_counter()
    oracle.conv_points_same(L, K, ii, jj)
    dt = time.perf_counter() - t0
    return n / dt / 1e6, n, dt, oracle.num_threads()


def run_reference(args, rank, world):
    """--impl reference: the FP64 oracle on the host cores, rank 0 only."""
    import numpy as np
    import synth
    if rank != 0:
        return
    wl = load_workload(args.workload)
    L = wl.radiance()
    Ks = wl.psfs()
    K = Ks[0]
    # per-step sample sized so that warmup + steps take about two minutes
    rate, _, _, cores = oracle_rate(L, K, 2.0, wl.seed + 7)
    per_step = max(16, int(rate * 1e6 * 120.0 / max(1, args.steps + args.warmup)))
    import oracle
    H, W = L.shape
    tot_px, tot_s = 0, 0.0
    for s in range(args.warmup + args.steps):
        ii, jj = synth.sample_pixels(H, W, per_step, wl.seed + 1000 + s)
        t0 = time.perf_counter()
        for Kk in Ks:
            oracle.conv_points_same(L, Kk, ii, jj)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            tot_px += per_step * len(Ks)
            tot_s += dt
    value = tot_px / tot_s / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * tot_s / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(wl, None),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{per_step} seeded output pixels per step per PSF "
                                   f"({len(Ks)} PSF) of the {H}x{W} map, FP64 direct sum"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


class _PaperShape:
    """The paper's own map shape (Sec. 3) with its two PSFs."""
    def __init__(self):
        import synth
        p = synth.PAPER_SHAPE
        self.name, self.H, self.W, self.px_km = p["name"], p["H"], p["W"], p["px_km"]
        self.seed = p["seed"]
        self.psf_side = p["alr_side"]
        self.psf_params = ("alr", "zsb")
        self._p = p

    def radiance(self):
        import synth
        return synth.paper_shape_inputs()[0]

    def psfs(self):
        import synth
        p = self._p
        return [synth.psf_alr(p["alr_side"], p["px_km"]),
                synth.psf_power_exp(p["zsb_side"], p["px_km"], 0.1, 1.25, 26.0)]


def load_workload(name):
    import synth
    if name == synth.PAPER_SHAPE["name"]:
        return _PaperShape()
    return synth.WORKLOADS[name]


def workload_config(wl, pad):
    c = {"workload": wl.name, "map": f"{wl.H}x{wl.W}", "psf": f"{wl.psf_side}x{wl.psf_side}",
         "n_psf": len(wl.psf_params), "pixel_km": wl.px_km,
         "l2": "flushed between steps (256 MiB write, outside the timed events)"}
    if pad is not None:
        c["padded"] = f"{pad[0]}x{pad[1]}"
    return c


# ----------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------

def cufft_comparator(L, Ks, ny, nx, flush, steps, stream):
    import torch
    H, W = L.shape
    dev = L.device
    khs = []
    for K in Ks:
        hk, wk = K.shape
        Kd = torch.from_numpy(K).to(dev)
        Kw = torch.roll(torch.nn.functional.pad(Kd, (0, nx - wk, 0, ny - hk)),
                        shifts=(-(hk // 2), -(wk // 2)), dims=(0, 1))
        khs.append(torch.fft.rfft2(Kw).to(torch.complex64))
    outs = [None] * len(Ks)

    def step():
        Lh = torch.fft.rfft2(L, s=(ny, nx))
        for k, kh in enumerate(khs):
            outs[k] = torch.fft.irfft2(Lh * kh, s=(ny, nx))[:H, :W]

    for _ in range(3):
        step()
    torch.cuda.synchronize()
    e0 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    e1 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    for i in range(steps):
        flush.zero_()
        e0[i].record(stream)
        step()
        e1[i].record(stream)
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in zip(e0, e1)) / steps
    return {"value": H * W * len(Ks) / (ms / 1e3) / 1e6, "unit": UNIT, "ms_per_step": ms,
            "what": "torch.fft rfft2 (zero-padded) x spectrum -> irfft2 -> crop, FP32, same workload"}


def _host_fft():
    try:
        import scipy.fft as sf
        return sf, "scipy.fft (pocketfft)", os.cpu_count() or 1
    except ImportError:
        import numpy.fft as sf
        return sf, "numpy.fft (one thread: scipy absent)", 1


def host_fft_spectrum(K, ny, nx, dtype):
    """rfft2 of the PSF zero-padded to ny x nx with its centre at (0, 0)."""
    import numpy as np
    sf, _, workers = _host_fft()
    kw = {"workers": workers} if workers > 1 else {}
    hk, wk = K.shape
    Kw = np.zeros((ny, nx), dtype)
    Kw[:hk, :wk] = K
    Kw = np.roll(Kw, (-(hk // 2), -(wk // 2)), axis=(0, 1))
    return sf.rfft2(Kw, **kw)


def host_fft_map(L, khat, ny, nx, dtype):
    """The paper's method on the host: zero-padded rfft2 of the map, product
    with the spectrum, irfft2, crop to the map region."""
    import numpy as np
    sf, _, workers = _host_fft()
    kw = {"workers": workers} if workers > 1 else {}
    H, W = L.shape
    Lp = np.zeros((ny, nx), dtype)
    Lp[:H, :W] = L
    return sf.irfft2(sf.rfft2(Lp, **kw) * khat, s=(ny, nx), **kw)[:H, :W].copy()


def cpu_fft_comparator(L, Ks, ny, nx, reps=2):
    """The paper's own method on the host cores (bench only, not the product
    path): host_fft_map with scipy.fft (pocketfft) on all cores, in FP64 and
    FP32; the PSF spectra are computed once, outside the timing."""
    import numpy as np
    _, lib, workers = _host_fft()
    H, W = L.shape
    res = {"unit": UNIT, "cores": workers, "kind": lib + " rfft2 / irfft2, same workload and padding",
           "reps": reps}
    for name, rdt, cdt in (("fp64", np.float64, np.complex128), ("fp32", np.float32, np.complex64)):
        khs = [host_fft_spectrum(K, ny, nx, rdt).astype(cdt) for K in Ks]
        best = None
        for _ in range(reps):
            t0 = time.perf_counter()
            for kh in khs:
                host_fft_map(L, kh, ny, nx, rdt)
            dt = time.perf_counter() - t0
            best = dt if best is None else min(best, dt)
        res[name] = H * W * len(Ks) / best / 1e6
    return res


def _time_maps(lp, ctx, L, specs, outs, prec, steps, warmup, flush, stream, per_spectrum=False):
    """Device ms of each of `steps` maps (CUDA events on the launching stream
    around each call, L2 flushed between calls outside the events).  With
    per_spectrum, a step is one single-spectrum call per spectrum (the plain
    path without a shared forward transform)."""
    import torch

    def one():
        if per_spectrum:
            for s, o in zip(specs, outs):
                lp.lp_map(ctx, L, [s], [o], prec=prec)
        else:
            lp.lp_map(ctx, L, specs, outs, prec=prec)

    for _ in range(warmup):
        flush.zero_()
        one()
    lp.lp_sync_status(ctx)
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    torch.cuda.synchronize()
    for k in range(steps):
        flush.zero_()
        ev0[k].record(stream)
        one()
        ev1[k].record(stream)
    torch.cuda.synchronize()
    lp.lp_sync_status(ctx)
    return [a.elapsed_time(b) for a, b in zip(ev0, ev1)]


def _time_passes(lp, ctx, L, specs, outs, prec, pk, flush):
    """Per-pass durations from the library's pass events over pk maps (a loop
    of its own: events between the passes stop their launch overlap)."""
    lp.lp_set_pass_timing(ctx, True)
    lp.lp_get_pass_timing(ctx)
    for _ in range(pk):
        flush.zero_()
        lp.lp_map(ctx, L, specs, outs, prec=prec)
    lp.lp_sync_status(ctx)
    passes = lp.lp_get_pass_timing(ctx)
    lp.lp_set_pass_timing(ctx, False)
    return passes


def _roofline(passes, model, pk, peak):
    """Dominant pass: algorithmic bytes per launch (3-pass model x units per
    launch) / its average event-timed launch duration."""
    dom = max(PASSES, key=lambda p: passes[p][0])
    ms_tot, launches = passes[dom]
    per_launch_s = ms_tot / 1e3 / max(1, launches)
    per_launch_bytes = model[dom] * (pk / max(1, launches))
    achieved = per_launch_bytes / per_launch_s / 1e9
    return dom, achieved, per_launch_bytes, achieved / peak


def _pass_table(passes, model, pk):
    return {p: {"ms_per_launch": passes[p][0] / max(1, passes[p][1]), "launches": passes[p][1],
                "algorithmic_gbs": model[p] * pk / max(1, passes[p][1]) /
                (passes[p][0] / 1e3 / max(1, passes[p][1])) / 1e9}
            for p in PASSES}


def cpu_baseline_leg_error(L, Ks, outs, seed, n=4096, top=64):
    """The CPU-baseline leg's accuracy check: max |B - B_ref| / max |B_ref| of
    the GPU maps against the FP64 direct sum (the oracle), on n seeded pixels
    plus the `top` brightest pixels of each GPU output (so that the
    denominator is the map maximum).  Runs outside every timed region."""
    import numpy as np
    import oracle
    import synth
    H, W = L.shape
    worst = 0.0
    for k, (K, o) in enumerate(zip(Ks, outs)):
        B = o.cpu().numpy()
        ii, jj = synth.sample_pixels(H, W, n, seed + k)
        flat = np.argpartition(B.ravel(), -top)[-top:]
        ii = np.concatenate([ii, flat // W])
        jj = np.concatenate([jj, flat % W])
        ref = oracle.conv_points_same(L, K, ii, jj)
        err = float(np.max(np.abs(B[ii, jj].astype(np.float64) - ref)) / np.max(np.abs(ref)))
        worst = max(worst, err)
    return worst


def _form_map(lp, args, wl, prec_name, flush, stream, dev, compare_fp32=True, per_spectrum_plain=False):
    """One 'form' of the path on its own workload: Mpix/s, the dominant pass's
    roofline fraction on its byte model, the error against the oracle, and
    the plain FP32 path on the same workload beside it."""
    import torch
    peak, peak_kind = measured_peak()
    H, W = wl.H, wl.W
    L_host = wl.radiance()
    Ks = wl.psfs()
    n = len(Ks)
    hk_max = max(K.shape[0] for K in Ks)
    ctx = lp.lp_create(dev.index or 0)
    try:
        L = torch.from_numpy(L_host).to(dev)
        split = prec_name == "split_bf16"
        prec = lp.LP_PREC_SPLIT_BF16 if split else lp.LP_PREC_FP32
        ny = lp.lp_supported_size(H + hk_max - 1)
        if split:
            ny = min(n_ for n_ in lp.supported_sizes() if n_ >= H + hk_max - 1 and lp.lp_split_supported(n_))
        nx = lp.lp_supported_size(W + hk_max - 1)
        Kd = [torch.from_numpy(K).to(dev) for K in Ks]
        specs = [lp.lp_kernel_spectrum(ctx, K, pad_ny=ny, pad_nx=nx, prec=prec) for K in Kd]
        info = lp.lp_spectrum_info(specs[0])
        s_k = 4 if info["is_real"] else 8
        outs = [torch.empty((H, W), dtype=torch.float32, device=dev) for _ in range(n)]
        steps, warm = max(3, min(args.steps, 20)), max(3, min(args.warmup, 5))
        ms = statistics.mean(_time_maps(lp, ctx, L, specs, outs, prec, steps, warm, flush, stream))
        pk = min(args.steps, 50)
        passes = _time_passes(lp, ctx, L, specs, outs, prec, pk, flush)
        model = pass_bytes(H, W, ny, nx, n, s_k)
        dom, achieved, per_launch, frac = _roofline(passes, model, pk, peak)
        err = cpu_baseline_leg_error(L_host, Ks, outs, wl.seed + 300)
        rec = {"workload": wl.name, "map": f"{H}x{W}", "psf": f"{wl.psf_side}x{wl.psf_side}", "n_psf": n,
               "padded": f"{ny}x{nx}", "precision": prec_name, "mpix_s": H * W * n / (ms / 1e3) / 1e6,
               "ms_per_step": ms, "steps": steps,
               "roofline": {"kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                            "frac": frac, "peak_kind": peak_kind, "algorithmic_bytes_per_launch": per_launch},
               "passes": _pass_table(passes, model, pk), "max_norm_err": err,
               "tolerance": 2e-4 if split else 1e-5}
        for s in specs:
            lp.lp_spectrum_release(ctx, s)
        # the plain FP32 path on the same workload: FP32 spectra, and for the
        # batched form one single-spectrum call per PSF (no shared transform)
        if compare_fp32:
            nyp = lp.lp_supported_size(H + hk_max - 1)
            sp = [lp.lp_kernel_spectrum(ctx, K, pad_ny=nyp, pad_nx=nx) for K in Kd]
            pms = statistics.mean(_time_maps(lp, ctx, L, sp, outs, lp.LP_PREC_FP32, steps, warm, flush, stream,
                                             per_spectrum=per_spectrum_plain))
            rec["plain_fp32"] = {"mpix_s": H * W * n / (pms / 1e3) / 1e6, "ms_per_step": pms,
                                 "padded": f"{nyp}x{nx}",
                                 "what": ("one single-spectrum map call per PSF" if per_spectrum_plain
                                          else "FP32 column pass")}
            rec["speedup_vs_plain_fp32"] = rec["mpix_s"] / rec["plain_fp32"]["mpix_s"]
            for s in sp:
                lp.lp_spectrum_release(ctx, s)
        lp.lp_sync_status(ctx)
        return rec
    finally:
        lp.lp_destroy(ctx)


def _form_tiled(lp, args, wl, flush, stream, dev):
    """The tiled form: a map longer than the longest FFT length, in
    overlap-save tiles (lp_map_tiled) at the padded size lp_tiled_pad picks;
    Mpix/s, the error against the oracle, and the plain FP32 path beside it
    on the largest square sub-map one transform of the longest length
    holds."""
    import torch
    H, W = wl.H, wl.W
    L_host = wl.radiance()
    (K,) = wl.psfs()
    hk = K.shape[0]
    n_max = max(lp.supported_sizes())
    ctx = lp.lp_create(dev.index or 0)
    try:
        L = torch.from_numpy(L_host).to(dev)
        Kd = torch.from_numpy(K).to(dev)
        ny, nx = lp.lp_tiled_pad(H, W, hk, hk)
        spec = lp.lp_kernel_spectrum(ctx, Kd, pad_ny=ny, pad_nx=nx)
        out = torch.empty((H, W), dtype=torch.float32, device=dev)
        steps, warm = max(3, min(args.steps, 10)), max(3, min(args.warmup, 5))

        def one():
            lp.lp_map_tiled(ctx, L, [spec], [out])

        for _ in range(warm):
            flush.zero_()
            one()
        lp.lp_sync_status(ctx)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        torch.cuda.synchronize()
        for a, b in ev:
            flush.zero_()
            a.record(stream)
            one()
            b.record(stream)
        torch.cuda.synchronize()
        lp.lp_sync_status(ctx)
        ms = statistics.mean(a.elapsed_time(b) for a, b in ev)
        th, tw = ny - (hk - 1), nx - (hk - 1)
        tiles = -(-H // th) * -(-W // tw)
        err = cpu_baseline_leg_error(L_host, [K], [out], wl.seed + 300)
        lp.lp_spectrum_release(ctx, spec)
        rec = {"workload": wl.name, "map": f"{H}x{W}", "psf": f"{hk}x{hk}", "n_psf": 1,
               "padded": f"{ny}x{nx}", "tiles": tiles, "tile_output": f"{th}x{tw}", "precision": "fp32",
               "mpix_s": H * W / (ms / 1e3) / 1e6, "ms_per_step": ms, "steps": steps,
               "max_norm_err": err, "tolerance": 1e-5}
        # the plain path on the largest sub-map one transform of the longest
        # length holds
        spec = lp.lp_kernel_spectrum(ctx, Kd, pad_ny=n_max, pad_nx=n_max)
        side = n_max - (hk - 1)
        sub = L[:side, :side]
        osub = out[:side, :side]
        pms = statistics.mean(_time_maps(lp, ctx, sub, [spec], [osub], lp.LP_PREC_FP32, steps, warm, flush,
                                         stream))
        rec["plain_fp32"] = {"map": f"{side}x{side}", "mpix_s": side * side / (pms / 1e3) / 1e6,
                             "ms_per_step": pms, "padded": f"{n_max}x{n_max}",
                             "what": "lp_map on the largest square sub-map one transform holds"}
        rec["speedup_vs_plain_fp32"] = rec["mpix_s"] / rec["plain_fp32"]["mpix_s"]
        lp.lp_spectrum_release(ctx, spec)
        lp.lp_sync_status(ctx)
        return rec
    finally:
        lp.lp_destroy(ctx)


def _form_same_pad(lp, args, wl, flush, stream, dev):
    """The SAME crop at its own padding: a map that one transform holds,
    through lp_map_tiled in one tile at the padding lp_tiled_pad picks
    (h + (hk - 1) / 2 instead of lp_map's h + hk - 1), against lp_map on the
    same map; Mpix/s and the error against the oracle."""
    import torch
    H, W = wl.H, wl.W
    L_host = wl.radiance()
    (K,) = wl.psfs()
    hk = K.shape[0]
    ctx = lp.lp_create(dev.index or 0)
    try:
        L = torch.from_numpy(L_host).to(dev)
        Kd = torch.from_numpy(K).to(dev)
        ny, nx = lp.lp_tiled_pad(H, W, hk, hk)
        spec = lp.lp_kernel_spectrum(ctx, Kd, pad_ny=ny, pad_nx=nx)
        out = torch.empty((H, W), dtype=torch.float32, device=dev)
        steps, warm = max(3, min(args.steps, 20)), max(3, min(args.warmup, 5))
        ev = []
        for k in range(warm + steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            lp.lp_map_tiled(ctx, L, [spec], [out])
            b.record(stream)
            if k >= warm:
                ev.append((a, b))
        torch.cuda.synchronize()
        lp.lp_sync_status(ctx)
        ms = statistics.mean(a.elapsed_time(b) for a, b in ev)
        err = cpu_baseline_leg_error(L_host, [K], [out], wl.seed + 400)
        lp.lp_spectrum_release(ctx, spec)
        nyp, nxp = lp.lp_supported_size(H + hk - 1), lp.lp_supported_size(W + hk - 1)
        sp = lp.lp_kernel_spectrum(ctx, Kd, pad_ny=nyp, pad_nx=nxp)
        pms = statistics.mean(_time_maps(lp, ctx, L, [sp], [out], lp.LP_PREC_FP32, steps, warm, flush, stream))
        lp.lp_spectrum_release(ctx, sp)
        lp.lp_sync_status(ctx)
        return {"workload": wl.name, "map": f"{H}x{W}", "psf": f"{hk}x{hk}", "padded": f"{ny}x{nx}",
                "tiles": 1 if (H <= ny - (hk - 1) // 2 and W <= nx - (hk - 1) // 2) else None,
                "precision": "fp32", "mpix_s": H * W / (ms / 1e3) / 1e6, "ms_per_step": ms, "steps": steps,
                "max_norm_err": err, "tolerance": 1e-5,
                "plain_fp32": {"mpix_s": H * W / (pms / 1e3) / 1e6, "ms_per_step": pms, "padded": f"{nyp}x{nxp}",
                               "what": "lp_map, padded to h + hk - 1 (Sec. 2.5)"},
                "speedup_vs_plain_fp32": pms / ms,
                "what": "lp_map_tiled in one tile padded to h + (hk - 1) / 2, enough for the SAME crop"}
    finally:
        lp.lp_destroy(ctx)


def _graph_case(lp, flush, dev, side, psf, n_maps, steps, seed):
    """n_maps maps of side^2 with one psf^2 PSF, each its own input and
    output: direct lp_map_noalloc calls against one replay of the same calls
    captured into a CUDA graph.  Device time per loop by CUDA events (L2
    flushed before each loop) and host time to enqueue the loop."""
    import numpy as np
    import torch
    import oracle
    import synth
    K = synth.psf_power_exp(psf, 1.0, 0.25, 1.25, 40.0)
    ctx = lp.lp_create(dev.index or 0)
    try:
        spec = lp.lp_kernel_spectrum(ctx, torch.from_numpy(K).to(dev), max_h=side, max_w=side)
        lp.lp_sync_status(ctx)
        Ls = [torch.from_numpy(synth.radiance_map(side, side, 12, seed + i)).to(dev) for i in range(n_maps)]
        outs = [torch.empty_like(L) for L in Ls]
        s = torch.cuda.Stream()

        def loop():
            for L, o in zip(Ls, outs):
                lp.lp_map_noalloc(ctx, L, [spec], [o])

        with torch.cuda.stream(s):
            loop()
        s.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            loop()

        def timed(fn):
            dev_ms, host_ms = [], []
            with torch.cuda.stream(s):
                for k in range(steps + 3):
                    flush.zero_()
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record(s)
                    t0 = time.perf_counter()
                    fn()
                    t1 = time.perf_counter()
                    b.record(s)
                    b.synchronize()
                    if k >= 3:
                        dev_ms.append(a.elapsed_time(b))
                        host_ms.append((t1 - t0) * 1e3)
            return statistics.mean(dev_ms), statistics.mean(host_ms)

        d_ms, d_host = timed(loop)
        g_ms, g_host = timed(g.replay)
        B = outs[0].cpu().numpy().astype(np.float64)
        ref = oracle.conv_same(Ls[0].cpu().numpy(), K)
        err = float(np.max(np.abs(B - ref)) / np.max(np.abs(ref)))
        px = side * side * n_maps
        del g
        lp.lp_spectrum_release(ctx, spec)
        lp.lp_sync_status(ctx)
        return {"map": f"{side}x{side}", "psf": f"{psf}x{psf}", "maps_per_step": n_maps,
                "kernels_per_step": 3 * n_maps,
                "graph": {"mpix_s": px / (g_ms / 1e3) / 1e6, "ms_per_step": g_ms, "host_ms_per_step": g_host},
                "direct": {"mpix_s": px / (d_ms / 1e3) / 1e6, "ms_per_step": d_ms, "host_ms_per_step": d_host},
                "speedup_vs_direct": d_ms / g_ms, "max_norm_err": err, "tolerance": 1e-5}
    finally:
        lp.lp_destroy(ctx)


def _form_graph(lp, args, flush, stream, dev):
    """The launch-bound form: loops of small maps as direct calls and as one
    CUDA-graph replay, for 64^2 tiles (31^2 PSF) and for the 256^2 map with
    the 101^2 PSF."""
    steps = max(3, min(args.steps, 20))
    return {"what": "lp_map_noalloc loops: launched one by one (direct) against one replay of the "
                    "same calls captured into a CUDA graph (graph); device time by CUDA events, host "
                    "time to enqueue",
            "cases": [_graph_case(lp, flush, dev, 64, 31, 256, steps, 1907_02891 + 600),
                      _graph_case(lp, flush, dev, 256, 101, 64, steps, 1907_02891 + 700)]}


def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch
    import synth
    from paper_1907_02891_gb300 import lp

    dist = world > 1
    if dist:
        import torch.distributed as td
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    wl = load_workload(args.workload)
    H, W = wl.H, wl.W
    L_host = wl.radiance()
    Ks = wl.psfs()
    n = len(Ks)
    hk_max = max(K.shape[0] for K in Ks)

    ctx = lp.lp_create(local_rank)
    stream = torch.cuda.current_stream()
    L = torch.from_numpy(L_host).to(dev)
    prec = lp.LP_PREC_SPLIT_BF16 if args.prec == "split_bf16" else lp.LP_PREC_FP32
    t0 = time.perf_counter()
    # one padded size for all PSFs: the largest PSF's N_L + N_K - 1, rounded up
    # (for the split precision, to a column length that has that pass)
    ny = lp.lp_supported_size(H + hk_max - 1)
    if prec == lp.LP_PREC_SPLIT_BF16:
        ny = min(n_ for n_ in lp.supported_sizes() if n_ >= H + hk_max - 1 and lp.lp_split_supported(n_))
    nx = lp.lp_supported_size(W + hk_max - 1)
    specs = [lp.lp_kernel_spectrum(ctx, torch.from_numpy(K).to(dev), pad_ny=ny, pad_nx=nx, prec=prec)
             for K in Ks]
    torch.cuda.synchronize()
    s0_ms = 1e3 * (time.perf_counter() - t0) / n
    info = lp.lp_spectrum_info(specs[0])
    ny, nx = info["ny"], info["nx"]
    s_k = 4 if info["is_real"] else 8
    outs = [torch.empty((H, W), dtype=torch.float32, device=dev) for _ in range(n)]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    for _ in range(args.warmup):
        flush.zero_()
        lp.lp_map(ctx, L, specs, outs, prec=prec)
    lp.lp_sync_status(ctx)
    # timed region: events around each map only (per-pass events would sit
    # between the passes and cost ~8 % here, as they stop each pass's launch
    # from overlapping the tail of the one before)
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clocks = Clocks(local_rank)
    clocks.start()
    time.sleep(0.3)
    if dist:
        td.barrier()
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    for k in range(args.steps):
        flush.zero_()
        ev0[k].record(stream)
        lp.lp_map(ctx, L, specs, outs, prec=prec)
        ev1[k].record(stream)
    torch.cuda.synchronize()
    if dist:
        td.barrier()
    wall_s = time.perf_counter() - w0
    clk = clocks.stop()
    lp.lp_sync_status(ctx)
    step_ms = [a.elapsed_time(b) for a, b in zip(ev0, ev1)]
    dev_ms = float(sum(step_ms))
    dev_ms = max_over_ranks(dev_ms, dev)
    value = whole_job_mpix_s(float(H) * W * n, args.steps, world, dev_ms)

    # per-pass durations and the roofline of the dominant pass
    pk = min(args.steps, 500)
    passes = _time_passes(lp, ctx, L, specs, outs, prec, pk, flush)
    launches_per_step = sum(passes[p][1] for p in PASSES) / pk
    model = pass_bytes(H, W, ny, nx, n, s_k)
    peak, peak_kind = measured_peak()
    dom, achieved, per_launch_bytes, frac = _roofline(passes, model, pk, peak)
    traffic = dram_traffic(dom + ("_tc" if prec != lp.LP_PREC_FP32 and dom == "p2_cols" else ""), wl.name,
                           (ny, nx))

    # end to end through the host-buffer entry point (pinned host memory)
    e2e = None
    if args.e2e_steps > 0:
        Lh = torch.from_numpy(L_host).pin_memory()
        oh = [torch.empty((H, W), dtype=torch.float32).pin_memory() for _ in range(n)]
        for _ in range(3):
            lp.lp_map_host(ctx, Lh, specs, oh, prec=prec)
        lp.lp_sync_status(ctx)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        if dist:
            td.barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.e2e_steps):
            lp.lp_map_host(ctx, Lh, specs, oh, prec=prec)
        e1.record(stream)
        torch.cuda.synchronize()
        e_ms = max_over_ranks(e0.elapsed_time(e1), dev)
        e2e = {"value": whole_job_mpix_s(float(H) * W * n, args.e2e_steps, world, e_ms),
               "unit": UNIT, "h2d_bytes_per_step": 4 * H * W,
               "d2h_bytes_per_step": 4 * H * W * n, "steps": args.e2e_steps,
               "host_memory": "pinned"}

    # comparator (bench only, not the product path): the same map through
    # torch.fft, i.e. cuFFT -- zero-padded rfft2, product with the spectrum of
    # the wrap-placed PSF, irfft2, crop
    cufft = None
    if not args.no_cufft:
        cufft = cufft_comparator(L, Ks, ny, nx, flush, min(args.steps, 200), stream)

    cpu_fft = None
    if rank == 0 and world == 1 and not args.no_cpu_fft:
        cpu_fft = cpu_fft_comparator(L_host, Ks, ny, nx)

    # CPU-baseline leg (rank 0, N = 1): the oracle's accuracy check of this
    # run's maps, then the oracle timed on the host cores
    cpu = None
    max_err = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        max_err = cpu_baseline_leg_error(L_host, Ks, outs, wl.seed + 100)
        rate, npx, secs, cores = oracle_rate(L_host, Ks[0], args.cpu_seconds, wl.seed + 7)
        cpu = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{npx} seeded output pixels of the {H}x{W} map with the first "
                         f"{wl.psf_side}x{wl.psf_side} PSF, FP64 direct sum, {secs:.1f} s"}

    for s in specs:
        lp.lp_spectrum_release(ctx, s)
    lp.lp_destroy(ctx)

    # the batched, split-precision and served forms, each beside the plain
    # FP32 path on the same GPU (rank 0, N = 1)
    forms = None
    if rank == 0 and world == 1 and args.forms and not args.no_cpu_baseline:
        forms = {}
        want = set(args.forms.split(","))
        if "batched" in want:
            forms["batched"] = _form_map(lp, args, synth.WORKLOADS["map8192_psf601x16"], "fp32", flush,
                                         stream, dev, per_spectrum_plain=True)
            forms["batched"]["what"] = ("one call, 16 spectra: one forward row transform shared by all, "
                                        "plain = 16 single-spectrum calls")
        if "split_bf16" in want:
            forms["split_bf16"] = _form_map(lp, args, synth.WORKLOADS["map16384_psf801"], "split_bf16",
                                            flush, stream, dev)
        if "graph" in want:
            forms["graph"] = _form_graph(lp, args, flush, stream, dev)
        if "same_pad" in want:
            forms["same_pad"] = _form_same_pad(lp, args, synth.WORKLOADS["map4096_psf541"], flush, stream, dev)
        if "tiled" in want:
            forms["tiled"] = _form_tiled(lp, args, synth.WORKLOADS["map17800x21000_psf801"], flush, stream, dev)
        if "serve" in want:
            # over capacity (continuous batching against back to back), and
            # at 70 % load (latency beside throughput)
            forms["serve"] = serve_measure(args.forms_serve_requests, 1.3, args.slots, local_rank)
            forms["serve_load70"] = serve_measure(args.forms_serve_requests, 0.7, args.slots, local_rank,
                                                  check=False)
    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dev_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if prec == lp.LP_PREC_FP32 else "bf16-split (hi/lo) products, f32 accumulate",
        "data": "synthetic", "config": dict(workload_config(wl, (ny, nx)),
                       **({} if prec == lp.LP_PREC_FP32 else {"precision": args.prec})),
        "max_norm_err": max_err,
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": frac, "peak_kind": peak_kind,
                     "traffic": traffic,
                     "algorithmic_bytes_per_launch": per_launch_bytes,
                     "frac_of_nominal_8tbs": achieved / 8000.0},
        "passes": _pass_table(passes, model, pk),
        "whole_step_gbs": sum(model.values()) / (dev_ms / args.steps / 1e3) / 1e9 / world,
        "e2e": e2e, "cpu_baseline": cpu, "clocks": clk,
        "gpu_launches": int(round(launches_per_step * args.steps)),
        "pass_timing": f"per-pass CUDA events in a second loop of {pk} steps (the timed loop has none)",
        "cufft_comparator": cufft, "cpu_fft_comparator": cpu_fft,
        "spectrum_build_ms": s0_ms, "wall_s": wall_s,
        "forms": forms,
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------
# serving run
# ----------------------------------------------------------------------------

def serve_measure(n_requests, load, slots, local_rank, check=True, log_path=None):
    """Poisson arrivals of map requests (tile side uniform on 256..8192, 1-8
    PSFs of a bank of 8 cached 201^2 spectra) through the request scheduler;
    p50/p99 latency and Mpix/s.  The same requests run back to back through
    lp_map on one stream give the queue-alone reference.  With `check`, the
    last requests' outputs are compared bitwise with the same requests run
    alone, and the last one against the oracle (CPU-baseline leg).  With
    `log_path`, the scheduler appends one JSON line per timed request there
    (lp_serve_log)."""
    import threading
    import numpy as np
    import torch
    import synth
    from paper_1907_02891_gb300 import lp

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    ctx = lp.lp_create(local_rank)
    bank = [torch.from_numpy(K).to(dev) for K in synth.serve_bank()]
    sides = synth.SERVE_TILE_SIDES
    spectra = {(s, i): lp.lp_kernel_spectrum(ctx, K, max_h=s, max_w=s)
               for s in sides for i, K in enumerate(bank)}
    maps = {s: torch.from_numpy(synth.radiance_map(s, s, max(4, s * s // 42000), synth.SERVE_SEED + s,
                                                   lit_fraction=0.05)).to(dev) for s in sides}
    ring = 12
    outs = {s: [[torch.empty((s, s), device=dev) for _ in range(8)] for _ in range(ring)] for s in sides}
    torch.cuda.synchronize()

    def call_args(rq, r):
        s = rq.side
        return maps[s], [spectra[(s, i)] for i in rq.kernels], outs[s][r % ring][:len(rq.kernels)]

    # capacity: the request mix back to back on one stream
    probe = synth.request_stream(200, 1.0, seed=synth.SERVE_SEED + 99)
    for rq in probe[:20]:
        L, sp, o = call_args(rq, 0)
        lp.lp_map(ctx, L, sp, o)
    lp.lp_sync_status(ctx)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    px_probe = 0
    for r, rq in enumerate(probe):
        L, sp, o = call_args(rq, r)
        lp.lp_map(ctx, L, sp, o)
        px_probe += rq.side * rq.side * len(rq.kernels)
    e1.record()
    torch.cuda.synchronize()
    seq_s = e0.elapsed_time(e1) / 1e3
    seq_mpix = px_probe / seq_s / 1e6
    mean_service = seq_s / len(probe)
    rate = load / mean_service

    reqs = synth.request_stream(n_requests, rate)
    lp.lp_serve_start(ctx, slots)
    # warm every slot's workspace with the largest request
    big = max(reqs, key=lambda q: (q.side, len(q.kernels)))
    warm = [lp.lp_serve_submit(ctx, *call_args(big, k)) for k in range(slots)]
    for t in warm:
        lp.lp_serve_poll(ctx, t)
    if log_path:
        lp.lp_serve_log(ctx, log_path)
    tickets = [None] * len(reqs)
    lat = [None] * len(reqs)
    done_t = [0.0] * len(reqs)

    def poller():
        for r in range(len(reqs)):
            while tickets[r] is None:
                time.sleep(20e-6)
            lat[r] = lp.lp_serve_poll(ctx, tickets[r])
            done_t[r] = time.perf_counter()

    th = threading.Thread(target=poller)
    th.start()
    clocks = Clocks(local_rank)
    clocks.start()
    t0 = time.perf_counter()
    for r, rq in enumerate(reqs):
        now = time.perf_counter() - t0
        if rq.arrival_s > now:
            time.sleep(rq.arrival_s - now)
        if r >= ring:  # output ring: the request using these buffers must be done
            while lat[r - ring] is None:
                time.sleep(20e-6)
        tickets[r] = lp.lp_serve_submit(ctx, *call_args(rq, r))
    th.join()
    clk = clocks.stop()
    makespan = max(done_t) - t0
    lp.lp_serve_stop(ctx)
    px = sum(q.side * q.side * len(q.kernels) for q in reqs)
    lat_ms = np.array(lat, dtype=np.float64)
    by_side = {}
    for s in sides:
        sel = np.array([q.side == s for q in reqs])
        if sel.any():
            by_side[str(s)] = {"n": int(sel.sum()), "p50_ms": float(np.percentile(lat_ms[sel], 50)),
                               "p99_ms": float(np.percentile(lat_ms[sel], 99)),
                               "max_ms": float(lat_ms[sel].max())}
    same, err = None, None
    if check:
        # the last `ring` requests' buffers are still intact: rerun each alone
        same = True
        for r in range(max(0, len(reqs) - ring), len(reqs)):
            L, sp, o = call_args(reqs[r], r)
            alone = [torch.empty_like(x) for x in o]
            lp.lp_map(ctx, L, sp, alone)
            lp.lp_sync_status(ctx)
            same = same and all(torch.equal(x, y) for x, y in zip(o, alone))
        rq = reqs[-1]
        L, sp, o = call_args(rq, len(reqs) - 1)
        bank_np = synth.serve_bank()
        err = cpu_baseline_leg_error(L.cpu().numpy(), [bank_np[i] for i in rq.kernels], o,
                                     synth.SERVE_SEED + 500)
    line = {
        "metric": "serve p50/p99 ms", "value": float(np.percentile(lat_ms, 50)),
        "p99_ms": float(np.percentile(lat_ms, 99)), "unit": "ms", "higher_is_better": False,
        "n_gpus": 1, "requests": len(reqs), "slots": slots, "offered_load": load,
        "same_as_alone_bitwise": same, "max_norm_err": err,
        "speedup_vs_back_to_back": (px / makespan / 1e6) / seq_mpix,
        "arrival_rate_hz": rate, "served_mpix_s": px / makespan / 1e6,
        "back_to_back_mpix_s": seq_mpix, "mean_service_ms": 1e3 * mean_service,
        "makespan_s": makespan, "max_ms": float(lat_ms.max()), "by_side": by_side,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": "serve_tiles256-8192_bank8_psf201", "tile_sides": list(sides),
                   "psf": "201x201", "kernels_per_request": "1-8", "arrivals": "Poisson"},
        "clocks": clk,
    }
    lp.lp_destroy(ctx)
    return line


def run_serve(args, rank, world, local_rank):
    if rank != 0:
        return
    print(json.dumps(serve_measure(args.requests, args.load, args.slots, local_rank, log_path=args.serve_log)),
          flush=True)


def main():
    args = parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.mode == "serve":
        run_serve(args, rank, world, local_rank)
        return
    if world > 1:
        import torch
        import torch.distributed as td
        torch.cuda.set_device(local_rank)
        td.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    try:
        run_ours(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as td
            td.destroy_process_group()


if __name__ == "__main__":
    main()
