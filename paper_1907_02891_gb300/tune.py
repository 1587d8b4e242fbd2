"""Autotuner of the FFT plans per length.

For each length N it builds small variant libraries that contain only N,
each with one candidate plan of the in-place engine (radix order, two
transforms per block or one, threads per block, minimum resident blocks
per SM), times the three passes of a map whose padded size is N x N on the
GPU, and keeps, for the radix order with the best total, the best launch
setting of each pass; with several spectra per map it also compares the
batched column pass (one forward transform, parked) with one
single-spectrum pass per spectrum.  The result is written to
``tuned_plans.json`` beside this file (key "v2" of each length);
``build.py`` uses it for every length it lists.

    python -m paper_1907_02891_gb300.tune --sizes 4704 [--quick] \
        [--map-side 4096 --psf 541 --nspec 1] [--plan 12,8,7,7 ...]

The passes are timed one by one, with events between them, which stops the
launch overlap between passes of a real map; check a stored plan on the
whole map as well.

Needs nvcc and one GPU.  Each variant is timed in a fresh subprocess (the
variant libraries export the same symbols).
"""

from __future__ import annotations

import argparse
import concurrent.futures as cf
import hashlib
import itertools
import json
import os
import subprocess
import sys
import time
from typing import Dict, List, Tuple

from . import build as B

TUNE_DIR = os.path.join(B.OUT, "tune")
TUNED_JSON = os.path.join(B.HERE, "tuned_plans.json")
COMMON_SRCS = ("api.cu", "spectrum.cu", "noalloc.cu", "serve.cpp")


def _prod(p) -> int:
    r = 1
    for x in p:
        r *= x
    return r


def candidate_plans(n: int, pair: bool, limit: int = 3) -> List[Tuple[int, ...]]:
    """Radix orders of the in-place engine with the least modelled cost."""
    esize = 16 if pair else 8
    facs = B._ip_factorizations(n)
    smin = min(len(f) for f in facs)
    scored = []
    for f in {tuple(sorted(f)) for f in facs if len(f) <= smin + 1}:
        for perm in set(itertools.permutations(f)):
            if perm[-1] % 2 == 0 and any(r % 2 for r in perm):
                continue
            if pair and max(perm) > 16:
                continue
            T, blocks, score = B.ip_launch(n, perm, pair)
            scored.append((B.ip_cost(n, perm, esize) / max(score, 1e-3), perm))
    scored.sort()
    return [p for _, p in scored[:limit]]


def launch_options(n: int, rs, pair: bool) -> List[Tuple[int, int]]:
    """(threads per block, minimum resident blocks) around the planner's
    choice: its own, and the best-balanced shapes with one resident block
    more or less."""
    esize = 16 if pair else 8
    regs = B.ip_regs(rs, pair)
    by_smem = B.SMEM_SM // (n * esize + 1024)
    out = []
    T0, m0, _ = B.ip_launch(n, rs, pair)
    out.append((T0, m0))
    for m in sorted({m0 - 1, m0 + 1, by_smem}):
        if m < 1 or m > by_smem:
            continue
        best = None
        for T in range(64, 1025, 32):
            if T * m > 2048 or 65536 // (T * m) < min(regs, 96) - 8:
                continue
            nbs = [n // r for r in rs]
            eff = sum(nbs) / (T * sum((x + T - 1) // T for x in nbs))
            key = eff * min(1.0, T * m / 32 / 20.0)
            if best is None or key > best[0] + 1e-9:
                best = (key, T)
        if best and (best[1], m) not in out:
            out.append((best[1], m))
    return out


def _compile_common(jobs: int) -> List[str]:
    os.makedirs(os.path.join(TUNE_DIR, "common"), exist_ok=True)
    deps = max(os.path.getmtime(h) for h in B._headers())
    srcs = [os.path.join(B.CSRC, f) for f in COMMON_SRCS]
    objs = []
    with cf.ThreadPoolExecutor(jobs) as ex:
        objs = list(ex.map(lambda s: B._compile(s, deps), srcs))
    return objs


def _variant_lib(n: int, plan: dict, common: List[str]) -> str:
    key = json.dumps([n, plan], sort_keys=True)
    vid = hashlib.sha1(key.encode()).hexdigest()[:12]
    d = os.path.join(TUNE_DIR, vid)
    lib = os.path.join(d, "liblp.so")
    if os.path.exists(lib):
        return lib
    os.makedirs(d, exist_ok=True)
    text = B._tu_text(n, plan)
    src = os.path.join(d, f"size_{n}.cu")
    with open(src, "w") as fh:
        fh.write(text)
    reg = os.path.join(d, "registry.cu")
    with open(reg, "w") as fh:
        fh.write(B._REGISTRY_TU.format(decls=f"extern const SizeKernels kSize_{n};",
                                       ptrs=f"&kSize_{n}", count=1))
    objs = []
    for s in (src, reg):
        o = s[:-3] + ".o"
        cmd = ["nvcc", *B.ARCH, *B.NVCC_FLAGS, "-I", B.CSRC, "-I", os.path.join(B.ROOT, "include"),
               "-c", s, "-o", o]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"nvcc failed for variant {vid}:\n{res.stderr}")
        objs.append(o)
    res = subprocess.run(["nvcc", *B.ARCH, "-shared", "-o", lib, *common, *objs, "-lcudart"],
                         capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"link failed for variant {vid}:\n{res.stderr}")
    return lib


_RUNNER = r"""
import json, sys, time
import numpy as np
import torch
sys.path.insert(0, {root!r})
import paper_1907_02891_gb300.lp as lp
lp.load_library({lib!r})
n, reps, side, psf, nspec = {n}, {reps}, {side}, {psf}, {nspec}
hk = psf if psf > 0 else min(541, max(3, (n // 8) | 1))
h = w = side if side > 0 else n - hk + 1
dev = torch.device("cuda", 0)
ctx = lp.lp_create(0)
g = np.random.default_rng(1)
L = torch.from_numpy(g.random((h, w), dtype=np.float32)).to(dev)
r = np.hypot(*np.meshgrid(np.arange(hk) - hk // 2, np.arange(hk) - hk // 2, indexing="ij"))
specs = [lp.lp_kernel_spectrum(ctx, torch.from_numpy((r * r + 0.1) ** -(1.0 + 0.25 * i)).to(dev),
                               pad_ny=n, pad_nx=n) for i in range(nspec)]
outs = [torch.empty_like(L) for _ in specs]
flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
for _ in range(5):
    lp.lp_map(ctx, L, specs, outs)
lp.lp_sync_status(ctx)
lp.lp_set_pass_timing(ctx, True)
lp.lp_get_pass_timing(ctx)
for _ in range(reps):
    flush.zero_()
    lp.lp_map(ctx, L, specs, outs)
lp.lp_sync_status(ctx)
t = lp.lp_get_pass_timing(ctx)
print(json.dumps({{k: v[0] / max(1, v[1]) for k, v in t.items()}}))
lp.lp_destroy(ctx)
"""


def time_variant(lib: str, n: int, reps: int, side: int = 0, psf: int = 0, nspec: int = 1) -> Dict[str, float]:
    code = _RUNNER.format(root=B.ROOT, lib=lib, n=n, reps=reps, side=side, psf=psf, nspec=nspec)
    res = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600)
    if res.returncode != 0:
        raise RuntimeError(f"timing failed for {lib}:\n{res.stderr[-2000:]}")
    return json.loads(res.stdout.strip().splitlines()[-1])


def tune_size(n: int, quick: bool, jobs: int, common: List[str], log, side: int = 0, psf: int = 0,
              nspec: int = 1, plans: List[Tuple[int, ...]] = ()) -> dict:
    base = B.plan_table()[n]
    pairs = [1, 0] if 16 * n + 1024 <= B.SMEM_SM else [0]
    variants = []
    for pair in pairs:
        rlist = [tuple(p) for p in plans] or candidate_plans(n, bool(pair), 2 if quick else 3)
        for rs in rlist:
            for T, m in launch_options(n, rs, bool(pair)):
                p = dict(base)
                p.update(ip=list(rs), pair=[pair] * 3, t=[T] * 3, m=[m] * 3, batch=True)
                variants.append(p)
    t0 = time.time()

    def build_or_error(p):
        try:
            return _variant_lib(n, p, common)
        except RuntimeError as e:  # a variant that does not compile is skipped
            return e

    with cf.ThreadPoolExecutor(jobs) as ex:
        libs = list(ex.map(build_or_error, variants))
    log(f"N={n}: built {sum(isinstance(l, str) for l in libs)} of {len(libs)} variants in {time.time() - t0:.0f} s")
    reps = 200 if n <= 5200 else 40
    results = []
    for p, lib in zip(variants, libs):
        tag = f"{p['ip']} pair={p['pair'][0]} T={p['t'][0]} m={p['m'][0]}"
        if not isinstance(lib, str):
            log(f"  skip {tag}: build failed: {str(lib).strip().splitlines()[-1][:120]}")
            continue
        try:
            t = time_variant(lib, n, reps, side, psf, nspec)
        except Exception as e:  # a variant that does not launch (resources) is skipped
            log(f"  skip {tag}: {str(e).splitlines()[-1][:120]}")
            continue
        results.append((p, t))
        log(f"  {tag}: " + " ".join(f"{k}={v * 1e3:.1f}us" for k, v in t.items()))
    if not results:
        raise RuntimeError(f"no variant of {n} ran")
    # per radix order: the best (pair, threads, blocks) of each pass; then the
    # order with the best total
    best = None
    for rs in sorted({tuple(p["ip"]) for p, _ in results}):
        rr = [(p, t) for p, t in results if tuple(p["ip"]) == rs]
        choice, total = {}, 0.0
        for name in ("p1_rows", "p2_cols", "p3_rows"):
            p, t = min(rr, key=lambda x: x[1][name])
            choice[name] = p
            total += t[name]
        if best is None or total < best[0]:
            best = (total, rs, choice)
    total, rs, choice = best
    names = ("p1_rows", "p2_cols", "p3_rows")
    v2 = dict(ip=list(rs), pair=[choice[k]["pair"][0] for k in names], t=[choice[k]["t"][0] for k in names],
              m=[choice[k]["m"][0] for k in names], batch=True, tuned_total_us=total * 1e3)
    log(f"N={n}: chose {v2} (sum of best passes {total * 1e3:.1f} us)")
    if nspec > 1:
        p = dict(base)
        p.update(v2, batch=False)
        lib = build_or_error(p)
        if isinstance(lib, str):
            try:
                t = time_variant(lib, n, reps, side, psf, nspec)
                log(f"  batch=0: " + " ".join(f"{k}={v * 1e3:.1f}us" for k, v in t.items()))
                pbest = min(t2["p2_cols"] for p2, t2 in results if tuple(p2["ip"]) == rs)
                if t["p2_cols"] < pbest * 0.99:
                    v2["batch"] = False
            except Exception as e:
                log(f"  skip batch=0: {str(e).splitlines()[-1][:120]}")
        log(f"N={n}: batch={v2['batch']}")
    return v2


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--sizes", type=int, nargs="+", required=True)
    ap.add_argument("--quick", action="store_true")
    ap.add_argument("--jobs", type=int, default=0)
    ap.add_argument("--out", default=TUNED_JSON)
    ap.add_argument("--log", default=None)
    ap.add_argument("--plan", action="append", default=[],
                    help="radix sequence to try, e.g. 12,8,7,7 (repeatable; default: the candidate list)")
    ap.add_argument("--psf", type=int, default=0, help="PSF side of the timed maps (default min(541, N/8))")
    ap.add_argument("--nspec", type=int, default=1, help="spectra per timed map (one forward transform)")
    ap.add_argument("--map-side", type=int, default=0,
                    help="time maps of this side instead of N - PSF + 1, to compare "
                         "padded lengths for one workload")
    args = ap.parse_args()
    jobs = args.jobs or (os.cpu_count() or 1)
    logf = open(args.log, "a") if args.log else None

    def log(msg):
        print(msg, flush=True)
        if logf:
            logf.write(msg + "\n")
            logf.flush()

    for n in args.sizes:
        if n not in B.SIZES:
            raise SystemExit(f"{n} is not in the supported size list")
    plans = [tuple(int(x) for x in p.split(",")) for p in args.plan]
    for p in plans:
        if len(args.sizes) != 1 or _prod(p) != args.sizes[0] or max(p) > 16:
            raise SystemExit(f"plan {p} is not a radix sequence of length {args.sizes}")
    common = _compile_common(jobs)
    table = {}
    if os.path.exists(args.out):
        with open(args.out) as fh:
            table = json.load(fh)
    for n in args.sizes:
        v2 = tune_size(n, args.quick, jobs, common, log, args.map_side, args.psf, args.nspec, plans)
        v2["tuned_on"] = {"map_side": args.map_side, "psf": args.psf, "nspec": args.nspec}
        table.setdefault(str(n), {})["v2"] = v2
        with open(args.out, "w") as fh:
            json.dump(table, fh, indent=1, sort_keys=True)
    log(f"wrote {args.out}")


if __name__ == "__main__":
    main()
