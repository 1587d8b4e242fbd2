"""Autotuner of the FFT plans (radix order and launch shape) per length.

For each length N it builds small variant libraries that contain only N,
each with one candidate radix sequence and one setting of the launch knobs
of the prefetching kernels (work units per block, minimum resident blocks per
SM, spectrum-column staging), times the three passes of a map whose padded
size is N x N on the GPU, and keeps, for the fastest radix sequence, the best
knob setting of each pass, then refines it (double-buffered exchange; with
several spectra per map, one single-spectrum column pass per spectrum
against the batched kernel).  The result is written to ``tuned_plans.json``
beside this file (or to the file $LP_TUNE_CACHE names); ``build.py`` uses
it for every length it lists.

    python -m paper_1907_02891_gb300.tune --sizes 4704 [--quick] \
        [--map-side 4096 --psf 541 --nspec 1] [--plan 21,16,14 ...]

The passes are timed one by one, with events between them, which stops the
launch overlap between passes of a real map; check a stored plan on the
whole map as well (a setting that speeds one pass up can slow the map down).

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
COMMON_SRCS = ("api.cu", "spectrum.cu", "noalloc.cu", "serve.cpp")


def _prod(p) -> int:
    r = 1
    for x in p:
        r *= x
    return r


def candidate_plans(n: int, limit: int = 3) -> List[Tuple[int, ...]]:
    """Radix sequences ordered like build.choose_plan, then the other orders
    of the same multisets (first radix odd / large first)."""
    scored = []
    for f in B.factorizations(n):
        if B.threads_for(n, f) > B.MAX_THREADS:
            continue
        scored.append(((len(f), max(f), -min(f)), f))
    scored.sort()
    out: List[Tuple[int, ...]] = []
    for _, f in scored:
        for perm in (tuple(sorted(f, reverse=True)), tuple(sorted(f))):
            if perm not in out:
                out.append(perm)
        if len(out) >= limit:
            break
    return out[:limit]


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
    r = list(plan["radices"])
    text = B._SIZE_TU.format(n=n, seq=", ".join(map(str, r)), f1=plan["f1"], f3=plan["f3"], ns=len(r),
                             tt=plan.get("tt", 0),
                             upb1=plan["upb"][0], upb2=plan["upb"][1], upb3=plan["upb"][2],
                             minb1=plan["minb"][0], minb2=plan["minb"][1], minb3=plan["minb"][2],
                             kstage="true" if plan["kstage"] else "false",
                             pf1=B._b(plan["pf"][0]), pf2=B._b(plan["pf"][1]), pf3=B._b(plan["pf"][2]),
                             db1=B._b(plan["db"][0]), db2=B._b(plan["db"][1]), db3=B._b(plan["db"][2]),
                             batch=B._b(plan.get("batch", True)),
                             kst2=B._b(plan.get("kst2", False)), packed=int(bool(plan.get("packed", False))),
                             late1=B._b(plan.get("late", B.DEFAULT_LATE)[0]), late2=B._b(plan.get("late", B.DEFAULT_LATE)[1]),
                             rad6=", ".join(map(str, r + [0] * (6 - len(r)))))
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
# a length below the linear-convolution padding (the SAME crop's own one)
# maps in one tile through lp_map_tiled
mapf = lp.lp_map if min(h, w) + hk - 1 <= n else (lambda c, L, s, o: lp.lp_map_tiled(c, L, s, o))
for _ in range(5):
    mapf(ctx, L, specs, outs)
lp.lp_sync_status(ctx)
if {whole}:
    # whole maps, CUDA events around each (the passes overlap as in use)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    for a, b in ev:
        flush.zero_()
        a.record()
        mapf(ctx, L, specs, outs)
        b.record()
    torch.cuda.synchronize()
    print(json.dumps({{"map": sum(a.elapsed_time(b) for a, b in ev) / len(ev)}}))
    lp.lp_destroy(ctx)
    sys.exit(0)
lp.lp_set_pass_timing(ctx, True)
lp.lp_get_pass_timing(ctx)
for _ in range(reps):
    flush.zero_()
    mapf(ctx, L, specs, outs)
lp.lp_sync_status(ctx)
t = lp.lp_get_pass_timing(ctx)
print(json.dumps({{k: v[0] / max(1, v[1]) for k, v in t.items()}}))
lp.lp_destroy(ctx)
"""


def time_variant(lib: str, n: int, reps: int, side: int = 0, psf: int = 0, nspec: int = 1,
                 whole: bool = False) -> Dict[str, float]:
    """Mean ms per launch of each pass (pass events), or with whole the mean
    ms of whole maps ({"map": ms}), whose passes overlap as in use."""
    code = _RUNNER.format(root=B.ROOT, lib=lib, n=n, reps=reps, side=side, psf=psf, nspec=nspec,
                          whole="True" if whole else "False")
    res = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600)
    if res.returncode != 0:
        raise RuntimeError(f"timing failed for {lib}:\n{res.stderr[-2000:]}")
    return json.loads(res.stdout.strip().splitlines()[-1])


def tune_size(n: int, quick: bool, jobs: int, common: List[str], log, side: int = 0, psf: int = 0,
              nspec: int = 1, plans: List[Tuple[int, ...]] = (), packed: bool = False) -> dict:
    base = dict(B.plan_table_entry(n), packed=packed)
    plans = list(plans) or candidate_plans(n, 2 if quick else 3)
    knobs = []
    for upb, minb, kst in itertools.product((1, 2, 3), (1, 2, 3), (False, True)):
        if quick and (minb == 3 and upb == 1):
            continue
        if upb == 3 and (quick or kst):
            continue
        knobs.append((upb, minb, kst, 1))
    knobs.append((1, 1, False, 0))   # one-unit-per-block kernels (no prefetch)
    knobs.append((1, 2, False, 0))
    knobs.append((1, 3, False, 0))
    variants = []
    for r in plans:
        # threads per transform: one butterfly per thread in every stage (0),
        # or as many as the stage with the fewest butterflies (whole warps)
        tts = [0]
        few = (n // max(r) + 31) // 32 * 32
        if few < B.threads_for(n, r):
            tts.append(few)
        for tt in tts:
            for upb, minb, kst, pf in knobs:
                if tt and (kst or not pf):   # staging / no-prefetch only at the default thread count
                    continue
                p = dict(base)
                p.update(radices=list(r), threads=tt or B.threads_for(n, r), upb=[upb] * 3,
                         minb=[minb] * 3, kstage=kst, tt=tt, pf=[pf] * 3, db=[0, 0, 0])
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
    results = []
    for p, lib in zip(variants, libs):
        if not isinstance(lib, str):
            log(f"  skip {p['radices']} upb={p['upb'][0]} minb={p['minb'][0]}: build failed: "
                f"{str(lib).strip().splitlines()[-1][:120]}")
            continue
        try:
            t = time_variant(lib, n, 200 if n <= 5200 else 40, side, psf, nspec)
        except Exception as e:  # a variant that does not launch (resources) is skipped
            log(f"  skip {p['radices']} upb={p['upb'][0]} minb={p['minb'][0]} kstage={p['kstage']}: "
                f"{str(e).splitlines()[-1][:120]}")
            continue
        results.append((p, t))
        log(f"  {p['radices']} tt={p['tt']} pf={p['pf'][0]} upb={p['upb'][0]} minb={p['minb'][0]} kstage={int(p['kstage'])}: "
            + " ".join(f"{k}={v * 1e3:.1f}us" for k, v in t.items()))
    if not results:
        raise RuntimeError(f"no variant of {n} ran")
    # per (radix plan, threads per transform): best knob per pass; then the
    # combination with the best total
    best = None
    for r, tt in sorted({(tuple(p["radices"]), p["tt"]) for p, _ in results}):
        rs = [(p, t) for p, t in results if tuple(p["radices"]) == r and p["tt"] == tt]
        if not rs:
            continue
        choice, total = {}, 0.0
        for k, name in enumerate(("p1_rows", "p2_cols", "p3_rows")):
            # fastest setting; among those within 1 % of it (a knob the
            # timed workload does not exercise), the fewest resident blocks
            # (highest register cap), fewest units per block, no staging
            tbest = min(t[name] for _, t in rs)
            near = [(p, t) for p, t in rs if t[name] <= tbest * 1.01]
            p, t = min(near, key=lambda x: (x[0]["minb"][k], x[0]["upb"][k], x[0]["kstage"], x[1][name]))
            choice[name] = p
            total += t[name]
        if best is None or total < best[0]:
            best = (total, r, choice, tt)
    total, r, choice, tt = best
    out = dict(base)
    out.update(radices=list(r), threads=tt or B.threads_for(n, r), tt=tt,
               upb=[choice["p1_rows"]["upb"][0], choice["p2_cols"]["upb"][1], choice["p3_rows"]["upb"][2]],
               minb=[choice["p1_rows"]["minb"][0], choice["p2_cols"]["minb"][1], choice["p3_rows"]["minb"][2]],
               kstage=choice["p2_cols"]["kstage"], tuned_total_us=total * 1e3,
               pf=[choice["p1_rows"]["pf"][0], choice["p2_cols"]["pf"][1], choice["p3_rows"]["pf"][2]])
    log(f"N={n}: chose {out['radices']} tt={out['tt']} pf={out['pf']} upb={out['upb']} minb={out['minb']} kstage={out['kstage']} "
        f"(sum of best passes {total * 1e3:.1f} us)")
    # refinement: double-buffered exchange on top of the choice, with each
    # resident-block setting; kept per pass where it is faster
    best_pass = {name: min(t[name] for p, t in results if tuple(p["radices"]) == tuple(out["radices"])
                           and p["tt"] == out["tt"] and p["upb"][i] == out["upb"][i] and p["pf"][i] == out["pf"][i]
                           and p["minb"][i] == out["minb"][i] and (i != 1 or p["kstage"] == out["kstage"]))
                 for i, name in enumerate(("p1_rows", "p2_cols", "p3_rows"))}
    refine = []
    for minb in (1, 2, 3):
        p = dict(out)
        p.update(db=[1, 1, 1], minb=[minb] * 3)
        refine.append(p)
    with cf.ThreadPoolExecutor(jobs) as ex:
        rlibs = list(ex.map(build_or_error, refine))
    db, minb = [0, 0, 0], list(out["minb"])
    for p, lib in zip(refine, rlibs):
        if not isinstance(lib, str):
            continue
        try:
            t = time_variant(lib, n, 200 if n <= 5200 else 40, side, psf, nspec)
        except Exception as e:
            log(f"  skip db=1 minb={p['minb'][0]}: {str(e).splitlines()[-1][:120]}")
            continue
        log(f"  db=1 minb={p['minb'][0]}: " + " ".join(f"{k}={v * 1e3:.1f}us" for k, v in t.items()))
        for i, name in enumerate(("p1_rows", "p2_cols", "p3_rows")):
            if t[name] < best_pass[name] * 0.99:
                best_pass[name] = t[name]
                db[i], minb[i] = 1, p["minb"][0]
    out.update(db=db, minb=minb, tuned_total_us=sum(best_pass.values()) * 1e3)
    log(f"N={n}: refined db={db} minb={minb} (sum {out['tuned_total_us']:.1f} us)")
    # packed FP32x2 DFT arithmetic: one switch for the whole length (its
    # constants take registers, which can make a register-capped kernel
    # spill); kept where all three passes together are faster
    p = dict(out, packed=not out.get("packed", False))
    lib = build_or_error(p)
    if isinstance(lib, str):
        try:
            t = time_variant(lib, n, 200 if n <= 5200 else 40, side, psf, nspec)
            log(f"  packed={int(p['packed'])}: " + " ".join(f"{k}={v * 1e3:.1f}us" for k, v in t.items()))
            if sum(t.values()) < sum(best_pass.values()) * 0.99:
                best_pass = dict(t)
                out.update(packed=p["packed"], tuned_total_us=sum(best_pass.values()) * 1e3)
        except Exception as e:
            log(f"  skip packed={int(p['packed'])}: {str(e).splitlines()[-1][:120]}")
    log(f"N={n}: packed={out.get('packed', False)}")
    # whole-map refinement: the pass timings above stop the launch overlap
    # between passes, which decides the trigger point and interacts with the
    # forward row pass's resident blocks; time whole maps of the choice and
    # of those neighbours, keep the fastest
    reps = 200 if n <= 5200 else 40
    late0 = list(out.get("late", B.DEFAULT_LATE))
    cands = [dict(out, late=late0), dict(out, late=[0, 0, 0])]
    m1 = out["minb"][0]
    for mb in (m1 - 1, m1 + 1):
        if 1 <= mb <= 3:
            cands.append(dict(out, late=late0, minb=[mb] + list(out["minb"][1:])))
    best_map = None
    for p in cands:
        lib = build_or_error(p)
        if not isinstance(lib, str):
            continue
        try:
            ms = min(time_variant(lib, n, reps, side, psf, nspec, whole=True)["map"] for _ in range(2))
        except Exception as e:
            log(f"  skip whole map late={p['late']} minb={p['minb']}: {str(e).splitlines()[-1][:120]}")
            continue
        log(f"  whole map late={p['late']} minb={p['minb']}: {ms * 1e3:.1f} us")
        if best_map is None or ms < best_map[0] * 0.995:
            best_map = (ms, p)
    if best_map is not None:
        out.update(late=best_map[1]["late"], minb=best_map[1]["minb"], tuned_map_us=best_map[0] * 1e3)
    log(f"N={n}: late={out.get('late')} minb={out['minb']} (whole map {out.get('tuned_map_us', 0):.1f} us)")
    if nspec > 1:
        # several spectra: the batched column kernel against one single-
        # spectrum pass per spectrum
        p = dict(out, batch=False)
        lib = build_or_error(p)
        if isinstance(lib, str):
            try:
                t = time_variant(lib, n, 200 if n <= 5200 else 40, side, psf, nspec)
                log(f"  batch=0: " + " ".join(f"{k}={v * 1e3:.1f}us" for k, v in t.items()))
                if t["p2_cols"] < best_pass["p2_cols"] * 0.99:
                    best_pass["p2_cols"] = t["p2_cols"]
                    out.update(batch=False, tuned_total_us=sum(best_pass.values()) * 1e3)
            except Exception as e:
                log(f"  skip batch=0: {str(e).splitlines()[-1][:120]}")
        log(f"N={n}: batch={out.get('batch', True)} (sum {out['tuned_total_us']:.1f} us)")
    return out


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--sizes", type=int, nargs="+", required=True)
    ap.add_argument("--quick", action="store_true")
    ap.add_argument("--jobs", type=int, default=0)
    ap.add_argument("--out", default=B.tuned_json_path(),
                    help="plan file to update (default: $LP_TUNE_CACHE, else tuned_plans.json)")
    ap.add_argument("--log", default=None)
    ap.add_argument("--plan", action="append", default=[],
                    help="radix sequence to try, e.g. 7,7,8,12 (repeatable; default: the candidate list)")
    ap.add_argument("--psf", type=int, default=0, help="PSF side of the timed maps (default min(541, N/8))")
    ap.add_argument("--nspec", type=int, default=1, help="spectra per timed map (one forward transform)")
    ap.add_argument("--map-side", type=int, default=0,
                    help="time maps of this side instead of N - PSF + 1, to compare "
                         "padded lengths for one workload")
    ap.add_argument("--packed", action="store_true",
                    help="search the knobs with packed FP32x2 arithmetic (the last step still tries both)")
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
        if len(args.sizes) != 1 or _prod(p) != args.sizes[0] or max(p) > 32:
            raise SystemExit(f"plan {p} is not a radix sequence of length {args.sizes}")
    common = _compile_common(jobs)
    table = {}
    if os.path.exists(args.out):
        with open(args.out) as fh:
            table = json.load(fh)
    for n in args.sizes:
        table[str(n)] = tune_size(n, args.quick, jobs, common, log, args.map_side, args.psf, args.nspec, plans,
                                  args.packed)
        table[str(n)]["tuned_on"] = {"map_side": args.map_side, "psf": args.psf, "nspec": args.nspec}
        with open(args.out, "w") as fh:
            json.dump(table, fh, indent=1, sort_keys=True)
    log(f"wrote {args.out}")


if __name__ == "__main__":
    main()
