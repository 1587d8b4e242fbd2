"""Build liblp.so (sm_103a) in-tree.

The FP32 FFT kernels are templates over the radix sequence of each supported
transform length.  This script picks one radix sequence per length (the
plan table below), writes one small translation unit per length into
``_build/gen``, and compiles everything with nvcc in parallel:

    python -m paper_1907_02891_gb300.build          # or build() from Python

Output: ``paper_1907_02891_gb300/_build/liblp.so``.
"""

from __future__ import annotations

import concurrent.futures as cf
import hashlib
import json
import os
import shutil
import subprocess
import sys
from typing import Dict, List, Sequence, Tuple

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
GEN = os.path.join(OUT, "gen")
OBJ = os.path.join(OUT, "obj")
LIB = os.path.join(OUT, "liblp.so")
# debug build (LP_DEBUG=1: the passes check every work unit's extents in
# every buffer first and report a miss in the device status word); a
# library of its own, loaded by lp.py when $LP_DEBUG is set
DEBUG_OBJ = os.path.join(OUT, "debug", "obj")
DEBUG_LIB = os.path.join(OUT, "debug", "liblp.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "--expt-relaxed-constexpr", "-lineinfo",
              "-Xcompiler", "-fPIC", "-Xcompiler", "-O2"]

# radices the in-register DFTs are instantiated for (7-smooth, <= 32)
RADICES = (2, 3, 4, 5, 6, 7, 8, 9, 10, 12, 14, 15, 16, 18, 20, 21, 24, 25, 27, 28, 30, 32)
MAX_THREADS = 1024
PF_UNITS = 2          # work units per block of the prefetching kernels
# trigger of the next pass at block exit for the forward row pass and the
# one-spectrum column pass (the inverse row pass triggers at block start):
# measured faster or equal on the whole map at 4608, 4704, 8820 (one and 16
# spectra) and 17280
DEFAULT_LATE = [1, 1, 0]
SMEM_LIMIT = 227 * 1024

# Supported transform lengths.  Every length is 7-smooth; the list covers
# the workload sizes (360, 480, 720, 1260, 2250, 4320, 4704, 8400, 8820,
# 17280; 4608 = 4096 + 512 for the 4096^2 map's SAME crop with a 541^2 PSF
# in one tile), powers of two, and a ladder in between.
SIZES = (
    45, 64, 96, 100, 120, 128, 160, 192, 210, 240, 256, 288, 320, 360, 384, 420, 480, 512,
    560, 640, 720, 768, 840, 960, 1024, 1120, 1260, 1344, 1536, 1680, 1792, 2048, 2250, 2520,
    2688, 3072, 3360, 3584, 4096, 4320, 4608, 4704, 4800, 4860, 5040, 5120, 5376, 6144, 6720, 7168,
    8192, 8400, 8640, 8820, 9000, 9216,
    10080, 10752, 12288, 13440, 15360, 16384, 17280,
)


def spad_size(n: int) -> int:
    return n + (n >> 5) + 1


def factorizations(n: int, max_stages: int = 4) -> List[Tuple[int, ...]]:
    out: List[Tuple[int, ...]] = []

    def rec(rem: int, start: int, cur: List[int]) -> None:
        if rem == 1:
            out.append(tuple(cur))
            return
        if len(cur) == max_stages:
            return
        for i in range(start, len(RADICES)):
            r = RADICES[i]
            if rem % r == 0:
                rec(rem // r, i, cur + [r])

    rec(n, 0, [])
    return out


def threads_for(n: int, radices: Sequence[int]) -> int:
    return (n // min(radices) + 31) // 32 * 32


def choose_plan(n: int) -> Tuple[int, ...]:
    """Fewest stages; then the smallest largest radix (register pressure);
    then the largest smallest radix (fewer threads).  Forward order is
    descending, so the last forward radix -- whose outputs stay in registers
    across the spectrum product -- is the smallest."""
    best = None
    for f in factorizations(n):
        if threads_for(n, f) > MAX_THREADS:
            continue
        key = (len(f), max(f), -min(f))
        if best is None or key < best[0]:
            best = (key, f)
    if best is None:
        raise ValueError(f"no radix plan for {n}")
    return tuple(sorted(best[1], reverse=True))


TUNED_JSON = os.path.join(HERE, "tuned_plans.json")


def tuned_json_path() -> str:
    """The measured plans: the file named by $LP_TUNE_CACHE when set (same
    form, e.g. plans re-measured on another GPU), else tuned_plans.json
    beside this file."""
    return os.environ.get("LP_TUNE_CACHE") or TUNED_JSON


def plan_table_entry(n: int) -> dict:
    """Heuristic plan of one length (used when the autotuner has not
    measured it)."""
    r = choose_plan(n)
    t = threads_for(n, r)
    smem = 8 * (n + n // 16 + 16)   # upper bound of the padded extent
    if smem > SMEM_LIMIT:
        raise ValueError(f"length {n} needs {smem} bytes of shared memory")

    def fits(f: int) -> bool:
        return f * t <= MAX_THREADS and f * smem <= 100 * 1024

    # transforms per block of the one-unit-per-block row kernels: two when
    # they fit (32-byte column segments in T and U), one otherwise; more for
    # tiny lengths
    f = 1
    for cand in (8, 4, 2):
        if fits(cand) and (cand <= 2 or cand * t <= 256):
            f = cand
            break
    return dict(radices=list(r), threads=t, f1=f, f3=f, smem=smem,
                upb=[PF_UNITS] * 3, minb=[1, 1, 1], kstage=True, tt=0, pf=[1, 1, 1], db=[0, 0, 0],
                batch=True)


def plan_table() -> Dict[int, dict]:
    """Plan of every supported length: the autotuner's measured choice from
    tuned_plans.json where there is one, the heuristic otherwise."""
    tuned = {}
    path = tuned_json_path()
    if os.path.exists(path):
        with open(path) as fh:
            tuned = json.load(fh)
    table = {}
    for n in SIZES:
        e = plan_table_entry(n)
        t = tuned.get(str(n))
        if t:
            e.update(radices=list(t["radices"]), threads=threads_for(n, t["radices"]),
                     upb=list(t["upb"]), minb=list(t["minb"]), kstage=bool(t["kstage"]),
                     tt=int(t.get("tt", 0)), pf=list(t.get("pf", [1, 1, 1])),
                     db=list(t.get("db", [0, 0, 0])), batch=bool(t.get("batch", True)),
                     kst2=bool(t.get("kst2", False)), packed=bool(t.get("packed", False)),
                     late=list(t.get("late", DEFAULT_LATE)))
            if e["tt"]:
                e["threads"] = e["tt"]
        table[n] = e
    return table


_SIZE_TU = """// generated by paper_1907_02891_gb300/build.py -- one supported FFT length
// packed FP32x2 complex arithmetic in this length's DFTs
#define LP_PACKED_FP32 {packed}
#include "conv_kernels.cuh"
#include "lp_internal.h"
#include "tc_kernels.cuh"

namespace lpk {{
namespace {{
constexpr int kN = {n};
using P = Plan<kN, Seq<{seq}>, {tt}>;   // threads per transform (0 = one butterfly each)
constexpr int kF1 = {f1}, kF3 = {f3};
constexpr int kSmem = P::SMEM_BYTES;
constexpr long long kMaxSmem = 227 * 1024;
// tuned parameters of the prefetching kernels: work units per block and
// minimum resident blocks per SM (register cap) per pass; spectrum staging
constexpr int kUPB1 = {upb1}, kUPB2 = {upb2}, kUPB3 = {upb3};
constexpr int kMINB1 = {minb1}, kMINB2 = {minb2}, kMINB3 = {minb3};
constexpr bool kKSTAGE = {kstage};
constexpr bool kPF1 = {pf1}, kPF2 = {pf2}, kPF3 = {pf3};   // prefetching form allowed per pass
constexpr bool kDB1 = {db1}, kDB2 = {db2}, kDB3 = {db3};   // double-buffered exchange per pass
// forward row pass / one-spectrum column pass: the next kernel launches as
// this one's blocks exit instead of once they have all started
constexpr bool kLATE1 = {late1}, kLATE2 = {late2};
// several spectra: the batched column kernel (forward column parked in global
// memory, one product + inverse per spectrum) or one single-spectrum pass per
// spectrum (forward transform repeated)
constexpr bool kBatch = {batch};
// the batched column kernel parks its forward column in shared memory where
// it fits next to the exchange buffer, else in global memory
constexpr bool kParkG = P::SMEM_BYTES + 8 * kN > kMaxSmem;
constexpr int kSmemM = kParkG ? kSmem : kSmem + 8 * kN;
constexpr int kX1 = kDB1 ? 2 : 1, kX2 = kDB2 ? 2 : 1, kX3 = kDB3 ? 2 : 1;
// one-unit-per-block column kernel: spectrum column staged in shared memory
// (where the staging fits next to the exchange buffer)
constexpr bool kKST2 = {kst2};
constexpr bool kKstOk(bool kreal)
{{
    return kKST2 && (long long)kX2 * kSmem + (kreal ? 4 : 8) * ((kN + 3) / 4 * 4) <= kMaxSmem;
}}
constexpr int kKst(bool kreal) {{ return kKstOk(kreal) ? (kreal ? 4 : 8) * ((kN + 3) / 4 * 4) : 0; }}
// split-precision tensor-core column pass (0 shared bytes: not available)
using TP = TcPlan<P, kN>;
constexpr bool kTC = TP::FITS;
constexpr int kTcSmem = kTC ? TP::SMEM_BYTES : 0;

template <class K>
cudaError_t attr(K k, int bytes)
{{
    return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}}

// blocks of a prefetching launch: each block takes upb units
inline int persistent_grid(int units, int upb) {{ return (units + upb - 1) / upb; }}

cudaError_t set_attrs()
{{
    cudaError_t e;
    if ((e = attr(p1_rows<P, kN, kF1, kLATE1>, kF1 * kSmem)) != cudaSuccess) return e;
    if ((e = attr(p2_cols<P, kN, true, false, kMINB2, kDB2, kKstOk(true), false, kLATE2>, kX2 * kSmem + kKst(true))) != cudaSuccess) return e;
    if ((e = attr(p2_cols<P, kN, false, false, kMINB2, kDB2, kKstOk(false), false, kLATE2>, kX2 * kSmem + kKst(false))) != cudaSuccess) return e;
    if ((e = attr(p2_cols<P, kN, true, true, 1, false, false, kParkG>, kSmemM)) != cudaSuccess) return e;
    if ((e = attr(p2_cols<P, kN, false, true, 1, false, false, kParkG>, kSmemM)) != cudaSuccess) return e;
    if ((e = attr(p2_multiclass<P, kN, true>, kSmem)) != cudaSuccess) return e;
    if ((e = attr(p2_multiclass<P, kN, false>, kSmem)) != cudaSuccess) return e;
    if ((e = attr(p3_rows<P, kN, kF3>, kF3 * kSmem)) != cudaSuccess) return e;
    if constexpr (kTC) {{
        if ((e = attr(p2_cols_tc<P, kN, true>, kTcSmem)) != cudaSuccess) return e;
        if ((e = attr(p2_cols_tc<P, kN, false>, kTcSmem)) != cudaSuccess) return e;
    }}
    if ((e = attr(p1_rows_pf<P, kN, kUPB1, kMINB1, kDB1, kLATE1>, (int)kMaxSmem)) != cudaSuccess) return e;
    if ((e = attr(p2_cols_pf<P, kN, true, kUPB2, kMINB2, kKSTAGE, kDB2, kLATE2>, (int)kMaxSmem)) != cudaSuccess) return e;
    if ((e = attr(p2_cols_pf<P, kN, false, kUPB2, kMINB2, kKSTAGE, kDB2, kLATE2>, (int)kMaxSmem)) != cudaSuccess) return e;
    return attr(p3_rows_pf<P, kN, kUPB3, kMINB3, kDB3>, (int)kMaxSmem);
}}

cudaError_t p1(const P1Args& a, cudaStream_t s)
{{
    const long long sm = kX1 * kSmem + p1_stage_bytes(a.Wst);
    if (kPF1 && sm <= kMaxSmem)
        return launch_pdl(p1_rows_pf<P, kN, kUPB1, kMINB1, kDB1, kLATE1>, dim3(persistent_grid(a.npairs - a.pair0, kUPB1)),
                          dim3(P::T), sm, s, a);
    return launch_pdl(p1_rows<P, kN, kF1, kLATE1>, dim3((a.npairs - a.pair0 + kF1 - 1) / kF1), dim3(P::T * kF1),
                      kF1 * kSmem, s, a);
}}

cudaError_t p2(const P2Args& a, bool kreal, cudaStream_t s)
{{
    const bool multi = a.nspec > 1;
    const long long sm = kX2 * kSmem + p2_stage_bytes(a.ldT, a.ldK, kreal, kKSTAGE);
    if (!multi) {{
        const dim3 gpf(persistent_grid(a.ncols, kUPB2));
        if (kPF2 && sm <= kMaxSmem)
            return kreal ? launch_pdl(p2_cols_pf<P, kN, true, kUPB2, kMINB2, kKSTAGE, kDB2, kLATE2>, gpf, dim3(P::T), sm, s, a)
                         : launch_pdl(p2_cols_pf<P, kN, false, kUPB2, kMINB2, kKSTAGE, kDB2, kLATE2>, gpf, dim3(P::T), sm, s, a);
        return kreal ? launch_pdl(p2_cols<P, kN, true, false, kMINB2, kDB2, kKstOk(true), false, kLATE2>, dim3(a.ncols), dim3(P::T),
                                  kX2 * kSmem + kKst(true), s, a)
                     : launch_pdl(p2_cols<P, kN, false, false, kMINB2, kDB2, kKstOk(false), false, kLATE2>, dim3(a.ncols), dim3(P::T),
                                  kX2 * kSmem + kKst(false), s, a);
    }}
    if (kBatch && (!kParkG || a.park)) {{
        return kreal ? launch_pdl(p2_cols<P, kN, true, true, 1, false, false, kParkG>, dim3(a.ncols), dim3(P::T), kSmemM, s, a)
                     : launch_pdl(p2_cols<P, kN, false, true, 1, false, false, kParkG>, dim3(a.ncols), dim3(P::T), kSmemM, s, a);
    }} else {{
        // one single-spectrum pass per spectrum (no room to park the forward
        // column, or the plan measured this faster)
        for (int i = 0; i < a.nspec; ++i) {{
            P2Args b = a;
            b.K[0] = a.K[i];
            b.nspec = 1;
            b.U = a.U + (long long)i * a.specU;
            b.u_elems = a.u_elems - (long long)i * a.specU;
            cudaError_t e = p2(b, kreal, s);
            if (e != cudaSuccess) return e;
        }}
        return cudaSuccess;
    }}
}}

cudaError_t p2m(const P2MArgs& a, bool kreal, cudaStream_t s)
{{
    return kreal ? launch_pdl(p2_multiclass<P, kN, true>, dim3(a.ncols), dim3(P::T), kSmem, s, a)
                 : launch_pdl(p2_multiclass<P, kN, false>, dim3(a.ncols), dim3(P::T), kSmem, s, a);
}}

// persistent grid of the tensor-core column pass: resident blocks per SM
// (registers, shared memory, threads, TMEM columns) times the SMs, computed
// once, for the device of the first launch (a different GPU model in the
// same process would only get a less fitting grid, never a wrong result)
template <bool KREAL>
int tc_grid(int ncols)
{{
    static int cap = 0;
    if (cap == 0) {{
        int dev = 0, sms = 0, smem_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        cudaFuncAttributes fa{{}};
        cudaFuncGetAttributes(&fa, p2_cols_tc<P, kN, KREAL>);
        const int warps = TP::THREADS / 32;
        const int regs_warp = (fa.numRegs * 32 + 255) / 256 * 256;
        int occ = regs_warp > 0 ? 65536 / (regs_warp * warps) : 1;
        const int by_smem = smem_sm / (kTcSmem + 1024);
        const int by_thr = 2048 / TP::THREADS;
        const int by_tmem = 512 / TP::TMEM_COLS;
        occ = occ < by_smem ? occ : by_smem;
        occ = occ < by_thr ? occ : by_thr;
        occ = occ < by_tmem ? occ : by_tmem;
        cap = (occ < 1 ? 1 : occ) * sms;
    }}
    return ncols < cap ? ncols : cap;
}}

cudaError_t p2tc(const P2TcArgs& a, bool kreal, cudaStream_t s)
{{
    if constexpr (kTC) {{
        return kreal ? launch_pdl(p2_cols_tc<P, kN, true>, dim3(tc_grid<true>(a.a.ncols)), dim3(TP::THREADS), kTcSmem, s, a)
                     : launch_pdl(p2_cols_tc<P, kN, false>, dim3(tc_grid<false>(a.a.ncols)), dim3(TP::THREADS), kTcSmem, s, a);
    }} else {{
        return cudaErrorNotSupported;
    }}
}}

cudaError_t p3(const P3Args& a, int nspec, cudaStream_t s)
{{
    const long long sm = kX3 * kSmem + p3_stage_bytes(a.ncols);
    if (kPF3 && sm <= kMaxSmem)
        return launch_pdl(p3_rows_pf<P, kN, kUPB3, kMINB3, kDB3>, dim3(persistent_grid(a.npairs - a.pair0, kUPB3), nspec),
                          dim3(P::T), sm, s, a);
    return launch_pdl(p3_rows<P, kN, kF3>, dim3((a.npairs - a.pair0 + kF3 - 1) / kF3, nspec), dim3(P::T * kF3),
                      kF3 * kSmem, s, a);
}}
}}  // namespace

extern const SizeKernels kSize_{n} = {{kN, {ns}, {{{rad6}}}, P::T, kF1, kF3, kSmem, kBatch ? 1 : 0,
                                       set_attrs, p1, p2, p2m, p3,
                                       kTC ? TP::THREADS : 0, kTcSmem, p2tc}};
}}  // namespace lpk
"""

_REGISTRY_TU = """// generated by paper_1907_02891_gb300/build.py -- table of supported lengths
#include "lp_internal.h"

namespace lpk {{
{decls}
const SizeKernels* const kAllSizes[] = {{{ptrs}}};
const int kNumSizes = {count};
}}  // namespace lpk
"""


def _b(x) -> str:
    return "true" if x else "false"


def _write_if_changed(path: str, text: str) -> None:
    if os.path.exists(path):
        with open(path) as fh:
            if fh.read() == text:
                return
    with open(path, "w") as fh:
        fh.write(text)


def generate(sizes: Sequence[int] = ()) -> List[str]:
    """Write one translation unit per supported length (all, or `sizes`)
    and the registry of the lengths written; returns their paths.  A
    subset goes to its own directory, so that it never replaces the
    registry of the full build."""
    table = plan_table()
    gen = GEN
    if sizes:
        table = {n: table[n] for n in sorted(set(sizes))}
        gen = os.path.join(OUT, "gen_" + "_".join(map(str, table)))
    os.makedirs(gen, exist_ok=True)
    files = []
    for n, p in table.items():
        r = list(p["radices"])
        text = _SIZE_TU.format(n=n, seq=", ".join(map(str, r)), f1=p["f1"], f3=p["f3"], ns=len(r),
                               tt=p.get("tt", 0),
                               upb1=p["upb"][0], upb2=p["upb"][1], upb3=p["upb"][2],
                               minb1=p["minb"][0], minb2=p["minb"][1], minb3=p["minb"][2],
                               kstage="true" if p["kstage"] else "false",
                               pf1=_b(p["pf"][0]), pf2=_b(p["pf"][1]), pf3=_b(p["pf"][2]),
                               db1=_b(p["db"][0]), db2=_b(p["db"][1]), db3=_b(p["db"][2]),
                               batch=_b(p.get("batch", True)),
                               kst2=_b(p.get("kst2", False)), packed=int(bool(p.get("packed", False))),
                               late1=_b(p.get("late", DEFAULT_LATE)[0]), late2=_b(p.get("late", DEFAULT_LATE)[1]),
                               rad6=", ".join(map(str, r + [0] * (6 - len(r)))))
        path = os.path.join(gen, f"size_{n}.cu")
        _write_if_changed(path, text)
        files.append(path)
    decls = "\n".join(f"extern const SizeKernels kSize_{n};" for n in table)
    ptrs = ", ".join(f"&kSize_{n}" for n in table)
    path = os.path.join(gen, "registry.cu")
    _write_if_changed(path, _REGISTRY_TU.format(decls=decls, ptrs=ptrs, count=len(table)))
    files.append(path)
    return files


def _headers() -> List[str]:
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    hs.append(os.path.join(ROOT, "include", "lp.h"))
    return hs


def _compile(src: str, deps_mtime: float, debug: bool = False) -> str:
    name = os.path.splitext(os.path.basename(src))[0]
    digest = hashlib.sha1(src.encode()).hexdigest()[:8]
    obj = os.path.join(DEBUG_OBJ if debug else OBJ, f"{name}_{digest}.o")
    if os.path.exists(obj) and os.path.getmtime(obj) >= max(os.path.getmtime(src), deps_mtime):
        return obj
    cmd = ["nvcc", *ARCH, *NVCC_FLAGS, *(["-DLP_DEBUG=1"] if debug else []), "-I", CSRC,
           "-I", os.path.join(ROOT, "include"), "-c", src, "-o", obj + ".tmp"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    os.replace(obj + ".tmp", obj)
    return obj


def build(jobs: int = 0, verbose: bool = False, debug: bool = False, sizes: Sequence[int] = ()) -> str:
    """Compile every CUDA/C++ source of the library for sm_103a and link
    liblp.so (with debug, the bounds-checked library DEBUG_LIB, optionally
    with only the FFT lengths `sizes`).  Returns the library path."""
    if sizes and not debug:
        raise ValueError("a subset of lengths is for the debug build only")
    if shutil.which("nvcc") is None:
        raise RuntimeError("nvcc not found on PATH")
    obj_dir, lib = (DEBUG_OBJ, DEBUG_LIB) if debug else (OBJ, LIB)
    os.makedirs(obj_dir, exist_ok=True)
    gen = generate(sizes)
    srcs = [os.path.join(CSRC, f) for f in sorted(os.listdir(CSRC)) if f.endswith((".cu", ".cpp"))]
    srcs += gen
    deps = max(os.path.getmtime(h) for h in _headers() + [os.path.abspath(__file__)])
    jobs = jobs or max(1, os.cpu_count() or 1)
    with cf.ThreadPoolExecutor(jobs) as ex:
        objs = list(ex.map(lambda s: _compile(s, deps, debug), srcs))
    # relink when an object is newer or the set of objects differs (a debug
    # build of another subset of lengths)
    manifest = lib + ".objs"
    listed = open(manifest).read() if os.path.exists(manifest) else ""
    if (not os.path.exists(lib) or listed != "\n".join(objs) or
            os.path.getmtime(lib) < max(os.path.getmtime(o) for o in objs)):
        tmp = lib + f".tmp{os.getpid()}"
        cmd = ["nvcc", *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, lib)
        with open(manifest, "w") as fh:
            fh.write("\n".join(objs))
    if verbose:
        print(lib)
    return lib


if __name__ == "__main__":
    build(verbose=True, debug="--debug" in sys.argv[1:])
    sys.exit(0)
