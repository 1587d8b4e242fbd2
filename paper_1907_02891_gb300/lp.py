"""Thin ctypes binding of liblp.so (include/lp.h).

Argument marshalling only: every step of the map runs in the library's CUDA
kernels.  Functions keep the C names.  Device buffers are torch CUDA
tensors (their data_ptr is passed); streams are torch.cuda.Stream objects or
raw cudaStream_t integers (None = the current torch stream).  There is no
CPU fallback: if the compiled library is missing, loading fails loudly.
"""

from __future__ import annotations

import ctypes
import os
from typing import List, Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# $LP_DEBUG (not "" or "0") selects the bounds-checked debug build
# (build.build(debug=True)): every work unit of the passes checks its extents
# in every buffer first and reports a miss as bit 3 of the device status word
DEBUG_LIB_PATH = os.path.join(_HERE, "_build", "debug", "liblp.so")
LIB_PATH = (DEBUG_LIB_PATH if os.environ.get("LP_DEBUG", "") not in ("", "0")
            else os.path.join(_HERE, "_build", "liblp.so"))

LP_OK, LP_ERR_INVALID, LP_ERR_OOM, LP_ERR_CUDA, LP_ERR_TIMEOUT = 0, 1, 2, 3, 4
LP_ERR_UNSUPPORTED, LP_ERR_BUSY, LP_ERR_DEVICE, LP_ERR_CANCELLED = 5, 6, 7, 8
LP_PREC_FP32, LP_PREC_SPLIT_BF16, LP_PREC_SPLIT_FP16 = 0, 1, 2
LP_OUT_SAME, LP_OUT_FULL = 0, 1

STATUS_NAMES = {0: "LP_OK", 1: "LP_ERR_INVALID", 2: "LP_ERR_OOM", 3: "LP_ERR_CUDA",
                4: "LP_ERR_TIMEOUT", 5: "LP_ERR_UNSUPPORTED", 6: "LP_ERR_BUSY",
                7: "LP_ERR_DEVICE", 8: "LP_ERR_CANCELLED"}

# every entry point declared in include/lp.h
EXPORTS = (
    "lp_version", "lp_last_error", "lp_create", "lp_destroy", "lp_bytes_in_use",
    "lp_num_supported_sizes", "lp_supported_size_at", "lp_supported_size", "lp_split_supported",
    "lp_kernel_spectrum", "lp_spectrum_info", "lp_spectrum_copy", "lp_spectrum_release",
    "lp_map", "lp_map_host", "lp_map_multiclass", "lp_map_tiled", "lp_tiled_pad", "lp_map_workspace_bytes", "lp_sync_status",
    "lp_set_pass_timing", "lp_get_pass_timing", "lp_map_noalloc", "lp_map_noalloc_scratch_bytes",
    "lp_set_test_hook",
    "lp_serve_start", "lp_serve_submit", "lp_serve_poll", "lp_serve_stats", "lp_serve_stop",
    "lp_serve_log", "lp_serve_cancel",
)


class LpError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None
_vp = ctypes.c_void_p
_i = ctypes.c_int
_sz = ctypes.c_size_t


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load liblp.so (raises OSError when it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError(f"liblp.so not built at {path}: run paper_1907_02891_gb300.build.build()")
    lib = ctypes.CDLL(path)
    sig = {
        "lp_version": ([], _i),
        "lp_last_error": ([], ctypes.c_char_p),
        "lp_create": ([ctypes.POINTER(_vp), _i, _sz], _i),
        "lp_destroy": ([_vp], None),
        "lp_bytes_in_use": ([_vp], _sz),
        "lp_num_supported_sizes": ([], _i),
        "lp_supported_size_at": ([_i], _i),
        "lp_supported_size": ([_i], _i),
        "lp_split_supported": ([_i], _i),
        "lp_kernel_spectrum": ([_vp, _vp, _i, _i, _i, _i, _i, _i, _i, _vp, ctypes.POINTER(_vp)], _i),
        "lp_spectrum_info": ([_vp] + [ctypes.POINTER(_i)] * 5, _i),
        "lp_spectrum_copy": ([_vp, _vp, _sz, _vp], _i),
        "lp_spectrum_release": ([_vp, _vp], _i),
        "lp_map": ([_vp, _vp, _i, _i, _i, _vp, _i, _vp, _i, _i, _i, _vp], _i),
        "lp_map_host": ([_vp, _vp, _i, _i, _i, _vp, _i, _vp, _i, _i, _i, _vp], _i),
        "lp_map_tiled": ([_vp, _vp, _i, _i, _i, _vp, _i, _vp, _i, _i, _vp], _i),
        "lp_tiled_pad": ([_i, _i, _i, _i, _i, ctypes.POINTER(_i), ctypes.POINTER(_i)], _i),
        "lp_map_multiclass": ([_vp, _vp, _i, _i, _i, _i, _vp, _vp, _i, _i, _i, _vp], _i),
        "lp_map_workspace_bytes": ([_i, _i, _i, _i, _i, _i, _i, _i], _sz),
        "lp_sync_status": ([_vp, _vp, _i], _i),
        "lp_set_pass_timing": ([_vp, _i], _i),
        "lp_set_test_hook": ([_vp, _i], _i),
        "lp_map_noalloc": ([_vp, _vp, _i, _i, _i, _vp, _i, _vp, _i, _i, _i, _vp], _i),
        "lp_map_noalloc_scratch_bytes": ([], _sz),
        "lp_serve_start": ([_vp, _i], _i),
        "lp_serve_submit": ([_vp, _vp, _i, _i, _i, _vp, _i, _vp, _i, _i,
                             ctypes.POINTER(ctypes.c_uint64)], _i),
        "lp_serve_poll": ([_vp, ctypes.c_uint64, _i, ctypes.POINTER(ctypes.c_double)], _i),
        "lp_serve_stats": ([_vp, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64),
                            ctypes.POINTER(_i), ctypes.POINTER(_i)], _i),
        "lp_serve_stop": ([_vp], _i),
        "lp_serve_log": ([_vp, ctypes.c_char_p], _i),
        "lp_serve_cancel": ([_vp, ctypes.c_uint64], _i),
        "lp_get_pass_timing": ([_vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_i)], _i),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def _check(st: int, where: str) -> None:
    if st != LP_OK:
        msg = load_library().lp_last_error()
        raise LpError(st, where, msg.decode() if msg else "")


def _stream_handle(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _ptr_array(ptrs: Sequence[int]):
    return (_vp * len(ptrs))(*ptrs)


# --------------------------------------------------------------------------
# entry points (same names as the C ABI)
# --------------------------------------------------------------------------

def lp_version() -> int:
    return load_library().lp_version()


def lp_num_supported_sizes() -> int:
    return load_library().lp_num_supported_sizes()


def lp_supported_size_at(i: int) -> int:
    return load_library().lp_supported_size_at(i)


def lp_supported_size(n: int) -> int:
    return load_library().lp_supported_size(n)


def lp_split_supported(n: int) -> bool:
    """True if length n has the split-BF16 tensor-core column pass."""
    return bool(load_library().lp_split_supported(n))


def supported_sizes() -> List[int]:
    return [lp_supported_size_at(i) for i in range(lp_num_supported_sizes())]


def lp_create(device: int = 0, hbm_budget_bytes: int = 0) -> int:
    ctx = _vp()
    _check(load_library().lp_create(ctypes.byref(ctx), device, hbm_budget_bytes), "lp_create")
    return ctx.value


def lp_destroy(ctx: int) -> None:
    load_library().lp_destroy(ctx)


def lp_bytes_in_use(ctx: int) -> int:
    return load_library().lp_bytes_in_use(ctx)


def lp_kernel_spectrum(ctx: int, K, max_h: int = 0, max_w: int = 0, pad_ny: int = 0,
                       pad_nx: int = 0, prec: int = LP_PREC_FP32, stream=None) -> int:
    """K: CUDA float64 tensor (hk, wk), contiguous."""
    if not (K.is_cuda and K.dtype.is_floating_point and K.element_size() == 8 and K.is_contiguous()):
        raise ValueError("K must be a contiguous CUDA float64 tensor")
    hk, wk = K.shape
    spec = _vp()
    _check(load_library().lp_kernel_spectrum(ctx, K.data_ptr(), hk, wk, max_h, max_w, pad_ny,
                                             pad_nx, prec, _stream_handle(stream),
                                             ctypes.byref(spec)), "lp_kernel_spectrum")
    return spec.value


def lp_spectrum_info(spec: int) -> dict:
    v = [_i() for _ in range(5)]
    _check(load_library().lp_spectrum_info(spec, *[ctypes.byref(x) for x in v]), "lp_spectrum_info")
    ny, nx, hk, wk, real = (x.value for x in v)
    return dict(ny=ny, nx=nx, hk=hk, wk=wk, is_real=bool(real))


def lp_spectrum_copy(spec: int, dst, stream=None) -> None:
    """dst: CUDA float32 tensor with >= (nx/2+1)*ny*(1 or 2) elements."""
    _check(load_library().lp_spectrum_copy(spec, dst.data_ptr(), dst.numel(),
                                           _stream_handle(stream)), "lp_spectrum_copy")


def lp_spectrum_release(ctx: int, spec: int) -> None:
    _check(load_library().lp_spectrum_release(ctx, spec), "lp_spectrum_release")


def output_shape(h: int, w: int, hk: int, wk: int, mode: int) -> tuple:
    return (h + hk - 1, w + wk - 1) if mode == LP_OUT_FULL else (h, w)


def lp_map(ctx: int, L, spectra: Sequence[int], out: Sequence, mode: int = LP_OUT_SAME,
           prec: int = LP_PREC_FP32, stream=None) -> None:
    """L: CUDA float32 2-D tensor (row stride = ldl); out: CUDA float32 2-D
    tensors with unit column stride (row stride = ldo, equal for all)."""
    h, w = L.shape
    if L.stride(1) != 1 or any(o.stride(1) != 1 for o in out):
        raise ValueError("rows must be contiguous")
    ldo = out[0].stride(0)
    if any(o.stride(0) != ldo for o in out):
        raise ValueError("all outputs need the same row stride")
    _check(load_library().lp_map(ctx, L.data_ptr(), h, w, L.stride(0), _ptr_array(spectra),
                                 len(spectra), _ptr_array([o.data_ptr() for o in out]), ldo,
                                 mode, prec, _stream_handle(stream)), "lp_map")


def lp_map_tiled(ctx: int, L, spectra: Sequence[int], out: Sequence, prec: int = LP_PREC_FP32,
                 stream=None) -> None:
    """SAME-mode map of any size in overlap-save tiles of (Ny - hk + 1) x
    (Nx - wk + 1) output pixels; tensors as lp_map."""
    h, w = L.shape
    if L.stride(1) != 1 or any(o.stride(1) != 1 for o in out):
        raise ValueError("rows must be contiguous")
    ldo = out[0].stride(0)
    if any(o.stride(0) != ldo for o in out):
        raise ValueError("all outputs need the same row stride")
    _check(load_library().lp_map_tiled(ctx, L.data_ptr(), h, w, L.stride(0), _ptr_array(spectra),
                                       len(spectra), _ptr_array([o.data_ptr() for o in out]), ldo,
                                       prec, _stream_handle(stream)), "lp_map_tiled")


def lp_tiled_pad(h: int, w: int, hk: int, wk: int, prec: int = LP_PREC_FP32):
    """(pad_ny, pad_nx) that lp_map_tiled maps an h x w map with the fewest
    transformed points (host only)."""
    ny, nx = _i(), _i()
    _check(load_library().lp_tiled_pad(h, w, hk, wk, prec, ctypes.byref(ny), ctypes.byref(nx)), "lp_tiled_pad")
    return ny.value, nx.value


def lp_map_host(ctx: int, L: np.ndarray, spectra: Sequence[int], out: Sequence[np.ndarray],
                mode: int = LP_OUT_SAME, prec: int = LP_PREC_FP32, stream=None) -> None:
    """Host (numpy float32 or pinned CPU torch) buffers; asynchronous on the
    stream -- call lp_sync_status before reading out."""
    def ptr_ld(a):
        if isinstance(a, np.ndarray):
            if a.dtype != np.float32 or a.strides[1] != 4:
                raise ValueError("host arrays must be float32 with contiguous rows")
            return a.ctypes.data, a.strides[0] // 4
        return a.data_ptr(), a.stride(0)
    lp_, ldl = ptr_ld(L)
    h, w = L.shape
    outs = [ptr_ld(o) for o in out]
    ldo = outs[0][1]
    _check(load_library().lp_map_host(ctx, lp_, h, w, ldl, _ptr_array(spectra), len(spectra),
                                      _ptr_array([p for p, _ in outs]), ldo, mode, prec,
                                      _stream_handle(stream)), "lp_map_host")


def lp_map_multiclass(ctx: int, Ls: Sequence, spectra: Sequence[int], out,
                      mode: int = LP_OUT_SAME, prec: int = LP_PREC_FP32, stream=None) -> None:
    h, w = Ls[0].shape
    ldl = Ls[0].stride(0)
    if any(x.shape != (h, w) or x.stride(0) != ldl or x.stride(1) != 1 for x in Ls):
        raise ValueError("class maps must share shape and row stride")
    _check(load_library().lp_map_multiclass(ctx, _ptr_array([x.data_ptr() for x in Ls]), len(Ls),
                                            h, w, ldl, _ptr_array(spectra), out.data_ptr(),
                                            out.stride(0), mode, prec, _stream_handle(stream)),
           "lp_map_multiclass")


def lp_map_workspace_bytes(h, w, ny, nx, hk, wk, n, mode=LP_OUT_SAME) -> int:
    return load_library().lp_map_workspace_bytes(h, w, ny, nx, hk, wk, n, mode)


def lp_sync_status(ctx: int, stream=None, timeout_ms: int = 60000) -> None:
    _check(load_library().lp_sync_status(ctx, _stream_handle(stream), timeout_ms), "lp_sync_status")


def lp_sync_status_code(ctx: int, stream=None, timeout_ms: int = 60000) -> int:
    """Like lp_sync_status but returns the status instead of raising."""
    return load_library().lp_sync_status(ctx, _stream_handle(stream), timeout_ms)


def call_status(name: str, *args) -> int:
    """Raw call of an entry point returning its lp_status (for error tests)."""
    return getattr(load_library(), name)(*args)


PASS_NAMES = ("p1_rows", "p2_cols", "p3_rows")


LP_TEST_TC_NO_MMA = 1
LP_TEST_FP_COLLIDE = 2
LP_TEST_SERVE_FAIL = 4
LP_TEST_BOUNDS = 8


def lp_set_test_hook(ctx: int, hook: int) -> None:
    """Test hooks (failure-detection tests only); 0 clears them."""
    _check(load_library().lp_set_test_hook(ctx, hook), "lp_set_test_hook")


def lp_set_pass_timing(ctx: int, enable: bool) -> None:
    _check(load_library().lp_set_pass_timing(ctx, 1 if enable else 0), "lp_set_pass_timing")


def lp_get_pass_timing(ctx: int) -> dict:
    """{pass name: (total ms, launches)} since the last call; waits for them."""
    ms = (ctypes.c_double * 3)()
    n = (_i * 3)()
    _check(load_library().lp_get_pass_timing(ctx, ms, n), "lp_get_pass_timing")
    return {PASS_NAMES[i]: (ms[i], n[i]) for i in range(3)}


def lp_map_noalloc(ctx: int, L, spectra: Sequence[int], out: Sequence, mode: int = LP_OUT_SAME,
                   prec: int = LP_PREC_FP32, stream=None) -> None:
    """lp_map with its scratch in the library's static device array: for
    callers that cannot let the library allocate device memory while they
    run.  Same arguments as lp_map; maps whose workspace exceeds
    lp_map_noalloc_scratch_bytes() are rejected; concurrent calls race."""
    h, w = L.shape
    if L.stride(1) != 1 or any(o.stride(1) != 1 for o in out):
        raise ValueError("rows must be contiguous")
    ldo = out[0].stride(0)
    if any(o.stride(0) != ldo for o in out):
        raise ValueError("all outputs need the same row stride")
    _check(load_library().lp_map_noalloc(ctx, L.data_ptr(), h, w, L.stride(0),
                                         _ptr_array(spectra), len(spectra),
                                         _ptr_array([o.data_ptr() for o in out]), ldo, mode,
                                         prec, _stream_handle(stream)), "lp_map_noalloc")


def lp_map_noalloc_scratch_bytes() -> int:
    return load_library().lp_map_noalloc_scratch_bytes()


# --------------------------------------------------------------------------
# serving
# --------------------------------------------------------------------------

def lp_serve_start(ctx: int, n_slots: int = 4) -> None:
    _check(load_library().lp_serve_start(ctx, n_slots), "lp_serve_start")


def lp_serve_submit(ctx: int, L, spectra: Sequence[int], out: Sequence,
                    mode: int = LP_OUT_SAME) -> int:
    """Queue one map request (device tensors, as lp_map; the precision is the
    spectra's); returns its ticket.  Keep L and out alive until the ticket is
    polled (the request holds its own references on the spectra)."""
    h, w = L.shape
    ldo = out[0].stride(0)
    t = ctypes.c_uint64()
    _check(load_library().lp_serve_submit(ctx, L.data_ptr(), h, w, L.stride(0), _ptr_array(spectra),
                                          len(spectra), _ptr_array([o.data_ptr() for o in out]),
                                          ldo, mode, ctypes.byref(t)), "lp_serve_submit")
    return t.value


def lp_serve_poll(ctx: int, ticket: int, timeout_ms: int = -1):
    """Latency in ms when finished, None on timeout; raises on failure."""
    lat = ctypes.c_double()
    st = load_library().lp_serve_poll(ctx, ticket, timeout_ms, ctypes.byref(lat))
    if st == LP_ERR_TIMEOUT:
        return None
    _check(st, "lp_serve_poll")
    return lat.value


def lp_serve_stats(ctx: int) -> dict:
    c, f = ctypes.c_uint64(), ctypes.c_uint64()
    q, r = _i(), _i()
    _check(load_library().lp_serve_stats(ctx, ctypes.byref(c), ctypes.byref(f), ctypes.byref(q),
                                         ctypes.byref(r)), "lp_serve_stats")
    return dict(completed=c.value, failed=f.value, queued=q.value, running=r.value)


def lp_serve_log(ctx: int, path) -> None:
    """Append one JSON line per finished request to path (None: stop logging)."""
    _check(load_library().lp_serve_log(ctx, None if path is None else str(path).encode()), "lp_serve_log")


def lp_serve_cancel(ctx: int, ticket: int) -> None:
    """Cancel a queued request (raises LpError with LP_ERR_BUSY if it is
    already running or finished)."""
    _check(load_library().lp_serve_cancel(ctx, ticket), "lp_serve_cancel")


def lp_serve_stop(ctx: int) -> None:
    _check(load_library().lp_serve_stop(ctx), "lp_serve_stop")
