"""ctypes wrapper of ``oracle.c`` (FP64 direct sums).  Test infrastructure only.

``build()`` compiles ``oracle.c`` with gcc + OpenMP into ``oracle/_build``.
The wrappers take numpy arrays: the radiance map L as float32 (H, W), the PSF
K as float64 (hk, wk) with odd sides and its centre at ((hk-1)/2, (wk-1)/2).
"""

from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lib = None

_i64 = ctypes.c_int64
_p = ctypes.c_void_p


def build(force: bool = False) -> str:
    """Compile the oracle (plain C, -O2, OpenMP).  Returns the .so path."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    # -ffp-contract=off keeps every product and sum a separately rounded
    # FP64 operation, in the loop order written in oracle.c.
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        lib.oracle_conv_points.argtypes = [_p, _i64, _i64, _i64, _p, _i64, _i64,
                                           _p, _p, _i64, _p]
        lib.oracle_conv_points.restype = ctypes.c_int
        lib.oracle_conv_full.argtypes = [_p, _i64, _i64, _i64, _p, _i64, _i64, _p]
        lib.oracle_conv_full.restype = ctypes.c_int
        lib.oracle_dft2_points.argtypes = [_p, _i64, _i64, _i64, _p, _p, _i64, _p, _p]
        lib.oracle_dft2_points.restype = ctypes.c_int
        lib.oracle_num_threads.argtypes = []
        lib.oracle_num_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def num_threads() -> int:
    """OpenMP threads the oracle uses."""
    return int(_load().oracle_num_threads())


def _prep(L, K):
    L = np.ascontiguousarray(L, dtype=np.float32)
    K = np.ascontiguousarray(K, dtype=np.float64)
    if L.ndim != 2 or K.ndim != 2:
        raise ValueError("L and K must be 2-D")
    return L, K


def conv_points_full(L, K, ii, jj) -> np.ndarray:
    """Bfull at full-grid coordinates (ii, jj), Eq. (7) discretised."""
    L, K = _prep(L, K)
    ii = np.ascontiguousarray(ii, dtype=np.int64).ravel()
    jj = np.ascontiguousarray(jj, dtype=np.int64).ravel()
    if ii.shape != jj.shape:
        raise ValueError("ii and jj differ in length")
    out = np.empty(ii.shape[0], dtype=np.float64)
    H, W = L.shape
    hk, wk = K.shape
    rc = _load().oracle_conv_points(L.ctypes.data, H, W, W, K.ctypes.data, hk, wk,
                                    ii.ctypes.data, jj.ctypes.data, ii.shape[0],
                                    out.ctypes.data)
    if rc != 0:
        raise ValueError("oracle_conv_points rejected its arguments")
    return out


def conv_full(L, K) -> np.ndarray:
    """Full linear convolution, (H+hk-1) x (W+wk-1), FP64."""
    L, K = _prep(L, K)
    H, W = L.shape
    hk, wk = K.shape
    out = np.empty((H + hk - 1, W + wk - 1), dtype=np.float64)
    rc = _load().oracle_conv_full(L.ctypes.data, H, W, W, K.ctypes.data, hk, wk,
                                  out.ctypes.data)
    if rc != 0:
        raise ValueError("oracle_conv_full rejected its arguments")
    return out


def _centre(K):
    hk, wk = K.shape
    if hk % 2 == 0 or wk % 2 == 0:
        raise ValueError("the PSF must have odd sides so that its centre is a pixel")
    return (hk - 1) // 2, (wk - 1) // 2


def conv_same(L, K) -> np.ndarray:
    """B[i][j] = Bfull[i+cy][j+cx]: the map region, observer on the source grid."""
    cy, cx = _centre(K)
    H, W = np.shape(L)
    return conv_full(L, K)[cy:cy + H, cx:cx + W]


def conv_points_same(L, K, ii, jj) -> np.ndarray:
    """B at map-grid pixels (ii, jj) of the cropped ("same") result."""
    cy, cx = _centre(K)
    return conv_points_full(L, K, np.asarray(ii) + cy, np.asarray(jj) + cx)


def conv_multiclass_points_same(Ls, Ks, ii, jj) -> np.ndarray:
    """Eq. (4): sum over source classes t of (K_t * L_t), at map pixels."""
    if len(Ls) != len(Ks) or len(Ls) == 0:
        raise ValueError("need one PSF per source class")
    acc = np.zeros(np.asarray(ii).size, dtype=np.float64)
    for L, K in zip(Ls, Ks):
        acc += conv_points_same(L, K, ii, jj)
    return acc


def dft2_points(f, kk, ll) -> np.ndarray:
    """Eq. (10) at 0-based frequencies (kk, ll); returns complex128."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    N, M = f.shape
    kk = np.ascontiguousarray(kk, dtype=np.int64).ravel()
    ll = np.ascontiguousarray(ll, dtype=np.int64).ravel()
    re = np.empty(kk.shape[0], dtype=np.float64)
    im = np.empty(kk.shape[0], dtype=np.float64)
    rc = _load().oracle_dft2_points(f.ctypes.data, N, M, M, kk.ctypes.data,
                                    ll.ctypes.data, kk.shape[0], re.ctypes.data,
                                    im.ctypes.data)
    if rc != 0:
        raise ValueError("oracle_dft2_points rejected its arguments")
    return re + 1j * im


def op_count_ratio(n_map: int, n_psf: int) -> float:
    """Direct-sum over FFT operation counts, the estimate printed after
    Eq. (10): N_L^2 N_K^2 / [(N_L + N_K)^2 log2 (N_L + N_K)^2]."""
    s = float(n_map + n_psf)
    return (n_map ** 2) * (n_psf ** 2) / (s * s * math.log2(s * s))
