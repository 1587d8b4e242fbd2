"""Host-side checks of the C-ABI library: it loads, exports every entry point
declared in include/lp.h, and its size table and errors work without a GPU.
No compute call is made here."""

import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1907_02891_gb300 import build, lp
    if not os.path.exists(lp.LIB_PATH):
        build.build()
    return lp.load_library()


def _declared_symbols():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            with open(os.path.join(ROOT, "include", f)) as fh:
                text = fh.read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(lp_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_every_declared_symbol_is_exported(lib):
    from paper_1907_02891_gb300 import lp
    declared = _declared_symbols()
    assert len(declared) >= 15
    for name in declared:
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"
    assert set(lp.EXPORTS) <= set(declared)


def test_supported_sizes_cover_the_workloads(lib):
    from paper_1907_02891_gb300 import build, lp
    sizes = lp.supported_sizes()
    assert sizes == sorted(sizes) and len(sizes) == len(build.SIZES)
    for n in sizes:
        f = build.choose_plan(n)
        assert all(r in build.RADICES for r in f)
        p = 1
        for r in f:
            p *= r
        assert p == n
        m = n
        for q in (2, 3, 5, 7):
            while m % q == 0:
                m //= q
        assert m == 1, f"{n} is not 7-smooth"
    # padded sizes of the workloads: map + PSF - 1 -> smallest supported
    assert lp.lp_supported_size(356) == 360
    assert lp.lp_supported_size(4636) == 4704
    assert lp.lp_supported_size(8792) == 8820
    assert lp.lp_supported_size(17184) == 17280
    assert lp.lp_supported_size(10 ** 6) == -1
    assert lp.lp_supported_size_at(-1) == -1


def test_workspace_model(lib):
    from paper_1907_02891_gb300 import lp
    # T: 2354 x 4096 (2353 columns rounded up to whole 2-column blocks)
    # + U: 2356 x 4096 (whole 4-column blocks), complex64, + alignment slack
    b = lp.lp_map_workspace_bytes(4096, 4096, 4704, 4704, 541, 541, 1)
    assert b == 8 * (2354 * 4096 + 2356 * 4096) + 256
    assert lp.lp_map_workspace_bytes(0, 4096, 4704, 4704, 541, 541, 1) == 0


def test_no_gpu_errors_are_reported_not_raised(lib):
    import ctypes
    from paper_1907_02891_gb300 import lp
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    ctx = ctypes.c_void_p()
    st = lib.lp_create(ctypes.byref(ctx), 0, 0)
    assert st == lp.LP_ERR_CUDA and ctx.value is None
    assert b"no CUDA device" in lib.lp_last_error()
    assert lib.lp_create(None, 0, 0) == lp.LP_ERR_INVALID


def test_tiled_pad_minimises_transformed_points(lib):
    """lp_tiled_pad against a brute-force search of the size table: per
    dimension the length N >= k with the fewest points tiles * N over all
    tiles, one tile where n <= N - (k - 1) / 2, else ceil(n / (N - k + 1))
    (ties: fewer tiles); maps one transform holds get one tile at the SAME
    crop's padding."""
    from paper_1907_02891_gb300 import lp
    sizes = lp.supported_sizes()

    def brute(n, k, split=False):
        best = None
        for N in sizes:
            if N < k or (split and not lp.lp_split_supported(N)):
                continue
            tiles = 1 if n <= N - (k - 1) // 2 else -(-n // (N - k + 1))
            key = (tiles * N, tiles)
            if best is None or key < best[0]:
                best = (key, N)
        return best[1]

    for h, w, hk, wk in ((17800, 21000, 801, 801), (100000, 3000, 1485, 965), (300, 260, 31, 31),
                         (1, 1, 1, 1), (5000, 40000, 541, 1), (65, 65, 63, 63)):
        assert lp.lp_tiled_pad(h, w, hk, wk) == (brute(h, hk), brute(w, wk)), (h, w, hk, wk)
        assert lp.lp_tiled_pad(h, w, hk, wk, lp.LP_PREC_SPLIT_BF16)[0] == brute(h, hk, True)
    for side, k, n in ((256, 101, 320), (4096, 541, 4608), (8192, 601, 8640), (16384, 801, 17280)):
        assert n == lp.lp_supported_size(side + (k - 1) // 2)
        assert lp.lp_tiled_pad(side, side, k, k) == (n, n)
    for bad in ((0, 10, 3, 3), (10, 10, 4, 3), (10, 10, 3, -1)):
        with pytest.raises(lp.LpError):
            lp.lp_tiled_pad(*bad)
    with pytest.raises(lp.LpError):   # no supported length holds the PSF
        lp.lp_tiled_pad(10, 10, 2 * max(sizes) + 1, 3)


def test_debug_build_compiles_and_exports(lib):
    """The bounds-checked debug library (one length here) builds with the
    same toolchain and exports the same entry points."""
    import ctypes
    from paper_1907_02891_gb300 import build
    path = build.build(debug=True, sizes=(96,))
    assert path == build.DEBUG_LIB and os.path.exists(path)
    dl = ctypes.CDLL(path)
    for name in _declared_symbols():
        assert hasattr(dl, name), name
    dl.lp_num_supported_sizes.restype = ctypes.c_int
    dl.lp_supported_size_at.restype = ctypes.c_int
    assert dl.lp_num_supported_sizes() == 1 and dl.lp_supported_size_at(0) == 96
