"""The allocation-free map entry point, against lp_map.

lp_map_noalloc exists for callers that cannot let the library call
cudaMalloc while they run (a host framework owning all device memory through
its own pool, or a latency-bound loop): it keeps its scratch in a static
device array.  This file is collected last so that a failure here cannot
hide the rest of the suite; it passes alone in a fresh process and after the
other tests.
"""

import gc

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1907_02891_gb300 import lp  # noqa: E402

TOL_FP32 = 1e-5
TOL_SPLIT = 2e-4


def _rel(a, b):
    a = a.double()
    b = b.double()
    return float((a - b).abs().max() / b.abs().max())


def test_noalloc_matches_lp_map_on_two_calls_in_a_row():
    dev = torch.device("cuda:0")
    ctx = lp.lp_create(0)
    try:
        g = np.random.default_rng(21)
        # two different maps and PSF sets, so the second call runs on the
        # scratch contents the first call left behind
        cases = []
        for seed, (h, w), psfs in [(1, (256, 256), [(0.25, 1.25, 40.0)]),
                                   (2, (300, 211), [(0.1, 1.25, 80.0), (0.1, 2.0, 40.0)])]:
            L = synth.radiance_map(h, w, 8, seed, lit_fraction=0.02)
            Ks = [synth.psf_power_exp(101, 1.0, a, p, lam) for (a, p, lam) in psfs]
            Ks.append(g.uniform(0.0, 1.0, (101, 101)))            # complex spectrum too
            cases.append((L, Ks))
        for L, Ks in cases:
            h, w = L.shape
            Ld = torch.from_numpy(L).to(dev)
            specs = [lp.lp_kernel_spectrum(ctx, torch.from_numpy(K).to(dev), max_h=h, max_w=w)
                     for K in Ks]
            ws = lp.lp_map_workspace_bytes(h, w, *[lp.lp_spectrum_info(specs[0])[k] for k in ("ny", "nx", "hk", "wk")], len(Ks))
            assert ws <= lp.lp_map_noalloc_scratch_bytes()
            ref = [torch.empty((h, w), dtype=torch.float32, device=dev) for _ in Ks]
            got = [torch.full((h, w), float("nan"), dtype=torch.float32, device=dev) for _ in Ks]
            lp.lp_map(ctx, Ld, specs, ref)
            lp.lp_map_noalloc(ctx, Ld, specs, got)
            lp.lp_sync_status(ctx)
            for a, b in zip(got, ref):
                assert torch.isfinite(a).all()
                assert _rel(a, b) <= TOL_FP32
            for s in specs:
                lp.lp_spectrum_release(ctx, s)
    finally:
        lp.lp_destroy(ctx)


def test_noalloc_rejects_maps_beyond_its_scratch():
    dev = torch.device("cuda:0")
    ctx = lp.lp_create(0)
    try:
        K = torch.from_numpy(synth.psf_power_exp(541, 0.742, 0.1, 1.25, 80.0)).to(dev)
        s = lp.lp_kernel_spectrum(ctx, K, max_h=4096, max_w=4096)
        L = torch.zeros((4096, 4096), dtype=torch.float32, device=dev)
        out = torch.empty_like(L)
        with pytest.raises(lp.LpError) as e:
            lp.lp_map_noalloc(ctx, L, [s], [out])
        assert e.value.status == lp.LP_ERR_INVALID
        assert "static scratch" in str(e.value)
        lp.lp_spectrum_release(ctx, s)
    finally:
        lp.lp_destroy(ctx)


def _maps_and_specs(ctx, L, Ks, prec=0, pad=None):
    h, w = L.shape
    if pad is None:
        return [lp.lp_kernel_spectrum(ctx, torch.from_numpy(K).to("cuda:0"), max_h=h, max_w=w, prec=prec)
                for K in Ks]
    return [lp.lp_kernel_spectrum(ctx, torch.from_numpy(K).to("cuda:0"), pad_ny=pad[0], pad_nx=pad[1],
                                  prec=prec) for K in Ks]


def test_noalloc_allocates_nothing_on_a_fresh_stream():
    """The first map of a fresh context, on a fresh stream, through the
    no-alloc entry point: no context memory, no torch memory and no device
    memory change across the call (a fallback to the per-stream workspace
    would allocate ~18 MB here), and the result equals lp_map's."""
    dev = torch.device("cuda:0")
    L = synth.radiance_map(1024, 1024, 60, 31, lit_fraction=0.02)
    Ks = [synth.psf_power_exp(101, 0.742, 0.1, p, 80.0) for p in (1.0, 1.25, 2.0)]
    # load every kernel and the scratch array's module once, on another context
    warm = lp.lp_create(0)
    try:
        specs = _maps_and_specs(warm, L, Ks)
        o = [torch.empty((1024, 1024), device=dev) for _ in Ks]
        lp.lp_map(warm, torch.from_numpy(L).to(dev), specs, o)
        lp.lp_map_noalloc(warm, torch.from_numpy(L).to(dev), specs, o)
        lp.lp_sync_status(warm)
    finally:
        lp.lp_destroy(warm)
    ctx = lp.lp_create(0)
    try:
        specs = _maps_and_specs(ctx, L, Ks)
        Ld = torch.from_numpy(L).to(dev)
        got = [torch.full((1024, 1024), float("nan"), device=dev) for _ in Ks]
        ref = [torch.empty((1024, 1024), device=dev) for _ in Ks]
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            torch.zeros(1, device=dev).add_(1)     # the stream's first work, outside the check
        torch.cuda.synchronize()
        # no garbage collection inside the window: a collection there frees
        # tensors that earlier tests left in reference cycles, which moves
        # torch's counter without any allocation by the call
        gc.collect()
        gc.disable()
        try:
            before = (lp.lp_bytes_in_use(ctx), torch.cuda.memory_allocated(), torch.cuda.mem_get_info()[0])
            lp.lp_map_noalloc(ctx, Ld, specs, got, stream=s)
            lp.lp_sync_status(ctx, stream=s)
            after = (lp.lp_bytes_in_use(ctx), torch.cuda.memory_allocated(), torch.cuda.mem_get_info()[0])
        finally:
            gc.enable()
        assert before[0] == after[0], "context memory changed"
        assert before[1] == after[1], "torch memory changed"
        assert abs(before[2] - after[2]) < (1 << 20), "device memory changed"
        lp.lp_map(ctx, Ld, specs, ref)
        lp.lp_sync_status(ctx)
        for a, b in zip(got, ref):
            assert torch.isfinite(a).all()
            assert _rel(a, b) <= TOL_FP32
    finally:
        lp.lp_destroy(ctx)


def test_noalloc_full_mode_odd_height_against_the_oracle():
    """FULL output (r0/c0 offsets) with an odd h (the zeroed padding row of
    the intermediate spectra), against lp_map and the FP64 oracle."""
    dev = torch.device("cuda:0")
    ctx = lp.lp_create(0)
    try:
        g = np.random.default_rng(22)
        L = g.lognormal(0.0, 1.0, (201, 150)).astype(np.float32)
        Ks = [synth.psf_power_exp(41, 1.0, 0.25, 1.25, 40.0), g.uniform(0.1, 1.0, (41, 41))]
        specs = _maps_and_specs(ctx, L, Ks)
        Ld = torch.from_numpy(L).to(dev)
        shape = lp.output_shape(201, 150, 41, 41, lp.LP_OUT_FULL)
        for _ in range(2):
            got = [torch.full(shape, float("nan"), device=dev) for _ in Ks]
            ref = [torch.empty(shape, device=dev) for _ in Ks]
            lp.lp_map_noalloc(ctx, Ld, specs, got, mode=lp.LP_OUT_FULL)
            lp.lp_map(ctx, Ld, specs, ref, mode=lp.LP_OUT_FULL)
            lp.lp_sync_status(ctx)
            for a, b, K in zip(got, ref, Ks):
                assert _rel(a, b) <= TOL_FP32
                full = oracle.conv_full(L, K)
                err = np.max(np.abs(a.cpu().numpy().astype(np.float64) - full)) / np.max(np.abs(full))
                assert err <= TOL_FP32
    finally:
        lp.lp_destroy(ctx)


def test_noalloc_split_precision_against_the_oracle():
    """Split-BF16 spectra (one tensor-core column launch per spectrum into
    the static scratch), against lp_map and the FP64 oracle."""
    dev = torch.device("cuda:0")
    ctx = lp.lp_create(0)
    try:
        L = synth.radiance_map(300, 260, 12, 33, lit_fraction=0.02)
        g = np.random.default_rng(23)
        Ks = [synth.psf_power_exp(61, 1.0, 0.25, 1.25, 40.0), g.uniform(0.1, 1.0, (61, 61))]
        specs = _maps_and_specs(ctx, L, Ks, prec=lp.LP_PREC_SPLIT_BF16)
        Ld = torch.from_numpy(L).to(dev)
        for _ in range(2):
            got = [torch.full((300, 260), float("nan"), device=dev) for _ in Ks]
            ref = [torch.empty((300, 260), device=dev) for _ in Ks]
            lp.lp_map_noalloc(ctx, Ld, specs, got, prec=lp.LP_PREC_SPLIT_BF16)
            lp.lp_map(ctx, Ld, specs, ref, prec=lp.LP_PREC_SPLIT_BF16)
            lp.lp_sync_status(ctx)
            for a, b, K in zip(got, ref, Ks):
                assert _rel(a, b) <= TOL_FP32
                same = oracle.conv_same(L, K)
                err = np.max(np.abs(a.cpu().numpy().astype(np.float64) - same)) / np.max(np.abs(same))
                assert err <= TOL_SPLIT
    finally:
        lp.lp_destroy(ctx)


def test_noalloc_more_spectra_than_one_launch_takes():
    """33 spectra: more than one column launch takes (32), so the second
    chunk reuses the intermediate spectra's scratch."""
    dev = torch.device("cuda:0")
    ctx = lp.lp_create(0)
    try:
        g = np.random.default_rng(24)
        L = g.lognormal(0.0, 1.0, (96, 80)).astype(np.float32)
        Ks = [g.uniform(0.1, 1.0, (9, 9)) if k % 3 == 0 else synth.psf_power_exp(9, 1.0, 0.25, 1.0 + 0.03 * k, 40.0)
              for k in range(33)]
        specs = _maps_and_specs(ctx, L, Ks)
        Ld = torch.from_numpy(L).to(dev)
        for _ in range(2):
            got = [torch.full((96, 80), float("nan"), device=dev) for _ in Ks]
            ref = [torch.empty((96, 80), device=dev) for _ in Ks]
            lp.lp_map_noalloc(ctx, Ld, specs, got)
            lp.lp_map(ctx, Ld, specs, ref)
            lp.lp_sync_status(ctx)
            for a, b in zip(got, ref):
                assert _rel(a, b) <= TOL_FP32
        same = oracle.conv_same(L, Ks[32])
        err = np.max(np.abs(got[32].cpu().numpy().astype(np.float64) - same)) / np.max(np.abs(same))
        assert err <= TOL_FP32
    finally:
        lp.lp_destroy(ctx)
