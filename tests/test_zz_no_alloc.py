"""The allocation-free map entry point, against lp_map.

lp_map_noalloc exists for callers that cannot let the library call
cudaMalloc while they run (a host framework owning all device memory through
its own pool, or a latency-bound loop): it keeps its scratch in a static
device array.  This file is collected last so that a failure here cannot
hide the rest of the suite; it passes alone in a fresh process and after the
other tests.
"""

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1907_02891_gb300 import lp  # noqa: E402

TOL_FP32 = 1e-5


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
