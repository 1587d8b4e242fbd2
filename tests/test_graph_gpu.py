"""Maps captured into CUDA graphs.

A loop of small maps is launch-bound; captured into one graph it replays as
one launch.  The captured calls only enqueue kernels, so nothing runs until
the replay, and a replay after new data is written into the same input
buffers maps the new data.  Results are compared bitwise with the same maps
through uncaptured lp_map calls (the same kernels), and one with the FP64
oracle.
"""

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1907_02891_gb300 import lp  # noqa: E402

DEV = "cuda:0"
TOL_FP32 = 1e-5


@pytest.fixture(scope="module")
def ctx():
    c = lp.lp_create(0)
    yield c
    lp.lp_destroy(c)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _maps(n, side, seed):
    return [dev(synth.radiance_map(side, side, 12, seed + i, lit_fraction=0.05)) for i in range(n)]


def _uncaptured(ctx, Ls, spec):
    ref = [torch.empty_like(L) for L in Ls]
    for L, r in zip(Ls, ref):
        lp.lp_map(ctx, L, [spec], [r])
    lp.lp_sync_status(ctx)
    return ref


def test_noalloc_loop_replays_as_one_graph(ctx):
    wl = synth.WORKLOADS["map256_psf101"]
    K = wl.psfs()[0]
    spec = lp.lp_kernel_spectrum(ctx, dev(K), max_h=256, max_w=256)
    lp.lp_sync_status(ctx)
    Ls = _maps(16, 256, 1907_02891 + 70)
    outs = [torch.full((256, 256), float("nan"), device=DEV) for _ in Ls]
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):   # one uncaptured call first (scratch address, build seen complete)
        lp.lp_map_noalloc(ctx, Ls[0], [spec], [outs[0]])
    s.synchronize()
    outs[0].fill_(float("nan"))
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        for L, o in zip(Ls, outs):
            lp.lp_map_noalloc(ctx, L, [spec], [o])
    torch.cuda.synchronize()
    assert all(torch.isnan(o).all() for o in outs), "a captured call ran before the replay"
    g.replay()
    torch.cuda.synchronize()
    ref = _uncaptured(ctx, Ls, spec)
    for o, r in zip(outs, ref):
        assert torch.equal(o, r)
    Lh = Ls[3].cpu().numpy()
    B = outs[3].cpu().numpy().astype(np.float64)
    want = oracle.conv_same(Lh, K)
    assert np.max(np.abs(B - want)) / np.max(np.abs(want)) <= TOL_FP32
    # new data in the same buffers: the replay maps it
    for L, N in zip(Ls, _maps(16, 256, 1907_02891 + 90)):
        L.copy_(N)
    g.replay()
    torch.cuda.synchronize()
    for o, r in zip(outs, _uncaptured(ctx, Ls, spec)):
        assert torch.equal(o, r)
    lp.lp_spectrum_release(ctx, spec)


def test_lp_map_and_tiled_map_captured(ctx):
    """lp_map (its workspace sized by an uncaptured call) and the tiled map
    (20 tiles, 60 kernels) in one graph."""
    K = synth.psf_power_exp(31, 0.742, 0.1, 1.25, 80.0)
    L1 = dev(synth.radiance_map(300, 260, 20, 1907_02891 + 71, lit_fraction=0.05))
    L2 = dev(synth.radiance_map(180, 200, 10, 1907_02891 + 72, lit_fraction=0.05))
    tspec = lp.lp_kernel_spectrum(ctx, dev(K), pad_ny=96, pad_nx=96)
    mspec = lp.lp_kernel_spectrum(ctx, dev(K), max_h=180, max_w=200)
    lp.lp_sync_status(ctx)
    o1 = torch.full((300, 260), float("nan"), device=DEV)
    o2 = torch.full((180, 200), float("nan"), device=DEV)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        lp.lp_map_tiled(ctx, L1, [tspec], [o1])
        lp.lp_map(ctx, L2, [mspec], [o2])
    s.synchronize()
    o1.fill_(float("nan"))
    o2.fill_(float("nan"))
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        lp.lp_map_tiled(ctx, L1, [tspec], [o1])
        lp.lp_map(ctx, L2, [mspec], [o2])
    g.replay()
    torch.cuda.synchronize()
    for L, o in ((L1, o1), (L2, o2)):
        B = o.cpu().numpy().astype(np.float64)
        want = oracle.conv_same(L.cpu().numpy(), K)
        assert np.max(np.abs(B - want)) / np.max(np.abs(want)) <= TOL_FP32
    lp.lp_spectrum_release(ctx, tspec)
    lp.lp_spectrum_release(ctx, mspec)


def test_capture_refusals_leave_the_capture_usable(ctx):
    """A call that would allocate, or with pass timing on, is refused before
    it enqueues anything; the rest of the capture still replays correctly."""
    K = synth.psf_power_exp(31, 0.742, 0.1, 1.25, 80.0)
    spec = lp.lp_kernel_spectrum(ctx, dev(K), max_h=512, max_w=512)
    lp.lp_sync_status(ctx)
    small = dev(synth.radiance_map(64, 64, 4, 1907_02891 + 73, lit_fraction=0.05))
    big = dev(synth.radiance_map(512, 512, 12, 1907_02891 + 74, lit_fraction=0.05))
    o_small = torch.empty_like(small)
    o_big = torch.empty_like(big)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        lp.lp_map(ctx, small, [spec], [o_small])   # this stream's workspace: the small map only
    s.synchronize()
    errors = []
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        try:
            lp.lp_map(ctx, big, [spec], [o_big])
        except lp.LpError as e:
            errors.append(str(e))
        lp.lp_set_pass_timing(ctx, True)
        try:
            lp.lp_map_noalloc(ctx, small, [spec], [o_small])
        except lp.LpError as e:
            errors.append(str(e))
        lp.lp_set_pass_timing(ctx, False)
        lp.lp_map(ctx, small, [spec], [o_small])
    assert len(errors) == 2 and "captured" in errors[0] and "timing" in errors[1], errors
    o_small.fill_(float("nan"))
    g.replay()
    torch.cuda.synchronize()
    B = o_small.cpu().numpy().astype(np.float64)
    want = oracle.conv_same(small.cpu().numpy(), K)
    assert np.max(np.abs(B - want)) / np.max(np.abs(want)) <= TOL_FP32
    lp.lp_spectrum_release(ctx, spec)
