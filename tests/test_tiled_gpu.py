"""Maps larger than the padded size: overlap-save tiles (lp_map_tiled).

Each tile convolves the input window that covers it plus the PSF's reach;
the result must equal the plain SAME-mode convolution of Eq. (7) everywhere,
seams and map borders included, so every check here is against the FP64
oracle: the whole map for small cases, seeded samples, the 64 brightest
pixels and the pixels on both sides of every seam for a map larger than the
longest supported FFT length.
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
TOL_SPLIT = 2e-4


@pytest.fixture(scope="module")
def ctx():
    c = lp.lp_create(0)
    yield c
    lp.lp_destroy(c)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def err(got, ref):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))


def asym_psf(n, seed):
    """A PSF without point symmetry (complex spectrum)."""
    g = np.random.default_rng(seed)
    K = synth.psf_power_exp(n, 0.742, 0.1, 1.25, 40.0)
    return K * (1.0 + 0.5 * g.random(K.shape))


def tiled(ctx, L, Ks, pad, prec=lp.LP_PREC_FP32):
    specs = [lp.lp_kernel_spectrum(ctx, dev(K), pad_ny=pad[0], pad_nx=pad[1], prec=prec) for K in Ks]
    outs = [torch.full(L.shape, float("nan"), device=DEV) for _ in Ks]
    lp.lp_map_tiled(ctx, dev(L), specs, outs, prec=prec)
    lp.lp_sync_status(ctx)
    for s in specs:
        lp.lp_spectrum_release(ctx, s)
    return [o.cpu().numpy() for o in outs]


def test_tiles_cover_the_map_exactly(ctx):
    """300 x 260 map, 31^2 PSFs (one real, one complex spectrum), 96^2
    padding: tiles of 66 x 66 output pixels, a 5 x 4 grid with ragged last
    tiles; the whole output against the oracle."""
    L = synth.radiance_map(300, 260, 20, 1907_02891 + 60, lit_fraction=0.05)
    Ks = [synth.psf_power_exp(31, 0.742, 0.1, 1.25, 80.0), asym_psf(31, 7)]
    for K, B in zip(Ks, tiled(ctx, L, Ks, (96, 96))):
        assert np.isfinite(B).all()
        assert err(B, oracle.conv_same(L, K)) <= TOL_FP32


@pytest.mark.parametrize("shape,psf,pad", [
    ((66, 66), 31, (96, 96)),      # one tile (h <= Ny - cy = 81)
    ((81, 81), 31, (96, 96)),      # one tile at the SAME crop's padding limit, Ny = h + cy
    ((82, 133), 31, (96, 96)),     # one row / 52 columns past that: tiles of 66
    ((133, 67), 31, (96, 96)),     # the transpose
    ((1, 1), 31, (96, 96)),        # a single pixel
    ((40, 25), 31, (96, 96)),      # smaller than one tile
    ((257, 190), 45, (100, 64)),   # unequal paddings, tiles of 56 x 20
    ((129, 77), 1, (64, 64)),      # 1 x 1 PSF: tiles of the padded size, no margin
])
def test_ragged_and_degenerate_tilings(ctx, shape, psf, pad):
    # a dim floor keeps the oracle's maximum away from zero on the tiny maps
    L = synth.radiance_map(shape[0], shape[1], 6, 1907_02891 + 61 + shape[0], lit_fraction=0.05) + 0.01
    K = asym_psf(psf, shape[1])
    (B,) = tiled(ctx, L, [K], pad)
    assert np.isfinite(B).all()
    assert err(B, oracle.conv_same(L, K)) <= TOL_FP32


def test_one_tile_at_the_same_crops_padding(ctx):
    """A 4096^2 map with the 541^2 PSF in one 4608^2 transform (4096 + 270
    <= 4608 < 4096 + 540, the padding lp_map needs): sampled against the
    oracle, the pixels of the first and last rows and columns (where the
    wrap-around would land first) included."""
    wl = synth.WORKLOADS["map4096_psf541"]
    L, (K,) = wl.radiance(), wl.psfs()
    assert lp.lp_tiled_pad(4096, 4096, 541, 541) == (4608, 4608)
    (B,) = tiled(ctx, L, [K], (4608, 4608))
    H, W = B.shape
    g = np.random.default_rng(1907_02891 + 66)
    ii, jj = synth.sample_pixels(H, W, 4096, 1907_02891 + 67)
    flat = np.argpartition(B.ravel(), -64)[-64:]
    edge = np.array([0, 1, H - 2, H - 1])
    ii = np.concatenate([ii, flat // W, np.repeat(edge, 64), g.integers(0, H, 256)])
    jj = np.concatenate([jj, flat % W, g.integers(0, W, 256), np.repeat(edge, 64)])
    ref = oracle.conv_points_same(L, K, ii, jj)
    assert err(B[ii, jj], ref) <= TOL_FP32


def test_more_spectra_than_one_launch_takes_in_every_tile(ctx):
    """33 PSFs (one more than a column launch takes) over a 4 x 3 tile grid:
    every tile runs its spectra in two chunks; the first, the 32nd and the
    33rd output against the oracle, all of them finite."""
    L = synth.radiance_map(200, 150, 12, 1907_02891 + 68, lit_fraction=0.05)
    Ks = [synth.psf_power_exp(15, 0.742, 0.1, 1.0 + 0.03 * i, 40.0 + 5.0 * i) for i in range(33)]
    Bs = tiled(ctx, L, Ks, (64, 64))
    assert all(np.isfinite(B).all() for B in Bs)
    for i in (0, 31, 32):
        assert err(Bs[i], oracle.conv_same(L, Ks[i])) <= TOL_FP32, i


def test_tiled_split_precision(ctx):
    L = synth.radiance_map(300, 300, 20, 1907_02891 + 62, lit_fraction=0.05)
    K = synth.psf_power_exp(41, 0.742, 0.1, 1.25, 80.0)
    (B,) = tiled(ctx, L, [K], (128, 128), prec=lp.LP_PREC_SPLIT_BF16)
    assert err(B, oracle.conv_same(L, K)) <= TOL_SPLIT


def test_tiled_rejects_mixed_psf_sizes(ctx):
    a = lp.lp_kernel_spectrum(ctx, dev(synth.psf_power_exp(31, 0.742, 0.1, 1.25, 80.0)), pad_ny=96, pad_nx=96)
    b = lp.lp_kernel_spectrum(ctx, dev(synth.psf_power_exp(33, 0.742, 0.1, 1.25, 80.0)), pad_ny=96, pad_nx=96)
    L = torch.zeros((200, 200), device=DEV)
    outs = [torch.empty_like(L), torch.empty_like(L)]
    with pytest.raises(lp.LpError):
        lp.lp_map_tiled(ctx, L, [a, b], outs)
    with pytest.raises(lp.LpError):   # out overlapping L
        lp.lp_map_tiled(ctx, L, [a], [L])
    lp.lp_spectrum_release(ctx, a)
    lp.lp_spectrum_release(ctx, b)


@pytest.fixture(scope="module")
def big_map():
    H, W = 17800, 21000
    return synth.radiance_map(H, W, 8000, 1907_02891 + 63, lit_fraction=0.05)


@pytest.mark.parametrize("pad", [None, (17280, 17280)])
def test_map_beyond_the_longest_length_sampled(ctx, big_map, pad):
    """17800 x 21000 map (longer than the 17280-point transform), 801^2 PSF,
    spectra at the padded size lp_tiled_pad picks (10080 x 12288: 2 x 2
    tiles of 9280 x 11488) and at 17280^2 (2 x 2 tiles of 16480^2).  Seeded
    samples, the 64 brightest pixels and 512 pixels on each side of each
    seam, against the oracle."""
    L = big_map
    H, W = L.shape
    hk = 801
    ny, nx = pad if pad else lp.lp_tiled_pad(H, W, hk, hk)
    if pad is None:
        assert (ny, nx) == (10080, 12288)
    K = synth.psf_power_exp(hk, 0.742, 0.1, 1.25, 80.0)
    spec = lp.lp_kernel_spectrum(ctx, dev(K), pad_ny=ny, pad_nx=nx)
    Ld = dev(L)
    out = torch.empty((H, W), device=DEV)
    lp.lp_map_tiled(ctx, Ld, [spec], [out])
    lp.lp_sync_status(ctx)
    lp.lp_spectrum_release(ctx, spec)
    B = out.cpu().numpy()
    del Ld, out
    th, tw = ny - (hk - 1), nx - (hk - 1)
    g = np.random.default_rng(1907_02891 + 64)
    ii, jj = synth.sample_pixels(H, W, 4096, 1907_02891 + 65)
    flat = np.argpartition(B.ravel(), -64)[-64:]
    seam_r = np.concatenate([np.repeat(np.array([t - 2, t - 1, t, t + 1]), 128) for t in range(th, H, th)])
    seam_c = np.concatenate([np.repeat(np.array([t - 2, t - 1, t, t + 1]), 128) for t in range(tw, W, tw)])
    ii = np.concatenate([ii, flat // W, seam_r, g.integers(0, H, seam_c.size)])
    jj = np.concatenate([jj, flat % W, g.integers(0, W, seam_r.size), seam_c])
    ref = oracle.conv_points_same(L, K, ii, jj)
    assert np.isfinite(B[ii, jj]).all()
    assert err(B[ii, jj], ref) <= TOL_FP32
