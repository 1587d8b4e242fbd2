"""GPU parity of the CUDA path (through the C ABI) against the FP64 oracle.

Error metric: max |B - B_ref| / max |B_ref| over the evaluated pixels; the
bar for the FP32 path is 1e-5.  Full maps for small cases; on the full-size
workloads, 4096 seeded pixels plus the 64 brightest pixels of the GPU
output (so that the denominator is the global maximum).
"""

import json
import os

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1907_02891_gb300 import lp  # noqa: E402

TOL_FP32 = 1e-5
DEV = "cuda:0"


@pytest.fixture(scope="module")
def ctx():
    c = lp.lp_create(0)
    yield c
    lp.lp_destroy(c)


def err_maxnorm(got, ref):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    err = float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))
    record_error(err)
    return err


def record_error(err):
    """Append the measured error to $LP_PARITY_LOG (one JSON line per check)."""
    path = os.environ.get("LP_PARITY_LOG")
    if path:
        with open(path, "a") as fh:
            fh.write(json.dumps({"test": os.environ.get("PYTEST_CURRENT_TEST", "").split(" ")[0],
                                 "max_norm_err": err}) + "\n")


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def run_map(ctx, L, Ks, mode=lp.LP_OUT_SAME, pad=None):
    h, w = L.shape
    specs = []
    for K in Ks:
        if pad is None:
            specs.append(lp.lp_kernel_spectrum(ctx, dev(K), max_h=h, max_w=w))
        else:
            specs.append(lp.lp_kernel_spectrum(ctx, dev(K), pad_ny=pad[0], pad_nx=pad[1]))
    hk, wk = Ks[0].shape
    shape = lp.output_shape(h, w, hk, wk, mode)
    outs = [torch.empty(shape, dtype=torch.float32, device=DEV) for _ in Ks]
    lp.lp_map(ctx, dev(L), specs, outs, mode=mode)
    lp.lp_sync_status(ctx)
    res = [o.cpu().numpy() for o in outs]
    for s in specs:
        lp.lp_spectrum_release(ctx, s)
    return res


def wrap_place(K, ny, nx):
    hk, wk = K.shape
    cy, cx = (hk - 1) // 2, (wk - 1) // 2
    Kw = np.zeros((ny, nx))
    for y in range(hk):
        for x in range(wk):
            Kw[(y - cy) % ny, (x - cx) % nx] = K[y, x]
    return Kw


# --- S0: the spectrum is Eq. (10) of the wrap-placed PSF -------------------

@pytest.mark.parametrize("symmetric", [False, True])
def test_spectrum_is_eq10_dft(ctx, symmetric):
    g = np.random.default_rng(11)
    ny, nx = 45, 64
    if symmetric:
        K = synth.psf_power_exp(7, 1.0, 0.25, 1.25, 40.0)[:, 1:6]   # 7 x 5, point-symmetric
    else:
        K = g.uniform(0.1, 1.0, (5, 7))
    s = lp.lp_kernel_spectrum(ctx, dev(K), pad_ny=ny, pad_nx=nx)
    info = lp.lp_spectrum_info(s)
    assert (info["ny"], info["nx"], info["hk"], info["wk"]) == (ny, nx) + K.shape
    assert info["is_real"] == symmetric
    nc = nx // 2 + 1
    per = 1 if symmetric else 2
    buf = torch.empty(nc * ny * per, dtype=torch.float32, device=DEV)
    lp.lp_spectrum_copy(s, buf)
    torch.cuda.synchronize()
    got = buf.cpu().numpy().astype(np.float64)
    got = got.reshape(nc, ny) if symmetric else (got[0::2] + 1j * got[1::2]).reshape(nc, ny)
    uu, cc = np.meshgrid(np.arange(ny), np.arange(nc), indexing="ij")
    ref = oracle.dft2_points(wrap_place(K, ny, nx), uu, cc).reshape(ny, nc).T / (2.0 * ny * nx)
    scale = np.max(np.abs(ref))
    if symmetric:
        assert np.max(np.abs(ref.imag)) < 1e-12 * scale
        ref = ref.real
    assert np.max(np.abs(got - ref)) < 2e-7 * scale
    lp.lp_spectrum_release(ctx, s)


# --- the whole path, small and full ------------------------------------------

def test_map256_psf101_full_map(ctx):
    wl = synth.WORKLOADS["map256_psf101"]
    L, K = wl.radiance(), wl.psfs()[0]
    (B,) = run_map(ctx, L, [K])
    assert err_maxnorm(B, oracle.conv_same(L, K)) <= TOL_FP32
    (Bf,) = run_map(ctx, L, [K], mode=lp.LP_OUT_FULL)
    assert Bf.shape == (356, 356)
    assert err_maxnorm(Bf, oracle.conv_full(L, K)) <= TOL_FP32


def _pairs():
    sizes = lp.supported_sizes()
    n = len(sizes)
    return [(sizes[i], sizes[(i * 7 + 3) % n]) for i in range(n)]


@pytest.mark.parametrize("ny,nx", _pairs())
def test_every_fft_length(ctx, ny, nx):
    """Each supported length once as the column length (P2) and once as the
    row length (P1, P3); a ragged map inside the padded grid."""
    g = np.random.default_rng(ny * 100003 + nx)
    hk = 9 if min(ny, nx) >= 40 else 5
    wk = 7 if min(ny, nx) >= 40 else 3
    h = min(ny - hk + 1, 93)
    w = min(nx - wk + 1, 71)
    L = g.lognormal(0.0, 1.0, (h, w)).astype(np.float32)
    K = g.uniform(0.05, 1.0, (hk, wk))              # asymmetric: complex spectrum
    Ksym = synth.psf_power_exp(hk, 1.0, 0.25, 1.25, 40.0)[:, (hk - wk) // 2:(hk + wk) // 2]
    mode = lp.LP_OUT_FULL if (ny + nx) % 2 else lp.LP_OUT_SAME
    B, Bs = run_map(ctx, L, [K, Ksym], mode=mode, pad=(ny, nx))
    conv = oracle.conv_full if mode == lp.LP_OUT_FULL else oracle.conv_same
    assert err_maxnorm(B, conv(L, K)) <= TOL_FP32
    assert err_maxnorm(Bs, conv(L, Ksym)) <= TOL_FP32


def test_ragged_leading_dimensions_and_mixed_spectra(ctx):
    g = np.random.default_rng(12)
    big = g.lognormal(0.0, 1.0, (41, 64)).astype(np.float32)
    L = big[2:39, 5:58]                                   # 37 x 53, ldl = 64
    Ks = [g.uniform(0.1, 1.0, (9, 11)), synth.psf_power_exp(11, 1.0, 0.1, 1.25, 80.0),
          g.uniform(0.1, 1.0, (9, 11))]
    Ks[1] = Ks[1][1:10, :]
    Ld = dev(big)[2:39, 5:58]
    for mode in (lp.LP_OUT_SAME, lp.LP_OUT_FULL):
        specs = [lp.lp_kernel_spectrum(ctx, dev(K), max_h=37, max_w=53) for K in Ks]
        shape = lp.output_shape(37, 53, 9, 11, mode)
        store = torch.full((3, shape[0], shape[1] + 6), float("nan"), device=DEV)
        outs = [store[k, :, :shape[1]] for k in range(3)]
        lp.lp_map(ctx, Ld, specs, outs, mode=mode)
        lp.lp_sync_status(ctx)
        conv = oracle.conv_full if mode == lp.LP_OUT_FULL else oracle.conv_same
        for k in range(3):
            assert err_maxnorm(outs[k].cpu().numpy(), conv(np.ascontiguousarray(L), Ks[k])) <= TOL_FP32
        assert torch.isnan(store[:, :, shape[1]:]).all(), "wrote outside the output rows"
        for s in specs:
            lp.lp_spectrum_release(ctx, s)


def test_single_row_and_column_maps(ctx):
    g = np.random.default_rng(13)
    K = g.uniform(0.1, 1.0, (5, 5))
    for shape in [(1, 60), (60, 1), (1, 1)]:
        L = g.lognormal(0.0, 1.0, shape).astype(np.float32)
        (B,) = run_map(ctx, L, [K], mode=lp.LP_OUT_FULL)
        assert err_maxnorm(B, oracle.conv_full(L, K)) <= TOL_FP32


def test_zero_map_gives_zero(ctx):
    K = synth.psf_power_exp(21, 1.0, 0.25, 1.25, 40.0)
    (B,) = run_map(ctx, np.zeros((50, 70), np.float32), [K])
    assert np.all(B == 0.0)


def test_multiclass_eq4(ctx):
    g = np.random.default_rng(14)
    Ls = [g.lognormal(0.0, 1.0, (60, 75)).astype(np.float32) for _ in range(3)]
    Ks = [synth.psf_power_exp(15, 1.0, 0.25, p, 40.0) for p in (1.0, 1.5, 2.0)]
    specs = [lp.lp_kernel_spectrum(ctx, dev(K), max_h=60, max_w=75) for K in Ks]
    out = torch.empty((60, 75), dtype=torch.float32, device=DEV)
    lp.lp_map_multiclass(ctx, [dev(x) for x in Ls], specs, out)
    lp.lp_sync_status(ctx)
    ii, jj = np.meshgrid(np.arange(60), np.arange(75), indexing="ij")
    ref = oracle.conv_multiclass_points_same(Ls, Ks, ii, jj).reshape(60, 75)
    assert err_maxnorm(out.cpu().numpy(), ref) <= TOL_FP32
    for s in specs:
        lp.lp_spectrum_release(ctx, s)


def test_host_entry_point_matches_device(ctx):
    wl = synth.WORKLOADS["map256_psf101"]
    L, K = wl.radiance(), wl.psfs()[0]
    s = lp.lp_kernel_spectrum(ctx, dev(K), max_h=256, max_w=256)
    out_d = torch.empty((256, 256), dtype=torch.float32, device=DEV)
    lp.lp_map(ctx, dev(L), [s], [out_d])
    out_h = torch.empty((256, 256), dtype=torch.float32).pin_memory()
    L_h = torch.from_numpy(L).pin_memory()
    lp.lp_map_host(ctx, L_h, [s], [out_h])
    lp.lp_sync_status(ctx)
    assert torch.equal(out_h, out_d.cpu())
    lp.lp_spectrum_release(ctx, s)


def test_host_entry_point_banded_ragged_full_mode(ctx):
    """The pipelined host path (row bands copied while transformed) on an odd
    map size, FULL output, three spectra (one complex), leading dimensions."""
    g = np.random.default_rng(16)
    big = g.lognormal(0.0, 1.0, (77, 130)).astype(np.float32)
    L = big[:, 3:120]                                     # 77 x 117, ldl = 130
    Ks = [synth.psf_power_exp(21, 1.0, 0.25, 1.25, 40.0), g.uniform(0.1, 1.0, (21, 21)),
          synth.psf_power_exp(21, 1.0, 0.25, 2.0, 80.0)]
    specs = [lp.lp_kernel_spectrum(ctx, dev(K), max_h=77, max_w=117) for K in Ks]
    Ho, Wo = 77 + 20, 117 + 20
    host_out = [np.full((Ho, Wo + 5), np.nan, np.float32) for _ in Ks]
    lp.lp_map_host(ctx, L, specs, [o[:, :Wo] for o in host_out], mode=lp.LP_OUT_FULL)
    lp.lp_sync_status(ctx)
    dev_out = [torch.empty((Ho, Wo), dtype=torch.float32, device=DEV) for _ in Ks]
    lp.lp_map(ctx, dev(np.ascontiguousarray(L)), specs, dev_out, mode=lp.LP_OUT_FULL)
    lp.lp_sync_status(ctx)
    for k, K in enumerate(Ks):
        np.testing.assert_array_equal(host_out[k][:, :Wo], dev_out[k].cpu().numpy())
        assert np.isnan(host_out[k][:, Wo:]).all()
        assert err_maxnorm(host_out[k][:, :Wo], oracle.conv_full(np.ascontiguousarray(L), K)) <= TOL_FP32
    for s in specs:
        lp.lp_spectrum_release(ctx, s)


def test_host_entry_point_back_to_back_calls(ctx):
    """Consecutive host maps overlap (a map's upload with the previous map's
    passes, its passes with the previous map's download; input and output
    staging alternating between two buffers each): five calls
    with different maps and two spectra, one sync at the end, every output
    bitwise equal to the device path's."""
    g = np.random.default_rng(17)
    Ks = [synth.psf_power_exp(31, 1.0, 0.25, 1.25, 40.0), g.uniform(0.1, 1.0, (31, 31))]
    specs = [lp.lp_kernel_spectrum(ctx, dev(K), max_h=300, max_w=280) for K in Ks]
    Ls = [torch.from_numpy(g.lognormal(0.0, 1.0, (300, 280)).astype(np.float32)).pin_memory() for _ in range(5)]
    outs = [[torch.full((300, 280), float("nan")).pin_memory() for _ in Ks] for _ in Ls]
    for L, o in zip(Ls, outs):
        lp.lp_map_host(ctx, L, specs, o)
    lp.lp_sync_status(ctx)
    for L, o in zip(Ls, outs):
        ref = [torch.empty((300, 280), dtype=torch.float32, device=DEV) for _ in Ks]
        lp.lp_map(ctx, L.to(DEV), specs, ref)
        lp.lp_sync_status(ctx)
        for a, b in zip(o, ref):
            assert torch.equal(a, b.cpu())
    for s in specs:
        lp.lp_spectrum_release(ctx, s)


# --- full-size workloads, sampled against the oracle -------------------------

def _sampled_check(L, K, B, seed, n=4096, top=64):
    H, W = L.shape
    ii, jj = synth.sample_pixels(H, W, n, seed)
    flat = np.argpartition(B.ravel(), -top)[-top:]
    ii = np.concatenate([ii, flat // W])
    jj = np.concatenate([jj, flat % W])
    ref = oracle.conv_points_same(L, K, ii, jj)
    return err_maxnorm(B[ii, jj], ref)


def test_map4096_psf541_sampled(ctx):
    wl = synth.WORKLOADS["map4096_psf541"]
    L, K = wl.radiance(), wl.psfs()[0]
    (B,) = run_map(ctx, L, [K])
    assert _sampled_check(L, K, B, wl.seed + 100) <= TOL_FP32


def test_map8192_psf601x16_batched_sampled(ctx):
    wl = synth.WORKLOADS["map8192_psf601x16"]
    L, Ks = wl.radiance(), wl.psfs()
    Bs = run_map(ctx, L, Ks)
    for k, (K, B) in enumerate(zip(Ks, Bs)):
        assert _sampled_check(L, K, B, wl.seed + 100 + k) <= TOL_FP32, k


def test_map16384_psf801_sampled(ctx):
    wl = synth.WORKLOADS["map16384_psf801"]
    L, K = wl.radiance(), wl.psfs()[0]
    (B,) = run_map(ctx, L, [K])
    assert _sampled_check(L, K, B, wl.seed + 100) <= TOL_FP32


def test_paper_shape_two_maps_one_forward_transform(ctx):
    """Sec. 3: two maps (all-sky ratio, Eq. (12)-(13), 1485^2; zenith-brightness
    stand-in, 965^2) of an 11920 x 11804 map at 404.4 m, from one call."""
    L, Ks = synth.paper_shape_inputs()
    H, W = L.shape
    ny = lp.lp_supported_size(H + 1485 - 1)
    nx = lp.lp_supported_size(W + 1485 - 1)
    specs = [lp.lp_kernel_spectrum(ctx, dev(K), pad_ny=ny, pad_nx=nx) for K in Ks]
    outs = [torch.empty((H, W), dtype=torch.float32, device=DEV) for _ in Ks]
    lp.lp_map(ctx, dev(L), specs, outs)
    lp.lp_sync_status(ctx)
    for k, (K, o) in enumerate(zip(Ks, outs)):
        assert _sampled_check(L, K, o.cpu().numpy(), synth.PAPER_SHAPE["seed"] + 10 + k) <= TOL_FP32, k
    for s in specs:
        lp.lp_spectrum_release(ctx, s)


def _sampled_check_full(L, K, B, seed, n=4096, top=64):
    """As _sampled_check for LP_OUT_FULL output (Hout x Wout = H+hk-1 x W+wk-1)."""
    Ho, Wo = B.shape
    ii, jj = synth.sample_pixels(Ho, Wo, n, seed)
    flat = np.argpartition(B.ravel(), -top)[-top:]
    ii = np.concatenate([ii, flat // Wo])
    jj = np.concatenate([jj, flat % Wo])
    ref = oracle.conv_points_full(L, K, ii, jj)
    return err_maxnorm(B[ii, jj], ref)


def test_tight_padding_at_a_production_length(ctx):
    """h = Ny - hk + 1 exactly (4164 + 541 - 1 = 4704): the kept rows and
    columns reach the wrap boundary of the padded grid in both output modes.
    FULL mode is also checked on every pixel through Sum Bfull = Sum L * Sum K
    (sums in FP64 on the host), which holds for the uncropped linear
    convolution whatever the FFT did inside."""
    h = w = 4704 - 541 + 1
    L = synth.radiance_map(h, w, 400, 1907_02891 + 31, lit_fraction=0.05)
    K = synth.psf_power_exp(541, 0.742, 0.1, 1.25, 80.0)
    s = lp.lp_kernel_spectrum(ctx, dev(K), max_h=h, max_w=w)
    assert (lp.lp_spectrum_info(s)["ny"], lp.lp_spectrum_info(s)["nx"]) == (4704, 4704)
    Ld = dev(L)
    same = torch.empty((h, w), dtype=torch.float32, device=DEV)
    full = torch.empty((4704, 4704), dtype=torch.float32, device=DEV)
    lp.lp_map(ctx, Ld, [s], [same])
    lp.lp_map(ctx, Ld, [s], [full], mode=lp.LP_OUT_FULL)
    lp.lp_sync_status(ctx)
    B, Bf = same.cpu().numpy(), full.cpu().numpy()
    assert _sampled_check(L, K, B, 1907_02891 + 32) <= TOL_FP32
    # the first and last kept rows and columns, where the crop meets the wrap:
    # their values are small, so the error is normalised by the map maximum
    # (the metric's denominator everywhere else)
    edge = np.concatenate([np.arange(0, 4704, 97), [4703]])
    ii = np.concatenate([np.zeros_like(edge), np.full_like(edge, 4703), edge, edge])
    jj = np.concatenate([edge, edge, np.zeros_like(edge), np.full_like(edge, 4703)])
    ref = oracle.conv_points_full(L, K, ii, jj)
    err = float(np.max(np.abs(Bf[ii, jj].astype(np.float64) - ref)) / np.max(np.abs(Bf)))
    record_error(err)
    assert err <= TOL_FP32
    assert _sampled_check_full(L, K, Bf, 1907_02891 + 33) <= TOL_FP32
    total = float(np.sum(Bf, dtype=np.float64))
    expect = float(np.sum(L, dtype=np.float64)) * float(np.sum(K))
    rel = abs(total - expect) / expect
    record_error(rel)
    assert rel <= TOL_FP32
    lp.lp_spectrum_release(ctx, s)


def test_full_mode_sum_invariant_at_full_size(ctx):
    """Sum Bfull = Sum L * Sum K on the 4096^2 map with the 541^2 PSF (FULL
    output 4636^2, padded 4704^2): an oracle-free check of every output pixel
    at once, sums in FP64 on the host."""
    wl = synth.WORKLOADS["map4096_psf541"]
    L, K = wl.radiance(), wl.psfs()[0]
    (Bf,) = run_map(ctx, L, [K], mode=lp.LP_OUT_FULL)
    assert Bf.shape == (4096 + 540, 4096 + 540)
    total = float(np.sum(Bf, dtype=np.float64))
    expect = float(np.sum(L, dtype=np.float64)) * float(np.sum(K))
    rel = abs(total - expect) / expect
    record_error(rel)
    assert rel <= TOL_FP32


def test_multiclass_eq4_at_workload_size(ctx):
    """Sec. 2.2 Eq. (4) on 4096^2 maps: three source classes, each with its
    own 541^2 PSF, summed before one inverse transform; 4096 seeded pixels +
    the 64 brightest against the oracle's Eq. (4)."""
    H = W = 4096
    Ls = [synth.radiance_map(H, W, 400, 1907_02891 + 40 + t, lit_fraction=0.05) for t in range(3)]
    Ks = [synth.psf_power_exp(541, 0.742, 0.1, p, lam) for (p, lam) in ((1.25, 80.0), (1.5, 40.0), (2.0, 200.0))]
    specs = [lp.lp_kernel_spectrum(ctx, dev(K), max_h=H, max_w=W) for K in Ks]
    out = torch.empty((H, W), dtype=torch.float32, device=DEV)
    lp.lp_map_multiclass(ctx, [dev(x) for x in Ls], specs, out)
    lp.lp_sync_status(ctx)
    B = out.cpu().numpy()
    ii, jj = synth.sample_pixels(H, W, 4096, 1907_02891 + 44)
    flat = np.argpartition(B.ravel(), -64)[-64:]
    ii = np.concatenate([ii, flat // W])
    jj = np.concatenate([jj, flat % W])
    ref = oracle.conv_multiclass_points_same(Ls, Ks, ii, jj)
    assert err_maxnorm(B[ii, jj], ref) <= TOL_FP32
    for s in specs:
        lp.lp_spectrum_release(ctx, s)


def test_multiclass_eq4_at_the_longest_column_length(ctx):
    """Eq. (4) with the column transform at 17280 (the longest built length;
    the sums of the class products live in global memory, so every length
    takes several classes): a tall 16384 x 64 map per class, 31 x 31 PSFs,
    sampled against the oracle."""
    H, W = 16384, 64
    Ls = [synth.radiance_map(H, W, 200, 1907_02891 + 50 + t, lit_fraction=0.05) for t in range(3)]
    Ks = [synth.psf_power_exp(31, 1.0, 0.25, p, 40.0) for p in (1.0, 1.5, 2.0)]
    specs = [lp.lp_kernel_spectrum(ctx, dev(K), pad_ny=17280, pad_nx=96) for K in Ks]
    out = torch.empty((H, W), dtype=torch.float32, device=DEV)
    lp.lp_map_multiclass(ctx, [dev(x) for x in Ls], specs, out)
    lp.lp_sync_status(ctx)
    B = out.cpu().numpy()
    ii, jj = synth.sample_pixels(H, W, 4096, 1907_02891 + 51)
    flat = np.argpartition(B.ravel(), -64)[-64:]
    ii = np.concatenate([ii, flat // W])
    jj = np.concatenate([jj, flat % W])
    ref = oracle.conv_multiclass_points_same(Ls, Ks, ii, jj)
    assert err_maxnorm(B[ii, jj], ref) <= TOL_FP32
    for s in specs:
        lp.lp_spectrum_release(ctx, s)


# --- cache, budget, validation, bounded waits ---------------------------------

def test_spectrum_cache_confirms_hits_by_value(ctx):
    """With every fingerprint forced equal (test hook), two different PSFs of
    the same size still get their own spectra -- the stored copy of K is
    compared value by value -- and the same PSF again is a cache hit."""
    g = np.random.default_rng(18)
    K1 = g.uniform(0.1, 1.0, (21, 21))
    K2 = K1.copy()
    K2[3, 4] = np.nextafter(K2[3, 4], 2.0)                # one ulp apart
    L = g.lognormal(0.0, 1.0, (90, 80)).astype(np.float32)
    lp.lp_set_test_hook(ctx, lp.LP_TEST_FP_COLLIDE)
    try:
        a = lp.lp_kernel_spectrum(ctx, dev(K1), max_h=90, max_w=80)
        b = lp.lp_kernel_spectrum(ctx, dev(K2), max_h=90, max_w=80)
        a2 = lp.lp_kernel_spectrum(ctx, dev(K1), max_h=90, max_w=80)
        b2 = lp.lp_kernel_spectrum(ctx, dev(K2), max_h=90, max_w=80)
        assert a != b and a == a2 and b == b2
        Ld = dev(L)
        outs = [torch.empty((90, 80), dtype=torch.float32, device=DEV) for _ in range(2)]
        lp.lp_map(ctx, Ld, [a, b], outs)
        lp.lp_sync_status(ctx)
        assert err_maxnorm(outs[0].cpu().numpy(), oracle.conv_same(L, K1)) <= TOL_FP32
        assert err_maxnorm(outs[1].cpu().numpy(), oracle.conv_same(L, K2)) <= TOL_FP32
        for s in (a, a2, b, b2):
            lp.lp_spectrum_release(ctx, s)
    finally:
        lp.lp_set_test_hook(ctx, 0)


def test_map_waits_for_a_spectrum_still_being_built(ctx):
    """lp_kernel_spectrum is asynchronous on its stream.  A map on another
    stream, issued right after it without any synchronisation, must still
    see the finished spectrum (the map waits for the build in stream order);
    so must a request submitted to the scheduler (non-blocking streams)."""
    g = np.random.default_rng(19)
    K = g.uniform(0.1, 1.0, (601, 601))                    # complex spectrum, 8820^2 FP64 build
    L = dev(g.lognormal(0.0, 1.0, (512, 512)).astype(np.float32))
    c2 = lp.lp_create(0)                                   # fresh cache: the build really runs
    try:
        s_build, s_map = torch.cuda.Stream(), torch.cuda.Stream()
        torch.cuda.synchronize()
        spec = lp.lp_kernel_spectrum(c2, dev(K), pad_ny=8820, pad_nx=8820, stream=s_build)
        racing = torch.full((512, 512), float("nan"), device=DEV)
        lp.lp_map(c2, L, [spec], [racing], stream=s_map)
        lp.lp_serve_start(c2, 2)
        served = torch.full((512, 512), float("nan"), device=DEV)
        t = lp.lp_serve_submit(c2, L, [spec], [served])
        assert lp.lp_serve_poll(c2, t, timeout_ms=60000) is not None
        lp.lp_serve_stop(c2)
        torch.cuda.synchronize()
        ref = torch.empty((512, 512), device=DEV)
        lp.lp_map(c2, L, [spec], [ref])
        lp.lp_sync_status(c2)
        assert torch.equal(racing, ref)
        assert torch.equal(served, ref)
        lp.lp_spectrum_release(c2, spec)
    finally:
        lp.lp_destroy(c2)


def test_release_is_stream_ordered(ctx):
    """Releasing the last reference of a spectrum that enqueued maps still
    read returns at once (no device-wide wait); its memory is freed only
    after those maps have completed, and their results are intact."""
    wl = synth.WORKLOADS["map8192_psf601x16"]
    c2 = lp.lp_create(0)
    try:
        L = dev(synth.radiance_map(8192, 8192, 1600, wl.seed, lit_fraction=0.05))
        K = dev(wl.psfs()[0])
        spec = lp.lp_kernel_spectrum(c2, K, max_h=8192, max_w=8192)
        ref = torch.empty((8192, 8192), device=DEV)
        lp.lp_map(c2, L, [spec], [ref])
        side = torch.cuda.Stream()
        lp.lp_map(c2, L, [spec], [ref], stream=side)     # the side stream's workspace
        lp.lp_sync_status(c2)
        lp.lp_sync_status(c2, stream=side)
        held = lp.lp_bytes_in_use(c2)
        outs = [torch.full((8192, 8192), float("nan"), device=DEV) for _ in range(6)]
        for o in outs:
            lp.lp_map(c2, L, [spec], [o], stream=side)
        lp.lp_spectrum_release(c2, spec)                 # last reference, maps in flight
        busy = lp.lp_sync_status_code(c2, stream=side, timeout_ms=0)
        assert busy == lp.LP_ERR_TIMEOUT, "release waited for the device"
        assert lp.lp_bytes_in_use(c2) == held            # not freed under the running maps
        lp.lp_sync_status(c2, stream=side)               # reaps it
        assert lp.lp_bytes_in_use(c2) < held
        for o in outs:
            assert torch.equal(o, ref)
    finally:
        lp.lp_destroy(c2)


def test_spectrum_cache_refcount(ctx):
    K = dev(synth.psf_power_exp(11, 1.0, 0.25, 1.25, 40.0))
    a = lp.lp_kernel_spectrum(ctx, K, max_h=64, max_w=64)
    b = lp.lp_kernel_spectrum(ctx, K, max_h=64, max_w=64)
    c = lp.lp_kernel_spectrum(ctx, K, pad_ny=120, pad_nx=96)
    assert a == b and a != c
    lp.lp_spectrum_release(ctx, a)
    lp.lp_spectrum_release(ctx, b)
    lp.lp_spectrum_release(ctx, c)
    with pytest.raises(lp.LpError) as e:
        lp.lp_spectrum_release(ctx, a)
    assert e.value.status == lp.LP_ERR_INVALID


def test_budget_refuses_oversized_spectrum():
    c = lp.lp_create(0, 4 << 20)
    try:
        K = dev(synth.psf_power_exp(541, 0.742, 0.1, 1.25, 80.0))
        with pytest.raises(lp.LpError) as e:
            lp.lp_kernel_spectrum(c, K, max_h=4096, max_w=4096)
        assert e.value.status == lp.LP_ERR_OOM
        assert lp.lp_bytes_in_use(c) < 4 << 20
    finally:
        lp.lp_destroy(c)


def test_invalid_arguments(ctx):
    g = np.random.default_rng(15)
    L = dev(g.uniform(0, 1, (40, 50)).astype(np.float32))
    K = dev(g.uniform(0, 1, (9, 9)))
    with pytest.raises(lp.LpError) as e:
        lp.lp_kernel_spectrum(ctx, dev(g.uniform(0, 1, (8, 9))), max_h=40, max_w=50)
    assert e.value.status == lp.LP_ERR_INVALID
    with pytest.raises(lp.LpError) as e:
        lp.lp_kernel_spectrum(ctx, K, pad_ny=97, pad_nx=96)       # 97 not a built length
    assert e.value.status == lp.LP_ERR_UNSUPPORTED
    with pytest.raises(lp.LpError) as e:
        lp.lp_kernel_spectrum(ctx, K, max_h=40, max_w=50, prec=lp.LP_PREC_SPLIT_FP16)
    assert e.value.status == lp.LP_ERR_UNSUPPORTED
    s_small = lp.lp_kernel_spectrum(ctx, K, pad_ny=45, pad_nx=64)  # 45 < 40 + 9 - 1
    out = torch.empty((40, 50), dtype=torch.float32, device=DEV)
    with pytest.raises(lp.LpError) as e:
        lp.lp_map(ctx, L, [s_small], [out])
    assert e.value.status == lp.LP_ERR_INVALID
    s = lp.lp_kernel_spectrum(ctx, K, max_h=40, max_w=50)
    with pytest.raises(lp.LpError) as e:
        lp.lp_map(ctx, L, [s], [L])                               # in place
    assert e.value.status == lp.LP_ERR_INVALID
    with pytest.raises(lp.LpError) as e:
        lp.lp_map(ctx, L, [s], [out], prec=lp.LP_PREC_SPLIT_FP16)
    assert e.value.status == lp.LP_ERR_UNSUPPORTED
    st = lp.call_status("lp_map", ctx, L.data_ptr(), 40, 50, 30, None, 1, None, 50, 0, 0, None)
    assert st == lp.LP_ERR_INVALID
    lp.lp_spectrum_release(ctx, s)
    lp.lp_spectrum_release(ctx, s_small)


def test_sync_status_wait_is_bounded(ctx):
    wl = synth.WORKLOADS["map4096_psf541"]
    L = dev(wl.radiance())
    s = lp.lp_kernel_spectrum(ctx, dev(wl.psfs()[0]), max_h=4096, max_w=4096)
    out = torch.empty_like(L)
    lp.lp_sync_status(ctx)
    for _ in range(40):
        lp.lp_map(ctx, L, [s], [out])
    assert lp.lp_sync_status_code(ctx, timeout_ms=0) == lp.LP_ERR_TIMEOUT
    assert lp.lp_sync_status_code(ctx, timeout_ms=-1) == lp.LP_OK
    lp.lp_spectrum_release(ctx, s)
