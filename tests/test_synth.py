"""Host-side checks of the seeded input generators (no method arithmetic)."""

import json
import os

import numpy as np

import synth
from _golden import GOLDEN


def test_radiance_map_is_seeded_nonnegative_and_sparse():
    a = synth.radiance_map(128, 96, 10, seed=123, lit_fraction=0.05)
    b = synth.radiance_map(128, 96, 10, seed=123, lit_fraction=0.05)
    c = synth.radiance_map(128, 96, 10, seed=124, lit_fraction=0.05)
    assert a.dtype == np.float32 and a.shape == (128, 96)
    np.testing.assert_array_equal(a, b)
    assert not np.array_equal(a, c)
    assert np.all(a >= 0)
    assert 0.02 < np.mean(a > 0) < 0.6


def test_dynamic_range_clip():
    L = synth.radiance_map(256, 256, 40, seed=5, lit_fraction=0.05,
                           lit_range=(1e-3, 1e3), clip_range=(1e-3, 1e3))
    nz = L[L > 0]
    assert nz.min() >= np.float32(1e-3) and nz.max() <= np.float32(1e3)


def test_power_exp_psf_is_radial_and_centred():
    K = synth.psf_power_exp(101, 1.0, 0.25, 1.25, 40.0)
    assert K.shape == (101, 101) and K.dtype == np.float64
    assert K[50, 50] == 0.25 ** -1.25
    np.testing.assert_array_equal(K, K[::-1, :])
    np.testing.assert_array_equal(K, K.T)
    r = np.hypot(3.0, 4.0)
    assert abs(K[53, 54] - (r * r + 0.25) ** -1.25 * np.exp(-r / 40.0)) < 1e-18


def test_alr_psf_follows_eq12_13():
    with open(os.path.join(GOLDEN, "paper_constants.json")) as fh:
        g = json.load(fh)["alr_psf"]
    c = 1.0 / g["c_inverse"]
    # 1 km pixels: d = 1 km gives d^-alpha = 1, so K = c exactly
    K = synth.psf_alr(7, 1.0)
    assert K[3, 3] == c                       # d -> 0 limit
    assert abs(K[3, 4] - c) < 1e-18          # d = 1 km
    d = 2.0
    alpha = g["alpha_scale"] * (d / g["d_ref_km"]) ** g["alpha_power"]
    assert abs(K[3, 5] - c * d ** -alpha) < 1e-18
    # decreasing beyond 1 km (it rises above c for 0 < d < 1 km)
    K2 = synth.psf_alr(801, 0.4044)
    row = K2[400, 403:]
    assert np.all(np.diff(row) < 0)


def test_request_stream_is_seeded():
    a = synth.request_stream(50, 100.0, seed=9)
    b = synth.request_stream(50, 100.0, seed=9)
    assert a == b
    assert all(r.side in synth.SERVE_TILE_SIDES for r in a)
    assert all(1 <= len(r.kernels) <= 8 and len(set(r.kernels)) == len(r.kernels) for r in a)
    assert all(a[i].arrival_s < a[i + 1].arrival_s for i in range(49))
