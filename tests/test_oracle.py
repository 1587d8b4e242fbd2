"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test pins the oracle to something other than itself: a hand-worked
example, a closed form, an invariant, a special case that reduces to a
library routine, or brute force on tiny inputs.  A dropped term, a wrong sign
or index, a flipped (correlation instead of convolution) or transposed
operand fails at least one of them.
"""

import json
import math
import os

import numpy as np
import pytest

from _golden import GOLDEN, read_blocks

import synth


def _rel(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(np.max(np.abs(b)), 1e-300))


# --- Eq. (7) discretised: hand-worked example --------------------------------

def test_hand_worked_convolution(oracle_lib):
    g = read_blocks("conv_hand_2x2_3x3.txt")
    L = g["L"].astype(np.float32)
    K = g["K"]
    np.testing.assert_array_equal(oracle_lib.conv_full(L, K), g["Bfull"])
    np.testing.assert_array_equal(oracle_lib.conv_same(L, K), g["Bsame"])


# --- delta source: B is K itself, shifted (exact) ----------------------------

@pytest.mark.parametrize("a,b", [(0, 0), (4, 7), (8, 10), (3, 0)])
def test_delta_source_returns_shifted_kernel(oracle_lib, a, b):
    g = np.random.default_rng(1)
    K = g.uniform(0.5, 2.0, (5, 7))            # asymmetric on purpose
    H, W = 9, 11
    L = np.zeros((H, W), np.float32)
    L[a, b] = 1.0
    expect = np.zeros((H + 4, W + 6))
    expect[a:a + 5, b:b + 7] = K
    np.testing.assert_array_equal(oracle_lib.conv_full(L, K), expect)


def test_delta_same_crop_puts_psf_centre_on_the_source(oracle_lib):
    g = np.random.default_rng(2)
    K = g.uniform(0.5, 2.0, (7, 5))
    cy, cx = 3, 2
    L = np.zeros((10, 12), np.float32)
    L[4, 6] = 1.0
    B = oracle_lib.conv_same(L, K)
    # observer at the source sees the PSF centre; one row below sees K[cy+1]
    assert B[4, 6] == K[cy, cx]
    assert B[5, 6] == K[cy + 1, cx]
    assert B[4, 7] == K[cy, cx + 1]
    assert B[0, 0] == 0.0


# --- linearity (linear regime of Sec. 2.1) -----------------------------------

def test_linearity(oracle_lib):
    g = np.random.default_rng(3)
    # integer-valued maps so that 3 L1 - 2 L2 is exact in FP32
    L1 = g.integers(0, 1000, (23, 19)).astype(np.float32)
    L2 = g.integers(0, 1000, (23, 19)).astype(np.float32)
    K = g.uniform(0.0, 1.0, (9, 7))
    lhs = oracle_lib.conv_full(3.0 * L1 - 2.0 * L2, K)
    rhs = 3.0 * oracle_lib.conv_full(L1, K) - 2.0 * oracle_lib.conv_full(L2, K)
    assert _rel(lhs, rhs) < 1e-13


# --- invariant: sum(Bfull) = sum(L) sum(K) ------------------------------------

def test_sum_invariant(oracle_lib):
    g = np.random.default_rng(4)
    L = g.lognormal(0.0, 1.5, (40, 33)).astype(np.float32)
    K = g.uniform(0.0, 1.0, (11, 13))
    B = oracle_lib.conv_full(L, K)
    s = math.fsum(L.astype(np.float64).ravel()) * math.fsum(K.ravel())
    assert abs(math.fsum(B.ravel()) - s) / s < 1e-13
    assert B.shape == (40 + 10, 33 + 12)


# --- mirror and transpose symmetry with a radial PSF --------------------------

def test_mirror_and_transpose(oracle_lib):
    g = np.random.default_rng(5)
    L = g.lognormal(0.0, 1.0, (21, 17)).astype(np.float32)
    K = synth.psf_power_exp(9, 1.0, 0.25, 1.25, 40.0)       # radial, square
    B = oracle_lib.conv_same(L, K)
    np.testing.assert_allclose(oracle_lib.conv_same(L[::-1, :], K), B[::-1, :], rtol=1e-14)
    np.testing.assert_allclose(oracle_lib.conv_same(L[:, ::-1], K), B[:, ::-1], rtol=1e-14)
    np.testing.assert_allclose(oracle_lib.conv_same(np.ascontiguousarray(L.T), K), B.T,
                               rtol=1e-14)


# --- amplitude: Gaussian * Gaussian closed form -------------------------------

@pytest.mark.parametrize("a,b", [(1.5, 2.0), (2.5, 3.0)])
def test_gaussian_closed_form(oracle_lib, a, b):
    def gauss(s, r):
        u = np.arange(-r, r + 1, dtype=np.float64)
        return np.exp(-(u[:, None] ** 2 + u[None, :] ** 2) / (2 * s * s))
    ra, rb = int(math.ceil(8 * a)), int(math.ceil(8 * b))
    L = gauss(a, ra).astype(np.float32)
    K = gauss(b, rb)
    B = oracle_lib.conv_full(L, K)
    c = np.sqrt(a * a + b * b)
    amp = 2 * np.pi * a * a * b * b / (a * a + b * b)
    # Bfull[ra+rb+di][ra+rb+dj] is the convolution at offset (di, dj)
    r = ra + rb
    u = np.arange(B.shape[0], dtype=np.float64) - r
    expect = amp * np.exp(-(u[:, None] ** 2 + u[None, :] ** 2) / (2 * c * c))
    # FP32 rounding of L (2^-24 relative, all terms positive) bounds the error
    assert np.max(np.abs(B - expect)) / amp < 2e-7
    assert abs(B[r, r] / amp - 1.0) < 2e-7


# --- separable PSF reduces to two 1-D numpy.convolve passes -----------------

def test_separable_kernel_matches_numpy_convolve(oracle_lib):
    g = np.random.default_rng(6)
    L = g.uniform(0.0, 5.0, (30, 26)).astype(np.float32)
    ky = g.uniform(0.0, 1.0, 7)
    kx = g.uniform(0.0, 1.0, 11)
    K = np.outer(ky, kx)
    Ld = L.astype(np.float64)
    rows = np.array([np.convolve(r, kx) for r in Ld])                # along j
    ref = np.array([np.convolve(c, ky) for c in rows.T]).T            # along i
    assert _rel(oracle_lib.conv_full(L, K), ref) < 1e-13


# --- brute force on tiny inputs against an FP64 numpy FFT ---------------------

@pytest.mark.parametrize("shape,kshape", [((13, 17), (5, 7)), ((8, 8), (3, 3)), ((1, 9), (1, 5))])
def test_tiny_against_numpy_fft(oracle_lib, shape, kshape):
    g = np.random.default_rng(7)
    L = g.standard_normal(shape).astype(np.float32)
    K = g.standard_normal(kshape)
    Ho, Wo = shape[0] + kshape[0] - 1, shape[1] + kshape[1] - 1
    ref = np.fft.irfft2(np.fft.rfft2(L.astype(np.float64), (Ho, Wo)) *
                        np.fft.rfft2(K, (Ho, Wo)), (Ho, Wo))
    assert _rel(oracle_lib.conv_full(L, K), ref) < 1e-12


def test_points_agree_with_full_map(oracle_lib):
    g = np.random.default_rng(8)
    L = g.lognormal(0.0, 1.0, (31, 29)).astype(np.float32)
    K = g.uniform(0.0, 1.0, (9, 5))
    B = oracle_lib.conv_full(L, K)
    ii = g.integers(-3, B.shape[0] + 3, 400)
    jj = g.integers(-3, B.shape[1] + 3, 400)
    inside = (ii >= 0) & (jj >= 0) & (ii < B.shape[0]) & (jj < B.shape[1])
    got = oracle_lib.conv_points_full(L, K, ii, jj)
    np.testing.assert_array_equal(got[inside], B[ii[inside], jj[inside]])
    assert np.all(got[~inside] == 0.0)
    Bs = oracle_lib.conv_same(L, K)
    si, sj = g.integers(0, 31, 50), g.integers(0, 29, 50)
    np.testing.assert_array_equal(oracle_lib.conv_points_same(L, K, si, sj), Bs[si, sj])


def test_multiclass_sum_eq4(oracle_lib):
    g = np.random.default_rng(9)
    L1 = g.integers(0, 100, (15, 14)).astype(np.float32)
    L2 = g.integers(0, 100, (15, 14)).astype(np.float32)
    K1 = g.uniform(0, 1, (5, 5))
    K2 = g.uniform(0, 1, (5, 5))
    ii, jj = np.meshgrid(np.arange(15), np.arange(14), indexing="ij")
    got = oracle_lib.conv_multiclass_points_same([L1, L2], [K1, K2], ii, jj).reshape(15, 14)
    ref = oracle_lib.conv_same(L1, K1) + oracle_lib.conv_same(L2, K2)
    np.testing.assert_allclose(got, ref, rtol=1e-14)
    # one class with the same PSF is linear in the map
    same = oracle_lib.conv_multiclass_points_same([L1, L2], [K1, K1], ii, jj).reshape(15, 14)
    np.testing.assert_allclose(same, oracle_lib.conv_same(L1 + L2, K1), rtol=1e-13)


# --- Eq. (10): the DFT ---------------------------------------------------------

def test_dft_hand_worked(oracle_lib):
    g = read_blocks("dft_hand_2x3.txt")
    F = g["F"]
    got = oracle_lib.dft2_points(g["f"], F[:, 0].astype(int), F[:, 1].astype(int))
    np.testing.assert_allclose(got.real, F[:, 2], atol=1e-13)
    np.testing.assert_allclose(got.imag, F[:, 3], atol=1e-13)


def test_dft_delta_closed_form(oracle_lib):
    N, M, n0, m0 = 12, 10, 5, 3
    f = np.zeros((N, M))
    f[n0, m0] = 1.0
    kk, ll = np.meshgrid(np.arange(N), np.arange(M), indexing="ij")
    got = oracle_lib.dft2_points(f, kk, ll).reshape(N, M)
    ref = np.exp(-2j * np.pi * (kk * n0 / N + ll * m0 / M))
    np.testing.assert_allclose(got, ref, atol=1e-14)


def test_dft_against_numpy_and_parseval(oracle_lib):
    g = np.random.default_rng(10)
    N, M = 9, 14
    f = g.standard_normal((N, M))
    kk, ll = np.meshgrid(np.arange(N), np.arange(M), indexing="ij")
    got = oracle_lib.dft2_points(f, kk, ll).reshape(N, M)
    np.testing.assert_allclose(got, np.fft.fft2(f), atol=1e-12)
    assert abs(np.sum(np.abs(got) ** 2) / (N * M) - np.sum(f * f)) < 1e-11
    # real input: Hermitian symmetry F(N-k, M-l) = conj F(k, l)
    np.testing.assert_allclose(got[(-kk) % N, (-ll) % M], np.conj(got), atol=1e-12)
    # constant: all energy in the zero frequency
    c = oracle_lib.dft2_points(np.ones((N, M)), kk, ll).reshape(N, M)
    assert abs(c[0, 0] - N * M) < 1e-12
    c[0, 0] = 0
    assert np.max(np.abs(c)) < 1e-12


# --- the paper's worked cost example ------------------------------------------

def test_cost_model_worked_example(oracle_lib):
    with open(os.path.join(GOLDEN, "paper_constants.json")) as fh:
        ex = json.load(fh)["cost_model_example"]
    n_map = int(round(ex["map_km"] / ex["pixel_km"]))
    n_psf = int(round(ex["psf_km"] / ex["pixel_km"]))
    r = oracle_lib.op_count_ratio(n_map, n_psf)
    # "about 1e4": within half an order of magnitude
    assert 10 ** -0.5 < r / ex["claimed_ratio_order"] < 10 ** 0.5
    assert abs(r - 2000 ** 2 * 600 ** 2 / (2600 ** 2 * math.log2(2600 ** 2))) < 1e-6
