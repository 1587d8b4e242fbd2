"""Seeded synthetic inputs shared by the tests, the smoke check and the bench.

This module only draws inputs: radiance maps shaped like the paper's
satellite-radiance workloads, sampled PSF matrices, pixel samples and request
streams.  It holds none of the method's arithmetic (no transform, no
convolution) and imports neither the oracle nor the product library.

The paper's own data (the VIIRS 2016 "vcm-orm-ntl" composite reprojected to a
404.4 m UTM grid, Sec. 3, and the LPTRAN PSF it cites) are not available, so
these generators stand in for them: non-negative, mostly dark maps of
Gaussian city blobs with log-normal peak radiance, optionally a sparse field
of isolated lit pixels, up to a 1e6 dynamic range.

Random generator: numpy ``Generator(PCG64(seed))``; the per-workload seed is
1907_02891 + workload index.
"""

from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

BASE_SEED = 1907_02891


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def radiance_map(H: int, W: int, n_cities: int, seed: int,
                 lit_fraction: float = 0.0,
                 lit_range: Optional[Tuple[float, float]] = None,
                 clip_range: Optional[Tuple[float, float]] = None) -> np.ndarray:
    """FP32 H x W radiance map L1 (row-major), background 0.

    * ``n_cities`` blobs: centre uniform in [0,H) x [0,W), sigma ~ U(1,5) px,
      peak ~ LogNormal(0, 1.5); each adds peak*exp(-d^2 / 2 sigma^2) inside a
      +-ceil(5 sigma) pixel window.
    * ``lit_fraction``: Bernoulli mask of isolated lit pixels; their values
      are LogNormal(0, 1.5), or log-uniform in ``lit_range`` when given.
    * ``clip_range`` (lo, hi): after generation values < lo become 0 and
      values > hi become hi (the 1e-3..1e3 dynamic-range workload).
    """
    g = rng(seed)
    L = np.zeros((H, W), dtype=np.float64)
    cy = g.uniform(0.0, H, n_cities)
    cx = g.uniform(0.0, W, n_cities)
    sig = g.uniform(1.0, 5.0, n_cities)
    peak = g.lognormal(0.0, 1.5, n_cities)
    for y0, x0, s, a in zip(cy, cx, sig, peak):
        r = int(math.ceil(5.0 * s))
        i0, i1 = max(0, int(y0) - r), min(H, int(y0) + r + 1)
        j0, j1 = max(0, int(x0) - r), min(W, int(x0) + r + 1)
        if i0 >= i1 or j0 >= j1:
            continue
        di = np.arange(i0, i1, dtype=np.float64)[:, None] - y0
        dj = np.arange(j0, j1, dtype=np.float64)[None, :] - x0
        L[i0:i1, j0:j1] += a * np.exp(-(di * di + dj * dj) / (2.0 * s * s))
    L = L.astype(np.float32)
    if lit_fraction > 0.0:
        # row blocks keep the temporary at a few hundred MB for 16384^2 maps
        rows = max(1, (1 << 24) // max(W, 1))
        for r0 in range(0, H, rows):
            r1 = min(H, r0 + rows)
            mask = g.random((r1 - r0, W)) < lit_fraction
            cnt = int(mask.sum())
            if lit_range is None:
                vals = g.lognormal(0.0, 1.5, cnt)
            else:
                lo, hi = lit_range
                vals = np.exp(g.uniform(math.log(lo), math.log(hi), cnt))
            blk = L[r0:r1]
            blk[mask] += vals.astype(np.float32)
    if clip_range is not None:
        lo, hi = clip_range
        L[L < lo] = 0.0
        np.minimum(L, np.float32(hi), out=L)
    return L


def radial_grid(n: int, px_km: float) -> np.ndarray:
    """Distance in km of each cell of an n x n PSF matrix from its centre."""
    if n % 2 == 0:
        raise ValueError("PSF side must be odd")
    c = (n - 1) // 2
    u = np.arange(n, dtype=np.float64) - c
    return px_km * np.hypot(u[:, None], u[None, :])


def psf_power_exp(n: int, px_km: float, a: float, p: float, lam_km: float) -> np.ndarray:
    """FP64 PSF K(r) = (r^2 + a)^(-p) * exp(-r / lam), r in km, square support
    with corners included, centre at the middle element.  Not normalised."""
    r = radial_grid(n, px_km)
    return (r * r + a) ** (-p) * np.exp(-r / lam_km)


def psf_alr(n: int, px_km: float) -> np.ndarray:
    """All-sky light-pollution-ratio PSF of Sec. 3, Eq. (12)-(13):
    K(d) = c d^(-alpha(d)), alpha(d) = 2.3 (d/350)^0.28, c = 1/562.72, d in
    km.  At d = 0 the limit is c (alpha -> 0 faster than log d diverges)."""
    d = radial_grid(n, px_km)
    c = 1.0 / 562.72
    out = np.full_like(d, c)
    nz = d > 0
    alpha = 2.3 * (d[nz] / 350.0) ** 0.28
    out[nz] = c * d[nz] ** (-alpha)
    return out


def sample_pixels(H: int, W: int, n: int, seed: int) -> Tuple[np.ndarray, np.ndarray]:
    """n seeded uniform map pixels (with repetition)."""
    g = rng(seed)
    return g.integers(0, H, n, dtype=np.int64), g.integers(0, W, n, dtype=np.int64)


# ----------------------------------------------------------------------------
# Workloads
# ----------------------------------------------------------------------------

@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    H: int
    W: int
    px_km: float
    n_cities: int
    lit_fraction: float
    lit_range: Optional[Tuple[float, float]]
    clip_range: Optional[Tuple[float, float]]
    psf_side: int
    psf_params: Tuple[Tuple[float, float, float], ...]  # (a, p, lam_km) per PSF
    seed: int

    def radiance(self) -> np.ndarray:
        return radiance_map(self.H, self.W, self.n_cities, self.seed,
                            self.lit_fraction, self.lit_range, self.clip_range)

    def psfs(self) -> List[np.ndarray]:
        return [psf_power_exp(self.psf_side, self.px_km, a, p, lam)
                for (a, p, lam) in self.psf_params]


def _family(a: float, ps: Sequence[float], lams: Sequence[float]):
    return tuple((a, p, lam) for lam in lams for p in ps)


WORKLOADS = {
    # 256^2 map, 1 km pixels, 12 cities, 101^2 PSF (r^2+0.25)^-1.25 e^(-r/40 km)
    "map256_psf101": Workload("map256_psf101", 256, 256, 1.0, 12, 0.0, None, None,
                              101, ((0.25, 1.25, 40.0),), BASE_SEED + 0),
    # 4096^2 map, 0.742 km pixels, 400 cities + 5% lit pixels, 541^2 PSF
    "map4096_psf541": Workload("map4096_psf541", 4096, 4096, 0.742, 400, 0.05, None, None,
                               541, ((0.1, 1.25, 80.0),), BASE_SEED + 1),
    # 8192^2 map, 1600 cities + 5% lit, 16 PSFs of side 601 (4 lambda x 4 p)
    "map8192_psf601x16": Workload("map8192_psf601x16", 8192, 8192, 0.742, 1600, 0.05, None,
                                  None, 601,
                                  _family(0.1, (1.0, 1.25, 1.5, 2.0), (40.0, 80.0, 120.0, 200.0)),
                                  BASE_SEED + 2),
    # 16384^2 map, 6400 cities, lit field log-uniform 1e-3..1e3, clipped to it
    "map16384_psf801": Workload("map16384_psf801", 16384, 16384, 0.742, 6400, 0.05,
                                (1e-3, 1e3), (1e-3, 1e3), 801, ((0.1, 1.25, 80.0),),
                                BASE_SEED + 3),
    # 17800 x 21000 map (longer than the longest FFT length): the tiled form,
    # same generator and PSF as the 16384^2 workload
    "map17800x21000_psf801": Workload("map17800x21000_psf801", 17800, 21000, 0.742, 8900, 0.05,
                                      None, None, 801, ((0.1, 1.25, 80.0),), BASE_SEED + 6),
}

# The paper's own shape (Sec. 3): an 11920 x 11804 map of 404.4 m pixels and
# two maps from it -- the all-sky light-pollution ratio PSF of Eq. (12)-(13)
# out to 300 km (1485 x 1485 support) and a zenith-brightness stand-in out to
# the 195 km reach used for the LPTRAN PSF (965 x 965 support; the LPTRAN
# values are not available, a power-law-exponential PSF stands in).
PAPER_SHAPE = dict(name="map11920x11804_alr1485_zsb965", H=11920, W=11804, px_km=0.4044,
                   n_cities=3300, lit_fraction=0.05, seed=BASE_SEED + 5,
                   alr_side=1485, zsb_side=965)


def paper_shape_inputs():
    """Radiance map and the two PSFs (ALR Eq. (12)-(13); ZSB stand-in)."""
    p = PAPER_SHAPE
    L = radiance_map(p["H"], p["W"], p["n_cities"], p["seed"], lit_fraction=p["lit_fraction"])
    K_alr = psf_alr(p["alr_side"], p["px_km"])
    K_zsb = psf_power_exp(p["zsb_side"], p["px_km"], 0.1, 1.25, 26.0)
    return L, [K_alr, K_zsb]


# Serving bank: 8 PSFs of side 201 (radius 100 px), lambda x p in {1.25, 2.0}
SERVE_BANK_PARAMS = _family(0.1, (1.25, 2.0), (40.0, 80.0, 120.0, 200.0))
SERVE_PSF_SIDE = 201
SERVE_PX_KM = 0.742
SERVE_TILE_SIDES = (256, 512, 1024, 2048, 4096, 8192)
SERVE_SEED = BASE_SEED + 4


def serve_bank() -> List[np.ndarray]:
    return [psf_power_exp(SERVE_PSF_SIDE, SERVE_PX_KM, a, p, lam)
            for (a, p, lam) in SERVE_BANK_PARAMS]


@dataclasses.dataclass(frozen=True)
class Request:
    arrival_s: float
    side: int
    kernels: Tuple[int, ...]
    seed: int


def request_stream(n: int, rate_hz: float, seed: int = SERVE_SEED,
                   sides: Sequence[int] = SERVE_TILE_SIDES,
                   max_kernels: int = 8, bank_size: int = 8) -> List[Request]:
    """Poisson arrivals (exponential gaps at ``rate_hz``); tile side uniform
    on ``sides``; 1..max_kernels PSFs drawn without replacement from the
    bank."""
    g = rng(seed)
    t = 0.0
    out = []
    for r in range(n):
        t += g.exponential(1.0 / rate_hz)
        side = int(sides[g.integers(0, len(sides))])
        k = int(g.integers(1, max_kernels + 1))
        ks = tuple(int(x) for x in g.choice(bank_size, size=k, replace=False))
        out.append(Request(t, side, ks, seed * 1000 + r))
    return out
