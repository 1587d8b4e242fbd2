"""FP64 CPU oracle for the light-pollution convolution (arXiv:1907.02891).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline / reference arms of ``bench.py``.  The product library
never imports, links or runs anything here.

Functions and the passage each follows:

* ``conv_points_full`` / ``conv_full`` -- Sec. 2.3 Eq. (7) discretised (the
  full linear convolution of size N_L + N_K - 1, Sec. 2.5).
* ``conv_same`` / ``conv_points_same`` -- the same sum cropped to the map
  region (observer pixels on the source grid, Sec. 2.4 / Sec. 3: sources
  beyond the region only contribute).
* ``conv_multiclass_points_same`` -- Sec. 2.2 Eq. (4): T factorable source
  classes, B = sum_t K_t * L_t.
* ``dft2_points`` -- Sec. 2.3 Eq. (10), the 2-D DFT, by direct summation.
* ``op_count_ratio`` -- the order-of-magnitude cost comparison printed after
  Eq. (10) (direct O(N_L^2 N_K^2) against FFT O[(N_L+N_K)^2 log2 (N_L+N_K)^2]).

All pins live in ``tests/test_oracle.py``.
"""

from .oracle import (  # noqa: F401
    build,
    conv_full,
    conv_multiclass_points_same,
    conv_points_full,
    conv_points_same,
    conv_same,
    dft2_points,
    num_threads,
    op_count_ratio,
)
