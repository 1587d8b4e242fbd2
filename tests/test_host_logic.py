"""Host-side logic that needs no GPU: the byte model behind the bench's
roofline, the plan table the library is built from, the bench's kernel
fingerprint, and the host-core FFT comparator against the oracle."""

import json
import os

import numpy as np
import pytest

import oracle
import synth

import bench
from paper_1907_02891_gb300 import build as B
from paper_1907_02891_gb300 import tune


def test_three_pass_byte_model_at_the_bench_workload():
    # 4096^2 map, 541^2 point-symmetric PSF (real spectrum, 4 bytes per
    # bin), padded 4704^2, one spectrum: 4HW + 16 H (Nx/2+1) + s_K Ny
    # (Nx/2+1) + 16 H (Nx/2+1) + 4HW = 487 MB
    m = bench.pass_bytes(4096, 4096, 4704, 4704, 1, 4)
    nc = 4704 // 2 + 1
    assert m["p1_rows"] == 4 * 4096 * 4096 + 8 * 4096 * nc
    assert m["p2_cols"] == 8 * 4096 * nc + 4 * 4704 * nc + 8 * 4096 * nc
    assert m["p3_rows"] == 8 * 4096 * nc + 4 * 4096 * 4096
    assert abs(sum(m.values()) / 1e6 - 487.0) < 1.0
    # n spectra share P1's bytes; P2 and P3 scale with n
    m16 = bench.pass_bytes(4096, 4096, 4704, 4704, 16, 4)
    assert m16["p1_rows"] == m["p1_rows"]
    assert m16["p3_rows"] == 16 * m["p3_rows"]


def _seven_smooth(n):
    for p in (2, 3, 5, 7):
        while n % p == 0:
            n //= p
    return n == 1


def test_plan_table_is_consistent():
    table = B.plan_table()
    assert sorted(table) == sorted(B.SIZES)
    for n, p in table.items():
        assert _seven_smooth(n), n
        r = p["radices"]
        assert int(np.prod(r)) == n and max(r) <= 32 and all(x in B.RADICES for x in r), (n, r)
        assert p["threads"] <= B.MAX_THREADS
        assert len(p["upb"]) == len(p["minb"]) == len(p["pf"]) == len(p["db"]) == 3
        assert all(1 <= u <= 3 for u in p["upb"]) and all(1 <= b <= 3 for b in p["minb"])
        assert isinstance(p["batch"], bool)


def test_tuned_plans_record_their_workload_and_knobs():
    with open(B.TUNED_JSON) as fh:
        tuned = json.load(fh)
    for n, e in tuned.items():
        assert int(n) in B.SIZES
        assert tune._prod(e["radices"]) == int(n)
        assert e["tuned_total_us"] > 0


def test_fingerprint_ignores_notes_but_not_knobs(tmp_path, monkeypatch):
    with open(B.TUNED_JSON) as fh:
        tuned = json.load(fh)
    e = dict(tuned["4704"])
    base = bench.kernel_source_sha(lengths=(4704,))
    alt = dict(tuned)
    alt["4704"] = dict(e, note="another note", tuned_total_us=1.0)
    p = tmp_path / "plans.json"
    p.write_text(json.dumps(alt))
    monkeypatch.setattr(bench, "TUNED_PLANS", os.path.relpath(p, bench.ROOT))
    assert bench.kernel_source_sha(lengths=(4704,)) == base
    alt["4704"] = dict(e, minb=[3, 3, 3])
    p.write_text(json.dumps(alt))
    assert bench.kernel_source_sha(lengths=(4704,)) != base
    monkeypatch.setattr(bench, "TUNED_PLANS", os.path.relpath(B.TUNED_JSON, bench.ROOT))
    assert bench.kernel_source_sha(lengths=(4704,)) == base
    # the generated sources' template and the compiler flags are part of it
    monkeypatch.setattr(B, "NVCC_FLAGS", B.NVCC_FLAGS + ["-DX"])
    assert bench.kernel_source_sha(lengths=(4704,)) != base
    monkeypatch.undo()
    monkeypatch.setattr(B, "_SIZE_TU", B._SIZE_TU + "\n")
    assert bench.kernel_source_sha(lengths=(4704,)) != base


def test_tune_cache_env_names_the_plan_file(tmp_path, monkeypatch):
    """$LP_TUNE_CACHE replaces tuned_plans.json for the build's plan table,
    the tuner's default output and the bench's kernel fingerprint."""
    with open(B.TUNED_JSON) as fh:
        tuned = json.load(fh)
    base_plan = B.plan_table()[4704]
    base_sha = bench.kernel_source_sha(lengths=(4704,))
    alt = dict(tuned)
    alt["4704"] = dict(tuned["4704"], radices=[14, 16, 21], minb=[1, 1, 1])
    p = tmp_path / "plans.json"
    p.write_text(json.dumps(alt))
    monkeypatch.setenv("LP_TUNE_CACHE", str(p))
    assert B.tuned_json_path() == str(p)
    got = B.plan_table()[4704]
    assert got["radices"] == [14, 16, 21] and got["minb"] == [1, 1, 1]
    assert got["threads"] == B.threads_for(4704, [14, 16, 21])
    assert bench.kernel_source_sha(lengths=(4704,)) != base_sha
    monkeypatch.delenv("LP_TUNE_CACHE")
    assert B.tuned_json_path() == B.TUNED_JSON
    assert B.plan_table()[4704] == base_plan
    assert bench.kernel_source_sha(lengths=(4704,)) == base_sha


def test_host_fft_comparator_computes_eq7():
    pytest.importorskip("scipy")
    oracle.build()
    wl = synth.WORKLOADS["map256_psf101"]
    L, K = wl.radiance(), wl.psfs()[0]
    ref = oracle.conv_same(L, K)
    for dt, tol in ((np.float64, 1e-12), (np.float32, 1e-5)):
        got = bench.host_fft_map(L, bench.host_fft_spectrum(K, 360, 360, dt), 360, 360, dt)
        assert got.shape == (256, 256)
        assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) < tol
    r = bench.cpu_fft_comparator(L, [K], 360, 360, reps=1)
    assert r["fp64"] > 0 and r["fp32"] > 0
