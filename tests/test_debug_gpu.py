"""The bounds-checked debug build (LP_DEBUG=1).

In the debug library every work unit of the passes checks its extents in
every buffer before it touches global memory, and a miss sets bit 3 of the
device status word instead of faulting.  Here the debug library (built for
four lengths, which covers the prefetching and the one-unit kernels, the
batched column kernel, the tensor-core pass, the tiled and the Eq. (4)
paths) runs in a child process:

* on correct calls every check passes (status word 0) and every result
  equals the release library's bitwise, and the oracle within 1e-5;
* with LP_TEST_BOUNDS (T declared one column block short) the checks of the
  last columns fire: LP_ERR_DEVICE with bit 3, no fault, and the next call
  is clean again.
"""

import json
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1907_02891_gb300 import build, lp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
DEBUG_SIZES = (96, 210, 240, 4704)
DEV = "cuda:0"


def _inputs():
    L = synth.radiance_map(200, 180, 12, 1907_02891 + 80, lit_fraction=0.05)
    g = np.random.default_rng(81)
    K1 = synth.psf_power_exp(31, 0.742, 0.1, 1.25, 80.0)
    K2 = K1 * (1.0 + 0.5 * g.random(K1.shape))          # complex spectrum
    K3 = synth.psf_power_exp(31, 0.742, 0.1, 2.0, 40.0)
    L2 = synth.radiance_map(200, 180, 12, 1907_02891 + 82, lit_fraction=0.05)
    Lt = synth.radiance_map(300, 260, 20, 1907_02891 + 83, lit_fraction=0.05)
    Lb = synth.radiance_map(600, 600, 30, 1907_02891 + 84, lit_fraction=0.05)
    return L, L2, Lt, Lb, [K1, K2, K3]


def run_cases(lp, hook=0):
    """Every case through the loaded library; returns {name: [arrays]} and
    {name: status of the lp_sync_status after it}."""
    L, L2, Lt, Lb, Ks = _inputs()
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(DEV)  # noqa: E731
    ctx = lp.lp_create(0)
    outs, status = {}, {}

    def sync(name):
        try:
            lp.lp_sync_status(ctx)
            status[name] = 0
        except lp.LpError as e:
            status[name] = e.status

    try:
        lp.lp_set_test_hook(ctx, hook)
        Ld, L2d, Ltd, Lbd = dev(L), dev(L2), dev(Lt), dev(Lb)
        sp = [lp.lp_kernel_spectrum(ctx, dev(K), max_h=200, max_w=180) for K in Ks]
        sync("spectra")
        o = [torch.empty((200, 180), device=DEV) for _ in Ks]
        lp.lp_map(ctx, Ld, sp, o)                         # batched, real and complex
        sync("same")
        outs["same"] = [x.cpu().numpy() for x in o]
        of = [torch.empty((230, 210), device=DEV)]
        lp.lp_map(ctx, Ld, sp[:1], of, mode=lp.LP_OUT_FULL)
        sync("full")
        outs["full"] = [x.cpu().numpy() for x in of]
        ss = lp.lp_kernel_spectrum(ctx, dev(Ks[0]), max_h=200, max_w=180, prec=lp.LP_PREC_SPLIT_BF16)
        os_ = [torch.empty((200, 180), device=DEV)]
        lp.lp_map(ctx, Ld, [ss], os_, prec=lp.LP_PREC_SPLIT_BF16)
        sync("split")
        outs["split"] = [x.cpu().numpy() for x in os_]
        tsp = lp.lp_kernel_spectrum(ctx, dev(Ks[0]), pad_ny=96, pad_nx=96)
        ot = [torch.empty((300, 260), device=DEV)]
        lp.lp_map_tiled(ctx, Ltd, [tsp], ot)
        sync("tiled")
        outs["tiled"] = [x.cpu().numpy() for x in ot]
        om = torch.empty((200, 180), device=DEV)
        lp.lp_map_multiclass(ctx, [Ld, L2d], sp[:1] + sp[2:3], om)
        sync("multiclass")
        outs["multiclass"] = [om.cpu().numpy()]
        bsp = [lp.lp_kernel_spectrum(ctx, dev(K), pad_ny=4704, pad_nx=4704) for K in Ks[:2]]
        ob = [torch.empty((600, 600), device=DEV) for _ in bsp]
        lp.lp_map(ctx, Lbd, bsp, ob)                      # 4704: the one-unit column kernel
        sync("len4704")
        outs["len4704"] = [x.cpu().numpy() for x in ob]
        if hook:
            lp.lp_set_test_hook(ctx, 0)
            lp.lp_map(ctx, Ld, sp, o)
            sync("after")
            outs["after"] = [x.cpu().numpy() for x in o]
        return outs, status
    finally:
        lp.lp_destroy(ctx)


_CHILD = r"""
import json, os, sys
import numpy as np
sys.path.insert(0, {root!r})
sys.path.insert(0, os.path.join({root!r}, "tests"))
from paper_1907_02891_gb300 import lp
assert lp.LIB_PATH.endswith(os.path.join("debug", "liblp.so")), lp.LIB_PATH
import test_debug_gpu as T
outs, status = T.run_cases(lp, hook={hook})
np.savez({npz!r}, **{{f"{{k}}_{{i}}": a for k, v in outs.items() for i, a in enumerate(v)}})
print(json.dumps(status))
"""


@pytest.fixture(scope="module")
def debug_lib():
    return build.build(debug=True, sizes=DEBUG_SIZES)


def _child(tmp_path, hook):
    npz = str(tmp_path / f"debug_{hook}.npz")
    env = dict(os.environ, LP_DEBUG="1")
    r = subprocess.run([sys.executable, "-c", _CHILD.format(root=ROOT, hook=hook, npz=npz)],
                       capture_output=True, text=True, env=env, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    status = json.loads(r.stdout.strip().splitlines()[-1])
    with np.load(npz) as z:
        arrays = {k: z[k] for k in z.files}
    return arrays, status


def test_debug_build_checks_pass_and_change_no_result(debug_lib, tmp_path):
    arrays, status = _child(tmp_path, 0)
    assert all(v == 0 for v in status.values()), status
    release, rstatus = run_cases(lp)
    assert all(v == 0 for v in rstatus.values()), rstatus
    for name, outs in release.items():
        for i, a in enumerate(outs):
            assert np.array_equal(arrays[f"{name}_{i}"], a), (name, i)
    L, L2, Lt, Lb, Ks = _inputs()
    for K, B in zip(Ks, release["same"]):
        ref = oracle.conv_same(L, K)
        assert np.max(np.abs(B - ref)) / np.max(np.abs(ref)) <= 1e-5
    ref = oracle.conv_same(L, Ks[0]) + oracle.conv_same(L2, Ks[2])
    B = release["multiclass"][0]
    assert np.max(np.abs(B - ref)) / np.max(np.abs(ref)) <= 1e-5


def test_debug_build_reports_a_declared_extent_miss(debug_lib, tmp_path):
    arrays, status = _child(tmp_path, lp.LP_TEST_BOUNDS)
    for name in ("same", "full", "split", "tiled", "multiclass", "len4704"):
        assert status[name] == lp.LP_ERR_DEVICE, (name, status)
    assert status["spectra"] == 0 and status["after"] == 0, status
    release, _ = run_cases(lp)
    for i, a in enumerate(release["same"]):
        assert np.array_equal(arrays[f"after_{i}"], a)
