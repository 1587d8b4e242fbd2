"""Serving (continuous batching) through the C ABI.

Each result must be the same alone (lp_map, one request at a time) and in
the mix (many requests in flight on several streams); the kernels are
deterministic, so the comparison is exact.  One request is also checked
against the FP64 oracle.
"""

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1907_02891_gb300 import lp  # noqa: E402

DEV = "cuda:0"


def _bank(ctx, sides, n_psf=4, psf_side=31):
    Ks = [synth.psf_power_exp(psf_side, 0.742, 0.1, p, lam)
          for (p, lam) in [(1.25, 40.0), (2.0, 80.0), (1.25, 120.0), (2.0, 200.0)][:n_psf]]
    spectra = {}
    for s in sides:
        for i, K in enumerate(Ks):
            spectra[(s, i)] = lp.lp_kernel_spectrum(ctx, torch.from_numpy(K).to(DEV), max_h=s, max_w=s)
    return Ks, spectra


def _requests(n, sides, seed):
    g = np.random.default_rng(seed)
    reqs = []
    for r in range(n):
        s = int(sides[g.integers(0, len(sides))])
        k = int(g.integers(1, 5))
        ks = [int(x) for x in g.choice(4, size=k, replace=False)]
        L = torch.from_numpy(synth.radiance_map(s, s, 6, seed * 100 + r, lit_fraction=0.02)).to(DEV)
        reqs.append((s, ks, L))
    return reqs


def test_results_same_alone_and_in_the_mix():
    sides = (64, 160, 256, 512)
    ctx = lp.lp_create(0)
    try:
        Ks, spectra = _bank(ctx, sides)
        reqs = _requests(40, sides, 3)
        alone = []
        for s, ks, L in reqs:
            outs = [torch.empty((s, s), device=DEV) for _ in ks]
            lp.lp_map(ctx, L, [spectra[(s, i)] for i in ks], outs)
            lp.lp_sync_status(ctx)
            alone.append(outs)
        lp.lp_serve_start(ctx, 4)
        mixed, tickets = [], []
        for s, ks, L in reqs:
            outs = [torch.full((s, s), float("nan"), device=DEV) for _ in ks]
            tickets.append(lp.lp_serve_submit(ctx, L, [spectra[(s, i)] for i in ks], outs))
            mixed.append(outs)
        lats = [lp.lp_serve_poll(ctx, t, timeout_ms=60000) for t in tickets]
        assert all(x is not None and x > 0 for x in lats)
        st = lp.lp_serve_stats(ctx)
        assert st["completed"] == len(reqs) and st["failed"] == 0 and st["queued"] == 0
        lp.lp_serve_stop(ctx)
        for a, b in zip(alone, mixed):
            for x, y in zip(a, b):
                assert torch.equal(x, y)
        # one request against the oracle
        s, ks, L = reqs[0]
        Lh = L.cpu().numpy()
        ref = oracle.conv_same(Lh, Ks[ks[0]])
        got = mixed[0][0].cpu().numpy().astype(np.float64)
        assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) <= 1e-5
    finally:
        lp.lp_destroy(ctx)


def test_admission_waits_for_memory_and_refuses_oversize():
    # budget: spectra + room for about one 512^2 request's workspace
    ctx = lp.lp_create(0, 64 << 20)
    try:
        Ks, spectra = _bank(ctx, (512,), n_psf=2)
        reqs = [(512, [0, 1], torch.from_numpy(synth.radiance_map(512, 512, 6, r)).to(DEV))
                for r in range(6)]
        lp.lp_serve_start(ctx, 4)
        tickets, outs_all = [], []
        for s, ks, L in reqs:
            outs = [torch.empty((s, s), device=DEV) for _ in ks]
            tickets.append(lp.lp_serve_submit(ctx, L, [spectra[(s, i)] for i in ks], outs))
            outs_all.append(outs)
        for t in tickets:
            assert lp.lp_serve_poll(ctx, t, timeout_ms=60000) is not None
        assert lp.lp_serve_stats(ctx)["failed"] == 0
        # a request whose workspace exceeds the whole serving capacity
        big = torch.zeros((8192, 8192), device=DEV)
        Kb = torch.from_numpy(synth.psf_power_exp(31, 0.742, 0.1, 1.25, 40.0)).to(DEV)
        with pytest.raises(lp.LpError) as e:
            sb = lp.lp_kernel_spectrum(ctx, Kb, max_h=8192, max_w=8192)
        assert e.value.status == lp.LP_ERR_OOM
        lp.lp_serve_stop(ctx)
    finally:
        lp.lp_destroy(ctx)


def test_serving_errors_and_bounded_poll():
    ctx = lp.lp_create(0)
    try:
        Ks, spectra = _bank(ctx, (2048,), n_psf=1)
        L = torch.from_numpy(synth.radiance_map(2048, 2048, 40, 5)).to(DEV)
        out = torch.empty_like(L)
        with pytest.raises(lp.LpError) as e:
            lp.lp_serve_submit(ctx, L, [spectra[(2048, 0)]], [out])
        assert e.value.status == lp.LP_ERR_BUSY
        lp.lp_serve_start(ctx, 2)
        with pytest.raises(lp.LpError) as e:
            lp.lp_serve_start(ctx, 2)
        assert e.value.status == lp.LP_ERR_BUSY
        with pytest.raises(lp.LpError) as e:
            lp.lp_serve_poll(ctx, 12345, 0)
        assert e.value.status == lp.LP_ERR_INVALID
        outs = [torch.empty_like(L) for _ in range(8)]
        ts = [lp.lp_serve_submit(ctx, L, [spectra[(2048, 0)]], [o]) for o in outs]
        assert lp.lp_serve_poll(ctx, ts[-1], timeout_ms=0) is None      # still running
        for t in ts:
            assert lp.lp_serve_poll(ctx, t, timeout_ms=-1) is not None
        for o in outs[1:]:
            assert torch.equal(o, outs[0])
        lp.lp_serve_stop(ctx)
    finally:
        lp.lp_destroy(ctx)


def test_split_precision_requests_same_alone_and_in_the_mix():
    """The scheduler runs split-BF16 spectra too (the request takes the
    spectra's precision); results equal lp_map's bitwise."""
    ctx = lp.lp_create(0)
    try:
        sides = (256, 512)
        Ks = [synth.psf_power_exp(31, 0.742, 0.1, p, lam) for (p, lam) in [(1.25, 40.0), (2.0, 80.0)]]
        spectra = {(s, i): lp.lp_kernel_spectrum(ctx, torch.from_numpy(K).to(DEV), max_h=s, max_w=s,
                                                 prec=lp.LP_PREC_SPLIT_BF16)
                   for s in sides for i, K in enumerate(Ks)}
        reqs = []
        for r in range(12):
            s = sides[r % 2]
            ks = [0, 1] if r % 3 == 0 else [r % 2]
            reqs.append((s, ks, torch.from_numpy(synth.radiance_map(s, s, 6, 700 + r)).to(DEV)))
        alone = []
        for s, ks, L in reqs:
            outs = [torch.empty((s, s), device=DEV) for _ in ks]
            lp.lp_map(ctx, L, [spectra[(s, i)] for i in ks], outs, prec=lp.LP_PREC_SPLIT_BF16)
            alone.append(outs)
        lp.lp_sync_status(ctx)
        lp.lp_serve_start(ctx, 3)
        mixed, tickets = [], []
        for s, ks, L in reqs:
            outs = [torch.full((s, s), float("nan"), device=DEV) for _ in ks]
            tickets.append(lp.lp_serve_submit(ctx, L, [spectra[(s, i)] for i in ks], outs))
            mixed.append(outs)
        for t in tickets:
            assert lp.lp_serve_poll(ctx, t, timeout_ms=60000) is not None
        lp.lp_serve_stop(ctx)
        for a, b in zip(alone, mixed):
            for x, y in zip(a, b):
                assert torch.equal(x, y)
        s, ks, L = reqs[1]
        ref = oracle.conv_same(L.cpu().numpy(), Ks[ks[0]])
        got = mixed[1][0].cpu().numpy().astype(np.float64)
        assert np.max(np.abs(got - ref)) / np.max(np.abs(ref)) <= 2e-4
    finally:
        lp.lp_destroy(ctx)


def test_release_mid_run_does_not_stall_the_slots():
    """Spectra released while requests are queued or running: the requests
    hold their own references, so they finish with correct results; a
    spectrum whose last use has completed is freed at once; no release
    waits for the device, so the slots are still busy right after it."""
    ctx = lp.lp_create(0)
    try:
        Ks, spectra = _bank(ctx, (8192, 256), n_psf=4, psf_side=201)
        L = torch.from_numpy(synth.radiance_map(8192, 8192, 1600, 9)).to(DEV)
        ref = [torch.empty((8192, 8192), device=DEV) for _ in range(4)]
        lp.lp_map(ctx, L, [spectra[(8192, i)] for i in range(4)], ref)
        lp.lp_sync_status(ctx)
        lp.lp_serve_start(ctx, 2)
        # size both slots' workspaces first, so that nothing else allocates below
        wouts = [[torch.empty((8192, 8192), device=DEV) for _ in range(4)] for _ in range(2)]
        warm = [lp.lp_serve_submit(ctx, L, [spectra[(8192, i)] for i in range(4)], w) for w in wouts]
        for t in warm:
            assert lp.lp_serve_poll(ctx, t, timeout_ms=60000) is not None
        outs = [[torch.full((8192, 8192), float("nan"), device=DEV) for _ in range(4)] for _ in range(4)]
        tickets = [lp.lp_serve_submit(ctx, L, [spectra[(8192, i)] for i in range(4)], o) for o in outs]
        for i in range(4):                      # drop the caller's references
            lp.lp_spectrum_release(ctx, spectra[(8192, i)])
        held = lp.lp_bytes_in_use(ctx)
        lp.lp_spectrum_release(ctx, spectra[(256, 0)])   # unused by the queue: freed at once
        assert lp.lp_serve_poll(ctx, tickets[-1], timeout_ms=0) is None, "a release waited for the device"
        assert lp.lp_bytes_in_use(ctx) < held
        for t in tickets:
            assert lp.lp_serve_poll(ctx, t, timeout_ms=60000) is not None
        lp.lp_serve_stop(ctx)
        for o in outs:
            for x, y in zip(o, ref):
                assert torch.equal(x, y)
    finally:
        lp.lp_destroy(ctx)


def test_request_log_lines(tmp_path):
    """The per-request JSON-lines log: one line per finished request, with
    its sizes and host-clock times in order (submit <= start <= end) and the
    latency lp_serve_poll returned."""
    import json
    sides = (64, 256)
    ctx = lp.lp_create(0)
    try:
        _, spectra = _bank(ctx, sides)
        reqs = _requests(12, sides, 5)
        lp.lp_serve_start(ctx, 2)
        with pytest.raises(lp.LpError):
            lp.lp_serve_log(ctx, str(tmp_path / "no_such_dir" / "x.jsonl"))
        path = tmp_path / "serve.jsonl"
        lp.lp_serve_log(ctx, path)
        outs, tickets = [], []
        for s, ks, L in reqs:
            o = [torch.empty((s, s), device=DEV) for _ in ks]
            tickets.append(lp.lp_serve_submit(ctx, L, [spectra[(s, i)] for i in ks], o))
            outs.append(o)
        lats = {t: lp.lp_serve_poll(ctx, t, timeout_ms=60000) for t in tickets}
        lp.lp_serve_stop(ctx)   # closes the log
        lines = [json.loads(x) for x in path.read_text().splitlines()]
        assert sorted(r["ticket"] for r in lines) == sorted(tickets)
        by = {r["ticket"]: r for r in lines}
        for t, (s, ks, _) in zip(tickets, reqs):
            r = by[t]
            assert r["status"] == 0 and r["h"] == s and r["w"] == s and r["n_psf"] == len(ks)
            assert r["mode"] == lp.LP_OUT_SAME and r["precision"] == lp.LP_PREC_FP32
            assert r["workspace_bytes"] > 0
            assert abs(r["output_mpix"] - s * s * len(ks) / 1e6) < 1e-6
            assert 0 <= r["submit_ms"] <= r["start_ms"] <= r["end_ms"]
            assert abs(r["latency_ms"] - (r["end_ms"] - r["submit_ms"])) < 1e-2
            assert abs(r["queue_ms"] - (r["start_ms"] - r["submit_ms"])) < 1e-2
            assert abs(r["latency_ms"] - lats[t]) < 1e-3
    finally:
        lp.lp_destroy(ctx)


def test_cancel_a_queued_request():
    """One slot, two long requests ahead: a request cancelled while queued
    never runs (its output keeps its NaNs) and polls as LP_ERR_CANCELLED; a
    running or finished one cannot be cancelled; the rest are unaffected."""
    ctx = lp.lp_create(0)
    try:
        _, spectra = _bank(ctx, (8192, 256), n_psf=4, psf_side=201)
        big = torch.from_numpy(synth.radiance_map(8192, 8192, 400, 21)).to(DEV)
        small = torch.from_numpy(synth.radiance_map(256, 256, 8, 22)).to(DEV)
        ref = torch.empty_like(small)
        lp.lp_map(ctx, small, [spectra[(256, 0)]], [ref])
        lp.lp_sync_status(ctx)
        lp.lp_serve_start(ctx, 1)
        bouts = [[torch.empty_like(big) for _ in range(4)] for _ in range(2)]
        t_big = [lp.lp_serve_submit(ctx, big, [spectra[(8192, i)] for i in range(4)], o) for o in bouts]
        o_cancel = torch.full_like(small, float("nan"))
        o_keep = torch.full_like(small, float("nan"))
        t_cancel = lp.lp_serve_submit(ctx, small, [spectra[(256, 0)]], [o_cancel])
        t_keep = lp.lp_serve_submit(ctx, small, [spectra[(256, 0)]], [o_keep])
        lp.lp_serve_cancel(ctx, t_cancel)
        with pytest.raises(lp.LpError) as e:
            lp.lp_serve_cancel(ctx, t_cancel)          # no longer queued
        assert e.value.status == lp.LP_ERR_BUSY
        with pytest.raises(lp.LpError) as e:
            lp.lp_serve_cancel(ctx, 10 ** 9)
        assert e.value.status == lp.LP_ERR_INVALID
        with pytest.raises(lp.LpError) as e:
            lp.lp_serve_poll(ctx, t_cancel, timeout_ms=1000)
        assert e.value.status == lp.LP_ERR_CANCELLED
        for t in t_big + [t_keep]:
            assert lp.lp_serve_poll(ctx, t, timeout_ms=60000) is not None
        with pytest.raises(lp.LpError) as e:
            lp.lp_serve_cancel(ctx, t_big[0])          # finished
        assert e.value.status == lp.LP_ERR_BUSY
        st = lp.lp_serve_stats(ctx)
        assert st["completed"] == 3 and st["failed"] == 0 and st["queued"] == 0
        lp.lp_serve_stop(ctx)
        assert torch.isnan(o_cancel).all()
        assert torch.equal(o_keep, ref)
    finally:
        lp.lp_destroy(ctx)


def test_injected_launch_failure_fails_one_request_only():
    """LP_TEST_SERVE_FAIL (host-side injection): the next admitted request
    fails with LP_ERR_CUDA and frees its slot; the others, before and after,
    finish with the results they have alone."""
    sides = (64, 256)
    ctx = lp.lp_create(0)
    try:
        _, spectra = _bank(ctx, sides)
        reqs = _requests(6, sides, 11)
        alone = []
        for s, ks, L in reqs:
            o = [torch.empty((s, s), device=DEV) for _ in ks]
            lp.lp_map(ctx, L, [spectra[(s, i)] for i in ks], o)
            alone.append(o)
        lp.lp_sync_status(ctx)
        lp.lp_serve_start(ctx, 1)
        outs, tickets = [], []
        for r, (s, ks, L) in enumerate(reqs):
            if r == 2:   # the first two have run; the next admitted request fails
                for t in tickets:
                    assert lp.lp_serve_poll(ctx, t, timeout_ms=60000) is not None
                lp.lp_set_test_hook(ctx, lp.LP_TEST_SERVE_FAIL)
            o = [torch.full((s, s), float("nan"), device=DEV) for _ in ks]
            tickets.append(lp.lp_serve_submit(ctx, L, [spectra[(s, i)] for i in ks], o))
            outs.append(o)
        status = []
        for t in tickets[2:]:
            try:
                lp.lp_serve_poll(ctx, t, timeout_ms=60000)
                status.append(lp.LP_OK)
            except lp.LpError as e:
                status.append(e.status)
        assert status == [lp.LP_ERR_CUDA, lp.LP_OK, lp.LP_OK, lp.LP_OK]
        st = lp.lp_serve_stats(ctx)
        assert st["failed"] == 1 and st["completed"] == 5
        lp.lp_serve_stop(ctx)
        for r, (a, b) in enumerate(zip(alone, outs)):
            for x, y in zip(a, b):
                if r == 2:
                    assert torch.isnan(y).all()
                else:
                    assert torch.equal(x, y)
    finally:
        lp.lp_set_test_hook(ctx, 0)
        lp.lp_destroy(ctx)
