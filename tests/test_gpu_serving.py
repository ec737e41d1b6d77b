"""Serving (ext_submit / ext_poll / ext_drain): continuous batching on the GPU.

Requests of mixed sizes, boundary rules and directions are submitted while others are running;
each result must equal what ext_solve gives for that request alone (bit for bit: every slot runs
the same kernels and its reductions do not depend on the other slots), and admission by HBM
footprint must refuse requests larger than the budget.
"""

import threading
import time

import numpy as np
import pytest
import torch

from paper_1704_08897_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ext():
    assert torch.cuda.is_available()
    from paper_1704_08897_gb300 import build_ext, ext as e
    build_ext.build()
    e.load()
    return e


def _stream(count, seed):
    reqs = synth.serving_stream(count=count, rate=400.0, seed=seed, side_lo=48, side_hi=200)
    return [r.problem for r in reqs], [r.arrival_s for r in reqs]


@pytest.mark.parametrize("prec", ["fp32", "mixed_bf16"])
def test_served_results_equal_solo_results(ext, prec):
    probs, arrivals = _stream(24, 11)
    solo = ext.ext_create(ext.options(prec))
    served = ext.ext_create(ext.options(prec, max_slots=8))
    try:
        ref = []
        for p in probs:
            out = torch.empty(p.phi.shape, device="cuda")
            r = ext.ext_solve(solo, ext.problem_of(p), torch.from_numpy(p.phi).cuda(),
                              torch.from_numpy(p.f).cuda(), out)
            ref.append((r, out))
        phis = [torch.from_numpy(p.phi).cuda() for p in probs]
        fs = [torch.from_numpy(p.f).cuda() for p in probs]
        outs = [torch.full(p.phi.shape, float("nan"), device="cuda") for p in probs]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        tickets = []
        for p, a, phi, f, o in zip(probs, arrivals, phis, fs, outs):
            while time.perf_counter() - t0 < a:  # arrivals while earlier requests are running
                time.sleep(1e-4)
            tickets.append(ext.ext_submit(served, ext.problem_of(p), phi, f, o))
        ext.ext_drain(served)
        for (r1, o1), t, o2 in zip(ref, tickets, outs):
            r2 = ext.ext_poll(served, t)
            assert r2["rc"] == 0 and r2["status"] == 0
            assert r2["iters"] == r1["iters"]
            assert torch.equal(o1, o2)
            assert r2["ms_queue"] >= 0 and r2["ms_solve"] > 0
        assert ext.ext_poll(served, tickets[0])["rc"] == ext.EXT_ENOTFOUND
    finally:
        ext.ext_destroy(solo)
        ext.ext_destroy(served)


def test_served_host_buffers_and_threads(ext):
    probs, _ = _stream(8, 12)
    c = ext.ext_create(ext.options("fp32", max_slots=4))
    try:
        outs = [np.full(p.phi.shape, np.nan, np.float32) for p in probs]
        tickets = [None] * len(probs)

        def submit(k):
            p = probs[k]
            tickets[k] = ext.ext_submit(c, ext.problem_of(p), np.ascontiguousarray(p.phi),
                                        np.ascontiguousarray(p.f), outs[k])

        threads = [threading.Thread(target=submit, args=(k,)) for k in range(len(probs))]
        for th in threads:
            th.start()
        for th in threads:
            th.join()
        ext.ext_drain(c)
        for p, t, o in zip(probs, tickets, outs):
            r = ext.ext_poll(c, t)
            assert r["rc"] == 0, r
            ref = torch.empty(p.phi.shape, device="cuda")
            ext.ext_solve(c, ext.problem_of(p), torch.from_numpy(p.phi).cuda(),
                          torch.from_numpy(p.f).cuda(), ref)
            np.testing.assert_array_equal(o, ref.cpu().numpy())
    finally:
        ext.ext_destroy(c)


def test_admission_refuses_requests_beyond_the_budget(ext):
    c = ext.ext_create(ext.options("fp32", hbm_budget=4 << 20))
    try:
        small = synth.circle(48)
        big = synth.circle(512)
        o1 = torch.empty(small.phi.shape, device="cuda")
        o2 = torch.empty(big.phi.shape, device="cuda")
        t1 = ext.ext_submit(c, ext.problem_of(small), torch.from_numpy(small.phi).cuda(),
                            torch.from_numpy(small.f).cuda(), o1)
        t2 = ext.ext_submit(c, ext.problem_of(big), torch.from_numpy(big.phi).cuda(),
                            torch.from_numpy(big.f).cuda(), o2)
        ext.ext_drain(c)
        assert ext.ext_poll(c, t1)["rc"] == 0
        assert ext.ext_poll(c, t2)["rc"] == ext.EXT_EADMIT
        assert ext.ext_poll(c, 987654321)["rc"] == ext.EXT_ENOTFOUND
    finally:
        ext.ext_destroy(c)
