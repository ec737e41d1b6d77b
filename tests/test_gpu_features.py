"""Entry points and result fields beyond the single solve, through the C ABI (GB300).

* ext_solve_multi: several fields sharing one phi (the paper's level-set application extends more
  than one field per step): each field's answer equals its ext_solve answer bit for bit and is
  within the error bound of the oracle's direct solve at rel-res 1e-8.
* ext_result.err_est: CG's step terms estimate the relative A-norm error of the returned iterate;
  compared here with the error computed on the CPU against the direct solve.
* the stencil tile autotuner: tiles of 16 and 32 rows and the autotuned choice give the same
  results bit for bit (the p.q partials are summed over fixed row segments, not tiles).
* ext_options.wait_cycles: a wait bound short enough that the kernels' first waits for their own
  tensor copies run out.  The kernels drain what they issued and return; the call reports
  EXT_ETIMEOUT and a fresh context then reproduces a reference solve bit for bit.
"""

import numpy as np
import pytest
import torch

from oracle import biharmonic as ob
from paper_1704_08897_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ext():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1704_08897_gb300 import build_ext, ext as e
    build_ext.build()
    e.load()
    return e


def dev(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


@pytest.mark.parametrize("prec,tol", [("fp32", 1e-6), ("mixed_bf16", 1e-5)])
def test_multi_field_solve_equals_single_solves_and_oracle(ext, prec, tol):
    p = synth.circle(128, "symmetric", "out")
    X, Y, _, _ = synth.grid(128, 128, "symmetric", "symmetric")
    fields = [p.f, (np.sin(2 * X) * np.cos(Y)).astype(np.float32),
              (0.3 + X * Y).astype(np.float32)]
    prob = ext.problem_of(p)
    c = ext.ext_create(ext.options(prec, rtol=1e-8))
    try:
        singles = []
        for f in fields:
            o = torch.empty(p.phi.shape, device="cuda")
            ext.ext_solve(c, prob, dev(p.phi), dev(f), o)
            singles.append(o)
        outs = [torch.empty(p.phi.shape, device="cuda") for _ in fields]
        rc, res = ext.ext_solve_multi(c, prob, dev(p.phi), [dev(f) for f in fields], outs)
    finally:
        ext.ext_destroy(c)
    phi64 = p.phi.astype(np.float64)
    known = ob.known_mask(phi64, p.direction)
    for f, o, s, r in zip(fields, outs, singles, res):
        assert r["status"] == 0 and r["relres_true"] <= 1e-8, r
        assert torch.equal(o, s)
        ref, _ = ob.extend(phi64, f.astype(np.float64), p.direction, p.bc_x, p.bc_y, p.hx, p.hy,
                           method="direct")
        assert ob.max_rel_error(o.cpu().numpy(), ref, known) <= tol


@pytest.mark.parametrize("prec", ["fp32", "mixed_bf16"])
def test_error_estimate_tracks_the_a_norm_error(ext, prec):
    ratios = []
    for p in (synth.wobbly(128, 1), synth.wobbly(192, 3), synth.star(160, "periodic", "in")):
        phi64, f64 = p.phi.astype(np.float64), p.f.astype(np.float64)
        A, b, unk, known = ob.system(phi64, f64, p.direction, p.bc_x, p.bc_y, p.hx, p.hy)
        xs = ob.solve_direct(A, b)
        for rtol in (1e-6, 1e-8):
            c = ext.ext_create(ext.options(prec, rtol=rtol))
            try:
                out64 = torch.empty(p.phi.shape, device="cuda", dtype=torch.float64)
                res = ext.ext_solve_f64(c, ext.problem_of(p), dev(p.phi), dev(p.f), out64)
            finally:
                ext.ext_destroy(c)
            e = xs - out64.cpu().numpy().ravel()[unk]
            true = np.sqrt(e @ (A @ e)) / np.sqrt(xs @ (A @ xs))
            assert res["err_est"] > 0
            ratios.append(res["err_est"] / true)
    # an estimate for the iterate eight steps before the end: above the returned iterate's error,
    # and not by orders of magnitude
    assert min(ratios) >= 0.5 and max(ratios) <= 50.0, ratios


@pytest.mark.parametrize("prec", ["fp32", "mixed_bf16"])
def test_wait_bound_runs_out_and_the_next_context_is_unaffected(ext, prec):
    p = synth.wobbly(128, 2)  # nx % 16 == 0: the stencil's windows arrive by tensor copies
    prob = ext.problem_of(p)
    c = ext.ext_create(ext.options(prec, rtol=1e-8))
    try:
        ref = torch.empty(p.phi.shape, device="cuda")
        r0 = ext.ext_solve(c, prob, dev(p.phi), dev(p.f), ref)
    finally:
        ext.ext_destroy(c)
    c = ext.ext_create(ext.options(prec, rtol=1e-8, wait_cycles=1))
    try:
        out = torch.empty(p.phi.shape, device="cuda")
        r1 = ext.ext_solve(c, prob, dev(p.phi), dev(p.f), out, check=False)
    finally:
        ext.ext_destroy(c)
    assert r1["rc"] == ext.EXT_ETIMEOUT, r1
    c = ext.ext_create(ext.options(prec, rtol=1e-8))
    try:
        again = torch.empty(p.phi.shape, device="cuda")
        r2 = ext.ext_solve(c, prob, dev(p.phi), dev(p.f), again)
    finally:
        ext.ext_destroy(c)
    assert r2["iters"] == r0["iters"] and torch.equal(again, ref)


@pytest.mark.parametrize("prec", ["fp32", "mixed_bf16"])
def test_tile_heights_and_autotuned_tiles_give_identical_results(ext, prec):
    probs = [synth.wobbly(s, i) for i, s in enumerate([128, 192, 97, 256])]
    X, Y, hx, hy = synth.grid(80, 72, "symmetric", "periodic")
    probs.append(synth.Problem((np.sqrt(X ** 2 + Y ** 2) - 0.5).astype(np.float32),
                               np.sin(2 * X + Y).astype(np.float32), "symmetric", "periodic",
                               "out", hx, 0.7 * hy))
    results = {}
    for name, kw in (("fixed32", dict(autotune=0, tile_y=32)), ("fixed16", dict(autotune=0, tile_y=16)),
                     ("tuned", dict(autotune=1))):
        c = ext.ext_create(ext.options(prec, rtol=1e-8, **kw))
        try:
            outs = [torch.empty(p.phi.shape, device="cuda") for p in probs]
            rc, res = ext.ext_solve_batch(c, [ext.problem_of(p) for p in probs],
                                          [dev(p.phi) for p in probs], [dev(p.f) for p in probs], outs)
            tile = ext.ext_stencil_tile(c)
        finally:
            ext.ext_destroy(c)
        results[name] = (outs, res, tile)
    assert results["fixed32"][2] == (64, 32) and results["fixed16"][2] == (64, 16)
    assert results["tuned"][2] in ((64, 16), (64, 32))
    ref_outs, ref_res, _ = results["fixed32"]
    for name in ("fixed16", "tuned"):
        outs, res, _ = results[name]
        for o1, o2, r1, r2 in zip(ref_outs, outs, ref_res, res):
            assert r1["iters"] == r2["iters"] and torch.equal(o1, o2), name


@pytest.mark.parametrize("fold", [0, 1])
def test_low_mode_correction_cuts_iterations_and_keeps_parity(ext, fold):
    """The lowest 32 x 32 modes of the mixed path's preconditioner (of each mirror class when the
    transforms are folded) come from six-slice products (about 48 bits) instead of the four-slice
    stages: on batch-workload grids the iteration count at rel-res 1e-8 falls, and both answers
    stay within the mixed path's bound of the direct solve."""
    its = {}
    for p in (synth.wobbly(256, 0), synth.wobbly(384, 5), synth.star(256, "periodic", "in")):
        phi64, f64 = p.phi.astype(np.float64), p.f.astype(np.float64)
        ref, _ = ob.extend(phi64, f64, p.direction, p.bc_x, p.bc_y, p.hx, p.hy, method="direct")
        known = ob.known_mask(phi64, p.direction)
        for low in (0, 1):
            c = ext.ext_create(ext.options("mixed_bf16", rtol=1e-8, low_modes=low, fold=fold))
            try:
                out64 = torch.empty(p.phi.shape, device="cuda", dtype=torch.float64)
                res = ext.ext_solve_f64(c, ext.problem_of(p), dev(p.phi), dev(p.f), out64)
            finally:
                ext.ext_destroy(c)
            o = out64.cpu().numpy()
            rr = ob.true_relative_residual(o, phi64, f64, p.direction, p.bc_x, p.bc_y, p.hx, p.hy)
            assert res["status"] == 0 and rr <= 1.05e-8, (p.name, low, rr, res)
            assert ob.max_rel_error(o, ref, known) <= 1e-5
            its[(p.name, low)] = res["iters"]
    for name in {k[0] for k in its}:
        assert its[(name, 1)] <= 0.9 * its[(name, 0)], its


def test_automatic_low_modes_follow_the_call_size(ext):
    """low_modes = 2 (the default) turns the correction on for every grid of a call whose grids
    hold at least 2048^2 nodes together, and leaves it off for the same grids solved one by one
    or with low_modes = 0 (seen in the per-kernel launch counts)."""
    probs = [synth.wobbly(512, i) for i in range(17)]  # 17 x 512^2 = 4.46 M nodes >= 2048^2
    assert sum(p.nx * p.ny for p in probs) >= 2048 * 2048 > 512 * 512

    def low_launches(low_modes, batch):
        kw = {} if low_modes is None else {"low_modes": low_modes}
        c = ext.ext_create(ext.options("mixed_bf16", rtol=1e-2, profile=1, **kw))
        try:
            sel = probs if batch else probs[:2]
            outs = [torch.empty(p.phi.shape, device="cuda") for p in sel]
            if batch:
                rc, res = ext.ext_solve_batch(c, [ext.problem_of(p) for p in sel],
                                              [dev(p.phi) for p in sel], [dev(p.f) for p in sel], outs)
                assert all(r["status"] == 0 for r in res), res
            else:
                for p, o in zip(sel, outs):
                    assert ext.ext_solve(c, ext.problem_of(p), dev(p.phi), dev(p.f), o)["status"] == 0
            prof = ext.ext_profile_read(c)
        finally:
            ext.ext_destroy(c)
        return prof["low_fwd"][1], prof["low_inv"][1]

    fwd, inv = low_launches(None, True)
    assert fwd > 0 and inv == fwd
    assert low_launches(None, False) == (0, 0)
    assert low_launches(0, True) == (0, 0)
