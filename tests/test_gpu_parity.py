"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.  Needs a GB300.

Bars:
* integer/bitwise: the masked 13-point operator on integer vectors, the right-hand side for integer
  fields, the known-node copy, batch-vs-single equality;
* validity at rel-res 1e-8: the FP64 true relative residual, recomputed on the CPU from the GPU's
  FP64 iterate, is <= 1e-8;
* error at rel-res 1e-8: the answer of a solve stopped at rel-res 1e-8 is within max-norm relative
  error 1e-6 (FP32 path) or 1e-5 (mixed path) of the oracle's direct solve, on small grids of
  every boundary pair and on grids of the benchmark workloads solved in the benchmark's own
  launch configuration (one batched call);
* uniqueness: solved to rel-res 1e-11 the GPU iterate matches the direct solve to the same bound.
"""

import numpy as np
import pytest
import torch

from oracle import biharmonic as ob
from paper_1704_08897_gb300 import synth

pytestmark = pytest.mark.gpu

BCN = ["symmetric", "periodic", "dirichlet"]
PAIRS = [(bx, by) for bx in BCN for by in BCN]
TOL_FP32 = 1e-6


@pytest.fixture(scope="module")
def ext():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1704_08897_gb300 import build_ext, ext as e
    build_ext.build()
    e.load()
    return e


@pytest.fixture(scope="module")
def ctx(ext):
    c = ext.ext_create(ext.options("fp32", rtol=1e-8))
    yield c
    ext.ext_destroy(c)


@pytest.fixture(scope="module", params=[32, 16], ids=["tile32", "tile16"])
def ctx_tile(ext, request):
    c = ext.ext_create(ext.options("fp32", rtol=1e-8, autotune=0, tile_y=request.param))
    yield c
    ext.ext_destroy(c)


@pytest.fixture(scope="module")
def ctx_tight(ext):
    c = ext.ext_create(ext.options("fp32", rtol=1e-11))
    yield c
    ext.ext_destroy(c)


def dev(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def _rand_phi(nx, ny, seed, frac=0.4):
    rng = np.random.default_rng(seed)
    phi = rng.uniform(-1, 1, (ny, nx)).astype(np.float32)
    phi[rng.uniform(size=(ny, nx)) > frac] = 1.0
    return phi


# ----------------------------------------------------------------------------------------------
# operator and right-hand side, bitwise on integers
# ----------------------------------------------------------------------------------------------
@pytest.mark.parametrize("bc_x,bc_y", PAIRS)
@pytest.mark.parametrize("nx,ny", [(4, 4), (5, 7), (64, 16), (65, 17), (100, 37), (130, 129),
                                   (48, 40), (256, 96), (512, 384), (200, 300)])
def test_operator_bitwise_on_integers(ext, ctx_tile, bc_x, bc_y, nx, ny):
    """ext_apply_biharmonic runs the solver's stencil kernel (iteration 0, beta = 0, z = p).  With
    h = 1 and integer p (|p| <= 2^10) every 13-point sum is an exact integer below 2^24, so q must
    equal the oracle's operator bit for bit, for both stencil tile heights (16 and 32 rows).  nx a
    multiple of 16 (48, 64, 256, 512) takes the tensor-copy window path, other widths the
    plain-load path; the sizes cover interior, edge and corner tiles and ragged last tiles in
    both axes."""
    phi = _rand_phi(nx, ny, nx * 7 + ny)
    known = ob.known_mask(phi.astype(np.float64), "out")
    rng = np.random.default_rng(nx + 3 * ny)
    p = rng.integers(-1024, 1025, (ny, nx)).astype(np.float32)
    p[known] = 0
    L2 = ob.squared_laplacian_kron(nx, ny, bc_x, bc_y)
    ref = (L2 @ p.astype(np.float64).ravel()).reshape(ny, nx)
    ref[known] = 0
    q = torch.empty((ny, nx), device="cuda")
    pq = ext.ext_apply_biharmonic(ctx_tile, ext.problem(nx, ny, bc_x, bc_y, "out"), dev(phi), dev(p), q)
    np.testing.assert_array_equal(q.cpu().numpy().astype(np.float64), ref)
    exact = float(p.astype(np.float64).ravel() @ ref.ravel())
    assert abs(pq - exact) <= 1e-9 * abs(exact), (pq, exact)


@pytest.mark.parametrize("bc_x,bc_y", PAIRS)
def test_operator_anisotropic_spacing(ext, ctx, bc_x, bc_y):
    nx, ny, hx, hy = 70, 45, 0.02, 0.031
    phi = _rand_phi(nx, ny, 11)
    known = ob.known_mask(phi.astype(np.float64), "out")
    p = np.random.default_rng(2).standard_normal((ny, nx)).astype(np.float32)
    p[known] = 0
    L2 = ob.squared_laplacian_kron(nx, ny, bc_x, bc_y, hx, hy)
    ref = (L2 @ p.astype(np.float64).ravel()).reshape(ny, nx)
    ref[known] = 0
    # the library scales the operator by max(1/hx^2, 1/hy^2)^-2 (CG is scale-free)
    s = max(1 / hx ** 2, 1 / hy ** 2) ** 2
    q = torch.empty((ny, nx), device="cuda")
    ext.ext_apply_biharmonic(ctx, ext.problem(nx, ny, bc_x, bc_y, "out", hx, hy), dev(phi), dev(p), q)
    np.testing.assert_allclose(q.cpu().numpy() * s, ref, rtol=2e-6, atol=1e-6 * np.abs(ref).max())


@pytest.mark.parametrize("bc_x,bc_y", PAIRS)
@pytest.mark.parametrize("direction", ["out", "in"])
def test_rhs_bitwise_on_integers(ext, ctx, bc_x, bc_y, direction):
    nx, ny = 67, 35
    phi = _rand_phi(nx, ny, 5)
    if direction == "in":
        phi = -phi
    f = np.random.default_rng(9).integers(-300, 301, (ny, nx)).astype(np.float32)
    ref = ob.rhs_padded(phi.astype(np.float64), f.astype(np.float64), direction, bc_x, bc_y)
    b = torch.empty((ny, nx), device="cuda", dtype=torch.float64)
    ext.ext_rhs(ctx, ext.problem(nx, ny, bc_x, bc_y, direction), dev(phi), dev(f), b)
    np.testing.assert_array_equal(b.cpu().numpy(), ref)


# ----------------------------------------------------------------------------------------------
# preconditioner: z / scale against the oracle's scipy.fft pseudo-inverse of L^2
# ----------------------------------------------------------------------------------------------
@pytest.mark.parametrize("bc_x,bc_y", PAIRS)
@pytest.mark.parametrize("nx,ny", [(16, 16), (40, 24), (130, 100)])
def test_preconditioner_matches_fast_poisson(ext, ctx, bc_x, bc_y, nx, ny):
    phi = _rand_phi(nx, ny, 3)
    known = ob.known_mask(phi.astype(np.float64), "out")
    r = np.random.default_rng(4).standard_normal((ny, nx)).astype(np.float32)
    r[known] = 0
    ref = ob.poisson_squared_pinv(r.astype(np.float64), bc_x, bc_y)
    ref[known] = 0
    z = torch.empty((ny, nx), device="cuda")
    scale = ext.ext_apply_preconditioner(ctx, ext.problem(nx, ny, bc_x, bc_y, "out"), dev(phi),
                                         dev(r), z)
    got = z.cpu().numpy().astype(np.float64) / scale
    np.testing.assert_allclose(got, ref, rtol=0, atol=2e-5 * np.abs(ref).max())


# ----------------------------------------------------------------------------------------------
# full solves
# ----------------------------------------------------------------------------------------------
def _check_solution(ext, ctx, ctx_tight, p, tol=TOL_FP32, rtol=1e-8):
    prob = ext.problem_of(p)
    phi64, f64 = p.phi.astype(np.float64), p.f.astype(np.float64)
    ref, info = ob.extend(phi64, f64, p.direction, p.bc_x, p.bc_y, p.hx, p.hy, method="direct")
    known = ob.known_mask(phi64, p.direction)
    # validity at the solver's tolerance, by the CPU's own FP64 residual of the GPU iterate
    out64 = torch.empty(p.phi.shape, device="cuda", dtype=torch.float64)
    res = ext.ext_solve_f64(ctx, prob, dev(p.phi), dev(p.f), out64)
    assert res["status"] == 0, res
    o64 = out64.cpu().numpy()
    rr = ob.true_relative_residual(o64, phi64, f64, p.direction, p.bc_x, p.bc_y, p.hx, p.hy)
    assert rr <= rtol * 1.05, (rr, res)
    assert abs(res["relres_true"] - rr) <= 0.05 * rr + 1e-15
    assert np.array_equal(o64[known], f64[known])
    # the error bound holds at the solver's own tolerance (rel-res 1e-8), not only when tighter
    err_at_rtol = ob.max_rel_error(o64, ref, known)
    assert err_at_rtol <= tol, (err_at_rtol, res)
    # the FP32 output: known nodes bit-exact, unknown nodes the rounded FP64 iterate
    out = torch.empty(p.phi.shape, device="cuda")
    res32 = ext.ext_solve(ctx, prob, dev(p.phi), dev(p.f), out)
    o32 = out.cpu().numpy()
    assert np.array_equal(o32[known], p.f[known])
    np.testing.assert_array_equal(o32[~known], o64[~known].astype(np.float32))
    assert res32["iters"] == res["iters"]
    # uniqueness: a tight solve reproduces the oracle's solution
    tight = torch.empty(p.phi.shape, device="cuda", dtype=torch.float64)
    rt = ext.ext_solve_f64(ctx_tight, prob, dev(p.phi), dev(p.f), tight)
    assert rt["status"] == 0 and rt["relres_true"] <= 1e-11, rt
    err = ob.max_rel_error(tight.cpu().numpy(), ref, known)
    assert err <= tol, (err, rt)
    return res, err_at_rtol, err


@pytest.mark.parametrize("bc_x,bc_y", PAIRS)
@pytest.mark.parametrize("direction", ["out", "in"])
def test_solve_small_all_boundaries(ext, ctx, ctx_tight, bc_x, bc_y, direction):
    n = 48
    X, Y, hx, hy = synth.grid(n, n + 5, bc_x, bc_y)
    phi = (np.sqrt((X - 0.1) ** 2 + Y ** 2) - 0.55).astype(np.float32)
    f = (np.cos(2 * X) * np.sin(3 * Y) + 0.5 * X).astype(np.float32)
    p = synth.Problem(phi, f, bc_x, bc_y, direction, hx, hy)
    _check_solution(ext, ctx, ctx_tight, p)


@pytest.mark.parametrize("n", [64, 97, 130, 256])  # 64, 256: tensor-copy stencil windows
def test_solve_circle_symmetric(ext, ctx, ctx_tight, n):
    _check_solution(ext, ctx, ctx_tight, synth.circle(n))


def test_solve_star_periodic_512(ext, ctx, ctx_tight):
    res, _, _ = _check_solution(ext, ctx, ctx_tight, synth.star(512, "periodic", "in"))
    assert res["iters"] < 5000


def test_solve_wobbly_batch_member(ext, ctx, ctx_tight):
    _check_solution(ext, ctx, ctx_tight, synth.wobbly(192, 3))


@pytest.mark.parametrize("nx", [60, 64])  # plain-load and tensor-copy stencil windows
def test_solve_anisotropic(ext, ctx, ctx_tight, nx):
    X, Y, hx, hy = synth.grid(nx, 90, "symmetric", "periodic")
    hy = hy * 0.7
    phi = (np.sqrt(X ** 2 + Y ** 2) - 0.5).astype(np.float32)
    f = (np.sin(2 * X + Y)).astype(np.float32)
    _check_solution(ext, ctx, ctx_tight, synth.Problem(phi, f, "symmetric", "periodic", "out", hx, hy))


# ----------------------------------------------------------------------------------------------
# batch = single, host buffers, edge cases
# ----------------------------------------------------------------------------------------------
def test_batch_results_equal_single_solves_bitwise(ext, ctx):
    probs = [synth.wobbly(s, i) for i, s in enumerate([128, 192, 128, 256, 97])]
    probs.append(synth.star(100, "periodic", "in"))
    singles = []
    for p in probs:
        out = torch.empty(p.phi.shape, device="cuda")
        singles.append((ext.ext_solve(ctx, ext.problem_of(p), dev(p.phi), dev(p.f), out), out))
    outs = [torch.empty(p.phi.shape, device="cuda") for p in probs]
    rc, res = ext.ext_solve_batch(ctx, [ext.problem_of(p) for p in probs],
                                  [dev(p.phi) for p in probs], [dev(p.f) for p in probs], outs)
    for (r1, o1), r2, o2 in zip(singles, res, outs):
        assert r2["status"] == 0 and r1["iters"] == r2["iters"]
        assert torch.equal(o1, o2)


def test_host_buffers_give_the_device_result(ext, ctx):
    p = synth.wobbly(128, 5)
    out_d = torch.empty(p.phi.shape, device="cuda")
    ext.ext_solve(ctx, ext.problem_of(p), dev(p.phi), dev(p.f), out_d)
    out_h = np.empty_like(p.f)
    ext.ext_solve(ctx, ext.problem_of(p), np.ascontiguousarray(p.phi), np.ascontiguousarray(p.f),
                  out_h)
    np.testing.assert_array_equal(out_h, out_d.cpu().numpy())


def test_out_may_alias_f(ext, ctx):
    p = synth.circle(64)
    out = torch.empty(p.phi.shape, device="cuda")
    ext.ext_solve(ctx, ext.problem_of(p), dev(p.phi), dev(p.f), out)
    fa = dev(p.f)
    ext.ext_solve(ctx, ext.problem_of(p), dev(p.phi), fa, fa)
    assert torch.equal(fa, out)


def test_all_known_returns_f(ext, ctx):
    n = 32
    phi = -np.ones((n, n), np.float32)
    f = np.random.default_rng(0).standard_normal((n, n)).astype(np.float32)
    out = torch.empty((n, n), device="cuda")
    res = ext.ext_solve(ctx, ext.problem(n, n, "symmetric", "symmetric", "out"), dev(phi), dev(f), out)
    assert res["iters"] == 0 and np.array_equal(out.cpu().numpy(), f)


def test_nothing_known(ext, ctx):
    n = 16
    phi = np.ones((n, n), np.float32)
    f = np.ones((n, n), np.float32)
    out = torch.empty((n, n), device="cuda")
    res = ext.ext_solve(ctx, ext.problem(n, n, "dirichlet", "symmetric", "out"), dev(phi), dev(f), out)
    assert res["status"] == 0 and torch.all(out == 0)
    res = ext.ext_solve(ctx, ext.problem(n, n, "periodic", "symmetric", "out"), dev(phi), dev(f),
                        out, check=False)
    assert res["rc"] == ext.EXT_ENOKNOWN


def test_invalid_inputs_are_rejected(ext, ctx):
    n = 16
    phi = np.ones((n, n), np.float32)
    phi[3, 4] = np.nan
    f = np.zeros((n, n), np.float32)
    out = torch.empty((n, n), device="cuda")
    res = ext.ext_solve(ctx, ext.problem(n, n), dev(phi), dev(f), out, check=False)
    assert res["rc"] == ext.EXT_EINVAL
    for bad in (ext.problem(3, 16), ext.problem(16, 16, hx=0.0), ext.problem(16, 16, hx=float("nan"))):
        r = ext.ext_solve(ctx, bad, dev(np.ones((16, 16), np.float32)), dev(f), out, check=False)
        assert r["rc"] == ext.EXT_EINVAL
    bad = ext.problem(16, 16)
    bad.bc_x = 7
    assert ext.ext_solve(ctx, bad, dev(phi), dev(f), out, check=False)["rc"] == ext.EXT_EINVAL


def test_non_finite_known_value_is_rejected(ext, ctx):
    """A non-finite field value at a known node would turn b, and every CG scalar after it, into
    NaN; the set-up counts such values beside NaN phi and the solve returns EXT_EINVAL with the
    known nodes of the output untouched by any iteration."""
    p = synth.circle(64)
    known = ob.known_mask(p.phi.astype(np.float64), p.direction)
    for bad in (np.nan, np.inf):
        f = p.f.copy()
        ky, kx = np.argwhere(known)[len(np.argwhere(known)) // 2]
        f[ky, kx] = bad
        out = torch.empty(p.phi.shape, device="cuda")
        res = ext.ext_solve(ctx, ext.problem_of(p), dev(p.phi), dev(f), out, check=False)
        assert res["rc"] == ext.EXT_EINVAL, res
        assert res["iters"] == 0
    # a non-finite value at an unknown node is ignored (only known values are data)
    f = p.f.copy()
    uy, ux = np.argwhere(~known)[0]
    f[uy, ux] = np.nan
    out = torch.empty(p.phi.shape, device="cuda")
    res = ext.ext_solve(ctx, ext.problem_of(p), dev(p.phi), dev(f), out)
    assert res["status"] == 0 and np.all(np.isfinite(out.cpu().numpy()))


def test_maxit_reports_not_converged_with_best_iterate(ext):
    c = ext.ext_create(ext.options("fp32", rtol=1e-12, maxit=20))
    try:
        p = synth.wobbly(128, 1)
        out = torch.empty(p.phi.shape, device="cuda")
        res = ext.ext_solve(c, ext.problem_of(p), dev(p.phi), dev(p.f), out, check=False)
        assert res["rc"] == ext.EXT_ENOTCONV and res["iters"] == 20
        assert 0 < res["relres_true"] < 1
        known = ob.known_mask(p.phi.astype(np.float64), p.direction)
        assert np.array_equal(out.cpu().numpy()[known], p.f[known])
    finally:
        ext.ext_destroy(c)


# ----------------------------------------------------------------------------------------------
# full-size single solve (1024^2 star, periodic, extend in): properties that hold at any size
# ----------------------------------------------------------------------------------------------
def test_full_size_star_1024(ext, ctx):
    p = synth.single_star_case(1024)
    # make the inputs exactly even in y (the float32 node coordinates are symmetric to 1 ulp)
    p.phi = np.ascontiguousarray((p.phi + p.phi[::-1, :]) * np.float32(0.5))
    p.f = np.ascontiguousarray((p.f + p.f[::-1, :]) * np.float32(0.5))
    prob = ext.problem_of(p)
    out64 = torch.empty(p.phi.shape, device="cuda", dtype=torch.float64)
    res = ext.ext_solve_f64(ctx, prob, dev(p.phi), dev(p.f), out64)
    assert res["status"] == 0
    o = out64.cpu().numpy()
    phi64, f64 = p.phi.astype(np.float64), p.f.astype(np.float64)
    rr = ob.true_relative_residual(o, phi64, f64, p.direction, p.bc_x, p.bc_y, p.hx, p.hy)
    assert rr <= 1.05e-8
    known = ob.known_mask(phi64, p.direction)
    assert np.array_equal(o[known], f64[known])
    # the star and the field are even in y: the extension is mirror-symmetric in y
    sym = np.abs(o - o[::-1, :]).max() / np.abs(o).max()
    assert sym < 1e-5, sym


# ----------------------------------------------------------------------------------------------
# CG trajectory: after k iterations the GPU iterate equals the oracle's FP64 PCG iterate x_k
# (same preconditioner, same Fletcher-Reeves beta) up to FP32 rounding.  Only the first two
# iterates are compared: on this operator FP32 and FP64 trajectories separate by 1e-2 within five
# iterations (an FP32-storage emulation of the same recurrences does the same).
# ----------------------------------------------------------------------------------------------
@pytest.mark.parametrize("k", [1, 2])
def test_cg_trajectory_matches_oracle(ext, k):
    p = synth.circle(64)
    phi64, f64 = p.phi.astype(np.float64), p.f.astype(np.float64)
    A, b, unk, known = ob.system(phi64, f64, p.direction, p.bc_x, p.bc_y)
    M = ob.fast_poisson_preconditioner(unk, 64, 64, p.bc_x, p.bc_y)
    x_k, it, _ = ob.cg(A, b, rtol=1e-30, maxit=k, precond=M)
    assert it == k
    c = ext.ext_create(ext.options("fp32", rtol=1e-15, maxit=k, flexible=0))
    try:
        out64 = torch.empty((64, 64), device="cuda", dtype=torch.float64)
        res = ext.ext_solve_f64(c, ext.problem_of(p), dev(p.phi), dev(p.f), out64, check=False)
    finally:
        ext.ext_destroy(c)
    assert res["iters"] == k, res
    got = out64.cpu().numpy().ravel()[unk]
    scale = np.abs(x_k).max()
    err = np.abs(got - x_k).max() / scale
    assert err < 1e-4 * k, (k, err)


# ----------------------------------------------------------------------------------------------
# mixed precision: tensor-core transforms from block-scaled integer slices in FP16 or BF16
# ----------------------------------------------------------------------------------------------
TOL_MIXED = 1e-5
MIXED = ["mixed_fp16", "mixed_bf16"]


@pytest.fixture(scope="module", params=MIXED)
def mixed(ext, request):
    c = ext.ext_create(ext.options(request.param, rtol=1e-8))
    ct = ext.ext_create(ext.options(request.param, rtol=1e-11))
    yield request.param, c, ct
    ext.ext_destroy(c)
    ext.ext_destroy(ct)


@pytest.mark.parametrize("bc_x,bc_y", [("symmetric", "symmetric"), ("periodic", "dirichlet"),
                                       ("dirichlet", "periodic")])
@pytest.mark.parametrize("nx,ny", [(40, 24), (130, 100), (256, 256)])
def test_mixed_preconditioner_matches_fast_poisson(ext, mixed, bc_x, bc_y, nx, ny):
    _, c, _ = mixed
    phi = _rand_phi(nx, ny, 3)
    known = ob.known_mask(phi.astype(np.float64), "out")
    r = np.random.default_rng(4).standard_normal((ny, nx)).astype(np.float32)
    r[known] = 0
    ref = ob.poisson_squared_pinv(r.astype(np.float64), bc_x, bc_y)
    ref[known] = 0
    z = torch.empty((ny, nx), device="cuda")
    scale = ext.ext_apply_preconditioner(c, ext.problem(nx, ny, bc_x, bc_y, "out"), dev(phi), dev(r), z)
    got = z.cpu().numpy().astype(np.float64) / scale
    np.testing.assert_allclose(got, ref, rtol=0, atol=5e-6 * np.abs(ref).max())


@pytest.fixture(scope="module")
def fold_ctxs(ext):
    # folded, full-size, and folded with the low-mode correction
    cs = [ext.ext_create(ext.options("mixed_bf16", rtol=1e-8, fold=f, low_modes=lm))
          for f, lm in ((1, 0), (0, 0), (1, 1))]
    yield cs
    for c in cs:
        ext.ext_destroy(c)


@pytest.mark.parametrize("bc_x", ob.BCS)
@pytest.mark.parametrize("bc_y", ob.BCS)
# both axes folded (odd and even n), x only (y = 128 does not pay), y only (x = 300 does not)
@pytest.mark.parametrize("nx,ny", [(255, 200), (256, 193), (255, 128), (300, 255)])
def test_folded_preconditioner_matches_fast_poisson(ext, fold_ctxs, bc_x, bc_y, nx, ny):
    """The transforms run per mirror class (even / odd vectors under i -> n-1-i) on axes where
    that halves the work: the same operator as the full-size transforms and the oracle's."""
    phi = _rand_phi(nx, ny, 5)
    known = ob.known_mask(phi.astype(np.float64), "out")
    r = np.random.default_rng(6).standard_normal((ny, nx)).astype(np.float32)
    r[known] = 0
    ref = ob.poisson_squared_pinv(r.astype(np.float64), bc_x, bc_y)
    ref[known] = 0
    got = []
    for c in fold_ctxs:
        z = torch.empty((ny, nx), device="cuda")
        scale = ext.ext_apply_preconditioner(c, ext.problem(nx, ny, bc_x, bc_y, "out"), dev(phi), dev(r), z)
        got.append(z.cpu().numpy().astype(np.float64) / scale)
        np.testing.assert_allclose(got[-1], ref, rtol=0, atol=5e-6 * np.abs(ref).max())
        assert np.all(got[-1][known] == 0)


@pytest.mark.parametrize("bc_x", ob.BCS)
@pytest.mark.parametrize("bc_y", ob.BCS)
@pytest.mark.parametrize("nx,ny", [(255, 200), (300, 255)])
def test_folded_preconditioner_fp32(ext, bc_x, bc_y, nx, ny):
    """The CUDA-core path folds the same axes: its preconditioner per mirror class equals the
    oracle's, folded and not."""
    phi = _rand_phi(nx, ny, 7)
    known = ob.known_mask(phi.astype(np.float64), "out")
    r = np.random.default_rng(8).standard_normal((ny, nx)).astype(np.float32)
    r[known] = 0
    ref = ob.poisson_squared_pinv(r.astype(np.float64), bc_x, bc_y)
    ref[known] = 0
    for fold in (1, 0):
        c = ext.ext_create(ext.options("fp32", rtol=1e-8, fold=fold))
        try:
            z = torch.empty((ny, nx), device="cuda")
            scale = ext.ext_apply_preconditioner(c, ext.problem(nx, ny, bc_x, bc_y, "out"), dev(phi),
                                                 dev(r), z)
        finally:
            ext.ext_destroy(c)
        got = z.cpu().numpy().astype(np.float64) / scale
        np.testing.assert_allclose(got, ref, rtol=0, atol=1e-6 * np.abs(ref).max())


@pytest.mark.parametrize("prec", ["mixed_bf16", "fp32"])
@pytest.mark.parametrize("bc", ob.BCS)
def test_folded_solve_on_odd_sides(ext, bc, prec):
    """A grid with odd sides on both folded axes (middle nodes in the even classes) solves to
    rel-res 1e-8 within the mixed path's bound of the direct solve, folded and not."""
    nx, ny = 255, 193
    X, Y = np.meshgrid(np.linspace(-1, 1, nx), np.linspace(-1, 1, ny))
    phi = (np.hypot(X - 0.1, Y + 0.05) - 0.45 - 0.05 * np.cos(5 * np.arctan2(Y, X))).astype(np.float32)
    f = (np.cos(3 * X + 1) * np.sin(2 * Y) + 0.3 * X * Y).astype(np.float32)
    phi64, f64 = phi.astype(np.float64), f.astype(np.float64)
    ref, _ = ob.extend(phi64, f64, "out", bc, bc, method="direct")
    known = ob.known_mask(phi64, "out")
    for fold in (1, 0):
        c = ext.ext_create(ext.options(prec, rtol=1e-8, maxit=40 * nx, fold=fold))
        try:
            out64 = torch.empty((ny, nx), device="cuda", dtype=torch.float64)
            res = ext.ext_solve_f64(c, ext.problem(nx, ny, bc, bc, "out"), dev(phi), dev(f), out64)
        finally:
            ext.ext_destroy(c)
        o = out64.cpu().numpy()
        rr = ob.true_relative_residual(o, phi64, f64, "out", bc, bc)
        assert res["status"] == 0 and rr <= 1.05e-8, (bc, fold, rr, res)
        assert ob.max_rel_error(o, ref, known) <= (TOL_MIXED if prec != "fp32" else TOL_FP32)


@pytest.mark.parametrize("maker", [lambda: synth.circle(64), lambda: synth.wobbly(192, 3),
                                   lambda: synth.star(256, "periodic", "in")])
def test_mixed_solve_validity_and_uniqueness(ext, mixed, maker):
    _, c, ct = mixed
    _check_solution(ext, c, ct, maker(), tol=TOL_MIXED)


def test_mixed_batch_equals_single_bitwise(ext, mixed):
    _, c, _ = mixed
    probs = [synth.wobbly(s, i) for i, s in enumerate([128, 192, 256])]
    singles = []
    for p in probs:
        out = torch.empty(p.phi.shape, device="cuda")
        singles.append((ext.ext_solve(c, ext.problem_of(p), dev(p.phi), dev(p.f), out), out))
    outs = [torch.empty(p.phi.shape, device="cuda") for p in probs]
    rc, res = ext.ext_solve_batch(c, [ext.problem_of(p) for p in probs], [dev(p.phi) for p in probs],
                                  [dev(p.f) for p in probs], outs)
    for (r1, o1), r2, o2 in zip(singles, res, outs):
        assert r2["status"] == 0 and r1["iters"] == r2["iters"]
        assert torch.equal(o1, o2)


def test_fp16_and_bf16_slices_give_identical_results(ext):
    """The slices are integers of at most 9 bits, exact in both formats, and every k-block sum is
    exact: the two tensor-core modes must agree bit for bit."""
    p = synth.wobbly(192, 4)
    outs = []
    for prec in MIXED:
        c = ext.ext_create(ext.options(prec))
        try:
            out = torch.empty(p.phi.shape, device="cuda")
            ext.ext_solve(c, ext.problem_of(p), dev(p.phi), dev(p.f), out)
            outs.append(out)
        finally:
            ext.ext_destroy(c)
    assert torch.equal(outs[0], outs[1])


# ----------------------------------------------------------------------------------------------
# scale: the extension is linear in f.  The iteration runs on 2^e b with e chosen from ||b||, so a
# power-of-two scale of f gives the same iterates and an exactly scaled answer, and fields far
# from unit size (whose FP32 pairwise products would overflow or underflow) still converge.
# ----------------------------------------------------------------------------------------------
@pytest.mark.parametrize("prec", ["fp32", "mixed_bf16"])
@pytest.mark.parametrize("s", [2.0 ** -70, 2.0 ** 70, 1e-25, 1e25])
def test_solution_scales_with_the_field(ext, prec, s):
    p = synth.wobbly(192, 3)
    c = ext.ext_create(ext.options(prec, rtol=1e-8))
    try:
        outs = []
        for k in (1.0, s):
            f = (p.f.astype(np.float64) * k).astype(np.float32)
            assert np.all(np.isfinite(f)) and np.all(f[p.f != 0] != 0)
            out = torch.empty(p.phi.shape, device="cuda")
            r = ext.ext_solve(c, ext.problem_of(p), dev(p.phi), dev(f), out)
            assert r["status"] == 0 and r["relres_true"] <= 1.05e-8, (k, r)
            outs.append(out.cpu().numpy())
        if np.log2(s) == np.round(np.log2(s)):
            # exact power of two: the same iterates, the answer scaled bit for bit
            assert np.array_equal(outs[1], (outs[0].astype(np.float64) * s).astype(np.float32))
        else:
            a = outs[0].astype(np.float64)
            b = outs[1].astype(np.float64) / s
            assert np.abs(b - a).max() <= 1e-4 * np.abs(a).max()
    finally:
        ext.ext_destroy(c)


# ----------------------------------------------------------------------------------------------
# Fletcher-Reeves beta (flexible=0) over many residual replacements: after a replacement the
# beta of the current iteration is recomputed with the previous iteration's r.z.
# ----------------------------------------------------------------------------------------------
@pytest.mark.parametrize("prec", ["fp32", "mixed_bf16"])
def test_fletcher_reeves_converges_through_residual_replacements(ext, prec):
    p = synth.wobbly(128, 2)
    its = {}
    for flex in (1, 0):
        c = ext.ext_create(ext.options(prec, rtol=1e-8, flexible=flex, true_res_every=20))
        try:
            out = torch.empty(p.phi.shape, device="cuda")
            r = ext.ext_solve(c, ext.problem_of(p), dev(p.phi), dev(p.f), out, check=False)
        finally:
            ext.ext_destroy(c)
        assert r["status"] == 0 and r["relres_true"] <= 1.05e-8, (flex, r)
        its[flex] = r["iters"]
    # both betas are exact CG for a fixed symmetric preconditioner: comparable counts
    assert its[0] <= 2 * its[1], its


# ----------------------------------------------------------------------------------------------
# workload-shaped parity at the solver's tolerance: the first twelve grids of the batch workload
# (wobbly interfaces, sides drawn from {128, ..., 512}) solved together in one ext_solve_batch
# call, as the benchmark runs them, each against the oracle's direct solve
# ----------------------------------------------------------------------------------------------
@pytest.fixture(scope="module")
def batch12():
    sides = synth.batch_sides(256)[:12]
    probs = [synth.wobbly(s, i) for i, s in enumerate(sides)]
    refs = []
    for p in probs:
        ref, _ = ob.extend(p.phi.astype(np.float64), p.f.astype(np.float64), p.direction, p.bc_x,
                           p.bc_y, p.hx, p.hy, method="direct")
        refs.append(ref)
    return probs, refs


@pytest.mark.parametrize("prec,tol", [("fp32", TOL_FP32), ("mixed_bf16", 1e-5)])
def test_workload_batch_grids_at_rtol_1e8(ext, batch12, prec, tol):
    probs, refs = batch12
    c = ext.ext_create(ext.options(prec, rtol=1e-8, maxit=40 * 512))
    try:
        outs = [torch.empty(p.phi.shape, device="cuda") for p in probs]
        rc, res = ext.ext_solve_batch(c, [ext.problem_of(p) for p in probs],
                                      [dev(p.phi) for p in probs], [dev(p.f) for p in probs], outs)
    finally:
        ext.ext_destroy(c)
    errs = []
    for p, r, o, ref in zip(probs, res, outs, refs):
        assert r["status"] == 0 and r["relres_true"] <= 1e-8, (p.name, r)
        known = ob.known_mask(p.phi.astype(np.float64), p.direction)
        o = o.cpu().numpy()
        assert np.array_equal(o[known], p.f[known])
        errs.append(ob.max_rel_error(o, ref, known))
    assert max(errs) <= tol, (prec, errs)


@pytest.mark.parametrize("prec,tol", [("fp32", TOL_FP32), ("mixed_bf16", 1e-5)])
def test_full_size_star_1024_error_at_rtol_1e8(ext, prec, tol):
    """The 1024^2 six-lobed star (periodic, extend in) at rel-res 1e-8 against the direct solve:
    the CPU's FP64 residual of the GPU's FP64 iterate, and the max-norm error bound."""
    p = synth.single_star_case(1024)
    phi64, f64 = p.phi.astype(np.float64), p.f.astype(np.float64)
    ref, _ = ob.extend(phi64, f64, p.direction, p.bc_x, p.bc_y, p.hx, p.hy, method="direct")
    c = ext.ext_create(ext.options(prec, rtol=1e-8, maxit=40 * 1024))
    try:
        out64 = torch.empty(p.phi.shape, device="cuda", dtype=torch.float64)
        res = ext.ext_solve_f64(c, ext.problem_of(p), dev(p.phi), dev(p.f), out64)
    finally:
        ext.ext_destroy(c)
    o = out64.cpu().numpy()
    rr = ob.true_relative_residual(o, phi64, f64, p.direction, p.bc_x, p.bc_y, p.hx, p.hy)
    assert res["status"] == 0 and rr <= 1.05e-8, (rr, res)
    known = ob.known_mask(phi64, p.direction)
    err = ob.max_rel_error(o, ref, known)
    assert err <= tol, (prec, err, res)
