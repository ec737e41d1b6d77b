"""The operator apply that allocates nothing gives what the context-based entry point gives.

ext_apply_biharmonic_noalloc exists for callers that may not allocate device memory when they
need the operator: a host application that owns the whole device-memory budget, or a loop in
which cudaMalloc/cudaFree would synchronise the device.  Its scratch is
one fixed array per device, shared by every call, so the test makes two calls in a row with
different grids and checks each against ext_apply_biharmonic: q bit for bit (both evaluate the
same compensated 13-point sum, term by term in the same order) and the sum p.q to 1e-7 relative:
this entry point sums p times the FP32 q it returns, the context entry point the solver's
double-float q, which is the same q plus a low part of relative size 2^-24.  This file is collected last; it also passes when run alone.
"""

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _case(nx, ny, bc_x, bc_y, direction, seed, h=(1.0, 1.0)):
    rng = np.random.default_rng(seed)
    phi = rng.uniform(-1, 1, (ny, nx)).astype(np.float32)
    known = phi < 0 if direction == "out" else phi > 0
    p = rng.standard_normal((ny, nx)).astype(np.float32)
    p[known] = 0
    return phi, p, h


def test_noalloc_apply_matches_context_apply_on_two_calls():
    assert torch.cuda.is_available(), "GPU test"
    from paper_1704_08897_gb300 import build_ext, ext
    build_ext.build()
    ext.load()
    ctx = ext.ext_create(ext.options("fp32"))
    try:
        cases = [(300, 170, "symmetric", "periodic", "out", 1, (1.0, 1.0)),
                 (97, 513, "dirichlet", "symmetric", "in", 2, (0.02, 0.03))]
        for nx, ny, bx, by, d, seed, h in cases:
            phi, p, h = _case(nx, ny, bx, by, d, seed, h)
            prob = ext.problem(nx, ny, bx, by, d, h[0], h[1])
            phi_d = torch.from_numpy(phi).cuda()
            p_d = torch.from_numpy(p).cuda()
            q_ref = torch.empty_like(p_d)
            s_ref = ext.ext_apply_biharmonic(ctx, prob, phi_d, p_d, q_ref)
            q = torch.full_like(p_d, float("nan"))
            rc, s = ext.ext_apply_biharmonic_noalloc(prob, phi_d, p_d, q)
            assert rc == ext.EXT_OK
            assert torch.equal(q, q_ref)
            assert abs(s - s_ref) <= 1e-7 * abs(s_ref)
    finally:
        ext.ext_destroy(ctx)


def test_noalloc_rejects_grids_beyond_its_scratch():
    from paper_1704_08897_gb300 import ext
    ext.load()
    phi = torch.zeros((1025, 1024), device="cuda")
    p = torch.zeros_like(phi)
    q = torch.empty_like(phi)
    rc, _ = ext.ext_apply_biharmonic_noalloc(ext.problem(1024, 1025), phi, p, q, check=False)
    assert rc == ext.EXT_EINVAL
    assert "too large" in ext.load().ext_noalloc_last_error().decode()
