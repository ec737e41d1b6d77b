"""Pins of the FP64 oracle against what the paper and the mathematics fix (CPU only).

Each test names the passage it follows.  None of them re-types the oracle's own formula: they use
a second construction, a variational characterisation, an invariance, or a value the paper prints.
"""

import os

import numpy as np
import pytest

from oracle import biharmonic as ob
from paper_1704_08897_gb300 import synth

BC_PAIRS = [(bx, by) for bx in ob.BCS for by in ob.BCS]
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _random_problem(nx, ny, seed, frac=0.35):
    rng = np.random.default_rng(seed)
    phi = rng.uniform(-1, 1, (ny, nx))
    phi[rng.uniform(size=(ny, nx)) > frac] = 1.0  # mostly unknown in 'out'
    f = rng.standard_normal((ny, nx))
    return phi, f


# -------------------------------------------------------------------------------------------
# Operator: three constructions agree; interior coefficients are eq. discrete_biharmonic
# -------------------------------------------------------------------------------------------
@pytest.mark.parametrize("bc_x,bc_y", BC_PAIRS)
@pytest.mark.parametrize("nx,ny", [(4, 4), (5, 7), (8, 6), (9, 9)])
def test_operator_constructions_agree_exactly(bc_x, bc_y, nx, ny):
    """Kronecker form == 13-point taps with ghost maps == Algorithm 1's padded two-pass form.

    With h = 1 every entry is an integer, so the comparison is exact.
    """
    K = ob.squared_laplacian_kron(nx, ny, bc_x, bc_y).toarray()
    S = ob.squared_laplacian_stencil(nx, ny, bc_x, bc_y).toarray()
    N = nx * ny
    P = np.zeros((N, N))
    for j in range(N):
        e = np.zeros(N)
        e[j] = 1.0
        P[:, j] = ob.apply_squared_laplacian_padded(e.reshape(ny, nx), bc_x, bc_y).ravel()
    assert np.array_equal(K, S)
    assert np.array_equal(K, P)
    assert np.array_equal(K, np.round(K))


@pytest.mark.parametrize("bc_x,bc_y", [("symmetric", "dirichlet"), ("periodic", "symmetric")])
def test_operator_constructions_agree_anisotropic(bc_x, bc_y):
    hx, hy = 0.3, 0.7
    K = ob.squared_laplacian_kron(7, 6, bc_x, bc_y, hx, hy).toarray()
    S = ob.squared_laplacian_stencil(7, 6, bc_x, bc_y, hx, hy).toarray()
    np.testing.assert_allclose(K, S, rtol=1e-13, atol=1e-9 * np.abs(K).max())


def test_interior_row_is_the_13_point_stencil():
    """Eq. discrete_biharmonic: 20 at the centre, -8 at edge neighbours, 2 diagonal, 1 at 2."""
    nx = ny = 9
    K = ob.squared_laplacian_kron(nx, ny, "dirichlet", "dirichlet")
    j, i = 4, 4
    row = K.getrow(j * nx + i).toarray().reshape(ny, nx)
    expect = np.zeros((ny, nx))
    expect[j, i] = 20
    for dj, di in [(-1, 0), (1, 0), (0, -1), (0, 1)]:
        expect[j + dj, i + di] = -8
    for dj, di in [(-1, -1), (-1, 1), (1, -1), (1, 1)]:
        expect[j + dj, i + di] = 2
    for dj, di in [(-2, 0), (2, 0), (0, -2), (0, 2)]:
        expect[j + dj, i + di] = 1
    assert np.array_equal(row, expect)


def test_dirichlet_padding_gives_zero_laplacian_on_boundary():
    """Algorithm 1's padding makes f = 0 and lap f = 0 on the boundary (eq. boundary conditions):
    the padded two-pass result equals T^2 with T = tridiag(-1, 2, -1) in 1-D rows."""
    n = 6
    T = np.diag(np.full(n, 2.0)) - np.diag(np.ones(n - 1), 1) - np.diag(np.ones(n - 1), -1)
    F = np.zeros((n, n))
    F[2, :] = np.arange(1, n + 1)
    out = ob.apply_squared_laplacian_padded(F, "dirichlet", "dirichlet")
    L = np.kron(T, np.eye(n)) + np.kron(np.eye(n), T)
    np.testing.assert_array_equal(out.ravel(), L @ L @ F.ravel())


# -------------------------------------------------------------------------------------------
# SPD (Sec. 2.2 calls the system symmetric positive definite)
# -------------------------------------------------------------------------------------------
@pytest.mark.parametrize("bc_x,bc_y", BC_PAIRS)
def test_operator_is_spd_with_bounded_spectrum(bc_x, bc_y):
    phi, f = _random_problem(9, 8, 3)
    A, b, unk, known = ob.system(phi, f, "out", bc_x, bc_y)
    Ad = A.toarray()
    rng = np.random.default_rng(0)
    for _ in range(5):
        x, y = rng.standard_normal((2, Ad.shape[0]))
        assert abs(x @ Ad @ y - y @ Ad @ x) <= 1e-14 * np.abs(Ad).sum() * np.abs(x).max() * np.abs(y).max()
        assert x @ Ad @ x > 0
    ev = np.linalg.eigvalsh(Ad)
    # Cauchy interlacing with L^2, whose eigenvalues are (lambda_x + lambda_y)^2 < 64 for h = 1
    assert ev.min() > 0 and ev.max() <= 64.0


# -------------------------------------------------------------------------------------------
# Solution: brute force by least squares on the Laplacian (a different characterisation)
# -------------------------------------------------------------------------------------------
@pytest.mark.parametrize("bc_x,bc_y", BC_PAIRS)
@pytest.mark.parametrize("direction", ["out", "in"])
@pytest.mark.parametrize("nx,ny", [(6, 6), (11, 9), (16, 16)])
def test_solution_minimises_laplacian_energy(bc_x, bc_y, direction, nx, ny):
    """The extension minimises ||L F||^2 over full-grid F that equal f on Omega (the discrete
    bending energy behind the thin plate spline, Sec. 2.1).  Solve that least-squares problem
    densely and compare with the direct, CG and PCG solutions of A x = b."""
    phi, f = _random_problem(nx, ny, nx * 31 + ny, frac=0.5)
    if direction == "in":
        phi = -phi
    known = ob.known_mask(phi, direction)
    if not known.any():
        pytest.skip("no known node")
    L = ob.laplacian(nx, ny, bc_x, bc_y).toarray()
    unk = np.flatnonzero(~known.ravel())
    fk = np.where(known, f, 0.0).ravel()
    x_ls, *_ = np.linalg.lstsq(L[:, unk], -L @ fk, rcond=None)
    ref = ob.assemble(x_ls, f, unk, known)
    scale = np.abs(ref).max()
    for method in ("direct", "cg", "pcg"):
        out, info = ob.extend(phi, f, direction, bc_x, bc_y, method=method, rtol=1e-13)
        np.testing.assert_allclose(out, ref, rtol=0, atol=1e-9 * scale, err_msg=method)


def test_known_nodes_are_reproduced_bitwise():
    p = synth.single_fp64_case()
    out, _ = ob.extend(p.phi, p.f, p.direction, p.bc_x, p.bc_y, method="direct")
    known = ob.known_mask(p.phi.astype(np.float64), p.direction)
    assert np.array_equal(out[known], p.f.astype(np.float64)[known])


def test_phi_zero_is_unknown_in_both_directions():
    phi = np.array([[-1.0, 0.0, 1.0]])
    assert ob.known_mask(phi, "out").tolist() == [[True, False, False]]
    assert ob.known_mask(phi, "in").tolist() == [[False, False, True]]


@pytest.mark.parametrize("bc", ["symmetric", "periodic"])
def test_constant_field_extends_to_constant(bc):
    """L^2 annihilates constants on symmetric/periodic grids, so a constant is the extension."""
    p = synth.circle(32, bc)
    f = np.full_like(p.f, 2.5)
    out, _ = ob.extend(p.phi, f, "out", bc, bc, method="direct")
    np.testing.assert_allclose(out, 2.5, rtol=0, atol=1e-11)


def test_no_known_node_is_rejected_for_symmetric_edges():
    with pytest.raises(ValueError):
        ob.extend(np.ones((8, 8)), np.zeros((8, 8)), "out", "symmetric", "periodic")
    out, info = ob.extend(np.ones((8, 8)), np.zeros((8, 8)), "out", "dirichlet", "symmetric")
    assert np.all(out == 0)


# -------------------------------------------------------------------------------------------
# Symmetry and periodicity (Sec. 1; Example 3's half-grid claim; Examples 2 and 4)
# -------------------------------------------------------------------------------------------
def test_mirror_symmetric_input_gives_mirror_symmetric_output():
    n = 40
    X, Y, hx, hy = synth.grid(n, n, "symmetric", "symmetric")
    phi = np.sqrt(X ** 2 + (Y - 0.1) ** 2) - 0.45 + 0.05 * np.cos(3 * Y)
    f = np.cos(2 * X) * np.sin(3 * Y) + X ** 2
    out, _ = ob.extend(phi, f, "out", "symmetric", "symmetric", hx, hy)
    np.testing.assert_allclose(out, out[:, ::-1], rtol=0, atol=1e-12 * np.abs(out).max())


def test_half_grid_with_symmetric_edge_equals_full_grid():
    """Example 3: solving on half the domain with a symmetry edge reproduces the full solution.
    On a cell-centred grid the mirror line lies between nodes, so the half grid is the right half
    of the full grid with a symmetric left edge."""
    n = 48
    X, Y, hx, hy = synth.grid(n, n, "symmetric", "dirichlet")
    r = np.sqrt(X ** 2 + Y ** 2)
    phi = np.abs(r - 0.6) - 0.15  # annulus band known
    f = Y / np.log(1.0 + 4 * r)
    full, _ = ob.extend(phi, f, "out", "symmetric", "dirichlet", hx, hy)
    half, _ = ob.extend(phi[:, n // 2:], f[:, n // 2:], "out", "symmetric", "dirichlet", hx, hy)
    np.testing.assert_allclose(half, full[:, n // 2:], rtol=0, atol=1e-11 * np.abs(full).max())


def test_periodic_shift_equivariance():
    p = synth.star(36, "periodic", "in")
    sy, sx = 5, 11
    out, _ = ob.extend(p.phi, p.f, "in", "periodic", "periodic")
    sh, _ = ob.extend(np.roll(p.phi, (sy, sx), (0, 1)), np.roll(p.f, (sy, sx), (0, 1)), "in",
                      "periodic", "periodic")
    np.testing.assert_allclose(sh, np.roll(out, (sy, sx), (0, 1)), rtol=0,
                               atol=1e-11 * np.abs(out).max())


def test_inner_region_decoupled_from_outer_boundary_rule():
    """Example 3: unknowns enclosed by a known annulus at least two cells wide are coupled only
    to the annulus, so they do not depend on the outer boundary rule."""
    n = 40
    X, Y, hx, hy = synth.grid(n, n, "symmetric", "symmetric")
    r = np.sqrt(X ** 2 + Y ** 2)
    phi = np.abs(r - 0.5) - 0.2  # known for 0.3 < r < 0.7 (about 8 cells wide)
    f = np.sin(3 * X) + Y
    a, _ = ob.extend(phi, f, "out", "dirichlet", "dirichlet", hx, hy)
    b, _ = ob.extend(phi, f, "out", "symmetric", "symmetric", hx, hy)
    inner = r < 0.3
    np.testing.assert_allclose(a[inner], b[inner], rtol=0, atol=1e-11)
    assert np.abs(a - b)[r > 0.7].max() > 1e-3  # the outside does feel the boundary rule


# -------------------------------------------------------------------------------------------
# Manufactured solution and the fast Poisson preconditioner
# -------------------------------------------------------------------------------------------
@pytest.mark.parametrize("bc_x,bc_y", BC_PAIRS)
def test_manufactured_solution(bc_x, bc_y):
    phi, f = _random_problem(20, 18, 7)
    A, _, unk, known = ob.system(phi, f, "out", bc_x, bc_y)
    g = np.random.default_rng(1).standard_normal(unk.size)
    for method in ("direct", "pcg"):
        if method == "direct":
            x = ob.solve_direct(A, A @ g)
        else:
            M = ob.fast_poisson_preconditioner(unk, 18, 20, bc_x, bc_y)
            x, it, _ = ob.cg(A, A @ g, rtol=1e-13, precond=M)
        np.testing.assert_allclose(x, g, rtol=0, atol=1e-8)


@pytest.mark.parametrize("bc_x,bc_y", BC_PAIRS)
@pytest.mark.parametrize("hx,hy", [(1.0, 1.0), (0.5, 0.8)])
def test_fast_poisson_inverts_squared_laplacian(bc_x, bc_y, hx, hy):
    """(L^2)^+ L^2 v = v, or v minus its mean when both axes carry a constant null vector."""
    nx, ny = 12, 10
    v = np.random.default_rng(5).standard_normal((ny, nx))
    L2 = ob.squared_laplacian_kron(nx, ny, bc_x, bc_y, hx, hy)
    z = ob.poisson_squared_pinv((L2 @ v.ravel()).reshape(ny, nx), bc_x, bc_y, hx, hy)
    expect = v - v.mean() if (bc_x != "dirichlet" and bc_y != "dirichlet") else v
    np.testing.assert_allclose(z, expect, rtol=0, atol=1e-10 * np.abs(v).max())


def test_preconditioned_cg_is_exact_with_nothing_known():
    """With Omega empty and Dirichlet edges the preconditioner is A^-1: one PCG iteration."""
    n = 16
    phi = np.ones((n, n))
    A, _, unk, _ = ob.system(phi, np.zeros((n, n)), "out", "dirichlet", "dirichlet")
    b = np.random.default_rng(2).standard_normal(unk.size)
    M = ob.fast_poisson_preconditioner(unk, n, n, "dirichlet", "dirichlet")
    x, it, rel = ob.cg(A, b, rtol=1e-10, precond=M)
    assert it == 1 and rel < 1e-12


def test_preconditioner_cuts_iterations():
    p = synth.single_fp64_case()
    _, i_cg = ob.extend(p.phi, p.f, p.direction, p.bc_x, p.bc_y, method="cg", rtol=1e-10)
    _, i_pcg = ob.extend(p.phi, p.f, p.direction, p.bc_x, p.bc_y, method="pcg", rtol=1e-10)
    assert i_pcg["iters"] * 5 < i_cg["iters"]
    assert i_cg["relres"] < 1e-9 and i_pcg["relres"] < 1e-9


# -------------------------------------------------------------------------------------------
# The paper's printed numbers (Example 1, Table 1)
# -------------------------------------------------------------------------------------------
def _example1(n, bc):
    a, b = -np.pi, np.pi
    if bc == "dirichlet":
        h = (b - a) / (n + 1)
        xs = a + (np.arange(n) + 1) * h
    else:
        h = (b - a) / n
        xs = a + (np.arange(n) + 0.5) * h
    X, Y = np.meshgrid(xs, xs)
    phi = np.minimum(np.hypot(X - 0.8, Y) - 1, np.hypot(X + 0.8, Y) - 1)
    return phi, np.cos(X) * np.sin(Y), h


def _golden_table1():
    rows = {}
    with open(os.path.join(GOLDEN, "example1_table1.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            bc, n, it, err = line.split()
            rows[(bc, int(n))] = (int(it), float(err))
    return rows


@pytest.mark.parametrize("bc", ["dirichlet", "symmetric"])
def test_example1_errors_and_iterations_match_table1(bc):
    """Example 1 at 128^2 and 256^2: errors within 4 cells of the interface match Table 1 to
    about 20% (node placement is not stated in the paper), the estimated order is about 2, and
    the PCG iteration counts at tol 1e-6 are within 20% of the printed ones."""
    table = _golden_table1()
    errs = []
    for n in (128, 256):
        phi, f, h = _example1(n, bc)
        out, info = ob.extend(phi, f, "out", bc, bc, h, h, method="pcg", rtol=1e-6)
        err = np.abs(out - f)[np.abs(phi) <= 4 * h].max()
        it_ref, err_ref = table[(bc, n)]
        assert abs(err / err_ref - 1) < 0.2, (n, err, err_ref)
        assert abs(info["iters"] / it_ref - 1) < 0.2, (n, info["iters"], it_ref)
        errs.append(err)
    order = np.log2(errs[0] / errs[1])
    assert 1.7 < order < 2.2


# -------------------------------------------------------------------------------------------
# Right-hand side on the full grid (Algorithm 1, first statement) and the residual measure
# -------------------------------------------------------------------------------------------
@pytest.mark.parametrize("bc_x,bc_y", BC_PAIRS)
@pytest.mark.parametrize("direction", ["out", "in"])
def test_rhs_padded_equals_system_rhs_on_integers(bc_x, bc_y, direction):
    """rhs_padded (Algorithm 1's padded two-pass stencil on the grid) scattered against b of the
    assembled system (Kronecker construction, restricted to the unknowns): two independent routes
    to -R L^2 E_K f.  With h = 1 and integer f both are exact integers, so they agree bit for bit;
    known nodes hold zero."""
    nx, ny = 13, 11
    phi, _ = _random_problem(nx, ny, 17)
    if direction == "in":
        phi = -phi
    f = np.random.default_rng(5).integers(-300, 301, (ny, nx)).astype(np.float64)
    A, b, unk, known = ob.system(phi, f, direction, bc_x, bc_y)
    B = ob.rhs_padded(phi, f, direction, bc_x, bc_y)
    full = np.zeros(nx * ny)
    full[unk] = b
    assert np.array_equal(B.ravel(), full)
    assert np.all(B[known] == 0)
    # the sign: for one known node of value 1 in the interior, b at its edge neighbour is +8
    # (minus the -8 coefficient of eq. discrete_biharmonic)
    phi1 = np.ones((9, 9)) * (1.0 if direction == "out" else -1.0)
    phi1[4, 4] = -phi1[4, 4]
    f1 = np.zeros((9, 9))
    f1[4, 4] = 1.0
    B1 = ob.rhs_padded(phi1, f1, direction, bc_x, bc_y)
    assert B1[4, 5] == 8.0 and B1[5, 5] == -2.0 and B1[4, 6] == -1.0 and B1[4, 4] == 0.0


def test_rhs_padded_anisotropic_matches_system():
    phi, f = _random_problem(10, 7, 23)
    hx, hy = 0.4, 0.9
    A, b, unk, known = ob.system(phi, f, "out", "periodic", "dirichlet", hx, hy)
    B = ob.rhs_padded(phi, f, "out", "periodic", "dirichlet", hx, hy)
    np.testing.assert_allclose(B.ravel()[unk], b, rtol=1e-13, atol=1e-12 * np.abs(b).max())


@pytest.mark.parametrize("bc_x,bc_y", BC_PAIRS)
def test_true_relative_residual_against_dense_brute_force(bc_x, bc_y):
    """true_relative_residual is ||b - A x|| / ||b|| on the unknowns.  The reference builds A and
    b densely from the 13-point tap table (a construction the function does not use), and a
    planted residual pins the value: x = x* + A^-1 v has residual exactly -v."""
    nx, ny = 12, 10
    phi, f = _random_problem(nx, ny, 41, frac=0.5)
    known = ob.known_mask(phi, "out")
    L2 = ob.squared_laplacian_stencil(nx, ny, bc_x, bc_y).toarray()
    unk = np.flatnonzero(~known.ravel())
    Ad = L2[np.ix_(unk, unk)]
    bd = -(L2 @ np.where(known, f, 0.0).ravel())[unk]
    xs = np.linalg.solve(Ad, bd)
    rng = np.random.default_rng(7)
    v = rng.standard_normal(unk.size) * 1e-3 * np.linalg.norm(bd) / np.sqrt(unk.size)
    x = xs + np.linalg.solve(Ad, v)
    out = ob.assemble(x, f, unk, known)
    got = ob.true_relative_residual(out, phi, f, "out", bc_x, bc_y)
    want = np.linalg.norm(v) / np.linalg.norm(bd)
    assert abs(got - want) <= 1e-9 * want
    # values at known nodes of `out` are not part of the measure
    out2 = out.copy()
    out2[known] += 123.0
    assert ob.true_relative_residual(out2, phi, f, "out", bc_x, bc_y) == got
    # the exact solution has a residual at round-off level
    assert ob.true_relative_residual(ob.assemble(xs, f, unk, known), phi, f, "out", bc_x, bc_y) < 1e-12
