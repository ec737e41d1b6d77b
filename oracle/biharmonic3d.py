"""FP64 CPU oracle for the three-dimensional biharmonic field extension (Moroney et al., arXiv
1704.08897, Sec. 3 Example 2: the same equations in three dimensions).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` may import it.  It shares no code with the CUDA library; it reuses the
two-dimensional oracle's per-axis pieces (the 1-D second difference, ghost padding, transforms and
the CG loop), which are pinned there.

What it computes: for a level set function phi on an nz-by-ny-by-nx grid (row-major, x
contiguous) and a field f known on Omega, the solution of

    A x = b,   A = R (L_z (+) L_y (+) L_x)^2 R^T,   b = -R (L_z (+) L_y (+) L_x)^2 E_K f

with L_a = T_a / h_a^2 the 1-D second difference of axis a under its boundary rule (the same
three rules as in two dimensions).  For hx = hy = hz the operator at an interior node is the
squared 7-point Laplacian, a 25-point stencil: 42 at the centre, -12 at the six face neighbours,
2 at the twelve edge neighbours and 1 at the six nodes two steps along an axis, divided by h^4.

Three constructions are kept so the tests can pin each against the others: the Kronecker form,
the pad-then-apply-the-7-point-Laplacian-twice form (Algorithm 1 in three dimensions), and a
25-point tap table with per-axis ghost maps.  The preconditioner is the fast Poisson solve of
L^2 on the box by separable transforms along the three axes (Example 2 uses discrete Fourier
transforms in all three), with the zero eigenvalue dropped when no axis is Dirichlet.
"""

from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from oracle import biharmonic as ob

AXES = ("z", "y", "x")


def laplacian3(nx, ny, nz, bc_x, bc_y, bc_z, hx=1.0, hy=1.0, hz=1.0) -> sp.csr_matrix:
    """L = L_z (+) L_y (+) L_x on the full grid, [z][y][x] row-major (x fastest)."""
    Tx = ob.axis_second_difference(nx, bc_x, hx)
    Ty = ob.axis_second_difference(ny, bc_y, hy)
    Tz = ob.axis_second_difference(nz, bc_z, hz)
    Ix, Iy, Iz = sp.identity(nx), sp.identity(ny), sp.identity(nz)
    return (sp.kron(sp.kron(Tz, Iy), Ix) + sp.kron(sp.kron(Iz, Ty), Ix)
            + sp.kron(sp.kron(Iz, Iy), Tx)).tocsr()


def squared_laplacian3_kron(nx, ny, nz, bc_x, bc_y, bc_z, hx=1.0, hy=1.0, hz=1.0) -> sp.csr_matrix:
    """Construction 1: L^2 as the product of the Kronecker-sum Laplacian with itself."""
    L = laplacian3(nx, ny, nz, bc_x, bc_y, bc_z, hx, hy, hz)
    return (L @ L).tocsr()


def apply_squared_laplacian3_padded(F, bc_x, bc_y, bc_z, hx=1.0, hy=1.0, hz=1.0) -> np.ndarray:
    """Construction 2: L^2 F by padding two ghost layers per axis and applying the 7-point
    Laplacian twice (first on the grid plus one ghost layer, then on the grid)."""
    P = np.asarray(F, dtype=np.float64)
    for axis, bc in ((0, bc_z), (1, bc_y), (2, bc_x)):
        P = ob._pad_axis(P, axis, bc)
    c = (1.0 / (hz * hz), 1.0 / (hy * hy), 1.0 / (hx * hx))

    def lap(Q):
        C = Q[1:-1, 1:-1, 1:-1]
        return ((2 * c[0] + 2 * c[1] + 2 * c[2]) * C
                - c[0] * (Q[:-2, 1:-1, 1:-1] + Q[2:, 1:-1, 1:-1])
                - c[1] * (Q[1:-1, :-2, 1:-1] + Q[1:-1, 2:, 1:-1])
                - c[2] * (Q[1:-1, 1:-1, :-2] + Q[1:-1, 1:-1, 2:]))

    return lap(lap(P))


def stencil25_taps(hx=1.0, hy=1.0, hz=1.0):
    """Tap table (dz, dy, dx, weight) of the squared 7-point Laplacian: with c_a = 1/h_a^2,
    L^2 = sum_a c_a^2 T_a^2 + 2 sum_{a<b} c_a c_b T_a T_b, T = [-1, 2, -1] along its axis."""
    c = {"z": 1.0 / (hz * hz), "y": 1.0 / (hy * hy), "x": 1.0 / (hx * hx)}
    unit = {"z": (1, 0, 0), "y": (0, 1, 0), "x": (0, 0, 1)}
    taps = {(0, 0, 0): 6 * sum(v * v for v in c.values())
            + 8 * (c["z"] * c["y"] + c["z"] * c["x"] + c["y"] * c["x"])}
    for a in AXES:
        others = sum(c[b] for b in AXES if b != a)
        for s in (-1, 1):
            taps[tuple(s * u for u in unit[a])] = -4 * c[a] * c[a] - 4 * c[a] * others
        for s in (-2, 2):
            taps[tuple(s * u for u in unit[a])] = c[a] * c[a]
    for i, a in enumerate(AXES):
        for b in AXES[i + 1:]:
            for sa in (-1, 1):
                for sb in (-1, 1):
                    off = tuple(sa * ua + sb * ub for ua, ub in zip(unit[a], unit[b]))
                    taps[off] = 2 * c[a] * c[b]
    return [(dz, dy, dx, w) for (dz, dy, dx), w in taps.items()]


def squared_laplacian3_stencil(nx, ny, nz, bc_x, bc_y, bc_z, hx=1.0, hy=1.0, hz=1.0):
    """Construction 3: full-grid L^2 assembled from the 25 taps and per-axis ghost maps."""
    rows, cols, vals = [], [], []
    taps = stencil25_taps(hx, hy, hz)
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                r = (k * ny + j) * nx + i
                for dz, dy, dx, w in taps:
                    gz = ob._ghost(k + dz, nz, bc_z)
                    gy = ob._ghost(j + dy, ny, bc_y)
                    gx = ob._ghost(i + dx, nx, bc_x)
                    if gz is None or gy is None or gx is None:
                        continue
                    rows.append(r)
                    cols.append((gz[0] * ny + gy[0]) * nx + gx[0])
                    vals.append(w * gz[1] * gy[1] * gx[1])
    N = nx * ny * nz
    return sp.csr_matrix((vals, (rows, cols)), shape=(N, N))


def system3(phi, f, direction, bcs, hs=(1.0, 1.0, 1.0), construction="kron"):
    """(A, b, unknown_index, known_mask) for the 3-D extension; bcs = (bc_x, bc_y, bc_z),
    hs = (hx, hy, hz)."""
    nz, ny, nx = phi.shape
    known = ob.known_mask(phi, direction)
    if construction == "kron":
        L2 = squared_laplacian3_kron(nx, ny, nz, *bcs, *hs)
    elif construction == "stencil":
        L2 = squared_laplacian3_stencil(nx, ny, nz, *bcs, *hs)
    else:
        raise ValueError(construction)
    unk = np.flatnonzero(~known.ravel())
    fk = np.where(known, f, 0.0).astype(np.float64).ravel()
    b = -(L2 @ fk)[unk]
    A = L2[unk][:, unk].tocsr()
    return A, b, unk, known


def rhs3_padded(phi, f, direction, bcs, hs=(1.0, 1.0, 1.0)):
    """b on the full grid (zeros at known nodes) through the padded two-pass stencil."""
    known = ob.known_mask(phi, direction)
    fk = np.where(known, f, 0.0).astype(np.float64)
    B = -apply_squared_laplacian3_padded(fk, *bcs, *hs)
    return np.where(known, 0.0, B)


def poisson_squared_pinv3(B, bcs, hs=(1.0, 1.0, 1.0)) -> np.ndarray:
    """Z = (L^2)^+ B on the box: transform the three axes, divide by the squared eigenvalue
    sums, transform back; the zero eigenvalue (no Dirichlet axis) is dropped."""
    nz, ny, nx = B.shape
    bc_x, bc_y, bc_z = bcs
    hx, hy, hz = hs
    Z = ob._forward(ob._forward(ob._forward(B.astype(np.float64), 2, bc_x), 1, bc_y), 0, bc_z)
    LL = (ob.axis_eigenvalues(nz, bc_z, hz)[:, None, None] + ob.axis_eigenvalues(ny, bc_y, hy)[None, :, None]
          + ob.axis_eigenvalues(nx, bc_x, hx)[None, None, :])
    with np.errstate(divide="ignore"):
        W = np.where(LL > 0, 1.0 / (LL * LL), 0.0)
    if "dirichlet" not in bcs:
        W[0, 0, 0] = 0.0
    Z = ob._inverse(ob._inverse(ob._inverse(Z * W, 0, bc_z), 1, bc_y), 2, bc_x)
    return np.real(Z)


def fast_poisson_preconditioner3(unk, shape, bcs, hs=(1.0, 1.0, 1.0)):
    """z = R (L^2)^+ R^T r by zero-augmentation to the box and the transform solve."""
    def apply(r):
        B = np.zeros(int(np.prod(shape)))
        B[unk] = r
        return poisson_squared_pinv3(B.reshape(shape), bcs, hs).ravel()[unk]
    return apply


def extend3(phi, f, direction="out", bcs=("periodic",) * 3, hs=(1.0, 1.0, 1.0), method="direct",
            rtol=1e-10, maxit=None):
    """Biharmonic extension of f from Omega to the whole box; method 'direct' or 'pcg'.
    Returns (out, info) with info = {iters, relres, n_unknown, n_known}."""
    phi = np.asarray(phi, dtype=np.float64)
    f = np.asarray(f)
    known = ob.known_mask(phi, direction)
    if not known.any() and "dirichlet" not in bcs:
        raise ValueError("no known node: the extension is not unique without a Dirichlet axis")
    A, b, unk, known = system3(phi, f, direction, bcs, hs)
    info = {"n_unknown": int(unk.size), "n_known": int(known.sum())}
    if method == "direct":
        x = ob.solve_direct(A, b)
        it = 0
    elif method == "pcg":
        M = fast_poisson_preconditioner3(unk, phi.shape, bcs, hs)
        x, it, _ = ob.cg(A, b, rtol=rtol, maxit=maxit, precond=M)
    else:
        raise ValueError(method)
    bn = np.linalg.norm(b)
    info["iters"] = it
    info["relres"] = float(np.linalg.norm(b - A @ x) / bn) if bn > 0 else 0.0
    return ob.assemble(x, f, unk, known), info


def true_relative_residual3(out, phi, f, direction, bcs, hs=(1.0, 1.0, 1.0)):
    """||b - A x|| / ||b|| for a full-grid answer ``out``, FP64."""
    A, b, unk, _ = system3(np.asarray(phi, np.float64), np.asarray(f), direction, bcs, hs)
    x = np.asarray(out, dtype=np.float64).ravel()[unk]
    bn = np.linalg.norm(b)
    return float(np.linalg.norm(b - A @ x) / bn) if bn > 0 else float(np.linalg.norm(A @ x))
