"""FP64 CPU oracle for the biharmonic field extension (Moroney et al., arXiv 1704.08897).

TEST INFRASTRUCTURE ONLY.  This module is the plain, slow, obviously correct statement of what
the GPU path computes.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it.  It shares no code with the CUDA library and imports nothing from the
package.

What it computes (Sec. 2.1, eqs. ``biharmonic`` .. ``biharmonic_interpolation_constraints`` and
``discrete_biharmonic``): given a level set function phi on an ny-by-nx grid (row-major, x
contiguous) and a field f whose values are known on Omega, the extension is the unique solution of

    A x = b,   A = R (L_y (+) L_x)^2 R^T,   b = -R (L_y (+) L_x)^2 E_K f

where R restricts to the unknown nodes D\\Omega, E_K embeds the known values with zeros elsewhere,
and L_a = T_a / h_a^2 is the 1-D 5-point second difference for the boundary rule of axis a:

* ``dirichlet``: the padding of Algorithm 1 (boundary node zero, outer ghost is the negated first
  node), which gives T = tridiag(-1, 2, -1);
* ``symmetric`` (the Neumann case of Example 1): half-sample reflection u[-1] = u[0],
  u[-2] = u[1], which gives T with T[0,0] = T[n-1,n-1] = 1;
* ``periodic`` (Example 2, Example 4): wrap-around ghosts, T the circulant.

For hx = hy the operator at every unknown node is exactly the 13-point stencil of eq.
``discrete_biharmonic`` divided by h^4.

Three independent constructions of the operator are kept so the tests can pin each against the
others: the Kronecker form, Algorithm 1's pad-then-apply-the-5-point-Laplacian-twice form, and a
13-point tap table with per-axis ghost maps.

Solvers: sparse direct (SuperLU), own-loop unpreconditioned CG, and CG preconditioned by the fast
Poisson solve of Algorithm 1 / Sec. 2.2 (the embedding of D\\Omega into D by zero-augmentation and
a separable transform solve of L^2 on the rectangle), built on ``scipy.fft``.

Readings where the paper is silent: the zero eigenvalue of L^2 for symmetric/periodic axes is
dropped (pseudo-inverse); phi == 0 counts as unknown in both directions; the tolerance is the
relative 2-norm residual on the unknowns with x0 = 0.
"""

from __future__ import annotations

import numpy as np
import scipy.fft as sfft
import scipy.sparse as sp
import scipy.sparse.linalg as spla

BCS = ("symmetric", "periodic", "dirichlet")
EXTEND_OUT = "out"  # field known inside (phi < 0), Fig. 1(a)
EXTEND_IN = "in"    # field known outside (phi > 0), Fig. 1(b)


# ----------------------------------------------------------------------------------------------
# Known region (Sec. 2.1; Example 1 defines Omega by a strict inequality on phi)
# ----------------------------------------------------------------------------------------------
def known_mask(phi: np.ndarray, direction: str) -> np.ndarray:
    """Boolean mask of the known nodes Omega.

    Extend out (Fig. 1(a)): the field is known inside the interface, phi < 0.
    Extend in (Fig. 1(b)): the field is known outside, phi > 0.  phi == 0 is unknown either way.
    """
    if direction == EXTEND_OUT:
        return phi < 0
    if direction == EXTEND_IN:
        return phi > 0
    raise ValueError(f"direction must be 'out' or 'in', got {direction!r}")


# ----------------------------------------------------------------------------------------------
# Operator, construction 1: Kronecker form R (L_y (+) L_x)^2 R^T
# ----------------------------------------------------------------------------------------------
def axis_second_difference(n: int, bc: str, h: float = 1.0) -> sp.csr_matrix:
    """1-D negative second difference T/h^2 of size n for one axis's boundary rule."""
    if n < 3:
        raise ValueError("each axis needs at least 3 nodes")
    main = np.full(n, 2.0)
    off = np.full(n - 1, -1.0)
    T = sp.diags([off, main, off], [-1, 0, 1], shape=(n, n), format="lil")
    if bc == "symmetric":
        T[0, 0] = 1.0
        T[n - 1, n - 1] = 1.0
    elif bc == "periodic":
        T[0, n - 1] += -1.0
        T[n - 1, 0] += -1.0
    elif bc != "dirichlet":
        raise ValueError(f"unknown bc {bc!r}")
    return (T.tocsr() / (h * h)).tocsr()


def laplacian(nx: int, ny: int, bc_x: str, bc_y: str, hx: float = 1.0, hy: float = 1.0):
    """Full-grid negative Laplacian L = L_y (x) I + I (x) L_x for row-major [y][x] storage."""
    Lx = axis_second_difference(nx, bc_x, hx)
    Ly = axis_second_difference(ny, bc_y, hy)
    return (sp.kron(Ly, sp.identity(nx)) + sp.kron(sp.identity(ny), Lx)).tocsr()


def squared_laplacian_kron(nx, ny, bc_x, bc_y, hx=1.0, hy=1.0) -> sp.csr_matrix:
    L = laplacian(nx, ny, bc_x, bc_y, hx, hy)
    return (L @ L).tocsr()


# ----------------------------------------------------------------------------------------------
# Operator, construction 2: Algorithm 1's padded array, 5-point Laplacian applied twice
# ----------------------------------------------------------------------------------------------
def _pad_axis(F: np.ndarray, axis: int, bc: str) -> np.ndarray:
    """Pad two ghost layers on both ends of one axis, following the boundary rule.

    Dirichlet follows Algorithm 1: the first ghost is the (zero) boundary node, the second ghost is
    the negated first interior node.  Symmetric is half-sample reflection; periodic wraps.
    """
    F = np.moveaxis(F, axis, 0)
    n = F.shape[0]
    out = np.zeros((n + 4,) + F.shape[1:], dtype=F.dtype)
    out[2:n + 2] = F
    if bc == "dirichlet":
        out[1] = 0.0
        out[0] = -F[0]
        out[n + 2] = 0.0
        out[n + 3] = -F[n - 1]
    elif bc == "symmetric":
        out[1] = F[0]
        out[0] = F[1]
        out[n + 2] = F[n - 1]
        out[n + 3] = F[n - 2]
    elif bc == "periodic":
        out[1] = F[n - 1]
        out[0] = F[n - 2]
        out[n + 2] = F[0]
        out[n + 3] = F[1]
    else:
        raise ValueError(bc)
    return np.moveaxis(out, 0, axis)


def apply_squared_laplacian_padded(F: np.ndarray, bc_x: str, bc_y: str,
                                   hx: float = 1.0, hy: float = 1.0) -> np.ndarray:
    """L^2 F on the full grid by padding and two passes of the 5-point Laplacian (Algorithm 1).

    F is [ny][nx].  The padding is applied once to the field (two ghost layers); the first pass
    evaluates the Laplacian on the grid plus one ghost layer, the second on the grid itself.
    For periodic and symmetric axes the once-padded Laplacian on the ghost layer equals the
    reflected/wrapped Laplacian, so the two passes compose to (L_y (+) L_x)^2.
    """
    P = _pad_axis(_pad_axis(np.asarray(F, dtype=np.float64), 0, bc_y), 1, bc_x)
    cx, cy = 1.0 / (hx * hx), 1.0 / (hy * hy)
    # first pass on rows/cols 1..n+2 of the padded array (grid plus one ghost ring)
    C = P[1:-1, 1:-1]
    Lp = (2 * cx + 2 * cy) * C - cx * (P[1:-1, :-2] + P[1:-1, 2:]) - cy * (P[:-2, 1:-1] + P[2:, 1:-1])
    C2 = Lp[1:-1, 1:-1]
    return ((2 * cx + 2 * cy) * C2 - cx * (Lp[1:-1, :-2] + Lp[1:-1, 2:])
            - cy * (Lp[:-2, 1:-1] + Lp[2:, 1:-1]))


# ----------------------------------------------------------------------------------------------
# Operator, construction 3: the 13-point stencil of eq. discrete_biharmonic with ghost maps
# ----------------------------------------------------------------------------------------------
def _ghost(i: int, n: int, bc: str):
    """Map an index that may lie up to 2 outside [0, n) to (index, sign) or None (a zero node)."""
    if 0 <= i < n:
        return i, 1.0
    if bc == "periodic":
        return i % n, 1.0
    if bc == "symmetric":
        return (-1 - i, 1.0) if i < 0 else (2 * n - 1 - i, 1.0)
    # dirichlet: the node at distance 1 is the boundary (zero); distance 2 is the odd reflection
    if i == -1 or i == n:
        return None
    return (-i - 2, -1.0) if i < 0 else (2 * n - i, -1.0)


def stencil13_taps(hx: float = 1.0, hy: float = 1.0):
    """Tap table (dy, dx, weight) of the squared 5-point Laplacian.

    For hx = hy = 1 these are the coefficients of eq. discrete_biharmonic: 20 at the centre, -8 at
    the four edge neighbours, 2 on the diagonals and 1 at distance two.
    """
    a, c = 1.0 / (hx * hx), 1.0 / (hy * hy)
    taps = [(0, 0, 6 * a * a + 8 * a * c + 6 * c * c)]
    taps += [(0, s, -4 * a * a - 4 * a * c) for s in (-1, 1)]
    taps += [(s, 0, -4 * c * c - 4 * a * c) for s in (-1, 1)]
    taps += [(sy, sx, 2 * a * c) for sy in (-1, 1) for sx in (-1, 1)]
    taps += [(0, s, a * a) for s in (-2, 2)]
    taps += [(s, 0, c * c) for s in (-2, 2)]
    return taps


def squared_laplacian_stencil(nx, ny, bc_x, bc_y, hx=1.0, hy=1.0) -> sp.csr_matrix:
    """Full-grid L^2 assembled row by row from the 13-point taps and per-axis ghost maps."""
    rows, cols, vals = [], [], []
    taps = stencil13_taps(hx, hy)
    for j in range(ny):
        for i in range(nx):
            r = j * nx + i
            for dy, dx, w in taps:
                gy = _ghost(j + dy, ny, bc_y)
                gx = _ghost(i + dx, nx, bc_x)
                if gy is None or gx is None:
                    continue
                rows.append(r)
                cols.append(gy[0] * nx + gx[0])
                vals.append(w * gy[1] * gx[1])
    N = nx * ny
    return sp.csr_matrix((vals, (rows, cols)), shape=(N, N))


# ----------------------------------------------------------------------------------------------
# Linear system (Algorithm 1: right-hand side from the known values, operator on D\Omega)
# ----------------------------------------------------------------------------------------------
def system(phi, f, direction, bc_x, bc_y, hx=1.0, hy=1.0, construction="kron"):
    """Return (A, b, unknown_index, known_mask) for the extension problem.

    b = -R L^2 E_K f: the stencil applied to the field with the unknowns zeroed, restricted to the
    unknowns (the first statement of Algorithm 1).
    """
    ny, nx = phi.shape
    known = known_mask(phi, direction)
    if construction == "kron":
        L2 = squared_laplacian_kron(nx, ny, bc_x, bc_y, hx, hy)
    elif construction == "stencil":
        L2 = squared_laplacian_stencil(nx, ny, bc_x, bc_y, hx, hy)
    else:
        raise ValueError(construction)
    unk = np.flatnonzero(~known.ravel())
    fk = np.where(known, f, 0.0).astype(np.float64).ravel()
    b = -(L2 @ fk)[unk]
    A = L2[unk][:, unk].tocsr()
    return A, b, unk, known


def rhs_padded(phi, f, direction, bc_x, bc_y, hx=1.0, hy=1.0):
    """b on the full grid (zeros at known nodes) through Algorithm 1's padded two-pass stencil."""
    known = known_mask(phi, direction)
    fk = np.where(known, f, 0.0).astype(np.float64)
    B = -apply_squared_laplacian_padded(fk, bc_x, bc_y, hx, hy)
    return np.where(known, 0.0, B)


def assemble(x_unknown, f, unk, known):
    """out = f at the known nodes (bit copy), x at the unknown nodes (Algorithm 1, last step)."""
    out = np.array(f, dtype=np.float64, copy=True)
    flat = out.ravel()
    flat[unk] = x_unknown
    return flat.reshape(f.shape)


# ----------------------------------------------------------------------------------------------
# Solvers
# ----------------------------------------------------------------------------------------------
def solve_direct(A, b):
    """Sparse direct solve (the role of MATLAB's chol in Sec. 2.2), SuperLU."""
    if A.shape[0] == 0:
        return np.zeros(0)
    return spla.spsolve(A.tocsc(), b)


def cg(A, b, rtol=1e-10, maxit=None, precond=None):
    """Conjugate gradients from x0 = 0 with an optional preconditioner z = M(r).

    Textbook PCG (Hestenes-Stiefel with beta = rho_new / rho_old).  Stops when the recursively
    updated residual satisfies ||r|| <= rtol ||b||; returns (x, iterations, true relative residual).
    b = 0 gives x = 0 after 0 iterations.
    """
    n = b.shape[0]
    maxit = 10 * n if maxit is None else maxit
    x = np.zeros(n)
    bnorm = np.linalg.norm(b)
    if n == 0 or bnorm == 0.0:
        return x, 0, 0.0
    r = b.copy()
    z = precond(r) if precond is not None else r.copy()
    p = z.copy()
    rho = r @ z
    it = 0
    while it < maxit:
        q = A @ p
        alpha = rho / (p @ q)
        x += alpha * p
        r -= alpha * q
        it += 1
        if np.linalg.norm(r) <= rtol * bnorm:
            break
        z = precond(r) if precond is not None else r.copy()
        rho_new = r @ z
        p = z + (rho_new / rho) * p
        rho = rho_new
    relres = np.linalg.norm(b - A @ x) / bnorm
    return x, it, relres


# ----------------------------------------------------------------------------------------------
# Fast Poisson preconditioner (Algorithm 1, Sec. 2.2), separable transforms via scipy.fft
# ----------------------------------------------------------------------------------------------
def axis_eigenvalues(n: int, bc: str, h: float = 1.0) -> np.ndarray:
    """Eigenvalues of T/h^2 in the order the transform of ``_forward`` returns its coefficients."""
    k = np.arange(n)
    if bc == "dirichlet":      # sine transform, Algorithm 1
        lam = 2.0 - 2.0 * np.cos(np.pi * (k + 1) / (n + 1))
    elif bc == "symmetric":    # cosine transform (Example 1, Neumann)
        lam = 2.0 - 2.0 * np.cos(np.pi * k / n)
    elif bc == "periodic":     # discrete Fourier transform (Example 2)
        lam = 2.0 - 2.0 * np.cos(2.0 * np.pi * k / n)
    else:
        raise ValueError(bc)
    return lam / (h * h)


def _forward(a, axis, bc):
    if bc == "dirichlet":
        return sfft.dst(a, type=1, axis=axis, norm="ortho")
    if bc == "symmetric":
        return sfft.dct(a, type=2, axis=axis, norm="ortho")
    return sfft.fft(a, axis=axis)


def _inverse(a, axis, bc):
    if bc == "dirichlet":
        return sfft.idst(a, type=1, axis=axis, norm="ortho")
    if bc == "symmetric":
        return sfft.idct(a, type=2, axis=axis, norm="ortho")
    return sfft.ifft(a, axis=axis)


def poisson_squared_pinv(B: np.ndarray, bc_x: str, bc_y: str, hx=1.0, hy=1.0) -> np.ndarray:
    """Z = (L^2)^+ B on the full rectangle: transform both axes, divide by the squared
    eigenvalue sums, transform back.  The zero eigenvalue (both axes symmetric/periodic) is
    dropped, i.e. the pseudo-inverse.
    """
    ny, nx = B.shape
    Z = _forward(_forward(B.astype(np.float64), 1, bc_x), 0, bc_y)
    LL = axis_eigenvalues(ny, bc_y, hy)[:, None] + axis_eigenvalues(nx, bc_x, hx)[None, :]
    with np.errstate(divide="ignore"):
        W = np.where(LL > 0, 1.0 / (LL * LL), 0.0)
    # the exact zero eigenvalue sits at index (0, 0); guard against round-off in LL there
    if bc_x != "dirichlet" and bc_y != "dirichlet":
        W[0, 0] = 0.0
    Z = _inverse(_inverse(Z * W, 0, bc_y), 1, bc_x)
    return np.real(Z)


def fast_poisson_preconditioner(unk, ny, nx, bc_x, bc_y, hx=1.0, hy=1.0):
    """z = R (L^2)^+ R^T r: map to D by zero-augmentation, invert on the rectangle, map back."""
    def apply(r):
        B = np.zeros(ny * nx)
        B[unk] = r
        return poisson_squared_pinv(B.reshape(ny, nx), bc_x, bc_y, hx, hy).ravel()[unk]
    return apply


# ----------------------------------------------------------------------------------------------
# End-to-end extension
# ----------------------------------------------------------------------------------------------
def extend(phi, f, direction="out", bc_x="symmetric", bc_y="symmetric", hx=1.0, hy=1.0,
           method="direct", rtol=1e-10, maxit=None):
    """Biharmonic extension of f from Omega (chosen by sign(phi)) to the whole grid.

    method: 'direct' (SuperLU), 'cg' (unpreconditioned) or 'pcg' (fast Poisson preconditioner).
    Returns (out, info) with info = {iters, relres, n_unknown, n_known}.
    Raises ValueError when no node is known and no axis is Dirichlet (solution unique only up to a
    constant).
    """
    phi = np.asarray(phi, dtype=np.float64)
    f = np.asarray(f)
    known = known_mask(phi, direction)
    if not known.any() and bc_x != "dirichlet" and bc_y != "dirichlet":
        raise ValueError("no known node: the extension is not unique for symmetric/periodic edges")
    A, b, unk, known = system(phi, f, direction, bc_x, bc_y, hx, hy)
    ny, nx = phi.shape
    info = {"n_unknown": int(unk.size), "n_known": int(known.sum())}
    if method == "direct":
        x = solve_direct(A, b)
        it = 0
    elif method == "cg":
        x, it, _ = cg(A, b, rtol=rtol, maxit=maxit)
    elif method == "pcg":
        M = fast_poisson_preconditioner(unk, ny, nx, bc_x, bc_y, hx, hy)
        x, it, _ = cg(A, b, rtol=rtol, maxit=maxit, precond=M)
    else:
        raise ValueError(method)
    bn = np.linalg.norm(b)
    info["iters"] = it
    info["relres"] = float(np.linalg.norm(b - A @ x) / bn) if bn > 0 else 0.0
    return assemble(x, f, unk, known), info


def true_relative_residual(out, phi, f, direction, bc_x, bc_y, hx=1.0, hy=1.0):
    """||b - A x|| / ||b|| for a full-grid answer ``out`` (x = out at the unknown nodes), FP64."""
    A, b, unk, _ = system(np.asarray(phi, np.float64), np.asarray(f), direction,
                          bc_x, bc_y, hx, hy)
    x = np.asarray(out, dtype=np.float64).ravel()[unk]
    bn = np.linalg.norm(b)
    return float(np.linalg.norm(b - A @ x) / bn) if bn > 0 else float(np.linalg.norm(A @ x))


def max_rel_error(out, ref, known):
    """max over unknown nodes of |out - ref| divided by the max |ref| over all nodes."""
    den = float(np.max(np.abs(ref)))
    d = np.abs(np.asarray(out, np.float64) - np.asarray(ref, np.float64))[~known]
    num = float(d.max()) if d.size else 0.0
    return num / den if den > 0 else num
