"""Host logic of the library, without a GPU: the transform bases of the fast Poisson
preconditioner (Algorithm 1, sine transform; Example 1, cosine transform; Example 2, Fourier
transform) that the library builds on the host, pinned against the oracle's independent sparse
construction of each axis's negative second difference T."""

import numpy as np
import pytest

from oracle import biharmonic as ob


@pytest.fixture(scope="module")
def ext():
    from paper_1704_08897_gb300 import build_ext, ext as e
    try:
        build_ext.build()
    except RuntimeError as err:  # no nvcc on this host
        pytest.skip(str(err))
    e.load()
    return e


@pytest.mark.parametrize("bc", ob.BCS)
@pytest.mark.parametrize("n", [4, 5, 7, 16, 33, 64, 100, 129])
def test_axis_basis_diagonalises_the_oracle_second_difference(ext, bc, n):
    Q, lam = ext.ext_axis_basis(n, bc)
    T = ob.axis_second_difference(n, bc).toarray()
    np.testing.assert_allclose(Q.T @ Q, np.eye(n), rtol=0, atol=1e-13)   # orthonormal
    np.testing.assert_allclose(Q.T @ T @ Q, np.diag(lam), rtol=0, atol=1e-12)  # T = Q diag Q^T
    # the same spectrum as the closed form the oracle's scipy.fft preconditioner divides by
    np.testing.assert_allclose(np.sort(lam), np.sort(ob.axis_eigenvalues(n, bc)), rtol=0,
                               atol=1e-13)


@pytest.mark.parametrize("bc", ["symmetric", "periodic"])
def test_zero_mode_is_the_constant_in_column_zero(ext, bc):
    # the pseudo-inverse drops exactly the (0, 0) mode: its eigenvalue must be an exact zero and
    # its eigenvector the normalised constant, on both axes kinds that have one
    n = 48
    Q, lam = ext.ext_axis_basis(n, bc)
    assert lam[0] == 0.0
    np.testing.assert_allclose(Q[:, 0], np.full(n, n ** -0.5), rtol=0, atol=1e-15)
    assert np.all(lam[1:] > 1e-3)


def test_dirichlet_spectrum_is_positive(ext):
    _, lam = ext.ext_axis_basis(40, "dirichlet")
    assert np.all(lam > 0.0)


def test_axis_basis_rejects_bad_arguments(ext):
    for n, bc in ((3, 0), (32769, 0), (8, 3), (8, -1)):
        Q = np.empty((4, 4))
        lam = np.empty(4)
        rc = ext.load().ext_axis_basis(n, bc, Q.ctypes.data, lam.ctypes.data)
        assert rc == ext.EXT_EINVAL, (n, bc)
    assert ext.load().ext_axis_basis(8, 0, None, None) == ext.EXT_EINVAL


def _decode(codes, type_):
    if type_ == "fp16":
        return codes.view(np.float16).astype(np.float64)
    return (codes.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


@pytest.mark.parametrize("type_", ["fp16", "bf16"])
@pytest.mark.parametrize("bc", ob.BCS)
@pytest.mark.parametrize("n", [4, 100, 128, 200])
def test_axis_slices_are_exact_block_scaled_integers(ext, type_, bc, n):
    """The tensor-core operand form of Q and Q^T: four integer slices per 128-wide block of a
    row, |c0| <= 255 and |c1..c3| <= 128 (exact in FP16 and BF16), reproduce every entry to
    2^(E-33) of its block's scale, and the padding is zero."""
    codes, exps = ext.ext_axis_slices(n, bc, type_)
    Q, _ = ext.ext_axis_basis(n, bc)
    npad = codes.shape[-1]
    assert npad % 128 == 0 and npad - 128 < n <= npad
    c = _decode(codes, type_)                       # [2, 4, np, np]
    assert np.array_equal(c, np.round(c))           # integers
    assert np.abs(c[:, 0]).max() <= 255 and np.abs(c[:, 1:]).max() <= 128
    E = np.repeat(exps.astype(np.float64), 128, axis=2)  # [2, np, np] exponent of each entry
    recon = sum(c[:, k] * np.exp2(E - 8 * (k + 1)) for k in range(4))
    for t, M in enumerate((Q, Q.T)):
        ref = np.zeros((npad, npad))
        ref[:n, :n] = M
        err = np.abs(recon[t] - ref)
        assert np.all(err <= np.exp2(E[t] - 33)), (t, err.max())
        # each block's largest entry sits in [2^(E-1), 2^E): the scale is the block's own
        blk = np.abs(ref).reshape(npad, npad // 128, 128).max(axis=2)
        e = exps[t].astype(np.float64)
        nz = blk > 0
        assert np.all(blk[nz] < np.exp2(e[nz])) and np.all(blk[nz] >= np.exp2(e[nz] - 2))
    assert np.all(recon[:, n:, :] == 0) and np.all(recon[:, :, n:] == 0)


def test_axis_slices_rejects_bad_arguments(ext):
    codes = np.empty(8, np.uint16)
    exps = np.empty(8, np.int8)
    lib = ext.load()
    for n, bc, t in ((3, 0, 1), (32769, 0, 1), (8, 3, 1), (8, 0, 2)):
        assert lib.ext_axis_slices(n, bc, t, codes.ctypes.data, exps.ctypes.data) == ext.EXT_EINVAL
    assert lib.ext_axis_slices(8, 0, 1, None, None) == ext.EXT_EINVAL


def _fold(r, cls):
    """Mirror fold of an axis vector (i -> n-1-i) for class cls: sum (even) or difference (odd) of
    each node and its mirror on the first ceil(n/2) nodes; the middle node of an odd n alone."""
    n = r.shape[0]
    h = (n + 1) // 2
    m = r[::-1][:h]
    v = r[:h] + m if cls == 0 else r[:h] - m
    if n % 2:
        v[h - 1] = r[h - 1] if cls == 0 else 0.0
    return v


def _unfold(E, O, n):
    """Inverse of the fold: E + O on the first ceil(n/2) nodes, E - O on their mirrors."""
    h, k = (n + 1) // 2, n // 2  # k nodes have a distinct mirror
    y = np.empty(n)
    y[:h] = E + O
    y[n - 1 - np.arange(k)] = (E - O)[:k]
    return y


@pytest.mark.parametrize("bc", ob.BCS)
@pytest.mark.parametrize("n", [4, 5, 7, 16, 33, 64, 100, 129])
def test_mirror_classes_apply_the_same_function_of_T(ext, bc, n):
    # g(T) r with g = 1/(1 + lambda), through the two half-size class bases (fold, transform,
    # scale, inverse transform, unfold), against a dense solve with the oracle's T
    T = ob.axis_second_difference(n, bc).toarray()
    rng = np.random.default_rng(n)
    r = rng.standard_normal(n)
    ref = np.linalg.solve(np.eye(n) + T, r)
    parts = []
    for cls in (0, 1):
        F, lam = ext.ext_axis_class_basis(n, bc, cls)
        c = F.T @ _fold(r, cls)
        parts.append(F @ (c / (1.0 + lam)))
    y = _unfold(parts[0], parts[1], n)
    np.testing.assert_allclose(y, ref, rtol=0, atol=1e-12 * np.abs(ref).max())


@pytest.mark.parametrize("bc", ob.BCS)
@pytest.mark.parametrize("n", [5, 16, 33, 128])
def test_mirror_classes_split_the_spectrum(ext, bc, n):
    h = (n + 1) // 2
    w = np.full(h, 2.0)
    if n % 2:
        w[h - 1] = 1.0  # the middle node is its own mirror
    lams, count = [], 0
    for cls in (0, 1):
        F, lam = ext.ext_axis_class_basis(n, bc, cls)
        live = np.abs(F).sum(axis=0) > 0
        k = int(live.sum())
        assert live[:k].all() and not live[k:].any()        # the class's modes come first
        assert np.all(np.diff(lam[:k]) >= -1e-15)             # in ascending order
        # orthonormal as full-length vectors (each node and its mirror)
        np.testing.assert_allclose(F[:, :k].T @ (w[:, None] * F[:, :k]), np.eye(k), rtol=0, atol=1e-13)
        lams.append(lam[:k])
        count += k
    assert count == n
    np.testing.assert_allclose(np.sort(np.concatenate(lams)), np.sort(ob.axis_eigenvalues(n, bc)),
                               rtol=0, atol=1e-13)
