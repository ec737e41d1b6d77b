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
