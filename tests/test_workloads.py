"""The seeded generators of the paper-shaped solver inputs (Sec. 4.2 ACG
boxes, Sec. 4.3 random graph Laplacians): structure checked against
brute-force constructions and the properties the solvers rely on."""
import itertools

import numpy as np
import pytest
import scipy.sparse as sp

import workloads


def _dense(rp, col, val):
    n = rp.shape[0] - 1
    return sp.csr_matrix((val, col, rp), shape=(n, n)).toarray()


@pytest.mark.parametrize("shape", [(4, 3, 2), (5, 1, 1), (3, 4, 1), (2, 2, 3)])
def test_stencil27_matches_brute_force(shape):
    nx, ny, nz = shape
    rp, col, val = workloads.stencil27(nx, ny, nz)
    n = nx * ny * nz
    ref = np.zeros((n, n))
    for z, y, x in itertools.product(range(nz), range(ny), range(nx)):
        i = x + nx * (y + ny * z)
        for dz, dy, dx in itertools.product((-1, 0, 1), repeat=3):
            X, Y, Z = x + dx, y + dy, z + dz
            if 0 <= X < nx and 0 <= Y < ny and 0 <= Z < nz:
                ref[i, X + nx * (Y + ny * Z)] = 27.0 if (dx, dy, dz) == (0, 0, 0) else -1.0
    np.testing.assert_array_equal(_dense(rp, col, val), ref)
    for r in range(n):  # columns ascending within every row
        assert np.all(np.diff(col[rp[r]:rp[r + 1]]) > 0)


def test_stencil27_spd_and_ones_solution():
    rp, col, val = workloads.stencil27(7, 6, 5)
    A = _dense(rp, col, val)
    assert np.array_equal(A, A.T)
    assert np.linalg.eigvalsh(A).min() > 0
    b = workloads.ones_rhs(rp, col, val)
    np.testing.assert_array_equal(b, A @ np.ones(A.shape[0]))
    # interior rows: 27 - 26 neighbours = 1; a corner of a 3-D box: 27 - 7 = 20
    assert b.min() == 1.0 and b[0] == 20.0


def test_stencil27_chimney_sizes():
    rp, col, val = workloads.stencil27(100, 100, 1)
    assert rp.shape[0] - 1 == 10**4 and rp[-1] == 9 * 98 * 98 + 6 * 4 * 98 + 4 * 4  # 9-point in one plane
    rp, col, val = workloads.stencil27(100, 100, 10)
    assert rp.shape[0] - 1 == 10**5 and col.dtype == np.int32 and rp.dtype == np.int64


@pytest.mark.parametrize("n,degree", [(50, 3), (300, 8), (2000, 8)])
def test_graph_laplacian_properties(n, degree):
    rp, col, val = workloads.graph_laplacian(n, degree, seed=5)
    L = sp.csr_matrix((val, col, rp), shape=(n, n))
    assert abs(L - L.T).max() == 0
    np.testing.assert_array_equal(np.asarray(L.sum(axis=1)).ravel(), np.zeros(n))
    off = L - sp.diags(L.diagonal())
    assert set(np.unique(off.data).tolist()) <= {-1.0, 0.0}
    assert L.diagonal().min() >= 0
    if n <= 300:
        assert np.linalg.eigvalsh(L.toarray()).min() > -1e-9
    # each vertex drew `degree` partners: every degree is at least that minus self loops
    assert L.diagonal().sum() >= n * degree * 0.9
    rp2, col2, val2 = workloads.graph_laplacian(n, degree, seed=5)
    assert np.array_equal(rp, rp2) and np.array_equal(col, col2)
