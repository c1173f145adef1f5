"""Pins of the oracle's Theorem-1 quantities: the explicit matrix of A is the
forward projector column by column (and its transpose the adjoint), the
sketch deviation ||U^T (S^T S - I) U|| has the closed form N_S - 1 when U
spans single rows, vanishes without sketching, and averages to zero over
the interleaved offsets (S^T S is unbiased)."""
import numpy as np

import oracle as O
from paper_2411_05771_gb300 import inputs as I


def test_explicit_matrix_is_the_projector_and_its_transpose_the_adjoint():
    N, n_ang = 6, 8
    ang = I.uniform_angles(n_ang)
    nd = O.ndet(N)
    A = O.explicit_matrix(N, ang, nd)
    rng = np.random.default_rng(0)
    x = rng.standard_normal((N, N))
    p = rng.standard_normal((n_ang, nd))
    np.testing.assert_allclose(A @ x.ravel(), O.proj_fwd(x[None], ang, nd).ravel(), atol=1e-12)
    np.testing.assert_allclose(A.T @ p.ravel(), O.proj_adj(p[None], ang, N).ravel(), atol=1e-12)


def test_deviation_closed_form_for_coordinate_columns():
    """A whose columns are distinct coordinate vectors: U is those columns,
    U^T (ns P - I) U = diag(ns or 0) - I has eigenvalues ns - 1 and -1."""
    n_ang, nd, ns = 6, 3, 3
    A = np.zeros((n_ang * nd, 4))
    for j, row in enumerate((0, 4, 7, 16)):
        A[row, j] = 1.0 + j
    d, s = O.sketch_gram_deviation(A, n_ang, nd, ns)
    assert s.size == 4
    np.testing.assert_allclose(d, ns - 1.0, rtol=1e-12)
    d1, _ = O.sketch_gram_deviation(A, n_ang, nd, 1)
    np.testing.assert_allclose(d1, 0.0, atol=1e-12)


def test_deviation_averages_to_zero_over_offsets():
    N, n_ang, ns = 8, 12, 4
    ang = I.uniform_angles(n_ang)
    nd = O.ndet(N)
    A = O.explicit_matrix(N, ang, nd)
    U, s, _ = np.linalg.svd(A, full_matrices=False)
    k = int(np.sum(s > 1e-10 * s[0]))
    U = U[:, :k]
    acc = np.zeros((k, k))
    for o in range(ns):
        mask = np.zeros(n_ang)
        mask[o::ns] = 1.0
        rows = np.repeat(mask, nd) > 0
        acc += ns * U[rows].T @ U[rows] - np.eye(k)
    assert np.abs(acc).max() <= 1e-10
    d, _ = O.sketch_gram_deviation(A, n_ang, nd, ns)
    assert np.all(d > 0) and np.all(d <= ns - 1 + 1e-12)
