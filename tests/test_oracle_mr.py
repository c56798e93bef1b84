"""Pins of the oracle's MR approximate inverse of C_a (c_solver=2, Sec. 4.3,
Algorithm 2: self-preconditioned global MR iterations with dual-threshold
dropping, from X_0 = diag(C_a)^-1; the solve applies the symmetric part
(X + X^T)/2).

Expected values are derived by hand or formed densely from the definitions:
C_a over the interface nodes from A and the partition, its inverse by LAPACK.
The oracle's X is read back column by column through A0 solves with unit
vectors on the interface nodes.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W


def _interface(A, part):
    Ad = W.to_dense(A)
    pv = np.asarray(part)
    idx = np.where(((Ad != 0) & (pv[:, None] != pv[None, :])).any(axis=1))[0]
    C = Ad[np.ix_(idx, idx)] + np.eye(len(idx))
    return idx, C


def _xdense(orc, n, idx):
    X = np.zeros((len(idx), len(idx)))
    for j, g in enumerate(idx):
        x = np.zeros(n)
        x[g] = 1.0
        X[:, j] = orc.a0_solve(x)[idx]
    return X


def test_one_step_closed_form():
    """1-D Laplacian tridiag(-1, 2, -1), n = 4, parts {0,1 | 2,3}, a = 1:
    C_a = [[3, -1], [-1, 3]], X_0 = I/3, R_0 = I - C_a X_0 = [[0, 1/3],
    [1/3, 0]], Z_0 = X_0 R_0 = [[0, 1/9], [1/9, 0]], C_a Z_0 = [[-1/9, 1/3],
    [1/3, -1/9]], tr(R_0^T C_a Z_0) = 2/9, ||C_a Z_0||_F^2 = 20/81, so
    beta = 9/10 and X_1 = [[1/3, 1/10], [1/10, 1/3]] (no dropping)."""
    A = W.laplacian((4,))
    part = np.array([0, 0, 1, 1], dtype=np.int32)
    orc = O.Oracle(A, part, 2, k=1, factor=1, c_solver=2, mr_iters=1, mr_lfil=2, mr_droptol=0.0)
    X = _xdense(orc, 4, np.array([1, 2]))
    np.testing.assert_allclose(X, [[1 / 3, 1 / 10], [1 / 10, 1 / 3]], rtol=0, atol=1e-15)
    # zero iterations: X_0 = diag(C_a)^-1
    orc0 = O.Oracle(A, part, 2, k=1, factor=1, c_solver=2, mr_iters=0)
    np.testing.assert_allclose(_xdense(orc0, 4, np.array([1, 2])), np.eye(2) / 3, rtol=0, atol=1e-15)


def test_without_dropping_converges_to_the_inverse():
    """No dropping: the self-preconditioned MR residual I - C_a X squares from
    one iteration to the next near convergence; after 6 iterations X = C_a^-1."""
    A = W.laplacian((12, 12))
    part, p = W.box_partition((12, 12), (2, 2))
    idx, C = _interface(A, part)
    Ci = np.linalg.inv(C)
    res = []
    for it in range(7):
        orc = O.Oracle(A, part, p, k=2, factor=1, c_solver=2, mr_iters=it, mr_lfil=len(idx), mr_droptol=0.0)
        X = _xdense(orc, A[0], idx)
        res.append(np.linalg.norm(np.eye(len(idx)) - C @ X))
    assert all(res[i + 1] < res[i] for i in range(5))
    assert res[4] < res[3] ** 1.5              # superlinear near the end
    np.testing.assert_allclose(X, Ci, rtol=0, atol=1e-13)


def test_dropping_bounds_the_fill_and_keeps_the_residual_falling():
    A = W.laplacian((12, 12))
    part, p = W.box_partition((12, 12), (2, 2))
    idx, C = _interface(A, part)
    prev = np.inf
    for it in range(6):
        orc = O.Oracle(A, part, p, k=2, factor=1, c_solver=2, mr_iters=it, mr_lfil=4, mr_droptol=1e-3)
        X = _xdense(orc, A[0], idx)
        np.testing.assert_array_equal(X, X.T)                            # symmetric part applied
        assert (X != 0).sum(axis=0).max() <= 2 * (1 + 4 * it)            # columns of X and X^T
        r = np.linalg.norm(np.eye(len(idx)) - C @ X)
        assert r < prev
        prev = r


def test_mr_preconditioner_solves():
    """IC(0) interior blocks, defaults (3 iterations, 8 entries per column,
    drop tolerance 1e-3): PCG converges in both variants, within a few
    iterations of the factored C_a."""
    A = W.laplacian((16, 16, 16))
    part, p = W.box_partition((16, 16, 16), (2, 2, 2))
    b = W.rhs(A[0], 0)
    for variant in (1, 2):
        its = {}
        for cs in (0, 2):
            orc = O.Oracle(A, part, p, variant=variant, k=8, factor=0, c_solver=cs, mr_lfil=8)
            _, its[cs], rel, st = orc.pcg(b, 1e-8)
            assert st == "OK" and rel <= 1e-8
        assert its[2] <= its[0] + max(4, its[0] // 5)


def test_mr_rejects_bad_options():
    A = W.laplacian((8, 8))
    part, p = W.box_partition((8, 8), (2, 2))
    for kw in (dict(c_solver=3), dict(c_solver=2, mr_iters=-1), dict(c_solver=2, mr_lfil=0),
               dict(c_solver=2, mr_droptol=-1.0)):
        with pytest.raises(O.OracleError, match="INVALID"):
            O.Oracle(A, part, p, k=2, **kw)
