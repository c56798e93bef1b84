"""Pins of the oracle's LDL^T local factors: factor=2 (incomplete LDL^T on
the pattern) and factor=3 (exact dense LDL^T without pivoting), the local
solver Sec. 5 names for the indefinite problems ("incomplete Cholesky or
LDL").

Facts fixed independently of the oracle (dense LAPACK, the definitions):
* (L D L^T)_ij = (A0)_ij on the lower pattern of every block, L unit lower
  (everywhere for the exact factor);
* where every pivot is positive, L D L^T and the Cholesky factor describe the
  same matrix (L_chol = L D^1/2), so ILDL(0) and IC(0), and exact LDL^T and
  exact Cholesky, give the same A0 solve;
* Sylvester's law of inertia: the exact LDL^T of A0 has as many negative
  pivots as A0 has negative eigenvalues;
* with an indefinite A0 the exact LDL^T solve is the dense solve, and SMW
  still gives M^-1 = A^-1 at full rank, so GMRES takes one step, while
  exact Cholesky refuses that A0;
* tridiagonal blocks have no fill: ILDL(0) equals the exact LDL^T there.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from dense_ddlr import DenseDDLR, oracle_matrix


def _factor(orc, n):
    r, c, v = orc.factor_coo()
    L = np.zeros((n, n))
    L[r, c] = v
    d = np.diag(L).copy()
    np.fill_diagonal(L, 1.0)
    return L, d


@pytest.fixture(scope="module")
def indef_a0():
    """12x12 Laplacian minus 1.3 I, 2x2 boxes: A0 itself is indefinite."""
    A = W.shifted_laplacian((12, 12), 1.3)
    part, p = W.box_partition((12, 12), (2, 2))
    D = DenseDDLR(A, part, p)
    A0 = D.to_original(D.A0)
    assert int((np.linalg.eigvalsh(A0) < 0).sum()) == 4
    return A, part, p, D, A0


@pytest.fixture(scope="module")
def nine_point():
    A = W.nine_point(12, 2.0)
    part, p = W.box_partition((12, 12), (2, 2))
    D = DenseDDLR(A, part, p)
    A0 = D.to_original(D.A0)
    assert int((np.linalg.eigvalsh(A0) < 0).sum()) > 0
    return A, part, p, D, A0


@pytest.mark.parametrize("problem", ["indef_a0", "nine_point"])
@pytest.mark.parametrize("factor,c_order", [(2, 0), (2, 1), (3, 0)])
def test_ldl_defining_property(request, problem, factor, c_order):
    A, part, p, D, A0 = request.getfixturevalue(problem)
    orc = O.Oracle(A, part, p, k=2, factor=factor, c_order=c_order, b_order=c_order, indefinite=1)
    L, d = _factor(orc, D.n)
    LDLt = L @ np.diag(d) @ L.T
    if factor == 3:
        np.testing.assert_allclose(LDLt, A0, atol=1e-11)
    else:
        mask = A0 != 0
        np.testing.assert_allclose(LDLt[mask], A0[mask], atol=1e-11)
        assert np.sum(L != 0) == (np.sum(mask) + D.n) // 2


def test_inertia_and_exact_solve(indef_a0):
    A, part, p, D, A0 = indef_a0
    orc = O.Oracle(A, part, p, k=2, factor=3, indefinite=1)
    _, d = _factor(orc, D.n)
    assert int((d < 0).sum()) == int((np.linalg.eigvalsh(A0) < 0).sum())
    x = W.rhs(D.n, 3)
    y = orc.a0_solve(x)
    ref = np.linalg.solve(A0, x)
    assert np.abs(y - ref).max() <= 1e-10 * np.abs(ref).max()
    with pytest.raises(O.OracleError, match="BREAKDOWN"):
        O.Oracle(A, part, p, k=2, factor=1, indefinite=1)


@pytest.mark.parametrize("variant", [1, 2])
def test_full_rank_is_exact_with_indefinite_a0(indef_a0, variant):
    A, part, p, D, _ = indef_a0
    orc = O.Oracle(A, part, p, variant=variant, k=D.s, factor=3, indefinite=1)
    Ainv = np.linalg.inv(W.to_dense(A))
    assert np.abs(oracle_matrix(orc, D.n) - Ainv).max() <= 1e-9 * np.abs(Ainv).max()
    _, its, rel, st = orc.gmres(W.rhs(D.n, 0), 1e-10)
    assert st == "OK" and its == 1 and rel <= 1e-10


def test_ldl_equals_cholesky_when_pivots_are_positive():
    A = W.laplacian((12, 12))
    part, p = W.box_partition((12, 12), (2, 2))
    x = W.rhs(144, 4)
    for c_order in (0, 1):
        kw = dict(k=4, c_order=c_order, b_order=c_order)
        for chol, ldl in ((0, 2), (1, 3)):
            y0 = O.Oracle(A, part, p, factor=chol, **kw).a0_solve(x)
            y1 = O.Oracle(A, part, p, factor=ldl, **kw).a0_solve(x)
            assert np.abs(y1 - y0).max() <= 1e-12 * np.abs(y0).max()
        L, d = _factor(O.Oracle(A, part, p, factor=2, **kw), 144)
        Lc, dc = _factor(O.Oracle(A, part, p, factor=0, **kw), 144)
        assert np.all(d > 0)
        np.testing.assert_allclose(np.sqrt(d), dc, rtol=1e-13)
        np.testing.assert_allclose(L * np.sqrt(d)[None, :], Lc - np.eye(144) + np.diag(dc), atol=1e-13)


def test_ildl0_is_exact_on_tridiagonal_blocks():
    A = W.shifted_laplacian((40,), 0.7)
    part, p = W.box_partition((40,), (4,))
    D = DenseDDLR(A, part, p)
    assert (np.linalg.eigvalsh(D.A0) < 0).sum() > 0
    x = W.rhs(40, 1)
    y2 = O.Oracle(A, part, p, k=2, factor=2, indefinite=1).a0_solve(x)
    y3 = O.Oracle(A, part, p, k=2, factor=3, indefinite=1).a0_solve(x)
    assert np.abs(y2 - y3).max() <= 1e-12 * np.abs(y3).max()


def test_bad_factor_option(indef_a0):
    A, part, p, _, _ = indef_a0
    with pytest.raises(O.OracleError, match="INVALID"):
        O.Oracle(A, part, p, k=2, factor=4)
