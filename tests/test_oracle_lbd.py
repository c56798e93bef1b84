"""Pins of the oracle's Lanczos bidiagonalisation for DDLR-2
(lowrank_method=2, Sec. 4.4: the alternative that computes U_k and V_k at the
same time).

Golub-Kahan bidiagonalisation of K = A0^-1 E from a start vector v_1 gives
K V_m = U_m B_m, and B_m^T B_m is the tridiagonal matrix that Lanczos on
K^T K = E^T A0^-2 E gives from the same v_1: in exact arithmetic the two
produce the same Ritz values and the same preconditioner.  That identity, and
exactness at full rank, are what these tests check; the Lanczos side is the
oracle's own, independent implementation.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from dense_ddlr import oracle_matrix


@pytest.fixture(scope="module")
def small():
    A = W.laplacian((12, 12))
    part, p = W.box_partition((12, 12), (2, 2))
    return A, part, p


@pytest.mark.parametrize("m", [10, 20])
def test_bidiagonalisation_equals_lanczos_on_normal_operator(small, m):
    A, part, p = small
    kw = dict(variant=2, k=6, factor=1, lanczos_max=m, lanczos_eps=1e-300)
    ol = O.Oracle(A, part, p, **kw)
    ob = O.Oracle(A, part, p, lowrank_method=2, **kw)
    assert ol.msteps == ob.msteps == m
    np.testing.assert_allclose(ob.ritz[:6], ol.ritz[:6], rtol=1e-12)
    for seed in (1, 2):
        x = W.rhs(A[0], seed)
        yl = ol.apply(x)
        assert np.abs(ob.apply(x) - yl).max() <= 1e-8 * np.abs(yl).max()


def test_full_rank_is_exact(small):
    A, part, p = small
    ob = O.Oracle(A, part, p, variant=2, k=44, factor=1, lowrank_method=2)
    Ainv = np.linalg.inv(W.to_dense(A))
    assert np.abs(oracle_matrix(ob, A[0]) - Ainv).max() <= 1e-12 * np.abs(Ainv).max()
    _, its, rel, st = ob.pcg(W.rhs(A[0], 0), 1e-8)
    assert st == "OK" and its == 1


def test_same_pcg_as_lanczos_with_ic0():
    A = W.laplacian((16, 16, 16))
    part, p = W.box_partition((16, 16, 16), (2, 2, 2))
    b = W.rhs(A[0], 0)
    res = {}
    for lm in (0, 2):
        o = O.Oracle(A, part, p, variant=2, k=8, factor=0, lowrank_method=lm)
        _, its, rel, st = o.pcg(b, 1e-8)
        assert st == "OK" and rel <= 1e-8
        res[lm] = (o.msteps, its)
    assert res[0][0] == res[2][0] and abs(res[0][1] - res[2][1]) <= 1


def test_bidiagonalisation_is_ddlr2_only(small):
    A, part, p = small
    with pytest.raises(O.OracleError, match="INVALID"):
        O.Oracle(A, part, p, variant=1, k=4, lowrank_method=2)
    with pytest.raises(O.OracleError, match="INVALID"):
        O.Oracle(A, part, p, variant=2, k=4, lowrank_method=3)
