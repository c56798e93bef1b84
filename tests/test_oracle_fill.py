"""Pins of the oracle's level-of-fill incomplete factors (fill_level k > 0
with factor 0 or 2): the pattern keeps the entries whose level of fill is at
most k, where A0's entries have level 0 and eliminating pivot t gives entry
(i, j) of two later neighbours i, j of t the level lev(i,t) + lev(j,t) + 1.

Fixed independently here: the pattern, recomputed in the test by eliminating
the pivots one after the other (the oracle builds it row by row); the
incomplete factor's defining property L L^T = A0 (or L D L^T = A0) on that
pattern; k = 0 is IC(0) and a level above the block size is the exact
Cholesky factor; patterns grow with k.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from dense_ddlr import DenseDDLR


def _factor(orc, n):
    r, c, v = orc.factor_coo()
    L = np.zeros((n, n))
    L[r, c] = v
    return L


def _blocks(A, part, p):
    n, rp, ci, _ = A
    part = np.asarray(part)
    iface = np.array([np.any(part[ci[rp[i]:rp[i + 1]]] != part[i]) for i in range(n)])
    return [np.flatnonzero((part == b) & ~iface) for b in range(p)] + [np.flatnonzero(iface)]


def _level_pattern(A0, nodes, k):
    """Lower pattern {(i, j)}, i > j in natural order, of the level-k factor of
    A0 restricted to nodes, by right-looking elimination of the pivots."""
    nodes = sorted(int(x) for x in nodes)
    lev = {}
    for a in nodes:
        for b in nodes:
            if b < a and A0[a, b] != 0:
                lev[(a, b)] = 0
    for t in nodes:
        below = sorted((i, lv) for (i, c), lv in lev.items() if c == t)
        for x in range(len(below)):
            for y in range(x):
                (i, li), (j, lj) = below[x], below[y]
                cand = li + lj + 1
                if cand <= k and cand < lev.get((i, j), k + 1):
                    lev[(i, j)] = cand
    return {key for key, lv in lev.items() if lv <= k}


@pytest.fixture(scope="module")
def lap2d():
    A = W.laplacian((14, 12))
    part, p = W.box_partition((14, 12), (2, 2))
    D = DenseDDLR(A, part, p)
    return A, part, p, D.to_original(D.A0)


@pytest.fixture(scope="module")
def nine_point():
    A = W.nine_point(12, 0.0)
    part, p = W.box_partition((12, 12), (2, 2))
    D = DenseDDLR(A, part, p)
    return A, part, p, D.to_original(D.A0)


@pytest.fixture(scope="module")
def lap3d_cuts():
    A = W.laplacian((9, 9, 9))
    part, p = W.random_cut_partition(9, 2, 1, 3, 6)
    D = DenseDDLR(A, part, p)
    return A, part, p, D.to_original(D.A0)


@pytest.mark.parametrize("problem", ["lap2d", "nine_point", "lap3d_cuts"])
@pytest.mark.parametrize("k", [1, 2, 3])
def test_pattern_and_defining_property(request, problem, k):
    A, part, p, A0 = request.getfixturevalue(problem)
    n = A[0]
    orc = O.Oracle(A, part, p, k=2, fill_level=k)
    L = _factor(orc, n)
    for nodes in _blocks(A, part, p):
        want = _level_pattern(A0, nodes, k)
        sub = np.ix_(nodes, nodes)
        got = {(int(nodes[a]), int(nodes[b])) for a, b in zip(*np.nonzero(np.tril(L[sub], -1)))}
        assert got <= want
        # entries kept by the rule can cancel to zero only by accident; none here
        assert got == want
        LLt = L[sub] @ L[sub].T
        mask = np.zeros_like(LLt, dtype=bool)
        idx = {int(x): t for t, x in enumerate(nodes)}
        for i, j in want:
            mask[idx[i], idx[j]] = mask[idx[j], idx[i]] = True
        mask |= np.eye(len(nodes), dtype=bool)
        np.testing.assert_allclose(LLt[mask], A0[sub][mask], atol=1e-12)


def test_level_zero_is_ic0_and_large_level_is_exact(lap2d):
    A, part, p, _ = lap2d
    n = A[0]
    x = W.rhs(n, 2)
    L0 = _factor(O.Oracle(A, part, p, k=2), n)
    assert np.array_equal(_factor(O.Oracle(A, part, p, k=2, fill_level=0), n), L0)
    big = O.Oracle(A, part, p, k=2, fill_level=10 ** 6)
    exact = O.Oracle(A, part, p, k=2, factor=1)
    assert np.abs(big.a0_solve(x) - exact.a0_solve(x)).max() <= 1e-12 * np.abs(exact.a0_solve(x)).max()
    Lb, Le = _factor(big, n), _factor(exact, n)
    assert np.array_equal(Lb != 0, Le != 0)


def test_patterns_grow_with_the_level(lap2d):
    A, part, p, _ = lap2d
    n = A[0]
    prev = None
    for k in range(4):
        nz = _factor(O.Oracle(A, part, p, k=2, fill_level=k), n) != 0
        if prev is not None:
            assert np.all(nz >= prev) and nz.sum() > prev.sum()
        prev = nz


def test_incomplete_ldl_with_fill_on_indefinite_a0():
    A = W.shifted_laplacian((12, 12), 1.3)
    part, p = W.box_partition((12, 12), (2, 2))
    D = DenseDDLR(A, part, p)
    A0 = D.to_original(D.A0)
    n = A[0]
    orc = O.Oracle(A, part, p, k=2, factor=2, fill_level=2, indefinite=1)
    F = _factor(orc, n)
    d = np.diag(F).copy()
    Lu = F.copy()
    np.fill_diagonal(Lu, 1.0)
    for nodes in _blocks(A, part, p):
        sub = np.ix_(nodes, nodes)
        want = _level_pattern(A0, nodes, 2)
        M = Lu[sub] @ np.diag(d[nodes]) @ Lu[sub].T
        idx = {int(x): t for t, x in enumerate(nodes)}
        for i, j in want:
            assert abs(M[idx[i], idx[j]] - A0[i, j]) <= 1e-11
        assert np.allclose(np.diag(M), np.diag(A0[sub]), atol=1e-11)


def test_negative_level_is_invalid(lap2d):
    A, part, p, _ = lap2d
    with pytest.raises(O.OracleError, match="INVALID"):
        O.Oracle(A, part, p, k=2, fill_level=-1)
