"""Pins of the oracle's randomized low-rank build (lowrank_method=1): the
randomized subspace iteration the paper's conclusion names as a faster
alternative to Lanczos for the eigenpairs of H = E^T A0^-1 E (DDLR-1) or
E^T A0^-2 E (DDLR-2).

Expected values come from dense LAPACK on matrices formed from the paper's
definitions (tests/dense_ddlr.py) and from the Rayleigh-Ritz theory: Ritz
values of H on any ell-dimensional subspace lie below the ell largest
eigenvalues one by one (Cauchy interlacing), a full subspace gives them
exactly, and the error shrinks with the power steps.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from dense_ddlr import DenseDDLR, oracle_matrix


@pytest.fixture(scope="module")
def small():
    A = W.laplacian((12, 12))
    part, p = W.box_partition((12, 12), (2, 2))
    return A, part, p, DenseDDLR(A, part, p)


def _h2_eigs(D):
    X = D.A0inv @ D.E
    K2 = X.T @ X
    return np.sort(np.linalg.eigvalsh(0.5 * (K2 + K2.T)))[::-1]


@pytest.mark.parametrize("variant", [1, 2])
def test_full_subspace_is_exact(small, variant):
    """ell = s: B = Q^T H Q is similar to H, so the Ritz values are H's
    eigenvalues; with exact local factors and k = s, M^-1 = A^-1 and PCG
    takes one iteration (both variants)."""
    A, part, p, D = small
    s = D.s
    orc = O.Oracle(A, part, p, variant=variant, k=s, factor=1, lowrank_method=1, rand_oversample=0,
                   rand_power=0)
    lam = D.lam if variant == 1 else _h2_eigs(D)
    assert orc.msteps == s
    np.testing.assert_allclose(orc.ritz, lam, rtol=0, atol=1e-12)
    Ainv = np.linalg.inv(W.to_dense(A))
    M = oracle_matrix(orc, A[0])
    assert np.abs(M - Ainv).max() <= 1e-11 * np.abs(Ainv).max()
    _, its, rel, st = orc.pcg(W.rhs(A[0], 0), 1e-8)
    assert st == "OK" and its == 1


def test_ritz_values_interlace_and_improve_with_power_steps(small):
    A, part, p, D = small
    k, over = 6, 10
    errs = []
    for q in (0, 1, 2, 4, 8):
        orc = O.Oracle(A, part, p, k=k, factor=1, lowrank_method=1, rand_oversample=over, rand_power=q)
        ell = k + over
        assert orc.msteps == ell
        r = orc.ritz
        assert np.all(np.diff(r) <= 1e-15)                       # descending
        assert np.all(r <= D.lam[:ell] + 1e-13)                  # Cauchy interlacing
        errs.append(np.abs(r[:k] - D.lam[:k]).max())
        U, lam, _ = orc.lowrank()
        np.testing.assert_allclose(U.T @ U, np.eye(k), atol=1e-12)
        assert abs(orc.theta - r[k]) == 0.0                      # theta = Ritz_{k+1}
    assert all(errs[i + 1] < errs[i] for i in range(len(errs) - 1))
    assert errs[-1] < 1e-3 and errs[-1] < 1e-2 * errs[0]


def test_randomized_preconditioner_solves(small):
    """IC(0), k = 8, default oversampling and power steps: PCG converges in
    both variants, within a few iterations of the Lanczos-built preconditioner."""
    A = W.laplacian((16, 16, 16))
    part, p = W.box_partition((16, 16, 16), (2, 2, 2))
    b = W.rhs(A[0], 0)
    for variant in (1, 2):
        its = {}
        for method in (0, 1):
            orc = O.Oracle(A, part, p, variant=variant, k=8, factor=0, lowrank_method=method)
            _, its[method], rel, st = orc.pcg(b, 1e-8)
            assert st == "OK" and rel <= 1e-8
        assert its[1] <= its[0] + max(3, its[0] // 10)


def test_randomized_rejects_bad_options():
    A = W.laplacian((8, 8))
    part, p = W.box_partition((8, 8), (2, 2))
    for kw in (dict(lowrank_method=2), dict(lowrank_method=1, rand_oversample=-1),
               dict(lowrank_method=1, rand_power=-1)):
        with pytest.raises(O.OracleError, match="INVALID"):
            O.Oracle(A, part, p, k=2, **kw)
