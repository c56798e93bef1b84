"""Pins of the oracle's indefinite mode and its right-preconditioned GMRES(m)
(Sec. 5: GMRES(40) for the indefinite model problems -Lap u - c u and for
preconditioners that are not SPD).

What fixes them, independently of the oracle:
* Sylvester's law of inertia: A = A0^{1/2} (I - A0^{-1/2} E E^T A0^{-1/2})
  A0^{1/2}, so with A0 positive definite the number of eigenvalues of
  H = E^T A0^-1 E above 1 equals the number of negative eigenvalues of A
  (dense LAPACK on both sides; the oracle's full-rank Ritz values too);
* the SMW identity still holds for indefinite A: exact factors and k = s give
  M^-1 = A^-1, hence one GMRES step, in both variants (this also pins the
  Gauss-Jordan inverse of an indefinite I - K);
* GMRES's defining property: after j steps from x0 = 0 its residual is the
  least-squares minimum of ||b - A M^-1 y|| over the Krylov space
  K_j(A M^-1, b), computed here from an explicit, QR-orthonormalised basis;
  the residual never grows within a cycle; restarting can only cost steps.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from dense_ddlr import DenseDDLR, oracle_matrix


@pytest.fixture(scope="module")
def indef2d():
    A = W.shifted_laplacian((24, 24), 0.1)
    part, p = W.box_partition((24, 24), (2, 2))
    return A, part, p


def test_inertia_of_h_matches_a(indef2d):
    A, part, p = indef2d
    d = DenseDDLR(A, part, p)
    assert np.linalg.eigvalsh(d.A0).min() > 0
    neg = int((np.linalg.eigvalsh(W.to_dense(A)) < 0).sum())
    assert neg == 3
    assert int((d.lam > 1.0).sum()) == neg
    o = O.Oracle(A, part, p, k=d.s, factor=1, indefinite=1)
    np.testing.assert_allclose(np.sort(o.ritz)[::-1], d.lam, atol=1e-10)


def test_spd_mode_refuses_and_indefinite_mode_accepts(indef2d):
    A, part, p = indef2d
    with pytest.raises(O.OracleError, match="NOT_SPD"):
        O.Oracle(A, part, p, k=8, factor=1)
    o = O.Oracle(A, part, p, k=8, factor=1, indefinite=1)
    assert o.ritz[0] > 1.0


@pytest.mark.parametrize("variant", [1, 2])
def test_full_rank_is_exact_for_indefinite_a(indef2d, variant):
    A, part, p = indef2d
    o = O.Oracle(A, part, p, variant=variant, k=92, factor=1, indefinite=1)
    assert o.s == 92
    Ainv = np.linalg.inv(W.to_dense(A))
    assert np.abs(oracle_matrix(o, A[0]) - Ainv).max() <= 1e-10 * np.abs(Ainv).max()
    _, its, rel, st = o.gmres(W.rhs(A[0], 0), 1e-10)
    assert st == "OK" and its == 1 and rel <= 1e-10


@pytest.mark.parametrize("variant", [1, 2])
def test_gmres_residual_is_the_krylov_minimum(indef2d, variant):
    A, part, p = indef2d
    n = A[0]
    o = O.Oracle(A, part, p, variant=variant, k=8, indefinite=1)
    Ad = W.to_dense(A)
    AM = Ad @ oracle_matrix(o, n)
    b = W.rhs(n, 0)
    K = np.empty((n, 12))
    v = b.copy()
    for j in range(12):
        K[:, j] = v
        v = AM @ v
    prev = np.inf
    for j in range(1, 13):
        Q, _ = np.linalg.qr(K[:, :j])
        c, *_ = np.linalg.lstsq(AM @ Q, b, rcond=None)
        rmin = np.linalg.norm(b - AM @ (Q @ c)) / np.linalg.norm(b)
        x, its, rel, st = o.gmres(b, 1e-14, maxit=j, restart=40)
        assert its == j
        np.testing.assert_allclose(rel, rmin, rtol=1e-6)
        assert np.linalg.norm(b - Ad @ x) / np.linalg.norm(b) == pytest.approx(rel, rel=1e-10)
        assert rel <= prev * (1 + 1e-12)
        prev = rel


def test_restart_and_exact_termination(indef2d):
    A, part, p = indef2d
    b = W.rhs(A[0], 1)
    o = O.Oracle(A, part, p, k=8, indefinite=1)
    _, its40, rel40, st40 = o.gmres(b, 1e-8, 500, 40)
    _, its10, rel10, st10 = o.gmres(b, 1e-8, 2000, 10)
    assert st40 == "OK" and st10 == "OK" and rel40 <= 1e-8 and rel10 <= 1e-8
    assert its10 >= its40
    # a 6x6 problem: full GMRES ends within n steps at any tolerance
    As = W.shifted_laplacian((6,), 1.0)
    ps = np.array([0, 0, 0, 1, 1, 1], dtype=np.int32)
    os_ = O.Oracle(As, ps, 2, k=1, indefinite=1)
    _, its, rel, st = os_.gmres(W.rhs(6, 2), 1e-13, 6, 6)
    assert st == "OK" and its <= 6 and rel <= 1e-13


def test_gmres_on_spd_problem_matches_pcg_quality():
    A = W.laplacian((16, 16, 16))
    part, p = W.box_partition((16, 16, 16), (2, 2, 2))
    o = O.Oracle(A, part, p, k=8)
    b = W.rhs(A[0], 0)
    _, its_g, rel_g, st_g = o.gmres(b, 1e-8)
    _, its_c, rel_c, st_c = o.pcg(b, 1e-8)
    assert st_g == st_c == "OK" and rel_g <= 1e-8
    # GMRES minimises the residual norm over the same Krylov space CG uses
    assert its_g <= its_c + 1


def test_bad_gmres_arguments(indef2d):
    A, part, p = indef2d
    o = O.Oracle(A, part, p, k=4, indefinite=1)
    _, _, _, st = o.gmres(W.rhs(A[0], 0), 1e-8, 10, 0)
    assert st == "INVALID"
    x, its, rel, st = o.gmres(np.zeros(A[0]), 1e-8)
    assert st == "OK" and its == 0 and not x.any()
