"""Pins of the oracle's Chebyshev solve with C_a (Sec. 4.3).

The expected values are formed here, densely, from the definitions alone:
C_a = C + a^2 I over the interface nodes, D_a = the part of C_a that couples
interface nodes of the same subdomain (the block Jacobi preconditioner made of
the local diagonal blocks), the generalized eigenpairs C_a V = D_a V L from
LAPACK, and the Chebyshev polynomials T_t from numpy.  The Chebyshev iterate
after t steps from x_0 = 0 on [lo, hi] (centre c, half-width d) is fixed by the
error polynomial:  x_t = V (1 - T_t((c - L)/d) / T_t(c/d)) L^-1 V^T y.
"""
import numpy as np
import pytest
import scipy.linalg as sl
from numpy.polynomial import chebyshev as npc

import oracle as O
import workloads as W
from dense_ddlr import oracle_matrix

CASES = [
    ("2d_12x12_2x2", lambda: (W.laplacian((12, 12)),) + W.box_partition((12, 12), (2, 2))),
    ("3d_6x6x6_2x2x2", lambda: (W.laplacian((6, 6, 6)),) + W.box_partition((6, 6, 6), (2, 2, 2))),
    ("2d_13x11_3x2", lambda: (W.laplacian((13, 11)),) + W.box_partition((13, 11), (3, 2))),
]


def _dense(A, part, alpha=1.0):
    """(dense A, interface indices ascending, C_a, D_a)"""
    Ad = W.to_dense(A)
    part = np.asarray(part)
    off = (Ad != 0) & (part[:, None] != part[None, :])
    idx = np.where(off.any(axis=1))[0]
    C = Ad[np.ix_(idx, idx)] + alpha ** 2 * np.eye(len(idx))
    D = C * (part[idx][:, None] == part[idx][None, :])
    return Ad, idx, C, D


def _cheb_closed_form(lam, V, y, lo, hi, t):
    c, d = 0.5 * (hi + lo), 0.5 * (hi - lo)
    coef = [0] * t + [1]
    P = npc.chebval((c - lam) / d, coef) / npc.chebval(c / d, coef)
    return V @ (((1.0 - P) / lam) * (V.T @ y))


@pytest.fixture(scope="module", params=CASES, ids=[c[0] for c in CASES])
def case(request):
    A, part, p = request.param[1]()
    Ad, idx, C, D = _dense(A, part)
    lam, V = sl.eigh(C, D)          # V^T D V = I
    return A, part, p, Ad, idx, C, D, lam, V


@pytest.mark.parametrize("t", [1, 2, 3, 5, 8])
def test_chebyshev_iterate_is_the_chebyshev_polynomial(case, t):
    """Exact local factors, so the oracle's D_a solve is D_a^-1; the interface
    part of A0^-1 x must be the closed-form Chebyshev iterate, for the exact
    spectrum, a wider interval, and an interval that cuts the spectrum."""
    A, part, p, Ad, idx, C, D, lam, V = case
    orc = O.Oracle(A, part, p, k=2, factor=1, c_solver=1, cheb_steps=t)
    rng = np.random.default_rng(t)
    x = rng.standard_normal(A[0])
    for lo, hi in [(lam[0], lam[-1]), (0.8 * lam[0], 1.3 * lam[-1]), (lam[2], lam[-3])]:
        orc.set_cheb_bounds(lo, hi)
        z = orc.a0_solve(x)
        ref = _cheb_closed_form(lam, V, x[idx], lo, hi, t)
        assert np.linalg.norm(z[idx] - ref) <= 1e-13 * np.linalg.norm(ref)
        # the interior blocks are untouched by the choice of C_a solver
        inter = np.setdiff1d(np.arange(A[0]), idx)
        ze = O.Oracle(A, part, p, k=2, factor=1).a0_solve(x)
        np.testing.assert_allclose(z[inter], ze[inter], rtol=0, atol=1e-14 * np.abs(ze).max())


def test_spectrum_estimate_encloses_and_converges(case):
    """Lanczos estimate on (C_a, D_a), widened by the residual norms: the
    interval contains the spectrum of D_a^-1 C_a and is within 1e-4 of it."""
    A, part, p, Ad, idx, C, D, lam, V = case
    orc = O.Oracle(A, part, p, k=2, factor=1, c_solver=1)
    lo, hi = orc.cheb_bounds
    assert lo <= lam[0] and hi >= lam[-1]
    assert lam[0] - lo <= 1e-4 * lam[0] and hi - lam[-1] <= 1e-4 * lam[-1]
    # two steps are not enough to converge, but the widening keeps hi >= the
    # Ritz value it came from and lo > 0
    lo2, hi2 = O.Oracle(A, part, p, k=2, factor=1, c_solver=1, cheb_lanczos=2).cheb_bounds
    assert 0 < lo2 <= hi2


def test_error_bound(case):
    """||x - x_t||_C <= ||x||_C / T_t(c/d) when [lo, hi] contains the spectrum."""
    A, part, p, Ad, idx, C, D, lam, V = case
    y = np.random.default_rng(7).standard_normal(len(idx))
    xs = np.linalg.solve(C, y)
    cnorm = lambda v: np.sqrt(v @ C @ v)
    for t in (2, 5, 9):
        orc = O.Oracle(A, part, p, k=2, factor=1, c_solver=1, cheb_steps=t)
        lo, hi = orc.cheb_bounds
        x = np.zeros(A[0])
        x[idx] = y
        xt = orc.a0_solve(x)[idx]
        c, d = 0.5 * (hi + lo), 0.5 * (hi - lo)
        bound = cnorm(xs) / npc.chebval(c / d, [0] * t + [1])
        assert cnorm(xs - xt) <= bound * (1 + 1e-10)


def test_block_jacobi_factor_is_d_alpha(case):
    """With exact local factors, L L^T of the C_a block equals D_a: couplings
    across subdomains dropped, a^2 added, nothing else changed."""
    A, part, p, Ad, idx, C, D, lam, V = case
    orc = O.Oracle(A, part, p, k=2, factor=1, c_solver=1)
    r, c, v = orc.factor_coo()
    pos = {g: j for j, g in enumerate(idx)}
    sel = np.array([ri in pos and ci in pos for ri, ci in zip(r, c)])
    L = np.zeros((len(idx), len(idx)))
    for ri, ci, vi in zip(r[sel], c[sel], v[sel]):
        L[pos[ri], pos[ci]] = vi
    partv = np.asarray(part)[idx]
    assert not np.any((L != 0) & (partv[:, None] != partv[None, :]))
    np.testing.assert_allclose(L @ L.T, D, rtol=0, atol=1e-13)


@pytest.mark.parametrize("variant", [1, 2])
def test_full_rank_with_converged_chebyshev_is_exact(variant):
    """k = s with exact local factors: M^-1 = (A0~ - E E^T)^-1 for the A0~ that
    the C_a solve implements; 40 Chebyshev steps make A0~ = A0 to rounding, so
    M^-1 = A^-1 and PCG needs one iteration."""
    A = W.laplacian((12, 12))
    part, p = W.box_partition((12, 12), (2, 2))
    s = _dense(A, part)[1].size
    orc = O.Oracle(A, part, p, variant=variant, k=s, factor=1, c_solver=1, cheb_steps=40)
    Ainv = np.linalg.inv(W.to_dense(A))
    M = oracle_matrix(orc, A[0])
    assert np.abs(M - Ainv).max() <= 1e-11 * np.abs(Ainv).max()
    _, its, rel, st = orc.pcg(W.rhs(A[0], 0), 1e-8)
    assert st == "OK" and its == 1 and rel <= 1e-8


def test_default_chebyshev_preconditions_pcg():
    """IC(0) local factors and the paper's 5 Chebyshev steps: PCG converges, in
    about as many iterations as with C_a factored (the solve with C_a is
    accurate to about 1e-3 on these grids)."""
    A = W.laplacian((16, 16, 16))
    part, p = W.box_partition((16, 16, 16), (2, 2, 2))
    b = W.rhs(A[0], 0)
    its = {}
    for cs in (0, 1):
        orc = O.Oracle(A, part, p, k=8, factor=0, c_solver=cs)
        _, its[cs], rel, st = orc.pcg(b, 1e-8)
        assert st == "OK" and rel <= 1e-8
    assert its[1] <= its[0] + 3


def test_chebyshev_rejects_bad_options():
    A = W.laplacian((8, 8))
    part, p = W.box_partition((8, 8), (2, 2))
    for kw in (dict(c_solver=3), dict(c_solver=1, cheb_steps=0), dict(c_solver=1, cheb_lanczos=0)):
        with pytest.raises(O.OracleError, match="INVALID"):
            O.Oracle(A, part, p, k=2, **kw)
