"""GPU parity of the L D L^T local factors (factor 2: incomplete on the
block pattern, factor 3: exact on the symbolic fill pattern; Sec. 5's
"incomplete Cholesky or LDL" for indefinite problems) against the oracle,
through the C ABI.

Bars: factor entries (unit L, d in the diagonal slot) and the A0 solve
within 1e-12 of the oracle's on problems whose A0 is indefinite (a shifted
5-point Laplacian and a shifted 9-point stencil, whose triangles exercise the
update terms inside the pattern) and on a 3-D shifted Laplacian, both
elimination orders; GMRES steps within +-1 of the oracle's and the true
residual; full rank with exact factors takes one step; on an SPD problem the
incomplete L D L^T gives the IC(0) solve; the options it excludes are
refused; several right-hand sides are solved one at a time, bitwise as alone.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle as O  # noqa: E402
import paper_1505_04341_gb300 as pkg  # noqa: E402
import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu

PROBLEMS = {
    "2d_12_s1.3": lambda: (W.shifted_laplacian((12, 12), 1.3),) + W.box_partition((12, 12), (2, 2)),
    "9pt_16_s2": lambda: (W.nine_point(16, 2.0),) + W.box_partition((16, 16), (2, 2)),
    "3d_10_s0.9": lambda: (W.shifted_laplacian((10, 10, 10), 0.9),) + W.box_partition((10, 10, 10), (2, 2, 2)),
}


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _coo_dense(r, c, v, n):
    M = np.zeros((n, n))
    M[r, c] = v
    return M


@pytest.fixture(scope="module", autouse=True)
def _built():
    pkg.build()
    O.build()


@pytest.mark.parametrize("order", [0, 1])
@pytest.mark.parametrize("factor", [2, 3])
@pytest.mark.parametrize("name", list(PROBLEMS))
def test_factor_and_a0_solve_match_oracle(name, factor, order):
    A, part, p = PROBLEMS[name]()
    n = A[0]
    kw = dict(factor=factor, c_order=order, b_order=order, indefinite=1)
    h = pkg.DDLR(A, part, p, rank_k=4, **kw)
    orc = O.Oracle(A, part, p, k=4, **kw)
    Fg = _coo_dense(*h.factor_coo(), n)
    Fo = _coo_dense(*orc.factor_coo(), n)
    assert np.abs(Fg - Fo).max() <= 1e-12 * np.abs(Fo).max()
    for seed in (1, 2):
        x = W.rhs(n, seed)
        y = h.a0_solve(torch.tensor(x, device="cuda")).cpu().numpy()
        assert _rel(y, orc.a0_solve(x)) < 1e-12
    h.close()


@pytest.mark.parametrize("variant", [1, 2])
@pytest.mark.parametrize("factor", [2, 3])
@pytest.mark.parametrize("name", ["2d_12_s1.3", "9pt_16_s2"])
def test_gmres_matches_oracle(name, factor, variant):
    A, part, p = PROBLEMS[name]()
    kw = dict(variant=variant, factor=factor, c_order=1, b_order=1, indefinite=1)
    h = pkg.DDLR(A, part, p, rank_k=8, **kw)
    orc = O.Oracle(A, part, p, k=8, **kw)
    assert h.info()["lanczos_steps"] == orc.msteps
    b = W.rhs(A[0], 0)
    x, info = h.gmres(torch.tensor(b, device="cuda"), tol=1e-8)
    _, its_o, _, st = orc.gmres(b, 1e-8)
    assert st == "OK" and info["status"] == "OK" and abs(info["its"] - its_o) <= 1
    S = W.to_scipy(A)
    assert np.linalg.norm(b - S @ x.cpu().numpy()) <= 1e-8 * (1 + 1e-6) * np.linalg.norm(b)
    h.close()


@pytest.mark.parametrize("variant", [1, 2])
def test_full_rank_exact_ldl(variant):
    A, part, p = PROBLEMS["2d_12_s1.3"]()
    h = pkg.DDLR(A, part, p, variant=variant, rank_k=44, factor=3, indefinite=1)
    assert h.info()["s"] == 44
    _, info = h.gmres(W.rhs(A[0], 0), tol=1e-10)
    assert info["status"] == "OK" and info["its"] == 1
    with pytest.raises(pkg.DdlrError, match="BREAKDOWN"):
        pkg.DDLR(A, part, p, variant=variant, rank_k=44, factor=1, indefinite=1)
    h.close()


def test_spd_problem_matches_ic0_and_refused_options():
    A = W.laplacian((16, 16, 16))
    part, p = W.box_partition((16, 16, 16), (2, 2, 2))
    x = W.rhs(A[0], 3)
    h0 = pkg.DDLR(A, part, p, rank_k=8, c_order=1, b_order=1)
    h2 = pkg.DDLR(A, part, p, rank_k=8, c_order=1, b_order=1, factor=2)
    assert _rel(h2.a0_solve(x), h0.a0_solve(x)) < 1e-12
    _, i0 = h0.pcg(x, tol=1e-8)
    _, i2 = h2.pcg(x, tol=1e-8)
    assert i2[0]["status"] == "OK" and abs(i2[0]["its"] - i0[0]["its"]) <= 1
    # several right-hand sides on an L D L^T handle: one at a time, bitwise
    X = np.asfortranarray(np.stack([W.rhs(A[0], s) for s in range(3)], axis=1))
    Y = h2.apply(X)
    for j in range(3):
        assert np.array_equal(Y[:, j], h2.apply(np.ascontiguousarray(X[:, j])))
    h0.close()
    h2.close()
    for kw in (dict(factor=2, precision=1), dict(factor=2, c_solver=1), dict(factor=3, lowrank_method=1),
               dict(factor=4)):
        with pytest.raises(pkg.DdlrError, match="INVALID"):
            pkg.DDLR(A, part, p, rank_k=8, **kw)
