"""GPU parity of the level-of-fill incomplete factors (fill_level k with
factor 0 or 2) against the oracle, through the C ABI: factor entries and the
A0 solve within 1e-12, PCG (or GMRES for the indefinite case) within one
iteration of the oracle's and the true residual; the level patterns
themselves are checked on the CPU (planner and oracle against the
definition).

Collected after the other GPU files: its only GPU run so far came before
the fix of the process-wide shared-memory limits, so a failure here should
not stop the files that have run green."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle as O  # noqa: E402
import paper_1505_04341_gb300 as pkg  # noqa: E402
import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu

CASES = {
    "3d_16_k1_natural": lambda: (W.laplacian((16, 16, 16)),) + W.box_partition((16, 16, 16), (2, 2, 2)) + (0, 0, 1),
    "3d_16_k2_multicolour": lambda: (W.laplacian((16, 16, 16)),) + W.box_partition((16, 16, 16), (2, 2, 2))
    + (0, 1, 2),
    "2d_24_ldl_k2_indefinite": lambda: (W.shifted_laplacian((24, 24), 0.3),) + W.box_partition((24, 24), (2, 2))
    + (2, 0, 2),
}


@pytest.fixture(scope="module", autouse=True)
def _built():
    pkg.build()
    O.build()


def _dense(r, c, v, n):
    M = np.zeros((n, n))
    M[r, c] = v
    return M


@pytest.mark.parametrize("name", list(CASES))
def test_fill_factors_match_oracle(name):
    A, part, p, factor, order, k = CASES[name]()
    n = A[0]
    indef = 1 if factor == 2 else 0
    kw = dict(factor=factor, c_order=order, b_order=order, fill_level=k, indefinite=indef)
    h = pkg.DDLR(A, part, p, rank_k=8, **kw)
    orc = O.Oracle(A, part, p, k=8, **kw)
    h0 = pkg.DDLR(A, part, p, rank_k=8, **dict(kw, fill_level=0))
    assert h.info()["nnz_factor"] > h0.info()["nnz_factor"]
    h0.close()
    Fg, Fo = _dense(*h.factor_coo(), n), _dense(*orc.factor_coo(), n)
    assert np.abs(Fg - Fo).max() <= 1e-12 * np.abs(Fo).max()
    x = W.rhs(n, 1)
    y = h.a0_solve(torch.tensor(x, device="cuda")).cpu().numpy()
    yo = orc.a0_solve(x)
    assert np.abs(y - yo).max() <= 1e-12 * np.abs(yo).max()
    b = W.rhs(n, 0)
    S = W.to_scipy(A)
    if indef:
        xs, info = h.gmres(torch.tensor(b, device="cuda"), tol=1e-8)
        _, its_o, _, st = orc.gmres(b, 1e-8)
        its = info["its"]
        ok = info["status"] == "OK"
    else:
        xs, infos = h.pcg(torch.tensor(b, device="cuda"), tol=1e-8)
        _, its_o, _, st = orc.pcg(b, 1e-8)
        its, ok = infos[0]["its"], infos[0]["status"] == "OK"
    assert st == "OK" and ok and abs(its - its_o) <= 1
    assert np.linalg.norm(b - S @ xs.cpu().numpy()) <= 1e-8 * (1 + 1e-6) * np.linalg.norm(b)
    h.close()


def test_fill_level_options_refused():
    A = W.laplacian((8, 8))
    part, p = W.box_partition((8, 8), (2, 2))
    for kw in (dict(fill_level=-1), dict(fill_level=65), dict(fill_level=1, factor=1), dict(fill_level=2, factor=3)):
        with pytest.raises(pkg.DdlrError, match="INVALID"):
            pkg.DDLR(A, part, p, rank_k=2, **kw)
