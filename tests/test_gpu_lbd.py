"""GPU parity of the Lanczos bidiagonalisation for DDLR-2 (lowrank_method=2)
against the oracle, and against the GPU's own Lanczos on E^T A0^-2 E from the
same start vector (the two give the same Ritz values and preconditioner in
exact arithmetic).

Bars: converged Ritz values within 1e-8 relative; M^-1 x of the two GPU
builds within 1e-7; PCG within +-1 iteration of the oracle; exact at full
rank; DDLR-1 refused.
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
    "2d_40x30_exact": lambda: (W.laplacian((40, 30)),) + W.box_partition((40, 30), (3, 2)) + (1, 0),
    "3d_20_multicolour": lambda: (W.laplacian((20, 20, 20)),) + W.box_partition((20, 20, 20), (2, 2, 2)) + (0, 3),
    "3d_24_natural": lambda: (W.laplacian((24, 24, 24)),) + W.box_partition((24, 24, 24), (3, 2, 2)) + (0, 0),
}


def _orders(o):
    return dict(c_order=o & 1, b_order=o >> 1)


@pytest.fixture(scope="module", autouse=True)
def _built():
    pkg.build()
    O.build()


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_matches_oracle_and_gpu_lanczos(name, monkeypatch):
    A, part, p, factor, orders = PROBLEMS[name]()
    kw = dict(variant=2, factor=factor, **_orders(orders))
    h = pkg.DDLR(A, part, p, rank_k=8, lowrank_method=2, **kw)
    orc = O.Oracle(A, part, p, k=8, lowrank_method=2, **kw)
    assert h.info()["lanczos_steps"] == orc.msteps
    np.testing.assert_allclose(h.ritz()[:8], orc.ritz[:8], rtol=1e-8)
    b = W.rhs(A[0], 0)
    x, info = h.pcg(torch.tensor(b, device="cuda"), tol=1e-8)
    _, its_o, _, st = orc.pcg(b, 1e-8)
    assert st == "OK" and info[0]["status"] == "OK" and info[0]["relres"] <= 1e-8
    assert abs(info[0]["its"] - its_o) <= 1
    # the GPU's Lanczos on E^T A0^-2 E (kernel-per-phase, same forced length)
    monkeypatch.setenv("DDLR_PERSIST", "0")
    m = h.info()["lanczos_steps"]
    hl = pkg.DDLR(A, part, p, rank_k=8, lanczos_max=m, lanczos_eps=1e-300, **kw)
    hb = pkg.DDLR(A, part, p, rank_k=8, lanczos_max=m, lanczos_eps=1e-300, lowrank_method=2, **kw)
    np.testing.assert_allclose(hb.ritz()[:8], hl.ritz()[:8], rtol=1e-8)
    xv = torch.tensor(W.rhs(A[0], 3), device="cuda")
    yl, yb = hl.apply(xv).cpu().numpy(), hb.apply(xv).cpu().numpy()
    assert np.abs(yb - yl).max() <= 1e-7 * np.abs(yl).max()
    for hh in (h, hl, hb):
        hh.close()


def test_full_rank_is_exact():
    A = W.laplacian((12, 12))
    part, p = W.box_partition((12, 12), (2, 2))
    h = pkg.DDLR(A, part, p, variant=2, rank_k=44, factor=1, lowrank_method=2)
    _, info = h.pcg(torch.tensor(W.rhs(A[0], 0), device="cuda"), tol=1e-10)
    assert info[0]["status"] == "OK" and info[0]["its"] == 1
    h.close()


def test_mixed_precision_and_refactor():
    A = W.laplacian((24, 24, 24))
    part, p = W.box_partition((24, 24, 24), (3, 2, 2))
    h = pkg.DDLR(A, part, p, variant=2, rank_k=16, lowrank_method=2, precision=1, uk_bf16=1, c_order=1, b_order=1)
    r0 = h.ritz()
    h.refactor()
    assert np.array_equal(h.ritz(), r0)
    _, info = h.pcg(torch.tensor(W.rhs(A[0], 1), device="cuda"), tol=1e-8)
    assert info[0]["status"] == "OK" and info[0]["relres"] <= 1e-8
    h.close()


def test_bidiagonalisation_rejects_ddlr1():
    A = W.laplacian((16, 16))
    part, p = W.box_partition((16, 16), (2, 2))
    with pytest.raises(pkg.DdlrError, match="INVALID"):
        pkg.DDLR(A, part, p, variant=1, rank_k=4, lowrank_method=2)
