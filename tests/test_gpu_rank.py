"""Raising the rank of a built preconditioner (Sec. 3.4, improving a given
preconditioner): the Lanczos process continues from its last step.

With a convergence tolerance that never stops the process, the steps run to
the limit (5 k) and the Krylov sequence from the same start vector is fixed,
so raising k from 6 to 12 must give what a fresh setup with k = 12 gives:
the same Ritz values, the same U_k, the same PCG, and the oracle's values.
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

MC = dict(c_order=1, b_order=1)


@pytest.fixture(scope="module", autouse=True)
def _built():
    pkg.build()
    O.build()


@pytest.mark.parametrize("persist", ["1", "0"])
@pytest.mark.parametrize("variant", [1, 2])
def test_increase_rank_equals_fresh_setup(variant, persist, monkeypatch):
    monkeypatch.setenv("DDLR_PERSIST", persist)
    A = W.laplacian((24, 24, 24))
    part, p = W.box_partition((24, 24, 24), (3, 2, 2))
    kw = dict(variant=variant, factor=0, lanczos_eps=1e-300, **MC)
    h = pkg.DDLR(A, part, p, rank_k=6, **kw)
    assert h.info()["lanczos_steps"] == 30
    h.increase_rank(12)
    f = pkg.DDLR(A, part, p, rank_k=12, **kw)
    hi, fi = h.info(), f.info()
    assert hi["k"] == 12 and hi["lanczos_steps"] == fi["lanczos_steps"] == 60
    rh, rf = h.ritz(), f.ritz()
    np.testing.assert_allclose(rh, rf, rtol=1e-10, atol=1e-13 * np.abs(rf).max())
    orc = O.Oracle(A, part, p, variant=variant, k=12, factor=0, lanczos_eps=1e-300, **MC)
    np.testing.assert_allclose(rh[:13], orc.ritz[:13], rtol=1e-8)
    Uh, Uf = h.lowrank()[0], f.lowrank()[0]
    if variant == 1:
        np.testing.assert_allclose(Uh.T @ Uh, np.eye(12), atol=1e-10)
    b = W.rhs(A[0], 0)
    bd = torch.tensor(b, device="cuda")
    _, ih = h.pcg(bd, tol=1e-8)
    _, iff = f.pcg(bd, tol=1e-8)
    _, its_o, _, st = orc.pcg(b, 1e-8)
    assert st == "OK" and ih[0]["status"] == "OK" and ih[0]["relres"] <= 1e-8
    assert abs(ih[0]["its"] - iff[0]["its"]) <= 1 and abs(ih[0]["its"] - its_o) <= 1
    h.close()
    f.close()


def test_increase_rank_twice_and_mixed_precision(monkeypatch):
    """Two raises in a row on a mixed-precision handle (the FP32/BF16 copies of
    U_k are rebuilt each time); the solve still reaches tol."""
    A = W.laplacian((24, 24, 24))
    part, p = W.box_partition((24, 24, 24), (3, 2, 2))
    h = pkg.DDLR(A, part, p, variant=1, rank_k=4, factor=0, precision=1, uk_bf16=1, **MC)
    b = torch.tensor(W.rhs(A[0], 2), device="cuda")
    _, i4 = h.pcg(b, tol=1e-8)
    h.increase_rank(8)
    h.increase_rank(16)
    assert h.info()["k"] == 16
    _, i16 = h.pcg(b, tol=1e-8)
    assert i16[0]["status"] == "OK" and i16[0]["relres"] <= 1e-8
    assert i16[0]["its"] <= i4[0]["its"]
    h.close()


def test_increase_rank_rejects_bad_ranks():
    A = W.laplacian((16, 16))
    part, p = W.box_partition((16, 16), (2, 2))
    h = pkg.DDLR(A, part, p, variant=1, rank_k=4, factor=0)
    s = h.info()["s"]
    for k_new in (4, 3, s + 1):
        with pytest.raises(pkg.DdlrError, match="INVALID"):
            h.increase_rank(k_new)
    x = torch.tensor(W.rhs(A[0], 0), device="cuda")
    _, info = h.pcg(x, tol=1e-8)
    assert info[0]["status"] == "OK"
    h.close()
