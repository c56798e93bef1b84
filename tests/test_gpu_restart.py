"""The true-residual confirmation and restart of PCG (stopping rule of the
design notes: the recursive residual passing tol is confirmed on b - A x;
if that fails, r is replaced by b - A x and CG restarts from x).

A tolerance below what FP64 can reach (1e-16 here, where the true residual
stalls near 3e-16) makes the recursive residual pass it while the true
residual cannot, so every check fails and restarts CG until maxit: the solve
must end NOCONV at maxit, as the oracle does, with x still accurate.  Run in
every PCG form: persistent and per-phase single RHS, batched FP64 and mixed.
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
TOL, MAXIT = 1e-16, 120


@pytest.fixture(scope="module", autouse=True)
def _built():
    pkg.build()
    O.build()


@pytest.fixture(scope="module")
def prob():
    A = W.laplacian((20, 20, 20))
    part, p = W.box_partition((20, 20, 20), (2, 2, 2))
    S = W.to_scipy(A)
    import scipy.sparse.linalg as spl
    B = np.stack([W.rhs(A[0], s) for s in range(4)], axis=1)
    X = np.stack([spl.spsolve(S.tocsc(), B[:, j]) for j in range(4)], axis=1)
    return A, part, p, S, B, X


def _check(S, b, x, xs, info):
    assert info["status"] == "NOCONV" and info["its"] == MAXIT
    # at this level b - A x is rounding noise, so the host's recomputation and
    # the reported true residual agree in magnitude only
    rel = np.linalg.norm(b - S @ x) / np.linalg.norm(b)
    assert rel < 1e-13 and info["relres"] < 1e-13
    assert np.linalg.norm(x - xs) <= 1e-11 * np.linalg.norm(xs)


def test_oracle_ends_at_maxit(prob):
    A, part, p, S, B, X = prob
    orc = O.Oracle(A, part, p, k=8, factor=0, **MC)
    x, its, rel, st = orc.pcg(B[:, 0], TOL, MAXIT)
    assert st == "NOCONV" and its == MAXIT and rel < 1e-13


@pytest.mark.parametrize("persist", ["1", "0"])
def test_single_rhs_restarts(prob, persist, monkeypatch):
    monkeypatch.setenv("DDLR_PERSIST", persist)
    A, part, p, S, B, X = prob
    h = pkg.DDLR(A, part, p, rank_k=8, factor=0, **MC)
    assert bool(h.info()["persistent"] & 1) == (persist == "1")
    x, info = h.pcg(torch.tensor(B[:, 0], device="cuda"), tol=TOL, maxit=MAXIT, check=False)
    _check(S, B[:, 0], x.cpu().numpy(), X[:, 0], info[0])
    h.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_batched_restarts(prob, precision):
    A, part, p, S, B, X = prob
    h = pkg.DDLR(A, part, p, rank_k=8, factor=0, precision=precision, uk_bf16=1, max_nrhs=4, **MC)
    Xg, infos = h.pcg(np.asfortranarray(B), tol=TOL, maxit=MAXIT, check=False)
    for j in range(4):
        _check(S, B[:, j], Xg[:, j], X[:, j], infos[j])
    h.close()
