"""Full-size configurations, checked by properties that hold at any size.

The FP64 oracle takes minutes at these sizes, so instead of element-wise
parity these tests check what the solver must satisfy whatever its size: the
true relative residual ||b - A x|| / ||b|| <= tol, recomputed here on the host
from the CSR matrix; the mixed-precision solution against the FP64 one; the
batched solve against single solves; the Lanczos build's U_k orthonormal.

* 128^3 7-point Laplacian, 512 boxes, k = 32 (n = 2,097,152), FP64 and mixed.
* 96^3 jump-coefficient problem, 125 uneven boxes, k = 24, a block of right-
  hand sides in one batched FP32/FP64 solve.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1505_04341_gb300 as pkg  # noqa: E402
import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu

MC = dict(c_order=1, b_order=1)


@pytest.fixture(scope="module", autouse=True)
def _built():
    pkg.build()


def _true_relres(S, b, x):
    return np.linalg.norm(b - S @ x) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def lap128():
    w = W.workload("lap3d_128_b8")
    return w["A"], w["part"], w["p"], W.to_scipy(w["A"])


def test_lap128_fp64_and_mixed(lap128):
    A, part, p, S = lap128
    b = W.rhs(A[0], 0)
    bd = torch.tensor(b, device="cuda")
    xs = {}
    its = {}
    for name, kw in (("fp64", dict(precision=0)), ("bf16", dict(precision=1, uk_bf16=1))):
        h = pkg.DDLR(A, part, p, variant=1, rank_k=32, factor=0, **MC, **kw)
        if name == "fp64":
            U = h.lowrank()[0]
            assert np.abs(U.T @ U - np.eye(32)).max() < 1e-10
            assert h.info()["persistent"] & 2      # the Lanczos process ran as one launch
        x, info = h.pcg(bd, tol=1e-8)
        xs[name] = x.cpu().numpy()
        its[name] = info[0]["its"]
        assert info[0]["status"] == "OK" and info[0]["relres"] <= 1e-8
        assert _true_relres(S, b, xs[name]) <= 1e-8 * (1 + 1e-6)
        h.close()
    assert abs(its["bf16"] - its["fp64"]) <= max(3, its["fp64"] // 10)
    assert np.linalg.norm(xs["bf16"] - xs["fp64"]) <= 1e-6 * np.linalg.norm(xs["fp64"])


def test_lap128_noalloc_rejects_beyond_its_limit(lap128):
    """n = 2,097,152 exceeds the 1,048,576-row array of the no-allocation A0
    solve: the call fails with INVALID and a message, and the handle stays
    usable."""
    A, part, p, S = lap128
    h = pkg.DDLR(A, part, p, variant=1, rank_k=4, factor=0, lanczos_max=8, **MC)
    x = torch.tensor(W.rhs(A[0], 1), device="cuda")
    with pytest.raises(pkg.DdlrError, match="limit"):
        h.a0_solve_noalloc(x, torch.empty_like(x))
    y = h.a0_solve(x)
    assert torch.isfinite(y).all()
    h.close()


def test_jump96_batched_mixed():
    w = W.workload("jump3d_96_cut5")
    A, part, p = w["A"], w["part"], w["p"]
    S = W.to_scipy(A)
    n = A[0]
    R = 8
    B = np.asfortranarray(np.stack([W.rhs(n, s) for s in range(R)], axis=1))
    h = pkg.DDLR(A, part, p, variant=1, rank_k=24, factor=0, scale_diag=1, precision=1, uk_bf16=0,
                 max_nrhs=R, **MC)
    X, infos = h.pcg(B, tol=1e-8, maxit=3000)
    for j in range(R):
        assert infos[j]["status"] == "OK" and infos[j]["relres"] <= 1e-8
        assert _true_relres(S, B[:, j], X[:, j]) <= 1e-8 * (1 + 1e-6)
    x0, inf0 = h.pcg(np.ascontiguousarray(B[:, 0]), tol=1e-8, maxit=3000)
    # the batched and single-RHS FP32 preconditioners round differently, and
    # over ~1,300 flexible-CG iterations on 10^+-3 jumps that moves the stop
    # by a few iterations (the single-RHS path has its own kernels)
    assert abs(inf0[0]["its"] - infos[0]["its"]) <= 3
    assert np.linalg.norm(x0 - X[:, 0]) <= 1e-6 * np.linalg.norm(x0)
    h.close()
