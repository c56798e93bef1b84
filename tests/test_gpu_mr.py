"""GPU parity of the MR approximate inverse of C_a (c_solver=2, Sec. 4.3,
Algorithm 2) against the oracle, through the C ABI.

Without dropping the approximate inverse is a fixed function of C_a, so the
A0 solve must match the oracle to 1e-12.  With the default dual-threshold
dropping, grid symmetry makes exactly equal magnitudes common, and which of
two equal entries survives is decided by rounding, so there the comparison
is on what is unique: PCG reaches tol within two iterations of the oracle.
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
    "2d_12x12_exact": lambda: (W.laplacian((12, 12)),) + W.box_partition((12, 12), (2, 2)) + (1, 0),
    "3d_20_multicolour": lambda: (W.laplacian((20, 20, 20)),) + W.box_partition((20, 20, 20), (2, 2, 2)) + (0, 3),
    "3d_24_natural": lambda: (W.laplacian((24, 24, 24)),) + W.box_partition((24, 24, 24), (3, 2, 2)) + (0, 0),
    "jump_32_multicolour": lambda: (W.jump_coefficient_fv(32, 8, 0),) + W.random_cut_partition(32, 3, 0, 6, 16) + (0, 3),
}


def _orders(o):
    return dict(c_order=o & 1, b_order=o >> 1)


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.fixture(scope="module", autouse=True)
def _built():
    pkg.build()
    O.build()


def test_one_step_closed_form():
    """C_a = [[3, -1], [-1, 3]]: one MR step from diag(C_a)^-1 gives
    beta = 9/10 and X_1 = [[1/3, 1/10], [1/10, 1/3]]."""
    A = W.laplacian((4,))
    part = np.array([0, 0, 1, 1], dtype=np.int32)
    h = pkg.DDLR(A, part, 2, rank_k=1, factor=1, c_solver=2, mr_iters=1, mr_lfil=2, mr_droptol=0.0)
    X = np.zeros((2, 2))
    for j, g in enumerate((1, 2)):
        x = np.zeros(4)
        x[g] = 1.0
        X[:, j] = h.a0_solve(torch.tensor(x, device="cuda")).cpu().numpy()[[1, 2]]
    np.testing.assert_allclose(X, [[1 / 3, 1 / 10], [1 / 10, 1 / 3]], rtol=0, atol=1e-15)
    h.close()


@pytest.mark.parametrize("name", list(PROBLEMS))
def test_no_dropping_matches_oracle(name):
    """One MR step keeps the pattern of C_a (at most 7 entries per column
    here), so lfil = 8 and tolerance 0 drop nothing."""
    A, part, p, factor, orders = PROBLEMS[name]()
    scale = 1 if name.startswith("jump") else 0
    kw = dict(factor=factor, scale_diag=scale, c_solver=2, mr_iters=1, mr_lfil=8, mr_droptol=0.0,
              **_orders(orders))
    h = pkg.DDLR(A, part, p, rank_k=4, **kw)
    orc = O.Oracle(A, part, p, k=4, **kw)
    assert h.info()["persistent"] == 0
    for seed in (1, 2):
        x = W.rhs(A[0], seed)
        y = h.a0_solve(torch.tensor(x, device="cuda")).cpu().numpy()
        assert _rel(y, orc.a0_solve(x)) < 1e-12
    x = W.rhs(A[0], 3)
    assert np.array_equal(h.a0_solve(x), h.a0_solve(torch.tensor(x, device="cuda")).cpu().numpy())
    h.close()


@pytest.mark.parametrize("variant", [1, 2])
@pytest.mark.parametrize("name", list(PROBLEMS))
def test_default_dropping_pcg_matches_oracle(name, variant):
    A, part, p, factor, orders = PROBLEMS[name]()
    scale = 1 if name.startswith("jump") else 0
    kw = dict(variant=variant, factor=factor, scale_diag=scale, c_solver=2, **_orders(orders))
    h = pkg.DDLR(A, part, p, rank_k=8, **kw)
    orc = O.Oracle(A, part, p, k=8, mr_lfil=8, **kw)
    b = W.rhs(A[0], 0)
    x, info = h.pcg(torch.tensor(b, device="cuda"), tol=1e-8, maxit=2000)
    _, its_o, _, st = orc.pcg(b, 1e-8, 2000)
    assert st == "OK" and info[0]["status"] == "OK" and info[0]["relres"] <= 1e-8
    assert abs(info[0]["its"] - its_o) <= 2
    S = W.to_scipy(A)
    xn = x.cpu().numpy()
    assert np.linalg.norm(b - S @ xn) <= 1e-8 * (1 + 1e-6) * np.linalg.norm(b)
    # the build is deterministic: a refactor gives the same bits
    y0 = h.a0_solve(torch.tensor(b, device="cuda")).cpu().numpy()
    h.refactor()
    assert np.array_equal(h.a0_solve(torch.tensor(b, device="cuda")).cpu().numpy(), y0)
    h.close()


def test_mixed_precision_and_batched():
    A = W.laplacian((24, 24, 24))
    part, p = W.box_partition((24, 24, 24), (3, 2, 2))
    S = W.to_scipy(A)
    B = np.asfortranarray(np.stack([W.rhs(A[0], s) for s in range(3)], axis=1))
    for kw in (dict(precision=1, uk_bf16=1), dict(max_nrhs=3), dict(lowrank_method=1)):
        h = pkg.DDLR(A, part, p, rank_k=16, c_solver=2, c_order=1, b_order=1, **kw)
        X, infos = h.pcg(B, tol=1e-8)
        for j in range(3):
            assert infos[j]["status"] == "OK"
            assert np.linalg.norm(B[:, j] - S @ X[:, j]) <= 1e-8 * (1 + 1e-6) * np.linalg.norm(B[:, j])
        h.close()


def test_mr_rejects_bad_options():
    A = W.laplacian((16, 16))
    part, p = W.box_partition((16, 16), (2, 2))
    for kw in (dict(c_solver=3), dict(c_solver=2, mr_lfil=0), dict(c_solver=2, mr_iters=4, mr_lfil=8),
               dict(c_solver=2, mr_droptol=-1.0), dict(c_solver=2, mr_iters=-1)):
        with pytest.raises(pkg.DdlrError, match="INVALID"):
            pkg.DDLR(A, part, p, rank_k=4, **kw)
