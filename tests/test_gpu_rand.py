"""GPU parity of the randomized low-rank build (lowrank_method=1) against the
oracle: the same test matrix (SplitMix64 streams over the interface nodes in
ascending original index), the same power steps, so the same subspace and the
same Rayleigh quotient up to rounding.

Bars: the ell Ritz values within 1e-10 relative; U_k orthonormal; with a full
subspace and exact factors the preconditioner is exact (PCG in one
iteration); PCG iterations within +-1 of the oracle with each side's own
setup; the build is bitwise repeatable.
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
    "3d_33x17x21_ragged": lambda: (W.laplacian((33, 17, 21)),) + W.box_partition((33, 17, 21), (3, 2, 2)) + (0, 1),
}


def _orders(o):
    return dict(c_order=o & 1, b_order=o >> 1)


@pytest.fixture(scope="module", autouse=True)
def _built():
    pkg.build()
    O.build()


@pytest.mark.parametrize("variant", [1, 2])
@pytest.mark.parametrize("name", list(PROBLEMS))
def test_ritz_values_and_pcg_match_oracle(name, variant):
    A, part, p, factor, orders = PROBLEMS[name]()
    kw = dict(variant=variant, factor=factor, **_orders(orders))
    h = pkg.DDLR(A, part, p, rank_k=8, lowrank_method=1, rand_oversample=10, rand_power=2, **kw)
    orc = O.Oracle(A, part, p, k=8, lowrank_method=1, rand_oversample=10, rand_power=2, **kw)
    rh, ro = h.ritz(), orc.ritz
    assert len(rh) == len(ro) == 18 and h.info()["lanczos_steps"] == 18
    np.testing.assert_allclose(rh, ro, rtol=1e-10, atol=1e-14 * np.abs(ro).max())
    if variant == 1:
        U = h.lowrank()[0]
        np.testing.assert_allclose(U.T @ U, np.eye(8), atol=1e-10)
        assert abs(h.info()["theta"] - orc.theta) <= 1e-10 * abs(orc.theta)
    b = W.rhs(A[0], 0)
    x, info = h.pcg(torch.tensor(b, device="cuda"), tol=1e-8)
    _, its_o, _, st = orc.pcg(b, 1e-8)
    assert st == "OK" and info[0]["status"] == "OK" and info[0]["relres"] <= 1e-8
    assert abs(info[0]["its"] - its_o) <= 1
    # the build is deterministic: a refactor gives the same bits
    h.refactor()
    assert np.array_equal(h.ritz(), rh)
    h.close()


@pytest.mark.parametrize("variant", [1, 2])
def test_full_subspace_is_exact(variant):
    """ell = s = 44 with exact local factors and k = s: M^-1 = A^-1."""
    A = W.laplacian((12, 12))
    part, p = W.box_partition((12, 12), (2, 2))
    h = pkg.DDLR(A, part, p, variant=variant, rank_k=44, factor=1, lowrank_method=1, rand_oversample=0,
                 rand_power=0)
    assert h.info()["s"] == 44
    x, info = h.pcg(torch.tensor(W.rhs(A[0], 0), device="cuda"), tol=1e-10)
    assert info[0]["status"] == "OK" and info[0]["its"] == 1
    h.close()


def test_mixed_precision_chebyshev_and_batched():
    """The randomized build under the other options: mixed precision with
    BF16 U_k, the Chebyshev C_a solve, batched right-hand sides."""
    A = W.laplacian((24, 24, 24))
    part, p = W.box_partition((24, 24, 24), (3, 2, 2))
    S = W.to_scipy(A)
    B = np.asfortranarray(np.stack([W.rhs(A[0], s) for s in range(3)], axis=1))
    for kw in (dict(precision=1, uk_bf16=1), dict(c_solver=1), dict(max_nrhs=3)):
        h = pkg.DDLR(A, part, p, rank_k=16, lowrank_method=1, c_order=1, b_order=1, **kw)
        X, infos = h.pcg(B, tol=1e-8)
        for j in range(3):
            assert infos[j]["status"] == "OK"
            assert np.linalg.norm(B[:, j] - S @ X[:, j]) <= 1e-8 * (1 + 1e-6) * np.linalg.norm(B[:, j])
        h.close()


def test_randomized_rejects_bad_options_and_rank_raise():
    A = W.laplacian((16, 16))
    part, p = W.box_partition((16, 16), (2, 2))
    for kw in (dict(lowrank_method=2), dict(lowrank_method=1, rand_oversample=60),
               dict(lowrank_method=1, rand_power=-1)):
        with pytest.raises(pkg.DdlrError, match="INVALID"):
            pkg.DDLR(A, part, p, rank_k=8, **kw)
    h = pkg.DDLR(A, part, p, rank_k=4, lowrank_method=1)
    with pytest.raises(pkg.DdlrError, match="INVALID"):
        h.increase_rank(8)
    _, info = h.pcg(torch.tensor(W.rhs(A[0], 0), device="cuda"), tol=1e-8)
    assert info[0]["status"] == "OK"
    h.close()
