"""GPU parity: the CUDA path through the C ABI against the FP64 CPU oracle.

Tolerances (FP64 path): A0^-1 x, local factors and M^-1 x (with the oracle's
low-rank data injected, since Lanczos vectors of clustered eigenvalues are not
unique) within 1e-12 relative; Lanczos Ritz values of converged pairs within
1e-8 relative; PCG iteration counts within +-1 and the true relative residual
<= tol.
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
    "2d_64x64_C1_exact": lambda: (W.laplacian((64, 64)),) + W.box_partition((64, 64), (2, 2)) + (1, 0),
    "3d_24_ic0_natural": lambda: (W.laplacian((24, 24, 24)),) + W.box_partition((24, 24, 24), (3, 2, 2)) + (0, 0),
    "3d_20_ic0_multicolour": lambda: (W.laplacian((20, 20, 20)),) + W.box_partition((20, 20, 20), (2, 2, 2)) + (0, 1),
    "3d_33x17x21_ragged": lambda: (W.laplacian((33, 17, 21)),) + W.box_partition((33, 17, 21), (3, 2, 2)) + (0, 0),
    "jump_32_cuts": lambda: (W.jump_coefficient_fv(32, 8, 0),) + W.random_cut_partition(32, 3, 0, 6, 16) + (0, 1),
    "3d_24_ic0_multicolour_all": lambda: (W.laplacian((24, 24, 24)),) + W.box_partition((24, 24, 24), (3, 2, 2)) + (0, 3),
    "jump_32_multicolour_all": lambda: (W.jump_coefficient_fv(32, 8, 0),) + W.random_cut_partition(32, 3, 0, 6, 16) + (0, 3),
}


def _orders(c_order):
    """c_order bit 0: C_a multicolour; bit 1: interior blocks multicolour"""
    return dict(c_order=c_order & 1, b_order=c_order >> 1)


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.fixture(scope="module", autouse=True)
def _built():
    pkg.build()
    O.build()


@pytest.mark.parametrize("kind", ["sf", "tma", "plain"])
@pytest.mark.parametrize("name", list(PROBLEMS))
def test_a0_solve_and_factor_parity(name, kind, monkeypatch):
    """Every interior-solve kernel (synchronisation-free, TMA-pipelined level
    schedule, plain level schedule) against the oracle."""
    A, part, p, factor, c_order = PROBLEMS[name]()
    k = 4
    monkeypatch.setenv("DDLR_SOLVE", kind)
    h = pkg.DDLR(A, part, p, rank_k=k, factor=factor, **_orders(c_order))
    orc = O.Oracle(A, part, p, k=k, factor=factor, **_orders(c_order))
    n = A[0]
    for seed in (1, 2):
        x = W.rhs(n, seed)
        y = h.a0_solve(torch.tensor(x, device="cuda")).cpu().numpy()
        assert _rel(y, orc.a0_solve(x)) < 1e-12
    # host-pointer path gives the same bits as the device path
    x = W.rhs(n, 3)
    yh = h.a0_solve(x)
    yd = h.a0_solve(torch.tensor(x, device="cuda")).cpu().numpy()
    assert np.array_equal(yh, yd)
    r, c, v = h.factor_coo()
    ro, co, vo = orc.factor_coo()
    assert len(r) == len(ro)
    ia = np.lexsort((c, r))
    ib = np.lexsort((co, ro))
    assert np.array_equal(r[ia], ro[ib]) and np.array_equal(c[ia], co[ib])
    assert np.abs(v[ia] - vo[ib]).max() <= 1e-12 * np.abs(vo).max()
    h.close()


@pytest.mark.parametrize("rows", ["1", "2", "4"])
@pytest.mark.parametrize("name", ["3d_20_ic0_multicolour", "3d_24_ic0_multicolour_all", "jump_32_multicolour_all"])
def test_level_chunk_solve_rows_per_thread(name, rows, monkeypatch):
    """The level-chunk solve with 1, 2 or 4 rows per thread (all blocks of a
    level per launch) against the oracle, FP64 and FP32; the FP64 result
    does not depend on the rows per thread."""
    A, part, p, factor, c_order = PROBLEMS[name]()
    monkeypatch.setenv("DDLR_CHUNK_ROWS", rows)
    monkeypatch.setenv("DDLR_PERSIST", "0")
    orc = O.Oracle(A, part, p, k=4, factor=factor, **_orders(c_order))
    x = W.rhs(A[0], 5)
    ref = orc.a0_solve(x)
    for precision, tol in ((0, 1e-12), (1, 1e-4)):
        h = pkg.DDLR(A, part, p, rank_k=4, factor=factor, precision=precision, **_orders(c_order))
        y = h.a0_solve(torch.tensor(x, device="cuda")).cpu().numpy()
        assert _rel(y, ref) < tol, (precision, _rel(y, ref))
        if precision == 0:
            monkeypatch.setenv("DDLR_CHUNK_ROWS", "1")
            h1 = pkg.DDLR(A, part, p, rank_k=4, factor=factor, **_orders(c_order))
            assert np.array_equal(h1.a0_solve(torch.tensor(x, device="cuda")).cpu().numpy(), y)
            h1.close()
            monkeypatch.setenv("DDLR_CHUNK_ROWS", rows)
        h.close()


@pytest.mark.parametrize("variant", [1, 2])
@pytest.mark.parametrize("name", ["2d_64x64_C1_exact", "3d_24_ic0_natural", "3d_20_ic0_multicolour",
                                  "jump_32_cuts", "3d_24_ic0_multicolour_all"])
def test_apply_parity_injected_lowrank(name, variant):
    A, part, p, factor, c_order = PROBLEMS[name]()
    k = 8
    scale = 1 if name.startswith("jump") else 0
    h = pkg.DDLR(A, part, p, variant=variant, rank_k=k, factor=factor, scale_diag=scale,
                 **_orders(c_order))
    orc = O.Oracle(A, part, p, variant=variant, k=k, factor=factor, scale_diag=scale,
                   **_orders(c_order))
    U, lam, Hk, rows = orc.lowrank_original_order()
    h.set_lowrank(U, lam, orc.theta, Hk)
    n = A[0]
    X = np.asfortranarray(np.stack([W.rhs(n, s) for s in (7, 8, 9)], axis=1))
    Y = h.apply(X)
    for j in range(3):
        assert _rel(Y[:, j], orc.apply(X[:, j])) < 1e-12
    h.close()


@pytest.mark.parametrize("variant", [1, 2])
def test_lanczos_ritz_values_and_orthogonality(variant):
    """Same start vector and the same forced number of steps as the oracle:
    converged Ritz values agree to 1e-8; U_k has orthonormal columns (DDLR-1)."""
    A = W.laplacian((40, 30))
    part, p = W.box_partition((40, 30), (3, 2))
    k, m = 6, 40
    h = pkg.DDLR(A, part, p, variant=variant, rank_k=k, factor=0, lanczos_max=m,
                 lanczos_check=0, seed=3)
    orc = O.Oracle(A, part, p, variant=variant, k=k, factor=0, lanczos_max=m,
                   lanczos_check=0, seed=3)
    rg, ro = h.ritz(), orc.ritz
    assert len(rg) == len(ro) == m
    np.testing.assert_allclose(rg[:k + 1], ro[:k + 1], rtol=1e-8)
    U, lam, theta, Hk = h.lowrank()
    if variant == 1:
        np.testing.assert_allclose(U.T @ U, np.eye(k), atol=1e-10)
        assert abs(theta - orc.theta) < 1e-8 * abs(orc.theta)
    else:
        np.testing.assert_allclose(Hk, Hk.T, atol=1e-12)
    h.close()


def test_lanczos_convergence_rule_matches_oracle():
    A = W.laplacian((64, 64))
    part, p = W.box_partition((64, 64), (2, 2))
    h = pkg.DDLR(A, part, p, variant=1, rank_k=8, factor=1)
    orc = O.Oracle(A, part, p, variant=1, k=8, factor=1)
    assert h.info()["lanczos_steps"] == orc.msteps
    np.testing.assert_allclose(h.ritz()[:8], orc.ritz[:8], rtol=1e-8)
    h.close()


@pytest.mark.parametrize("variant", [1, 2])
def test_full_rank_exact_one_iteration(variant):
    """k = s with exact local factors: M^-1 = A^-1 (eq. split3), PCG takes one
    iteration."""
    A = W.laplacian((16, 16))
    part, p = W.box_partition((16, 16), (2, 2))
    orc = O.Oracle(A, part, p, variant=variant, k=2, factor=1)
    s = orc.s
    h = pkg.DDLR(A, part, p, variant=variant, rank_k=s, factor=1)
    b = W.rhs(A[0], 0)
    x, info = h.pcg(torch.tensor(b, device="cuda"), tol=1e-10)
    assert info[0]["its"] == 1 and info[0]["relres"] < 1e-10
    Ad = W.to_dense(A)
    assert _rel(x.cpu().numpy(), np.linalg.solve(Ad, b)) < 1e-10
    h.close()


CONFIGS = [
    # (workload, variant, k, factor, orders: bit 0 C_a, bit 1 interior multicolour)
    ("lap2d_64_b2x2", 1, 8, 1, 0),
    ("lap3d_64_b4", 1, 16, 0, 0),
    ("lap3d_64_b4", 1, 16, 0, 1),
    ("lap3d_64_b4", 2, 16, 0, 1),
    ("lap3d_64_b4", 1, 32, 0, 1),
    ("lap3d_64_b4", 1, 16, 0, 3),
    ("lap3d_64_b4", 2, 16, 0, 3),
]


@pytest.mark.parametrize("wl,variant,k,factor,c_order", CONFIGS)
def test_pcg_parity(wl, variant, k, factor, c_order):
    w = W.workload(wl)
    A, part, p = w["A"], w["part"], w["p"]
    h = pkg.DDLR(A, part, p, variant=variant, rank_k=k, factor=factor, **_orders(c_order))
    orc = O.Oracle(A, part, p, variant=variant, k=k, factor=factor, **_orders(c_order))
    b = W.rhs(A[0], 0)
    x, info = h.pcg(torch.tensor(b, device="cuda"), tol=1e-8)
    xo, its_o, rel_o, st = orc.pcg(b, 1e-8)
    assert st == "OK"
    assert info[0]["status"] == "OK" and info[0]["relres"] <= 1e-8
    assert abs(info[0]["its"] - its_o) <= 1, (info, its_o)
    assert _rel(x.cpu().numpy(), xo) < 1e-6
    h.close()


def test_mixed_precision_reaches_tol():
    w = W.workload("lap3d_64_b4")
    A, part, p = w["A"], w["part"], w["p"]
    b = W.rhs(A[0], 0)
    orc = O.Oracle(A, part, p, variant=1, k=16, factor=0, c_order=1)
    xo, its_o, _, _ = orc.pcg(b, 1e-8)
    for bf16 in (0, 1):
        h = pkg.DDLR(A, part, p, variant=1, rank_k=16, factor=0, c_order=1, precision=1,
                     uk_bf16=bf16)
        x, info = h.pcg(torch.tensor(b, device="cuda"), tol=1e-8)
        assert info[0]["status"] == "OK" and info[0]["relres"] <= 1e-8
        assert abs(info[0]["its"] - its_o) <= max(3, its_o // 10), (info, its_o)
        assert _rel(x.cpu().numpy(), xo) < 1e-6
        h.close()


def test_error_statuses_without_fault():
    A = W.laplacian((10, 10))
    part, p = W.box_partition((10, 10), (2, 2))
    n, rp, ci, va = A
    va3 = va.copy()
    va3[rp[0]] = -10.0   # indefinite first block: non-positive pivot
    with pytest.raises(pkg.DdlrError) as e:
        pkg.DDLR((n, rp, ci, va3), part, p, rank_k=2)
    assert e.value.status == "BREAKDOWN"
    h = pkg.DDLR(A, part, p, rank_k=2)
    b = W.rhs(n, 0)
    x, info = h.pcg(b, tol=1e-14, maxit=2, check=False)
    assert info[0]["status"] == "NOCONV" and info[0]["its"] == 2
    bn = b.copy()
    bn[5] = np.nan
    x, info = h.pcg(bn, tol=1e-8, check=False)
    assert info[0]["status"] == "NAN"
    h.close()
