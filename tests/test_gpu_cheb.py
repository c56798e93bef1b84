"""GPU parity of the Chebyshev solve with C_a (c_solver=1, Sec. 4.3) against
the FP64 CPU oracle, through the C ABI.

Tolerances as for the factored C_a: A0^-1 x and M^-1 x within 1e-12 relative
with the oracle's spectrum interval (and low-rank data, for M^-1) injected;
the interval estimated on the GPU within 1e-10 of the oracle's (same start
vector, same steps); PCG iteration counts within +-1 and the true relative
residual <= tol.
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

# (A, part, p, factor, orders): orders bit 0 = C_a / D_a multicolour, bit 1 =
# interior blocks multicolour.  Natural orders take the deep-factor path
# (CTA per interior block, C_a branch on a second stream), multicolour ones
# the all-blocks level sweeps.
PROBLEMS = {
    "2d_12x12_exact": lambda: (W.laplacian((12, 12)),) + W.box_partition((12, 12), (2, 2)) + (1, 0),
    "3d_24_ic0_natural": lambda: (W.laplacian((24, 24, 24)),) + W.box_partition((24, 24, 24), (3, 2, 2)) + (0, 0),
    "3d_20_ic0_c_multicolour": lambda: (W.laplacian((20, 20, 20)),) + W.box_partition((20, 20, 20), (2, 2, 2)) + (0, 1),
    "3d_33x17x21_ragged": lambda: (W.laplacian((33, 17, 21)),) + W.box_partition((33, 17, 21), (3, 2, 2)) + (0, 0),
    "3d_24_multicolour_all": lambda: (W.laplacian((24, 24, 24)),) + W.box_partition((24, 24, 24), (3, 2, 2)) + (0, 3),
    "jump_32_multicolour_all": lambda: (W.jump_coefficient_fv(32, 8, 0),) + W.random_cut_partition(32, 3, 0, 6, 16) + (0, 3),
}


def _orders(o):
    return dict(c_order=o & 1, b_order=o >> 1)


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.fixture(scope="module", autouse=True)
def _built():
    pkg.build()
    O.build()


def _pair(name, steps=5, **kw):
    A, part, p, factor, orders = PROBLEMS[name]()
    scale = 1 if name.startswith("jump") else 0
    opts = dict(factor=factor, scale_diag=scale, **_orders(orders), **kw)
    h = pkg.DDLR(A, part, p, c_solver=1, cheb_steps=steps, **opts)
    orc = O.Oracle(A, part, p, c_solver=1, cheb_steps=steps, factor=factor, scale_diag=scale,
                   **_orders(orders), **{("k" if a == "rank_k" else a): v for a, v in kw.items()})
    return A, h, orc


@pytest.mark.parametrize("steps", [1, 2, 5])
@pytest.mark.parametrize("name", list(PROBLEMS))
def test_a0_solve_parity_and_interval(name, steps):
    A, h, orc = _pair(name, steps, rank_k=4)
    inf = h.info()
    assert inf["persistent"] == 0
    lo, hi = orc.cheb_bounds
    assert abs(inf["cheb_lo"] - lo) <= 1e-10 * lo and abs(inf["cheb_hi"] - hi) <= 1e-10 * hi
    assert inf["cheb_lanczos_steps"] == 20
    h.set_cheb_bounds(lo, hi)
    n = A[0]
    for seed in (1, 2):
        x = W.rhs(n, seed)
        y = h.a0_solve(torch.tensor(x, device="cuda")).cpu().numpy()
        assert _rel(y, orc.a0_solve(x)) < 1e-12
    # host-pointer path gives the same bits as the device path
    x = W.rhs(n, 3)
    assert np.array_equal(h.a0_solve(x), h.a0_solve(torch.tensor(x, device="cuda")).cpu().numpy())
    h.close()


@pytest.mark.parametrize("variant", [1, 2])
@pytest.mark.parametrize("name", ["3d_24_ic0_natural", "3d_20_ic0_c_multicolour", "jump_32_multicolour_all"])
def test_apply_parity_injected(name, variant):
    A, h, orc = _pair(name, variant=variant, rank_k=8)
    h.set_cheb_bounds(*orc.cheb_bounds)
    U, lam, Hk, rows = orc.lowrank_original_order()
    h.set_lowrank(U, lam, orc.theta, Hk)
    n = A[0]
    X = np.asfortranarray(np.stack([W.rhs(n, s) for s in (7, 8, 9)], axis=1))
    Y = h.apply(X)                       # batched path (3 right-hand sides)
    for j in range(3):
        ref = orc.apply(X[:, j])
        assert _rel(Y[:, j], ref) < 1e-12
        y1 = h.apply(torch.tensor(X[:, j], device="cuda")).cpu().numpy()
        assert _rel(y1, ref) < 1e-12
    h.close()


@pytest.mark.parametrize("variant", [1, 2])
@pytest.mark.parametrize("name", ["3d_24_ic0_natural", "3d_24_multicolour_all", "3d_33x17x21_ragged"])
def test_pcg_iterations_match_oracle(name, variant):
    """Each side with its own setup (GPU Lanczos, GPU interval)."""
    A, h, orc = _pair(name, variant=variant, rank_k=8)
    b = W.rhs(A[0], 0)
    x, info = h.pcg(torch.tensor(b, device="cuda"), tol=1e-8)
    _, its_o, rel_o, st_o = orc.pcg(b, 1e-8)
    assert st_o == "OK" and info[0]["status"] == "OK"
    assert info[0]["relres"] <= 1e-8 and abs(info[0]["its"] - its_o) <= 1
    S = W.to_scipy(A)
    xn = x.cpu().numpy()
    assert np.linalg.norm(b - S @ xn) <= 1e-8 * (1 + 1e-6) * np.linalg.norm(b)
    h.close()


def test_pcg_follows_a_new_interval():
    """The coefficients live in a device table: a PCG solve (captured CUDA
    graph) after set_cheb_bounds uses the new interval, as the oracle does."""
    A, h, orc = _pair("3d_24_multicolour_all", rank_k=8)
    b = W.rhs(A[0], 1)
    bd = torch.tensor(b, device="cuda")
    h.pcg(bd, tol=1e-8)
    lo, hi = orc.cheb_bounds
    for lo2, hi2 in ((0.5 * lo, 1.5 * hi), (lo, hi)):
        h.set_cheb_bounds(lo2, hi2)
        orc.set_cheb_bounds(lo2, hi2)
        x = W.rhs(A[0], 4)
        assert _rel(h.a0_solve(torch.tensor(x, device="cuda")).cpu().numpy(), orc.a0_solve(x)) < 1e-12
        _, info = h.pcg(bd, tol=1e-8)
        _, its_o, _, st = orc.pcg(b, 1e-8)
        assert info[0]["status"] == "OK" and abs(info[0]["its"] - its_o) <= 1
    h.close()


def test_two_node_interface_closed_form():
    """1-D Laplacian tridiag(-1, 2, -1), n = 4, parts {0,1 | 2,3}, a = 1: the
    interface nodes 1 and 2 give C_a = [[3, -1], [-1, 3]] and D_a = 3 I, so
    D_a^-1 C_a has eigenvalues 2/3 and 4/3.  The estimate meets the invariant
    subspace at step 2 and returns that interval; one Chebyshev step (centre
    1) is x = D_a^-1 y = y / 3."""
    A = W.laplacian((4,))
    part = np.array([0, 0, 1, 1], dtype=np.int32)
    for t in (1, 3):
        h = pkg.DDLR(A, part, 2, rank_k=1, factor=1, c_solver=1, cheb_steps=t)
        orc = O.Oracle(A, part, 2, k=1, factor=1, c_solver=1, cheb_steps=t)
        inf = h.info()
        assert inf["cheb_lanczos_steps"] == 2
        assert abs(inf["cheb_lo"] - 2 / 3) < 1e-13 and abs(inf["cheb_hi"] - 4 / 3) < 1e-13
        x = np.array([0.0, 1.0, -2.0, 0.0])
        y = h.a0_solve(torch.tensor(x, device="cuda")).cpu().numpy()
        assert _rel(y, orc.a0_solve(x)) < 1e-12
        if t == 1:
            np.testing.assert_allclose(y, [0.0, 1 / 3, -2 / 3, 0.0], rtol=0, atol=1e-15)
        h.close()


def test_mixed_precision_and_batched_solve():
    A = W.laplacian((24, 24, 24))
    part, p = W.box_partition((24, 24, 24), (3, 2, 2))
    n = A[0]
    h = pkg.DDLR(A, part, p, rank_k=8, c_solver=1, precision=1, uk_bf16=1, max_nrhs=4, c_order=1, b_order=1)
    h64 = pkg.DDLR(A, part, p, rank_k=8, c_solver=1, max_nrhs=4, c_order=1, b_order=1)
    B = np.asfortranarray(np.stack([W.rhs(n, s) for s in range(4)], axis=1))
    S = W.to_scipy(A)
    for hh in (h, h64):
        X, infos = hh.pcg(B, tol=1e-8)
        for j in range(4):
            assert infos[j]["status"] == "OK" and infos[j]["relres"] <= 1e-8
            assert np.linalg.norm(B[:, j] - S @ X[:, j]) <= 1e-8 * (1 + 1e-6) * np.linalg.norm(B[:, j])
        x0, i0 = hh.pcg(np.ascontiguousarray(B[:, 0]), tol=1e-8)
        assert abs(i0[0]["its"] - infos[0]["its"]) <= 1
    h.close()
    h64.close()


def test_bad_chebyshev_options_and_bounds():
    A = W.laplacian((16, 16))
    part, p = W.box_partition((16, 16), (2, 2))
    for kw in (dict(c_solver=3), dict(c_solver=1, cheb_steps=0), dict(c_solver=1, cheb_steps=65),
               dict(c_solver=1, cheb_lanczos=0)):
        with pytest.raises(pkg.DdlrError, match="INVALID"):
            pkg.DDLR(A, part, p, rank_k=4, **kw)
    h0 = pkg.DDLR(A, part, p, rank_k=4)
    with pytest.raises(pkg.DdlrError, match="INVALID"):
        h0.set_cheb_bounds(0.5, 1.5)
    h0.close()
    h = pkg.DDLR(A, part, p, rank_k=4, c_solver=1)
    for lo, hi in ((0.0, 1.0), (1.0, 0.5), (-1.0, 2.0)):
        with pytest.raises(pkg.DdlrError, match="INVALID"):
            h.set_cheb_bounds(lo, hi)
    x = torch.tensor(W.rhs(A[0], 0), device="cuda")
    _, info = h.pcg(x, tol=1e-8)
    assert info[0]["status"] == "OK"
    h.close()
