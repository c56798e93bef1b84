"""The persistent whole-solve kernels against the FP64 oracle and against the
kernel-per-phase path.

With shallow local factors (greedy multicolour orders of the interior blocks
and of C_a) a PCG solve runs as one cooperative launch and so does the whole
Lanczos process, convergence tests included.  DDLR_PERSIST=0 keeps the path
of one kernel per phase.  Both must meet the same bars: PCG iterations within
+-1 of the oracle's, the true relative residual <= tol, Ritz values within
1e-8 of the oracle's, the number of Lanczos steps chosen by eq. converge equal
to the oracle's.
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


def _handle(monkeypatch, persist, A, part, p, **kw):
    monkeypatch.setenv("DDLR_PERSIST", persist)
    return pkg.DDLR(A, part, p, **kw)


def _families(h):
    return {k for k, v in h.counters()["families"].items() if v["launches"] > 0}


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


CASES = {
    "lap3d_32_v1": (lambda: (W.laplacian((32, 32, 32)),) + W.box_partition((32, 32, 32), (2, 2, 2)), 1, 8, 0),
    "lap3d_32_v2": (lambda: (W.laplacian((32, 32, 32)),) + W.box_partition((32, 32, 32), (2, 2, 2)), 2, 8, 0),
    "jump_32_scaled_v1": (lambda: (W.jump_coefficient_fv(32, 8, 0),) + W.random_cut_partition(32, 3, 0, 6, 16),
                          1, 8, 1),
    "jump_32_scaled_v2": (lambda: (W.jump_coefficient_fv(32, 8, 0),) + W.random_cut_partition(32, 3, 0, 6, 16),
                          2, 8, 1),
    "lap3d_33x17x21_ragged_v1": (lambda: (W.laplacian((33, 17, 21)),) + W.box_partition((33, 17, 21), (3, 2, 2)),
                                 1, 6, 0),
}


@pytest.mark.parametrize("persist", ["1", "0"])
@pytest.mark.parametrize("case", list(CASES))
def test_pcg_matches_oracle(case, persist, monkeypatch):
    build, variant, k, sd = CASES[case]
    A, part, p = build()
    h = _handle(monkeypatch, persist, A, part, p, variant=variant, rank_k=k, factor=0, scale_diag=sd, **MC)
    orc = O.Oracle(A, part, p, variant=variant, k=k, factor=0, scale_diag=sd, **MC)
    assert h.info()["lanczos_steps"] == orc.msteps
    np.testing.assert_allclose(h.ritz()[:k + 1], orc.ritz[:k + 1], rtol=1e-8)
    b = W.rhs(A[0], 0)
    h.reset_counters()
    x, info = h.pcg(torch.tensor(b, device="cuda"), tol=1e-8)
    xo, its_o, _, st = orc.pcg(b, 1e-8)
    assert st == "OK"
    assert info[0]["status"] == "OK" and info[0]["relres"] <= 1e-8
    assert abs(info[0]["its"] - its_o) <= 1, (info, its_o)
    assert _rel(x.cpu().numpy(), xo) < 1e-6
    fam = _families(h)
    assert ("pcg_persist" in fam) == (persist == "1"), fam
    h.close()


@pytest.mark.parametrize("variant", [1, 2])
def test_lanczos_persistent_equals_phase_path(variant, monkeypatch):
    """Same start vector and forced step count: the Ritz values of the two
    paths agree with each other and with the oracle's; U_k is orthonormal."""
    A = W.laplacian((40, 30))
    part, p = W.box_partition((40, 30), (3, 2))
    k, m = 6, 40
    kw = dict(variant=variant, rank_k=k, factor=0, lanczos_max=m, lanczos_check=0, seed=3, **MC)
    hp = _handle(monkeypatch, "1", A, part, p, **kw)
    hk = _handle(monkeypatch, "0", A, part, p, **kw)
    orc = O.Oracle(A, part, p, variant=variant, k=k, factor=0, lanczos_max=m, lanczos_check=0, seed=3, **MC)
    rp, rk, ro = hp.ritz(), hk.ritz(), orc.ritz
    assert len(rp) == len(rk) == len(ro) == m
    np.testing.assert_allclose(rp[:k + 1], ro[:k + 1], rtol=1e-8)
    np.testing.assert_allclose(rp, rk, rtol=1e-9, atol=1e-12 * np.abs(rk).max())
    if variant == 1:
        Up = hp.lowrank()[0]
        np.testing.assert_allclose(Up.T @ Up, np.eye(k), atol=1e-10)
    hp.close()
    hk.close()


@pytest.mark.parametrize("persist", ["1", "0"])
@pytest.mark.parametrize("variant", [1, 2])
def test_breakdown_restart_full_rank(variant, persist, monkeypatch):
    """k = s: the Krylov space is exhausted inside the Lanczos process (a
    breakdown and a restart).  With exact local factors M^-1 = A^-1 in exact
    arithmetic (eq. split3): DDLR-1 takes one PCG iteration; both variants
    match the oracle's count within one and solve to 1e-10."""
    A = W.laplacian((16, 16))
    part, p = W.box_partition((16, 16), (2, 2))
    s = O.Oracle(A, part, p, variant=variant, k=2, factor=1, **MC).s
    orc = O.Oracle(A, part, p, variant=variant, k=s, factor=1, **MC)
    h = _handle(monkeypatch, persist, A, part, p, variant=variant, rank_k=s, factor=1, **MC)
    assert h.info()["lanczos_steps"] == orc.msteps
    b = W.rhs(A[0], 0)
    x, info = h.pcg(torch.tensor(b, device="cuda"), tol=1e-10)
    _, its_o, _, st = orc.pcg(b, 1e-10)
    assert st == "OK" and info[0]["relres"] < 1e-10
    assert abs(info[0]["its"] - its_o) <= 1, (info, its_o)
    if variant == 1:
        assert info[0]["its"] == 1
    assert _rel(x.cpu().numpy(), np.linalg.solve(W.to_dense(A), b)) < 1e-8
    h.close()


def test_convergence_rule_persistent(monkeypatch):
    A = W.laplacian((64, 64))
    part, p = W.box_partition((64, 64), (2, 2))
    h = _handle(monkeypatch, "1", A, part, p, variant=1, rank_k=8, factor=1, **MC)
    orc = O.Oracle(A, part, p, variant=1, k=8, factor=1, **MC)
    assert h.info()["lanczos_steps"] == orc.msteps
    np.testing.assert_allclose(h.ritz()[:8], orc.ritz[:8], rtol=1e-8)
    h.close()


def test_pcg_maxit_and_zero_rhs(monkeypatch):
    """NOCONV after maxit iterations, and b = 0 gives x = 0 in no iteration."""
    A = W.laplacian((32, 32, 32))
    part, p = W.box_partition((32, 32, 32), (2, 2, 2))
    h = _handle(monkeypatch, "1", A, part, p, variant=1, rank_k=4, factor=0, **MC)
    b = torch.tensor(W.rhs(A[0], 1), device="cuda")
    x, info = h.pcg(b, tol=1e-14, maxit=3, check=False)
    assert info[0]["status"] == "NOCONV" and info[0]["its"] == 3
    x0, info0 = h.pcg(torch.zeros_like(b), tol=1e-8)
    assert info0[0]["its"] == 0 and float(x0.abs().max()) == 0.0
    h.close()


@pytest.mark.parametrize("persist", ["1", "0"])
@pytest.mark.parametrize("bf16", [0, 1])
@pytest.mark.parametrize("case", ["lap3d_32_v1", "lap3d_32_v2", "jump_32_scaled_v1"])
def test_mixed_precision_pcg(case, bf16, persist, monkeypatch):
    """FP32 factors and solves, U_k in FP32 or BF16, flexible CG in FP64: the
    true relative residual reaches tol and the iteration count stays within
    max(3, 10%) of the FP64 oracle's."""
    build, variant, k, sd = CASES[case]
    A, part, p = build()
    h = _handle(monkeypatch, persist, A, part, p, variant=variant, rank_k=k, factor=0, scale_diag=sd,
                precision=1, uk_bf16=bf16, **MC)
    orc = O.Oracle(A, part, p, variant=variant, k=k, factor=0, scale_diag=sd, **MC)
    b = W.rhs(A[0], 0)
    h.reset_counters()
    x, info = h.pcg(torch.tensor(b, device="cuda"), tol=1e-8)
    xo, its_o, _, st = orc.pcg(b, 1e-8)
    assert st == "OK"
    assert info[0]["status"] == "OK" and info[0]["relres"] <= 1e-8
    assert abs(info[0]["its"] - its_o) <= max(3, its_o // 10), (info, its_o)
    assert _rel(x.cpu().numpy(), xo) < 1e-6
    assert ("pcg_persist" in _families(h)) == (persist == "1")
    assert (h.info()["persistent"] & 1) == (persist == "1")
    h.close()


def test_refused_cooperative_launch_falls_back(monkeypatch):
    """A refused cooperative launch (faked on the host) leaves the handle on
    the per-phase kernels: setup and PCG still meet the oracle bars."""
    build, variant, k, sd = CASES["lap3d_32_v1"]
    A, part, p = build()
    monkeypatch.setenv("DDLR_FAKE_COOP_REFUSAL", "1")
    h = _handle(monkeypatch, "1", A, part, p, variant=variant, rank_k=k, factor=0, **MC)
    assert h.info()["persistent"] == 0
    orc = O.Oracle(A, part, p, variant=variant, k=k, factor=0, **MC)
    assert h.info()["lanczos_steps"] == orc.msteps
    b = W.rhs(A[0], 0)
    x, info = h.pcg(torch.tensor(b, device="cuda"), tol=1e-8)
    _, its_o, _, _ = orc.pcg(b, 1e-8)
    assert info[0]["status"] == "OK" and info[0]["relres"] <= 1e-8
    assert abs(info[0]["its"] - its_o) <= 1
    h.close()


@pytest.mark.parametrize("persist", ["1", "0"])
@pytest.mark.parametrize("variant", [1, 2])
@pytest.mark.parametrize("reorth", [0, 1])
def test_reorthogonalisation_passes(reorth, variant, persist, monkeypatch):
    """Full reorthogonalisation with the second Gram-Schmidt pass on
    cancellation (lanczos_reorth 0) or every step (1): the GPU takes the same
    passes as the oracle, the same steps, Ritz values within 1e-8, an
    orthonormal U_k; near full rank the second pass is taken."""
    A = W.laplacian((32, 32, 32))
    part, p = W.box_partition((32, 32, 32), (2, 2, 2))
    kw = dict(variant=variant, factor=0, lanczos_reorth=reorth, **MC)
    h = _handle(monkeypatch, persist, A, part, p, rank_k=8, **kw)
    orc = O.Oracle(A, part, p, k=8, **kw)
    inf = h.info()
    assert inf["lanczos_steps"] == orc.msteps
    np.testing.assert_allclose(h.ritz()[:9], orc.ritz[:9], rtol=1e-8)
    assert inf["reorth_passes"] == orc.reorth_passes
    assert inf["reorth_passes"] == (2 if reorth else 1) * orc.msteps
    # the persistent kernel forms the corrections in FP32 where their error
    # bound is below FP64 rounding of w; the per-phase path keeps FP64
    if persist == "1":
        assert 0 < inf["reorth_fp32"] <= inf["reorth_passes"]
    else:
        assert inf["reorth_fp32"] == 0
    if variant == 1:
        U = h.lowrank()[0]
        np.testing.assert_allclose(U.T @ U, np.eye(8), atol=1e-10)
    h.close()
    # exhausting the Krylov space: cancellation, so the criterion takes the
    # second pass too (exact 2-D factors, k = s)
    A2 = W.laplacian((16, 16))
    part2, p2 = W.box_partition((16, 16), (2, 2))
    s = O.Oracle(A2, part2, p2, variant=variant, k=2, factor=1, **MC).s
    kw2 = dict(variant=variant, factor=1, lanczos_reorth=reorth, **MC)
    h2 = _handle(monkeypatch, persist, A2, part2, p2, rank_k=s, **kw2)
    orc2 = O.Oracle(A2, part2, p2, k=s, **kw2)
    assert h2.info()["lanczos_steps"] == orc2.msteps
    assert h2.info()["reorth_passes"] == orc2.reorth_passes > orc2.msteps
    h2.close()
