"""GPU: the batched (multi right-hand side) path against the single-RHS path
and against the oracle; batch invariance (a column's result does not depend on
the other columns of its batch)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle as O  # noqa: E402
import paper_1505_04341_gb300 as pkg  # noqa: E402
import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu


def _block(n, seeds):
    return np.asfortranarray(np.stack([W.rhs(n, s) for s in seeds], axis=1))


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("variant", [1, 2])
@pytest.mark.parametrize("b_order", [1, 0])
def test_batched_apply_matches_oracle(variant, b_order):
    A = W.laplacian((24, 20, 18))
    part, p = W.box_partition((24, 20, 18), (3, 2, 2))
    k = 8
    h = pkg.DDLR(A, part, p, variant=variant, rank_k=k, c_order=1, b_order=b_order)
    orc = O.Oracle(A, part, p, variant=variant, k=k, c_order=1, b_order=b_order)
    U, lam, Hk, _ = orc.lowrank_original_order()
    h.set_lowrank(U, lam, orc.theta, Hk)
    n = A[0]
    X = _block(n, range(11, 16))
    Y = h.apply(X)                       # host block, batched path
    Yd = h.apply(torch.tensor(X, device="cuda").T.contiguous().T).cpu().numpy()
    assert np.array_equal(Y, Yd)
    for j in range(X.shape[1]):
        assert _rel(Y[:, j], orc.apply(np.ascontiguousarray(X[:, j]))) < 1e-12
    h.close()


@pytest.mark.parametrize("precision", [0, 1])
def test_batched_pcg_matches_single(precision):
    w = W.workload("lap3d_64_b4")
    A, part, p = w["A"], w["part"], w["p"]
    n = A[0]
    h = pkg.DDLR(A, part, p, variant=1, rank_k=16, c_order=1, b_order=1, precision=precision,
                 uk_bf16=precision)
    B = _block(n, range(0, 6))
    X, infos = h.pcg(B, tol=1e-8)
    for j in range(B.shape[1]):
        xs, inf1 = h.pcg(np.ascontiguousarray(B[:, j]), tol=1e-8)
        assert infos[j]["status"] == "OK" and infos[j]["relres"] <= 1e-8
        assert abs(infos[j]["its"] - inf1[0]["its"]) <= 1
        assert _rel(X[:, j], xs) < 1e-6
    info = h.info()
    assert info["batch_block_chunks"] > 0 and info["batch_block_elem"] > 0
    h.close()


def test_batch_invariance_bitwise():
    """The same right-hand side solved inside two different batches gives the
    same bits (fixed row partition and order in every reduction)."""
    A = W.jump_coefficient_fv(32, 8, 0)
    part, p = W.random_cut_partition(32, 3, 0, 6, 16)
    n = A[0]
    h = pkg.DDLR(A, part, p, variant=1, rank_k=8, c_order=1, b_order=1, scale_diag=1,
                 precision=1, uk_bf16=1)
    b0 = W.rhs(n, 100)
    X1, i1 = h.pcg(np.asfortranarray(np.stack([b0, W.rhs(n, 1), W.rhs(n, 2)], 1)), tol=1e-8)
    X2, i2 = h.pcg(np.asfortranarray(np.stack([W.rhs(n, 7), b0], 1)), tol=1e-8)
    assert i1[0]["its"] == i2[1]["its"] and i1[0]["status"] == "OK"
    assert np.array_equal(X1[:, 0], X2[:, 1])
    h.close()


def test_batched_jump_coefficients_mixed_oracle():
    """Jump coefficients with diagonal scaling, uneven random-cut boxes, FP32
    inner / FP64 outer, 8 right-hand sides: each column converges to 1e-8 and
    agrees with the FP64 oracle solution."""
    A = W.jump_coefficient_fv(40, 8, 0)
    part, p = W.random_cut_partition(40, 3, 0, 8, 20)
    n = A[0]
    k = 12
    h = pkg.DDLR(A, part, p, variant=1, rank_k=k, c_order=1, b_order=1, scale_diag=1,
                 precision=1, uk_bf16=1)
    orc = O.Oracle(A, part, p, variant=1, k=k, c_order=1, b_order=1, scale_diag=1)
    B = _block(n, range(20, 28))
    X, infos = h.pcg(B, tol=1e-8)
    for j in (0, 7):
        xo, its_o, rel_o, st = orc.pcg(np.ascontiguousarray(B[:, j]), 1e-8)
        assert infos[j]["status"] == "OK" and infos[j]["relres"] <= 1e-8
        assert abs(infos[j]["its"] - its_o) <= max(3, its_o // 10)
        assert _rel(X[:, j], xo) < 1e-6
    h.close()


@pytest.mark.parametrize("precision", [1, 0])
def test_batch_invariance_across_kernel_forms(precision):
    """Widths that are a multiple of the 16-byte vector (4 FP32 / 2 FP64
    columns) take the vector form of the batched level solve, others the
    scalar form; a column gives the same bits in either."""
    A = W.jump_coefficient_fv(24, 8, 0)
    part, p = W.random_cut_partition(24, 3, 0, 6, 12)
    n = A[0]
    h = pkg.DDLR(A, part, p, variant=1, rank_k=8, c_order=1, b_order=1, scale_diag=1,
                 precision=precision, uk_bf16=precision)
    b0 = W.rhs(n, 100)
    outs = []
    for width in (4, 5, 8, 3):
        B = np.asfortranarray(np.stack([b0] + [W.rhs(n, 10 + j) for j in range(width - 1)], 1))
        X, inf = h.pcg(B, tol=1e-8)
        assert inf[0]["status"] == "OK"
        outs.append((X[:, 0].copy(), inf[0]["its"]))
    for x, its in outs[1:]:
        assert its == outs[0][1] and np.array_equal(x, outs[0][0])
    h.close()
