"""GPU: the tensor-core forms (mma.sync, TF32 operands split in two for FP32
accuracy, FP32 accumulation) of the multi-right-hand-side U_k products of the
mixed-precision batched path, against the scalar CUDA-core forms
(DDLR_BATCH_TC=0) and against the FP64 oracle.

Both forms compute the same FP32 products; only the summation order inside
the tensor-core instruction differs, so the batched applies agree to FP32
rounding (1e-5 relative).  Against the FP64 oracle the FP32 / BF16 apply keeps
its usual error.  Tile edges are covered: k = 3 and 40 (partial 16-row
tiles), R = 2, 5, 13 (partial 8-column tiles), up to R = 64 and k = 64.
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


@pytest.fixture(scope="module", autouse=True)
def _built():
    pkg.build()
    O.build()


def _block(n, seeds):
    return np.asfortranarray(np.stack([W.rhs(n, s) for s in seeds], axis=1))


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


CASES = [(1, 3, 5, 1), (1, 24, 32, 0), (1, 40, 13, 1), (2, 8, 2, 0), (2, 16, 64, 1), (1, 64, 16, 0)]


@pytest.mark.parametrize("variant,k,R,bf16", CASES)
def test_tc_products_match_scalar_and_oracle(variant, k, R, bf16, monkeypatch):
    A = W.laplacian((24, 20, 18))
    part, p = W.box_partition((24, 20, 18), (3, 2, 2))
    X = _block(A[0], range(40, 40 + R))
    kw = dict(variant=variant, rank_k=k, c_order=1, b_order=1, precision=1, uk_bf16=bf16, max_nrhs=R)
    out = {}
    for tc in ("1", "0"):
        monkeypatch.setenv("DDLR_BATCH_TC", tc)
        h = pkg.DDLR(A, part, p, **kw)
        h.reset_counters()
        out[tc] = h.apply(X)
        fams = {f for f, v in h.counters()["families"].items() if v["launches"] > 0}
        assert "utx_mr" in fams
        h.close()
    assert _rel(out["1"], out["0"]) < 1e-5
    # against the FP64 oracle, with the oracle's low-rank data injected
    orc = O.Oracle(A, part, p, variant=variant, k=k, c_order=1, b_order=1)
    Uo, lam, Hk, _ = orc.lowrank_original_order()
    hm = pkg.DDLR(A, part, p, **dict(kw))
    hm.set_lowrank(Uo, lam, orc.theta, Hk)
    Ym = hm.apply(X)
    for j in (0, R - 1):
        yo = orc.apply(np.ascontiguousarray(X[:, j]))
        # FP32 factors and sweeps (BF16 U_k: 2^-8 relative on the low-rank term)
        assert _rel(Ym[:, j], yo) < (2e-2 if bf16 else 1e-4)
    hm.close()


def test_tc_batched_pcg_matches_scalar(monkeypatch):
    """A batched mixed-precision PCG with the tensor-core products converges
    like the scalar form: the same iterations within two, solutions within
    1e-6, true residuals <= tol."""
    A = W.jump_coefficient_fv(32, 8, 0)
    part, p = W.random_cut_partition(32, 3, 0, 6, 16)
    B = _block(A[0], range(0, 12))
    res = {}
    for tc in ("1", "0"):
        monkeypatch.setenv("DDLR_BATCH_TC", tc)
        h = pkg.DDLR(A, part, p, variant=1, rank_k=12, c_order=1, b_order=1, scale_diag=1, precision=1,
                     uk_bf16=0, max_nrhs=12)
        res[tc] = h.pcg(B, tol=1e-8, maxit=2000)
        h.close()
    (X1, i1), (X0, i0) = res["1"], res["0"]
    for j in range(B.shape[1]):
        assert i1[j]["status"] == "OK" and i1[j]["relres"] <= 1e-8
        assert abs(i1[j]["its"] - i0[j]["its"]) <= 2
        assert _rel(X1[:, j], X0[:, j]) < 1e-6
