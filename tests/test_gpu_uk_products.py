"""The U_k products of the M^-1 apply (U_k^T y, the G^-1 epilogue of
Algorithm 1, and U_k (H_k U_k^T x) of eq. Form2a) for every rank class the
kernels dispatch on: vector loads (a row of U_k is 1..32 loads of 16 bytes),
shared-memory row tiles (FP64, k even, k <= 64) and the scalar kernels
(other k).  FP64 against the oracle with its low-rank data injected (1e-12);
the vector/tiled kernels against the scalar ones (DDLR_UVEC=0) in FP32/BF16.
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


@pytest.fixture(scope="module")
def prob():
    A = W.laplacian((28, 24, 20))
    part, p = W.box_partition((28, 24, 20), (2, 2, 2))
    return A, part, p


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("k", [3, 8, 16, 32, 64, 70])
@pytest.mark.parametrize("variant", [1, 2])
def test_fp64_apply_matches_oracle(prob, variant, k):
    A, part, p = prob
    h = pkg.DDLR(A, part, p, variant=variant, rank_k=k, factor=0, lanczos_max=max(5 * k, 40), **MC)
    orc = O.Oracle(A, part, p, variant=variant, k=k, factor=0, lanczos_max=max(5 * k, 40), **MC)
    U, lam, Hk, _ = orc.lowrank_original_order()
    h.set_lowrank(U, lam, orc.theta, Hk)
    for seed in (1, 2):
        x = W.rhs(A[0], seed)
        y = h.apply(torch.tensor(x, device="cuda")).cpu().numpy()
        assert _rel(y, orc.apply(x)) < 1e-12
    h.close()


@pytest.mark.parametrize("k", [8, 16, 32, 64])
@pytest.mark.parametrize("bf16", [0, 1])
@pytest.mark.parametrize("variant", [1, 2])
def test_low_precision_vector_kernels_match_scalar(prob, variant, bf16, k, monkeypatch):
    A, part, p = prob
    x = torch.tensor(W.rhs(A[0], 3), device="cuda")
    out = {}
    for uv in ("1", "0"):
        monkeypatch.setenv("DDLR_UVEC", uv)
        h = pkg.DDLR(A, part, p, variant=variant, rank_k=k, factor=0, precision=1, uk_bf16=bf16,
                     lanczos_max=max(5 * k, 40), **MC)
        out[uv] = h.apply(x).cpu().numpy()
        _, info = h.pcg(x, tol=1e-8)
        assert info[0]["status"] == "OK" and info[0]["relres"] <= 1e-8
        h.close()
    # same FP32 arithmetic in a different summation order
    assert _rel(out["1"], out["0"]) < 1e-5
