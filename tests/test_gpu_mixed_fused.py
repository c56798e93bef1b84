"""GPU: the mixed-precision DDLR-1 apply without separate precision casts.

On shallow (multicolour) factors the FP32 preconditioner reads the FP64
residual where it needs it and its last sweeps write the FP64 result; the
rounding is the same as that of separate cast kernels (FP64 -> FP32 to
nearest as read, FP32 -> FP64 exactly), so the results must be bitwise those of
the path with the casts (DDLR_NO_FUSED_CAST=1), for the apply and for a whole
kernel-per-phase PCG solve, with FP32 and BF16 U_k."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1505_04341_gb300 as pkg  # noqa: E402
import workloads as W  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("bf16", [0, 1])
@pytest.mark.parametrize("k", [8, 16])
def test_fused_casts_bitwise(bf16, k, monkeypatch):
    A = W.laplacian((30, 28, 26))
    part, p = W.box_partition((30, 28, 26), (2, 2, 2))
    b = torch.tensor(W.rhs(A[0], 3), device="cuda")
    out = {}
    for fused in ("0", "1"):
        monkeypatch.setenv("DDLR_NO_FUSED_CAST", fused)
        monkeypatch.setenv("DDLR_PERSIST", "0")
        h = pkg.DDLR(A, part, p, variant=1, rank_k=k, c_order=1, b_order=1, precision=1, uk_bf16=bf16)
        h.reset_counters()
        y = h.apply(b)
        fams = h.counters()["families"]
        x, info = h.pcg(b, tol=1e-8)
        out[fused] = (y.cpu().numpy(), x.cpu().numpy(), info[0]["its"],
                      fams.get("vec", {"launches": 0})["launches"])
        h.close()
    (y0, x0, i0, v0), (y1, x1, i1, v1) = out["0"], out["1"]
    assert v0 == 0 and v1 > 0                  # no cast kernels on the fused path
    assert np.array_equal(y0, y1)
    assert i0 == i1 and np.array_equal(x0, x1)
