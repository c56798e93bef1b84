"""The A0 solve that allocates no device memory (its temporaries sit in a
static device array) against the ordinary A0 solve, through the C ABI.

Kept in a file of its own that pytest collects last, so that it runs both
alone in a fresh process and after every other test of the session.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def _handle(name, **kw):
    from paper_1505_04341_gb300 import DDLR
    w = W.workload(name)
    return DDLR(w["A"], w["part"], w["p"], **kw), w["A"][0]


@pytest.mark.parametrize("name,kw", [
    ("lap2d_64_b2x2", dict(variant=1, rank_k=8, factor=0)),
    ("lap3d_32", dict(variant=2, rank_k=8, factor=0, c_order=1, b_order=1)),
    # the other A0 branches: Chebyshev and MR solves with C_a, L D L^T factors
    ("lap3d_32", dict(variant=1, rank_k=8, factor=0, c_order=1, b_order=1, c_solver=1)),
    ("lap2d_64_b2x2", dict(variant=1, rank_k=8, factor=0, c_solver=2)),
    ("lap3d_32", dict(variant=1, rank_k=8, factor=2, c_order=1, b_order=1)),
])
def test_noalloc_matches_a0_solve_twice(name, kw):
    import torch
    h, n = _handle(name, **kw)
    try:
        for seed in (0, 1):      # two calls in a row, different right-hand sides
            x = torch.tensor(W.rhs(n, seed), device="cuda")
            y_ref = h.a0_solve(x, torch.zeros_like(x))
            y = torch.full_like(x, float("nan"))
            h.a0_solve_noalloc(x, y)
            torch.cuda.synchronize()
            yr, yn = y_ref.cpu().numpy(), y.cpu().numpy()
            assert np.all(np.isfinite(yn))
            err = np.max(np.abs(yn - yr)) / np.max(np.abs(yr))
            assert err <= 1e-12, err
    finally:
        h.close()


def test_noalloc_rejects_bad_arguments():
    import torch
    from paper_1505_04341_gb300.ddlr import DdlrError
    h, n = _handle("lap2d_64_b2x2", variant=1, rank_k=4)
    try:
        x = torch.tensor(W.rhs(n, 0))          # host tensor
        with pytest.raises(DdlrError, match="device memory"):
            h.a0_solve_noalloc(x, torch.zeros_like(x))
    finally:
        h.close()
    h32, n = _handle("lap2d_64_b2x2", variant=1, rank_k=4, precision=1)
    try:
        x = torch.tensor(W.rhs(n, 0), device="cuda")
        with pytest.raises(DdlrError, match="FP64"):
            h32.a0_solve_noalloc(x, torch.zeros_like(x))
    finally:
        h32.close()


def test_noalloc_leaves_free_device_memory_unchanged():
    """The call allocates nothing: after one call has loaded the kernels, the
    free device memory (cudaMemGetInfo) is the same before and after repeated
    calls, the first call on a freshly set-up handle included."""
    import torch
    h0, n = _handle("lap3d_32", variant=1, rank_k=8, factor=0, c_order=1, b_order=1)
    x = torch.tensor(W.rhs(n, 0), device="cuda")
    y = torch.empty_like(x)
    h0.a0_solve_noalloc(x, y)
    torch.cuda.synchronize()
    h1, _ = _handle("lap3d_32", variant=1, rank_k=8, factor=0, c_order=1, b_order=1)
    try:
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        for _ in range(4):
            h1.a0_solve_noalloc(x, y)
            h0.a0_solve_noalloc(x, y)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
    finally:
        h0.close()
        h1.close()
