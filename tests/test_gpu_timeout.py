"""Bounded device waits: a wait that runs out ends the kernel and the call
with DDLR_ERR_TIMEOUT, without faulting the GPU, and the handle stays usable.

The persistent kernels separate their phases by grid barriers whose waits are
limited by the handle's wait_limit_s.  DDLR_TEST_UNMET_BARRIER=1 makes the
first barrier of a launch wait for one arrival more than the grid has (an
arrival that nothing provides), so every CTA's wait runs out after the limit:
each CTA records it and returns, and the host reads the flag.
"""
import time

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


@pytest.mark.parametrize("variant", [1, 2])
def test_grid_barrier_runs_out_and_handle_recovers(variant, monkeypatch):
    A = W.laplacian((32, 32, 32))
    part, p = W.box_partition((32, 32, 32), (2, 2, 2))
    h = pkg.DDLR(A, part, p, variant=variant, rank_k=8, factor=0, **MC)
    assert h.info()["persistent"] == 3          # PCG and Lanczos persistent
    b = torch.tensor(W.rhs(A[0], 0), device="cuda")
    x0, inf0 = h.pcg(b, tol=1e-8)
    x0 = x0.clone()

    h.set_wait_limit(1e-3)
    monkeypatch.setenv("DDLR_TEST_UNMET_BARRIER", "1")
    t = time.perf_counter()
    with pytest.raises(pkg.DdlrError) as e:
        h.pcg(b, tol=1e-8)
    assert e.value.status == "TIMEOUT"
    # every CTA gave up after the 1 ms limit (the default limit is 2 s)
    assert time.perf_counter() - t < 1.0
    with pytest.raises(pkg.DdlrError) as e:
        h.refactor()                            # the persistent Lanczos process
    assert e.value.status == "TIMEOUT"

    monkeypatch.delenv("DDLR_TEST_UNMET_BARRIER")
    h.set_wait_limit(2.0)
    h.refactor()
    x1, inf1 = h.pcg(b, tol=1e-8)
    assert inf1[0]["status"] == "OK" and inf1[0]["relres"] <= 1e-8
    assert inf1[0]["its"] == inf0[0]["its"]
    assert torch.equal(x1, x0)                  # the same bits as before the timeouts
    orc = O.Oracle(A, part, p, variant=variant, k=8, factor=0, **MC)
    _, its_o, _, st = orc.pcg(W.rhs(A[0], 0), 1e-8)
    assert st == "OK" and abs(inf1[0]["its"] - its_o) <= 1
    h.close()


def test_wait_limit_arguments():
    A = W.laplacian((12, 12))
    part, p = W.box_partition((12, 12), (2, 2))
    with pytest.raises(pkg.DdlrError) as e:
        pkg.DDLR(A, part, p, rank_k=4, wait_limit_s=0.0)
    assert e.value.status == "INVALID"
    h = pkg.DDLR(A, part, p, rank_k=4, wait_limit_s=0.5)
    for bad in (0.0, -1.0, 1e9, float("nan")):
        with pytest.raises(pkg.DdlrError):
            h.set_wait_limit(bad)
    h.set_wait_limit(3.0)
    x, info = h.pcg(np.asarray(W.rhs(A[0], 0)), tol=1e-8)
    assert info[0]["status"] == "OK"
    h.close()
