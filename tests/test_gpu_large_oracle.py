"""The kernel-per-phase PCG path against the FP64 oracle above the size rule
of the persistent solve.

The whole-solve persistent kernel serves problems of at most 3,000 rows per
SM (456,000 rows on 152 SMs); larger problems, the 128^3 configuration among
them, run one kernel per phase inside a CUDA graph per iteration.  These
tests run that path at 80^3 (n = 512,000, 125 boxes of 16^3, rank 32, greedy
multicolour orders) against the oracle, which finishes there in tens of
seconds:

* FP64, both variants: PCG iterations within one of the oracle's, the true
  relative residual (recomputed here from the CSR matrix) <= tol, and the
  solution within 1e-6 of the oracle's (Sec. 5 stopping rule, Algorithm 1).
* Mixed precision (FP32 factors and sweeps, BF16 or FP32 U_k, FP64 flexible
  CG): the true residual <= tol, iterations within max(3, 10 %) of the FP64
  oracle's, and the error against the oracle's solution stated and bounded.
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

SHAPE = (80, 80, 80)
K = {1: 32, 2: 32}
OPTS = dict(factor=0, c_order=1, b_order=1)


@pytest.fixture(scope="module", autouse=True)
def _built():
    pkg.build()
    O.build()


@pytest.fixture(scope="module")
def problem():
    A = W.laplacian(SHAPE)
    part, p = W.box_partition(SHAPE, (5, 5, 5))
    b = W.rhs(A[0], 0)
    return A, part, p, b, W.to_scipy(A)


_ORACLE = {}


def _oracle(problem, variant):
    if variant not in _ORACLE:
        A, part, p, b, _ = problem
        orc = O.Oracle(A, part, p, variant=variant, k=K[variant], **OPTS)
        x, its, rel, st = orc.pcg(b, 1e-8)
        assert st == "OK" and rel <= 1e-8
        _ORACLE[variant] = (x, its, orc.msteps)
    return _ORACLE[variant]


def _relres(S, b, x):
    return np.linalg.norm(b - S @ x) / np.linalg.norm(b)


@pytest.mark.parametrize("variant", [1, 2])
def test_fp64_per_phase_pcg_matches_oracle(problem, variant):
    A, part, p, b, S = problem
    assert A[0] > 3000 * torch.cuda.get_device_properties(0).multi_processor_count
    xo, its_o, m_o = _oracle(problem, variant)
    h = pkg.DDLR(A, part, p, variant=variant, rank_k=K[variant], precision=0, **OPTS)
    inf = h.info()
    assert not (inf["persistent"] & 1)          # PCG: one kernel per phase
    assert inf["lanczos_steps"] == m_o
    x, info = h.pcg(torch.tensor(b, device="cuda"), tol=1e-8)
    x = x.cpu().numpy()
    assert info[0]["status"] == "OK"
    assert abs(info[0]["its"] - its_o) <= 1, (info, its_o)
    assert _relres(S, b, x) <= 1e-8 * (1 + 1e-6)
    assert np.linalg.norm(x - xo) <= 1e-6 * np.linalg.norm(xo)
    h.close()


@pytest.mark.parametrize("variant", [1, 2])
@pytest.mark.parametrize("uk_bf16", [1, 0])
def test_mixed_per_phase_pcg_against_oracle(problem, variant, uk_bf16):
    A, part, p, b, S = problem
    xo, its_o, _ = _oracle(problem, variant)
    h = pkg.DDLR(A, part, p, variant=variant, rank_k=K[variant], precision=1, uk_bf16=uk_bf16, **OPTS)
    assert not (h.info()["persistent"] & 1)
    x, info = h.pcg(torch.tensor(b, device="cuda"), tol=1e-8)
    x = x.cpu().numpy()
    assert info[0]["status"] == "OK"
    assert abs(info[0]["its"] - its_o) <= max(3, its_o // 10), (info, its_o)
    assert _relres(S, b, x) <= 1e-8 * (1 + 1e-6)
    # both solutions satisfy the 1e-8 residual bound; on this well-conditioned
    # Laplacian their difference is far below it
    assert np.linalg.norm(x - xo) <= 1e-6 * np.linalg.norm(xo)
    h.close()
