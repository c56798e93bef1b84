"""GPU: the binary64 <-> binary32 conversions that the batched casts write out
on the bit patterns (IEEE 754 rounding to nearest, ties to even; exact
widening) give the same bits as the device's conversion instructions, over
random bit patterns of every exponent, the halfway cases, both ends of the
normal binary32 range and the special values."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1505_04341_gb300 as pkg  # noqa: E402
from paper_1505_04341_gb300 import ddlr as D  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    pkg.build()


def _narrowing_cases():
    rng = np.random.default_rng(7)
    bits = rng.integers(0, 2**63, size=400_000, dtype=np.uint64) | (
        rng.integers(0, 2, size=400_000, dtype=np.uint64) << np.uint64(63))
    vals = [bits.view(np.float64)]
    # values around the binary32 range ends and every binary32 exponent
    e = rng.integers(860, 1190, size=400_000).astype(np.uint64)
    m = rng.integers(0, 2**52, size=400_000, dtype=np.uint64)
    vals.append(((e << np.uint64(52)) | m).view(np.float64))
    # exact halfway cases (dropped bits 1000...0) with odd and even kept bits
    h = (m & ~np.uint64(0x1FFFFFFF)) | np.uint64(0x10000000)
    vals.append(((e << np.uint64(52)) | h).view(np.float64))
    vals.append(((e << np.uint64(52)) | (h + np.uint64(1))).view(np.float64))
    vals.append(((e << np.uint64(52)) | (h - np.uint64(1))).view(np.float64))
    f32 = np.finfo(np.float32)
    special = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, float(f32.max), float(f32.tiny),
                        float(f32.max) * (1 + 2**-25), float(f32.max) * (1 + 2**-23), 1e-46, 1e-39,
                        1.0, -1.0, 3.0000001, 2.0**-126, 2.0**-127, 2.0**128], dtype=np.float64)
    vals.append(special)
    return np.concatenate(vals)


def test_narrowing_matches_device():
    x = torch.tensor(_narrowing_cases(), dtype=torch.float64, device="cuda")
    assert D.selftest_conversions(x, 0) == 0


def test_widening_matches_device():
    rng = np.random.default_rng(8)
    lo = rng.integers(0, 2**32, size=500_000, dtype=np.uint64)
    special = np.array([0, 0x80000000, 0x7F800000, 0xFF800000, 0x7FC00000, 0x00000001,
                        0x007FFFFF, 0x00800000, 0x7F7FFFFF], dtype=np.uint64)
    x = torch.tensor(np.concatenate([lo, special]).view(np.float64), dtype=torch.float64, device="cuda")
    assert D.selftest_conversions(x, 1) == 0


def test_bad_arguments():
    x = np.zeros(4)
    with pytest.raises(pkg.DdlrError):
        D.selftest_conversions(x, 0)            # host memory
    xd = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(pkg.DdlrError):
        D.selftest_conversions(xd, 2)
