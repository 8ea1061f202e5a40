"""The tensor-core product unit of the segment sweeps (tcgen05, kind::tf32):
its products in every operand form the sweep issues agree with CUDA-core
FP32 products of the same operands to the TF32 rounding of the operands
(10 mantissa bits: unit roundoff 2^-11 ~ 4.9e-4 per operand, normwise
differences of order 1e-3 over K = 128 terms), and X - X with the second
product negated cancels to FP32 accumulation rounding."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1809_06360_gb300 import build, lqr
    build.build()
    return lqr


def test_tensor_core_products_match_cuda_cores(lib):
    errs = lib.lqr_tc_selftest(0)
    print("tc selftest", errs)
    assert errs[4] == 0.0
    for e in errs[:3]:
        assert 1e-6 < e < 1e-2, errs  # TF32 rounding is visible, layout errors are O(1)
    assert errs[3] < 1e-5, errs
