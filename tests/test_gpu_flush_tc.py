"""The tcgen05 tensor-core flush of the delayed updates (TF32 three-product
split) reproduces W - U V^T at FP32 accuracy against an FP64 reference."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("cplx", [0, 1])
@pytest.mark.parametrize("N,rank", [(128, 8), (200, 32), (512, 64), (384, 72), (4096, 64)])
def test_flush_tc_accuracy(cplx, N, rank):
    from paper_2412_01737_gb300 import GGF
    ctx = GGF(0)
    err = ctx.selftest_flush(cplx, N, rank)
    ctx.close()
    assert err < 2e-6, err
