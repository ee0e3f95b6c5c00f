"""GPU checks of the learned brick codec's tensor-core path (tcgen05): products
through the shared-memory layouts and descriptors the codec kernels use, against
numpy in FP64 on the same BF16 values."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vr():
    from paper_1205_0282_gb300 import vr
    return vr


@pytest.mark.parametrize("a_mn,b_mn", [(0, 0), (1, 0), (0, 1), (1, 1)])
@pytest.mark.parametrize("K,N", [(16, 16), (32, 64), (64, 32), (64, 64)])
def test_tensor_core_product(vr, a_mn, b_mn, K, N):
    rng = np.random.default_rng(K * 100 + N + 7 * a_mn + 13 * b_mn)
    A = vr.to_bf16_bits(rng.normal(size=(128, K)))
    B = vr.to_bf16_bits(rng.normal(size=(N, K)))
    D = vr.vr_codec_gemm_check(A, B, a_mn, b_mn)
    a = vr.bf16_bits_to_float(A).astype(np.float64)
    b = vr.bf16_bits_to_float(B).astype(np.float64)
    ref = a @ b.T
    scale = np.abs(a) @ np.abs(b).T
    assert np.all(np.abs(D - ref) <= 1e-6 * scale + 1e-30)
