"""Tensor-core (tcgen05) kernels of the learned part against numpy.

The GEMM takes bf16 operands and accumulates in FP32; the reference is the
FP64 product of the same bf16-rounded operands, so the only difference is
the FP32 accumulation: the tensor cores add K/16 partial products of 16
terms each into the FP32 accumulator, so
|C - ref| <= (K/16 + 2) 2^-24 sum_k |A_ik B_jk|."""
import numpy as np
import pytest

from paper_2305_19768_gb300 import qmc

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("M,N,K", [(128, 16, 16), (128, 256, 64), (256, 48, 256), (256, 128, 80),
                                   (2048, 256, 2048), (384, 32, 528)])
def test_gemm_bf16_tensor_cores(M, N, K):
    rng = np.random.default_rng(M * 7 + N * 3 + K)
    A = qmc.to_bf16_bits(rng.normal(size=(M, K)).astype(np.float32))
    B = qmc.to_bf16_bits(rng.normal(size=(N, K)).astype(np.float32))
    C = qmc.qmc_gemm_bf16(A, B)
    a = qmc.from_bf16_bits(A).astype(np.float64)
    b = qmc.from_bf16_bits(B).astype(np.float64)
    ref = a @ b.T
    bound = (K / 16 + 2) * 2.0 ** -24 * (np.abs(a) @ np.abs(b).T) + 1e-30
    assert np.all(np.abs(C - ref) <= bound), float(np.max(np.abs(C - ref) / bound))


def test_gemm_rejects_bad_shapes():
    A = np.zeros((100, 16), dtype=np.uint16)
    with pytest.raises(qmc.QmcError):
        qmc.qmc_gemm_bf16(A, np.zeros((16, 16), dtype=np.uint16))
