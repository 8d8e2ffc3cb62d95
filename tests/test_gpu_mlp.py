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


def _net():
    return qmc.Mlp(2, 256, 4, 42, seed=7)


def test_mlp_forward_and_gradient_match_oracle():
    from oracle import mlp as omlp

    net = _net()
    try:
        rng = np.random.default_rng(11)
        B = 300
        x = rng.uniform(-1, 1, size=(B, 2)).astype(np.float32)
        y = rng.normal(size=(B, 42)).astype(np.float32)
        wt = rng.uniform(0.5, 2.0, size=42).astype(np.float32)
        p = net.params()
        out = net.forward(x)
        ref, _ = omlp.forward(p, x, 2, 256, 4, 42, bf16=True)
        scale = np.abs(ref).max()
        # identical bf16 rounding points; differences come from FP32 accumulation and the
        # occasional bf16 rounding flip that this causes (one bf16 ulp = 2^-8 relative)
        assert np.abs(out - ref).max() <= 5e-3 * scale
        assert np.abs(out - ref).mean() <= 5e-4 * scale
        loss, g = net.grad(x, y, wt)
        rloss, rg = omlp.loss_and_grad(p, x, y, wt, 2, 256, 4, 42, bf16=True)
        assert abs(loss - rloss) <= 1e-3 * abs(rloss)
        cos = float(g @ rg / (np.linalg.norm(g) * np.linalg.norm(rg)))
        assert cos > 0.9999, cos
        assert np.abs(g - rg).max() <= 2e-2 * np.abs(rg).max()
        # against the unrounded FP64 gradient the bf16 model is still close
        _, g64 = omlp.loss_and_grad(p, x, y, wt, 2, 256, 4, 42, bf16=False)
        cos64 = float(g @ g64 / (np.linalg.norm(g) * np.linalg.norm(g64)))
        assert cos64 > 0.999, cos64
    finally:
        net.close()


def test_mlp_training_fits_a_smooth_map():
    net = _net()
    try:
        rng = np.random.default_rng(12)
        x = rng.uniform(-1, 1, size=(2000, 2)).astype(np.float32)
        def target(x):
            return np.stack([np.sin(2 * x[:, 0] + 0.1 * k * x[:, 1]) * (1 + 0.02 * k) for k in range(42)],
                            axis=1).astype(np.float32)

        y = target(x)
        losses = net.train(x, y, 600, 1e-3)
        assert losses[-1] < losses[0] / 100, (losses[0], losses[-1])
        xt = rng.uniform(-1, 1, size=(500, 2)).astype(np.float32)
        assert np.sqrt(np.mean((net.forward(xt) - target(xt)) ** 2)) < 0.05
    finally:
        net.close()


@pytest.mark.parametrize("M,N,K", [(256, 256, 2048), (2048, 48, 256), (19456, 256, 1024)])
def test_gemm_bf16_device_buffers_and_split_k(M, N, K):
    # device-pointer entry point: split-K (few M tiles, long K) and a grid of
    # one M tile per SM; reference = FP64 product of the same bf16 operands
    torch = pytest.importorskip("torch")
    g = torch.Generator(device="cuda").manual_seed(M + N + K)
    A = torch.randn(M, K, device="cuda", generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, device="cuda", generator=g).to(torch.bfloat16)
    C = torch.empty(M, N, device="cuda", dtype=torch.float32)
    err = torch.zeros(1, device="cuda", dtype=torch.int32)
    qmc.qmc_gemm_bf16_device(A.data_ptr(), B.data_ptr(), C.data_ptr(), M, N, K, err.data_ptr())
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    a, b = A.double(), B.double()
    ref = a @ b.T
    bound = (K / 16 + 2) * 2.0 ** -24 * (a.abs() @ b.abs().T) + 1e-30
    worst = float(((C.double() - ref).abs() / bound).max())
    assert worst <= 1.0, worst


@pytest.mark.parametrize("M,N,K", [(512, 256, 1024), (19456, 256, 1024)])
def test_gemm_wait_timeout_sets_the_error_word_and_frees_tensor_memory(M, N, K):
    # every pipeline wait given zero polls: each CTA must give up, count
    # itself in the error word, drain its copies and MMAs, free its tensor
    # memory and return; a normal GEMM right after must then allocate tensor
    # memory again and be exact. (512: split-K, one K chunk per CTA, only the
    # MMA-side waits run out; 19456: 16 chunks per CTA, the producer's
    # stage-free waits run out too.)
    torch = pytest.importorskip("torch")
    g = torch.Generator(device="cuda").manual_seed(7)
    A = torch.randn(M, K, device="cuda", generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, device="cuda", generator=g).to(torch.bfloat16)
    C = torch.empty(M, N, device="cuda", dtype=torch.float32)
    err = torch.zeros(1, device="cuda", dtype=torch.int32)
    qmc.qmc_gemm_bf16_device_limit(A.data_ptr(), B.data_ptr(), C.data_ptr(), M, N, K, err.data_ptr(), 0)
    torch.cuda.synchronize()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    mt, nchunks = M // 128, (K + 63) // 64
    splits = max(1, min(nchunks, sms // mt))
    per = (nchunks + splits - 1) // splits
    splits = (nchunks + per - 1) // per
    assert int(err.item()) == mt * splits
    err.zero_()
    for limit in (None, 1 << 26):
        C.zero_()
        if limit is None:
            qmc.qmc_gemm_bf16_device(A.data_ptr(), B.data_ptr(), C.data_ptr(), M, N, K, err.data_ptr())
        else:
            qmc.qmc_gemm_bf16_device_limit(A.data_ptr(), B.data_ptr(), C.data_ptr(), M, N, K, err.data_ptr(), limit)
        torch.cuda.synchronize()
        assert int(err.item()) == 0
        a, b = A.double(), B.double()
        bound = (K / 16 + 2) * 2.0 ** -24 * (a.abs() @ b.abs().T) + 1e-30
        assert float(((C.double() - a @ b.T).abs() / bound).max()) <= 1.0
