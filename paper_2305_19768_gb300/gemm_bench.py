"""Time the tensor-core BF16 GEMM of the learned model on device buffers.

    python -m paper_2305_19768_gb300.gemm_bench [--m 19456] [--n 256] [--k 8192] [--reps 20]

Prints one JSON line: the shape, milliseconds per call (CUDA events on the
launching stream, after 3 warm-up calls) and TFLOP/s (2 M N K / time).
"""
from __future__ import annotations

import argparse
import json


def main():
    import torch

    from . import qmc

    ap = argparse.ArgumentParser()
    ap.add_argument("--m", type=int, default=19456)
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--k", type=int, default=8192)
    ap.add_argument("--reps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    a = ap.parse_args()
    g = torch.Generator(device="cuda").manual_seed(1)
    A = torch.randn(a.m, a.k, device="cuda", generator=g).to(torch.bfloat16)
    B = torch.randn(a.n, a.k, device="cuda", generator=g).to(torch.bfloat16)
    C = torch.empty(a.m, a.n, device="cuda", dtype=torch.float32)
    err = torch.zeros(1, device="cuda", dtype=torch.int32)
    stream = torch.cuda.current_stream()
    call = lambda: qmc.qmc_gemm_bf16_device(A.data_ptr(), B.data_ptr(), C.data_ptr(), a.m, a.n, a.k,  # noqa: E731
                                            err.data_ptr(), stream.cuda_stream)
    for _ in range(a.warmup):
        call()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(a.reps):
        call()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / max(1, a.reps)
    print(json.dumps({"m": a.m, "n": a.n, "k": a.k, "ms": ms, "tflops": 2.0 * a.m * a.n * a.k / (ms * 1e-3) / 1e12,
                      "wait_errors": int(err.item())}))
    return 0 if int(err.item()) == 0 else 1


if __name__ == "__main__":
    raise SystemExit(main())
