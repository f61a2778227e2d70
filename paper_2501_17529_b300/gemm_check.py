"""Time the tensor-core GEMM of the screener on given shapes.

    python -m paper_2501_17529_b300.gemm_check 8192x8192x8192 65536x256x3840

Draws bf16 A [M, K] and B [N, K], runs D = A B^T through ``dcflow_gemm_bf16``
(3 warm-up calls, then 10 timed with CUDA events) and prints one JSON line
with ms and TF/s per shape.
"""
from __future__ import annotations

import json
import sys


def main(argv=None):
    import torch

    from .csrc import build
    from .dcflow import dcflow_gemm_bf16
    shapes = (argv if argv is not None else sys.argv[1:]) or ["8192x8192x8192"]
    build.build()
    out = {}
    for sh in shapes:
        M, N, K = (int(x) for x in sh.lower().split("x"))
        A = torch.randn(M, K, device="cuda").to(torch.bfloat16)
        B = torch.randn(N, K, device="cuda").to(torch.bfloat16)
        D = torch.empty(M, N, device="cuda")
        for _ in range(3):
            dcflow_gemm_bf16(A, B, out=D)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(10):
            dcflow_gemm_bf16(A, B, out=D)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 10
        out[sh] = {"ms": ms, "tflops": 2.0 * M * N * K / ms / 1e9}
    print(json.dumps(out))


if __name__ == "__main__":
    main()
