"""Dense INT8 GEMM rate of this GPU through the vendor library (torch._int_mm -> cuBLASLt),
the number that decides whether an INT8 Toeplitz formulation of the external product could
compete with the integer NTT (it needs ~1.1e11 int8 multiply-adds per bootstrap).

Usage: python -m paper_2407_19871_gb300.peaks.int8_rate  -> one JSON line."""
import json

import torch


def rate(m: int, n: int, k: int, dtype: str, reps: int = 10) -> float:
    if dtype == "int8":
        a = torch.randint(-128, 127, (m, k), dtype=torch.int8, device="cuda")
        b = torch.randint(-128, 127, (k, n), dtype=torch.int8, device="cuda")
        f = lambda: torch._int_mm(a, b)
    else:
        a = torch.randn(m, k, dtype=torch.bfloat16, device="cuda")
        b = torch.randn(k, n, dtype=torch.bfloat16, device="cuda")
        f = lambda: a @ b
    for _ in range(3):
        f()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    best = float("inf")
    for _ in range(reps):
        e0.record()
        f()
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1) / 1e3)
    return 2.0 * m * n * k / best


if __name__ == "__main__":
    s = 8192
    i8 = rate(s, s, s, "int8")
    bf = rate(s, s, s, "bf16")
    ops_per_bootstrap = 630 * 2 * 1024 * 6144 * 7 * 2   # Toeplitz route: 7 surviving 8-bit limb pairs
    print(json.dumps({"int8_tops": i8 / 1e12, "bf16_tflops": bf / 1e12, "shape": [s, s, s],
                      "toeplitz_int8_ops_per_bootstrap": ops_per_bootstrap,
                      "toeplitz_bootstraps_per_s_at_this_rate": i8 / ops_per_bootstrap}))
