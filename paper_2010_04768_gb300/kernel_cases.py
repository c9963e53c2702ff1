"""Single-contraction cases for kernel profiling.

Each case runs one tensor-core contraction with the shape that the sigma product of a workload
runs, through the C ABI's self-test entry points (device memory: the operands, their digit planes
and the output only), on seeded random operands.  The first call of a shape also times the
autotuner's candidate tiles; later repeats run the chosen tile only.

    python -m paper_2010_04768_gb300.kernel_cases ring-ip-medium --repeat 2

Shapes (M rows of the operator, N planar columns, K contraction length):
  ring-ip-medium   IP ring contraction, o=40 v=200, 40 systems: M = K = o v, N = 2 * 40 * o
  ring-ea-medium   EA ring contraction, 40 systems: M = K = o v, N = 2 * 40 * v
  vvvv-ea-medium   EA vvvv contraction, 40 systems: M = K = v (v - 1) / 2, N = 2 * 40 * o
  ring-ip-medium-emu   the IP ring contraction as an FP64-accurate product from 8 digit planes
                       per operand, digit pairs i + j <= 9
  ring-ip-c60-half     the IP ring contraction of the C60-shaped workload (o=90 v=450, 30 systems:
                       N = 2 * 30 * o = 5400) with M = K = o v / 2 = 20250, so that the operator
                       (820 MB in BF16) is far larger than L2 as at full size (3.3 GB)
"""
from __future__ import annotations

import argparse
import time

import numpy as np

from . import gfcc

CASES = {
    "ring-ip-medium": (8000, 3200, 8000, None),
    "ring-ea-medium": (8000, 16000, 8000, None),
    "vvvv-ea-medium": (19900, 3200, 19900, None),
    "ring-ip-medium-emu": (8000, 3200, 8000, (8, 9)),
    "ring-ip-c60-half": (20250, 5400, 20250, None),
}


def run(case: str, repeat: int = 2) -> list[float]:
    M, N, K, emu = CASES[case]
    rng = np.random.default_rng(0)
    if emu is None:
        A = rng.standard_normal((M, K), dtype=np.float32)
        B = rng.standard_normal((N, K), dtype=np.float32)
    else:
        A = rng.standard_normal((M, K))
        B = rng.standard_normal((N, K))
    times = []
    for _ in range(repeat):
        t0 = time.perf_counter()
        if emu is None:
            gfcc.selftest_gemm_bf16(A, B)
        else:
            gfcc.selftest_gemm_f64emu(A, B, S=emu[0], P=emu[1])
        times.append(time.perf_counter() - t0)
    return times


def main() -> None:
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("case", choices=sorted(CASES))
    ap.add_argument("--repeat", type=int, default=2)
    args = ap.parse_args()
    gfcc.load()
    times = run(args.case, args.repeat)
    M, N, K, emu = CASES[args.case]
    print(f"{args.case}: M={M} N={N} K={K}{' digit planes ' + str(emu) if emu else ''}; "
          f"wall seconds per call (with host staging) {', '.join(f'{t:.3f}' for t in times)}")


if __name__ == "__main__":
    main()
