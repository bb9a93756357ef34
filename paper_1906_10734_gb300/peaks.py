"""Measured arithmetic peaks of GPU 0 (hpm_measure_alu_peaks), printed as JSON.

    python -m paper_1906_10734_gb300.peaks [--repeat R]

Runs the library's FP32 FFMA, FP64 DFMA and FP32 rsqrt microbenchmarks R times
and prints every measurement and the median of each rate. These are the
denominators of the rooflines of the kernels bound by CUDA-core arithmetic.
"""
from __future__ import annotations

import argparse
import json
import statistics


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--repeat", type=int, default=5)
    args = ap.parse_args()
    import torch

    from paper_1906_10734_gb300 import build as B, hpm
    B.build()
    torch.cuda.set_device(0)
    runs = [hpm.hpm_measure_alu_peaks() for _ in range(args.repeat)]
    med = {k: statistics.median(r[k] for r in runs) for k in ("fp32_tflops", "fp64_tflops", "rsqrt_gops")}
    print(json.dumps({"device": torch.cuda.get_device_name(0), "median": med, "runs": runs}))


if __name__ == "__main__":
    main()
