"""Build and run the integer-pipe throughput microbenchmark (int_peaks.cu) on the current GPU.

Usage: python -m paper_2407_19871_gb300.peaks.run   -> one JSON line with operations per SM
per clock for each measured instruction pattern."""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))


def main() -> int:
    from paper_2407_19871_gb300.build import ARCH, nvcc
    out_dir = os.path.join(ROOT, "_build")
    os.makedirs(out_dir, exist_ok=True)
    exe = os.path.join(out_dir, "int_peaks")
    src = os.path.join(HERE, "int_peaks.cu")
    subprocess.check_call([nvcc(), src, "-o", exe, "-O3"] + ARCH)
    return subprocess.call([exe])


if __name__ == "__main__":
    sys.exit(main())
