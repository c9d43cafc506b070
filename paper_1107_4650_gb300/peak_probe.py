"""Builds and runs the arithmetic issue-rate probe (csrc/peak_probe.cu) on cuda:0.

  python -m paper_1107_4650_gb300.peak_probe

Prints one JSON line per operation (DFMA, DADD, FFMA, FADD): lane-instructions per second and per SM per
clock.  The FP64 figure is the measured denominator of the FP64 step kernels' ALU roofline.
"""
from __future__ import annotations

import os
import subprocess
import sys

from .build import _nvcc

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc", "peak_probe.cu")
EXE = os.path.join(HERE, "_build", "peak_probe")


def main() -> int:
    os.makedirs(os.path.dirname(EXE), exist_ok=True)
    subprocess.check_call([_nvcc(), "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-I", os.path.dirname(SRC), "-o", EXE, SRC])
    return subprocess.call([EXE])


if __name__ == "__main__":
    sys.exit(main())
