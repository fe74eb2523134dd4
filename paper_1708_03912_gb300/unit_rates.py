"""Measure the per-SM unit rates used for the roofline of the assembly kernels.

python -m paper_1708_03912_gb300.unit_rates
Compiles csrc/unit_rates.cu for sm_103a into _build/ and runs it on the current GPU.
"""
import os
import subprocess
import sys

from .build import ARCH, BUILD, CSRC, _nvcc


def main():
    os.makedirs(BUILD, exist_ok=True)
    exe = os.path.join(BUILD, "unit_rates")
    src = os.path.join(CSRC, "unit_rates.cu")
    subprocess.run([_nvcc(), "-O3", "-o", exe, src] + ARCH, check=True)
    return subprocess.run([exe]).returncode


if __name__ == "__main__":
    sys.exit(main())
