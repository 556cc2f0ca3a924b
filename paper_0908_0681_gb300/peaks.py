"""Measure the FP32 and FP64 FMA pipes of the current GPU (roofline denominators).

    python -m paper_0908_0681_gb300.peaks

Builds probe/pipe_probe.cu for sm_103a into _build/ and runs it. The probe
also times a variant with a single active lane per warp: on GB300 an FP64 warp
instruction takes the same time with 1 or 32 active lanes.
"""
from __future__ import annotations

import json
import os
import subprocess
import sys

from .build import ARCH, HERE, _nvcc


def main() -> int:
    src = os.path.join(HERE, "probe", "pipe_probe.cu")
    exe = os.path.join(HERE, "_build", "pipe_probe")
    os.makedirs(os.path.dirname(exe), exist_ok=True)
    if not os.path.exists(exe) or os.path.getmtime(exe) < os.path.getmtime(src):
        subprocess.check_call([_nvcc(), *ARCH, "-O3", src, "-o", exe])
    out = subprocess.run([exe], capture_output=True, text=True)
    sys.stdout.write(out.stdout)
    if out.returncode == 0:
        json.loads(out.stdout.strip().splitlines()[-1])
    return out.returncode


if __name__ == "__main__":
    sys.exit(main())
