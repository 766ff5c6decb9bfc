"""Measure the CUDA-core FMA peaks (FP64, FP32) of cuda:0 and print one JSON line.

The measured peaks file has HBM and BF16 tensor throughput only; the
NFFT's window sums run on the CUDA cores, so their ALU roofline needs these.
Each figure is the best of `reps` runs of a kernel of independent FMA chains.
"""
from __future__ import annotations

import ctypes
import json
import subprocess

import torch

from . import _lib, build


def measure(reps: int = 3) -> dict:
    build.build()
    torch.cuda.init()
    out = {}
    for prec, iters in ((64, 1600), (32, 100000)):
        best = 0.0
        for _ in range(reps):
            v = ctypes.c_double()
            _lib.call("nfft3_fma_peak", prec, iters, None, ctypes.byref(v))
            best = max(best, v.value)
        out["fp%d_tflops" % prec] = best
    try:
        q = subprocess.run(["nvidia-smi", "-i", "0", "--query-gpu=clocks.sm,clocks.max.sm",
                            "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=10)
        sm, smax = [float(v) for v in q.stdout.strip().split(",")]
        out["sm_mhz_after"] = sm
        out["sm_max_mhz"] = smax
    except Exception:
        pass
    props = torch.cuda.get_device_properties(0)
    out["sms"] = props.multi_processor_count
    out["gpu"] = props.name
    return out


if __name__ == "__main__":
    print(json.dumps(measure()))
