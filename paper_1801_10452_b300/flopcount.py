"""Algorithmic operation count of one geodesic step, from the kernel source.

Compiles ``csrc/flopcount.cu`` for the host with nvcc: it instantiates the kernels'
templated arithmetic with a number type that counts each add, multiply, division and
elementary-function call (a fused multiply-add counts as 2 flops).  The result is cached
next to the library and regenerated when the sources change.
"""
from __future__ import annotations

import glob
import json
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc", "flopcount.cu")
OUT_DIR = os.path.join(HERE, "_build")
BIN = os.path.join(OUT_DIR, "flopcount")
CACHE = os.path.join(OUT_DIR, "flopcount.json")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")


def _stale(path):
    if not os.path.exists(path):
        return True
    t = os.path.getmtime(path)
    srcs = [SRC] + glob.glob(os.path.join(HERE, "csrc", "*.cuh"))
    return any(os.path.getmtime(s) > t for s in srcs)


def counts() -> dict:
    """Per-part operation counts (see flopcount.cu)."""
    os.makedirs(OUT_DIR, exist_ok=True)
    if _stale(CACHE):
        if _stale(BIN):
            subprocess.run([NVCC, "-O1", "-std=c++17", "-o", BIN, SRC], check=True, capture_output=True)
        out = subprocess.run([BIN], check=True, capture_output=True, text=True).stdout
        with open(CACHE, "w") as f:
            f.write(out)
    return json.load(open(CACHE))


def flops_per_step(n_freq: int = 1, plasma: str = "analytic") -> dict:
    """Flops of one accepted step with its transfer sample: geodesic (step size + RK4) +
    plasma sample + n_freq x (emissivity + transfer update).  The same source serves the
    FP32 and FP64 instantiations, so both carry the same algorithmic count."""
    c = counts()
    sample = c["sample_analytic"]["flops"] if plasma == "analytic" else c["sample_grid_" + plasma]["flops"]
    total = c["geodesic_step"]["flops"] + sample + n_freq * c["per_frequency"]["flops"]
    return {"fp64_step": total, "fp32_step": total, "geodesic_only": c["geodesic_step"]["flops"],
            "sample": sample, "per_frequency": c["per_frequency"]["flops"],
            "verlet_step": c["verlet_step"]["flops"] + sample + n_freq * c["per_frequency"]["flops"],
            "verlet_reeval_step": c["verlet_reeval_step"]["flops"] + sample + n_freq * c["per_frequency"]["flops"]}


# FP32 instructions of one double-float operation, counted from raptor_df64.cuh: add
# (two-sum 6, two adds, fast-two-sum 3) 11; multiply (product, error FMA, two cross FMAs; the
# pair is left unrenormalised) 4; division (approximate reciprocal, two residual products and
# subtractions, three quotient products, renormalisation) ~40; sincos of the polar angle
# (node index, offset in double-float, two short series with float tails, table load,
# angle addition) ~150.  The model gives ~5,400 instructions per step with its FP32
# transfer sample; ncu counts 5,281 executed per step of the FP64 phase (256^2 render).
DF64_FP32_INSTR = {"add": 11, "mul": 4, "div": 40, "sincos": 150}


def df64_instructions_per_step(n_freq: int = 1, plasma: str = "analytic") -> dict:
    """FP32 instructions of one double-float geodesic step (its transfer sample runs in FP32:
    one instruction per flop), and the resulting instructions per algorithmic flop."""
    c = counts()
    g = c["geodesic_step"]
    geo = sum(DF64_FP32_INSTR[k] * g[k] for k in DF64_FP32_INSTR)
    f = flops_per_step(n_freq, plasma)
    instr = geo + f["sample"] + n_freq * f["per_frequency"]
    return {"fp32_instructions": instr, "flops": f["fp64_step"], "instructions_per_flop": instr / f["fp64_step"]}
