"""Algorithmic flop count of one geodesic step (filled in by the source-level counter)."""


def flops_per_step():
    return {"fp64_step": None, "fp32_step": None}
