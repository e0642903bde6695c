"""Algorithmic work of the render kernels, for the roofline fraction.

The render and its gradient are bound by FP32 ALU work of BVH traversal,
ray/triangle tests and shading, on data that stays in L2.  Work is counted by
the kernels themselves (node visits, triangle tests, edge-BVH visits, edge
tests; fr_set_counters) and converted to FLOPs with the per-operation costs
below, counted from the code (an add, multiply, min/max, compare or FMA each
count as 1 FLOP except FMA = 2; divisions and square roots count as 1).
"""
from __future__ import annotations

# FLOPs per operation
NODE_VISIT = 40        # two child slab tests: 6 sub, 6 mul, 10 min/max, 2 cmp each
TRI_TEST = 40          # watertight test: 9 sub, 6 mul + 6 sub (shear), 9 edge-fn ops, 3+6 for T, div
EDGE_NODE_VISIT = 80   # two child boxes against 5 pyramid planes (3 sub + 5 for a dot each)
EDGE_TEST = 100        # 2 silhouette dots (16) + clip of 2 endpoints against 5 planes (~84)
SHADE_FWD = 150        # one light sample shaded (BRDF + geometry term)
SHADE_BWD = 420        # one light sample: forward recompute + adjoint
N_LIGHTS = 20

SMS = 152
FP32_LANES = 128


def forward_flops(cnt, samples: int, n_on: int) -> float:
    return cnt[0] * NODE_VISIT + cnt[1] * TRI_TEST + samples * n_on * SHADE_FWD


def backward_flops(cnt, samples: int, n_on: int) -> float:
    shading = samples * (N_LIGHTS * SHADE_BWD + 2 * n_on * SHADE_FWD)
    return (cnt[4] * NODE_VISIT + cnt[5] * TRI_TEST + cnt[6] * EDGE_NODE_VISIT + cnt[7] * EDGE_TEST + shading)


def fp32_peak_tflops(sm_mhz: float | None) -> float:
    mhz = sm_mhz if sm_mhz else 2070.0
    return SMS * FP32_LANES * 2 * mhz * 1e6 / 1e12
