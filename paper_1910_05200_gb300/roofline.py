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
EDGE_NODE_VISIT = 200  # two children: box vs 5 pyramid planes (~55) + normal-cone test (~45) each
EDGE_TEST = 110        # 2 silhouette tests (16) + clip of 2 endpoints against 5 planes (~94)

# Counting in k_bwd_sedge: the edge-BVH descent is shared by the 32 lanes of
# a warp (one traversal of the warp's bounding sphere), so an edge-BVH visit
# is counted once per warp; edge tests are per lane.

# DRAM bytes of one k_bwd_sedge launch at 256x256x16 spp from a 1-pass ncu
# capture of the current kernel (dram__bytes_read.sum + dram__bytes_write.sum);
# None until the kernel as it stands has been captured.
SEDGE_TRAFFIC_BYTES = None
SHADE_FWD = 150        # one light sample shaded (BRDF + geometry term)
SHADE_BWD = 420        # one light sample: forward recompute + adjoint
N_LIGHTS = 20

SMS = 152
FP32_LANES = 128


def forward_flops(cnt, samples: int, n_on: int) -> float:
    return cnt[0] * NODE_VISIT + cnt[1] * TRI_TEST + samples * n_on * SHADE_FWD


def backward_flops(cnt, samples: int, n_on: int) -> float:
    """All backward kernels: counters 4..15."""
    shading = samples * (N_LIGHTS * SHADE_BWD + 2 * n_on * SHADE_FWD)
    trav = 0
    for k in (4, 8, 12):
        trav += cnt[k] * NODE_VISIT + cnt[k + 1] * TRI_TEST + cnt[k + 2] * EDGE_NODE_VISIT + cnt[k + 3] * EDGE_TEST
    return trav + shading


def sedge_flops(cnt) -> float:
    """Shadow-edge kernel: counters 12..15 (its shadow rays, its edge search)."""
    return cnt[12] * NODE_VISIT + cnt[13] * TRI_TEST + cnt[14] * EDGE_NODE_VISIT + cnt[15] * EDGE_TEST


def fp32_peak_tflops(sm_mhz: float | None) -> float:
    mhz = sm_mhz if sm_mhz else 2070.0
    return SMS * FP32_LANES * 2 * mhz * 1e6 / 1e12
