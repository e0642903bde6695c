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
EDGE_NODE_VISIT = 400  # four children (4-wide edge hierarchy): box vs 5 pyramid planes (~45) + normal cone (~55) each
EDGE_TEST = 20         # exact silhouette test of a pair: 2 plane tests (3 sub, 3 mul, 2 add each) + signs
CLIP_TEST = 90         # adjacency check, clip of both endpoints against the 5 planes of the light pyramid
EDGE_CLASSIFY = 68     # an edge's 2 face planes bounded over a box: 2 corner evaluations (8 each), the
                       # rounding bound T (14) and the margin and compares (4), per face

# Counter layout (fr_get_counters): 6 per kernel -- ray BVH nodes, triangle
# tests, 4-wide edge-hierarchy nodes (once per warp: the 32 lanes share one
# descent), exact silhouette tests of (shading point, edge) pairs, clip tests,
# leaf edges classified against a warp's box of shading points (once per
# warp) -- for forward, interior, primary edges, shadow edges.
K_FWD, K_INTERIOR, K_PEDGE, K_SEDGE = 0, 6, 12, 18

# DRAM bytes of one k_bwd_sedge launch (the shadow-edge search and pick, two
# points per lane) at 256x256x16 spp from a 1-pass ncu capture of the kernel
# as it stands (dram__bytes_read.sum + dram__bytes_write.sum): 22.73 MB read,
# the edge records, hierarchies and meshes staying in L2, and 74.45 MB of
# the 117 MB of picks written back (the rest is still in L2 when the
# contributions read it).
SEDGE_TRAFFIC_BYTES = 22.73e6 + 74.45e6
# L2 bytes of the same launch: lts__t_sectors.sum x 32 B from the same
# 1-pass capture (291.43 M sectors), spills to local memory included.
SEDGE_L2_BYTES = 291.43e6 * 32
SHADE_FWD = 150        # one light sample shaded (BRDF + geometry term)
SHADE_BWD = 420        # one light sample: forward recompute + adjoint
N_LIGHTS = 20

FP32_LANES = 128


def _kernel_flops(cnt, k):
    return (cnt[k] * NODE_VISIT + cnt[k + 1] * TRI_TEST + cnt[k + 2] * EDGE_NODE_VISIT + cnt[k + 3] * EDGE_TEST
            + cnt[k + 4] * CLIP_TEST + cnt[k + 5] * EDGE_CLASSIFY)


def forward_flops(cnt, samples: int, n_on: int) -> float:
    return _kernel_flops(cnt, K_FWD) + samples * n_on * SHADE_FWD


def backward_flops(cnt, samples: int, n_on: int) -> float:
    """All backward kernels: interior adjoint (every light), primary edges
    (two one-sample radiance estimates per edge sample), shadow edges."""
    shading = samples * (N_LIGHTS * SHADE_BWD + 2 * n_on * SHADE_FWD)
    return sum(_kernel_flops(cnt, k) for k in (K_INTERIOR, K_PEDGE, K_SEDGE)) + shading


def step_flops(cnt, samples: int, n_on: int) -> float:
    """One fwd+loss+bwd step from the counters of that step."""
    return forward_flops(cnt, samples, n_on) + backward_flops(cnt, samples, n_on)


def sedge_flops(cnt) -> float:
    """Shadow-edge term: the edge search and the contributions' shadow rays."""
    return _kernel_flops(cnt, K_SEDGE)


def sedge_search_flops(cnt) -> float:
    """k_bwd_sedge, the shadow-edge search and pick: hierarchy nodes, leaf
    edge classifications, exact silhouette tests and clips."""
    k = K_SEDGE
    return (cnt[k + 2] * EDGE_NODE_VISIT + cnt[k + 3] * EDGE_TEST + cnt[k + 4] * CLIP_TEST
            + cnt[k + 5] * EDGE_CLASSIFY)


def sedge_add_flops(cnt) -> float:
    """k_bwd_sedge_add, the contributions of the picks: their shadow rays."""
    return cnt[K_SEDGE] * NODE_VISIT + cnt[K_SEDGE + 1] * TRI_TEST


def fp32_peak_tflops(sm_mhz: float, sm_count: int) -> float:
    """Nominal FP32 peak from the device's SM count and a clock (context for
    the measured FMA peak, which is the denominator)."""
    return sm_count * FP32_LANES * 2 * sm_mhz * 1e6 / 1e12
