"""Refitted against rebuilt hierarchies: the cost of building the triangle
and edge hierarchies once from the mean shape and refitting them to every
pose and expression.

For seeded full-face scenes at poses up to 30 degrees, the posed vertices of
the library (fr_geometry) become the mean shape of a second context without
bases and at zero pose, whose hierarchies are therefore built on the posed
shape itself.  The two contexts render the same geometry (the images must
agree to FP32 rounding), and the work counters of one render and one
gradient give the node visits of the rays and of the shadow-edge searches
of each.

    python -m paper_1910_05200_gb300.bvh_eval [--scenes N]
"""
from __future__ import annotations

import argparse
import json

import numpy as np
import torch

from . import facert
from . import roofline as RF
from . import synthetic as S


def counts(r, th, W, H, spp, seed):
    r.set_counters(True)
    img = r.render(th, W, H, spp, seed=seed)
    c_fwd = r.counters().copy()
    r.backward(th, torch.ones_like(img), W, H, spp, seed=seed)
    c_bwd = r.counters().copy()
    r.set_counters(False)
    return img, c_fwd, c_bwd


def run(n_scenes=4, device=0):
    scene, _, c = S.make_workload("full", seed=1)
    W, H, spp = c["W"], c["H"], c["spp"]
    r = facert.Renderer(scene, device=device)
    rows = []
    for k in range(n_scenes):
        theta = S.make_theta(scene, seed=700 + k, n_on=c["n_on"], max_angle_deg=30, t_std=0.05)
        th = torch.tensor(theta, device=r.device)
        X = r.geometry(th)["X"].cpu().numpy()
        o = S.param_offsets()
        posed = S.Scene(X.astype(np.float32), scene.tris, scene.uv, np.zeros((3 * scene.V, 0), np.float32),
                        np.zeros((3 * scene.V, 0), np.float32),
                        (scene.alb_mean + scene.B_alb.astype(np.float64) @ theta[o["delta"]:o["cspec"]]).astype(
                            np.float32),
                        np.zeros((3 * scene.V, 0), np.float32))
        r2 = facert.Renderer(posed, device=device)
        th2 = np.concatenate([theta[o["cspec"]:o["pose"]], np.zeros(6, np.float32), theta[o["lights"]:]])
        th2 = torch.tensor(th2.astype(np.float32), device=r.device)
        img1, f1, b1 = counts(r, th, W, H, spp, seed=k)
        img2, f2, b2 = counts(r2, th2, W, H, spp, seed=k)
        n = W * H * spp
        rows.append({
            "scene": k, "rotation_deg": float(np.degrees(np.abs(theta[o["pose"]:o["pose"] + 3]).max())),
            "image_max_rel_diff": float((img1 - img2).abs().max() / img1.abs().max()),
            "forward_ray_nodes_per_sample": {"refit": float(f1[0] / n), "rebuilt": float(f2[0] / n)},
            "forward_tri_tests_per_sample": {"refit": float(f1[1] / n), "rebuilt": float(f2[1] / n)},
            "shadow_edge_hierarchy_node_visits": {"refit": int(b1[RF.K_SEDGE + 2]), "rebuilt": int(b2[RF.K_SEDGE + 2])},
            "shadow_edge_lane_edge_tests": {"refit": int(b1[RF.K_SEDGE + 3]), "rebuilt": int(b2[RF.K_SEDGE + 3])},
            "backward_ray_nodes": {"refit": int(sum(b1[k] for k in (RF.K_INTERIOR, RF.K_PEDGE, RF.K_SEDGE))),
                                   "rebuilt": int(sum(b2[k] for k in (RF.K_INTERIOR, RF.K_PEDGE, RF.K_SEDGE)))},
        })
        del r2
    r.sync()
    return {"workload": f"full face {W}x{H}, {spp} spp, {c['n_on']} of 20 lights on, poses up to 30 degrees",
            "scenes": rows}


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--scenes", type=int, default=4)
    a = ap.parse_args()
    print(json.dumps(run(a.scenes), indent=1))
