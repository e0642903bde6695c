"""Batched frames: 32 frames of the 35,709-vertex face with crops of 128 to 320
pixels, 16 spp, one CUDA graph per step (geometry, render + loss + backward of
all frames in phased launches or one persistent launch, geometry adjoints).

Reports the autotuner's table (tuned on 8 of the frames, every fourth by
size, so that the sweep stays short), the step time and throughput of the
full batch with the chosen and the default configuration and with the
fastest configuration of each launch mode (phased, persistent), and the same
frames processed one by one through fr_render / fr_loss /
fr_render_backward.  Targets are the batch's own renders of other
parameters (seed + 1).

    python -m paper_1910_05200_gb300.batch_eval [--steps K] [--reps R]
"""
from __future__ import annotations

import argparse
import json

import numpy as np
import torch

from . import facert
from . import synthetic as S


def _timed(fn, steps):
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    fn(0)
    torch.cuda.synchronize()
    ev0.record()
    for i in range(steps):
        fn(i + 1)
    ev1.record()
    torch.cuda.synchronize()
    return ev0.elapsed_time(ev1) / steps


def _batch(r, frames, thetas, spp, target_thetas):
    b = facert.Batch(r, frames, spp)
    dev = r.device
    b.set_targets(torch.zeros(b.n_pix, 3, device=dev))
    ts, tf = facert.split_theta(torch.tensor(target_thetas, device=dev))
    _, _, _, tgt = b.step(ts[0], tf, iter=10_000)
    b.set_targets(tgt.clone())
    ts, tf = facert.split_theta(torch.tensor(thetas, device=dev))
    return b, ts[0].contiguous(), tf.contiguous()


def run(steps=5, reps=1, device=0):
    c = S.BATCH
    scene = S.make_scene(c["kind"], seed=0)
    kw = dict(n_on=c["n_on"], max_angle_deg=c["max_angle_deg"], t_std=c["t_std"])
    frames, thetas = S.make_batch(scene, n_frames=c["n_frames"], seed=c["seed"], **kw)
    _, target_thetas = S.make_batch(scene, n_frames=c["n_frames"], seed=c["seed"] + 1, **kw)
    spp = c["spp"]
    samples = sum(w * h for w, h, _ in frames) * spp
    r = facert.Renderer(scene, device=device)

    # --- autotune on 8 frames spanning the crop sizes --------------------------
    order = np.argsort([w * h for w, h, _ in frames])
    sub = sorted(order[::4].tolist())
    bs, ts_s, tf_s = _batch(r, [frames[i] for i in sub], thetas[sub], spp, target_thetas[sub])
    table, chosen = bs.autotune(ts_s, tf_s, reps=reps)
    bs.close()

    # --- full batch: chosen vs default configuration -----------------------------
    b, ts, tf = _batch(r, frames, thetas, spp, target_thetas)
    default = b.config()
    ms_default = _timed(lambda i: b.step(ts, tf, 0.02, 0.002, iter=i, images=False), steps)
    # the fastest configuration of each launch mode on the full batch
    by_mode = {}
    for fused, mode in ((0, "phased"), (1, "persistent")):
        best = min((t for t in table if t["fused"] == fused), key=lambda t: t["ms"])
        b.set_config(best["tile_w"], best["tile_h"], best["block"], best["min_blocks"], fused)
        by_mode[mode] = dict(config=best, ms_per_step=_timed(
            lambda i: b.step(ts, tf, 0.02, 0.002, iter=i, images=False), steps))
    b.set_config(chosen["tile_w"], chosen["tile_h"], chosen["block"], chosen["min_blocks"], chosen["fused"])
    l0 = r.launches()
    ms = _timed(lambda i: b.step(ts, tf, 0.02, 0.002, iter=i, images=False), steps)
    kernels_per_step = (r.launches() - l0) / (steps + 1)

    # --- the same frames one by one through the single-image entry points ------------
    dev = r.device
    th_all = torch.tensor(thetas, device=dev)
    tg = b.split(b.targets)
    d_images = [torch.empty(h, w, 3, device=dev) for w, h, _ in frames]
    grad = torch.zeros(th_all.shape[1], device=dev, dtype=torch.float64)

    def per_frame(i):
        for f, (w, h, seed) in enumerate(frames):
            img = r.render(th_all[f], w, h, spp, seed=seed, iter=i)
            r.loss(th_all[f], img, tg[f], None, None, 0.02, 0.002, d_images[f], grad)
            r.backward(th_all[f], d_images[f], w, h, spp, seed=seed, iter=i, grad=grad, accumulate=True)

    ms_single = _timed(per_frame, max(1, steps // 2))
    g_f = torch.empty_like(grad)
    images = [torch.empty(h, w, 3, device=dev) for w, h, _ in frames]

    def per_frame_step(i):
        for f, (w, h, seed) in enumerate(frames):
            r.step(th_all[f], tg[f], w, h, spp, seed=seed, iter=i, w1=0.02, w2=0.002, image=images[f],
                   d_image=d_images[f], grad=g_f)
            grad.add_(g_f)

    ms_single_step = _timed(per_frame_step, max(1, steps // 2))
    r.sync()
    return {
        "workload": f"{len(frames)} frames, full face (35,709 verts / 70,789 tris), square crops "
                    f"{min(w for w, _, _ in frames)}..{max(w for w, _, _ in frames)}, {spp} spp, "
                    f"{c['n_on']} of 20 lights on, shared alpha/delta/c_spec",
        "samples_per_step": samples,
        "autotune": {"frames": len(sub), "reps": reps, "table": table, "chosen": chosen},
        "default_config": default,
        "ms_per_step_default": ms_default,
        "full_batch_by_mode": by_mode,
        "ms_per_step": ms,
        "msamples_per_s": samples / ms / 1e3,
        "kernels_per_step": kernels_per_step,
        "ms_per_step_single_image_calls": ms_single,
        "speedup_vs_single_image_calls": ms_single / ms,
        "ms_per_step_single_image_fr_step": ms_single_step,
        "speedup_vs_single_image_fr_step": ms_single_step / ms,
    }


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--reps", type=int, default=1)
    a = ap.parse_args()
    print(json.dumps(run(a.steps, a.reps), indent=1))
