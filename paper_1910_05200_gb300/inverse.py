"""Inverse rendering: recover face, reflectance, pose and lights from an image.

Optimization paragraph: argmin E_data + w1 E_prior + w2 E_light over
alpha, beta, delta, c_spec, [R t] and the lights, in stages after the
multi-step strategy of Garrido et al. 2016 with a specular step and a light
step added.  Reading used here (the stage contents of Garrido et al.'s
Algorithm 1 are not in the paper):

    1. pose and lights           (rigid alignment, coarse lighting)
    2. + identity and expression (geometry)
    3. albedo and lights         (diffuse reflectance)
    4. specular map              (the added Cook-Torrance step)
    5. lights                    (the added light step)

Every step of an iteration runs in the library: render, loss and gradient
in one fr_step call (or, with the denoiser, render with its features, the
network, loss and gradient as separate calls), then Adam (fr_adam_step; a
learning rate of 0 freezes a group).  Samples change every iteration
(Philox key (seed, iter)).
"""
from __future__ import annotations

import dataclasses

import numpy as np
import torch

from . import synthetic as S

STAGES = [
    ("pose+lights", 0.2, ("pose_r", "pose_t", "lights")),
    ("identity+expression", 0.3, ("pose_r", "pose_t", "alpha", "beta", "lights")),
    ("albedo", 0.2, ("delta", "lights")),
    ("specular", 0.15, ("cspec",)),
    ("lights", 0.15, ("lights",)),
]
LEARNING_RATES = dict(alpha=0.05, beta=0.05, delta=0.05, cspec=0.02, pose_r=0.004, pose_t=0.002, lights=0.02)


def schedule(n_iter: int):
    """Stage index of every iteration (stages in order, lengths by fraction)."""
    bounds = np.cumsum([f for _, f, _ in STAGES])
    bounds = np.round(bounds / bounds[-1] * n_iter).astype(int)
    out = np.zeros(n_iter, np.int32)
    lo = 0
    for k, hi in enumerate(bounds):
        out[lo:hi] = k
        lo = hi
    return out


def group_slices(K=(S.K_ID, S.K_EXP, S.K_ALB)):
    o = S.param_offsets(*K)
    return dict(alpha=slice(o["alpha"], o["beta"]), beta=slice(o["beta"], o["delta"]),
                delta=slice(o["delta"], o["cspec"]), cspec=slice(o["cspec"], o["pose"]),
                pose_r=slice(o["pose"], o["pose"] + 3), pose_t=slice(o["pose"] + 3, o["lights"]),
                lights=slice(o["lights"], o["total"]))


def lr_vector(groups, K=(S.K_ID, S.K_EXP, S.K_ALB), rates=LEARNING_RATES):
    sl = group_slices(K)
    lr = np.zeros(S.param_offsets(*K)["total"], np.float32)
    for g in groups:
        lr[sl[g]] = rates[g]
    return lr


def initial_theta(K=(S.K_ID, S.K_EXP, S.K_ALB), light=0.8):
    """Mean face, grey specular map, frontal pose, every light on at `light`."""
    o = S.param_offsets(*K)
    th = np.zeros(o["total"], np.float32)
    th[o["cspec"]:o["pose"]] = 0.5
    th[o["lights"]:] = light
    return th


@dataclasses.dataclass
class Result:
    theta: np.ndarray
    loss: np.ndarray        # per iteration
    ms_per_iter: float


def save_checkpoint(path, it, step_in_stage, theta, mom, vel, losses):
    """The state of optimize() after `it` iterations, written atomically
    (a temporary file renamed over the target)."""
    import os
    tmp = f"{path}.tmp{os.getpid()}.npz"
    np.savez(tmp, it=np.int64(it), step_in_stage=np.int64(step_in_stage), theta=theta.cpu().numpy(),
             mom=mom.cpu().numpy(), vel=vel.cpu().numpy(), losses=losses.cpu().numpy())
    os.replace(tmp, path)


def optimize(r, target, W, H, spp, iters=500, seed=0, theta0=None, w1=0.02, w2=0.002, m=None,
             denoise=False, rates=LEARNING_RATES, api="step", checkpoint=None, checkpoint_every=50,
             resume=None, stop_after=None) -> Result:
    """Fit theta to the target image [H, W, 3] (device).  With denoise, the
    loss is taken on the denoised render and its residual is the image
    adjoint handed to the renderer (the network must be set on r).  api
    "calls" runs render, loss and backward as three calls instead of fr_step
    (same results up to the order of floating-point additions).

    checkpoint: a path where the state (iteration, stage step, theta, Adam
    moments, losses) is saved every checkpoint_every iterations and at the
    end; resume: a path written that way, from which the run continues (the
    samples of iteration i depend only on (seed, i), so a resumed run draws
    what an uninterrupted one would); stop_after: end after this many
    iterations of the schedule (a run interrupted on purpose)."""
    dev = r.device
    th = torch.tensor(initial_theta() if theta0 is None else theta0, device=dev)
    P = th.numel()
    mom = torch.zeros(P, device=dev)
    vel = torch.zeros(P, device=dev)
    grad = torch.zeros(P, device=dev, dtype=torch.float64)
    d_image = torch.empty(H, W, 3, device=dev)
    image = torch.empty(H, W, 3, device=dev)
    stages = schedule(iters)
    lrs = [torch.tensor(lr_vector(g, rates=rates), device=dev) for _, _, g in STAGES]
    losses = torch.zeros(iters, device=dev, dtype=torch.float64)
    step_in_stage = 0
    start = 0
    if resume is not None:
        z = np.load(resume)
        start, step_in_stage = int(z["it"]), int(z["step_in_stage"])
        th.copy_(torch.from_numpy(z["theta"]))
        mom.copy_(torch.from_numpy(z["mom"]))
        vel.copy_(torch.from_numpy(z["vel"]))
        losses[: len(z["losses"])] = torch.from_numpy(z["losses"][:iters])
    end = iters if stop_after is None else min(iters, stop_after)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for it in range(start, end):
        if it > 0 and stages[it] != stages[it - 1]:
            mom.zero_()
            vel.zero_()
            step_in_stage = 0
        step_in_stage += 1
        if denoise or api != "step":
            if denoise:
                _, aov = r.render(th, W, H, spp, seed=seed, iter=it, aov=True)
                img = r.denoise(aov)
            else:
                img = r.render(th, W, H, spp, seed=seed, iter=it, out=image)
            grad.zero_()
            losses[it:it + 1] = r.loss(th, img, target, m=m, w1=w1, w2=w2, d_image=d_image, grad=grad)
            r.backward(th, d_image, W, H, spp, seed=seed, iter=it, grad=grad, accumulate=True)
        else:
            losses[it:it + 1] = r.step(th, target, W, H, spp, seed=seed, iter=it, m=m, w1=w1, w2=w2,
                                       image=image, d_image=d_image, grad=grad)[1]
        r.adam_step(th, grad, mom, vel, lrs[stages[it]], step_in_stage)
        if checkpoint is not None and (it + 1) % checkpoint_every == 0:
            save_checkpoint(checkpoint, it + 1, step_in_stage, th, mom, vel, losses)
    ev1.record()
    torch.cuda.synchronize()
    if checkpoint is not None:
        save_checkpoint(checkpoint, end, step_in_stage, th, mom, vel, losses)
    return Result(th.cpu().numpy(), losses.cpu().numpy(), ev0.elapsed_time(ev1) / max(1, end - start))


def parameter_errors(theta, truth, K=(S.K_ID, S.K_EXP, S.K_ALB)):
    """Per-group error against the ground truth: relative RMSE for the
    coefficient groups and the lights, degrees and units for the pose."""
    sl = group_slices(K)
    out = {}
    for g in ("alpha", "beta", "delta", "cspec", "lights"):
        t = truth[sl[g]].astype(np.float64)
        out[g] = float(np.linalg.norm(theta[sl[g]] - t) / max(np.linalg.norm(t), 1e-12))
    out["rotation_deg"] = float(np.degrees(np.abs(theta[sl["pose_r"]] - truth[sl["pose_r"]]).max()))
    out["translation"] = float(np.abs(theta[sl["pose_t"]] - truth[sl["pose_t"]]).max())
    return out


def evaluate(n_targets=16, iters=500, spp_lo=4, spp_hi=64, device=0, denoiser_pairs=512, denoiser_steps=8000):
    """Full-face inverse problems (256x256): targets rendered at 256 spp from
    seeded ground truth (14 of 20 lights on, pose within 30 degrees); fits on
    every target at spp_lo plain, spp_lo denoised and spp_hi plain.  The
    denoiser is trained first, in this call, on denoiser_pairs scenes drawn
    like the targets (random lights included; denoiser_eval.make_pairs:
    4-spp features against 1024-spp radiance).  Returns per-variant mean
    parameter errors, final losses, time per iteration and per-target errors."""
    from . import denoiser_eval as D
    from . import facert
    scene, _, c = S.make_workload("full", seed=1)
    W, H = c["W"], c["H"]
    r = facert.Renderer(scene, device=device)
    out = {"workload": f"full face {W}x{H}, {iters} Adam iterations, 5 stages, {n_targets} targets"}
    if denoiser_pairs:
        X, Y, _ = D.make_pairs(r, scene, c, denoiser_pairs, r.device)
        D.train(r, X, Y, denoiser_steps)
        del X, Y
        out["denoiser"] = {"pairs": denoiser_pairs, "steps": denoiser_steps, "input_spp": 4, "target_spp": 1024}
    variants = [("plain_%dspp" % spp_lo, spp_lo, False), ("plain_%dspp" % spp_hi, spp_hi, False)]
    if denoiser_pairs:
        variants.insert(1, ("denoised_%dspp" % spp_lo, spp_lo, True))
    init_err = []
    for name, spp, den in variants:
        errs, losses, ms = [], [], []
        for k in range(n_targets):
            truth = S.make_theta(scene, seed=500 + k, n_on=c["n_on"], max_angle_deg=30, t_std=0.05)
            target = r.render(torch.tensor(truth, device=r.device), W, H, 256, seed=9)
            res = optimize(r, target, W, H, spp, iters=iters, seed=k, denoise=den)
            errs.append(parameter_errors(res.theta, truth))
            losses.append(float(res.loss[-10:].mean()))
            ms.append(res.ms_per_iter)
            if name == variants[0][0]:
                init_err.append(parameter_errors(initial_theta(), truth))
        mean = lambda es: {kk: float(np.mean([e[kk] for e in es])) for kk in es[0]}
        out[name] = {"targets": n_targets, "param_error": mean(errs), "final_loss": float(np.mean(losses)),
                     "ms_per_iter": float(np.mean(ms)), "per_target": errs}
    out["initial_param_error"] = {kk: float(np.mean([e[kk] for e in init_err])) for kk in init_err[0]}
    return out


def iteration_times(iters=60, spps=(4, 64), device=0):
    """Time per inverse iteration (render, loss, gradient, Adam) on the first
    target of evaluate(), through fr_step and through the three calls."""
    from . import facert
    scene, _, c = S.make_workload("full", seed=1)
    W, H = c["W"], c["H"]
    r = facert.Renderer(scene, device=device)
    truth = S.make_theta(scene, seed=500, n_on=c["n_on"], max_angle_deg=30, t_std=0.05)
    target = r.render(torch.tensor(truth, device=r.device), W, H, 256, seed=9)
    out = {}
    for spp in spps:
        for api in ("step", "calls"):
            optimize(r, target, W, H, spp, iters=5, seed=0, api=api)            # warm-up
            out[f"{spp}spp_{api}"] = optimize(r, target, W, H, spp, iters=iters, seed=0, api=api).ms_per_iter
    return out


if __name__ == "__main__":
    import argparse
    import json
    ap = argparse.ArgumentParser()
    ap.add_argument("--targets", type=int, default=16)
    ap.add_argument("--iters", type=int, default=500)
    ap.add_argument("--denoiser-pairs", type=int, default=512)
    ap.add_argument("--times", action="store_true", help="time per iteration only (iteration_times)")
    a = ap.parse_args()
    if a.times:
        print(json.dumps(iteration_times(), indent=1))
    else:
        print(json.dumps(evaluate(n_targets=a.targets, iters=a.iters, denoiser_pairs=a.denoiser_pairs), indent=1))
