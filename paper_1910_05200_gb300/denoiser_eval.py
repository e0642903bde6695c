"""Train the per-pixel denoiser and measure what it buys: error and time of the
denoised low-spp path against the plain path at equal error.

The network (denoise.cu) is trained on pairs (4-spp features, high-spp
radiance) that the renderer itself produces from faces with random shape,
expression, albedo, specular map and pose under one light-stage
configuration.  On held-out faces it reports, against a high-spp reference:
* image rRMSE of the plain render at each spp of a sweep and of the denoised
  4-spp render, and the plain spp with the same error (error ~ spp^-1/2);
* gradient rRMSE (loss = |image - target|^2, 1,340 parameters) of the plain
  gradient at each spp and of two denoised gradients at 4 spp: "jacobian"
  back-propagates the denoised loss through the network (J^T applied to the
  image adjoint), "residual" hands the renderer the adjoint 2 (denoised -
  target) directly (the network cleans the residual, not the derivative);
* device time per fwd+bwd at each spp and of the network, and the speedup
  T_plain(equal-error spp) / T_denoised(4 spp).

    python -m paper_1910_05200_gb300.denoiser_eval [--quick]
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np
import torch

from . import facert
from . import synthetic as S

NIN = 14


def init_weights(aov, sout, seed=0):
    """He-uniform hidden layers, zero output layer (starts at the identity),
    standardisation constants from the training features."""
    rng = np.random.default_rng(seed)
    parts = []
    for n_out, n_in in [(64, 14), (64, 64), (64, 64)]:
        lim = math.sqrt(6.0 / n_in)
        parts += [rng.uniform(-lim, lim, (n_out, n_in)).ravel(), np.zeros(n_out)]
    parts += [np.zeros(3 * 64), np.zeros(3)]
    x = aov.reshape(-1, NIN).astype(np.float64).copy()
    x[:, 12] = np.sqrt(np.maximum(x[:, 12], 0))
    parts += [x.mean(0), 1.0 / np.maximum(x.std(0), 1e-6), np.array([sout])]
    return np.concatenate(parts).astype(np.float32)


def rrmse(x, ref):
    return float(torch.linalg.norm((x - ref).double()) / torch.linalg.norm(ref.double()))


def timed(fn, reps=3):
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    fn()
    torch.cuda.synchronize()
    ev0.record()
    for _ in range(reps):
        fn()
    ev1.record()
    torch.cuda.synchronize()
    return ev0.elapsed_time(ev1) / reps


def run(quick=False, device=0):
    dev = torch.device("cuda", device)
    scene, _, c = S.make_workload("full", seed=1)
    W, H = c["W"], c["H"]
    n_train = 8 if quick else 32
    n_test = 2 if quick else 4
    spp_in = 4
    spp_target = 64 if quick else 256
    spp_ref = 1024 if quick else 4096
    r = facert.Renderer(scene, device=device)
    lights_off = S.param_offsets()["lights"]
    lights = S.make_theta(scene, seed=4242, n_on=c["n_on"], max_angle_deg=30, t_std=0.05)[lights_off:]

    def face(seed):
        th = S.make_theta(scene, seed=seed, n_on=c["n_on"], max_angle_deg=30, t_std=0.05)
        th[lights_off:] = lights
        return torch.tensor(th, device=dev)

    # --- training set --------------------------------------------------------
    t0 = time.time()
    X, Y = [], []
    for k in range(n_train):
        th = face(10_000 + k)
        _, aov = r.render(th, W, H, spp_in, seed=k, aov=True)
        X.append(aov.reshape(-1, NIN).clone())
        Y.append(r.render(th, W, H, spp_target, seed=100_000 + k).reshape(-1, 3).clone())
    X, Y = torch.cat(X), torch.cat(Y)
    hit = X[:, 13] > 0
    X, Y = X[hit].contiguous(), Y[hit].contiguous()
    torch.cuda.synchronize()
    t_data = time.time() - t0
    noise = float((X[:, :3] - Y).std())
    r.set_denoiser(init_weights(X.cpu().numpy(), noise))
    steps = 1500 if quick else 6000
    gen = torch.Generator(device=dev).manual_seed(0)
    t0 = time.time()
    losses = []
    for it in range(steps):
        idx = torch.randint(0, X.shape[0], (32768,), device=dev, generator=gen)
        lr = 2e-3 if it < 0.7 * steps else 2e-4
        l = r.denoiser_train_step(X[idx], Y[idx], lr)
        if it % (steps // 10) == 0 or it == steps - 1:
            losses.append(float(l))
    torch.cuda.synchronize()
    t_train = time.time() - t0

    # --- held-out evaluation ----------------------------------------------------
    sweep = [4, 8, 16, 32, 64, 128, 256] + ([] if quick else [1024])
    img_err = {s: [] for s in sweep}
    grad_err = {s: [] for s in sweep}
    den_img_err, den_grad_err, res_grad_err = [], [], []
    for k in range(n_test):
        th = face(90_000 + k)
        target = r.render(face(95_000 + k), W, H, spp_ref, seed=7)
        ref = r.render(th, W, H, spp_ref, seed=11)
        g_ref = r.backward(th, 2 * (ref - target), W, H, spp_ref // 4, seed=13)
        for s in sweep:
            img = r.render(th, W, H, s, seed=20 + s)
            img_err[s].append(rrmse(img, ref))
            g = r.backward(th, 2 * (img - target), W, H, s, seed=20 + s)
            grad_err[s].append(rrmse(g, g_ref))
        img, aov = r.render(th, W, H, spp_in, seed=999, aov=True)
        den, jt = r.denoise(aov, 2 * (r.denoise(aov) - target))
        den_img_err.append(rrmse(den, ref))
        g = r.backward(th, jt, W, H, spp_in, seed=999)
        den_grad_err.append(rrmse(g, g_ref))
        g = r.backward(th, (2 * (den - target)).contiguous(), W, H, spp_in, seed=999)
        res_grad_err.append(rrmse(g, g_ref))
    r.sync()
    e_img = {s: float(np.mean(v)) for s, v in img_err.items()}
    e_grad = {s: float(np.mean(v)) for s, v in grad_err.items()}
    e_den_img, e_den_grad = float(np.mean(den_img_err)), float(np.mean(den_grad_err))
    e_res_grad = float(np.mean(res_grad_err))
    # plain spp with the denoised error, from error ~ spp^-1/2 through the 4-spp point
    eq_img = spp_in * (e_img[spp_in] / e_den_img) ** 2
    eq_grad = spp_in * (e_grad[spp_in] / min(e_den_grad, e_res_grad)) ** 2

    # --- timing (fwd + bwd per frame) ---------------------------------------------
    th = face(1)
    tgt = r.render(face(2), W, H, 16, seed=3)
    t_plain = {}
    for s in sweep:
        def step(s=s):
            img = r.render(th, W, H, s, seed=5)
            r.backward(th, 2 * (img - tgt), W, H, s, seed=5)
        t_plain[s] = timed(step, reps=2 if s >= 256 else 3)

    def den_step():
        img, aov = r.render(th, W, H, spp_in, seed=5, aov=True)
        den, jt = r.denoise(aov, 2 * (img - tgt))
        r.backward(th, jt, W, H, spp_in, seed=5)
    t_den = timed(den_step)
    aov_t = r.render(th, W, H, spp_in, seed=5, aov=True)[1]
    t_mlp = timed(lambda: r.denoise(aov_t, aov_t[..., :3].contiguous()), reps=10)

    def t_at(spp):   # plain time at a non-swept spp: linear in spp between sweep points
        xs = sorted(t_plain)
        return float(np.interp(spp, xs, [t_plain[x] for x in xs]))

    r.weights_trained = r.denoiser_weights()
    out = {
        "workload": f"full face, {W}x{H}, {c['n_on']} of 20 lights on (fixed), train {n_train} faces, "
                    f"test {n_test} faces",
        "train": {"pixels": int(X.shape[0]), "steps": steps, "data_s": t_data, "train_s": t_train,
                  "loss_curve": losses, "input_spp": spp_in, "target_spp": spp_target},
        "reference_spp": spp_ref,
        "image_rrmse": {"plain": e_img, "denoised_4spp": e_den_img, "plain_spp_at_equal_error": eq_img},
        "gradient_rrmse": {"plain": e_grad, "denoised_4spp_jacobian": e_den_grad,
                           "denoised_4spp_residual": e_res_grad, "plain_spp_at_equal_error": eq_grad},
        "ms_fwd_bwd": {"plain": t_plain, "denoised_4spp": t_den, "mlp_infer_and_adjoint": t_mlp},
        "speedup_at_equal_image_error": t_at(eq_img) / t_den,
        "speedup_at_equal_gradient_error": t_at(eq_grad) / t_den,
        "reaches_1024spp_image_error": e_den_img <= e_img.get(1024, float("nan")),
    }
    out["_weights"] = r.weights_trained
    return out


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--quick", action="store_true")
    ap.add_argument("--save-weights", default="")
    a = ap.parse_args()
    res = run(a.quick)
    w = res.pop("_weights")
    if a.save_weights:
        np.save(a.save_weights, w)
    print(json.dumps(res, indent=1))
