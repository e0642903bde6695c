"""Train the per-pixel denoiser on renderer-made pairs and measure what it buys.

Training set (one denoiser configuration of the method's extension: a
per-pixel MLP on the renderer's 14 features, trained on low-spp/high-spp
pairs the renderer itself generates): full-face scenes drawn like the
benchmark workload -- random shape, expression, albedo, specular map, pose
within 30 degrees and random lights (14 of 20 on, intensities U[0, 2]) --
each giving the 4-spp features and the 1024-spp radiance of its face pixels.

Measured on held-out scenes drawn the same way:
* learning curve: held-out image rRMSE of the denoised 4-spp render after
  training on the first n pairs (same number of Adam steps for every n);
* image rRMSE of the plain render at each spp of a sweep and of the denoised
  4-spp render, against a 16,384-spp reference, and the plain spp with the
  denoised error (log-log interpolation over the sweep);
* gradient rRMSE (loss |image - target|^2, all 1,340 parameters) of the plain
  gradient at each spp and of the denoised 4-spp gradient, two ways:
  "jacobian" back-propagates the denoised loss through the network (the
  network's J^T applied to the image adjoint), "residual" hands the renderer
  the adjoint 2 (denoised - target) directly;
* device time of one fwd+loss+bwd at each spp (fr_step) and of the denoised
  path (render with features, network and its adjoint, loss, backward), and
  the speedups, read two ways:
  R1 -- the denoised 4-spp path against the plain path at the spp with the
       same error;
  R2 -- the plain path at 1024 spp against the cheapest plain spp whose
       error is within 1 % rRMSE of the 1024-spp render (the plain path's own
       speedup under the looser reading, reported as context).

    python -m paper_1910_05200_gb300.denoiser_eval [--pairs N] [--quick] [--save-weights F]
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


def loglog_spp(sweep, errs, e):
    """Plain spp at which the error equals e, by log-log interpolation over
    the sweep (extrapolated with error ~ spp^-1/2 beyond its ends)."""
    s = np.log(np.asarray(sweep, np.float64))
    v = np.log(np.asarray([errs[k] for k in sweep], np.float64))
    le = math.log(e)
    if le >= v[0]:
        return float(math.exp(s[0] - 2.0 * (le - v[0])))
    if le <= v[-1]:
        return float(math.exp(s[-1] - 2.0 * (le - v[-1])))
    for i in range(len(s) - 1):
        if v[i] >= le >= v[i + 1]:
            t = (le - v[i]) / (v[i + 1] - v[i]) if v[i + 1] != v[i] else 0.0
            return float(math.exp(s[i] + t * (s[i + 1] - s[i])))
    return float("nan")


def scene_theta(scene, c, seed, dev):
    """A scene drawn like the benchmark workload: shape, expression, albedo,
    specular map, pose and lights (14 of 20 on) all random."""
    th = S.make_theta(scene, seed=seed, n_on=c["n_on"], max_angle_deg=30, t_std=0.05)
    return torch.tensor(th, device=dev)


def make_pairs(r, scene, c, pairs, dev, spp_in=4, spp_target=1024):
    """Face pixels of (spp_in features, spp_target radiance) for scenes drawn
    like the benchmark workload (seeds 10,000 + k).  Returns X [n, 14], Y [n, 3]
    and the first pixel of each pair."""
    W, H = c["W"], c["H"]
    X, Y, bounds = [], [], [0]
    for k in range(pairs):
        th = scene_theta(scene, c, 10_000 + k, dev)
        _, aov = r.render(th, W, H, spp_in, seed=k, aov=True)
        y = r.render(th, W, H, spp_target, seed=100_000 + k)
        hit = aov[..., 13].reshape(-1) > 0
        X.append(aov.reshape(-1, NIN)[hit].clone())
        Y.append(y.reshape(-1, 3)[hit].clone())
        bounds.append(bounds[-1] + int(hit.sum()))
    return torch.cat(X), torch.cat(Y), bounds


def train(r, X, Y, steps, seed=0, batch=32768):
    noise = float((X[:, :3] - Y).std())
    r.set_denoiser(init_weights(X[: min(X.shape[0], 1 << 20)].cpu().numpy(), noise, seed=seed))
    gen = torch.Generator(device=X.device).manual_seed(seed)
    losses = []
    for it in range(steps):
        idx = torch.randint(0, X.shape[0], (batch,), device=X.device, generator=gen)
        lr = 2e-3 if it < 0.7 * steps else 2e-4
        loss = r.denoiser_train_step(X[idx], Y[idx], lr)
        if it % max(1, steps // 10) == 0 or it == steps - 1:
            losses.append(float(loss))
    return losses


def run(pairs=512, quick=False, device=0):
    dev = torch.device("cuda", device)
    scene, _, c = S.make_workload("full", seed=1)
    W, H = c["W"], c["H"]
    if quick:
        pairs = min(pairs, 16)
    n_test = 2 if quick else 4
    spp_in, spp_target = 4, (256 if quick else 1024)
    spp_ref = 4096 if quick else 16384
    steps = 1500 if quick else 8000
    r = facert.Renderer(scene, device=device)

    # --- training pairs (face pixels of 4-spp features and high-spp radiance) -------
    t0 = time.time()
    X, Y, bounds = make_pairs(r, scene, c, pairs, dev, spp_in, spp_target)
    torch.cuda.synchronize()
    t_data = time.time() - t0

    # --- held-out scenes ---------------------------------------------------------------
    tests = []
    for k in range(n_test):
        th = scene_theta(scene, c, 90_000 + k, dev)
        target = r.render(scene_theta(scene, c, 95_000 + k, dev), W, H, spp_target, seed=7)
        ref = r.render(th, W, H, spp_ref, seed=11)
        ref1024 = r.render(th, W, H, spp_target, seed=12)
        img4, aov4 = r.render(th, W, H, spp_in, seed=999, aov=True)
        tests.append(dict(th=th, target=target, ref=ref, ref1024=ref1024, img4=img4, aov4=aov4))

    # --- learning curve: fresh networks on the first n pairs ------------------------
    curve = []
    sizes = sorted({max(1, pairs // d) for d in (16, 8, 4, 2, 1)})
    for n in sizes:
        t0 = time.time()
        losses = train(r, X[: bounds[n]], Y[: bounds[n]], steps)
        t_tr = time.time() - t0
        e = [rrmse(r.denoise(t["aov4"]), t["ref"]) for t in tests]
        curve.append({"pairs": n, "pixels": bounds[n], "heldout_image_rrmse": float(np.mean(e)),
                      "final_train_loss": losses[-1], "train_s": t_tr})
    losses_full = losses            # the last network saw every pair

    # --- plain sweep and the denoised 4-spp path (the network trained on all pairs) ---
    sweep = [4, 8, 16, 32, 64, 128, 256, 1024]
    img_err = {s: [] for s in sweep}
    grad_err = {s: [] for s in sweep}
    err_vs_1024 = {s: [] for s in sweep}
    den_img, den_grad_j, den_grad_r = [], [], []
    for t in tests:
        th, target, ref = t["th"], t["target"], t["ref"]
        g_ref = r.backward(th, 2 * (ref - target), W, H, spp_ref // 4, seed=13)
        for s in sweep:
            img = r.render(th, W, H, s, seed=20 + s)
            img_err[s].append(rrmse(img, ref))
            err_vs_1024[s].append(rrmse(img, t["ref1024"]))
            g = r.backward(th, 2 * (img - target), W, H, s, seed=20 + s)
            grad_err[s].append(rrmse(g, g_ref))
        den = r.denoise(t["aov4"])
        den_img.append(rrmse(den, ref))
        den2, jt = r.denoise(t["aov4"], 2 * (den - target))
        den_grad_j.append(rrmse(r.backward(th, jt, W, H, spp_in, seed=999), g_ref))
        den_grad_r.append(rrmse(r.backward(th, (2 * (den - target)).contiguous(), W, H, spp_in, seed=999), g_ref))
    r.sync()
    mean = lambda d: {k: float(np.mean(v)) for k, v in d.items()}
    e_img, e_grad, e_1024 = mean(img_err), mean(grad_err), mean(err_vs_1024)
    e_den_img = float(np.mean(den_img))
    e_den_gj, e_den_gr = float(np.mean(den_grad_j)), float(np.mean(den_grad_r))
    eq_img = loglog_spp(sweep, e_img, e_den_img)
    eq_grad = loglog_spp(sweep, e_grad, min(e_den_gj, e_den_gr))

    # --- time of one fwd+loss+bwd ---------------------------------------------------------
    th = tests[0]["th"]
    tgt = tests[0]["target"]
    t_plain = {}
    for s in sweep:
        t_plain[s] = timed(lambda s=s: r.step(th, tgt, W, H, s, seed=5), reps=2 if s >= 256 else 3)
    d_image = torch.empty(H, W, 3, device=dev)
    grad = torch.zeros(r.P, device=dev, dtype=torch.float64)

    def den_step():
        _, aov = r.render(th, W, H, spp_in, seed=5, aov=True)
        den = r.denoise(aov)
        r.loss(th, den, tgt, d_image=d_image, grad=grad)
        r.backward(th, d_image, W, H, spp_in, seed=5, grad=grad, accumulate=True)
    t_den = timed(den_step)
    aov_t = tests[0]["aov4"]
    t_mlp = timed(lambda: r.denoise(aov_t, aov_t[..., :3].contiguous()), reps=10)

    def t_at(spp):
        xs = sorted(t_plain)
        return float(np.interp(spp, xs, [t_plain[x] for x in xs]))

    within1 = [s for s in sweep if e_1024[s] <= 0.01]
    out = {
        "workload": f"full face {W}x{H}; scenes with random shape, expression, albedo, specular map, pose and "
                    f"lights ({c['n_on']} of 20 on); train {pairs} pairs, test {n_test} scenes",
        "train": {"pairs": pairs, "pixels": int(X.shape[0]), "input_spp": spp_in, "target_spp": spp_target,
                  "steps_per_network": steps, "data_s": t_data, "loss_curve": losses_full},
        "learning_curve": curve,
        "reference_spp": spp_ref,
        "image_rrmse": {"plain": e_img, "denoised_4spp": e_den_img, "plain_spp_at_equal_error": eq_img,
                        "plain_vs_1024spp_render": e_1024},
        "gradient_rrmse": {"plain": e_grad, "denoised_4spp_jacobian": e_den_gj, "denoised_4spp_residual": e_den_gr,
                           "plain_spp_at_equal_error": eq_grad},
        "ms_fwd_bwd": {"plain": t_plain, "denoised_4spp": t_den, "mlp_infer_and_adjoint": t_mlp},
        "R1_speedup_at_equal_image_error": t_at(eq_img) / t_den,
        "R1_speedup_at_equal_gradient_error": t_at(eq_grad) / t_den,
        "R1_denoised_reaches_1024spp_image_error": e_den_img <= e_img[1024],
        "R1_denoised_reaches_1024spp_gradient_error": min(e_den_gj, e_den_gr) <= e_grad[1024],
        "R2_cheapest_plain_spp_within_1pct_of_1024spp": within1[0] if within1 else None,
        "R2_plain_speedup": (t_plain[1024] / t_plain[within1[0]]) if within1 else None,
    }
    out["_weights"] = r.denoiser_weights()
    return out


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--pairs", type=int, default=512)
    ap.add_argument("--quick", action="store_true")
    ap.add_argument("--save-weights", default="")
    a = ap.parse_args()
    res = run(a.pairs, a.quick)
    w = res.pop("_weights")
    if a.save_weights:
        np.save(a.save_weights, w)
    print(json.dumps(res, indent=1))
