"""How much the paper's open readings matter, measured with the renderer.

The Face Modeling paragraph names a Cook-Torrance reflectance and an
isotropically sampled hemisphere of 20 lights without their terms; the
library implements several readings (fr_config: brdf_model, fresnel,
light_layout).  For one seeded full-face parameter vector this reports
* the image difference (relative RMSE at 256 spp) of each reading against
  the default one;
* for each reading, a fit of its own render (the target) with the default
  reading (model mismatch) and with the reading itself (the inverse loop of
  inverse.py): parameter errors against the truth and the final loss;
* for each reading of m_j in E_light (fr_config.light_prior: the given m,
  here zero; the mean of the lights per channel; each light's channel mean),
  a fit of the default render: parameter errors and final loss.

    python -m paper_1910_05200_gb300.readings_eval [--iters N]
"""
from __future__ import annotations

import argparse
import json

import torch

from . import facert, inverse
from . import synthetic as S

READINGS = {
    "default (Beckmann + V-cavity, F in c_spec, Fibonacci lights)": dict(),
    "GGX + Smith": dict(brdf_model=1),
    "Schlick F": dict(fresnel=1),
    "GGX + Smith + Schlick F": dict(brdf_model=1, fresnel=1),
    "icosphere lights": dict(light_layout=1),
}

LIGHT_PRIORS = {"m given (zero)": 0, "mean of the lights per channel": 1, "each light's channel mean": 2}


def _rrmse(x, ref):
    return float(torch.linalg.norm((x - ref).double()) / torch.linalg.norm(ref.double()))


def run(iters=300, spp_fit=16, spp_ref=256, device=0):
    scene, _, c = S.make_workload("full", seed=1)
    W, H = c["W"], c["H"]
    truth = S.make_theta(scene, seed=500, n_on=c["n_on"], max_angle_deg=30, t_std=0.05)
    dev = torch.device("cuda", device)
    th = torch.tensor(truth, device=dev)
    rs = {k: facert.Renderer(scene, device=device, config=facert.default_config(**kw)) for k, kw in READINGS.items()}
    names = list(READINGS)
    base = rs[names[0]]
    ref = base.render(th, W, H, spp_ref, seed=9)
    out = {"workload": f"full face {W}x{H}, truth seed 500, targets at {spp_ref} spp, fits of {iters} Adam "
                       f"iterations at {spp_fit} spp (5 stages)", "readings": {}}
    for name in names:
        r = rs[name]
        target = r.render(th, W, H, spp_ref, seed=9)
        entry = {"image_rrmse_vs_default": _rrmse(target, ref)}
        for label, fitter in (("fit_with_default", base), ("fit_with_itself", r)):
            res = inverse.optimize(fitter, target, W, H, spp_fit, iters=iters, seed=1)
            entry[label] = {"param_error": inverse.parameter_errors(res.theta, truth),
                            "final_loss": float(res.loss[-10:].mean()), "ms_per_iter": res.ms_per_iter}
        out["readings"][name] = entry
    out["light_prior"] = {}
    for name, prior in LIGHT_PRIORS.items():
        r = rs[names[0]] if prior == 0 else \
            facert.Renderer(scene, device=device, config=facert.default_config(light_prior=prior))
        res = inverse.optimize(r, ref, W, H, spp_fit, iters=iters, seed=1)
        out["light_prior"][name] = {"param_error": inverse.parameter_errors(res.theta, truth),
                                    "final_loss": float(res.loss[-10:].mean()), "ms_per_iter": res.ms_per_iter}
        r.sync()
    for r in rs.values():
        r.sync()
    return out


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--iters", type=int, default=300)
    a = ap.parse_args()
    print(json.dumps(run(a.iters), indent=1))
