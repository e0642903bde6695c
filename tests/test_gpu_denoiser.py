"""Denoiser on the GPU against the FP64 references, and what training gains.

Tolerances: the kernels round weights, inputs and hidden activations to FP16
(unit roundoff 4.9e-4) and accumulate in FP32 in a different order than the
reference, so an activation next to an FP16 rounding boundary can round the
other way.  Outputs are compared at 2e-3 of their scale, the input adjoint
(four FP16 roundings in its chain) at 5e-3, training gradients (the
tensor-core backward also rounds each layer's gradient to FP16; the FP64
reference does not) at 1e-2 of each layer's largest entry.

Training set: faces with random shape, expression, albedo, specular map and
pose under one fixed light-stage configuration (the capture setting); the
per-pixel features carry no information about the light intensities, so a
network trained across random lighting cannot predict radiance.
"""
import numpy as np
import pytest
import torch

from oracle import default_config, mlp
from paper_1910_05200_gb300 import synthetic as S
from tests.parity import note

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def r(tiny):
    from paper_1910_05200_gb300 import build, facert
    build.build()
    return facert.Renderer(tiny[0], device=0)


def _features(n, seed):
    """Seeded synthetic features spanning the ranges the renderer produces."""
    rng = np.random.default_rng(seed)
    f = np.zeros((n, 14), np.float32)
    f[:, 0:3] = rng.uniform(0, 0.6, (n, 3))
    nrm = rng.normal(size=(n, 3))
    f[:, 3:6] = nrm / np.linalg.norm(nrm, axis=1, keepdims=True)
    f[:, 6:9] = rng.uniform(0.3, 0.7, (n, 3))
    f[:, 9] = rng.uniform(0, 1, n)
    f[:, 10] = rng.uniform(0.7, 1.1, n)
    f[:, 11] = rng.uniform(0, 1, n)
    f[:, 12] = rng.uniform(0, 0.01, n)
    f[:, 13] = rng.choice([0.0, 0.5, 1.0], n)
    return f


@pytest.mark.parametrize("W,H,spp", [(64, 64, 4), (37, 29, 3)])
def test_features_match_oracle(oracle, tiny, r, W, H, spp):
    scene, theta, _ = tiny
    img, aov = r.render(torch.tensor(theta, device="cuda:0"), W, H, spp, seed=4, aov=True)
    r.sync()
    ref_img, ref = oracle.render(default_config(W=W, H=H, spp=spp, seed=4), scene, theta, aov=True)
    got = aov.cpu().numpy().astype(np.float64)
    assert np.allclose(got[..., :3], img.cpu().numpy(), atol=1e-7)
    for k in range(14):
        scale = max(np.abs(ref[..., k]).max(), 1e-12)
        # FP32 interpolation of normals, albedo and the specular map (~1e-6 per op,
        # a few ops); feature 12, E[Y^2] - E[Y]^2, cancels in FP32
        tol = 2e-5 * scale if k != 12 else 1e-4 * scale
        err = np.abs(got[..., k] - ref[..., k]).max()
        note(f"denoiser feature {k} at {W}x{H}x{spp} (relative to its scale)", err / scale, tol / scale,
             n=ref[..., k].size)
        assert err <= tol, (k, err, scale)


def test_inference_and_adjoint_match_reference(r):
    f = _features(1000, 3)            # 1000: several warps and a ragged tail
    w = mlp.init_weights(7, scale_out=1.0, aov=_features(500, 9), sout=0.5)
    r.set_denoiser(w)
    d = np.random.default_rng(4).normal(size=(1000, 3)).astype(np.float32)
    d[::7] *= 1e-6                    # tiny adjoints keep their digits (per-pixel scaling)
    out, jt = r.denoise(torch.tensor(f, device="cuda:0"), torch.tensor(d, device="cuda:0"))
    r.sync()
    y_ref, _ = mlp.forward(w, f)
    jt_ref = mlp.input_adjoint(w, f, d)
    out, jt = out.cpu().numpy(), jt.cpu().numpy()
    e_out = np.abs(out - y_ref) / np.abs(y_ref).max()
    note("denoiser inference (relative to the output scale)", e_out.max(), 2e-3, n=out.size,
         p9999=np.quantile(e_out, 0.9999))
    assert np.abs(out - y_ref).max() <= 2e-3 * np.abs(y_ref).max()
    rel = np.abs(jt - jt_ref) / (np.abs(jt_ref).max(axis=1, keepdims=True) + 1e-30)
    note("denoiser input adjoint J^T (relative to each pixel's largest)", rel.max(), 5e-3, n=rel.size,
         p9999=np.quantile(rel, 0.9999))
    assert rel.max() <= 5e-3, rel.max()     # four FP16 roundings along the adjoint chain
    # inference alone gives the same output
    out2 = r.denoise(torch.tensor(f, device="cuda:0")).cpu().numpy()
    assert np.array_equal(out2, out)


def test_train_step_gradient_and_update(r):
    f = _features(3000, 5)
    w = mlp.init_weights(11, scale_out=1.0, aov=f, sout=0.5)
    r.set_denoiser(w)
    tgt = np.random.default_rng(6).uniform(0, 0.6, (3000, 3)).astype(np.float32)
    lr = 1e-3
    loss = r.denoiser_train_step(torch.tensor(f, device="cuda:0"), torch.tensor(tgt, device="cuda:0"), lr)
    g = r.denoiser_grad().astype(np.float64)
    w1 = r.denoiser_weights().astype(np.float64)
    lref, gref = mlp.loss_and_grad(w, f, tgt)
    note("denoiser training loss", abs(loss.item() - lref) / abs(lref), 1e-4)
    assert loss.item() == pytest.approx(lref, rel=1e-4)
    o = 0
    for name, shape in mlp.SIZES:
        n = int(np.prod(shape))
        gs, rs = g[o:o + n], gref[o:o + n]
        note(f"denoiser training gradient {name} (relative to the layer's largest)",
             np.abs(gs - rs).max() / max(np.abs(rs).max(), 1e-300), 1e-2, n=n)
        assert np.abs(gs - rs).max() <= 1e-2 * np.abs(rs).max() + 1e-12, name
        o += n
    wref, _, _ = mlp.adam_step(w.astype(np.float64), gref, np.zeros_like(gref), np.zeros_like(gref), 1, lr)
    # the first Adam step moves each weight by lr g / (|g| + eps): lr sign(g)
    # wherever |g| >> eps, so equal wherever the sign agrees, up to the relative
    # error of g for gradients near eps (the tensor-core backward rounds each
    # layer's gradient to FP16: about 1e-3 relative)
    agree = np.sign(g) == np.sign(gref)
    assert agree.mean() > 0.99
    assert np.abs(w1 - wref)[agree].max() <= 5e-3 * lr
    assert np.abs(w1 - wref).max() <= 2.0001 * lr


def test_training_reduces_error_on_held_out_faces(r, tiny):
    """What the trained network gains over the plain low-spp render."""
    scene = tiny[0]
    W = H = 64
    dev = "cuda:0"
    lights = S.make_theta(scene, seed=100, n_on=8)[S.param_offsets()["lights"]:]

    def face(seed):
        th = S.make_theta(scene, seed=seed, n_on=8)
        th[S.param_offsets()["lights"]:] = lights
        return torch.tensor(th, device=dev)

    feats, tgts = [], []
    for k in range(12):
        th = face(100 + k)
        _, aov = r.render(th, W, H, 4, seed=k, aov=True)
        feats.append(aov.reshape(-1, 14).clone())
        tgts.append(r.render(th, W, H, 256, seed=1000 + k).reshape(-1, 3).clone())
    X = torch.cat(feats)
    Y = torch.cat(tgts)
    noise = (X[:, :3] - Y).std().item()
    r.set_denoiser(mlp.init_weights(0, scale_out=0.0, aov=X.cpu().numpy(), sout=noise))
    gen = torch.Generator(device=dev).manual_seed(0)
    for it in range(3000):
        idx = torch.randint(0, X.shape[0], (16384,), device=dev, generator=gen)
        r.denoiser_train_step(X[idx], Y[idx], 2e-3 if it < 2000 else 2e-4)
    errs_noisy, errs_den = [], []
    for k in range(3):
        th = face(900 + k)
        img, aov = r.render(th, W, H, 4, seed=77 + k, aov=True)
        ref = r.render(th, W, H, 1024, seed=5000 + k)
        den = r.denoise(aov)
        nrm = torch.linalg.norm(ref)
        errs_noisy.append((torch.linalg.norm(img - ref) / nrm).item())
        errs_den.append((torch.linalg.norm(den - ref) / nrm).item())
    r.sync()
    print("rRMSE noisy", errs_noisy, "denoised", errs_den)
    # a per-pixel network only sees noisy features: the gain is modest but clear
    assert np.mean(errs_den) < 0.9 * np.mean(errs_noisy)
