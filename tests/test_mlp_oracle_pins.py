"""Pins of the FP64 denoiser reference (oracle/mlp.py) and of the oracle's
per-pixel denoiser features.

* backward and input adjoint against central differences of the forward
  (FP16 rounding switched off so that the function is smooth)
* Adam's first step in closed form (update = lr * sign(g) up to eps)
* zero hidden weights reduce the network to rgb + coverage * s_out * b4
* features of a plane facing the camera: normal, albedo, depth, coverage
"""
import numpy as np
import pytest

from oracle import default_config, mlp
from tests import closed_forms as CF


@pytest.fixture
def smooth(monkeypatch):
    monkeypatch.setattr(mlp, "h16", lambda x: np.asarray(x, np.float64))
    return mlp


def _batch(n=7, seed=0):
    rng = np.random.default_rng(seed)
    aov = rng.uniform(0, 1, size=(n, 14))
    aov[:, 3:6] = rng.normal(size=(n, 3))
    return aov


def test_weight_gradient_matches_central_differences(smooth):
    w = smooth.init_weights(3, scale_out=1.0, aov=_batch(40, 9), sout=0.7).astype(np.float64)
    aov = _batch()
    tgt = np.random.default_rng(1).uniform(size=(7, 3))
    _, g = smooth.loss_and_grad(w, aov, tgt)
    rng = np.random.default_rng(2)
    n_trained = sum(int(np.prod(sh)) for name, sh in smooth.SIZES if name in smooth.TRAINED)
    for idx in list(rng.choice(n_trained, 40, replace=False)) + [n_trained - 1, n_trained - 4]:
        wp, wm = w.copy(), w.copy()
        h = 1e-6
        wp[idx] += h
        wm[idx] -= h
        fd = (smooth.loss_and_grad(wp, aov, tgt)[0] - smooth.loss_and_grad(wm, aov, tgt)[0]) / (2 * h)
        assert g[idx] == pytest.approx(fd, rel=1e-5, abs=1e-9)


def test_input_adjoint_matches_central_differences(smooth):
    aov = _batch(5, 3)
    w = smooth.init_weights(4, scale_out=1.0, aov=_batch(40, 9), sout=0.7).astype(np.float64)
    d = np.random.default_rng(5).normal(size=(5, 3))
    jt = smooth.input_adjoint(w, aov, d)
    for c in range(3):
        ap, am = aov.copy(), aov.copy()
        ap[:, c] += 1e-6
        am[:, c] -= 1e-6
        fd = ((smooth.forward(w, ap)[0] - smooth.forward(w, am)[0]) * d).sum(1) / 2e-6
        assert np.allclose(jt[:, c], fd, rtol=1e-5, atol=1e-9)


def test_adam_first_step_closed_form():
    g = np.array([0.3, -2.0, 1e-3, 0.0])
    w, m, v = mlp.adam_step(np.zeros(4), g, np.zeros(4), np.zeros(4), 1, lr=0.01)
    # bias-corrected m / sqrt(v) = g / |g| on the first step
    assert np.allclose(w[:3], -0.01 * np.sign(g[:3]), rtol=1e-4)
    assert w[3] == 0.0


def test_zero_hidden_weights_is_identity_plus_bias():
    d = mlp.unpack(mlp.init_weights(0, aov=_batch(50, 1), sout=0.5))
    for k in ("W1", "W2", "W3", "W4"):
        d[k][:] = 0
    d["b4"][:] = [0.25, -0.5, 0.125]
    aov = _batch(9, 7)
    aov[0, 13] = 0.0                   # a background pixel passes through
    y, _ = mlp.forward(mlp.pack(d).astype(np.float32), aov)
    expect = aov[:, :3] + aov[:, 13:14] * 0.5 * np.array([0.25, -0.5, 0.125])
    assert np.allclose(y, expect, atol=0, rtol=1e-15)
    assert np.array_equal(y[0], aov[0, :3])


def test_standardisation_constants_get_no_gradient(smooth):
    aov = _batch(20, 8)
    w = smooth.init_weights(2, scale_out=1.0, aov=aov, sout=0.3)
    _, g = smooth.loss_and_grad(w, aov, np.zeros((20, 3)))
    n_trained = sum(int(np.prod(sh)) for name, sh in smooth.SIZES if name in smooth.TRAINED)
    assert np.all(g[n_trained:] == 0) and np.abs(g[:n_trained]).max() > 0


def test_plane_features(oracle):
    verts = [(-2, -2, 0), (2, -2, 0), (2, 2, 0), (-2, 2, 0)]
    sc = CF.plain_scene(verts, [(0, 1, 2), (0, 2, 3)])
    th = CF.plain_theta(lights_on=[5, 12, 19], cspec=0.25)
    cfg = default_config(W=8, H=8, spp=4)
    img, f = oracle.render(cfg, sc, th, aov=True)
    assert np.allclose(f[..., :3], img)
    assert np.allclose(f[..., 3:6], [0, 0, 1], atol=1e-12)       # shading normal
    assert np.allclose(f[..., 6:9], np.pi, atol=1e-6)            # albedo (plain scene: pi)
    assert np.allclose(f[..., 9], 0.25, atol=1e-9)               # specular map value
    assert np.allclose(f[..., 13], 1.0)                          # every sample hits
    assert np.allclose(f[..., 11], 1.0)                          # lights above the plane, no occluder
    # depth: distance along each ray to z = 0, divided by d_cam, between 1 and 1/cos(half fov)
    assert np.all(f[..., 10] >= 1.0 - 1e-9) and np.all(f[..., 10] <= 1.0 / np.cos(np.arctan(0.275 * np.sqrt(2))) + 1e-9)
    assert np.all(f[..., 12] >= 0)
