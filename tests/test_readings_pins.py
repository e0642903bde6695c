"""Pins of the alternative readings (configuration switches) in the oracle.

The paper names a Cook-Torrance reflectance and an isotropically sampled
hemisphere of 20 lights without their terms.  Besides the default reading
(Beckmann + V-cavity, F folded into c_spec, Fibonacci points), the library and
the oracle implement GGX with Smith masking, Schlick's Fresnel term and an
icosphere dome.  Each is checked here against facts that do not come from
retyping its formula:
* reciprocity, and the closed form at normal incidence,
  f = rho/pi + c_s / (4 pi m^2), which both distributions share;
* Schlick equals the folded reading at c_s = 1 and never falls below it;
* the directional albedo of the specular lobe is at most 1 and near 1 for a
  smooth GGX surface seen head-on (it fails for a wrong normalisation of the
  distribution or a wrong masking term);
* the oracle's gradient is the exact derivative of its own estimate
  (linearity in lights and texels, finite differences in geometry);
* the icosphere directions are the upper half of a once-subdivided
  icosahedron: every nearest-neighbour angle is atan(2)/2 or 36 degrees.
"""
import math

import numpy as np
import pytest

from oracle import default_config
from paper_1910_05200_gb300 import synthetic as S

VARIANTS = [(1, 0), (0, 1), (1, 1)]          # (brdf_model, fresnel); (0, 0) is pinned in test_oracle_pins


def _hemi(rng, k):
    v = rng.normal(size=(k, 3))
    v[:, 2] = np.abs(v[:, 2]) + 0.05
    return v / np.linalg.norm(v, axis=1, keepdims=True)


@pytest.mark.parametrize("model,fresnel", VARIANTS)
def test_brdf_reciprocity_and_normal_incidence(oracle, model, fresnel):
    cfg = default_config(brdf_model=model, fresnel=fresnel)
    n = np.array([0.0, 0.0, 1.0])
    rng = np.random.default_rng(3)
    for a, b in zip(_hemi(rng, 60), _hemi(rng, 60)):
        f1 = oracle.brdf(cfg, n, a, b, 0.0, 0.6)
        f2 = oracle.brdf(cfg, n, b, a, 0.0, 0.6)
        assert f1 > 0 and abs(f1 - f2) <= 1e-12 * max(1.0, f1)
    for m in (0.2, 0.3, 0.5):
        c = default_config(brdf_model=model, fresnel=fresnel, beckmann_m=m)
        m32 = float(np.float32(m))
        for rho, cs in ((0.0, 1.0), (0.4, 0.25), (0.7, 0.0)):
            f = oracle.brdf(c, n, n, n, rho, cs)
            assert f == pytest.approx(rho / math.pi + cs / (4 * math.pi * m32 * m32), rel=1e-12)


def test_schlick_against_folded(oracle):
    n = np.array([0.0, 0.0, 1.0])
    rng = np.random.default_rng(4)
    for model in (0, 1):
        c0 = default_config(brdf_model=model, fresnel=0)
        c1 = default_config(brdf_model=model, fresnel=1)
        for a, b in zip(_hemi(rng, 40), _hemi(rng, 40)):
            assert oracle.brdf(c1, n, a, b, 0.3, 1.0) == pytest.approx(oracle.brdf(c0, n, a, b, 0.3, 1.0), rel=1e-13)
            for cs in (0.0, 0.04, 0.5):
                assert oracle.brdf(c1, n, a, b, 0.0, cs) >= oracle.brdf(c0, n, a, b, 0.0, cs) * (1 - 1e-13)


def _albedo(oracle, cfg, theta_o, nt=256, nph=64):
    """Directional albedo of the specular lobe (rho = 0, c_s = 1), midpoint rule."""
    n = np.array([0.0, 0.0, 1.0])
    wo = np.array([math.sin(theta_o), 0.0, math.cos(theta_o)])
    th = (np.arange(nt) + 0.5) / nt * (math.pi / 2)
    ph = (np.arange(nph) + 0.5) / nph * 2 * math.pi
    tot = 0.0
    for t in th:
        st, ct = math.sin(t), math.cos(t)
        for p in ph:
            w = np.array([st * math.cos(p), st * math.sin(p), ct])
            tot += oracle.brdf(cfg, n, w, wo, 0.0, 1.0) * ct * st
    return tot * (math.pi / 2 / nt) * (2 * math.pi / nph)


@pytest.mark.parametrize("model", [0, 1])
def test_specular_albedo_at_most_one_and_near_one_when_smooth(oracle, model):
    for m in (0.1, 0.3, 0.6):
        cfg = default_config(brdf_model=model, fresnel=1, beckmann_m=m)
        for ang in (0.0, 0.7, 1.3):
            a = _albedo(oracle, cfg, ang)
            assert 0.2 < a <= 1.0 + 2e-3, (model, m, ang, a)
    a = _albedo(oracle, default_config(brdf_model=1, fresnel=1, beckmann_m=0.1), 0.0, nt=512)
    if model == 1:
        assert a >= 0.95, a


def _grad_setup(model, fresnel):
    scene, theta, _ = S.make_workload("tiny", seed=3)
    cfg = default_config(W=24, H=24, spp=2, seed=5, value_mesh=0, brdf_model=model, fresnel=fresnel)
    dI = np.random.default_rng(11).normal(size=(24, 24, 3))
    return scene, theta, cfg, dI


@pytest.mark.parametrize("model,fresnel", VARIANTS)
def test_gradient_linear_parameters_exact(oracle, model, fresnel):
    """The image is linear in each light channel and affine in each albedo
    coefficient and specular texel (Schlick is affine in c_s too)."""
    scene, theta, cfg, dI = _grad_setup(model, fresnel)
    o = S.param_offsets(*scene.K)
    g = oracle.render_backward(cfg, scene, theta, dI)
    for j, ch in [(0, 0), (7, 2), (13, 1)]:
        th = theta.copy()
        th[o["lights"]:] = 0
        th[o["lights"] + 3 * j + ch] = 1.0
        ref = float(np.sum(dI * oracle.render(cfg, scene, th)))
        assert g[o["lights"] + 3 * j + ch] == pytest.approx(ref, rel=1e-9, abs=1e-12)
    base = float(np.sum(dI * oracle.render(cfg, scene, theta)))
    for idx in [o["delta"] + 3, o["cspec"] + 5 * 32 + 9, o["cspec"] + 16 * 32 + 16]:
        th = theta.copy()
        th[idx] += 1.0
        ref = float(np.sum(dI * oracle.render(cfg, scene, th))) - base
        assert g[idx] == pytest.approx(ref, rel=1e-7, abs=1e-9 * max(1.0, abs(base)))


@pytest.mark.parametrize("model,fresnel", VARIANTS)
def test_geometry_gradient_fd(oracle, model, fresnel):
    scene, theta, cfg, dI = _grad_setup(model, fresnel)
    o = S.param_offsets(*scene.K)
    gi = oracle.render_backward(cfg, scene, theta, dI, terms=True)[1][0]
    _, sig0 = oracle.render(cfg, scene, theta, signature=True)
    checked = 0
    for idx, h in [(o["alpha"] + 0, 1e-4), (o["beta"] + 2, 1e-4), (o["pose"] + 1, 1e-5), (o["pose"] + 5, 1e-5)]:
        tp, tm = theta.copy(), theta.copy()
        tp[idx] += h
        tm[idx] -= h
        ip, sp = oracle.render(cfg, scene, tp, signature=True)
        im, sm = oracle.render(cfg, scene, tm, signature=True)
        if sp != sig0 or sm != sig0:
            continue                                   # a decision moved: not an interior difference
        fd = float(np.sum(dI * (ip - im))) / (np.float64(tp[idx]) - np.float64(tm[idx]))
        assert gi[idx] == pytest.approx(fd, rel=2e-4, abs=1e-6 * (1 + abs(fd))), (idx, gi[idx], fd)
        checked += 1
    assert checked >= 3


def test_icosphere_light_stage(oracle):
    L = oracle.light_stage(20, 3.0, layout=1).astype(np.float64)
    c, e1, e2, d = L[:, 0:3], L[:, 3:6], L[:, 6:9], L[:, 9:12]
    assert np.allclose(np.linalg.norm(d, axis=1), 1, atol=1e-6) and np.all(d[:, 2] > 0)
    assert np.allclose(c, 3.0 * d, atol=1e-6)
    assert np.allclose(np.sum(e1 * d, 1), 0, atol=1e-6) and np.allclose(np.cross(d, e1), e2, atol=1e-6)
    assert np.all(np.diff(d[:, 2]) <= 1e-6)                      # ordered by height
    ang = np.degrees(np.arccos(np.clip(d @ d.T, -1, 1)))
    np.fill_diagonal(ang, 180.0)
    nearest = ang.min(axis=1)
    half_edge = math.degrees(math.atan(2.0)) / 2                  # vertex to an adjacent edge midpoint
    for a in nearest:
        assert min(abs(a - half_edge), abs(a - 36.0)) < 1e-4, nearest
    assert ang.min() > half_edge - 1e-4
    # the default layout is unchanged by the switch
    assert np.array_equal(oracle.light_stage(20, 3.0, layout=0), oracle.light_stage(20, 3.0))
