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
  icosahedron: every nearest-neighbour angle is atan(2)/2 or 36 degrees;
* the light prior m_j of E_light (Eq. 1), read as the mean of the lights per
  channel or as each light's channel mean: E_light equals N times the
  per-channel variances, or 3 times the per-light variances (numpy's var);
  it vanishes for equal or grey lights; its gradient matches central
  differences, which are exact for a quadratic at dyadic steps.
"""
import math

import numpy as np
import pytest

from oracle import default_config
from paper_1910_05200_gb300 import synthetic as S
from tests import closed_forms as CF

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


# ---------------------------------------------------------------------------
# light prior readings: E_light = sum_j |l_j - m_j|^2 with m following the lights

def _prior_case(seed=4):
    sc = CF.plain_scene([(0, 0, 0), (1, 0, 0), (0, 1, 0)], [(0, 1, 2)])
    o = S.param_offsets(0, 0, 0)
    rng = np.random.default_rng(seed)
    th = CF.plain_theta()
    k = rng.integers(0, 129, size=(20, 3))
    k[19] += (-k.sum(axis=0)) % 5                          # column sums divisible by 5:
    L = k / 64.0                                           # values and channel means dyadic
    th[o["lights"]:o["lights"] + 60] = L.reshape(-1)
    img = np.zeros((1, 2, 3), np.float32)
    return sc, th, L, img, o


def _e_light(oracle, prior, th, sc, img, m=None, w2=1.0):
    cfg = default_config(W=2, H=1, light_prior=prior)
    val, _, gr = oracle.loss(cfg, sc, th, img, img, None, m, 0.0, w2)
    return val, gr


def test_light_prior_closed_forms(oracle):
    sc, th, L, img, o = _prior_case()
    v1, _ = _e_light(oracle, 1, th, sc, img)
    assert v1 == pytest.approx(20 * np.var(L, axis=0).sum(), rel=1e-13)
    v2, _ = _e_light(oracle, 2, th, sc, img)
    assert v2 == pytest.approx(3 * np.var(L, axis=1).sum(), rel=1e-13)
    # the given m is ignored when m follows the lights
    m = np.full(60, 7.0, np.float32)
    assert _e_light(oracle, 1, th, sc, img, m)[0] == v1 and _e_light(oracle, 2, th, sc, img, m)[0] == v2
    # mean over lights, frozen and given, has the same value and gradient:
    # the term through m is minus the mean of deviations that sum to zero
    mm = np.tile(L.mean(axis=0), 20).astype(np.float32)
    v0, g0 = _e_light(oracle, 0, th, sc, img, mm, w2=0.5)
    v1b, g1 = _e_light(oracle, 1, th, sc, img, None, w2=0.5)
    assert v0 == pytest.approx(v1b, rel=1e-13)
    np.testing.assert_allclose(g1, g0, rtol=0, atol=1e-13)


def test_light_prior_vanishes_on_equal_and_grey_lights(oracle):
    sc, th, L, img, o = _prior_case()
    eq = th.copy()
    eq[o["lights"]:o["lights"] + 60] = np.tile([0.5, 1.25, 2.0], 20)
    v, g = _e_light(oracle, 1, eq, sc, img)
    assert v == 0.0 and np.all(g == 0.0)
    assert _e_light(oracle, 2, eq, sc, img)[0] > 0
    grey = th.copy()
    grey[o["lights"]:o["lights"] + 60] = np.repeat(L[:, 0], 3)
    v, g = _e_light(oracle, 2, grey, sc, img)
    assert v == 0.0 and np.all(g == 0.0)
    assert _e_light(oracle, 1, grey, sc, img)[0] > 0


@pytest.mark.parametrize("prior", [0, 1, 2])
def test_light_prior_gradient_central_differences(oracle, prior):
    sc, th, L, img, o = _prior_case(seed=9)
    m = (np.arange(60) % 5 / 4.0).astype(np.float32)
    _, g = _e_light(oracle, prior, th, sc, img, m, w2=0.75)
    h = 1.0 / 64
    for k in (0, 1, 2, 7, 31, 59):
        tp, tm = th.copy(), th.copy()
        tp[o["lights"] + k] += h
        tm[o["lights"] + k] -= h
        fd = (_e_light(oracle, prior, tp, sc, img, m, w2=0.75)[0] -
              _e_light(oracle, prior, tm, sc, img, m, w2=0.75)[0]) / (2 * h)
        assert g[o["lights"] + k] == pytest.approx(fd, rel=1e-11, abs=1e-12)
