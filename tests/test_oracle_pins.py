"""Pins of the CPU oracle against closed forms, invariants and exact identities.

Each test ties one part of the oracle to something other than itself, chosen
so that a dropped term, a wrong sign or index, or a transposed operand fails:

* Philox known-answer vectors (Salmon et al. SC'11, Random123 distribution)
* morphable geometry and pose on one-hot inputs (Face Modeling paragraph)
* vertex normals on a plane and a sphere
* watertightness of the ray/triangle test on a shared edge
* Lambert's polygon formula for the unshadowed light integral
* polygon-clipped irradiance behind an occluder (self-shadows)
* BRDF reciprocity and energy bound (Cook-Torrance)
* exact linearity of the image in the lights, albedo and specular map
* central differences of the interior gradient with all decisions frozen
* the primary-visibility edge term against the exact derivative of pixel
  coverage (Li et al. 2018 edge sampling)
* the shadow-boundary edge term against the derivative of the clipped
  polygon irradiance, with respect to the occluder's vertices and to the
  receiver's (the shading point moving with its triangle), on one occluder
  and on a cluster of occluders with many candidate edges (exact union of
  their shadows by slab decomposition)
* the loss of Eq. 1 on a hand-computed case
"""
import os

import numpy as np
import pytest

from oracle import default_config
from paper_1910_05200_gb300 import synthetic as S
from tests import closed_forms as CF

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answers(oracle):
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = oracle.philox(v[4:6], v[0:4])
        assert out.tolist() == v[6:10]


def test_light_stage_frames(oracle):
    L = oracle.light_stage(20, 3.0).astype(np.float64)
    c, e1, e2, d = L[:, 0:3], L[:, 3:6], L[:, 6:9], L[:, 9:12]
    assert np.allclose(np.linalg.norm(d, axis=1), 1, atol=1e-6)
    assert np.allclose(np.linalg.norm(c, axis=1), 3, atol=1e-5)
    assert np.allclose((e1 * d).sum(1), 0, atol=1e-6) and np.allclose((e2 * d).sum(1), 0, atol=1e-6)
    assert np.allclose((e1 * e2).sum(1), 0, atol=1e-6)
    assert np.allclose(np.cross(e1, e2), d, atol=1e-6)          # right-handed, normal = d
    assert np.allclose(d[:, 2], (np.arange(20) + 0.5) / 20, atol=1e-6)   # equal-area bands
    assert np.all(d[:, 2] > 0)                                  # camera hemisphere
    # isotropic: the mean direction of equal-area samples of a hemisphere is (0, 0, 1/2)
    assert np.allclose(d.mean(0), [0, 0, 0.5], atol=0.05)


def _small_scene(K=(3, 2, 2), seed=0):
    mean, tris, uv = S.tiny_grid_mesh(6)
    rng = np.random.default_rng(seed)
    V = mean.shape[0]
    return S.Scene(mean, tris, uv, rng.normal(size=(3 * V, K[0])).astype(np.float32) * 0.01,
                   rng.normal(size=(3 * V, K[1])).astype(np.float32) * 0.01,
                   np.full(3 * V, 0.5, np.float32), rng.normal(size=(3 * V, K[2])).astype(np.float32) * 0.01)


def test_geometry_one_hot_and_pose(oracle):
    sc = _small_scene()
    cfg = default_config()
    o = S.param_offsets(*sc.K)
    th = np.zeros(o["total"], np.float32)
    th[o["alpha"] + 1] = 1.0
    g = oracle.geometry(cfg, sc, th)
    assert np.allclose(g["X"].reshape(-1), sc.mean.reshape(-1).astype(np.float64) + sc.B_id[:, 1], atol=1e-12)
    th[:] = 0
    th[o["beta"] + 1] = 2.0
    th[o["delta"] + 0] = -1.0
    g = oracle.geometry(cfg, sc, th)
    assert np.allclose(g["X"].reshape(-1), sc.mean.reshape(-1).astype(np.float64) + 2 * sc.B_exp[:, 1].astype(np.float64), atol=1e-12)
    assert np.allclose(g["albedo"].reshape(-1), 0.5 - sc.B_alb[:, 0].astype(np.float64), atol=1e-12)
    # rotation about x by 90 degrees: (x, y, z) -> (x, -z, y); then translation
    th[:] = 0
    th[o["pose"] + 0] = np.float32(np.pi / 2)
    th[o["pose"] + 3:o["pose"] + 6] = [0.5, -0.25, 0.125]
    g = oracle.geometry(cfg, sc, th)
    m = sc.mean.astype(np.float64)
    exp = np.stack([m[:, 0], -m[:, 2], m[:, 1]], 1) + [0.5, -0.25, 0.125]
    assert np.allclose(g["X"], exp, atol=1e-7)
    assert np.array_equal(g["X32"], g["X"].astype(np.float32))
    # rotation about z by 90 degrees: (x, y, z) -> (-y, x, z)
    th[:] = 0
    th[o["pose"] + 2] = np.float32(np.pi / 2)
    g = oracle.geometry(cfg, sc, th)
    assert np.allclose(g["X"], np.stack([-m[:, 1], m[:, 0], m[:, 2]], 1), atol=1e-7)
    # composition order R = Rz Ry Rx: rx then rz
    th[:] = 0
    th[o["pose"] + 0] = np.float32(np.pi / 2)
    th[o["pose"] + 2] = np.float32(np.pi / 2)
    g = oracle.geometry(cfg, sc, th)
    step = np.stack([m[:, 0], -m[:, 2], m[:, 1]], 1)
    assert np.allclose(g["X"], np.stack([-step[:, 1], step[:, 0], step[:, 2]], 1), atol=1e-7)


def test_normals_plane_and_sphere(oracle):
    cfg = default_config()
    verts = [(-1, -1, 0.2), (1, -1, 0.2), (1, 1, 0.2), (-1, 1, 0.2), (0, 0, 0.2)]
    tris = [(0, 1, 4), (1, 2, 4), (2, 3, 4), (3, 0, 4)]
    g = oracle.geometry(cfg, CF.plain_scene(verts, tris), CF.plain_theta())
    assert np.allclose(g["normals"], [0, 0, 1], atol=1e-12)
    mean, tris, uv = S.tiny_grid_mesh()
    sc = CF.plain_scene(mean, tris, uv)
    g = oracle.geometry(cfg, sc, CF.plain_theta())
    radial = g["X"] / np.linalg.norm(g["X"], axis=1, keepdims=True)
    n = mean.shape[0]
    side = int(np.sqrt(n))
    inner = np.array([i * side + j for i in range(1, side - 1) for j in range(1, side - 1)])
    err = np.linalg.norm(g["normals"][inner] - radial[inner], axis=1)
    assert err.max() < 5e-3          # O(h^2) with h = pi/39
    assert (g["normals"] * radial).sum(1).min() > 0.9


def test_watertight_shared_edge(oracle):
    cfg = default_config()
    verts = [(-1, -1, 0), (1, -1, 0), (1, 1, 0), (-1, 1, 0)]
    sc = CF.plain_scene(verts, [(0, 1, 2), (0, 2, 3)])
    th = CF.plain_theta(lights_on=[19])
    o = np.array([0, 0, 4], np.float32)
    rng = np.random.default_rng(1)
    faces = []
    for s in list(rng.uniform(-0.9, 0.9, 200)) + [0.0, 0.5, -0.25]:
        tgt = np.array([s, s, 0], np.float32)              # exactly on the shared diagonal
        _, f = oracle.point_shade(cfg, sc, th, o, (tgt - o).astype(np.float32), 19, 0.5, 0.5)
        faces.append(f)
    assert min(faces) >= 0                                  # never falls through the crack
    # off the plane: a clear miss
    _, f = oracle.point_shade(cfg, sc, th, o, np.array([0.5, 0, -1], np.float32), 19, 0.5, 0.5)
    assert f == -1


def _grid_mean(fn, n):
    u = (np.arange(n) + 0.5) / n
    acc = 0.0
    for a in u:
        for b in u:
            acc += fn(np.float32(a), np.float32(b))
    return acc / (n * n)


@pytest.mark.parametrize("j", [3, 12, 19])
def test_lambert_unshadowed(oracle, j):
    cfg = default_config()
    rng = np.random.default_rng(j)
    for _ in range(2):
        x = rng.uniform(-0.3, 0.3, 3)
        n = np.array([0.1, 0.0, 1.0]) + rng.normal(0, 0.1, 3)
        n /= np.linalg.norm(n)
        wo = np.array([0, 0, 4.0]) - x
        wo /= np.linalg.norm(wo)
        quad = CF.light_quad(j)
        if min((np.asarray(p) - x) @ n for p in quad) <= 0.05:
            continue
        est = _grid_mean(lambda a, b: oracle.light_estimate(cfg, x, n, wo, [np.pi] * 3, 0.0, [1, 1, 1], j, a, b)[0], 96)
        ref = CF.lambert_irradiance(x, n, quad)
        assert abs(est - ref) < 2e-4 * ref, (est, ref)


def test_brdf_reciprocity_and_energy(oracle):
    cfg = default_config()
    rng = np.random.default_rng(2)
    n = np.array([0.0, 0.0, 1.0])

    def hemi(k):
        v = rng.normal(size=(k, 3))
        v[:, 2] = np.abs(v[:, 2]) + 0.05
        return v / np.linalg.norm(v, axis=1, keepdims=True)

    wi, wo = hemi(50), hemi(50)
    for a, b in zip(wi, wo):
        f1 = oracle.brdf(cfg, n, a, b, 0.0, 1.0)
        f2 = oracle.brdf(cfg, n, b, a, 0.0, 1.0)
        assert f1 > 0 and abs(f1 - f2) <= 1e-12 * max(1.0, f1)
        assert abs(oracle.brdf(cfg, n, a, b, 0.7, 0.0) - 0.7 / np.pi) < 1e-14
    # directional albedo of the specular lobe <= 1 (midpoint rule on the hemisphere)
    nt, npz = 128, 256
    th = (np.arange(nt) + 0.5) / nt * (np.pi / 2)
    ph = (np.arange(npz) + 0.5) / npz * 2 * np.pi
    for ang in (0.0, 0.6, 1.2):
        wov = np.array([np.sin(ang), 0, np.cos(ang)])
        tot = 0.0
        for t in th:
            for p in ph[::4]:
                w = np.array([np.sin(t) * np.cos(p), np.sin(t) * np.sin(p), np.cos(t)])
                tot += oracle.brdf(cfg, n, w, wov, 0.0, 1.0) * np.cos(t) * np.sin(t)
        tot *= (np.pi / 2 / nt) * (2 * np.pi / (npz / 4))
        assert 0.2 < tot <= 1.0, (ang, tot)


def _occluder_scene(j=15):
    c, e1, e2, d = CF.light_frame(j)
    recv = [(-2, -2, 0), (2, -2, 0), (2, 2, 0), (-2, 2, 0)]
    occ = [d * 1.0, d * 1.0 + 0.15 * e1 + 0.02 * e2, d * 1.0 + 0.05 * e1 + 0.15 * e2]
    verts = recv + [tuple(v) for v in occ]
    tris = [(0, 1, 2), (0, 2, 3), (4, 5, 6)]
    return CF.plain_scene(verts, tris), np.asarray(occ)


def _lit_irradiance(x, n, occ, j):
    """E(quad) - E(quad intersected with the occluder's central projection from x)."""
    quad = CF.light_quad(j)
    c, e1, e2, d = CF.light_frame(j)
    D = (c - x) @ d
    proj = [x + (p - x) * (D / ((p - x) @ d)) for p in occ]
    to2 = lambda p: np.array([(p - c) @ e1, (p - c) @ e2])
    q2 = CF.ccw([to2(p) for p in quad])
    t2 = CF.ccw([to2(p) for p in proj])
    inter = CF.clip_polygon(t2, q2)
    E = CF.lambert_irradiance(x, n, quad)
    if len(inter) >= 3:
        E -= CF.lambert_irradiance(x, n, [c + p[0] * e1 + p[1] * e2 for p in inter])
    return E


def test_shadowed_irradiance(oracle):
    j = 15
    sc, occ = _occluder_scene(j)
    cfg = default_config()
    th = CF.plain_theta(lights_on=[j])
    o = np.array([0, 0, 4], np.float32)
    x = np.array([0.013, -0.021, 0.0])
    d = (x.astype(np.float32) - o).astype(np.float32)
    est = _grid_mean(lambda a, b: oracle.point_shade(cfg, sc, th, o, d, j, a, b)[0][0], 200)
    ref = _lit_irradiance(x, np.array([0, 0, 1.0]), occ, j)
    full = CF.lambert_irradiance(x, np.array([0, 0, 1.0]), CF.light_quad(j))
    assert ref < 0.9 * full                    # the occluder really casts a partial shadow
    assert abs(est - ref) < 4e-3 * full, (est, ref, full)


def test_loss_hand_case(oracle):
    cfg = default_config(W=2, H=1)
    sc = CF.plain_scene([(0, 0, 0), (1, 0, 0), (0, 1, 0)], [(0, 1, 2)])
    th = CF.plain_theta()
    o = S.param_offsets(0, 0, 0)
    th[o["lights"] + 0] = 2.0
    th[o["lights"] + 5] = -1.0
    img = np.array([[[1, 2, 3], [0, 0, 1]]], np.float32)
    tgt = np.array([[[1, 0, 0], [0, 0, 0]]], np.float32)
    m = np.zeros(60, np.float32)
    m[0] = 1.0
    val, dI, gr = oracle.loss(cfg, sc, th, img, tgt, None, m, w1=0.5, w2=0.25)
    # E_data = 4 + 9 + 1 = 14 ; E_prior = 0 (K = 0) ; E_light = (2-1)^2 + 1 = 2
    assert abs(val - (14 + 0.25 * 2)) < 1e-12
    assert np.allclose(dI.reshape(-1), 2 * (img - tgt).reshape(-1))
    assert gr[o["lights"]] == pytest.approx(2 * 0.25 * 1.0) and gr[o["lights"] + 5] == pytest.approx(2 * 0.25 * -1.0)
    val, dI, _ = oracle.loss(cfg, sc, th, img, tgt, np.array([0, 1], np.uint8), None, 0.0, 0.0)
    assert val == pytest.approx(1.0) and np.all(dI[0, 0] == 0)


# ---------------------------------------------------------------------------
# gradient pins on a small face-like scene

def _grad_setup():
    scene, theta, _ = S.make_workload("tiny", seed=3)
    cfg = default_config(W=24, H=24, spp=2, seed=5, value_mesh=0)
    rng = np.random.default_rng(11)
    dI = rng.normal(size=(24, 24, 3))
    return scene, theta, cfg, dI


def _dot(a, b):
    return float(np.sum(np.asarray(a) * np.asarray(b)))


def test_light_albedo_specular_exactly_linear(oracle):
    scene, theta, cfg, dI = _grad_setup()
    o = S.param_offsets(*scene.K)
    g = oracle.render_backward(cfg, scene, theta, dI)
    # lights: the image is linear in every light channel (all samples fixed)
    for j, ch in [(0, 0), (7, 2), (13, 1)]:
        th = theta.copy()
        th[o["lights"]:] = 0
        th[o["lights"] + 3 * j + ch] = 1.0
        ref = _dot(dI, oracle.render(cfg, scene, th))
        assert g[o["lights"] + 3 * j + ch] == pytest.approx(ref, rel=1e-9, abs=1e-12)
    # albedo coefficients and specular texels: exact differences of a linear map
    base = _dot(dI, oracle.render(cfg, scene, theta))
    for idx in [o["delta"] + 0, o["delta"] + 17, o["cspec"] + 5 * 32 + 9, o["cspec"] + 16 * 32 + 16]:
        th = theta.copy()
        th[idx] += 1.0
        ref = _dot(dI, oracle.render(cfg, scene, th)) - base
        assert g[idx] == pytest.approx(ref, rel=1e-7, abs=1e-9 * max(1.0, abs(base)))


def test_geometry_interior_gradient_fd(oracle):
    scene, theta, cfg, dI = _grad_setup()
    o = S.param_offsets(*scene.K)
    gi = oracle.render_backward(cfg, scene, theta, dI, terms=True)[1][0]
    _, sig0 = oracle.render(cfg, scene, theta, signature=True)
    checked = 0
    for idx, h in [(o["alpha"] + 0, 1e-4), (o["alpha"] + 5, 1e-4), (o["beta"] + 2, 1e-4),
                   (o["pose"] + 0, 1e-5), (o["pose"] + 1, 1e-5), (o["pose"] + 5, 1e-5)]:
        tp, tm = theta.copy(), theta.copy()
        tp[idx] += h
        tm[idx] -= h
        ip, sp = oracle.render(cfg, scene, tp, signature=True)
        im, sm = oracle.render(cfg, scene, tm, signature=True)
        if sp != sig0 or sm != sig0:
            continue                                         # a decision moved: not an interior-only difference
        heff = (np.float64(tp[idx]) - np.float64(tm[idx]))
        fd = (_dot(dI, ip) - _dot(dI, im)) / heff
        assert gi[idx] == pytest.approx(fd, rel=2e-4, abs=1e-6 * (1 + abs(fd))), (idx, gi[idx], fd)
        checked += 1
    assert checked >= 4


def test_geometry_adjoint_against_forward_fd(oracle):
    """grad(theta) = J^T dX: the backward's geometry adjoint against FD of the forward geometry."""
    scene, theta, cfg, dI = _grad_setup()
    o = S.param_offsets(*scene.K)
    g, dX = oracle.render_backward(cfg, scene, theta, dI, dX=True)
    for idx, h in [(o["alpha"] + 3, 1e-2), (o["beta"] + 40, 1e-2), (o["pose"] + 2, 1e-3), (o["pose"] + 4, 1e-3)]:
        tp, tm = theta.copy(), theta.copy()
        tp[idx] += h
        tm[idx] -= h
        J = (oracle.geometry(cfg, scene, tp)["X"] - oracle.geometry(cfg, scene, tm)["X"]) / (np.float64(tp[idx]) - np.float64(tm[idx]))
        assert g[idx] == pytest.approx(_dot(J, dX), rel=1e-6, abs=1e-9)


def _triangle_scene():
    verts = [(-0.5, -0.4, 0.0), (0.6, -0.3, 0.1), (0.0, 0.6, -0.05)]
    return CF.plain_scene(verts, [(0, 1, 2)])


def _screen(cfg, p):
    k = 2.0 * np.float64(np.float32(cfg.tan_half_fov)) / cfg.H
    cx = np.float64(np.float32(cfg.tan_half_fov)) * cfg.W / cfg.H
    cy = np.float64(np.float32(cfg.tan_half_fov))
    q = cfg.d_cam - p[2]
    return np.array([(p[0] / q + cx) / k, (cy - p[1] / q) / k])


def test_primary_edge_term_matches_coverage_derivative(oracle):
    """Flat shading (1 on the triangle, 0 elsewhere): pixel = covered area."""
    sc = _triangle_scene()
    verts = sc.mean.astype(np.float64)
    th = CF.plain_theta()
    W = H = 12
    pix_list = [(W * H, None)]           # total over the image
    # pick two pixels crossed by an edge
    cfg0 = default_config(W=W, H=H, spp=1, shade_mode=1)
    s2 = [_screen(cfg0, v) for v in verts]
    for py in range(H):
        for px in range(W):
            a = CF.triangle_pixel_area(s2, px, py)
            if 0.2 < a < 0.8 and len(pix_list) < 3:
                pix_list.append((py * W + px, None))

    def exact(vv, pid):
        s = [_screen(cfg0, v) for v in vv]
        if pid == W * H:
            return sum(CF.triangle_pixel_area(s, px, py) for py in range(H) for px in range(W))
        return CF.triangle_pixel_area(s, pid % W, pid // W)

    for pid, _ in pix_list:
        dI = np.zeros((H, W, 3))
        if pid == W * H:
            dI[..., 0] = 1.0
        else:
            dI[pid // W, pid % W, 0] = 1.0
        ests = []
        for seed in range(8):
            cfg = default_config(W=W, H=H, spp=64, seed=seed, shade_mode=1)
            _, dX = oracle.render_backward(cfg, sc, th, dI, dX=True)
            ests.append(dX.reshape(-1))
        ests = np.array(ests)
        mean, se = ests.mean(0), ests.std(0, ddof=1) / np.sqrt(len(ests))
        fd = np.zeros(9)
        for i in range(9):
            vp, vm = verts.copy(), verts.copy()
            vp[i // 3, i % 3] += 1e-6
            vm[i // 3, i % 3] -= 1e-6
            fd[i] = (exact(vp, pid) - exact(vm, pid)) / 2e-6
        scale = np.abs(fd).max()
        assert np.all(np.abs(mean - fd) <= 4.5 * se + 0.02 * scale), (pid, mean, fd, se)


def test_shadow_edge_term_matches_clipped_irradiance_derivative(oracle):
    j = 15
    sc, occ = _occluder_scene(j)
    th = CF.plain_theta(lights_on=[j])
    o = np.array([0, 0, 4], np.float32)
    x = np.array([0.013, -0.021, 0.0])
    d = (x.astype(np.float32) - o).astype(np.float32)
    n = np.array([0, 0, 1.0])
    fd = np.zeros(9)
    for i in range(9):
        op, om = occ.copy(), occ.copy()
        op[i // 3, i % 3] += 1e-6
        om[i // 3, i % 3] -= 1e-6
        fd[i] = (_lit_irradiance(x, n, op, j) - _lit_irradiance(x, n, om, j)) / 2e-6
    reps = 4000
    ests = []
    for seed in range(8):
        cfg = default_config(seed=seed)
        dX = oracle.shadow_edge_point(cfg, sc, th, o, d, j, [1.0, 0, 0], reps)
        ests.append(dX[4:7].reshape(-1) / reps)
    ests = np.array(ests)
    mean, se = ests.mean(0), ests.std(0, ddof=1) / np.sqrt(len(ests))
    scale = np.abs(fd).max()
    assert scale > 0
    assert np.all(np.abs(mean - fd) <= 4.5 * se + 0.01 * scale), (mean, fd, se)


def test_two_sided_shading_ignores_winding(oracle):
    """A surface seen from either side shades alike: reversing the winding changes nothing."""
    verts = [(-0.6, -0.6, 0.1), (0.6, -0.6, -0.1), (0.6, 0.6, 0.0), (-0.6, 0.6, 0.05)]
    th = CF.plain_theta(lights_on=[4, 11, 18], cspec=0.5)
    cfg = default_config(W=16, H=16, spp=2)
    a = oracle.render(cfg, CF.plain_scene(verts, [(0, 1, 2), (0, 2, 3)]), th)
    b = oracle.render(cfg, CF.plain_scene(verts, [(0, 2, 1), (0, 3, 2)]), th)
    assert a.max() > 0.01
    assert np.allclose(a, b, rtol=1e-12, atol=1e-15)


def _hit_point_on(verts, tri, o, d):
    """Intersection of the ray o + t d with the plane of triangle tri (FP64)."""
    P = [np.asarray(verts[k], np.float64) for k in tri]
    n = np.cross(P[1] - P[0], P[2] - P[0])
    t = ((P[0] - o) @ n) / (d @ n)
    return o + t * d


def _shadow_edge_estimates(oracle, sc, th, o, d, j, reps, seeds=8):
    ests = []
    for seed in range(seeds):
        dX = oracle.shadow_edge_point(default_config(seed=seed), sc, th, o, d, j, [1.0, 0, 0], reps)
        ests.append(dX.reshape(-1) / reps)
    ests = np.array(ests)
    return ests.mean(0), ests.std(0, ddof=1) / np.sqrt(seeds)


def test_shadow_edge_term_receiver_side(oracle):
    """The shading point x moves with its triangle (the camera ray fixed):
    the shadow on the light square moves with it.  The estimator's
    derivative with respect to the receiver's vertices against central
    differences of the exact lit irradiance in which only the visibility
    boundary sees the moved x (the integrand's own dependence on x belongs to
    the interior term)."""
    j = 15
    sc, occ = _occluder_scene(j)
    th = CF.plain_theta(lights_on=[j])
    o = np.array([0, 0, 4], np.float32)
    x = np.array([0.013, -0.021, 0.0])
    d = (x.astype(np.float32) - o).astype(np.float32)
    o64, d64 = o.astype(np.float64), d.astype(np.float64)
    verts = sc.mean.astype(np.float64)
    tri = (0, 1, 2)                                  # the receiver triangle under x (y < x)
    x0 = _hit_point_on(verts, tri, o64, d64)
    n = np.array([0, 0, 1.0])
    occ_tris = [occ]
    fd = np.zeros(12)
    for i in range(12):
        vp, vm = verts.copy(), verts.copy()
        vp[i // 3, i % 3] += 1e-6
        vm[i // 3, i % 3] -= 1e-6
        fp = CF.lit_irradiance(x0, n, occ_tris, j, x_vis=_hit_point_on(vp, tri, o64, d64))
        fm = CF.lit_irradiance(x0, n, occ_tris, j, x_vis=_hit_point_on(vm, tri, o64, d64))
        fd[i] = (fp - fm) / 2e-6
    mean, se = _shadow_edge_estimates(oracle, sc, th, o, d, j, 4000)
    scale = np.abs(fd).max()
    assert scale > 0 and np.all(fd[9:] == 0)        # vertex 3 is not on x's triangle
    assert np.all(np.abs(mean[:12] - fd) <= 4.5 * se[:12] + 0.01 * scale), (mean[:12], fd, se[:12])
    # the single-occluder closed form of the occluder-side pin is the same function
    assert CF.lit_irradiance(x0, n, occ_tris, j) == pytest.approx(_lit_irradiance(x0, n, occ, j), rel=1e-12)


def _occluder_cluster(j=15, seed=4):
    """Receiver plane plus a cluster of small occluders between x and light j:
    seven loose triangles at random offsets and tilts (every edge a boundary
    edge) and a Z-folded pair whose shared edge is a silhouette seen from x."""
    c, e1, e2, d = CF.light_frame(j)
    rng = np.random.default_rng(seed)
    recv = [(-2, -2, 0), (2, -2, 0), (2, 2, 0), (-2, 2, 0)]
    verts = [np.asarray(v, np.float64) for v in recv]
    tris = [(0, 1, 2), (0, 2, 3)]
    occ = []
    for _ in range(7):
        cen = d * rng.uniform(0.8, 1.2) + e1 * rng.uniform(-0.09, 0.09) + e2 * rng.uniform(-0.09, 0.09)
        a = rng.uniform(0, 2 * np.pi)
        tri = []
        for k in range(3):
            ang = a + 2 * np.pi * k / 3 + rng.uniform(-0.3, 0.3)
            r = rng.uniform(0.025, 0.05)
            tri.append(cen + r * (np.cos(ang) * e1 + np.sin(ang) * e2) + rng.uniform(-0.02, 0.02) * d)
        occ.append(tri)
    base = d * 1.0 - 0.06 * e2
    A, B = base - 0.05 * e1, base + 0.05 * e1
    occ.append([A, B, base + 0.06 * e2 + 0.03 * d])
    occ.append([B, A, base - 0.03 * e2 - 0.03 * d])
    for t in occ[:7]:
        k = len(verts)
        verts += list(t)
        tris.append((k, k + 1, k + 2))
    k = len(verts)
    verts += [A, B, occ[7][2], occ[8][2]]
    tris += [(k, k + 1, k + 2), (k + 1, k, k + 3)]
    return CF.plain_scene(np.asarray(verts), tris), occ


def test_shadow_edge_term_many_candidates(oracle):
    """A cluster of occluders: many candidate edges (silhouettes seen from x
    that cross the light square), some of them inside another occluder's
    shadow (no visibility change, no contribution).  The estimator's
    derivatives with respect to occluder and receiver vertices against
    central differences of the exact lit irradiance (Lambert's formula on
    the square minus the exact union of the occluders' projections)."""
    j = 15
    sc, occ = _occluder_cluster(j)
    th = CF.plain_theta(lights_on=[j])
    o = np.array([0, 0, 4], np.float32)
    x = np.array([0.013, -0.021, 0.0])
    d = (x.astype(np.float32) - o).astype(np.float32)
    o64, d64 = o.astype(np.float64), d.astype(np.float64)
    verts = sc.mean.astype(np.float64)
    x0 = _hit_point_on(verts, (0, 1, 2), o64, d64)
    n = np.array([0, 0, 1.0])
    full = CF.lambert_irradiance(x0, n, CF.light_quad(j))
    lit = CF.lit_irradiance(x0, n, occ, j)
    assert 0.1 * full < lit < 0.9 * full, (lit, full)        # a partial shadow
    # candidate edges (FP64 restatement of the candidate rule: silhouette seen
    # from x, central projection crossing the light square)
    c, e1, e2, dl = CF.light_frame(j)
    quad2 = CF.ccw([np.array([(p - c) @ e1, (p - c) @ e2]) for p in CF.light_quad(j)])
    tris = sc.tris
    edge_faces = {}
    for f, t in enumerate(tris):
        for k in range(3):
            key = tuple(sorted((int(t[k]), int(t[(k + 1) % 3]))))
            edge_faces.setdefault(key, []).append(f)

    def side(f):
        P = verts[tris[f]]
        return np.sign(np.cross(P[1] - P[0], P[2] - P[0]) @ (x0 - P[0]))

    n_cand = 0
    D = (c - x0) @ dl
    for (a, b), fs in edge_faces.items():
        if 0 in fs or 1 in fs and fs == [1]:
            continue
        if fs[0] in (0, 1):
            continue
        sil = len(fs) == 1 or side(fs[0]) != side(fs[1])
        if not sil:
            continue
        pa, pb = verts[a], verts[b]
        ya = x0 + (pa - x0) * (D / ((pa - x0) @ dl))
        yb = x0 + (pb - x0) * (D / ((pb - x0) @ dl))
        seg = [np.array([(ya - c) @ e1, (ya - c) @ e2]), np.array([(yb - c) @ e1, (yb - c) @ e2])]
        if len(CF.clip_polygon(seg + [seg[1] + 1e-12], quad2)) >= 2:
            n_cand += 1
    assert n_cand >= 10, n_cand
    mean, se = _shadow_edge_estimates(oracle, sc, th, o, d, j, 12000)
    checks = list(range(0, 9)) + [3 * v + k for v in (4, 5, 9, 27, 28) for k in range(3)]

    def lit(vv, i):
        if i < 12:          # a receiver vertex: x moves, the occluders stay
            return CF.lit_irradiance(x0, n, occ, j, x_vis=_hit_point_on(vv, (0, 1, 2), o64, d64))
        return CF.lit_irradiance(x0, n, [[vv[t] for t in tri] for tri in tris[2:]], j)

    fd = np.zeros(len(checks))
    for m, i in enumerate(checks):
        # median of three steps: the slab decomposition can jump by rounding
        # when two events nearly coincide at one particular step
        est = []
        for h in (1e-5, 2e-5, 4e-5):
            vp, vm = verts.copy(), verts.copy()
            vp[i // 3, i % 3] += h
            vm[i // 3, i % 3] -= h
            est.append((lit(vp, i) - lit(vm, i)) / (2 * h))
        fd[m] = np.median(est)
    got, s = mean[checks], se[checks]
    scale = np.abs(fd).max()
    assert scale > 0 and np.count_nonzero(np.abs(fd) > 0.05 * scale) >= 8
    assert np.all(np.abs(got - fd) <= 4.5 * s + 0.01 * scale), np.c_[got, fd, s]


def test_full_estimator_statistical_fd_on_tiny_face(oracle):
    """The whole gradient estimator (interior, primary-visibility and
    shadow-boundary terms) is unbiased for the derivative of the expected
    image: on a 6 x 6 window astride the tiny face's silhouette, the mean of
    the backward over 8 independent seeds x 512 spp (4,096 spp) against
    central differences (h = 1e-3) of the expected weighted image, each side
    rendered with common random numbers over 8 other seeds x 512 spp, for
    identity, expression, rotation, both in-plane translations and one light.
    The two means must agree within 3 standard errors of their difference."""
    scene, theta, _ = S.make_workload("tiny", seed=0)
    W = H = 64
    cov = oracle.render(default_config(W=W, H=H, spp=4, seed=0), scene, theta).sum(-1) > 0
    edge = cov & ~(np.roll(cov, 1, 0) & np.roll(cov, -1, 0) & np.roll(cov, 1, 1) & np.roll(cov, -1, 1))
    ys, xs = np.nonzero(edge)
    cy, cx = ys[len(ys) // 3], xs[len(xs) // 3]
    pix = np.array([y * W + x for y in range(cy - 3, cy + 3) for x in range(cx - 3, cx + 3)], np.int32)
    assert 6 <= cov.reshape(-1)[pix].sum() <= 30                      # the window straddles the silhouette
    rng = np.random.default_rng(1)
    wts = rng.uniform(0.5, 1.5, (len(pix), 3))
    dI = np.zeros((H * W, 3))
    dI[pix] = wts
    dI = dI.reshape(H, W, 3)
    o = S.param_offsets()
    h, seeds, spp = 1e-3, 8, 512
    G = np.array([oracle.render_backward(default_config(W=W, H=H, spp=spp, seed=100 + s), scene, theta, dI)
                  for s in range(seeds)])
    light = o["lights"] + int(np.argmax(np.abs(G[0, o["lights"]:])))     # the light channel that lights the window most
    params = [o["alpha"], o["beta"] + 3, o["pose"], o["pose"] + 3, o["pose"] + 5, light]
    G = G[:, params]
    FD = np.zeros((seeds, len(params)))
    for s in range(seeds):
        cfg = default_config(W=W, H=H, spp=spp, seed=200 + s)
        for m, i in enumerate(params):
            tp, tm = theta.copy(), theta.copy()
            tp[i] += h
            tm[i] -= h
            ip = oracle.render(cfg, scene, tp, pixels=pix)
            im = oracle.render(cfg, scene, tm, pixels=pix)
            FD[s, m] = (np.sum(wts * ip) - np.sum(wts * im)) / (np.float64(tp[i]) - np.float64(tm[i]))
    se = np.hypot(G.std(0, ddof=1), FD.std(0, ddof=1)) / np.sqrt(seeds)
    z = (G.mean(0) - FD.mean(0)) / se
    assert np.all(se > 0) and np.abs(G.mean(0)).max() > 1.0
    assert np.all(np.abs(z) <= 3.0), np.c_[G.mean(0), FD.mean(0), se, z]
