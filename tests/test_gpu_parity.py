"""GPU path against the CPU oracle, element by element, on identical seeded inputs.

Tolerances are those of tests/parity.py: per pixel 1e-4 relative with at
most 0.01 % flipped pixels; per gradient component 1e-3 relative with a
floor of 1e-3 of the parameter group's largest entry.  The GPU takes every
discrete decision in FP32 with the oracle's order of operations, so flips
are not expected; values differ by FP32 rounding.  Every check records its
strict error (tests/parity.py RECORD).
"""
import numpy as np
import pytest
import torch

from oracle import default_config
from paper_1910_05200_gb300 import synthetic as S
from tests.parity import (KAPPA, RECORD, assert_image, check_close, check_groups, check_same_values, face_pixels,
                          loss_bound, record_value)

pytestmark = pytest.mark.gpu

GROUPS = ["alpha", "beta", "delta", "cspec", "pose", "lights"]


@pytest.fixture(scope="module")
def fr():
    from paper_1910_05200_gb300 import build, facert
    build.build()
    return facert


@pytest.fixture(scope="module")
def tiny_r(fr, tiny):
    scene, theta, _ = tiny
    return fr.Renderer(scene, device=0)


@pytest.fixture(scope="module")
def full():
    scene, theta, c = S.make_workload("full", seed=1)
    return scene, theta, c


@pytest.fixture(scope="module")
def full_r(fr, full):
    return fr.Renderer(full[0], device=0)


def group_slices(K=(80, 90, 80)):
    o = S.param_offsets(*K)
    return {"alpha": slice(o["alpha"], o["beta"]), "beta": slice(o["beta"], o["delta"]),
            "delta": slice(o["delta"], o["cspec"]), "cspec": slice(o["cspec"], o["pose"]),
            "pose": slice(o["pose"], o["lights"]), "lights": slice(o["lights"], o["total"])}


def assert_grad(got, ref, mass=None, K=(80, 90, 80), what="", named=None, **kw):
    return check_groups(got, ref, group_slices(K), mass, named=named, what=what, **kw)


def assert_vertex_grad(dXg, dXo, mass, what=""):
    """Per-vertex position gradient (a diagnostic below the parameter level):
    relative 1e-3 for entries above 1 % of the largest, otherwise judged
    against that 1 % scale or KAPPA times the entry's L1 mass.  Entries that
    small come from a handful of samples at grazing angles, where cosines are
    near-cancelling FP32 dot products of unit vectors."""
    floor = 1e-2 * np.abs(dXo).max()
    strict = np.abs(dXg - dXo) / (1e-3 * np.maximum(np.abs(dXo), floor))
    tol = np.maximum(1e-3 * np.maximum(np.abs(dXo), floor), KAPPA * mass)
    err = np.abs(dXg - dXo) / tol
    RECORD.append(dict(kind="vertex", what=what, n=int(dXo.size), max=float(strict.max()) * 1e-3,
                       p9999=float(np.quantile(strict, 0.9999)) * 1e-3, n_mass_only=int((strict > 1).sum())))
    assert err.max() <= 1.0, f"{what}: per-vertex error {err.max():.3e} x tolerance"


def test_geometry_matches_oracle(oracle, tiny, tiny_r):
    scene, theta, _ = tiny
    geo = tiny_r.geometry(torch.tensor(theta, device="cuda:0"))
    ref = oracle.geometry(default_config(), scene, theta)
    X = geo["X"].cpu().numpy()
    # FP64 accumulation then rounding: bitwise equal up to rare rounding-boundary ties
    assert (X != ref["X32"]).mean() < 1e-3
    assert np.abs(X - ref["X"]).max() < 1e-6
    assert np.abs(geo["normals"].cpu().numpy() - ref["normals"]).max() < 2e-5
    assert np.abs(geo["albedo"].cpu().numpy() - ref["albedo"]).max() < 2e-5
    assert geo["n_silhouette"] == ref["n_silhouette"]


@pytest.mark.parametrize("W,H,spp,seed", [(64, 64, 4, 0), (37, 29, 3, 7), (8, 8, 32, 3), (1, 1, 1, 5)])
def test_forward_matches_oracle(oracle, tiny, tiny_r, W, H, spp, seed):
    scene, theta, _ = tiny
    img = tiny_r.render(torch.tensor(theta, device="cuda:0"), W, H, spp, seed=seed)
    tiny_r.sync()
    ref = oracle.render(default_config(W=W, H=H, spp=spp, seed=seed), scene, theta)
    if W * H > 1:
        assert ref.max() > 0
    assert_image(img.cpu().numpy().astype(np.float64), ref, what=f"forward {W}x{H}x{spp}")


@pytest.mark.parametrize("terms", [1, 2, 4])
def test_backward_terms_match_oracle(oracle, tiny, tiny_r, terms):
    scene, theta, _ = tiny
    W = H = 64
    spp = 4
    rng = np.random.default_rng(terms)
    dI = rng.normal(size=(H, W, 3)).astype(np.float32)
    g = tiny_r.backward(torch.tensor(theta, device="cuda:0"), torch.tensor(dI, device="cuda:0"), W, H, spp,
                        seed=2, terms=terms)
    tiny_r.sync()
    dXg = tiny_r.vertex_grad().cpu().numpy().astype(np.float64)
    cfg = default_config(W=W, H=H, spp=spp, seed=2, terms=terms)
    ref, dXo, mass, dXmass = oracle.render_backward(cfg, scene, theta, dI.astype(np.float64), dX=True, mass=True)
    got = g.cpu().numpy()
    assert np.abs(ref).max() > 0
    assert_vertex_grad(dXg, dXo, dXmass, what=f"terms={terms}")
    assert_grad(got, ref, mass, what=f"terms={terms}")


def test_backward_total_and_ragged(oracle, tiny, tiny_r):
    scene, theta, _ = tiny
    W, H, spp = 37, 29, 3
    rng = np.random.default_rng(9)
    dI = rng.normal(size=(H, W, 3)).astype(np.float32)
    g = tiny_r.backward(torch.tensor(theta, device="cuda:0"), torch.tensor(dI, device="cuda:0"), W, H, spp, seed=4)
    tiny_r.sync()
    ref, mass = oracle.render_backward(default_config(W=W, H=H, spp=spp, seed=4), scene, theta,
                                       dI.astype(np.float64), mass=True)
    assert_grad(g.cpu().numpy(), ref, mass, what="all terms, ragged")


def test_error_against_fp64_posed_mesh(oracle, tiny, tiny_r):
    """The oracle's values on its FP64 posed mesh (decisions still taken on
    the FP32 mesh, which is what makes sample identity possible) against the
    GPU, which evaluates everything on the FP32 mesh.  The difference is the
    FP32 rounding of the posed vertices (relative 6e-8 of coordinates of
    order 1, ~1e-6 of the tiny mesh's 0.08-unit triangles) propagated through
    the estimator, and it is measured here rather than hidden: image and
    gradient are held to the same tolerances as on the FP32 mesh."""
    scene, theta, _ = tiny
    W = H = 64
    spp = 4
    th = torch.tensor(theta, device="cuda:0")
    img = tiny_r.render(th, W, H, spp, seed=0)
    cfg = default_config(W=W, H=H, spp=spp, seed=0, value_mesh=0)
    assert_image(img.cpu().numpy().astype(np.float64), oracle.render(cfg, scene, theta),
                 what="forward 64x64x4 vs FP64 posed mesh")
    dI = np.random.default_rng(17).normal(size=(H, W, 3)).astype(np.float32)
    g = tiny_r.backward(th, torch.tensor(dI, device="cuda:0"), W, H, spp, seed=0).cpu().numpy()
    tiny_r.sync()
    ref, mass = oracle.render_backward(cfg, scene, theta, dI.astype(np.float64), mass=True)
    assert_grad(g, ref, mass, what="all terms 64x64x4 vs FP64 posed mesh")


def test_autograd_function(fr, tiny_r, tiny):
    scene, theta, _ = tiny
    th = torch.tensor(theta, device="cuda:0", requires_grad=True)
    img = fr.render(th, tiny_r, 32, 32, 2, 11)
    w = torch.randn(32, 32, 3, device="cuda:0", generator=torch.Generator("cuda:0").manual_seed(0))
    (img * w).sum().backward()
    direct = tiny_r.backward(th.detach(), w, 32, 32, 2, 11)
    # the same kernels: the two passes differ only in the order of FP32 atomic additions
    assert_sum_order_close(th.grad.double().cpu().numpy(), direct.cpu().numpy(), what="autograd vs direct")


def test_loss_matches_oracle(oracle, tiny, tiny_r):
    scene, theta, _ = tiny
    W, H = 40, 30
    rng = np.random.default_rng(3)
    img = rng.uniform(size=(H, W, 3)).astype(np.float32)
    tgt = rng.uniform(size=(H, W, 3)).astype(np.float32)
    mask = (rng.uniform(size=(H, W)) > 0.3).astype(np.uint8)
    m = rng.uniform(size=60).astype(np.float32)
    dev = lambda a: torch.tensor(a, device="cuda:0")
    d_image = torch.empty(H, W, 3, device="cuda:0")
    grad = torch.zeros(len(theta), device="cuda:0", dtype=torch.float64)
    loss = tiny_r.loss(dev(theta), dev(img), dev(tgt), dev(mask), dev(m), 0.3, 0.7, d_image, grad)
    val, dref, gref = oracle.loss(default_config(W=W, H=H), scene, theta, img, tgt, mask, m, 0.3, 0.7)
    record_value("loss E_data + w1 E_prior + w2 E_light", loss.item(), val, 1e-12)
    record_value("loss d_image", d_image.cpu().numpy()[dref != 0], dref[dref != 0], 1e-7)
    assert np.all(d_image.cpu().numpy()[dref == 0] == 0)
    assert np.allclose(grad.cpu().numpy(), gref, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("prior", [1, 2])
def test_light_prior_readings_match_oracle(oracle, fr, tiny, prior):
    """E_light with m following the lights (mean per channel; each light's
    channel mean): value and gradient against the oracle's chain rule."""
    scene, theta, _ = tiny
    W, H = 17, 9
    rng = np.random.default_rng(8)
    th = theta.copy()
    o = S.param_offsets(scene.B_id.shape[1], scene.B_exp.shape[1], scene.B_alb.shape[1])
    th[o["lights"]:o["lights"] + 60] = rng.uniform(0, 2, size=60)
    img = rng.uniform(size=(H, W, 3)).astype(np.float32)
    tgt = rng.uniform(size=(H, W, 3)).astype(np.float32)
    m = rng.uniform(size=60).astype(np.float32)            # ignored by these readings
    r = fr.Renderer(scene, device=0, config=fr.default_config(light_prior=prior))
    dev = lambda a: torch.tensor(a, device="cuda:0")
    grad = torch.zeros(len(th), device="cuda:0", dtype=torch.float64)
    loss = r.loss(dev(th), dev(img), dev(tgt), None, dev(m), 0.3, 0.7, None, grad)
    val, _, gref = oracle.loss(default_config(W=W, H=H, light_prior=prior), scene, th, img, tgt, None, None,
                               0.3, 0.7)
    record_value(f"loss, light prior reading {prior}", loss.item(), val, 1e-12)
    assert np.allclose(grad.cpu().numpy(), gref, rtol=1e-12, atol=1e-12)
    with pytest.raises(RuntimeError):
        fr.Renderer(scene, device=0, config=fr.default_config(light_prior=3))


def _three_calls(r, th, tgt, mask, m, W, H, spp, seed, w1, w2, terms=0):
    img = r.render(th, W, H, spp, seed=seed)
    d_image = torch.empty_like(img)
    loss = r.loss(th, img, tgt, mask, m, w1, w2, d_image)
    g = r.backward(th, d_image, W, H, spp, seed=seed, terms=terms)
    r.loss(th, img, tgt, mask, m, w1, w2, None, g)          # adds the prior and light terms' gradient
    r.sync()
    return img.cpu().numpy(), loss.item(), g.cpu().numpy(), d_image.cpu().numpy()


def assert_sum_order_close(got, ref, what=""):
    """Two GPU results that differ only in the order of floating-point atomic
    additions: 1e-4 of the group's largest entry plus 1e-3 of the entry."""
    check_close(got, ref, group_slices(), what=what)


@pytest.mark.parametrize("W,H,spp,terms", [(40, 33, 4, 0), (37, 29, 8, 0), (24, 24, 32, 0), (33, 17, 2, 1),
                                           (30, 20, 3, 0), (16, 9, 64, 0), (9, 7, 256, 0), (10, 6, 96, 0)])
def test_step_equals_render_loss_backward(oracle, fr, tiny, tiny_r, W, H, spp, terms):
    """fr_step (fused when spp divides 256, three calls otherwise) against
    fr_render + fr_loss + fr_render_backward: the same decisions, so image
    and d_image agree to FP32 rounding (the shading formulas compiled in two
    kernels may contract multiply-adds differently; above 32 spp fr_render
    also adds the samples atomically in no fixed order), the loss to 1e-6,
    the gradient up to the order of atomic additions; the 4-spp case also
    against the oracle's loss."""
    scene, theta, _ = tiny
    rng = np.random.default_rng(W * 100 + spp)
    tgt = rng.uniform(size=(H, W, 3)).astype(np.float32)
    mask = (rng.uniform(size=(H, W)) > 0.25).astype(np.uint8)
    m = rng.uniform(size=60).astype(np.float32)
    dev = lambda a: torch.tensor(a, device="cuda:0")
    th = dev(theta)
    w1, w2 = 0.02, 0.3
    ref_img, ref_loss, ref_g, ref_d = _three_calls(tiny_r, th, dev(tgt), dev(mask), dev(m), W, H, spp, 5, w1, w2,
                                                   terms)
    d_image = torch.empty(H, W, 3, device="cuda:0")
    img, loss, g = tiny_r.step(th, dev(tgt), W, H, spp, seed=5, mask=dev(mask), m=dev(m), w1=w1, w2=w2,
                               terms=terms, d_image=d_image)
    tiny_r.sync()
    rel = 1e-6 if spp <= 32 else 1e-5
    got_img = img.cpu().numpy()
    check_same_values(got_img, ref_img, what=f"fr_step image {W}x{H}x{spp} against fr_render", rel=rel)
    # d_image is 2 mask (image - target) of fr_step's own image
    d_own = 2.0 * mask[..., None] * (got_img.astype(np.float64) - tgt)
    assert np.all(np.abs(d_image.cpu().numpy() - d_own) <= 1e-6 * (np.abs(got_img) + np.abs(tgt)))
    img_scale = np.maximum(np.abs(ref_img), 1e-3 * np.abs(ref_img).max())
    assert np.all(np.abs(d_image.cpu().numpy() - ref_d) <= 2.0 * rel * img_scale + 1e-6 * np.abs(ref_d) + 1e-12)
    assert abs(loss.item() - ref_loss) <= 10 * rel * abs(ref_loss)
    assert_sum_order_close(g.cpu().numpy(), ref_g, what=f"step {W}x{H}x{spp}")
    if spp == 4:
        o_img = oracle.render(default_config(W=W, H=H, spp=spp, seed=5), scene, theta)
        val, _, _ = oracle.loss(default_config(W=W, H=H), scene, theta, o_img, tgt, mask, m, w1, w2)
        record_value(f"fr_step loss {W}x{H}x{spp}", loss.item(), val, loss_bound(o_img, tgt, mask) / abs(val))
    # without d_image the context's buffer is used; the results stay the same
    img2, loss2, g2 = tiny_r.step(th, dev(tgt), W, H, spp, seed=5, mask=dev(mask), m=dev(m), w1=w1, w2=w2,
                                  terms=terms)
    tiny_r.sync()
    if 32 % spp == 0:          # the same kernel again, a pixel's sum in one warp: bit for bit
        assert np.array_equal(img2.cpu().numpy(), img.cpu().numpy())
    else:                      # a pixel's samples may straddle two warps: atomic sums in no fixed order
        check_same_values(img2.cpu().numpy(), img.cpu().numpy(), what=f"fr_step image again {W}x{H}x{spp}",
                          rel=rel)
    assert abs(loss2.item() - loss.item()) <= (1e-12 if 32 % spp == 0 else 1e-6) * abs(ref_loss)
    assert_sum_order_close(g2.cpu().numpy(), ref_g, what="step, context d_image")


def test_counters_are_reset_per_call(fr, tiny, tiny_r):
    """Work counters describe the latest call: two identical calls report the
    same counts for every kernel."""
    _, theta, _ = tiny
    th = torch.tensor(theta, device="cuda:0")
    W, H, spp = 32, 24, 4
    d_image = torch.ones(H, W, 3, device="cuda:0")
    tiny_r.set_counters(True)
    try:
        seen = []
        for _ in range(2):
            tiny_r.render(th, W, H, spp, seed=2)
            tiny_r.backward(th, d_image, W, H, spp, seed=2)
            seen.append(tiny_r.counters().copy())
    finally:
        tiny_r.set_counters(False)
    assert np.array_equal(seen[0], seen[1]), (seen[0], seen[1])
    from paper_1910_05200_gb300 import roofline as RF
    c = seen[0]
    assert c[RF.K_FWD] > 0 and c[RF.K_INTERIOR] > 0 and c[RF.K_PEDGE] > 0 and c[RF.K_SEDGE + 2] > 0
    # every shadow-edge search classifies the leaf edges it reaches
    assert c[RF.K_SEDGE + 5] > 0


def test_all_lights_off_is_black(oracle, tiny, tiny_r):
    scene, theta, _ = tiny
    th = theta.copy()
    o = S.param_offsets()
    th[o["lights"]:] = 0
    t = torch.tensor(th, device="cuda:0")
    img = tiny_r.render(t, 16, 16, 2)
    assert img.abs().max().item() == 0
    dI = torch.ones(16, 16, 3, device="cuda:0")
    g = tiny_r.backward(t, dI, 16, 16, 2).cpu().numpy()
    ref, mass = oracle.render_backward(default_config(W=16, H=16, spp=2), scene, th, np.ones((16, 16, 3)),
                                       mass=True)
    assert np.all(g[:o["lights"]] == 0)         # nothing lit: no geometry, albedo or texture gradient
    assert np.abs(ref[o["lights"]:]).max() > 0   # but the lights still get their gradient
    assert_grad(g, ref, mass, what="lights off")


def test_errors_are_reported(fr, tiny):
    scene, theta, _ = tiny
    r = fr.Renderer(None, device=0)
    with pytest.raises(RuntimeError, match="not uploaded|upload"):
        r.P = len(theta)
        r.render(torch.tensor(theta, device="cuda:0"), 8, 8, 1)
    r2 = fr.Renderer(scene, device=0)
    with pytest.raises(RuntimeError, match="invalid argument"):
        r2.render(torch.tensor(theta, device="cuda:0"), 0, 8, 1)
    bad = S.Scene(scene.mean, np.concatenate([scene.tris, scene.tris[:1]]), scene.uv, scene.B_id, scene.B_exp,
                  scene.alb_mean, scene.B_alb)
    with pytest.raises(RuntimeError, match="shape"):
        fr.Renderer(bad, device=0)
    # fr_step: bad sizes and missing buffers are refused before any launch
    th = torch.tensor(theta, device="cuda:0")
    tgt = torch.zeros(8, 8, 3, device="cuda:0")
    with pytest.raises(RuntimeError, match="invalid argument"):
        r2.step(th, tgt, 8, 8, 0)
    import ctypes as C
    vp = lambda t: None if t is None else C.c_void_p(t.data_ptr())
    img = torch.empty(8, 8, 3, device="cuda:0")
    loss = torch.empty(1, device="cuda:0", dtype=torch.float64)
    g = torch.empty(r2.P, device="cuda:0", dtype=torch.float64)
    o = r2.opts(8, 8, 4)
    for missing in ("target", "image", "loss", "grad"):
        args = dict(target=tgt, image=img, loss=loss, grad=g)
        args[missing] = None
        rc = fr.load().fr_step(r2.ctx, vp(th), C.byref(o), vp(args["target"]), None, None, 0.0, 0.0,
                               vp(args["image"]), None, vp(args["loss"]), vp(args["grad"]))
        assert rc == -1, (missing, rc)
    with pytest.raises(RuntimeError, match="invalid argument"):
        fr.Renderer(scene, device=0, config=fr.default_config(light_prior=-1))


def test_large_image_and_size_limits(oracle, fr, tiny, tiny_r):
    """A 2048 x 1536 image (sampled pixels against the oracle) and a request
    of 2^31 samples, one beyond the limit, rejected before any work."""
    import ctypes as C
    scene, theta, _ = tiny
    th = torch.tensor(theta, device="cuda:0")
    W, H, spp = 2048, 1536, 2
    img = tiny_r.render(th, W, H, spp, seed=8)
    tiny_r.sync()
    got = img.cpu().numpy().reshape(-1, 3)
    lit = np.nonzero(got.sum(1) > 0)[0]
    assert len(lit) > 0
    pix = np.unique(np.concatenate([S.random_pixels(W, H, 32, seed=1),
                                    lit[:: max(1, len(lit) // 32)][:32]])).astype(np.int32)
    ref = oracle.render(default_config(W=W, H=H, spp=spp, seed=8), scene, theta, pixels=pix)
    assert_image(got[pix], ref, what="forward 2048x1536x2 sampled")
    opts = fr.FrRenderOpts(8192, 8192, 32, 0, 0, 0)
    small = torch.empty(3, device="cuda:0")
    rc = tiny_r.lib.fr_render(tiny_r.ctx, C.c_void_p(th.data_ptr()), C.byref(opts), C.c_void_p(small.data_ptr()),
                              None)
    assert rc == -1 and b"too large" in tiny_r.lib.fr_last_error(tiny_r.ctx)


# ---------------------------------------------------------------------------
# Full size (35,709 vertices, 256 x 256, 16 spp): sampled outputs

def test_full_size_forward_sampled_pixels(oracle, full, full_r):
    scene, theta, c = full
    W, H, spp = c["W"], c["H"], c["spp"]
    img = full_r.render(torch.tensor(theta, device="cuda:0"), W, H, spp, seed=3)
    full_r.sync()
    cfg = default_config(W=W, H=H, spp=spp, seed=3)
    # random pixels and pixels on the face (projected vertices of the oracle's mesh)
    pix = np.unique(np.concatenate([S.random_pixels(W, H, 48, seed=5),
                                    face_pixels(oracle, cfg, scene, theta, 48, seed=6)])).astype(np.int32)
    got = img.cpu().numpy().reshape(-1, 3)
    ref = oracle.render(cfg, scene, theta, pixels=pix)
    assert (ref.sum(1) > 0).sum() >= 40
    assert_image(got[pix], ref, what="full face forward 256x256x16 sampled")


def test_full_size_backward_masked_adjoint(oracle, full, full_r):
    """Gradient of <d_image, image> with d_image supported on a few pixels."""
    scene, theta, c = full
    W, H, spp = c["W"], c["H"], c["spp"]
    th = torch.tensor(theta, device="cuda:0")
    cfg = default_config(W=W, H=H, spp=spp, seed=3)
    rng = np.random.default_rng(0)
    pix = face_pixels(oracle, cfg, scene, theta, 12, seed=0)
    dI = np.zeros((H * W, 3), np.float32)
    dI[pix] = rng.normal(size=(len(pix), 3))
    dI = dI.reshape(H, W, 3)
    g = full_r.backward(th, torch.tensor(dI, device="cuda:0"), W, H, spp, seed=3).cpu().numpy()
    full_r.sync()
    ref, mass = oracle.render_backward(cfg, scene, theta, dI.astype(np.float64), mass=True)
    assert_grad(g, ref, mass, what="full size, masked adjoint")


def test_full_size_step_masked(oracle, full, full_r):
    """fr_step, the benchmarked call, at full size in its benchmarked launch
    configuration: E_data restricted by the mask to a few pixels on the face,
    a black target (d_image = 2 image there), w1 = w2 = 0.  Image on those
    pixels, loss and gradient against the oracle."""
    scene, theta, c = full
    W, H, spp = c["W"], c["H"], c["spp"]
    th = torch.tensor(theta, device="cuda:0")
    cfg = default_config(W=W, H=H, spp=spp, seed=4)
    pix = face_pixels(oracle, cfg, scene, theta, 12, seed=2)
    mask = np.zeros(H * W, np.uint8)
    mask[pix] = 1
    tgt = torch.zeros(H, W, 3, device="cuda:0")
    img, loss, g = full_r.step(th, tgt, W, H, spp, seed=4, mask=torch.tensor(mask.reshape(H, W), device="cuda:0"))
    full_r.sync()
    ref = oracle.render(cfg, scene, theta, pixels=pix)
    assert (ref.sum(1) > 0).sum() >= 10
    assert_image(img.cpu().numpy().reshape(-1, 3)[pix], ref, what="fr_step full face 256x256x16 masked pixels")
    e_ref = float(np.sum(ref ** 2))
    record_value("fr_step full face loss (masked pixels)", loss.item(), e_ref,
                 loss_bound(ref, np.zeros_like(ref)) / e_ref)
    dI = np.zeros((H * W, 3))
    dI[pix] = 2.0 * ref
    gref, mass = oracle.render_backward(cfg, scene, theta, dI.reshape(H, W, 3), mass=True)
    assert_grad(g.cpu().numpy(), gref, mass, what="fr_step full face gradient (masked pixels)")


@pytest.mark.parametrize("model,fresnel,layout", [(1, 0, 0), (0, 1, 0), (1, 1, 1)])
def test_alternative_readings_match_oracle(oracle, fr, tiny, model, fresnel, layout):
    """GGX + Smith, Schlick's Fresnel and the icosphere dome: light stage,
    forward image and all gradient terms against the oracle."""
    scene, theta, _ = tiny
    kw = dict(brdf_model=model, fresnel=fresnel, light_layout=layout)
    r = fr.Renderer(scene, device=0, config=fr.default_config(**kw))
    assert np.array_equal(r.light_stage(), oracle.light_stage(20, 3.0, layout))
    W, H, spp = 40, 33, 4
    th = torch.tensor(theta, device="cuda:0")
    img = r.render(th, W, H, spp, seed=6)
    r.sync()
    cfg = default_config(W=W, H=H, spp=spp, seed=6, **kw)
    assert_image(img.cpu().numpy(), oracle.render(cfg, scene, theta), what=f"readings {kw} forward")
    dI = np.random.default_rng(12).normal(size=(H, W, 3)).astype(np.float32)
    g = r.backward(th, torch.tensor(dI, device="cuda:0"), W, H, spp, seed=6).cpu().numpy()
    r.sync()
    ref, mass = oracle.render_backward(cfg, scene, theta, dI.astype(np.float64), mass=True)
    # named exceptions (tests/parity.py): components with a cancellation ratio
    # of 300 or more, against 1e-5 of their mass
    assert_grad(g, ref, mass, what=f"readings {kw}", cancel=300.0, kappa=1e-5)


def test_degenerate_images(oracle, tiny, tiny_r):
    """A one-pixel image at one sample, and a face moved out of view (no
    primary hit, no camera silhouette): black image, zero gradient."""
    scene, theta, _ = tiny
    th = torch.tensor(theta, device="cuda:0")
    img = tiny_r.render(th, 1, 1, 1, seed=2)
    tiny_r.sync()
    ref = oracle.render(default_config(W=1, H=1, spp=1, seed=2), scene, theta)
    assert_image(img.cpu().numpy(), ref, what="forward 1x1x1")
    g = tiny_r.backward(th, torch.ones(1, 1, 3, device="cuda:0"), 1, 1, 1, seed=2).cpu().numpy()
    tiny_r.sync()
    gref, mass = oracle.render_backward(default_config(W=1, H=1, spp=1, seed=2), scene, theta, np.ones((1, 1, 3)),
                                        mass=True)
    assert_grad(g, gref, mass, what="1x1")
    away = theta.copy()
    away[S.param_offsets()["pose"] + 3] = 50.0      # tx: far outside the field of view
    t = torch.tensor(away, device="cuda:0")
    img = tiny_r.render(t, 20, 12, 2)
    assert img.abs().max().item() == 0
    g = tiny_r.backward(t, torch.ones(12, 20, 3, device="cuda:0"), 20, 12, 2).cpu().numpy()
    tiny_r.sync()
    assert np.all(g == 0)
    assert np.abs(oracle.render(default_config(W=20, H=12, spp=2), scene, away)).max() == 0
