"""Batched frames: the persistent render + loss + backward in a CUDA graph.

Checked frame by frame against the oracle (images, loss, gradients of the
shared and per-frame parameters), against the single-image path of the same
library (same samples and decisions: images equal to FP32 rounding, gradients
equal up to the order of floating-point atomic additions), across launch
configurations of the autotuner, and at the full size of 32 frames of the
35,709-vertex face.

Tolerances (tests/parity.py): against the oracle, those of the single-image
parity tests (1e-3 of each entry with a floor of 1e-3 of the group's
largest); between two GPU runs that differ only in the order of FP32 atomic
additions, 1e-4 of the group's largest plus 1e-3 of the entry.
"""
import numpy as np
import pytest
import torch

from oracle import default_config
from paper_1910_05200_gb300 import synthetic as S
from tests.parity import assert_image, check_close, check_groups, check_same_values, record_value

pytestmark = pytest.mark.gpu

SIZES = [(24, 24), (19, 31), (40, 33)]       # uneven, ragged against every tile shape
SPP, ITER, W1, W2 = 4, 3, 0.02, 0.002
K = (80, 90, 80)


def shared_groups():
    return {"alpha": slice(0, 80), "delta": slice(80, 160), "cspec": slice(160, 1184)}


def frame_groups():
    return {"beta": slice(0, 90), "pose": slice(90, 96), "lights": slice(96, 156)}


def assert_groups(got, ref, groups, mass=None, what="", named=None):
    check_groups(got, ref, groups, mass, named=named, what=what)


def assert_atomic_close(got, ref, groups, what=""):
    check_close(got, ref, groups, what=what)


def combine(fr, per_frame, thetas, m, w1, w2):
    """Per-frame full gradients (data term) -> batch layout plus the prior and
    light terms, each parameter counted once (weights as the FP32 values the
    library receives)."""
    w1, w2 = float(np.float32(w1)), float(np.float32(w2))
    shared = sum(fr.split_theta(g)[0] for g in per_frame)
    frames = np.stack([fr.split_theta(g)[1] for g in per_frame])
    ts, tf = fr.split_theta(thetas.astype(np.float64))
    shared[:80] += 2 * w1 * ts[0, :80]
    shared[80:160] += 2 * w1 * ts[0, 80:160]
    frames[:, :90] += 2 * w1 * tf[:, :90]
    frames[:, 96:] += 2 * w2 * (tf[:, 96:] - m.astype(np.float64))
    reg = w1 * (np.sum(ts[0, :160] ** 2) + np.sum(tf[:, :90] ** 2)) + w2 * np.sum((tf[:, 96:] - m) ** 2)
    return shared, frames, reg


@pytest.fixture(scope="module")
def fr():
    from paper_1910_05200_gb300 import build, facert
    build.build()
    return facert


def dev(a):
    return torch.tensor(np.ascontiguousarray(a), device="cuda:0")


class Case:
    def __init__(self, fr, scene, sizes, spp, seed=7, config=None):
        self.fr, self.scene, self.spp = fr, scene, spp
        self.r = fr.Renderer(scene, device=0, config=config)
        self.frames, self.thetas = S.make_batch(scene, seed=seed, n_on=8, max_angle_deg=10.0, t_std=0.02,
                                                sizes=sizes)
        self.targets = S.noise_images(self.frames, seed=seed + 1)
        rng = np.random.default_rng(seed + 2)
        self.masks = (rng.uniform(size=len(self.targets)) > 0.2).astype(np.uint8)
        self.m = rng.uniform(0, 1, 60).astype(np.float32)
        self.b = fr.Batch(self.r, self.frames, spp)
        self.b.set_targets(dev(self.targets), dev(self.masks), dev(self.m))
        ts, tf = fr.split_theta(self.thetas)
        self.ts, self.tf = dev(ts[0]), dev(tf)

    def step(self, it=ITER):
        loss, gs, gf, img = self.b.step(self.ts, self.tf, W1, W2, iter=it)
        self.r.sync()
        return loss.item(), gs.cpu().numpy(), gf.cpu().numpy(), img.cpu().numpy()

    def frame_slices(self, packed):
        out, o = [], 0
        for w, h, _ in self.frames:
            out.append(packed[o:o + w * h].reshape(h, w, *packed.shape[1:]))
            o += w * h
        return out


@pytest.fixture(scope="module")
def case(fr, tiny):
    return Case(fr, tiny[0], SIZES, SPP)


@pytest.mark.parametrize("fused", [0, 1])
def test_batch_matches_oracle(oracle, fr, case, fused):
    case.b.set_config(4, 4, 256, 4, fused) if fused else case.b.set_config(8, 8, 256, 4, 0)
    loss, gs, gf, img = case.step()
    imgs = case.frame_slices(img)
    tgts = case.frame_slices(case.targets)
    masks = case.frame_slices(case.masks)
    per_frame, masses, e_data = [], [], 0.0
    for f, (w, h, seed) in enumerate(case.frames):
        cfg = default_config(W=w, H=h, spp=SPP, seed=seed, iter=ITER)
        ref = oracle.render(cfg, case.scene, case.thetas[f])
        assert_image(imgs[f], ref, what=f"batch ({'persistent' if fused else 'phased'}) frame {f} {w}x{h}x{SPP}")
        d = 2.0 * masks[f][..., None] * (ref - tgts[f])
        e_data += float(np.sum(masks[f][..., None] * (ref - tgts[f]) ** 2))
        g, mass = oracle.render_backward(cfg, case.scene, case.thetas[f], d, mass=True)
        per_frame.append(g)
        masses.append(mass)
    gs_ref, gf_ref, reg = combine(fr, per_frame, case.thetas, case.m, W1, W2)
    ms_ref, mf_ref, _ = combine(fr, masses, case.thetas * 0, case.m * 0, 0.0, 0.0)
    mode = "persistent" if fused else "phased"
    record_value(f"batch ({mode}) loss", loss, e_data + reg, 1e-5)
    assert_groups(gs, gs_ref, shared_groups(), ms_ref, what=f"batch ({mode}) shared")
    for f in range(len(case.frames)):
        assert_groups(gf[f], gf_ref[f], frame_groups(), mf_ref[f], what=f"batch ({mode}) frame {f}")


@pytest.mark.parametrize("fused", [0, 1])
def test_batch_equals_single_image_path(fr, case, fused):
    case.b.set_config(2, 2, 128, 2, fused) if fused else case.b.set_config(8, 8, 256, 3, 0)
    loss, gs, gf, img = case.step()
    imgs = case.frame_slices(img)
    tgts = case.frame_slices(case.targets)
    masks = case.frame_slices(case.masks)
    r = case.r
    per_frame, e_data = [], 0.0
    for f, (w, h, seed) in enumerate(case.frames):
        th = dev(case.thetas[f])
        single = r.render(th, w, h, SPP, seed=seed, iter=ITER)
        check_same_values(single.cpu().numpy(), imgs[f], what=f"batch frame {f} against fr_render")
        d_image = torch.empty(h, w, 3, device="cuda:0")
        e_data += r.loss(th, single, dev(tgts[f]), dev(masks[f]), None, 0.0, 0.0, d_image).item()
        per_frame.append(r.backward(th, d_image, w, h, SPP, seed=seed, iter=ITER).cpu().numpy())
    r.sync()
    gs_ref, gf_ref, reg = combine(fr, per_frame, case.thetas, case.m, W1, W2)
    assert abs(loss - (e_data + reg)) <= 1e-6 * abs(e_data + reg)
    assert_atomic_close(gs, gs_ref, shared_groups(), "shared")
    for f in range(len(case.frames)):
        assert_atomic_close(gf[f], gf_ref[f], frame_groups(), f"frame {f}")


def test_steps_are_deterministic_and_keyed_by_iter(case):
    l1, g1, f1, i1 = case.step(ITER)
    l2, g2, f2, i2 = case.step(ITER)
    l3, _, _, i3 = case.step(ITER + 1)
    assert np.array_equal(i1, i2)
    assert abs(l1 - l2) <= 1e-12 * abs(l1)
    assert_atomic_close(g2, g1, shared_groups(), "replay")
    assert not np.array_equal(i1, i3)


def test_autotuner_table_and_configuration_invariance(case):
    _, gs0, gf0, img0 = case.step()
    table, chosen = case.b.autotune(case.ts, case.tf, reps=1)
    keys = ("tile_w", "tile_h", "block", "min_blocks", "fused")
    assert len(table) == 6 and {t["fused"] for t in table} == {0, 1}
    best = min(table, key=lambda t: t["ms"])
    assert tuple(chosen[k] for k in keys) == tuple(best[k] for k in keys)
    for cfg in [(8, 8, 256, 3, 0), (8, 8, 256, 4, 0), (2, 2, 256, 2, 1), (4, 4, 128, 3, 1), (16, 8, 64, 4, 1),
                (5, 3, 96, 2, 1)]:
        case.b.set_config(*cfg)
        _, gs, gf, img = case.step()
        check_same_values(img, img0, what=f"batch config {cfg} against the first")
        assert_atomic_close(gs, gs0, shared_groups(), f"config {cfg}")
        for f in range(len(case.frames)):
            assert_atomic_close(gf[f], gf0[f], frame_groups(), f"config {cfg} frame {f}")
    case.b.set_config(8, 8, 256, 4, 0)


@pytest.mark.parametrize("fused", [0, 1])
def test_spp_multiple_of_32(fr, tiny, fused):
    """spp = 64 in both launch modes: the phased launches sum a pixel's
    samples over two warps of a block through shared memory; the persistent
    kernel takes each pixel in two passes (radiance, then the adjoints with
    the primary hit traced again).  The single-image forward sums such pixels
    with atomics, so images agree to rounding."""
    c = Case(fr, tiny[0], [(9, 7), (12, 10)], 64, seed=21)
    assert c.b.config()["fused"] == 0                 # phased by default: 64 divides 256
    if fused:
        c.b.set_config(4, 4, 256, 2, 1)
    loss, gs, gf, img = c.step()
    imgs = c.frame_slices(img)
    tgts, masks = c.frame_slices(c.targets), c.frame_slices(c.masks)
    per_frame = []
    for f, (w, h, seed) in enumerate(c.frames):
        th = dev(c.thetas[f])
        single = c.r.render(th, w, h, 64, seed=seed, iter=ITER).cpu().numpy()
        assert np.allclose(imgs[f], single, rtol=1e-5, atol=1e-7)
        d_image = torch.empty(h, w, 3, device="cuda:0")
        c.r.loss(th, dev(imgs[f]), dev(tgts[f]), dev(masks[f]), None, 0.0, 0.0, d_image)
        per_frame.append(c.r.backward(th, d_image, w, h, 64, seed=seed, iter=ITER).cpu().numpy())
    gs_ref, gf_ref, _ = combine(fr, per_frame, c.thetas, c.m, W1, W2)
    assert_atomic_close(gs, gs_ref, shared_groups(), f"spp 64 shared, fused {fused}")
    for f in range(len(c.frames)):
        assert_atomic_close(gf[f], gf_ref[f], frame_groups(), f"spp 64 frame {f}, fused {fused}")


def test_unsupported_spp_is_refused(fr, case):
    for spp in (3, 48):
        with pytest.raises(RuntimeError):
            fr.Batch(case.r, [(8, 8, 0)], spp)
    b96 = fr.Batch(case.r, [(8, 8, 0)], 96)
    assert b96.config()["fused"] == 1
    with pytest.raises(RuntimeError):
        b96.set_config(8, 8, 256, 4, 0)          # phased launches need spp dividing 256


def test_invalid_configurations_are_refused(case):
    for cfg in [(0, 8, 256, 2, 1), (65, 8, 256, 2, 1), (8, 8, 100, 2, 1), (8, 8, 256, 5, 1), (8, 8, 256, 2, 0),
                (8, 8, 256, 4, 2)]:
        with pytest.raises(RuntimeError):
            case.b.set_config(*cfg)


def test_full_size_batch_equals_single_frames(oracle, fr):
    """32 frames of the 35,709-vertex face, crops 128..320, 16 spp: images of
    two frames equal to fr_render up to FP32 rounding and sampled pixels against the
    oracle; the batch gradient equal to the sum of the single-image
    gradients of all frames."""
    cfg = S.BATCH
    scene = S.make_scene(cfg["kind"], seed=0)
    frames, thetas = S.make_batch(scene, n_frames=cfg["n_frames"], seed=cfg["seed"], n_on=cfg["n_on"],
                                  max_angle_deg=cfg["max_angle_deg"], t_std=cfg["t_std"])
    sides = [w for w, _, _ in frames]
    assert min(sides) >= 128 and max(sides) <= 320 and len(set(sides)) > 8
    spp = cfg["spp"]
    r = fr.Renderer(scene, device=0)
    b = fr.Batch(r, frames, spp)
    targets = S.noise_images(frames, seed=5, lo=0.0, hi=0.3)
    b.set_targets(dev(targets))
    ts, tf = fr.split_theta(thetas)
    loss, gs, gf, img = b.step(dev(ts[0]), dev(tf), 0.0, 0.0, iter=1)
    r.sync()
    gs, gf, img = gs.cpu().numpy(), gf.cpu().numpy(), img.cpu().numpy()
    assert np.isfinite(loss.item()) and np.all(np.isfinite(gs)) and np.all(np.isfinite(gf))
    imgs = b.split(img)
    tg = b.split(targets)
    per_frame = []
    for f, (w, h, seed) in enumerate(frames):
        th = dev(thetas[f])
        single = r.render(th, w, h, spp, seed=seed, iter=1)
        d_image = torch.empty(h, w, 3, device="cuda:0")
        r.loss(th, single, dev(tg[f]), None, None, 0.0, 0.0, d_image)
        per_frame.append(r.backward(th, d_image, w, h, spp, seed=seed, iter=1).cpu().numpy())
        if f in (int(np.argmin(sides)), int(np.argmax(sides))):
            s = single.cpu().numpy()
            check_same_values(s, imgs[f], what=f"full-size batch frame {f} against fr_render")
            lit = np.nonzero(s.reshape(-1, 3).sum(1) > 0)[0]
            pix = np.unique(np.concatenate([S.random_pixels(w, h, 16, seed=f),
                                            lit[:: max(1, len(lit) // 16)][:16]])).astype(np.int32)
            ref = oracle.render(default_config(W=w, H=h, spp=spp, seed=seed, iter=1), scene, thetas[f], pixels=pix)
            assert_image(s.reshape(-1, 3)[pix], ref, what=f"full-size batch frame {f} {w}x{h}x{spp} sampled")
    r.sync()
    gs_ref, gf_ref, _ = combine(fr, per_frame, thetas, np.zeros(60, np.float32), 0.0, 0.0)
    assert_atomic_close(gs, gs_ref, shared_groups(), "full size shared")
    for f in range(len(frames)):
        assert_atomic_close(gf[f], gf_ref[f], frame_groups(), f"full size frame {f}")


def test_targets_masks_and_prior_can_be_replaced(fr, tiny):
    """set_targets between steps: dropping the mask adds the masked-out
    pixels' E_data, dropping m turns the light term into w2 sum |l|^2;
    restoring both restores the loss."""
    c = Case(fr, tiny[0], [(16, 12), (9, 13)], 4, seed=31)
    l_full, _, _, img = c.step()
    c.b.set_targets(dev(c.targets))
    l_plain, _, _, img2 = c.step()
    assert np.array_equal(img, img2)
    c.b.set_targets(dev(c.targets), dev(c.masks), dev(c.m))
    l_again, _, _, _ = c.step()
    assert l_again == pytest.approx(l_full, rel=1e-12)
    w2 = float(np.float32(W2))
    out = c.masks == 0
    extra = float(np.sum((img[out].astype(np.float64) - c.targets[out]) ** 2))
    _, tf = fr.split_theta(c.thetas.astype(np.float64))
    lights = tf[:, 96:]
    prior_change = w2 * float(np.sum(lights ** 2) - np.sum((lights - c.m.astype(np.float64)) ** 2))
    assert l_plain - l_full == pytest.approx(extra + prior_change, rel=1e-9, abs=1e-9)


@pytest.mark.parametrize("prior", [1, 2])
def test_batch_light_prior_readings(oracle, fr, tiny, prior):
    """m following each frame's own lights (mean per channel; each light's
    channel mean): the light term of the batch loss and its gradient against
    the oracle frame by frame.  A second step with w2 = 0 takes out the data
    term; the given m is ignored."""
    c = Case(fr, tiny[0], [(16, 12), (9, 13)], 4, seed=51, config=fr.default_config(light_prior=prior))
    w2 = 5.0
    l0, _, f0, _ = c.b.step(c.ts, c.tf, W1, 0.0, iter=ITER, images=False)
    l1, _, f1, _ = c.b.step(c.ts, c.tf, W1, w2, iter=ITER, images=False)
    c.r.sync()
    o = S.param_offsets(*K)
    z = np.zeros((1, 1, 3), np.float32)
    e_light, g_light = 0.0, []
    for f in range(len(c.frames)):
        val, _, gr = oracle.loss(default_config(W=1, H=1, light_prior=prior), c.scene, c.thetas[f], z, z,
                                 None, None, 0.0, w2)
        e_light += val
        g_light.append(gr[o["lights"]:o["lights"] + 60])
    assert l1.item() - l0.item() == pytest.approx(e_light, rel=1e-9)
    dg = (f1 - f0).cpu().numpy()[:, 96:]
    for f in range(len(c.frames)):
        ref = g_light[f]
        assert np.all(np.abs(dg[f] - ref) <= 1e-4 * np.abs(ref).max() + 1e-6 * np.abs(ref)), f


def test_batch_refuses_after_new_mesh(fr, tiny):
    """A batch is sized for the mesh and bases of its context: after a new
    upload its steps are refused, and a new batch works."""
    c = Case(fr, tiny[0], [(8, 8)], 4, seed=41)
    c.step()
    c.r.upload(tiny[0])
    with pytest.raises(RuntimeError, match="not uploaded|changed"):
        c.b.step(c.ts, c.tf, W1, W2, iter=ITER)
    b2 = fr.Batch(c.r, c.frames, 4)
    b2.set_targets(dev(c.targets))
    loss, _, _, _ = b2.step(c.ts, c.tf, W1, W2, iter=ITER)
    c.r.sync()
    assert np.isfinite(loss.item())
