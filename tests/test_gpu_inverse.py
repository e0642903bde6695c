"""Inverse loop on the GPU: the staged Adam fit lowers the loss and moves the
parameters toward the ground truth; fr_adam_step matches the FP64 reference."""
import numpy as np
import pytest
import torch

from oracle import mlp
from paper_1910_05200_gb300 import inverse as INV
from paper_1910_05200_gb300 import synthetic as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def r(tiny):
    from paper_1910_05200_gb300 import build, facert
    build.build()
    return facert.Renderer(tiny[0], device=0)


def test_adam_step_matches_reference_and_constraints(r):
    P = r.P
    rng = np.random.default_rng(0)
    th = rng.normal(size=P).astype(np.float32)
    o = S.param_offsets()
    th[o["lights"]:] = rng.uniform(0, 0.01, P - o["lights"])
    g = rng.normal(size=P)
    lr = INV.lr_vector(("alpha", "cspec", "lights"))
    m = np.zeros(P, np.float32)
    v = np.zeros(P, np.float32)
    t = torch.tensor(th, device="cuda:0")
    mt, vt = torch.tensor(m, device="cuda:0"), torch.tensor(v, device="cuda:0")
    r.adam_step(t, torch.tensor(g, device="cuda:0"), mt, vt, torch.tensor(lr, device="cuda:0"), 1)
    got = t.cpu().numpy()
    ref, _, _ = mlp.adam_step(th.astype(np.float64), g, np.zeros(P), np.zeros(P), 1, lr.astype(np.float64))
    ref[o["lights"]:] = np.maximum(ref[o["lights"]:], 0)
    ref[o["cspec"]:o["pose"]] = np.clip(ref[o["cspec"]:o["pose"]], 0, 1)
    ref[lr == 0] = th[lr == 0]
    assert np.allclose(got, ref, rtol=1e-6, atol=2e-7)   # FP32 update of values ~1
    assert np.all(got[o["lights"]:] >= 0)


def test_inverse_loop_fits_tiny_face(r, tiny):
    scene, _, _ = tiny
    W = H = 32
    truth = S.make_theta(scene, seed=21, n_on=8)
    target = r.render(torch.tensor(truth, device="cuda:0"), W, H, 64, seed=3)
    res = INV.optimize(r, target, W, H, 4, iters=150, seed=1)
    first, last = res.loss[:5].mean(), res.loss[-10:].mean()
    e0 = INV.parameter_errors(INV.initial_theta(), truth)
    e1 = INV.parameter_errors(res.theta, truth)
    print("loss", first, "->", last, "errors", e0, "->", e1, "ms/iter", res.ms_per_iter)
    assert last < 0.3 * first
    assert e1["lights"] < e0["lights"]


def test_checkpoint_and_resume(r, tiny, tmp_path):
    """A run interrupted after 30 of 60 iterations and resumed from its
    checkpoint ends where an uninterrupted run ends: the state (theta, Adam
    moments, stage step, losses) is restored and the samples of an iteration
    depend only on (seed, iteration).  Two runs differ in the order of
    floating-point atomic additions inside each gradient, which Adam
    amplifies in components whose gradient is near zero (a flipped sign moves
    them by the learning rate), so the runs are compared by their losses and
    by the distance of their parameters relative to how far the second half
    moves them."""
    scene, _, _ = tiny
    W = H = 24
    truth = S.make_theta(scene, seed=22, n_on=8)
    target = r.render(torch.tensor(truth, device="cuda:0"), W, H, 64, seed=3)
    full = INV.optimize(r, target, W, H, 4, iters=60, seed=2)
    ck = str(tmp_path / "state.npz")
    part = INV.optimize(r, target, W, H, 4, iters=60, seed=2, checkpoint=ck, checkpoint_every=10, stop_after=30)
    z = np.load(ck)
    assert int(z["it"]) == 30 and int(z["step_in_stage"]) >= 1
    assert np.array_equal(z["theta"], part.theta)
    rest = INV.optimize(r, target, W, H, 4, iters=60, seed=2, resume=ck)
    d_rest = np.linalg.norm(rest.theta - full.theta)
    d_half = np.linalg.norm(part.theta - full.theta)
    assert d_rest <= 0.1 * d_half, (d_rest, d_half)
    # two uninterrupted runs already differ by up to about 2 % of |theta| here
    # (atomic order through Adam); 3 % still catches a resume that restored
    # the wrong state
    assert d_rest <= 3e-2 * np.linalg.norm(full.theta)
    assert np.array_equal(rest.loss[:30], part.loss[:30])          # restored from the checkpoint
    np.testing.assert_allclose(rest.loss[:30], full.loss[:30], rtol=1e-2)
    assert abs(rest.loss[-10:].mean() - full.loss[-10:].mean()) <= 2e-2 * full.loss[-10:].mean()
