"""Device-side limits reach the caller as FR_ERR_DEVICE_LIMIT (fr_sync).

Each limit is made to run out through fr_set_limits: a traversal step cap of
one node visit (every ray and every edge search stops at once) and a batch
wait limit of zero tries (an edge item of the persistent batch kernel that
finds its frame's tiles unfinished gives up at once).  Both are
host-visible error returns: nothing faults and nothing spins.  The test then
checks that the flag clears and that the next call with the default limits
gives the same results as before.
"""
import numpy as np
import pytest
import torch

from paper_1910_05200_gb300 import synthetic as S

pytestmark = pytest.mark.gpu
DEVICE_LIMIT = -5


@pytest.fixture(scope="module")
def fr():
    from paper_1910_05200_gb300 import build, facert
    build.build()
    return facert


def test_traversal_step_cap_is_reported(fr, tiny):
    scene, theta, _ = tiny
    r = fr.Renderer(scene, device=0)
    th = torch.tensor(theta, device="cuda:0")
    dI = torch.ones(32, 32, 3, device="cuda:0")
    ref = r.render(th, 32, 32, 2, seed=1).cpu().numpy()
    g_ref = r.backward(th, dI, 32, 32, 2, seed=1).cpu().numpy()
    assert r.sync_code() == 0
    r.set_limits(max_steps=1)
    r.render(th, 32, 32, 2, seed=1)
    assert r.sync_code() == DEVICE_LIMIT
    assert r.sync_code() == 0                     # fr_sync cleared the flag
    r.backward(th, dI, 32, 32, 2, seed=1)
    assert r.sync_code() == DEVICE_LIMIT
    r.set_limits()                                # defaults again
    img = r.render(th, 32, 32, 2, seed=1).cpu().numpy()
    g = r.backward(th, dI, 32, 32, 2, seed=1).cpu().numpy()
    assert r.sync_code() == 0
    assert np.array_equal(img, ref)
    assert np.abs(g - g_ref).max() <= 1e-4 * np.abs(g_ref).max()
    for bad in [(0, 10), (10, -1)]:
        with pytest.raises(RuntimeError, match="invalid argument"):
            r.set_limits(*bad)


def test_batch_wait_limit_is_reported(fr, tiny):
    """One 64 x 64 frame in the persistent kernel: its 64 tile items go to the
    first 64 warps, and the next warps take edge items while the tiles still
    render; with a wait limit of zero those items stop at once."""
    scene, _, _ = tiny
    r = fr.Renderer(scene, device=0)
    frames, thetas = S.make_batch(scene, n_frames=1, seed=9, n_on=8, max_angle_deg=10.0, t_std=0.02,
                                  sizes=[(64, 64)])
    b = fr.Batch(r, frames, 4)
    b.set_targets(torch.tensor(S.noise_images(frames, seed=3), device="cuda:0"))
    b.set_config(8, 8, 256, 4, 1)
    ts, tf = fr.split_theta(thetas)
    ts, tf = torch.tensor(ts[0], device="cuda:0"), torch.tensor(tf, device="cuda:0")
    l0, gs0, gf0, img0 = b.step(ts, tf, 0.01, 0.01, iter=2)
    l0, gs0, img0 = l0.item(), gs0.cpu().numpy(), img0.cpu().numpy()
    assert r.sync_code() == 0
    r.set_limits(wait_limit=0)
    b.step(ts, tf, 0.01, 0.01, iter=2)
    assert r.sync_code() == DEVICE_LIMIT
    r.set_limits()
    l1, gs1, _, img1 = b.step(ts, tf, 0.01, 0.01, iter=2)
    assert r.sync_code() == 0
    assert np.array_equal(img1.cpu().numpy(), img0)
    assert abs(l1.item() - l0) <= 1e-12 * abs(l0)
    assert np.abs(gs1.cpu().numpy() - gs0).max() <= 1e-4 * np.abs(gs0).max()
