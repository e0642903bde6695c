"""Host-side logic of batched frames: the seeded frame recipe and the split of
the parameter vector into shared and per-frame parts (no GPU)."""
import numpy as np

from paper_1910_05200_gb300 import facert
from paper_1910_05200_gb300 import synthetic as S


def test_split_join_round_trip():
    th = np.arange(1340, dtype=np.float32)
    sh, fr = facert.split_theta(th)
    assert sh.shape == (80 + 80 + 1024,) and fr.shape == (90 + 6 + 60,)
    assert np.array_equal(sh[:80], th[:80]) and np.array_equal(sh[80:160], th[170:250])
    assert np.array_equal(fr[:90], th[80:170]) and np.array_equal(fr[90:], th[1274:])
    assert np.array_equal(facert.join_theta(sh, fr), th)
    two = np.stack([th, th + 1])
    s2, f2 = facert.split_theta(two)
    assert s2.shape == (2, 1184) and f2.shape == (2, 156)


def test_batch_recipe():
    scene = S.make_scene("tiny", seed=0)
    frames, thetas = S.make_batch(scene, n_frames=32, seed=100)
    sides = [w for w, h, _ in frames]
    assert all(w == h for w, h, _ in frames)
    assert min(sides) >= 128 and max(sides) <= 320 and all(s % 8 == 0 for s in sides)
    assert len({sd for _, _, sd in frames}) == 32
    sh, fr = facert.split_theta(thetas)
    assert np.all(sh == sh[0])                          # alpha, delta, c_spec shared
    assert len({tuple(f[:90]) for f in fr}) == 32       # beta per frame
    assert len({tuple(f[90:96]) for f in fr}) == 32     # pose per frame
    lights = fr[:, 96:].reshape(32, 20, 3)
    assert np.all((lights != 0).any(-1).sum(-1) == 14)  # 14 of 20 lights on in every frame
    # the side distribution spans the range
    assert max(sides) - min(sides) >= 120


def test_noise_images_packing():
    frames = [(3, 2, 0), (5, 4, 1)]
    t = S.noise_images(frames, seed=1)
    assert t.shape == (26, 3) and t.dtype == np.float32 and t.min() >= 0 and t.max() <= 0.5
