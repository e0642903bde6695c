"""Host-side logic of batched frames: the seeded frame recipe and the split of
the parameter vector into shared and per-frame parts (no GPU)."""
import numpy as np
import pytest

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


SEDGE, PEDGE = 1 << 29, 1 << 30


def _check_plan(frames, spp, tw, th, n_lights):
    it = facert.batch_plan(frames, spp, tw, th, n_lights)
    x, y = it[:, 0], it[:, 1]
    kind = np.where(x & PEDGE, 2, np.where(x & SEDGE, 1, 0))
    f = x & ~(PEDGE | SEDGE)
    assert np.all(y >= 0) and np.all((f >= 0) & (f < len(frames)))
    # tile items, then shadow-edge items, then primary-edge items: every item
    # an edge item waits for (its frame's tiles) is ahead of it in the queue
    assert np.all(np.diff(kind) >= 0) and set(kind.tolist()) == {0, 1, 2}
    area = [w * h for w, h, _ in frames]
    order = sorted(range(len(frames)), key=lambda i: -area[i])      # stable: larger frames first
    for k in range(3):
        seq = f[kind == k]
        firsts = [int(v) for i, v in enumerate(seq) if i == 0 or seq[i - 1] != v]
        assert firsts == order, (k, firsts, order)                   # each frame's items contiguous, in order
    for i, (w, h, _) in enumerate(frames):
        n_tiles = -(-w // tw) * -(-h // th)
        assert sorted(y[(kind == 0) & (f == i)].tolist()) == list(range(n_tiles))
        nc = -(-(n_tiles * tw * th * spp) // 32)
        ys = y[(kind == 1) & (f == i)]
        jk = [(int(v) & 31, int(v) >> 5) for v in ys]
        assert jk == [(j, c) for j in range(n_lights) for c in range(nc)]   # light-major, each chunk once
        npe = -(-(w * h * spp) // 32)
        assert y[(kind == 2) & (f == i)].tolist() == list(range(npe))
    return it


def test_persistent_plan_order_and_coverage():
    """The persistent launch's work items (fr_batch_plan, host only): every
    tile, every (light, 32-sample chunk) and every primary-edge chunk of each
    frame exactly once; tile items before all edge items, which the bounded
    waits of the edge items rely on to end; shadow-edge items light-major."""
    frames = [(40, 24, 1), (17, 33, 2), (64, 64, 3), (8, 5, 4), (17, 33, 5)]
    _check_plan(frames, 4, 2, 2, 20)
    _check_plan(frames, 16, 5, 3, 14)
    _check_plan(frames, 64, 4, 4, 3)        # spp a multiple of 32
    one = _check_plan([(3, 2, 0)], 1, 4, 4, 1)     # one tile of 16 tile-order samples: one chunk each
    assert one.tolist() == [[0, 0], [SEDGE, 0], [PEDGE, 0]]


def test_persistent_plan_refusals():
    ok = [(16, 16, 0)]
    for args in [(ok, 3, 2, 2, 20), (ok, 48, 2, 2, 20), (ok, 4, 0, 2, 20), (ok, 4, 2, 65, 20), (ok, 4, 2, 2, 0),
                 (ok, 4, 2, 2, 33), ([(0, 16, 0)], 4, 2, 2, 20), ([(8192, 8193, 0)], 1, 2, 2, 20),
                 ([(8192, 8192, 0)], 16, 1, 1, 20)]:          # the last: too many chunks for the item encoding
        with pytest.raises(RuntimeError, match="invalid argument"):
            facert.batch_plan(*args)


def _simulate_queue(items, n_tiles, n_warps, rng):
    """A model of the persistent kernel's scheduling: n_warps resident warps
    each take the next item from the queue when idle; a tile item finishes
    after a random time; an edge item spins until its frame's tile items have
    all finished, then finishes after a random time.  Returns the number of
    items finished before no warp can make progress."""
    x = items[:, 0]
    kind = np.where(x & PEDGE, 2, np.where(x & SEDGE, 1, 0))
    f = x & ~(PEDGE | SEDGE)
    done_tiles = np.zeros(len(n_tiles), np.int64)
    nxt, finished = 0, 0
    warps = [None] * n_warps          # (item, remaining time) or None
    while True:
        for w in range(n_warps):
            if warps[w] is None and nxt < len(items):
                warps[w] = [nxt, int(rng.integers(1, 5))]
                nxt += 1
        progressed = False
        for w in range(n_warps):
            if warps[w] is None:
                continue
            i, t = warps[w]
            if kind[i] != 0 and done_tiles[f[i]] < n_tiles[f[i]]:
                continue                  # spinning on the frame's tiles
            progressed = True
            warps[w][1] = t - 1
            if warps[w][1] == 0:
                if kind[i] == 0:
                    done_tiles[f[i]] += 1
                warps[w] = None
                finished += 1
        if not progressed:
            return finished


def test_persistent_queue_waits_end():
    """However many warps are resident, every item of the plan finishes: an
    edge item only ever waits for tile items taken before it by warps that
    do not wait."""
    frames = [(24, 16, 1), (9, 13, 2), (32, 20, 3)]
    tw = th = 4
    items = facert.batch_plan(frames, 2, tw, th, 3)
    n_tiles = [-(-w // tw) * -(-h // th) for w, h, _ in frames]
    rng = np.random.default_rng(0)
    for n_warps in (1, 2, 5, 17, 64, 1000):
        assert _simulate_queue(items, n_tiles, n_warps, rng) == len(items), n_warps
    # the model is not vacuous: the same items with one edge item moved ahead
    # of a tile item of its frame stall a single warp
    bad = items.copy()
    first_edge = int(np.argmax(bad[:, 0] & (SEDGE | PEDGE) != 0))
    frame_of = bad[first_edge, 0] & ~(SEDGE | PEDGE)
    tile_pos = int(np.nonzero(bad[:, 0] == frame_of)[0][0])
    bad[[tile_pos, first_edge]] = bad[[first_edge, tile_pos]]
    assert _simulate_queue(bad, n_tiles, 1, rng) < len(bad)
