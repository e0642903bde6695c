"""The rounding bound behind the shadow-edge search's box classification.

The search drops a leaf edge for a whole warp when both of its face planes
are proven to have one sign over the box of the warp's shading points
(plane_sign_over_box in csrc/render_device.cuh).  The proof: the decision
form dot3r(n, sub3r(x, p)) of a point x (each term rounded at most four times
in FP32) differs from the exact n.(x - p) by at most gamma_4 T with
T = sum_i |n_i| max(|lo_i - p_i|, |hi_i - p_i|); the box's extremes are
evaluated at the corners chosen by the signs of n with the same bound, and a
margin of 1e-6 T (> 2 gamma_4 T) plus 1e-30 separates them from zero.

This test restates the bound in numpy FP32 (IEEE round to nearest; the
device's contraction of the box evaluation into FMAs is emulated too) and
checks it against the decision form itself: wherever the bound claims a
sign, every corner and many random points of the box must give that sign.
Cases include near-grazing planes, where the bound is tight.
"""
import numpy as np
import pytest

F = np.float32


def dot3r(a, b):
    """The decision form: products and sums each rounded to FP32, in order."""
    p = F(a[0]) * F(b[0])
    p = F(p + F(a[1]) * F(b[1]))
    return F(p + F(a[2]) * F(b[2]))


def sub3r(a, b):
    return [F(F(a[k]) - F(b[k])) for k in range(3)]


def fma32(a, b, c):
    # the product of two FP32 values is exact in FP64
    return F(np.float64(a) * np.float64(b) + np.float64(c))


def dot_plain(a, b, contract):
    if not contract:
        return F(F(F(a[0]) * F(b[0]) + F(a[1]) * F(b[1])) + F(a[2]) * F(b[2]))
    return fma32(a[0], b[0], fma32(a[1], b[1], F(F(a[2]) * F(b[2]))))


def plane_sign_over_box(n, p, lo, hi, contract):
    cmin = [lo[k] if n[k] > 0 else hi[k] for k in range(3)]
    cmax = [hi[k] if n[k] > 0 else lo[k] for k in range(3)]
    smin = dot_plain(n, [F(cmin[k] - p[k]) for k in range(3)], contract)
    smax = dot_plain(n, [F(cmax[k] - p[k]) for k in range(3)], contract)
    t = [F(abs(n[k])) * F(max(abs(F(lo[k] - p[k])), abs(F(hi[k] - p[k])))) for k in range(3)]
    T = F(F(t[0] + t[1]) + t[2]) if not contract else fma32(abs(n[0]), max(abs(F(lo[0] - p[0])), abs(F(hi[0] - p[0]))),
                                                             F(t[1] + t[2]))
    m = fma32(F(1e-6), T, F(1e-30)) if contract else F(F(F(1e-6) * T) + F(1e-30))
    return 1 if smin > m else (-1 if smax < -m else 0)


def _cases(rng, n_cases):
    for _ in range(n_cases):
        n = (rng.normal(size=3) * 10.0 ** rng.uniform(-7, 0)).astype(F)
        p = rng.uniform(-0.6, 0.6, size=3).astype(F)
        size = 10.0 ** rng.uniform(-6, -1.5)
        if rng.uniform() < 0.5:
            # a box near the plane through p: its centre 0..20 box sizes off the plane
            u = n.astype(np.float64) / np.linalg.norm(n.astype(np.float64))
            t = rng.normal(size=3)
            t -= t.dot(u) * u
            c = p + t * rng.uniform(0, 0.05) + u * size * rng.uniform(-20, 20)
        else:
            c = p + rng.normal(size=3) * rng.uniform(1e-4, 0.2)
        half = rng.uniform(0.1, 1.0, size=3) * size
        lo = (c - half).astype(F)
        hi = (c + half).astype(F)
        yield n, p, lo, hi


@pytest.mark.parametrize("contract", [False, True])
def test_box_sign_bound_holds_for_the_decision_form(contract):
    rng = np.random.default_rng(12 + contract)
    proven = 0
    for n, p, lo, hi in _cases(rng, 3000):
        sgn = plane_sign_over_box(n, p, lo, hi, contract)
        if sgn == 0:
            continue
        proven += 1
        pts = [np.array([(hi if (c >> k) & 1 else lo)[k] for k in range(3)], F) for c in range(8)]
        pts += list(rng.uniform(lo, hi, size=(64, 3)).astype(F))
        for x in pts:
            s = dot3r(n, sub3r(x, p))
            assert (s > 0 if sgn > 0 else s < 0), (n, p, lo, hi, x, s, sgn)
    assert proven > 1000          # the bound proves most boxes off the plane


@pytest.mark.parametrize("contract", [False, True])
def test_box_sign_bound_adversarial_corners(contract):
    """Boxes whose nearest corner lies within a few rounding units of the
    plane (offsets of 1e-9 .. 1e-5 of the terms' scale): the corner's decision
    form and the box evaluation round differently there, and only the margin
    keeps a claimed sign right."""
    rng = np.random.default_rng(40 + contract)
    proven = 0
    for _ in range(20000):
        n = (rng.normal(size=3) * 10.0 ** rng.uniform(-3, 0)).astype(F)
        p = rng.uniform(-0.6, 0.6, size=3).astype(F)
        nn = n.astype(np.float64)
        u = nn / np.linalg.norm(nn)
        t = rng.normal(size=3)
        t -= t.dot(u) * u
        scale = float(np.abs(nn).sum() * (np.abs(p).max() + 0.1))
        off = rng.choice([-1.0, 1.0]) * 10.0 ** rng.uniform(-9, -5) * scale / np.linalg.norm(nn)
        c = (p + t * rng.uniform(0.001, 0.05) + u * off).astype(F)
        size = 10.0 ** rng.uniform(-6, -3)
        # the box extends away from the plane from the corner c
        away = np.where(nn * np.sign(off) > 0, 1.0, -1.0) * size
        lo = np.minimum(c, c + away).astype(F)
        hi = np.maximum(c, c + away).astype(F)
        sgn = plane_sign_over_box(n, p, lo, hi, contract)
        if sgn == 0:
            continue
        proven += 1
        for k in range(8):
            x = np.array([(hi if (k >> i) & 1 else lo)[i] for i in range(3)], F)
            s = dot3r(n, sub3r(x, p))
            assert (s > 0 if sgn > 0 else s < 0), (n, p, lo, hi, x, s, sgn)
    assert proven > 100


def test_box_sign_bound_is_not_vacuous_near_the_plane():
    """A box straddling the plane is never classified; a box just off it is,
    once the offset exceeds the margin."""
    n = np.array([0.3, -0.5, 0.8], F)
    p = np.array([0.1, 0.2, -0.1], F)
    u = n.astype(np.float64) / np.linalg.norm(n.astype(np.float64))
    h = 1e-3
    straddle = (p - h, p + h)
    assert plane_sign_over_box(n, p, straddle[0].astype(F), straddle[1].astype(F), False) == 0
    off = p + u * 0.01
    box = ((off - h).astype(F), (off + h).astype(F))
    assert plane_sign_over_box(n, p, box[0], box[1], False) == 1
    box = ((p - u * 0.01 - h).astype(F), (p - u * 0.01 + h).astype(F))
    assert plane_sign_over_box(n, p, box[0], box[1], False) == -1
