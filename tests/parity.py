"""Parity checks of the CUDA path against the FP64 oracle, with a record of
every error they measure.

Tolerances (the target accuracy of the method, written here):

* image: |g - o| <= 1e-4 * max(|o|, 1e-4 * mean|o|) per pixel and channel;
  at most 0.01 % of pixels may differ by a flipped discrete decision.
* gradient: |g - o| <= 1e-3 * max(|o|, 1e-3 * max|o| over the parameter
  group), per component ("strict").
* named exceptions: a test may name, per parameter group, components (or
  a rule that names them: every component whose oracle L1 mass exceeds its
  value by a cancellation ratio of at least `cancel`) that are judged
  against kappa * mass instead, mass being the oracle's L1 mass of the
  component (sum of absolute contributions, an edge sample counted by both
  of its sides, propagated with absolute Jacobians).  Only the alternative
  reflectance readings use this, with kappa = 1e-5: their FP32 lobes carry a
  systematic relative bias of about 2e-7 (the FP32 roughness a^2 = m^2 and
  pi; measured by FP32 emulation against FP64), which sums with a
  cancellation ratio of 3e2 to 1e5 amplify beyond 1e-3 relative.  The strict
  error of every such component is still recorded.

Every check appends a row to RECORD: the result, its strict maximum and
99.99th percentile error, and the components that passed only through a
named exception.  With FACERT_PARITY_LOG set, tests/conftest.py writes the
rows to that file (JSON lines) when the session ends.
"""
from __future__ import annotations

import os

import numpy as np

KAPPA = 1e-4
RECORD: list[dict] = []

# FACERT_PARITY_MODE=record measures without asserting (a record of the
# errors of every result); the default asserts.
ASSERT = os.environ.get("FACERT_PARITY_MODE", "assert") != "record"


def _pct(a, q):
    a = np.asarray(a, np.float64).ravel()
    return float(np.quantile(a, q)) if a.size else 0.0


def image_errors(got, ref):
    scale = np.maximum(np.abs(ref), 1e-4 * np.abs(ref).mean() + 1e-30)
    rel = np.abs(np.asarray(got, np.float64) - ref) / scale
    bad_px = np.any(rel > 1e-4, axis=-1)
    return rel, bad_px


def assert_image(got, ref, what=""):
    rel, bad = image_errors(got, ref)
    n = bad.size
    allowed = int(1e-4 * n)
    RECORD.append(dict(kind="image", what=what, n=int(n), max=float(rel.max()) if rel.size else 0.0,
                       p9999=_pct(rel, 0.9999), flipped=int(bad.sum()), allowed=allowed))
    if ASSERT:
        assert bad.sum() <= allowed, f"{what}: {bad.sum()} of {n} pixels off (max rel {rel.max():.3e}, " \
                                     f"allowed {allowed})"


def check_groups(got, ref, groups, mass=None, named=None, what="", floor_rel=1e-3, cancel=None, kappa=KAPPA):
    """Strict per-component check over the parameter groups {name: slice}.

    named: {group: index array (relative to the group)} of the components
    judged against kappa * mass instead (needs mass); cancel: also name every
    component with mass >= cancel * |oracle value|."""
    named = dict(named or {})
    if cancel is not None:
        assert mass is not None, "a cancellation rule needs the oracle's mass"
        for name, sl in groups.items():
            o = np.abs(np.asarray(ref[sl], np.float64))
            hit = np.nonzero(np.asarray(mass[sl], np.float64) >= cancel * o)[0]
            named[name] = np.union1d(np.asarray(named.get(name, []), np.int64), hit)
    rows = []
    for name, sl in groups.items():
        o, g = np.asarray(ref[sl], np.float64), np.asarray(got[sl], np.float64)
        floor = floor_rel * np.abs(o).max()
        if floor == 0:
            row = dict(kind="grad", what=what, group=name, n=int(o.size), max=float(np.abs(g).max()),
                       p9999=float(np.abs(g).max()), zero=True, mass_only=[])
            RECORD.append(row)
            rows.append(row)
            if ASSERT:
                assert np.all(np.abs(g) <= 1e-9), (what, name, np.abs(g).max())
            continue
        strict = np.abs(g - o) / (1e-3 * np.maximum(np.abs(o), floor))
        ok = strict <= 1.0
        allowed = np.zeros(o.size, bool)
        idx = named.get(name)
        if idx is not None and len(idx):
            assert mass is not None, "named exceptions need the oracle's mass"
            ms = np.asarray(mass[sl], np.float64)
            allowed[np.asarray(idx)] = True
            ok = ok | (allowed & (np.abs(g - o) <= kappa * ms))
        mass_only = [int(i) for i in np.nonzero(ok & ~(strict <= 1.0))[0]]
        row = dict(kind="grad", what=what, group=name, n=int(o.size), max=float(strict.max()) * 1e-3,
                   p9999=_pct(strict, 0.9999) * 1e-3, zero=False, mass_only=mass_only,
                   n_named=int(allowed.sum()), kappa=kappa if allowed.any() else None)
        if mass is not None:
            ms = np.asarray(mass[sl], np.float64)
            row["cancel_max"] = float((ms / np.maximum(np.abs(o), 1e-300)).max())
            bad = np.nonzero(~(strict <= 1.0))[0]
            row["fail_strict"] = [dict(i=int(i), got=float(g[i]), ref=float(o[i]), mass=float(ms[i]),
                                       strict=float(strict[i]) * 1e-3) for i in bad[:12]]
        RECORD.append(row)
        rows.append(row)
        if ASSERT and not ok.all():
            i = int(np.argmax(np.where(ok, 0.0, strict)))
            raise AssertionError(f"{what} {name}: strict error {strict[i] * 1e-3:.3e} at {i} "
                                 f"(got {g[i]:.6e}, oracle {o[i]:.6e}, group max {np.abs(o).max():.3e})")
    return rows


def check_close(got, ref, groups, what="", rel=1e-3, grp=1e-4):
    """Two results of the same library that differ only in the order of FP32
    atomic additions: grp of the group's largest plus rel of the entry."""
    for name, sl in groups.items():
        o, g = np.asarray(ref[sl], np.float64), np.asarray(got[sl], np.float64)
        tol = grp * np.abs(o).max() + rel * np.abs(o) + 1e-12
        err = np.abs(g - o) / tol
        RECORD.append(dict(kind="same-library", what=what, group=name, n=int(o.size),
                           max=float((np.abs(g - o) / np.maximum(np.abs(o), 1e-300)).max()),
                           p9999=0.0, tol_frac=float(err.max())))
        if ASSERT:
            assert err.max() <= 1.0, f"{what} {name}: {err.max():.3e} x tolerance at {int(err.argmax())}"


def record_value(what, got, ref, tol):
    """A scalar (or small array) result compared with its oracle value."""
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    e = np.abs(got - ref) / np.maximum(np.abs(ref), 1e-300)
    RECORD.append(dict(kind="value", what=what, n=int(e.size), max=float(e.max()), p9999=_pct(e, 0.9999),
                       tol=tol))
    if ASSERT:
        assert e.max() <= tol, f"{what}: relative error {e.max():.3e} > {tol:.1e}"


def face_pixels(oracle, cfg, scene, theta, n, seed):
    """n distinct pixel indices covered by the face: projections of posed
    vertices (the oracle's FP64 geometry) that face the camera, through the
    pinhole camera of the configuration.  Chosen from oracle values only."""
    geo = oracle.geometry(cfg, scene, theta)
    X, N = geo["X"], geo["normals"]
    d = float(cfg.d_cam)
    tan = float(cfg.tan_half_fov)
    W, H = int(cfg.W), int(cfg.H)
    k, cx, cy = 2.0 * tan / H, tan * W / H, tan
    q = d - X[:, 2]
    sx = (X[:, 0] / q + cx) / k
    sy = (cy - X[:, 1] / q) / k
    facing = np.einsum("ij,ij->i", N, np.stack([-X[:, 0], -X[:, 1], d - X[:, 2]], 1)) > 0
    inside = facing & (sx >= 0) & (sx < W) & (sy >= 0) & (sy < H)
    pix = np.unique(np.floor(sy[inside]).astype(np.int64) * W + np.floor(sx[inside]).astype(np.int64))
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(pix, size=min(n, pix.size), replace=False)).astype(np.int32)


def loss_bound(ref_img, target, mask=None, rel=1e-4):
    """Bound on |E_data(g) - E_data(o)| when every image value g is within
    rel * max(|o|, rel * mean|o|) of the oracle's o (the image tolerance)."""
    o = np.asarray(ref_img, np.float64)
    t = np.asarray(target, np.float64)
    m = 1.0 if mask is None else np.asarray(mask, np.float64)[..., None]
    e = rel * np.maximum(np.abs(o), rel * np.abs(o).mean())
    return float(np.sum(m * (2.0 * np.abs(o - t) * e + e * e)))


def note(what, err, tol, n=1, p9999=None):
    """Record an error the calling test measured and asserts itself."""
    RECORD.append(dict(kind="value", what=what, n=int(n), max=float(err),
                       p9999=float(err if p9999 is None else p9999), tol=float(tol)))


def check_same_values(got, ref, what="", rel=1e-6):
    """Two results of the same library whose decisions are identical and
    whose values differ only by FP32 rounding (the same formulas compiled in
    two kernels may contract multiply-adds differently): |g - r| <= rel *
    max(|r|, 1e-3 max|r|)."""
    g, r = np.asarray(got, np.float64), np.asarray(ref, np.float64)
    scale = np.maximum(np.abs(r), 1e-3 * np.abs(r).max() + 1e-30)
    e = np.abs(g - r) / scale
    RECORD.append(dict(kind="same-library", what=what, group="values", n=int(e.size),
                       max=float(e.max()) if e.size else 0.0, p9999=_pct(e, 0.9999), tol_frac=float(e.max() / rel)
                       if e.size else 0.0))
    if ASSERT:
        assert e.size == 0 or e.max() <= rel, f"{what}: values differ by {e.max():.3e} (relative) > {rel:.1e}"
