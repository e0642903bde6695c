"""Closed forms used to pin the oracle (independent of oracle/ and of the CUDA path).

* Lambert's formula for the irradiance from a uniform polygonal emitter:
  E(x, n) = 1/2 * sum_k gamma_k * (n . g_k), where gamma_k is the angle the
  polygon edge k subtends at x and g_k the unit normal of the plane through x
  and that edge (Lambert, Photometria 1760; the form-factor version is in
  Cohen & Wallace, "Radiosity and Realistic Image Synthesis", 1993).
* Sutherland-Hodgman clipping of a polygon against a convex polygon.
* Shoelace area of a polygon, and the exact covered area of a pixel square by
  a triangle (clip, then shoelace).
"""
from __future__ import annotations

import numpy as np

from paper_1910_05200_gb300 import synthetic as S


def lambert_irradiance(x, n, poly):
    """Irradiance at x (unit normal n) from a uniform polygon of unit radiance."""
    x = np.asarray(x, np.float64)
    n = np.asarray(n, np.float64)
    r = [np.asarray(p, np.float64) - x for p in poly]
    r = [v / np.linalg.norm(v) for v in r]
    E = 0.0
    for k in range(len(r)):
        a, b = r[k], r[(k + 1) % len(r)]
        gamma = np.arccos(np.clip(a @ b, -1.0, 1.0))
        c = np.cross(a, b)
        nc = np.linalg.norm(c)
        if nc == 0:
            continue
        E += gamma * (n @ (c / nc))
    return abs(0.5 * E)


def clip_polygon(subject, clipper):
    """Sutherland-Hodgman: subject polygon clipped by a convex counter-clockwise clipper (2D)."""
    out = [np.asarray(p, np.float64) for p in subject]
    m = len(clipper)
    for i in range(m):
        a, b = np.asarray(clipper[i], np.float64), np.asarray(clipper[(i + 1) % m], np.float64)
        inp, out = out, []
        if not inp:
            break

        def inside(p):
            return (b[0] - a[0]) * (p[1] - a[1]) - (b[1] - a[1]) * (p[0] - a[0]) >= 0

        def inter(p, q):
            d1 = (b[0] - a[0]) * (p[1] - a[1]) - (b[1] - a[1]) * (p[0] - a[0])
            d2 = (b[0] - a[0]) * (q[1] - a[1]) - (b[1] - a[1]) * (q[0] - a[0])
            t = d1 / (d1 - d2)
            return p + t * (q - p)

        for k in range(len(inp)):
            p, q = inp[k], inp[(k + 1) % len(inp)]
            if inside(q):
                if not inside(p):
                    out.append(inter(p, q))
                out.append(q)
            elif inside(p):
                out.append(inter(p, q))
    return out


def shoelace(poly):
    if len(poly) < 3:
        return 0.0
    P = np.asarray(poly)
    return 0.5 * float(np.sum(P[:, 0] * np.roll(P[:, 1], -1) - np.roll(P[:, 0], -1) * P[:, 1]))


def ccw(poly2):
    return poly2 if shoelace(poly2) > 0 else poly2[::-1]


def triangle_pixel_area(tri2, px, py):
    """Exact area of (2D triangle) intersected with the unit pixel [px,px+1]x[py,py+1]."""
    sq = [(px, py), (px + 1, py), (px + 1, py + 1), (px, py + 1)]
    return abs(shoelace(clip_polygon(ccw([np.asarray(p) for p in tri2]), sq)))


# ---------------------------------------------------------------------------
# light stage restated (Fibonacci hemisphere) for building test geometry

def light_frame(j, n=20, radius=3.0):
    z = (j + 0.5) / n
    r = np.sqrt(1 - z * z)
    ph = j * np.pi * (3 - np.sqrt(5))
    d = np.array([r * np.cos(ph), r * np.sin(ph), z])
    e1 = np.array([d[2], 0.0, -d[0]])
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(d, e1)
    return radius * d, e1, e2, d


def light_quad(j, side=0.6, n=20, radius=3.0):
    c, e1, e2, d = light_frame(j, n, radius)
    h = side / 2
    return [c - h * e1 - h * e2, c + h * e1 - h * e2, c + h * e1 + h * e2, c - h * e1 + h * e2]


def plain_scene(verts, tris, uv=None):
    """Scene with no morphable bases (K = 0) around explicit geometry."""
    verts = np.asarray(verts, np.float32)
    V = verts.shape[0]
    uv = np.zeros((V, 2), np.float32) if uv is None else np.asarray(uv, np.float32)
    return S.Scene(mean=verts, tris=np.asarray(tris, np.int32), uv=uv,
                   B_id=np.zeros((3 * V, 0), np.float32), B_exp=np.zeros((3 * V, 0), np.float32),
                   alb_mean=np.full(3 * V, np.pi, np.float32), B_alb=np.zeros((3 * V, 0), np.float32))


def plain_theta(lights_on=(), rgb=(1.0, 1.0, 1.0), cspec=0.0):
    o = S.param_offsets(0, 0, 0)
    th = np.zeros(o["total"], np.float32)
    th[o["cspec"]:o["pose"]] = cspec
    for j in lights_on:
        th[o["lights"] + 3 * j:o["lights"] + 3 * j + 3] = rgb
    return th


# ---------------------------------------------------------------------------
# exact union of planar triangles (slab decomposition) for shadows cast by
# many occluder triangles at once

def _seg_cross_x(p, q, r, s):
    """x coordinate where segments pq and rs cross (None if they do not)."""
    d1, d2 = q - p, s - r
    den = d1[0] * d2[1] - d1[1] * d2[0]
    if den == 0.0:
        return None
    w = r - p
    a = (w[0] * d2[1] - w[1] * d2[0]) / den
    b = (w[0] * d1[1] - w[1] * d1[0]) / den
    if 0.0 < a < 1.0 and 0.0 < b < 1.0:
        return p[0] + a * d1[0]
    return None


def triangle_union_pieces(tris2):
    """Disjoint convex pieces (trapezoids, counter-clockwise) whose union is
    the union of the 2D triangles tris2 [k][3][2].  Vertical slabs between
    consecutive event abscissae (vertices and edge crossings) contain no event,
    so in each slab every triangle is bounded by one lower and one upper edge
    line and the union is a set of trapezoids found by merging intervals."""
    T = [np.asarray(t, np.float64) for t in tris2]
    edges = [(t[i], t[(i + 1) % 3]) for t in T for i in range(3)]
    xs = [p[0] for t in T for p in t]
    for i in range(len(edges)):
        for k in range(i + 1, len(edges)):
            x = _seg_cross_x(edges[i][0], edges[i][1], edges[k][0], edges[k][1])
            if x is not None:
                xs.append(x)
    xs = np.unique(np.asarray(xs))
    pieces = []

    def line_at(e, x):
        p, q = e
        return p[1] + (q[1] - p[1]) * (x - p[0]) / (q[0] - p[0])

    for xa, xb in zip(xs[:-1], xs[1:]):
        if not xb > xa:
            continue
        xm = 0.5 * (xa + xb)
        iv = []
        for t in T:
            if not (t[:, 0].min() < xm < t[:, 0].max()):
                continue
            es = [(t[i], t[(i + 1) % 3]) for i in range(3)
                  if min(t[i][0], t[(i + 1) % 3][0]) < xm < max(t[i][0], t[(i + 1) % 3][0])]
            if len(es) != 2:
                continue
            ys = [line_at(e, xm) for e in es]
            lo, hi = (es[0], es[1]) if ys[0] < ys[1] else (es[1], es[0])
            iv.append((min(ys), max(ys), lo, hi))
        iv.sort(key=lambda r: r[0])
        merged, cur = [], None
        for r in iv:
            if cur is None:
                cur = list(r)
            elif r[0] <= cur[1]:
                if r[1] > cur[1]:
                    cur[1], cur[3] = r[1], r[3]
            else:
                merged.append(cur)
                cur = list(r)
        if cur is not None:
            merged.append(cur)
        for _, _, lo, hi in merged:
            pieces.append([np.array([xa, line_at(lo, xa)]), np.array([xb, line_at(lo, xb)]),
                           np.array([xb, line_at(hi, xb)]), np.array([xa, line_at(hi, xa)])])
    return pieces


def lit_irradiance(x_int, n, occluders, j, x_vis=None):
    """Irradiance at x_int (normal n) from unit-radiance light j of the stage
    with the part hidden by the occluder triangles, as seen from x_vis
    (default x_int), removed: E(square) - E(square intersected with the union
    of the occluders' central projections from x_vis), Lambert's formula on
    exact polygons.  Splitting x_vis from x_int separates the visibility
    boundary's dependence on the shading point from that of the integrand."""
    x_int = np.asarray(x_int, np.float64)
    x_vis = x_int if x_vis is None else np.asarray(x_vis, np.float64)
    quad = light_quad(j)
    c, e1, e2, d = light_frame(j)
    D = (c - x_vis) @ d
    to2 = lambda p: np.array([(p - c) @ e1, (p - c) @ e2])
    proj = []
    for tri in occluders:
        tri = [np.asarray(p, np.float64) for p in tri]
        if min((p - x_vis) @ d for p in tri) <= 0:
            continue
        proj.append([to2(x_vis + (p - x_vis) * (D / ((p - x_vis) @ d))) for p in tri])
    q2 = ccw([to2(p) for p in quad])
    E = lambert_irradiance(x_int, n, quad)
    for piece in triangle_union_pieces(proj):
        inter = clip_polygon(ccw(piece), q2)
        if len(inter) >= 3:
            E -= lambert_irradiance(x_int, n, [c + p[0] * e1 + p[1] * e2 for p in inter])
    return E
