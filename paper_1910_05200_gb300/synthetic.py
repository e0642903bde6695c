"""Seeded synthetic scenes for the light-stage face renderer.

This module only draws inputs: meshes, morphable bases, parameter vectors and
targets.  It holds none of the renderer's arithmetic, so both the CUDA path and
the CPU oracle can consume its output without sharing method code.

The paper (Face Modeling paragraph) fits a morphable face model with identity
(80), expression (90) and albedo (80) coefficients, a 32x32 specular map, a
6-dof pose and 20 RGB light intensities.  Neither the morphable model nor real
photographs are available, so scenes are synthetic:

* ``tiny``: a 40x40 latitude/longitude patch of the unit sphere facing +z
  (1,600 vertices, 3,042 triangles), 8 of 20 lights on, 64x64 image, 4 spp.
* ``full``: a disk of concentric rings (35,709 vertices, 70,789 triangles,
  627 boundary vertices) displaced into a face-like height field (dome, nose
  ridge, eye sockets, mouth), 14 of 20 lights on, 256x256 image, 16 spp.

Basis columns are smooth random fields (random Fourier features of the mean
position) whose entries are Gaussian with standard deviation
``scale * exp(-k / 20)`` for column ``k``.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

N_LIGHTS = 20
CSPEC_RES = 32
K_ID, K_EXP, K_ALB = 80, 90, 80


@dataclasses.dataclass
class Scene:
    """A mesh with its morphable bases (all arrays little-endian, C order)."""
    mean: np.ndarray       # [V, 3] float32 mean shape
    tris: np.ndarray       # [F, 3] int32, counter-clockwise seen from outside
    uv: np.ndarray         # [V, 2] float32 in [0, 1]^2 (specular-map coordinates)
    B_id: np.ndarray       # [3V, K_id] float32, row 3v+c = coordinate c of vertex v
    B_exp: np.ndarray      # [3V, K_exp] float32
    alb_mean: np.ndarray   # [3V] float32 RGB albedo mean
    B_alb: np.ndarray      # [3V, K_alb] float32

    @property
    def V(self) -> int:
        return int(self.mean.shape[0])

    @property
    def F(self) -> int:
        return int(self.tris.shape[0])

    @property
    def K(self):
        return (int(self.B_id.shape[1]), int(self.B_exp.shape[1]), int(self.B_alb.shape[1]))

    @property
    def n_params(self) -> int:
        kid, kexp, kalb = self.K
        return kid + kexp + kalb + CSPEC_RES * CSPEC_RES + 6 + 3 * N_LIGHTS


def param_offsets(K_id=K_ID, K_exp=K_EXP, K_alb=K_ALB):
    """Offsets of the packed parameter vector theta.

    Layout: alpha[K_id] | beta[K_exp] | delta[K_alb] | c_spec[32*32] |
    pose[6] = (rx, ry, rz, tx, ty, tz) | lights[20*3].
    """
    o = {}
    o["alpha"] = 0
    o["beta"] = K_id
    o["delta"] = K_id + K_exp
    o["cspec"] = K_id + K_exp + K_alb
    o["pose"] = o["cspec"] + CSPEC_RES * CSPEC_RES
    o["lights"] = o["pose"] + 6
    o["total"] = o["lights"] + 3 * N_LIGHTS
    return o


# ---------------------------------------------------------------------------
# meshes

def tiny_grid_mesh(n: int = 40):
    """n x n latitude/longitude patch of the unit sphere, facing +z."""
    lon = np.linspace(-0.5 * math.pi, 0.5 * math.pi, n)
    lat = np.linspace(-0.45 * math.pi, 0.45 * math.pi, n)
    la, lo = np.meshgrid(lat, lon, indexing="ij")        # row = latitude, col = longitude
    pts = np.stack([np.sin(lo) * np.cos(la), np.sin(la), np.cos(lo) * np.cos(la)], -1)
    mean = pts.reshape(-1, 3)
    uv = np.stack(np.meshgrid(np.arange(n) / (n - 1), np.arange(n) / (n - 1), indexing="xy"), -1)
    uv = uv.reshape(-1, 2)
    tris = []
    for i in range(n - 1):
        for j in range(n - 1):
            a, b, c, d = i * n + j, i * n + j + 1, (i + 1) * n + j + 1, (i + 1) * n + j
            tris.append((a, b, c))
            tris.append((a, c, d))
    tris = np.asarray(tris, np.int64)
    tris = _orient_outward(mean, tris)
    return mean.astype(np.float32), tris.astype(np.int32), uv.astype(np.float32)


def _ring_sizes(n_total: int, n_outer: int):
    """Ring sizes n_1..n_R, growing linearly, summing to n_total, last = n_outer."""
    R = int(round(2.0 * n_total / n_outer - 1))
    sizes = [max(3, int(round(n_outer * r / R))) for r in range(1, R + 1)]
    sizes[-1] = n_outer
    diff = n_total - sum(sizes)
    k = R - 2
    while diff != 0:                       # spread the remainder over inner rings
        step = 1 if diff > 0 else -1
        if sizes[k] + step >= 3 and sizes[k] + step < sizes[k + 1]:
            sizes[k] += step
            diff -= step
        k -= 1
        if k < 0:
            k = R - 2
    return sizes


def full_face_mesh(n_verts: int = 35709, n_boundary: int = 627):
    """Disk of concentric rings displaced into a face-like height field.

    A triangulated disk with V vertices and B boundary vertices has
    F = 2V - B - 2 triangles and E = (3F + B) / 2 edges, so 35,709/627 gives
    70,789 triangles and 106,497 edges.
    """
    sizes = _ring_sizes(n_verts - 1, n_boundary)
    R = len(sizes)
    xy = [np.zeros((1, 2))]
    ang_all = [np.zeros(1)]
    rings = []
    start = 1
    for r, nr in enumerate(sizes, 1):
        off = 0.5 * (r % 2)
        ang = 2 * math.pi * (np.arange(nr) + off) / nr
        rad = r / R
        xy.append(np.stack([rad * np.cos(ang), rad * np.sin(ang)], -1))
        ang_all.append(ang)
        rings.append(np.arange(start, start + nr))
        start += nr
    xy = np.concatenate(xy, 0)
    tris = []
    inner = rings[0]
    for k in range(len(inner)):                       # centre fan
        tris.append((0, inner[k], inner[(k + 1) % len(inner)]))
    for r in range(R - 1):
        a_idx, b_idx = rings[r], rings[r + 1]
        a_ang = (ang_all[r + 1] / (2 * math.pi))
        b_ang = (ang_all[r + 2] / (2 * math.pi))
        na, nb = len(a_idx), len(b_idx)
        i = j = 0
        while i < na or j < nb:
            next_a = a_ang[(i + 1) % na] + (1.0 if i + 1 >= na else 0.0)
            next_b = b_ang[(j + 1) % nb] + (1.0 if j + 1 >= nb else 0.0)
            if j >= nb or (i < na and next_a < next_b):
                tris.append((a_idx[i % na], b_idx[j % nb], a_idx[(i + 1) % na]))
                i += 1
            else:
                tris.append((a_idx[i % na], b_idx[j % nb], b_idx[(j + 1) % nb]))
                j += 1
    tris = np.asarray(tris, np.int64)
    # fix orientation: counter-clockwise in the xy plane (the face looks at +z)
    p = xy[tris]
    area = (p[:, 1, 0] - p[:, 0, 0]) * (p[:, 2, 1] - p[:, 0, 1]) - (p[:, 2, 0] - p[:, 0, 0]) * (p[:, 1, 1] - p[:, 0, 1])
    flip = area < 0
    tris[flip] = tris[flip][:, [0, 2, 1]]
    x = 0.78 * xy[:, 0]
    y = 1.0 * xy[:, 1]
    rho2 = xy[:, 0] ** 2 + xy[:, 1] ** 2
    z = 0.62 * np.sqrt(np.maximum(0.0, 1.0 - 0.85 * rho2))
    z += 0.30 * np.exp(-(x / 0.10) ** 2 - ((y + 0.02) / 0.26) ** 2) * (0.6 + 0.4 * np.clip(0.2 - y, 0, 1))
    for sx in (-1.0, 1.0):
        z -= 0.08 * np.exp(-((x - sx * 0.30) / 0.13) ** 2 - ((y - 0.22) / 0.09) ** 2)
    z -= 0.04 * np.exp(-(x / 0.24) ** 2 - ((y + 0.46) / 0.045) ** 2)
    z += 0.03 * np.exp(-(x / 0.45) ** 2 - ((y - 0.38) / 0.05) ** 2)  # brow ridge
    z -= 0.35
    mean = np.stack([x, y, z], -1)
    mean /= np.max(np.linalg.norm(mean, axis=1))
    uv = (mean[:, :2] - mean[:, :2].min(0)) / (mean[:, :2].max(0) - mean[:, :2].min(0))
    return mean.astype(np.float32), tris.astype(np.int32), uv.astype(np.float32)


def _orient_outward(mean, tris):
    p = mean[tris]
    n = np.cross(p[:, 1] - p[:, 0], p[:, 2] - p[:, 0])
    c = p.mean(1)
    flip = (n * c).sum(1) < 0
    tris = tris.copy()
    tris[flip] = tris[flip][:, [0, 2, 1]]
    return tris


# ---------------------------------------------------------------------------
# bases and parameters

def smooth_basis(mean: np.ndarray, K: int, scale: float, rng: np.random.Generator,
                 n_feat: int = 8, freq: float = 1.0) -> np.ndarray:
    """[3V, K] basis whose column k is a smooth random field with std scale*exp(-k/20)."""
    V = mean.shape[0]
    P = mean.astype(np.float64)
    B = np.empty((3 * V, K), np.float64)
    for k in range(K):
        sig = scale * math.exp(-k / 20.0)
        om = rng.normal(0.0, 2 * math.pi * freq, size=(3, 3 * n_feat))
        ph = rng.uniform(0.0, 2 * math.pi, size=3 * n_feat)
        w = rng.normal(0.0, 1.0, size=3 * n_feat)
        feats = np.cos(P @ om + ph) * w * math.sqrt(2.0 / n_feat)   # [V, 3*n_feat]
        col = feats.reshape(V, 3, n_feat).sum(-1)                    # [V, 3]
        B[:, k] = sig * col.reshape(-1)
    return B.astype(np.float32)


def make_scene(kind: str = "tiny", seed: int = 0, K=(K_ID, K_EXP, K_ALB),
               geo_scale: float = 4e-3, alb_scale: float = 0.02) -> Scene:
    if kind == "tiny":
        mean, tris, uv = tiny_grid_mesh()
    elif kind == "full":
        mean, tris, uv = full_face_mesh()
    else:
        raise ValueError(kind)
    rng = np.random.default_rng(1000 + seed)
    kid, kexp, kalb = K
    B_id = smooth_basis(mean, kid, geo_scale, rng)
    B_exp = smooth_basis(mean, kexp, geo_scale, rng)
    B_alb = smooth_basis(mean, kalb, alb_scale, rng)
    alb_mean = np.tile(np.array([0.6, 0.45, 0.35], np.float32), mean.shape[0])
    return Scene(mean, tris, uv, B_id, B_exp, alb_mean, B_alb)


def make_theta(scene: Scene, seed: int = 0, n_on: int = 8, max_angle_deg: float = 10.0,
               t_std: float = 0.02) -> np.ndarray:
    """alpha, beta, delta ~ N(0,1); c_spec ~ U[0,1]; n_on of 20 lights U[0,2]^3."""
    rng = np.random.default_rng(seed)
    kid, kexp, kalb = scene.K
    o = param_offsets(kid, kexp, kalb)
    th = np.zeros(o["total"], np.float64)
    th[o["alpha"]:o["alpha"] + kid] = rng.normal(size=kid)
    th[o["beta"]:o["beta"] + kexp] = rng.normal(size=kexp)
    th[o["delta"]:o["delta"] + kalb] = rng.normal(size=kalb)
    th[o["cspec"]:o["pose"]] = rng.uniform(0.0, 1.0, CSPEC_RES * CSPEC_RES)
    a = math.radians(max_angle_deg)
    th[o["pose"]:o["pose"] + 3] = rng.uniform(-a, a, 3)
    th[o["pose"] + 3:o["pose"] + 6] = rng.normal(0.0, t_std, 3)
    on = rng.choice(N_LIGHTS, size=n_on, replace=False)
    L = np.zeros((N_LIGHTS, 3))
    L[on] = rng.uniform(0.0, 2.0, (n_on, 3))
    th[o["lights"]:] = L.reshape(-1)
    return th.astype(np.float32)


# Workload presets: (scene kind, W, H, spp, lights on, max pose angle, t std)
CONFIGS = {
    "tiny": dict(kind="tiny", W=64, H=64, spp=4, n_on=8, max_angle_deg=10.0, t_std=0.02),
    "full": dict(kind="full", W=256, H=256, spp=16, n_on=14, max_angle_deg=30.0, t_std=0.05),
}


def make_workload(name: str = "tiny", seed: int = 0):
    c = CONFIGS[name]
    scene = make_scene(c["kind"], seed=0)
    theta = make_theta(scene, seed=seed, n_on=c["n_on"], max_angle_deg=c["max_angle_deg"],
                       t_std=c["t_std"])
    return scene, theta, c


# Batched frames: frames of one face with shared identity, albedo and specular
# map and per-frame expression, pose and lights; square crops of side
# 128 + 8 floor(25 u), u ~ U[0,1) (128 ... 320 in steps of 8).
BATCH = dict(kind="full", n_frames=32, spp=16, n_on=14, max_angle_deg=30.0, t_std=0.05, seed=100,
             side_min=128, side_step=8, side_levels=25)


def batch_sides(n_frames: int, seed: int, side_min: int = 128, side_step: int = 8, levels: int = 25):
    rng = np.random.default_rng(seed)
    return [int(side_min + side_step * math.floor(levels * u)) for u in rng.uniform(size=n_frames)]


def make_batch(scene: Scene, n_frames: int = 32, seed: int = 100, n_on: int = 14, max_angle_deg: float = 30.0,
               t_std: float = 0.05, sizes=None):
    """Frames [(W, H, seed_f)] and full parameter vectors [n_frames, P] (FP32)
    whose alpha, delta and c_spec are the same in every frame.  sizes: list
    of (W, H); default square crops from batch_sides."""
    if sizes is None:
        sizes = [(w, w) for w in batch_sides(n_frames, seed)]
    kid, kexp, kalb = scene.K
    o = param_offsets(kid, kexp, kalb)
    base = make_theta(scene, seed=seed, n_on=n_on, max_angle_deg=max_angle_deg, t_std=t_std)
    thetas = []
    for f in range(len(sizes)):
        th = make_theta(scene, seed=seed * 1000 + 1 + f, n_on=n_on, max_angle_deg=max_angle_deg, t_std=t_std)
        th[o["alpha"]:o["beta"]] = base[o["alpha"]:o["beta"]]
        th[o["delta"]:o["pose"]] = base[o["delta"]:o["pose"]]
        thetas.append(th)
    frames = [(int(w), int(h), seed * 1000 + f) for f, (w, h) in enumerate(sizes)]
    return frames, np.stack(thetas)


def noise_images(frames, seed: int, lo: float = 0.0, hi: float = 0.5) -> np.ndarray:
    """Packed [sum W*H, 3] FP32 images, U[lo, hi] per channel."""
    n = sum(w * h for w, h, _ in frames)
    return np.random.default_rng(seed).uniform(lo, hi, (n, 3)).astype(np.float32)


def random_pixels(W: int, H: int, n: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(W * H, size=min(n, W * H), replace=False)).astype(np.int32)
