"""ctypes wrapper and build step for the C++ oracle (test infrastructure only).

The oracle is the FP64 brute-force restatement of the renderer in
``oracle.cpp``; see that file's header for what it computes and which paper
passage each part follows.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD = os.path.join(HERE, "_build")
ORACLE_SO = os.path.join(BUILD, "liboracle.so")
SRC = os.path.join(HERE, "oracle.cpp")


def build_oracle(force: bool = False) -> str:
    """Compile oracle.cpp with g++ (no fused multiply-add, IEEE semantics)."""
    os.makedirs(BUILD, exist_ok=True)
    if (not force and os.path.exists(ORACLE_SO)
            and os.path.getmtime(ORACLE_SO) >= os.path.getmtime(SRC)):
        return ORACLE_SO
    tmp = ORACLE_SO + f".tmp{os.getpid()}"
    cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-pthread", SRC, "-o", tmp]
    subprocess.check_call(cmd)
    os.replace(tmp, ORACLE_SO)
    return ORACLE_SO


class OracleConfig(C.Structure):
    _fields_ = [("W", C.c_int32), ("H", C.c_int32), ("spp", C.c_int32),
                ("seed", C.c_uint32), ("iter", C.c_uint32),
                ("tan_half_fov", C.c_float), ("d_cam", C.c_float),
                ("light_radius", C.c_float), ("light_side", C.c_float),
                ("beckmann_m", C.c_float), ("eps_pedge", C.c_float),
                ("eps_sedge", C.c_float), ("shadow_tmin", C.c_float),
                ("clip_kappa", C.c_float),
                ("n_lights", C.c_int32), ("shade_mode", C.c_int32),
                ("n_threads", C.c_int32), ("terms", C.c_int32), ("value_mesh", C.c_int32),
                ("brdf_model", C.c_int32), ("fresnel", C.c_int32), ("light_layout", C.c_int32),
                ("light_prior", C.c_int32)]


class OracleScene(C.Structure):
    _fields_ = [("V", C.c_int32), ("F", C.c_int32), ("K_id", C.c_int32),
                ("K_exp", C.c_int32), ("K_alb", C.c_int32),
                ("mean", C.c_void_p), ("tris", C.c_void_p), ("uv", C.c_void_p),
                ("B_id", C.c_void_p), ("B_exp", C.c_void_p),
                ("alb_mean", C.c_void_p), ("B_alb", C.c_void_p)]


# Scene constants (one reading of what the paper leaves open).
DEFAULTS = dict(tan_half_fov=0.275, d_cam=4.0, light_radius=3.0, light_side=0.6,
                beckmann_m=0.3, eps_pedge=1e-3, eps_sedge=2e-4, shadow_tmin=1e-4,
                clip_kappa=1e-5, n_lights=20, brdf_model=0, fresnel=0, light_layout=0,
                light_prior=0)


def default_config(W=64, H=64, spp=4, seed=0, iter=0, shade_mode=0, n_threads=0, terms=0,
                   value_mesh=1, **kw) -> OracleConfig:
    """value_mesh = 1 (default) evaluates the estimator on the posed mesh rounded
    to FP32, the mesh the renderer consumes; 0 keeps the FP64 posed mesh (used by
    finite-difference pins, where rounding steps would swamp small differences)."""
    d = dict(DEFAULTS)
    d.update(kw)
    return OracleConfig(W=W, H=H, spp=spp, seed=seed, iter=iter, shade_mode=shade_mode,
                        n_threads=n_threads, terms=terms, value_mesh=value_mesh, **d)


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p)


class Oracle:
    """Thin ctypes front end.  Arrays are converted to the C types it expects."""

    def __init__(self, so_path: str | None = None):
        self.lib = C.CDLL(so_path or os.environ.get("FACERT_ORACLE_SO") or build_oracle())
        L = self.lib
        vp = C.c_void_p
        L.oracle_philox.argtypes = [C.c_uint32] * 6 + [vp]
        L.oracle_n_edges.argtypes = [vp, vp, vp, vp]
        L.oracle_light_stage.argtypes = [C.c_int32, C.c_float, C.c_int32, vp]
        L.oracle_geometry.argtypes = [vp, vp, vp, vp, vp, vp, vp]
        L.oracle_render.argtypes = [vp, vp, vp, vp, C.c_int32, vp, vp, vp]
        L.oracle_render_backward.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, vp]
        L.oracle_loss.argtypes = [vp, vp, vp, vp, vp, vp, vp, C.c_float, C.c_float, vp, vp]
        L.oracle_loss.restype = C.c_double
        L.oracle_light_estimate.argtypes = [vp, vp, vp, vp, vp, C.c_double, vp, C.c_int32,
                                            C.c_float, C.c_float, vp]
        L.oracle_brdf.argtypes = [vp, vp, vp, vp, C.c_double, C.c_double, vp]
        L.oracle_point_shade.argtypes = [vp, vp, vp, vp, vp, C.c_int32, C.c_float, C.c_float, vp, vp]
        L.oracle_shadow_edge_point.argtypes = [vp, vp, vp, vp, vp, C.c_int32, vp, C.c_int32, vp]

    # -- helpers ---------------------------------------------------------------
    @staticmethod
    def _scene(scene):
        keep = dict(
            mean=np.ascontiguousarray(scene.mean, np.float32),
            tris=np.ascontiguousarray(scene.tris, np.int32),
            uv=np.ascontiguousarray(scene.uv, np.float32),
            B_id=np.ascontiguousarray(scene.B_id, np.float32),
            B_exp=np.ascontiguousarray(scene.B_exp, np.float32),
            alb_mean=np.ascontiguousarray(scene.alb_mean, np.float32),
            B_alb=np.ascontiguousarray(scene.B_alb, np.float32))
        s = OracleScene(V=keep["mean"].shape[0], F=keep["tris"].shape[0],
                        K_id=keep["B_id"].shape[1], K_exp=keep["B_exp"].shape[1],
                        K_alb=keep["B_alb"].shape[1],
                        **{k: _ptr(v) for k, v in keep.items()})
        s._keep = keep
        return s

    def philox(self, key, ctr):
        out = np.zeros(4, np.uint32)
        self.lib.oracle_philox(*[int(k) for k in key], *[int(c) for c in ctr], _ptr(out))
        return out

    def edges(self, cfg, scene):
        s = self._scene(scene)
        th = np.zeros(1, np.float32)
        n = self.lib.oracle_n_edges(C.byref(cfg), C.byref(s), _ptr(th), None)
        out = np.zeros((n, 4), np.int32)
        self.lib.oracle_n_edges(C.byref(cfg), C.byref(s), _ptr(th), _ptr(out))
        return out

    def light_stage(self, n=20, radius=3.0, layout=0):
        """[n, 12]: centre, e1, e2, unit direction of each light (layout 0
        Fibonacci, 1 icosphere, n = 20 only)."""
        out = np.zeros((n, 12), np.float32)
        self.lib.oracle_light_stage(n, radius, layout, _ptr(out))
        return out

    def geometry(self, cfg, scene, theta):
        s = self._scene(scene)
        th = np.ascontiguousarray(theta, np.float32)
        V = s.V
        X = np.zeros((V, 3)); X32 = np.zeros((V, 3), np.float32)
        A = np.zeros((V, 3)); N = np.zeros((V, 3))
        n_sil = self.lib.oracle_geometry(C.byref(cfg), C.byref(s), _ptr(th), _ptr(X), _ptr(X32),
                                         _ptr(A), _ptr(N))
        if n_sil < 0:
            raise RuntimeError(f"oracle_geometry failed: {n_sil}")
        return dict(X=X, X32=X32, albedo=A, normals=N, n_silhouette=n_sil)

    def render(self, cfg, scene, theta, pixels=None, signature=False, aov=False):
        """Image [H, W, 3] (or [n_pix, 3]); optionally the decision signature and
        the 14 denoiser features per pixel."""
        s = self._scene(scene)
        th = np.ascontiguousarray(theta, np.float32)
        if pixels is None:
            img = np.zeros((cfg.H, cfg.W, 3))
            pp, n = None, 0
        else:
            pixels = np.ascontiguousarray(pixels, np.int32)
            img = np.zeros((len(pixels), 3))
            pp, n = _ptr(pixels), len(pixels)
        sig = np.zeros(1, np.uint64)
        feats = np.zeros(img.shape[:-1] + (14,)) if aov else None
        rc = self.lib.oracle_render(C.byref(cfg), C.byref(s), _ptr(th), pp, n, _ptr(img), _ptr(sig),
                                    None if feats is None else _ptr(feats))
        if rc:
            raise RuntimeError(f"oracle_render failed: {rc}")
        out = [img]
        if signature:
            out.append(int(sig[0]))
        if aov:
            out.append(feats)
        return out[0] if len(out) == 1 else tuple(out)

    def render_backward(self, cfg, scene, theta, d_image, terms=False, dX=False, mass=False):
        """Gradient [P]; optionally the per-term parts [3, P], the per-vertex
        position gradient [V, 3], the L1 mass [P] of each component and (with
        dX and mass) the L1 mass [V, 3] of the per-vertex gradient."""
        s = self._scene(scene)
        th = np.ascontiguousarray(theta, np.float32)
        dI = np.ascontiguousarray(d_image, np.float64).reshape(cfg.H, cfg.W, 3)
        P = th.shape[0]
        g = np.zeros(P)
        gt = np.zeros((3, P))
        dXo = np.zeros((s.V, 3))
        gm = np.zeros(P)
        dXm = np.zeros((s.V, 3))
        rc = self.lib.oracle_render_backward(C.byref(cfg), C.byref(s), _ptr(th), _ptr(dI), _ptr(g),
                                             _ptr(gt), _ptr(dXo), _ptr(gm), _ptr(dXm))
        if rc:
            raise RuntimeError(f"oracle_render_backward failed: {rc}")
        out = [g]
        if terms:
            out.append(gt)
        if dX:
            out.append(dXo)
        if mass:
            out.append(gm)
            if dX:
                out.append(dXm)
        return out[0] if len(out) == 1 else tuple(out)

    def loss(self, cfg, scene, theta, image, target, mask=None, m=None, w1=0.0, w2=0.0):
        s = self._scene(scene)
        th = np.ascontiguousarray(theta, np.float32)
        img = np.ascontiguousarray(image, np.float32)
        tgt = np.ascontiguousarray(target, np.float32)
        mk = None if mask is None else np.ascontiguousarray(mask, np.uint8)
        mm = None if m is None else np.ascontiguousarray(m, np.float32)
        dI = np.zeros((cfg.H, cfg.W, 3))
        gr = np.zeros(th.shape[0])
        val = self.lib.oracle_loss(C.byref(cfg), C.byref(s), _ptr(th), _ptr(img), _ptr(tgt),
                                   None if mk is None else _ptr(mk), None if mm is None else _ptr(mm),
                                   w1, w2, _ptr(dI), _ptr(gr))
        return val, dI, gr

    def light_estimate(self, cfg, x, ns, wo, rho, cs, lrgb, j, u2, u3):
        a = [np.ascontiguousarray(v, np.float64) for v in (x, ns, wo, rho)]
        l = np.ascontiguousarray(lrgb, np.float32)
        out = np.zeros(3)
        self.lib.oracle_light_estimate(C.byref(cfg), *[_ptr(v) for v in a], float(cs), _ptr(l), int(j),
                                       float(u2), float(u3), _ptr(out))
        return out

    def brdf(self, cfg, n, wi, wo, rho, cs):
        a = [np.ascontiguousarray(v, np.float64) for v in (n, wi, wo)]
        out = np.zeros(1)
        self.lib.oracle_brdf(C.byref(cfg), *[_ptr(v) for v in a], float(rho), float(cs), _ptr(out))
        return float(out[0])

    def point_shade(self, cfg, scene, theta, o, d, j, u2, u3):
        s = self._scene(scene)
        th = np.ascontiguousarray(theta, np.float32)
        o = np.ascontiguousarray(o, np.float32); d = np.ascontiguousarray(d, np.float32)
        out = np.zeros(3)
        hf = np.zeros(1, np.int32)
        rc = self.lib.oracle_point_shade(C.byref(cfg), C.byref(s), _ptr(th), _ptr(o), _ptr(d), int(j),
                                         float(u2), float(u3), _ptr(out), _ptr(hf))
        if rc:
            raise RuntimeError(rc)
        return out, int(hf[0])

    def shadow_edge_point(self, cfg, scene, theta, o, d, j, wrgb, n_rep):
        s = self._scene(scene)
        th = np.ascontiguousarray(theta, np.float32)
        o = np.ascontiguousarray(o, np.float32); d = np.ascontiguousarray(d, np.float32)
        w = np.ascontiguousarray(wrgb, np.float64)
        dX = np.zeros((s.V, 3))
        rc = self.lib.oracle_shadow_edge_point(C.byref(cfg), C.byref(s), _ptr(th), _ptr(o), _ptr(d), int(j),
                                               _ptr(w), int(n_rep), _ptr(dX))
        if rc:
            raise RuntimeError(rc)
        return dX
