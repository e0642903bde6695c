"""Python binding of libfacert (include/facert.h): argument marshalling only.

Every step of the render and its gradient runs in the library's CUDA kernels;
PyTorch supplies device memory and the stream.  There is no CPU fallback: if
the compiled library is missing, loading fails with an error.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np
import torch

from . import build as _build

_LIB = None

FR_ERRORS = {-1: "invalid argument", -2: "inconsistent shapes", -3: "CUDA error", -4: "out of device memory",
             -5: "device traversal limit reached", -6: "mesh or bases not uploaded"}


class FrConfig(C.Structure):
    _fields_ = [("tan_half_fov", C.c_float), ("d_cam", C.c_float), ("light_radius", C.c_float),
                ("light_side", C.c_float), ("beckmann_m", C.c_float), ("eps_pedge", C.c_float),
                ("eps_sedge", C.c_float), ("shadow_tmin", C.c_float), ("clip_kappa", C.c_float),
                ("n_lights", C.c_int32), ("brdf_model", C.c_int32), ("fresnel", C.c_int32),
                ("light_layout", C.c_int32), ("light_prior", C.c_int32)]


class FrRenderOpts(C.Structure):
    _fields_ = [("W", C.c_int32), ("H", C.c_int32), ("spp", C.c_int32), ("seed", C.c_uint32),
                ("iter", C.c_uint32), ("terms", C.c_int32)]


class FrFrame(C.Structure):
    _fields_ = [("W", C.c_int32), ("H", C.c_int32), ("seed", C.c_uint32)]


class FrTileConfig(C.Structure):
    _fields_ = [("tile_w", C.c_int32), ("tile_h", C.c_int32), ("block", C.c_int32), ("min_blocks", C.c_int32),
                ("fused", C.c_int32), ("ms", C.c_float)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


EXPORTS = ["fr_default_config", "fr_create", "fr_destroy", "fr_set_stream", "fr_last_error", "fr_strerror",
           "fr_upload_mesh", "fr_upload_bases", "fr_n_params", "fr_render", "fr_render_backward", "fr_loss", "fr_step",
           "fr_geometry", "fr_geometry_noalloc", "fr_vertex_grad", "fr_light_stage", "fr_sync", "fr_set_counters", "fr_get_counters", "fr_set_timing", "fr_get_timings",
           "fr_launch_count", "fr_denoiser_n_weights", "fr_denoiser_set_weights", "fr_denoiser_get_weights",
           "fr_denoise", "fr_denoiser_train_step", "fr_denoiser_get_grad", "fr_adam_step",
           "fr_batch_n_shared", "fr_batch_n_frame", "fr_batch_create", "fr_batch_destroy", "fr_batch_set_targets",
           "fr_batch_step", "fr_batch_autotune", "fr_batch_get_config", "fr_batch_set_config", "fr_batch_plan",
           "fr_probe_peaks",
           "fr_set_limits", "fr_silhouettes"]


def probe_peaks(device: int = 0) -> dict:
    """Measured FP32 FMA throughput (TFLOP/s), L2 read bandwidth (GB/s) and SM
    count of the device (fr_probe_peaks)."""
    L = load()
    f = C.c_double(0.0)
    l2 = C.c_double(0.0)
    n = C.c_int32(0)
    rc = L.fr_probe_peaks(int(device), C.byref(f), C.byref(l2), C.byref(n))
    if rc:
        raise RuntimeError(f"fr_probe_peaks: {FR_ERRORS.get(rc, rc)}")
    return {"fp32_tflops": f.value, "l2_read_gbs": l2.value, "sm_count": n.value}


def lib_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Load libfacert.so (built by build.build()); raises if it is missing."""
    global _LIB
    if _LIB is not None:
        return _LIB
    p = path or lib_path()
    if not os.path.exists(p):
        raise RuntimeError(f"libfacert.so not found at {p}: run __graft_entry__.build() first")
    L = C.CDLL(p)
    vp, i32, f32 = C.c_void_p, C.c_int32, C.c_float
    L.fr_default_config.argtypes = [vp]
    L.fr_default_config.restype = None
    L.fr_create.argtypes = [C.POINTER(vp), vp, i32]
    L.fr_destroy.argtypes = [vp]
    L.fr_destroy.restype = None
    L.fr_set_stream.argtypes = [vp, vp]
    L.fr_last_error.argtypes = [vp]
    L.fr_last_error.restype = C.c_char_p
    L.fr_strerror.argtypes = [i32]
    L.fr_strerror.restype = C.c_char_p
    L.fr_upload_mesh.argtypes = [vp, vp, i32, vp, i32, vp]
    L.fr_upload_bases.argtypes = [vp, vp, i32, vp, i32, vp, vp, i32]
    L.fr_n_params.argtypes = [vp]
    L.fr_render.argtypes = [vp, vp, vp, vp, vp]
    L.fr_render_backward.argtypes = [vp, vp, vp, vp, vp, i32]
    L.fr_loss.argtypes = [vp, vp, i32, i32, vp, vp, vp, vp, f32, f32, vp, vp, vp]
    L.fr_step.argtypes = [vp, vp, vp, vp, vp, vp, f32, f32, vp, vp, vp, vp]
    L.fr_geometry.argtypes = [vp, vp, vp, vp, vp]
    L.fr_geometry_noalloc.argtypes = [vp, vp, vp, vp, vp]
    L.fr_light_stage.argtypes = [vp, vp]
    L.fr_vertex_grad.argtypes = [vp, vp]
    L.fr_sync.argtypes = [vp]
    L.fr_set_counters.argtypes = [vp, i32]
    L.fr_get_counters.argtypes = [vp, vp]
    L.fr_set_timing.argtypes = [vp, i32]
    L.fr_get_timings.argtypes = [vp, vp]
    L.fr_launch_count.argtypes = [vp]
    L.fr_launch_count.restype = C.c_uint64
    L.fr_probe_peaks.argtypes = [i32, vp, vp, vp]
    L.fr_set_limits.argtypes = [vp, i32, i32]
    L.fr_silhouettes.argtypes = [vp, vp, i32]
    L.fr_denoiser_n_weights.argtypes = []
    L.fr_denoiser_set_weights.argtypes = [vp, vp, i32]
    L.fr_denoiser_get_weights.argtypes = [vp, vp, i32]
    L.fr_denoise.argtypes = [vp, vp, i32, vp, vp, vp]
    L.fr_denoiser_train_step.argtypes = [vp, vp, vp, i32, f32, vp]
    L.fr_denoiser_get_grad.argtypes = [vp, vp, i32]
    L.fr_adam_step.argtypes = [vp, vp, vp, vp, vp, vp, i32]
    L.fr_batch_n_shared.argtypes = [vp]
    L.fr_batch_n_frame.argtypes = [vp]
    L.fr_batch_create.argtypes = [vp, vp, i32, i32, C.POINTER(vp)]
    L.fr_batch_destroy.argtypes = [vp]
    L.fr_batch_destroy.restype = None
    L.fr_batch_set_targets.argtypes = [vp, vp, vp, vp]
    L.fr_batch_step.argtypes = [vp, vp, vp, f32, f32, C.c_uint32, vp, vp, vp, vp]
    L.fr_batch_autotune.argtypes = [vp, vp, vp, i32, vp, i32, C.POINTER(i32)]
    L.fr_batch_get_config.argtypes = [vp, vp]
    L.fr_batch_set_config.argtypes = [vp, vp]
    L.fr_batch_plan.argtypes = [vp, i32, i32, i32, i32, i32, vp, C.c_int64, C.POINTER(C.c_int64)]
    _LIB = L
    return L


def default_config(**kw) -> FrConfig:
    c = FrConfig()
    load().fr_default_config(C.byref(c))
    for k, v in kw.items():
        setattr(c, k, v)
    return c


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _hptr(a):
    return a.ctypes.data_as(C.c_void_p)


class Renderer:
    """One library context on one CUDA device."""

    def __init__(self, scene=None, device: int = 0, config: FrConfig | None = None):
        self.lib = load()
        self.device = torch.device("cuda", device)
        self.cfg = config or default_config()
        h = C.c_void_p()
        rc = self.lib.fr_create(C.byref(h), C.byref(self.cfg), device)
        if rc:
            raise RuntimeError(f"fr_create failed: {FR_ERRORS.get(rc, rc)}")
        self.ctx = h
        self.P = 0
        if scene is not None:
            self.upload(scene)

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.fr_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, what):
        if rc < 0:
            msg = self.lib.fr_last_error(self.ctx).decode()
            raise RuntimeError(f"{what} failed ({FR_ERRORS.get(rc, rc)}): {msg}")
        return rc

    def _stream(self):
        s = torch.cuda.current_stream(self.device).cuda_stream
        self.lib.fr_set_stream(self.ctx, C.c_void_p(s))

    def upload(self, scene):
        mean = np.ascontiguousarray(scene.mean, np.float32)
        tris = np.ascontiguousarray(scene.tris, np.int32)
        uv = np.ascontiguousarray(scene.uv, np.float32)
        self._stream()
        self._check(self.lib.fr_upload_mesh(self.ctx, _hptr(mean), mean.shape[0], _hptr(tris), tris.shape[0],
                                            _hptr(uv)), "fr_upload_mesh")
        B = [np.ascontiguousarray(b, np.float32) for b in (scene.B_id, scene.B_exp, scene.alb_mean, scene.B_alb)]
        self._check(self.lib.fr_upload_bases(self.ctx, _hptr(B[0]), B[0].shape[1], _hptr(B[1]), B[1].shape[1],
                                             _hptr(B[2]), _hptr(B[3]), B[3].shape[1]), "fr_upload_bases")
        self.P = self.lib.fr_n_params(self.ctx)
        self.V = mean.shape[0]

    @staticmethod
    def opts(W, H, spp, seed=0, iter=0, terms=0) -> FrRenderOpts:
        return FrRenderOpts(W=W, H=H, spp=spp, seed=seed, iter=iter, terms=terms)

    def _theta(self, theta):
        assert theta.device == self.device and theta.dtype == torch.float32 and theta.is_contiguous()
        assert theta.numel() == self.P, (theta.numel(), self.P)
        return theta

    def render(self, theta, W, H, spp, seed=0, iter=0, out=None, aov=None):
        """Render; with aov (an [H, W, 14] float32 tensor, or True to allocate
        one) also writes the per-pixel denoiser features and returns (image, aov)."""
        theta = self._theta(theta)
        img = out if out is not None else torch.empty((H, W, 3), device=self.device, dtype=torch.float32)
        if aov is True:
            aov = torch.empty((H, W, 14), device=self.device, dtype=torch.float32)
        o = self.opts(W, H, spp, seed, iter)
        self._stream()
        self._check(self.lib.fr_render(self.ctx, _ptr(theta), C.byref(o), _ptr(img), _ptr(aov)), "fr_render")
        return img if aov is None else (img, aov)

    def backward(self, theta, d_image, W, H, spp, seed=0, iter=0, terms=0, grad=None, accumulate=False):
        theta = self._theta(theta)
        d_image = d_image.contiguous()
        assert d_image.dtype == torch.float32 and d_image.numel() == W * H * 3
        g = grad if grad is not None else torch.empty(self.P, device=self.device, dtype=torch.float64)
        o = self.opts(W, H, spp, seed, iter, terms)
        self._stream()
        self._check(self.lib.fr_render_backward(self.ctx, _ptr(theta), C.byref(o), _ptr(d_image), _ptr(g),
                                                1 if accumulate else 0), "fr_render_backward")
        return g

    def loss(self, theta, image, target, mask=None, m=None, w1=0.0, w2=0.0, d_image=None, grad=None):
        theta = self._theta(theta)
        H, W = image.shape[0], image.shape[1]
        loss = torch.empty(1, device=self.device, dtype=torch.float64)
        self._stream()
        self._check(self.lib.fr_loss(self.ctx, _ptr(theta), W, H, _ptr(image), _ptr(target), _ptr(mask), _ptr(m),
                                     float(w1), float(w2), _ptr(loss), _ptr(d_image), _ptr(grad)), "fr_loss")
        return loss

    def step(self, theta, target, W, H, spp, seed=0, iter=0, mask=None, m=None, w1=0.0, w2=0.0, terms=0,
             image=None, d_image=None, grad=None):
        """Render, loss (Eq. 1) and its gradient in one call (fr_step).
        Returns (image [H, W, 3], loss [1] FP64, grad [P] FP64)."""
        theta = self._theta(theta)
        target = target.contiguous()
        assert target.dtype == torch.float32 and target.numel() == W * H * 3
        img = image if image is not None else torch.empty((H, W, 3), device=self.device, dtype=torch.float32)
        g = grad if grad is not None else torch.empty(self.P, device=self.device, dtype=torch.float64)
        loss = torch.empty(1, device=self.device, dtype=torch.float64)
        o = self.opts(W, H, spp, seed, iter, terms)
        self._stream()
        self._check(self.lib.fr_step(self.ctx, _ptr(theta), C.byref(o), _ptr(target), _ptr(mask), _ptr(m),
                                     float(w1), float(w2), _ptr(img), _ptr(d_image), _ptr(loss), _ptr(g)), "fr_step")
        return img, loss, g

    def geometry(self, theta):
        theta = self._theta(theta)
        X = torch.empty((self.V, 3), device=self.device)
        N = torch.empty_like(X)
        A = torch.empty_like(X)
        self._stream()
        n_sil = self._check(self.lib.fr_geometry(self.ctx, _ptr(theta), _ptr(X), _ptr(N), _ptr(A)), "fr_geometry")
        return dict(X=X, normals=N, albedo=A, n_silhouette=n_sil)

    def vertex_grad(self):
        dX = torch.empty((self.V, 3), device=self.device)
        self._stream()
        self._check(self.lib.fr_vertex_grad(self.ctx, _ptr(dX)), "fr_vertex_grad")
        return dX

    def light_stage(self):
        out = np.zeros((self.cfg.n_lights, 12), np.float32)
        self._check(self.lib.fr_light_stage(self.ctx, _hptr(out)), "fr_light_stage")
        return out

    def sync(self):
        return self._check(self.lib.fr_sync(self.ctx), "fr_sync")

    def set_counters(self, on=True):
        self.lib.fr_set_counters(self.ctx, 1 if on else 0)

    def set_limits(self, max_steps=1 << 16, wait_limit=1 << 22):
        """Traversal step cap and batch wait limit of later calls (fr_set_limits)."""
        self._check(self.lib.fr_set_limits(self.ctx, int(max_steps), int(wait_limit)), "fr_set_limits")

    def silhouettes(self):
        """Canonical ids of the camera-silhouette edges of the last geometry
        preparation (fr_silhouettes), host int32 array."""
        n = self._check(self.lib.fr_silhouettes(self.ctx, None, 0), "fr_silhouettes")
        out = np.zeros(max(n, 1), np.int32)
        self._check(self.lib.fr_silhouettes(self.ctx, _hptr(out), n), "fr_silhouettes")
        return out[:n]

    def sync_code(self):
        """fr_sync's return code (0, or e.g. -5 = FR_ERR_DEVICE_LIMIT) without raising."""
        return int(self.lib.fr_sync(self.ctx))

    # -- denoiser -----------------------------------------------------------------
    def set_denoiser(self, w):
        w = np.ascontiguousarray(w, np.float32)
        self._check(self.lib.fr_denoiser_set_weights(self.ctx, _hptr(w), w.size), "fr_denoiser_set_weights")

    def denoiser_weights(self):
        w = np.zeros(self.lib.fr_denoiser_n_weights(), np.float32)
        self._check(self.lib.fr_denoiser_get_weights(self.ctx, _hptr(w), w.size), "fr_denoiser_get_weights")
        return w

    def denoiser_grad(self):
        g = np.zeros(self.lib.fr_denoiser_n_weights(), np.float32)
        self._check(self.lib.fr_denoiser_get_grad(self.ctx, _hptr(g), g.size), "fr_denoiser_get_grad")
        return g

    def denoise(self, aov, d_out=None):
        """aov [..., 14] -> denoised RGB [..., 3]; with d_out also returns J^T d_out."""
        aov = aov.contiguous()
        n = aov.numel() // 14
        out = torch.empty(aov.shape[:-1] + (3,), device=self.device, dtype=torch.float32)
        d_rgb = None if d_out is None else torch.empty_like(out)
        self._stream()
        self._check(self.lib.fr_denoise(self.ctx, _ptr(aov), n, _ptr(out),
                                        _ptr(None if d_out is None else d_out.contiguous()), _ptr(d_rgb)),
                    "fr_denoise")
        return out if d_out is None else (out, d_rgb)

    def denoiser_train_step(self, aov, target, lr):
        aov = aov.contiguous()
        target = target.contiguous()
        loss = torch.empty(1, device=self.device, dtype=torch.float64)
        self._stream()
        self._check(self.lib.fr_denoiser_train_step(self.ctx, _ptr(aov), _ptr(target), aov.numel() // 14,
                                                    float(lr), _ptr(loss)), "fr_denoiser_train_step")
        return loss

    def adam_step(self, theta, grad, m, v, lr, step):
        """In-place Adam step on theta (see fr_adam_step)."""
        self._stream()
        self._check(self.lib.fr_adam_step(self.ctx, _ptr(theta), _ptr(grad), _ptr(m), _ptr(v), _ptr(lr), int(step)),
                    "fr_adam_step")

    def launches(self) -> int:
        return int(self.lib.fr_launch_count(self.ctx))

    PHASES = ("geometry", "forward", "interior", "primary_edges", "shadow_edge_search", "adjoint", "loss",
              "shadow_edge_contributions")

    def set_timing(self, on=True):
        self._check(self.lib.fr_set_timing(self.ctx, 1 if on else 0), "fr_set_timing")

    def timings(self) -> dict:
        out = np.zeros(len(self.PHASES), np.float32)
        self._check(self.lib.fr_get_timings(self.ctx, _hptr(out)), "fr_get_timings")
        return dict(zip(self.PHASES, out.tolist()))

    def counters(self):
        out = np.zeros(24, np.uint64)
        self._check(self.lib.fr_get_counters(self.ctx, _hptr(out)), "fr_get_counters")
        return out


class FaceRender(torch.autograd.Function):
    """image = F(theta): forward renders, backward re-traces with the same samples."""

    @staticmethod
    def forward(ctx, theta, renderer: Renderer, W: int, H: int, spp: int, seed: int = 0, iter: int = 0):
        ctx.renderer = renderer
        ctx.args = (W, H, spp, seed, iter)
        ctx.save_for_backward(theta)
        return renderer.render(theta.detach().contiguous(), W, H, spp, seed, iter)

    @staticmethod
    def backward(ctx, d_image):
        (theta,) = ctx.saved_tensors
        W, H, spp, seed, iter = ctx.args
        g = ctx.renderer.backward(theta.detach().contiguous(), d_image.float().contiguous(), W, H, spp, seed, iter)
        return g.to(torch.float32), None, None, None, None, None, None


def render(theta, renderer: Renderer, W: int, H: int, spp: int, seed: int = 0, iter: int = 0):
    """Differentiable render (autograd entry point)."""
    return FaceRender.apply(theta, renderer, W, H, spp, seed, iter)


class Batch:
    """Batched frames (fr_batch_*): frames of one face with shared identity,
    albedo and specular map and per-frame expression, pose and lights, each
    at its own crop size; one step = one CUDA graph (geometry, the render +
    loss + backward of all frames, geometry adjoints)."""

    def __init__(self, renderer: Renderer, frames, spp: int):
        """frames: list of (W, H, seed)."""
        self.r = renderer
        self.lib = renderer.lib
        self.frames = [(int(w), int(h), int(sd)) for w, h, sd in frames]
        arr = (FrFrame * len(self.frames))(*[FrFrame(w, h, sd) for w, h, sd in self.frames])
        self.spp = int(spp)
        self.n_pix = sum(w * h for w, h, _ in self.frames)
        self.offsets = np.cumsum([0] + [w * h for w, h, _ in self.frames])
        self.Ps = self.lib.fr_batch_n_shared(renderer.ctx)
        self.Pf = self.lib.fr_batch_n_frame(renderer.ctx)
        h = C.c_void_p()
        renderer._stream()
        renderer._check(self.lib.fr_batch_create(renderer.ctx, C.cast(arr, C.c_void_p), len(self.frames), self.spp,
                                                 C.byref(h)), "fr_batch_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.fr_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def split(self, packed):
        """Per-frame [H, W, ...] views of a packed image tensor."""
        out = []
        for f, (w, h, _) in enumerate(self.frames):
            o0, o1 = int(self.offsets[f]), int(self.offsets[f + 1])
            out.append(packed[o0:o1].reshape(h, w, *packed.shape[1:]))
        return out

    def set_targets(self, targets, masks=None, m=None):
        """targets: packed [n_pix, 3] FP32 device; masks packed [n_pix] uint8."""
        self.r._stream()
        self.r._check(self.lib.fr_batch_set_targets(self.h, _ptr(targets.contiguous()),
                                                    _ptr(None if masks is None else masks.contiguous()),
                                                    _ptr(None if m is None else m.contiguous())),
                      "fr_batch_set_targets")
        self._keep = (targets, masks, m)     # alive until the asynchronous copies into the batch have run

    @property
    def targets(self):
        """The packed target images last given to set_targets (or None)."""
        return self._keep[0] if getattr(self, "_keep", None) else None

    def step(self, theta_shared, theta_frames, w1=0.0, w2=0.0, iter=0, images=True):
        """Returns (loss [1] FP64, grad_shared [Ps] FP64, grad_frames [F, Pf] FP64, images [n_pix, 3] or None)."""
        dev = self.r.device
        loss = torch.empty(1, device=dev, dtype=torch.float64)
        gs = torch.empty(self.Ps, device=dev, dtype=torch.float64)
        gf = torch.empty(len(self.frames), self.Pf, device=dev, dtype=torch.float64)
        img = torch.empty(self.n_pix, 3, device=dev) if images else None
        self.r._stream()
        self.r._check(self.lib.fr_batch_step(self.h, _ptr(theta_shared.contiguous()), _ptr(theta_frames.contiguous()),
                                             float(w1), float(w2), int(iter), _ptr(loss), _ptr(gs), _ptr(gf),
                                             _ptr(img)), "fr_batch_step")
        return loss, gs, gf, img

    def autotune(self, theta_shared, theta_frames, reps=1):
        """Time every launch configuration that fits; keep the fastest.  Returns
        the table (list of dicts) and the chosen configuration."""
        cap = 64
        tab = (FrTileConfig * cap)()
        n = C.c_int32()
        self.r._stream()
        self.r._check(self.lib.fr_batch_autotune(self.h, _ptr(theta_shared.contiguous()),
                                                 _ptr(theta_frames.contiguous()), int(reps), C.cast(tab, C.c_void_p),
                                                 cap, C.byref(n)), "fr_batch_autotune")
        return [tab[i].as_dict() for i in range(min(n.value, cap))], self.config()

    def config(self):
        c = FrTileConfig()
        self.r._check(self.lib.fr_batch_get_config(self.h, C.byref(c)), "fr_batch_get_config")
        return c.as_dict()

    def set_config(self, tile_w=8, tile_h=8, block=256, min_blocks=4, fused=0):
        c = FrTileConfig(int(tile_w), int(tile_h), int(block), int(min_blocks), int(fused), 0.0)
        self.r._check(self.lib.fr_batch_set_config(self.h, C.byref(c)), "fr_batch_set_config")


def batch_plan(frames, spp, tile_w, tile_h, n_lights=20):
    """Work items of the persistent batch launch, in queue order (fr_batch_plan;
    host only): an int32 array [n, 2] of (x, y) pairs."""
    L = load()
    frames = [(int(w), int(h), int(sd)) for w, h, sd in frames]
    arr = (FrFrame * len(frames))(*[FrFrame(w, h, sd) for w, h, sd in frames])
    n = C.c_int64(0)
    args = (C.cast(arr, C.c_void_p), len(frames), int(spp), int(tile_w), int(tile_h), int(n_lights))
    rc = L.fr_batch_plan(*args, None, 0, C.byref(n))
    if rc:
        raise RuntimeError(f"fr_batch_plan: {FR_ERRORS.get(rc, rc)}")
    out = np.zeros((n.value, 2), np.int32)
    rc = L.fr_batch_plan(*args, out.ctypes.data_as(C.c_void_p), n.value, C.byref(n))
    if rc:
        raise RuntimeError(f"fr_batch_plan: {FR_ERRORS.get(rc, rc)}")
    return out


def split_theta(theta, K=(80, 90, 80), n_lights=20):
    """Full parameter vector(s) -> (shared, frame) parts: shared = alpha,
    delta, c_spec; frame = beta, pose, lights.  theta: [..., P] array or tensor."""
    K_id, K_exp, K_alb = K
    o_b, o_d = K_id, K_id + K_exp
    o_c = o_d + K_alb
    o_p = o_c + 32 * 32
    lib = torch if isinstance(theta, torch.Tensor) else np
    cat = (lambda xs: torch.cat(xs, -1)) if lib is torch else (lambda xs: np.concatenate(xs, -1))
    shared = cat([theta[..., :o_b], theta[..., o_d:o_p]])
    frame = cat([theta[..., o_b:o_d], theta[..., o_p:]])
    return shared, frame


def join_theta(shared, frame, K=(80, 90, 80)):
    """Inverse of split_theta for one frame."""
    K_id, K_exp, K_alb = K
    lib = torch if isinstance(shared, torch.Tensor) else np
    cat = (lambda xs: torch.cat(xs, -1)) if lib is torch else (lambda xs: np.concatenate(xs, -1))
    return cat([shared[..., :K_id], frame[..., :K_exp], shared[..., K_id:], frame[..., K_exp:]])
