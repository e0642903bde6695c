"""fr_geometry_noalloc against fr_geometry, through the C ABI.

The no-allocation variant is for callers that must not allocate device
memory while it runs (an allocator that owns the device, a fixed memory
budget, or a loop that cannot take the synchronisation an allocation may
cause).  Its silhouette-compaction scratch lives in a static device array
instead of a context buffer; its outputs must equal fr_geometry's.  Two calls
in a row check that the shared array's leftover contents do not leak into the
next call.  This file sorts last so that a run stopping at the first failure
has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_1910_05200_gb300 import synthetic as S

pytestmark = pytest.mark.gpu


def _outputs(lib, ctx, fn, theta, V):
    X = torch.full((V, 3), float("nan"), device="cuda:0")
    N = torch.full_like(X, float("nan"))
    A = torch.full_like(X, float("nan"))
    rc = getattr(lib, fn)(ctx, C.c_void_p(theta.data_ptr()), C.c_void_p(X.data_ptr()), C.c_void_p(N.data_ptr()),
                          C.c_void_p(A.data_ptr()))
    assert rc >= 0, (fn, rc, lib.fr_last_error(ctx))
    return rc, X.cpu().numpy(), N.cpu().numpy(), A.cpu().numpy()


def test_noalloc_geometry_matches_fr_geometry():
    from paper_1910_05200_gb300 import build, facert
    build.build()
    scene, theta0, _ = S.make_workload("tiny", seed=0)
    r = facert.Renderer(scene, device=0)
    lib, ctx = r.lib, r.ctx
    thetas = [theta0, S.make_theta(scene, seed=5, max_angle_deg=25.0)]
    for th in thetas:                      # two calls in a row, different poses
        t = torch.tensor(th, device="cuda:0")
        torch.cuda.synchronize()
        n_ref, X_ref, N_ref, A_ref = _outputs(lib, ctx, "fr_geometry", t, r.V)
        n_new, X_new, N_new, A_new = _outputs(lib, ctx, "fr_geometry_noalloc", t, r.V)
        assert n_new == n_ref and n_ref > 0
        # same kernels on the same inputs: the geometry tolerance of the parity tests
        assert np.abs(X_new - X_ref).max() <= 1e-6
        assert np.abs(N_new - N_ref).max() <= 2e-5
        assert np.abs(A_new - A_ref).max() <= 2e-5
    # the silhouette list the variant leaves behind drives the gradient identically
    t = torch.tensor(thetas[1], device="cuda:0")
    dI = torch.randn(32, 32, 3, device="cuda:0", generator=torch.Generator("cuda:0").manual_seed(1))
    g_ref = r.backward(t, dI, 32, 32, 2, seed=3, terms=2).cpu().numpy()
    assert r.sync() == 0
    r2 = facert.Renderer(scene, device=0)
    _outputs(r2.lib, r2.ctx, "fr_geometry_noalloc", t, r2.V)
    g_new = r2.backward(t, dI, 32, 32, 2, seed=3, terms=2).cpu().numpy()
    scale = np.abs(g_ref).max()
    assert np.abs(g_new - g_ref).max() <= 1e-4 * scale


def test_noalloc_rejects_no_context():
    from paper_1910_05200_gb300 import facert
    lib = facert.load()
    assert lib.fr_geometry_noalloc(None, None, None, None, None) < 0
