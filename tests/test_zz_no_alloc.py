"""fr_geometry_noalloc against fr_geometry, through the C ABI.

The no-allocation variant is for callers that must not allocate device
memory while it runs (an allocator that owns the device, a fixed memory
budget, or a loop that cannot take the synchronisation an allocation may
cause).  Its silhouette-compaction scratch lives in a static device array
instead of a context buffer; its outputs, and the silhouette list that the
compaction writes, must equal fr_geometry's.  Two calls in a row check that
the shared array's leftover contents do not leak into the next call; a mesh
with more edges than the array covers is refused.  This file sorts last so
that a run stopping at the first failure has already run every other test.
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
    lists = []
    for th in thetas:                      # two calls in a row, different poses
        t = torch.tensor(th, device="cuda:0")
        torch.cuda.synchronize()
        n_ref, X_ref, N_ref, A_ref = _outputs(lib, ctx, "fr_geometry", t, r.V)
        sil_ref = r.silhouettes()
        n_new, X_new, N_new, A_new = _outputs(lib, ctx, "fr_geometry_noalloc", t, r.V)
        sil_new = r.silhouettes()
        assert n_new == n_ref and n_ref > 0
        # the list the compaction through the static array wrote: the same
        # canonical edge ids, in increasing order
        assert np.array_equal(sil_new, sil_ref)
        assert np.all(np.diff(sil_new) > 0)
        lists.append(sil_new)
        # same kernels on the same inputs: the geometry tolerance of the parity tests
        assert np.abs(X_new - X_ref).max() <= 1e-6
        assert np.abs(N_new - N_ref).max() <= 2e-5
        assert np.abs(A_new - A_ref).max() <= 2e-5
    assert not np.array_equal(lists[0], lists[1])     # the second pose has its own silhouettes


def test_noalloc_refuses_meshes_beyond_its_array():
    """A 593 x 593 vertex grid has 1,052,576 edges, more than the static
    array's 4096 blocks of 256 edges: refused before any kernel runs."""
    from paper_1910_05200_gb300 import build, facert
    build.build()
    n = 593
    iy, ix = np.mgrid[0:n, 0:n]
    verts = np.stack([ix.ravel() / (n - 1) - 0.5, iy.ravel() / (n - 1) - 0.5, np.zeros(n * n)], 1)
    q = (iy[:-1, :-1] * n + ix[:-1, :-1]).ravel()
    tris = np.concatenate([np.stack([q, q + 1, q + n + 1], 1), np.stack([q, q + n + 1, q + n], 1)])
    E = 3 * (n - 1) ** 2 + 2 * (n - 1)
    assert E > 4096 * 256
    scene = S.Scene(verts.astype(np.float32), tris.astype(np.int32), np.zeros((n * n, 2), np.float32),
                    np.zeros((3 * n * n, 0), np.float32), np.zeros((3 * n * n, 0), np.float32),
                    np.full(3 * n * n, 0.5, np.float32), np.zeros((3 * n * n, 0), np.float32))
    r = facert.Renderer(scene, device=0)
    th = torch.zeros(r.P, device="cuda:0")
    X = torch.empty(n * n, 3, device="cuda:0")
    rc = r.lib.fr_geometry_noalloc(r.ctx, C.c_void_p(th.data_ptr()), C.c_void_p(X.data_ptr()), None, None)
    assert rc == -1 and b"at most" in r.lib.fr_last_error(r.ctx)


def test_noalloc_rejects_no_context():
    from paper_1910_05200_gb300 import facert
    lib = facert.load()
    assert lib.fr_geometry_noalloc(None, None, None, None, None) < 0
