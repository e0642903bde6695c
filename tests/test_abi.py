"""CPU checks of the C-ABI library: it builds for sm_103a, loads, and exports
every entry point that include/facert.h declares (no GPU calls)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1910_05200_gb300 import build
    path = build.build()
    return C.CDLL(path)


def declared_functions():
    text = open(os.path.join(ROOT, "include", "facert.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(fr_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["fr_create", "fr_destroy", "fr_upload_mesh", "fr_upload_bases", "fr_render",
                     "fr_render_backward", "fr_loss", "fr_strerror"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header():
    from paper_1910_05200_gb300 import facert
    assert sorted(facert.EXPORTS) == declared_functions()


def test_host_only_calls(lib):
    lib.fr_strerror.restype = C.c_char_p
    assert lib.fr_strerror(-5) == b"device traversal limit reached"

    class Cfg(C.Structure):   # fr_config: 9 floats, n_lights, brdf_model, fresnel, light_layout, light_prior
        _fields_ = [(n, C.c_float) for n in ("a", "b", "c", "d", "e", "f", "g", "h", "i")] + \
                   [(n, C.c_int32) for n in ("n", "brdf", "fresnel", "layout", "prior")]

    from paper_1910_05200_gb300 import facert
    assert C.sizeof(Cfg) == C.sizeof(facert.FrConfig)
    c = Cfg()
    lib.fr_default_config(C.byref(c))
    assert c.n == 20 and abs(c.a - 0.275) < 1e-7 and abs(c.d - 0.6) < 1e-7
    assert (c.brdf, c.fresnel, c.layout, c.prior) == (0, 0, 0, 0)
    # creating a context without a GPU fails cleanly with a negative code
    h = C.c_void_p()
    rc = lib.fr_create(C.byref(h), None, 0)
    if rc == 0:
        lib.fr_destroy(h)
    else:
        assert rc < 0


def test_header_is_plain_c_and_links(tmp_path, lib):
    """A C99 program includes only include/facert.h, links against the
    library and calls host-only entry points (no GPU): the boundary needs
    neither C++ nor CUDA nor torch headers."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    from paper_1910_05200_gb300 import build
    src = tmp_path / "use_facert.c"
    src.write_text(r'''
#include <stdio.h>
#include "facert.h"
int main(void) {
  fr_config c;
  fr_ctx* ctx = 0;
  int rc;
  fr_default_config(&c);
  printf("%d %d %d %d %d %s\n", c.n_lights, c.brdf_model, c.fresnel, c.light_layout, c.light_prior,
         fr_strerror(FR_ERR_INVALID_ARG));
  c.light_prior = 7;                           /* refused before any device work */
  rc = fr_create(&ctx, &c, 0);
  printf("%d %d\n", rc, ctx == 0);
  return 0;
}
''')
    exe = tmp_path / "use_facert"
    libdir = os.path.dirname(build.LIB)
    subprocess.check_call([cc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
                           "-o", str(exe), "-L", libdir, "-l:" + os.path.basename(build.LIB),
                           "-Wl,-rpath," + libdir])
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    assert out[0] == "20 0 0 0 0 invalid argument"
    rc, null = out[1].split()
    assert int(rc) < 0 and null == "1"
