"""CPU checks of the C ABI: the library loads without a GPU and exports every entry point that
include/xtc.h declares, and the binding names the same set."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "xtc.h")


def declared():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"XTC_API\s+[\w\s\*]+?\b(xtc_\w+)\s*\(", src)))


def _lib_path():
    from paper_2304_07006_gb300 import xtc
    if not os.path.exists(xtc.LIB_PATH):
        from paper_2304_07006_gb300 import _build
        _build.build()
    return xtc.LIB_PATH


def test_header_declares_the_boundary():
    names = declared()
    for must in ("xtc_create", "xtc_set_jastrow", "xtc_build_1b2b", "xtc_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(_lib_path())
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_lists_the_declared_symbols():
    from paper_2304_07006_gb300 import xtc
    assert sorted(xtc.EXPORTED) == declared()


def test_strerror_and_defaults_without_gpu():
    from paper_2304_07006_gb300 import xtc
    lib = xtc.load(_lib_path())
    assert lib.xtc_strerror(0) == b"success"
    assert b"symmetric" in lib.xtc_strerror(-2)
    p = xtc.XtcParams()
    lib.xtc_default_params(ctypes.byref(p))
    assert p.precision == xtc.PREC_FP16X2 and p.grid_chunk == 0 and p.range_stages == 0
    # argument checks happen before any device call
    h = ctypes.c_void_p()
    assert lib.xtc_create(ctypes.byref(h), None) == -1
    p.grid_chunk = 100  # not a multiple of 128
    assert lib.xtc_create(ctypes.byref(h), ctypes.byref(p)) == -1
    p.grid_chunk = 0
    p.range_stages = 5  # ranges of 1..4 stages
    assert lib.xtc_create(ctypes.byref(h), ctypes.byref(p)) == -1


def test_missing_library_fails_loudly(tmp_path):
    from paper_2304_07006_gb300 import xtc
    saved = xtc._lib
    xtc._lib = None
    try:
        with pytest.raises(RuntimeError, match="missing"):
            xtc.load(str(tmp_path / "nope.so"))
    finally:
        xtc._lib = saved


def test_params_struct_layout_matches_the_header(tmp_path):
    """The binding's xtc_params has the size and field offsets that a C compiler gives the header's."""
    import shutil
    import subprocess
    from paper_2304_07006_gb300 import xtc
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    fields = [f[0] for f in xtc.XtcParams._fields_]
    body = " ".join(f'printf("%zu ", offsetof(xtc_params, {f}));' for f in fields)
    src = tmp_path / "layout.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "xtc.h"\n'
                   f'int main(void) {{ printf("%zu ", sizeof(xtc_params)); {body} return 0; }}\n')
    exe = tmp_path / "layout"
    subprocess.check_call([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    want = [ctypes.sizeof(xtc.XtcParams)] + [getattr(xtc.XtcParams, f).offset for f in fields]
    assert got == want


def _shell_context():
    """A Context without a device: the binding's argument checks run before any library call."""
    from paper_2304_07006_gb300 import Context
    c = Context.__new__(Context)
    c._h, c._lib = None, None
    return c


def test_binding_rejects_short_or_mistyped_buffers():
    import numpy as np
    c = _shell_context()
    n_grid, n = 10, 3
    grid, w, phi, g = np.zeros((n_grid, 3)), np.ones(n_grid), np.zeros((n_grid, n)), np.eye(n)
    with pytest.raises(ValueError, match="grid_xyz"):
        c.build(grid[:5], w, phi, g)
    with pytest.raises(ValueError, match="weights"):
        c.build(grid, w[:4], phi, g)
    with pytest.raises(ValueError, match="gamma"):
        c.build(grid, w, phi, np.eye(2))
    with pytest.raises(TypeError, match="dh must be float64"):
        c.build(grid, w, phi, g, dh=np.zeros((n, n), dtype=np.float32))
    with pytest.raises(ValueError, match="dU"):
        c.build(grid, w, phi, g, dU=np.zeros(n ** 3))
    with pytest.raises(TypeError, match="dU_f32 must be float32"):
        c.build(grid, w, phi, g, dU_f32=np.zeros(n ** 4))
    with pytest.raises(ValueError, match="dh_b"):
        c.build_rohf(grid, w, phi, g, g, dh_b=np.zeros(2))
    with pytest.raises(ValueError, match="L holds"):
        c.three_body_L(grid, w, phi, out=np.zeros(n ** 5))
    with pytest.raises(ValueError, match="V holds"):
        c.vfield(grid, w, phi, 0, 4, out=np.zeros(5))
    with pytest.raises(ValueError, match="r2"):
        c.jastrow_grad(np.zeros((4, 3)), np.zeros((2, 3)))
    with pytest.raises(ValueError, match="nuc_set"):
        c.set_jastrow(np.zeros((2, 3)), [0], np.array([(0, 0, 1)]), np.ones((1, 1)))
    with pytest.raises(ValueError, match="coef"):
        c.set_jastrow(np.zeros((2, 3)), [0, 0], np.array([(0, 0, 1)]), np.ones((1, 2)))
