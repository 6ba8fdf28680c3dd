"""The C ABI library builds for sm_103a, loads, and exports every symbol that
include/sph.h declares (no GPU needed: nothing is called that touches a device)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(sph_[a-z_0-9]+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    import paper_2004_13887_gb300 as pkg
    pkg.build()
    return pkg.load()


def test_every_declared_symbol_is_exported(lib):
    import paper_2004_13887_gb300 as pkg
    names = _declared()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n
        assert n in pkg.SIGNATURES, n


def test_host_only_calls(lib):
    import ctypes as C
    import paper_2004_13887_gb300 as pkg
    from inputs import Grid
    g = Grid(4, 5, 6, 1.0, 2.0, 0.5, 2.5, 0.0, 1.0)
    s = pkg._grid_struct(g)
    sizes = [lib.sph_field_size(C.byref(s), f) for f in range(5)]
    assert sizes == [4 * 5 * 6, 5 * 5 * 6, 4 * 6 * 6, 4 * 5 * 7, 4 * 5 * 6]
    assert lib.sph_strerror(-3).startswith(b"non-finite")
    # argument validation happens before any device work
    h = C.c_void_p()
    bad = pkg.sph_grid(1, 5, 6, 1.0, 2.0, 0.5, 2.5, 0.0, 1.0, 0)
    p = pkg.sph_params(1.4, 1.0, 1.0, 0.1, 0.0, 0.0, 0.0, 0)
    assert lib.sph_create(C.byref(bad), C.byref(p), None, C.byref(h)) == -1
    assert lib.sph_launch_count(None) == 0


def test_no_cpu_fallback_without_library(tmp_path):
    import paper_2004_13887_gb300 as pkg
    with pytest.raises(RuntimeError):
        pkg._lib_backup = pkg._lib
        try:
            pkg._lib = None
            pkg.load(str(tmp_path / "missing.so"))
        finally:
            pkg._lib = pkg._lib_backup
