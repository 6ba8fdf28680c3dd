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


def _defines():
    vals = {}
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            for name, v in re.findall(r"^#define\s+(SPH_[A-Z_0-9]+)\s+\(?(-?\d+)\)?\b", open(os.path.join(ROOT, "include", fn)).read(),
                                      flags=re.M):
                vals[name] = int(v)
    return vals


def test_binding_constants_match_header():
    """Every SPH_* constant of the Python binding has the header's value, and the
    stage names it reports follow the header's SPH_K_* order."""
    import paper_2004_13887_gb300 as pkg
    d = _defines()
    consts = {n: getattr(pkg, n) for n in dir(pkg) if n.startswith("SPH_") and isinstance(getattr(pkg, n), int)}
    assert {"SPH_PREC_FP64", "SPH_PREC_MIXED", "SPH_LINES_THOMAS", "SPH_LINES_PARTITIONED",
            "SPH_LINES_PARTITIONED_WARP", "SPH_LINES_PARTITIONED_NARROW"} <= set(consts)
    for n, v in consts.items():
        assert n in d and d[n] == v, (n, v, d.get(n))
    names = ["avg", "coef", "rhs", "sweep_r", "sweep_theta", "sweep_phi"]
    keys = ["SPH_K_AVG", "SPH_K_COEF", "SPH_K_RHS", "SPH_K_SWEEP_R", "SPH_K_SWEEP_TH", "SPH_K_SWEEP_PH"]
    assert [pkg.Solver.KERNELS[d[k]] for k in keys] == names
    # Solver.profile_read passes buffers of 8 entries
    assert d["SPH_NKERNELS"] == 8 and len(pkg.Solver.KERNELS) <= d["SPH_NKERNELS"]


def test_noalloc_binding_checks_shapes_before_the_library(monkeypatch):
    """block_thomas_noalloc rejects mismatched shapes, dtypes and devices before
    it loads or calls the library (a smaller A, C or d would be read past its
    end on the device)."""
    import torch
    import paper_2004_13887_gb300 as pkg

    def boom(*a, **k):
        raise AssertionError("the library must not be reached")
    monkeypatch.setattr(pkg, "load", boom)
    blk = lambda *s: torch.zeros(*s, dtype=torch.float64)
    good = (blk(4, 6, 3, 3), blk(4, 6, 3, 3), blk(4, 6, 3, 3), blk(4, 6, 3))
    for bad in ((blk(3, 6, 3, 3),) + good[1:],                      # fewer lines in A
                good[:2] + (blk(4, 5, 3, 3), good[3]),             # shorter C
                good[:3] + (blk(4, 6, 2),),                         # d's trailing dim
                good[:1] + (blk(4, 6, 9),) + good[2:]):             # B not 3x3 blocks
        with pytest.raises(ValueError):
            pkg.block_thomas_noalloc(*bad)
    with pytest.raises(TypeError):
        pkg.block_thomas_noalloc(good[0].float(), *good[1:])
    with pytest.raises(ValueError):   # host tensors: not CUDA
        pkg.block_thomas_noalloc(*good)
