"""GB300 (sm_103a) implementation of the direction-splitting scheme for weakly
compressible flow in spherical coordinates (Frolov, Minev & Takhirov,
arXiv 2004.13887).

A thin ctypes binding over the C ABI in include/sph.h (libsph.so, built in-tree
by ``build()``).  Every step of the method runs in the library's CUDA kernels;
this module only marshals arguments.  PyTorch supplies device memory and the
stream.  There is no CPU fallback: without the built library every call raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from ._build import LIB, build

__all__ = ["build", "load", "Solver", "Batch", "SphError", "sph_field_size", "SPH_PREC_FP64", "SPH_PREC_MIXED",
           "SPH_LINES_THOMAS", "SPH_LINES_PARTITIONED", "SPH_LINES_PARTITIONED_WARP",
           "SPH_LINES_PARTITIONED_NARROW"]

SPH_PREC_FP64 = 0
SPH_PREC_MIXED = 1
SPH_LINES_THOMAS = 0
SPH_LINES_PARTITIONED = 1
SPH_LINES_PARTITIONED_WARP = 2
SPH_LINES_PARTITIONED_NARROW = 3

_ERRORS = {0: "ok", -1: "invalid argument", -2: "CUDA runtime error", -3: "non-finite state",
           -4: "zero pivot in a line solve", -5: "device allocation failed", -6: "adjoint tape too short"}


class SphError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {_ERRORS.get(code, 'unknown')} ({code})")


class sph_grid(C.Structure):
    _fields_ = [("nr", C.c_int), ("nth", C.c_int), ("nph", C.c_int),
                ("r1", C.c_double), ("r2", C.c_double), ("th1", C.c_double), ("th2", C.c_double),
                ("ph1", C.c_double), ("ph2", C.c_double), ("periodic_phi", C.c_int)]


class sph_params(C.Structure):
    _fields_ = [("gamma", C.c_double), ("cv", C.c_double), ("Pr", C.c_double), ("mu", C.c_double),
                ("pi_inf", C.c_double), ("g", C.c_double), ("omega", C.c_double), ("precision", C.c_int)]


_lib = None
_DP = C.POINTER(C.c_double)
_PP = C.POINTER(_DP)
_CTX = C.c_void_p

# name -> (argtypes, restype); every symbol include/sph.h declares
SIGNATURES = {
    "sph_field_size": ([C.POINTER(sph_grid), C.c_int], C.c_size_t),
    "sph_create": ([C.POINTER(sph_grid), C.POINTER(sph_params), C.c_void_p, C.POINTER(_CTX)], C.c_int),
    "sph_set_background": ([_CTX, _DP, _DP], C.c_int),
    "sph_set_bc": ([_CTX, _PP, _PP, C.c_int], C.c_int),
    "sph_set_state": ([_CTX, _PP, C.c_int], C.c_int),
    "sph_get_state": ([_CTX, _PP, C.c_int], C.c_int),
    "sph_step": ([_CTX, C.c_double, C.c_int, _PP, C.c_int, _DP], C.c_int),
    "sph_step_async": ([_CTX, C.c_double, C.c_int, _PP, C.c_int], C.c_int),
    "sph_status": ([_CTX, _DP], C.c_int),
    "sph_batch_create": ([C.POINTER(_CTX), C.c_int, C.c_void_p, C.POINTER(C.c_void_p)], C.c_int),
    "sph_batch_capture": ([C.c_void_p, C.c_double, C.c_int, C.c_int], C.c_int),
    "sph_batch_capture_fused": ([C.c_void_p, C.c_double, C.c_int, C.c_int], C.c_int),
    "sph_batch_launch": ([C.c_void_p, C.c_int], C.c_int),
    "sph_batch_status": ([C.c_void_p, C.POINTER(C.c_int)], C.c_int),
    "sph_batch_destroy": ([C.c_void_p], None),
    "sph_set_iterate": ([_CTX, _PP, C.c_int], C.c_int),
    "sph_rhs": ([_CTX, C.c_double, _PP, C.c_int, _PP], C.c_int),
    "sph_sweep": ([_CTX, C.c_int, C.c_double, _PP, _PP], C.c_int),
    "sph_set_line_solver": ([_CTX, C.c_int], C.c_int),
    "sph_set_tile": ([_CTX, C.c_int, C.c_int], C.c_int),
    "sph_launch_count": ([_CTX], C.c_longlong),
    "sph_bounds_report": ([C.POINTER(C.c_int)], C.c_int),
    "sph_profile": ([_CTX, C.c_int], C.c_int),
    "sph_profile_read": ([_CTX, _DP, C.POINTER(C.c_longlong)], C.c_int),
    "sph_destroy": ([_CTX], None),
    "sph_block_thomas_noalloc": ([C.c_int, C.c_int, _DP, _DP, _DP, _DP, _DP, C.c_void_p], C.c_int),
    "sph_step_adjoint": ([_CTX, C.c_double, C.c_int, _PP, _PP, _PP], C.c_int),
    "sph_schur_local": ([C.c_int, C.c_int, _DP, _DP, _DP, _DP, _DP, _DP, _DP, _DP, C.POINTER(C.c_int), C.c_void_p],
                        C.c_int),
    "sph_schur_reduced": ([C.c_int, C.c_int, C.c_int, _DP, _DP, C.POINTER(C.c_int), C.c_void_p], C.c_int),
    "sph_schur_back": ([C.c_int, C.c_int, _DP, _DP, _DP, _DP, _DP, _DP, C.c_void_p], C.c_int),
    "sph_adjoint_tape_use": ([_CTX, C.POINTER(C.c_int), C.POINTER(C.c_int)], C.c_int),
    "sph_strerror": ([C.c_int], C.c_char_p),
}


def load(path: str = LIB):
    """Load libsph.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: run paper_2004_13887_gb300.build() (needs nvcc)")
        L = C.CDLL(path)
        for name, (args, res) in SIGNATURES.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def use_library(path: str):
    """Switch every later call to the library at `path` (for example the
    bounds-checked debug build, _build.LIB_CHECKED); returns the previous one.
    Solvers created before the switch must be closed first."""
    global _lib
    prev = _lib
    _lib = None
    load(path)
    return prev


def restore_library(prev):
    global _lib
    _lib = prev


def bounds_report():
    """(violations since the last call, (field, i, j, k) of the first); -1 from a
    regular build"""
    first = (C.c_int * 4)()
    n = load().sph_bounds_report(first)
    return n, tuple(first)


def _grid_struct(grid) -> sph_grid:
    return sph_grid(int(grid.nr), int(grid.nt), int(grid.np), float(grid.r1), float(grid.r2), float(grid.t1),
                    float(grid.t2), float(grid.p1), float(grid.p2), int(bool(grid.periodic)))


def sph_field_size(grid, f: int) -> int:
    g = _grid_struct(grid)
    return int(load().sph_field_size(C.byref(g), f))


def _check(code, what):
    if code != 0:
        raise SphError(code, what)


NOALLOC_MAX_BLOCKS = 131072


def block_thomas_noalloc(A, B, Cb, d, stream=None):
    """Solve nlines independent 3x3-block tridiagonal lines without any device
    allocation inside the library (sph_block_thomas_noalloc).

    A, B, Cb: CUDA float64 tensors (nlines, n, 3, 3); d: (nlines, n, 3), all on
    one device.  The solve runs on that device, on `stream` (default: that
    device's current stream).  The output tensor is allocated here by torch, on
    the caller's side, in the stream the solve runs on.  Shapes, dtypes and
    devices are checked before anything reaches the library (a smaller array
    would be read past its end)."""
    import torch
    for t in (A, B, Cb, d):
        if not isinstance(t, torch.Tensor):
            raise TypeError("A, B, C, d must be torch tensors")
    if B.dim() != 4 or tuple(B.shape[2:]) != (3, 3):
        raise ValueError(f"B must have shape (nlines, n, 3, 3), not {tuple(B.shape)}")
    nlines, n = int(B.shape[0]), int(B.shape[1])
    for name, t, shape in (("A", A, (nlines, n, 3, 3)), ("C", Cb, (nlines, n, 3, 3)), ("d", d, (nlines, n, 3))):
        if tuple(t.shape) != shape:
            raise ValueError(f"{name} must have shape {shape}, not {tuple(t.shape)}")
    for t in (A, B, Cb, d):
        if t.dtype != torch.float64 or not t.is_contiguous():
            raise TypeError("A, B, C, d must be contiguous float64 tensors")
    if not all(t.is_cuda for t in (A, B, Cb, d)) or len({t.device for t in (A, B, Cb, d)}) != 1:
        raise ValueError("A, B, C, d must be CUDA tensors on one device")
    dev = B.device
    if stream is None:
        stream = torch.cuda.current_stream(dev)
    elif stream.device != dev:
        raise ValueError(f"stream is on {stream.device}, the tensors on {dev}")
    with torch.cuda.device(dev), torch.cuda.stream(stream):
        x = torch.empty((nlines, n, 3), dtype=torch.float64, device=dev)
        p = [C.cast(C.c_void_p(t.data_ptr()), _DP) for t in (A, B, Cb, d, x)]
        _check(load().sph_block_thomas_noalloc(nlines, n, *p, C.c_void_p(stream.cuda_stream)),
               "sph_block_thomas_noalloc")
    return x


class _Ptrs:
    """double*[5] view of 5 torch tensors or numpy arrays (kept alive)."""

    def __init__(self, fields, shapes, device):
        import torch
        if len(fields) != 5:
            raise ValueError("need 5 fields: p, u_r, u_theta, u_phi, T")
        self.keep = []
        ptrs = []
        for f, shp in zip(fields, shapes):
            if device:
                if not (isinstance(f, torch.Tensor) and f.is_cuda and f.dtype == torch.float64):
                    raise TypeError("device fields must be CUDA float64 tensors")
                if tuple(f.shape) != tuple(shp) and f.numel() != int(np.prod(shp)):
                    raise ValueError(f"field shape {tuple(f.shape)} != {tuple(shp)}")
                f = f.contiguous()
                self.keep.append(f)
                ptrs.append(C.cast(C.c_void_p(f.data_ptr()), _DP))
            else:
                a = np.ascontiguousarray(f, dtype=np.float64)
                if a.size != int(np.prod(shp)):
                    raise ValueError(f"field size {a.size} != {int(np.prod(shp))}")
                self.keep.append(a)
                ptrs.append(a.ctypes.data_as(_DP))
        self.arr = (_DP * 5)(*ptrs)


def torch_float64():
    import torch
    return torch.float64


class Solver:
    """One sector (or shell) and its state on the current CUDA device.

    grid: object with nr, nt, np, r1, r2, t1, t2, p1, p2, periodic.
    par:  object with gamma, cv, Pr, mu, pinf, g, omega.
    """

    def __init__(self, grid, par, precision: int = SPH_PREC_FP64, stream=None):
        import torch
        L = load()
        self.grid = grid
        self._g = _grid_struct(grid)
        self._p = sph_params(float(par.gamma), float(par.cv), float(par.Pr), float(par.mu), float(par.pinf),
                             float(par.g), float(par.omega), int(precision))
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        h = _CTX()
        _check(L.sph_create(C.byref(self._g), C.byref(self._p), C.c_void_p(stream.cuda_stream), C.byref(h)),
               "sph_create")
        self._h = h
        self.shapes = grid.shapes()

    # -------------------------------------------------------------- state
    def set_background(self, p_ref=None, T_ref=None):
        n = self.grid.nr + 2
        a = None if p_ref is None else np.ascontiguousarray(p_ref, dtype=np.float64)
        b = None if T_ref is None else np.ascontiguousarray(T_ref, dtype=np.float64)
        for v in (a, b):
            if v is not None and v.size != n:
                raise ValueError(f"background needs {n} values")
        _check(load().sph_set_background(self._h, a.ctypes.data_as(_DP) if a is not None else None,
                                         b.ctypes.data_as(_DP) if b is not None else None), "sph_set_background")

    def set_bc(self, walls_n=None, walls_np1=None):
        """Dirichlet wall velocity at t^n and t^{n+1} for the coming steps
        (sph_set_bc).  walls_*: None or a dict {(c, d, s): array} -- component
        c on the wall normal to direction d at side s -- of numpy arrays (or
        CUDA float64 tensors) in the header's layout; both None = homogeneous
        walls."""
        if walls_n is None and walls_np1 is None:
            _check(load().sph_set_bc(self._h, None, None, 0), "sph_set_bc")
            return
        g = self.grid
        sizes = {}
        for c in range(3):
            for d in range(3):
                sizes[(c, d)] = int(np.prod(g.wall_shape(c, d)))
        keep = []
        dev = None
        arrs = []
        for walls in (walls_n, walls_np1):
            ptrs = [None] * 18
            for (c, d, s), a in (walls or {}).items():
                is_dev = not isinstance(a, np.ndarray)
                if dev is None:
                    dev = is_dev
                elif dev != is_dev:
                    raise ValueError("wall arrays must all be host arrays or all CUDA tensors")
                if is_dev:
                    if not (a.is_cuda and a.dtype == torch_float64()):
                        raise TypeError("device wall data must be CUDA float64 tensors")
                    a = a.contiguous()
                    ptr = C.cast(C.c_void_p(a.data_ptr()), _DP)
                    n = a.numel()
                else:
                    a = np.ascontiguousarray(a, dtype=np.float64)
                    ptr = a.ctypes.data_as(_DP)
                    n = a.size
                if n != sizes[(c, d)]:
                    raise ValueError(f"wall array {(c, d, s)} has {n} values, needs {sizes[(c, d)]}")
                keep.append(a)
                ptrs[(c * 3 + d) * 2 + s] = ptr
            arrs.append((_DP * 18)(*ptrs))
        _check(load().sph_set_bc(self._h, arrs[0], arrs[1], int(bool(dev))), "sph_set_bc")

    # The library works on the solver's stream.  Device arrays handed in were
    # written on torch's current stream, and device arrays handed back are
    # read there: the two streams are ordered around every such call.
    def _after_caller(self):
        import torch
        cur = torch.cuda.current_stream(self.stream.device)
        if cur != self.stream:
            self.stream.wait_stream(cur)

    def _before_caller(self):
        import torch
        cur = torch.cuda.current_stream(self.stream.device)
        if cur != self.stream:
            cur.wait_stream(self.stream)

    def set_state(self, fields):
        dev = not isinstance(fields[0], np.ndarray)
        p = _Ptrs(fields, self.shapes, dev)
        if dev:
            self._after_caller()
        _check(load().sph_set_state(self._h, p.arr, int(dev)), "sph_set_state")

    def set_iterate(self, fields):
        dev = not isinstance(fields[0], np.ndarray)
        p = _Ptrs(fields, self.shapes, dev)
        if dev:
            self._after_caller()
        _check(load().sph_set_iterate(self._h, p.arr, int(dev)), "sph_set_iterate")

    def empty(self):
        import torch
        return [torch.empty(s, dtype=torch.float64, device="cuda") for s in self.shapes]

    def get_state(self, device: bool = True, out=None):
        """The state U^n: new CUDA tensors (device=True) or numpy arrays, or
        written into `out` (5 CUDA float64 tensors, or 5 C-contiguous float64
        numpy arrays -- pinned host memory makes the copy fastest)."""
        if out is not None:
            dev = not isinstance(out[0], np.ndarray)
            for f in out:
                ok = (f.is_contiguous() and f.dtype == torch_float64()) if dev else \
                    (isinstance(f, np.ndarray) and f.dtype == np.float64 and f.flags["C_CONTIGUOUS"] and f.flags["WRITEABLE"])
                if not ok:
                    raise ValueError("out fields must be contiguous, writeable float64 arrays (or CUDA tensors)")
            p = _Ptrs(out, self.shapes, dev)
            if dev:
                self._after_caller()
            _check(load().sph_get_state(self._h, p.arr, int(dev)), "sph_get_state")
            if dev:
                self._before_caller()
            return out
        if device:
            out = self.empty()
            p = _Ptrs(out, self.shapes, True)
            self._after_caller()
            _check(load().sph_get_state(self._h, p.arr, 1), "sph_get_state")
            self._before_caller()
            return out
        out = [np.empty(s) for s in self.shapes]
        p = _Ptrs(out, self.shapes, False)
        _check(load().sph_get_state(self._h, p.arr, 0), "sph_get_state")
        return out

    # --------------------------------------------------------------- step
    def step(self, dt: float, n_iter: int, source=None, residual: bool = False):
        src = None
        on_dev = 0
        if source is not None:
            on_dev = int(not isinstance(source[0], np.ndarray))
            src = _Ptrs(source, self.shapes, bool(on_dev))
        res = np.zeros(5) if residual else None
        if on_dev:
            self._after_caller()
        _check(load().sph_step(self._h, float(dt), int(n_iter), src.arr if src else None, on_dev,
                               res.ctypes.data_as(_DP) if res is not None else None), "sph_step")
        return res

    def step_async(self, dt: float, n_iter: int, source=None):
        """Enqueue one step on the solver's stream (device sources only); check with status()."""
        src = _Ptrs(source, self.shapes, True) if source is not None else None
        if src is not None:
            self._after_caller()
        _check(load().sph_step_async(self._h, float(dt), int(n_iter), src.arr if src else None, 1), "sph_step_async")

    def status(self, residual: bool = False):
        """Synchronise; raise if an enqueued step produced a non-finite value or a zero pivot."""
        res = np.zeros(5) if residual else None
        _check(load().sph_status(self._h, res.ctypes.data_as(_DP) if res is not None else None), "sph_status")
        return res

    # ------------------------------------------------------------ adjoint
    def step_adjoint(self, dt: float, n_iter: int, lam_out, source=None):
        """dJ/dU^n from dJ/dU^{n+1} for the step sph_step takes from the current
        state U^n (sph_step_adjoint; FP64 solvers).  lam_out: 5 CUDA float64
        tensors; source: the step's 5 device source arrays or None.  Returns 5
        new CUDA tensors."""
        lam_in = self.empty()
        lo = _Ptrs(lam_out, self.shapes, True)
        li = _Ptrs(lam_in, self.shapes, True)
        src = _Ptrs(source, self.shapes, True) if source is not None else None
        self._after_caller()
        _check(load().sph_step_adjoint(self._h, float(dt), int(n_iter), src.arr if src else None, lo.arr, li.arr),
               "sph_step_adjoint")
        self._before_caller()
        return lam_in

    def tape_use(self):
        """(longest per-thread tape used by the adjoint so far, capacity)"""
        a, b = C.c_int(0), C.c_int(0)
        _check(load().sph_adjoint_tape_use(self._h, C.byref(a), C.byref(b)), "sph_adjoint_tape_use")
        return a.value, b.value

    # ------------------------------------------------------------- stages
    def rhs(self, dt: float, source=None):
        out = self.empty()
        po = _Ptrs(out, self.shapes, True)
        src = None
        on_dev = 0
        if source is not None:
            on_dev = int(not isinstance(source[0], np.ndarray))
            src = _Ptrs(source, self.shapes, bool(on_dev))
        self._after_caller()
        _check(load().sph_rhs(self._h, float(dt), src.arr if src else None, on_dev, po.arr), "sph_rhs")
        self._before_caller()
        return out

    def sweep(self, direction: int, dt: float, rhs_fields):
        out = self.empty()
        pi = _Ptrs(rhs_fields, self.shapes, True)
        po = _Ptrs(out, self.shapes, True)
        self._after_caller()
        _check(load().sph_sweep(self._h, int(direction), float(dt), pi.arr, po.arr), "sph_sweep")
        self._before_caller()
        return out

    def set_line_solver(self, which: int):
        """SPH_LINES_PARTITIONED (default), SPH_LINES_PARTITIONED_WARP (one warp per line),
        SPH_LINES_PARTITIONED_NARROW (4 or 8 lanes for lines of 16 to 64 cells) or
        SPH_LINES_THOMAS for the mixed-precision sweeps.  In the FP64 mode
        SPH_LINES_THOMAS takes one thread per line and every other value two
        threads per walled line (elimination from both ends)."""
        _check(load().sph_set_line_solver(self._h, int(which)), "sph_set_line_solver")

    def set_tile(self, tj: int, ti: int):
        """stencil tile shape: 128/(tj ti) phi points x tj theta rows x ti r rows"""
        _check(load().sph_set_tile(self._h, int(tj), int(ti)), "sph_set_tile")

    KERNELS = ("avg", "coef", "rhs", "sweep_r", "sweep_theta", "sweep_phi")

    def profile(self, enable: bool = True):
        """Start (clear) or stop per-kernel CUDA-event timing inside the library."""
        _check(load().sph_profile(self._h, int(bool(enable))), "sph_profile")

    def profile_read(self):
        """{kernel: (total ms, launches)} recorded since profile(True) (synchronises)."""
        ms = (C.c_double * 8)()
        cnt = (C.c_longlong * 8)()
        _check(load().sph_profile_read(self._h, ms, cnt), "sph_profile_read")
        return {k: (ms[i], cnt[i]) for i, k in enumerate(self.KERNELS)}

    @property
    def launches(self) -> int:
        return int(load().sph_launch_count(self._h))

    def close(self):
        if getattr(self, "_h", None):
            load().sph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Independent solvers stepped together by one CUDA graph (sph_batch_*):
    each solver's steps form a branch on its own stream, so the instances run
    concurrently and no host launch overhead remains per step."""

    def __init__(self, solvers, stream=None):
        import torch
        self.solvers = list(solvers)
        self.stream = stream if stream is not None else torch.cuda.Stream()
        arr = (_CTX * len(self.solvers))(*[s._h for s in self.solvers])
        h = C.c_void_p()
        _check(load().sph_batch_create(arr, len(self.solvers), C.c_void_p(self.stream.cuda_stream), C.byref(h)),
               "sph_batch_create")
        self._h = h
        self.steps = 0

    def capture(self, dt: float, n_iter: int, steps: int = 2, fused: bool = False):
        """Record `steps` steps (even) of every solver into the graph: one branch
        per solver (fused=False), or batched launches over all solvers, one per
        stage and line layout (fused=True, sph_batch_capture_fused)."""
        fn = "sph_batch_capture_fused" if fused else "sph_batch_capture"
        _check(getattr(load(), fn)(self._h, float(dt), int(n_iter), int(steps)), fn)
        self.steps = steps
        self.fused = fused

    def launch(self, times: int = 1):
        _check(load().sph_batch_launch(self._h, int(times)), "sph_batch_launch")

    def status(self):
        """Synchronise; raise SphError for the first failed solver (its index in .bad)."""
        bad = C.c_int(-1)
        code = load().sph_batch_status(self._h, C.byref(bad))
        self.bad = bad.value
        _check(code, f"sph_batch_status (solver {bad.value})")

    def close(self):
        if getattr(self, "_h", None):
            load().sph_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
