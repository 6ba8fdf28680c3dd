"""Block-tridiagonal lines split across ranks: the partitioned (Schur-complement)
block Thomas algorithm of Section 2.2, the way the paper solves a line whose
cells belong to several subdomains.

Every rank holds m >= 2 consecutive blocks of each line.  The arithmetic runs
in the library's kernels (sph_schur_local, sph_schur_reduced, sph_schur_back,
include/sph.h); this module orders them around the one exchange the algorithm
needs -- an all-gather of each rank's interface rows (42 values per line) --
and allocates the caller-side buffers with torch:

1. local: y, V, W with x = y - V x_left - W x_right on the rank's segment;
2. all-gather of (V_0, V_{m-1}, W_0, W_{m-1}, y_0, y_{m-1}) from every rank;
3. every rank solves the same 6P x 6P reduced system of the ranks' first and
   last blocks (cyclic when the line is);
4. back-substitution with the neighbours' boundary blocks.

`ops` carries the three arithmetic steps, so the communication order can be
exercised with any implementation of them (the tests run it on CPU ranks with
a plain reference of the same steps); the default is the CUDA library.
"""
from __future__ import annotations

import ctypes as C

IFACE = 42


class CudaOps:
    """The three steps on the GPU through the C ABI (torch float64 CUDA tensors)."""

    def _ptr(self, t):
        from . import _DP
        return C.cast(C.c_void_p(t.data_ptr()), _DP)

    def _stream(self, t):
        import torch
        return C.c_void_p(torch.cuda.current_stream(t.device).cuda_stream)

    def local(self, A, B, Cb, d):
        import torch
        from . import _check, load
        nl, m = int(B.shape[0]), int(B.shape[1])
        dev = B.device
        scr = torch.empty(30 * nl * m, dtype=torch.float64, device=dev)
        Y = torch.empty((nl, m, 3), dtype=torch.float64, device=dev)
        V = torch.empty((nl, m, 3, 3), dtype=torch.float64, device=dev)
        W = torch.empty((nl, m, 3, 3), dtype=torch.float64, device=dev)
        flag = torch.zeros(1, dtype=torch.int32, device=dev)
        keep = [t.contiguous() for t in (A, B, Cb, d)]   # alive until the call returns
        p = [self._ptr(t) for t in keep]
        _check(load().sph_schur_local(nl, m, *p, self._ptr(scr), self._ptr(Y), self._ptr(V), self._ptr(W),
                                      C.cast(C.c_void_p(flag.data_ptr()), C.POINTER(C.c_int)), self._stream(B)),
               "sph_schur_local")
        return Y, V, W

    def reduced(self, iface, cyclic):
        import torch
        from . import _check, load
        P, nl = int(iface.shape[0]), int(iface.shape[1])
        z = torch.empty((nl, 2 * P, 3), dtype=torch.float64, device=iface.device)
        flag = torch.zeros(1, dtype=torch.int32, device=iface.device)
        iface = iface.contiguous()
        _check(load().sph_schur_reduced(nl, P, int(bool(cyclic)), self._ptr(iface), self._ptr(z),
                                        C.cast(C.c_void_p(flag.data_ptr()), C.POINTER(C.c_int)),
                                        self._stream(iface)), "sph_schur_reduced")
        return z

    def back(self, Y, V, W, xl, xr):
        import torch
        from . import _check, load
        nl, m = int(Y.shape[0]), int(Y.shape[1])
        x = torch.empty_like(Y)
        # the contiguous copies of the neighbour blocks must stay alive until the
        # kernel has run: a copy freed at once could be handed to the next one
        xl, xr = xl.contiguous(), xr.contiguous()
        _check(load().sph_schur_back(nl, m, self._ptr(Y), self._ptr(V), self._ptr(W), self._ptr(xl),
                                     self._ptr(xr), self._ptr(x), self._stream(Y)), "sph_schur_back")
        torch.cuda.current_stream(Y.device).synchronize()
        return x


def interface_rows(Y, V, W):
    """the 42 values per line a rank contributes to the reduced system"""
    import torch
    nl = Y.shape[0]
    return torch.cat([V[:, 0].reshape(nl, 9), V[:, -1].reshape(nl, 9), W[:, 0].reshape(nl, 9),
                      W[:, -1].reshape(nl, 9), Y[:, 0], Y[:, -1]], dim=1)


def neighbour_blocks(z, rank, world, cyclic):
    """(x_left, x_right): rank-1's last block and rank+1's first block from the
    reduced solution z (nlines, 2P, 3), zero past a walled end"""
    import torch
    nl = z.shape[0]
    zero = torch.zeros((nl, 3), dtype=z.dtype, device=z.device)
    if rank > 0 or cyclic:
        xl = z[:, 2 * ((rank - 1) % world) + 1]
    else:
        xl = zero
    if rank < world - 1 or cyclic:
        xr = z[:, 2 * ((rank + 1) % world)]
    else:
        xr = zero
    return xl, xr


def solve(A, B, Cb, d, group=None, cyclic: bool = False, ops=None):
    """This rank's part x of the solution of the lines (shapes of d), the
    segments of all ranks in rank order forming the whole lines."""
    import torch
    import torch.distributed as dist
    ops = ops or CudaOps()
    world = dist.get_world_size(group) if dist.is_initialized() else 1
    rank = dist.get_rank(group) if dist.is_initialized() else 0
    Y, V, W = ops.local(A, B, Cb, d)
    mine = interface_rows(Y, V, W).contiguous()
    if world > 1:
        got = [torch.empty_like(mine) for _ in range(world)]
        dist.all_gather(got, mine, group=group)
    else:
        got = [mine]
    z = ops.reduced(torch.stack(got), cyclic)
    xl, xr = neighbour_blocks(z, rank, world, cyclic)
    return ops.back(Y, V, W, xl, xr)
