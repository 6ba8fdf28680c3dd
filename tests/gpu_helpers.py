"""Shared helpers of the GPU parity tests: run the CUDA library and the oracle on
the same seeded inputs and compare."""
import numpy as np

import paper_2004_13887_gb300 as sph


def rel_err(a, b):
    """max-norm error of a against b, relative to max |b| (per field)."""
    s = float(np.max(np.abs(b)))
    d = float(np.max(np.abs(np.asarray(a) - np.asarray(b))))
    return d / s if s > 0 else d


def to_host(fields):
    return [f.detach().cpu().numpy() for f in fields]


def to_dev(fields):
    import torch
    return [torch.from_numpy(np.array(f, dtype=np.float64, copy=True)).to("cuda") for f in fields]


def solver_for(grid, par, bg=None, state=None, precision=0):
    s = sph.Solver(grid, par, precision=precision)
    if bg is not None:
        s.set_background(bg[0], bg[1])
    if state is not None:
        s.set_state(state)
    return s


def perturbed(fields, scale, seed, grid):
    """fields + scale*noise with the wall-face normal velocity left unchanged"""
    rng = np.random.default_rng(seed)
    out = []
    for q, f in enumerate(fields):
        n = rng.standard_normal(f.shape) * scale[q]
        if q == 1:
            n[0] = n[-1] = 0
        if q == 2:
            n[:, 0] = n[:, -1] = 0
        if q == 3 and not grid.periodic:
            n[:, :, 0] = n[:, :, -1] = 0
        out.append(f + n)
    return out


def physical_fields(U, bg, par):
    """p, rho, theta, T and the velocity components of a state (perturbations +
    the radial background)"""
    p = U[0] + bg[0][1:-1][:, None, None]
    T = U[4] + bg[1][1:-1][:, None, None]
    Rg = par.cv * (par.gamma - 1.0)
    rho = (p + par.pinf) / (Rg * T)
    cp = par.gamma * par.cv
    p00 = float(bg[0][1]) if float(bg[0][1]) > 0 else 1.0
    theta = T * (p00 / p) ** (Rg / cp)
    return {"p": p, "rho": rho, "theta": theta, "T": T, "ur": U[1], "ut": U[2], "up": U[3]}


def l2_rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def velocity_l2(A, B):
    num = sum(np.linalg.norm(A[k] - B[k]) ** 2 for k in ("ur", "ut", "up"))
    den = sum(np.linalg.norm(B[k]) ** 2 for k in ("ur", "ut", "up"))
    return float(np.sqrt(num / max(den, 1e-300)))


def field_errors(U, Uref, bg, par):
    """relative L2 error of p, rho, theta, T and of the velocity (all three
    components together) of U against Uref"""
    A, B = physical_fields(U, bg, par), physical_fields(Uref, bg, par)
    out = {k: l2_rel(A[k], B[k]) for k in ("p", "rho", "theta", "T")}
    out["u"] = velocity_l2(A, B)
    return out
