"""Continuous right-hand side of the non-conservative system, eqs.
(nonconservmass)-(nonconserveos), evaluated symbolically through CARTESIAN
coordinates.

This is deliberately independent of the spherical-component formulas of
Appendix B: the spherical velocity is mapped to Cartesian components, every
derivative is taken by the chain rule in x, y, z, the stress divergence is
formed as div(sigma) of the full tensor (no vector-Laplacian identity), and the
momentum residual is projected back on e_r, e_theta, e_phi.  Tests use it to pin
the discrete operators (their sum must converge to it at second order) and to
build manufactured-solution sources.  Requires sympy (CPU side only).

Sign convention: the PDE is dU/dt + N(U) + G = S, with G = [0, g, 0, 0, 0]
(gravity g along e_r, added on the left as in eq. nonconservmom) and the
Coriolis term 2 omega x u for a rotation omega about the polar axis.
"""
from __future__ import annotations

import sympy as sp

r, th, ph, t = sp.symbols("r theta phi t", real=True, positive=True)


def _basis():
    st, ct, sp_, cp_ = sp.sin(th), sp.cos(th), sp.sin(ph), sp.cos(ph)
    e_r = (st * cp_, st * sp_, ct)
    e_t = (ct * cp_, ct * sp_, -st)
    e_p = (-sp_, cp_, sp.Integer(0))
    # d q_b / d x_a for q = (r, theta, phi)
    J = [
        [st * cp_, st * sp_, ct],
        [ct * cp_ / r, ct * sp_ / r, -st / r],
        [-sp_ / (r * st), cp_ / (r * st), sp.Integer(0)],
    ]
    return e_r, e_t, e_p, J


def operator(p, ur, ut, up, T, gamma, cv, Pr, mu, pinf=0, g=0, omega=0):
    """Return [N_p, N_ur, N_ut, N_up, N_T] + G as sympy expressions in (r, theta, phi)."""
    e_r, e_t, e_p, J = _basis()
    q = (r, th, ph)

    def D(f, a):  # d f / d x_a
        return sum(J[b][a] * sp.diff(f, q[b]) for b in range(3))

    U = [ur * e_r[a] + ut * e_t[a] + up * e_p[a] for a in range(3)]
    L = [[D(U[b], a) for b in range(3)] for a in range(3)]          # L[a][b] = dU_b/dx_a
    div = L[0][0] + L[1][1] + L[2][2]
    sig = [[mu * (L[a][b] + L[b][a] - sp.Rational(2, 3) * div * (1 if a == b else 0))
            for b in range(3)] for a in range(3)]
    divsig = [sum(D(sig[a][b], a) for a in range(3)) for b in range(3)]
    phi_visc = sum(L[a][b] * sig[a][b] for a in range(3) for b in range(3))
    kappa = mu * gamma * cv / Pr
    lapT = sum(D(D(T, a), a) for a in range(3))
    rho = (p + pinf) / (cv * (gamma - 1) * T)
    adv = lambda f: sum(U[a] * D(f, a) for a in range(3))
    # rotation about the polar axis: omega * e_z
    om = (0, 0, omega)
    cor = [2 * (om[1] * U[2] - om[2] * U[1]), 2 * (om[2] * U[0] - om[0] * U[2]),
           2 * (om[0] * U[1] - om[1] * U[0])]
    mom = [adv(U[b]) + D(p, b) / rho - divsig[b] / rho + g * e_r[b] + cor[b] for b in range(3)]
    Np = adv(p) + gamma * (p + pinf) * div - (gamma - 1) * kappa * lapT - (gamma - 1) * phi_visc
    NT = adv(T) + (gamma - 1) * T * div - (gamma - 1) * T / (p + pinf) * (kappa * lapT + phi_visc)
    Nr = sum(mom[b] * e_r[b] for b in range(3))
    Nt = sum(mom[b] * e_t[b] for b in range(3))
    Nph = sum(mom[b] * e_p[b] for b in range(3))
    return [Np, Nr, Nt, Nph, NT]


def lambdify(exprs, with_t=False):
    """numpy callables f(R, TH, PH[, t]) for a list of expressions (common subexpressions shared)."""
    args = (r, th, ph, t) if with_t else (r, th, ph)
    fns = []
    for e in exprs:
        fns.append(sp.lambdify(args, e, modules="numpy", cse=True))
    return fns
