"""Write inputs/_sector_mms_generated.py: numpy code for the exact fields and the
forcing S = dU/dt + N(U) + G of the sector manufactured solution (seed 20041388),
so that machines without sympy can build the same inputs.

Run:  python -m inputs.gen_sector_mms
"""
from __future__ import annotations

import os

import sympy as sp
from sympy.printing.numpy import NumPyPrinter

from . import cases
from .continuous import operator, r, th, ph, t

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "_sector_mms_generated.py")


def _fn(name, expr, printer):
    subs, (red,) = sp.cse([expr], optimizations="basic")
    lines = [f"def {name}(r, theta, phi, t):"]
    for sym, e in subs:
        lines.append(f"    {printer.doprint(sym)} = {printer.doprint(e)}")
    lines.append(f"    return {printer.doprint(red)}")
    return "\n".join(lines)


def main():
    par = cases.Params(**cases.SECTOR_PAR)
    exprs = cases.sector_mms_exprs(cases.SECTOR_SEED)
    p0 = cases.SECTOR_P0
    T0 = p0 / (par.cv * (par.gamma - 1))
    pert = [exprs[0] - p0, exprs[1], exprs[2], exprs[3], exprs[4] - T0]
    N = operator(*exprs, gamma=par.gamma, cv=par.cv, Pr=par.Pr, mu=par.mu)
    S = [sp.diff(e, t) + n for e, n in zip(exprs, N)]
    pr = NumPyPrinter({"fully_qualified_modules": False, "inline": True})
    names = ["p", "ur", "ut", "up", "T"]
    body = ['"""GENERATED by inputs/gen_sector_mms.py from the sympy definitions in',
            'inputs/cases.py (sector manufactured solution, seed 20041388). Do not edit."""',
            "from numpy import *  # noqa: F401,F403", ""]
    for nm, e in zip(names, pert):
        body += [_fn(f"exact_{nm}", e, pr), ""]
    for nm, e in zip(names, S):
        body += [_fn(f"source_{nm}", e, pr), ""]
    body.append("EXACT = [" + ", ".join(f"exact_{n}" for n in names) + "]")
    body.append("SOURCE = [" + ", ".join(f"source_{n}" for n in names) + "]")
    with open(OUT, "w") as f:
        f.write("\n".join(body) + "\n")
    print("wrote", OUT, os.path.getsize(OUT), "bytes")


if __name__ == "__main__":
    main()
