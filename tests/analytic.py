"""Closed-form test functions built with SymPy (independent of the oracle).

Functions are written as polynomials in the Cartesian position (x, y, z) and
direction (wx, wy, wz), then mapped into the doubly spherical coordinates of
Sect. 4.1 (position r, theta, phi; direction Theta, Phi measured in the local
frame, Eqs. omegax-omegaz). SymPy differentiates them symbolically, so the
expected values share no arithmetic with the oracle's spectral derivatives.
"""
from __future__ import annotations

import functools

import numpy as np
import sympy as sp

r, th, ph, Th, Ph = sp.symbols("r theta phi Theta Phi", real=True)
x, y, z, wx, wy, wz = sp.symbols("x y z wx wy wz", real=True)

SPH = {
    x: r * sp.sin(th) * sp.cos(ph),
    y: r * sp.sin(th) * sp.sin(ph),
    z: r * sp.cos(th),
    wx: sp.cos(Th) * sp.sin(th) * sp.cos(ph) + sp.sin(Th) * sp.cos(Ph) * sp.cos(th) * sp.cos(ph)
        - sp.sin(Th) * sp.sin(Ph) * sp.sin(ph),
    wy: sp.cos(Th) * sp.sin(th) * sp.sin(ph) + sp.sin(Th) * sp.cos(Ph) * sp.cos(th) * sp.sin(ph)
        + sp.sin(Th) * sp.sin(Ph) * sp.cos(ph),
    wz: sp.cos(Th) * sp.cos(th) - sp.sin(Th) * sp.cos(Ph) * sp.sin(th),
}

ARGS = (r, th, ph, Th, Ph)


def _lam(expr):
    f = sp.lambdify(ARGS, expr, "numpy")
    return f


def on_grid(expr, grid, groups=1):
    """Evaluate a SymPy expression in (r, th, ph, Th, Ph) on a grid's nodes,
    returning [G][Nr][Nth][Nph][NTh][NPh]."""
    f = _lam(expr)
    R, T, P, TT, PP = np.meshgrid(grid.r, grid.theta, grid.phi, grid.Theta, grid.Phi, indexing="ij")
    v = np.broadcast_to(np.asarray(f(R, T, P, TT, PP), dtype=np.float64), R.shape)
    return np.ascontiguousarray(np.broadcast_to(v, (groups,) + R.shape))


@functools.lru_cache(maxsize=None)
def cartesian_case(name):
    """(F, omega.grad F) as spherical SymPy expressions for a Cartesian polynomial."""
    P = CASES[name]
    adv = wx * sp.diff(P, x) + wy * sp.diff(P, y) + wz * sp.diff(P, z)
    return P.subs(SPH), adv.subs(SPH)


CASES = {
    "x": x,
    "z": z,
    "wx": wx,
    "wy*wz": wy * wz,
    "xy+wz": x * y + wz,
    "x*wy-z^2": x * wy - z ** 2,
    "cubic": x * y * wz + z ** 2 * wx - 0.5 * y * wy ** 2 + 0.25 * x ** 3,
    "iso4": (1 + 2 * wx + wy + wz / 2) ** 4,
}


def spherical_derivatives(expr):
    """Symbolic d/dr, d/dth, d/dph, d/dTh, d/dPh of a spherical expression."""
    return [sp.diff(expr, v) for v in ARGS]
