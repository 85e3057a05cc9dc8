"""Seeded synthetic inputs for the 6-D transport step.

This module holds no arithmetic of the method itself (no transform, derivative,
quadrature, collision, boundary or time-stage code). It only evaluates analytic
initial data and coefficient fields at node coordinates that the caller passes
in, and draws the random numbers those fields use. The CPU oracle and the CUDA
library each compute their own nodes; whoever calls this module hands it the
node arrays of the side it feeds.

Node arrays are 1-D numpy float64 arrays: ``r``, ``theta``, ``phi`` (position)
and ``Theta``, ``Phi`` (momentum direction, measured in the local frame of the
position, Sect. 4.1). Arrays returned for a field F have shape
``[G][Nr][Ntheta][Nphi][NTheta][NPhi]`` (Phi fastest); coefficient fields have
shape ``[G][Nr][Ntheta][Nphi]``.

Workload recipes (the paper measures on analytic problems, not datasets):
  * Gaussian shell in vacuum: F0 = exp(-((r-0.6)/0.1)^2) (1 + 0.5 cos Theta).
  * Seeded smooth field: F0 = sum_{k<=4} sum_{|a|<=3} c_{k,a} 2^-(k+|a|)
    T_k(x_r) m_a(xhat, omega), c ~ N(0,1) from numpy PCG64(seed); m_a runs over
    the monomials of total degree <= 3 in the six Cartesian components of the
    unit position vector xhat and the direction omega (Eqs. omegax-omegaz).
  * Absorber: kappa = 1 + 0.5 sin(theta) cos(phi), eta = kappa exp(-r^2),
    kappa_s = 0.5 (isotropic scattering).
  * Gradient workload: kappa in [0.5, 5] and eta from seeded smooth fields.
  * Batch of uneven problems: N_r in {17,33,65}, angular N in {8,16,24},
    1..24 groups, kappa scale s ~ U[0.1, 100].
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "dt_rule", "unit_position", "direction_cartesian", "gaussian_shell",
    "seeded_smooth", "absorber_fields", "gradient_fields", "inflow_from",
    "batch_problems", "ProblemSpec",
]


def dt_rule(R1: float, R2: float, Nr: int, cfl: float = 0.4) -> float:
    """Time step = cfl x the smallest radial node spacing of the
    Chebyshev-Gauss-Lobatto grid on [R1, R2] (radial Courant limit, Sect. 5.4).
    """
    return cfl * 0.5 * (R2 - R1) * (1.0 - math.cos(math.pi / (Nr - 1)))


def unit_position(theta, phi):
    """xhat = x/r as three arrays broadcast over [theta][phi]."""
    th = np.asarray(theta)[:, None]
    ph = np.asarray(phi)[None, :]
    return (np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th) + 0 * ph)


def direction_cartesian(theta, phi, Theta, Phi):
    """Cartesian components of the momentum direction, Eqs. (omegax)-(omegaz),
    Sect. 4.1, as arrays of shape [Ntheta][Nphi][NTheta][NPhi]."""
    th = np.asarray(theta)[:, None, None, None]
    ph = np.asarray(phi)[None, :, None, None]
    Th = np.asarray(Theta)[None, None, :, None]
    Ph = np.asarray(Phi)[None, None, None, :]
    ox = (np.cos(Th) * np.sin(th) * np.cos(ph) + np.sin(Th) * np.cos(Ph) * np.cos(th) * np.cos(ph)
          - np.sin(Th) * np.sin(Ph) * np.sin(ph))
    oy = (np.cos(Th) * np.sin(th) * np.sin(ph) + np.sin(Th) * np.cos(Ph) * np.cos(th) * np.sin(ph)
          + np.sin(Th) * np.sin(Ph) * np.cos(ph))
    oz = np.cos(Th) * np.cos(th) - np.sin(Th) * np.cos(Ph) * np.sin(th)
    return ox, oy, oz


def gaussian_shell(r, theta, phi, Theta, Phi, r0=0.6, width=0.1, groups=1):
    """F0 = exp(-((r-r0)/width)^2) (1 + 0.5 cos Theta), independent of theta,
    phi, Phi (the vacuum free-streaming workload)."""
    rr = np.asarray(r)[:, None, None, None, None]
    Th = np.asarray(Theta)[None, None, None, :, None]
    f = np.exp(-((rr - r0) / width) ** 2) * (1.0 + 0.5 * np.cos(Th))
    f = np.broadcast_to(f, (len(r), len(theta), len(phi), len(Theta), len(Phi)))
    return np.ascontiguousarray(np.broadcast_to(f, (groups,) + f.shape))


def _monomial_exponents(nvar: int, maxdeg: int):
    out = []
    for deg in range(maxdeg + 1):
        for combo in itertools.combinations_with_replacement(range(nvar), deg):
            e = [0] * nvar
            for v in combo:
                e[v] += 1
            out.append(tuple(e))
    return out


def _cheb_T(k: int, x):
    # T_k(x) = cos(k arccos x) for |x| <= 1: the definition of the input's radial profile.
    return np.cos(k * np.arccos(np.clip(x, -1.0, 1.0)))


def seeded_smooth(r, theta, phi, Theta, Phi, seed: int, R1: float, R2: float,
                  kmax: int = 4, maxdeg: int = 3, with_direction: bool = True):
    """One group of the seeded smooth field: sum_k sum_a c_{k,a} 2^-(k+|a|)
    T_k(x_r) m_a(xhat, omega). Returns [Nr][Nth][Nph][NTh][NPh] (or
    [Nr][Nth][Nph] when ``with_direction`` is False, in which case the
    monomials run over xhat only)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    xr = (2.0 * np.asarray(r) - R1 - R2) / (R2 - R1)
    xh = unit_position(theta, phi)
    if with_direction:
        om = direction_cartesian(theta, phi, Theta, Phi)
        shp = (len(theta), len(phi), len(Theta), len(Phi))
        variables = [np.broadcast_to(v[:, :, None, None], shp) for v in xh] + [om[0], om[1], om[2]]
    else:
        shp = (len(theta), len(phi))
        variables = [np.broadcast_to(v, shp) for v in xh]
    exps = _monomial_exponents(len(variables), maxdeg)
    coef = rng.standard_normal((kmax + 1, len(exps)))
    # powers of each variable up to maxdeg
    pw = [[np.ones(shp)] + [None] * maxdeg for _ in variables]
    for vi, v in enumerate(variables):
        for p in range(1, maxdeg + 1):
            pw[vi][p] = pw[vi][p - 1] * v
    mono = []
    for e in exps:
        m = np.ones(shp)
        for vi, p in enumerate(e):
            if p:
                m = m * pw[vi][p]
        mono.append(m)
    out = np.zeros((len(r),) + shp)
    for k in range(kmax + 1):
        Q = np.zeros(shp)
        for ai, e in enumerate(exps):
            Q += coef[k, ai] * 2.0 ** (-(k + sum(e))) * mono[ai]
        out += _cheb_T(k, xr).reshape((-1,) + (1,) * len(shp)) * Q[None]
    return out


def absorber_fields(r, theta, phi, groups=1, kappa_s=0.5):
    """kappa = 1 + 0.5 sin(theta) cos(phi), eta = kappa exp(-r^2), kappa_s const.
    Returns (kappa, eta, kappa_s), each [G][Nr][Nth][Nph]."""
    rr = np.asarray(r)[:, None, None]
    th = np.asarray(theta)[None, :, None]
    ph = np.asarray(phi)[None, None, :]
    kap = (1.0 + 0.5 * np.sin(th) * np.cos(ph)) + 0.0 * rr
    eta = kap * np.exp(-rr ** 2)
    ks = np.full_like(kap, kappa_s)
    rep = lambda a: np.ascontiguousarray(np.broadcast_to(a, (groups,) + a.shape))
    return rep(kap), rep(eta), rep(ks)


def _normalised(field_):
    lo, hi = field_.min(), field_.max()
    return 2.0 * (field_ - lo) / (hi - lo) - 1.0


def gradient_fields(r, theta, phi, groups, seed, R1, R2, kappa_s=0.5):
    """kappa_g = 0.5 + 4.5 (1 + s_g)/2 and eta_g = kappa_g exp(-r^2)(1 + 0.3 s'_g),
    with s_g, s'_g seeded smooth position-only fields normalised to [-1, 1]
    (so kappa lies in [0.5, 5]). Returns (kappa, eta, kappa_s) [G][Nr][Nth][Nph]."""
    kap = np.empty((groups, len(r), len(theta), len(phi)))
    eta = np.empty_like(kap)
    rr = np.asarray(r)[:, None, None]
    for g in range(groups):
        s = _normalised(seeded_smooth(r, theta, phi, None, None, seed + 1000 + g, R1, R2,
                                      with_direction=False))
        s2 = _normalised(seeded_smooth(r, theta, phi, None, None, seed + 2000 + g, R1, R2,
                                       with_direction=False))
        kap[g] = 0.5 + 4.5 * (1.0 + s) / 2.0
        eta[g] = kap[g] * np.exp(-rr ** 2) * (1.0 + 0.3 * s2)
    return kap, eta, np.full_like(kap, kappa_s)


def nucleon_densities(r, theta, phi, groups, seed, R1, R2):
    """Neutron and proton scattering amplitudes A_n, A_p, each [G][Nr][Nth][Nph]
    (density times the per-nucleon coefficient of the neutrino-nucleon kernels),
    scaled so that 4 pi (A_n + A_p) is of order one: A_n = (0.75 + 0.25 s)/(4 pi),
    A_p = (0.3 + 0.2 s')/(4 pi), with s, s' seeded smooth position-only fields
    normalised to [-1, 1] (proton fraction between about 0.06 and 0.5)."""
    An = np.empty((groups, len(r), len(theta), len(phi)))
    Ap = np.empty_like(An)
    for g in range(groups):
        s = _normalised(seeded_smooth(r, theta, phi, None, None, seed + 3000 + g, R1, R2,
                                      with_direction=False))
        s2 = _normalised(seeded_smooth(r, theta, phi, None, None, seed + 4000 + g, R1, R2,
                                       with_direction=False))
        An[g] = (0.75 + 0.25 * s) / (4 * np.pi)
        Ap[g] = (0.3 + 0.2 * s2) / (4 * np.pi)
    return An, Ap


def signed_field(r, theta, phi, groups, seed, R1, R2):
    """A seeded smooth position-only field normalised to [-1, 1] per group,
    [G][Nr][Nth][Nph] (e.g. a scattering anisotropy covering its whole range)."""
    return np.stack([_normalised(seeded_smooth(r, theta, phi, None, None, seed + 5000 + g, R1, R2,
                                               with_direction=False)) for g in range(groups)])


def lambert_inflow(Theta, Ntheta, Nphi, NPhi, groups=1, F0=1.0):
    """Inflow data of a Lambert emitter at the inner sphere: F(R1) = F0 cos(Theta)
    on the outgoing directions (cos Theta > 0, the first NTheta/2 nodes), nothing
    entering at R2. Returns (g_R1, g_R2), each [G][Ntheta][Nphi][NTheta/2][NPhi]."""
    h = len(Theta) // 2
    c = np.cos(np.asarray(Theta[:h]))[None, None, None, :, None]
    gR1 = np.ascontiguousarray(np.broadcast_to(F0 * c, (groups, Ntheta, Nphi, h, NPhi)))
    return gR1, np.zeros_like(gR1)


def shell_scattering(r, theta, phi, R1, R2, tau, groups=1):
    """Scattering coefficient of the shell plasma n0 [1 + 0.1 r sin(th) cos(ph) cos(th)]
    [1 - (r - R1)/(R2 - R1)]^8 (largest at R1, vanishing at R2), scaled so that
    the radial optical depth of the unmodulated profile, int kappa_s dr, is tau.
    Returns [G][Nr][Nth][Nph]."""
    rr = np.asarray(r)[:, None, None]
    th = np.asarray(theta)[None, :, None]
    ph = np.asarray(phi)[None, None, :]
    k0 = 9.0 * tau / (R2 - R1)
    ks = k0 * (1.0 + 0.1 * rr * np.sin(th) * np.cos(ph) * np.cos(th)) * (1.0 - (rr - R1) / (R2 - R1)) ** 8
    return np.ascontiguousarray(np.broadcast_to(ks, (groups,) + ks.shape))


def inflow_from(F, NTheta):
    """Static inflow data equal to F's own values at the inflow nodes:
    r = R1 for the directions with cos Theta > 0 (the first NTheta/2 Theta
    nodes) and r = R2 for the rest. Returns (g_R1, g_R2), each
    [G][Nth][Nph][NTheta/2][NPhi]."""
    h = NTheta // 2
    return (np.ascontiguousarray(F[:, 0, :, :, :h, :]),
            np.ascontiguousarray(F[:, -1, :, :, h:, :]))


@dataclass
class ProblemSpec:
    Nr: int
    Ntheta: int
    Nphi: int
    NTheta: int
    NPhi: int
    groups: int
    kappa_scale: float
    seed: int
    R1: float = 0.2
    R2: float = 1.0

    @property
    def points(self) -> int:
        return self.Nr * self.Ntheta * self.Nphi * self.NTheta * self.NPhi * self.groups


def batch_problems(n: int = 64, seed: int = 1104):
    """The uneven batch: per problem N_r uniform on {17,33,65}, each angular
    axis independently uniform on {8,16,24}, groups uniform on 1..24, kappa
    scale s ~ U[0.1, 100]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for p in range(n):
        Nr = int(rng.choice([17, 33, 65]))
        ang = [int(v) for v in rng.choice([8, 16, 24], size=4)]
        G = int(rng.integers(1, 25))
        s = float(rng.uniform(0.1, 100.0))
        out.append(ProblemSpec(Nr, ang[0], ang[1], ang[2], ang[3], G, s, seed + 17 * p))
    return out


def batch_fields(spec: ProblemSpec, r, theta, phi):
    """kappa = s (1 + 0.5 sin theta cos phi), eta = kappa exp(-r^2), kappa_s = 0.5
    for every group of one batch problem."""
    kap, eta, ks = absorber_fields(r, theta, phi, groups=spec.groups)
    return spec.kappa_scale * kap, spec.kappa_scale * eta, ks
