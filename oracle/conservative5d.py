"""Plain FP64 CPU oracle of the conservative 5-D formulation (App. A, Eq. Cohercons).

TEST INFRASTRUCTURE ONLY. The tests and the benchmark's CPU leg are the only
callers; the CUDA library never calls this module and this module imports
nothing from the library.

What it computes (Bonazzola, Vasset & Peres 2011, App. A): the transport
equation of Sect. 4.1 multiplied by the phase-space volume element, for the
conservative variable
    Fhat = J F,   J = r^2 sin(th) sin(Th),
in flux form (Eq. Cohercons, every flux written through Fhat):
    dFhat/dt = - [ d_r (cos Th Fhat) + d_th (sin Th cos Ph Fhat / r)
                   + d_ph (sin Th sin Ph Fhat / (r sin th))
                   - d_Th (sin Th Fhat / r) - d_Ph (sin Th sin Ph cot th Fhat / r) ]
               + J CT(Fhat / J)
with CT the collision term of the plain form (absorption, emission and the
scattering kernels (kappa_s/4pi)(1 + b mu + c (mu^2 - 1/3))). Integrated over
the shell it gives the number balance dN/dt + J_R2 - J_R1 = S (Eq. Cons), S the
integral of J (eta - kappa F) (zero for pure scattering), N = int Fhat (Eq. Npho)
and J_R = int cos Th Fhat(R) (Eq. Flux).

Readings taken here:
  * r: the radial velocity cos Th does not depend on r: cos Th D_r Fhat with the
    plain form's coefficient-space Chebyshev derivative.
  * th, ph: their velocities do not depend on th (resp. ph): velocity x the
    derivative of Fhat. Fhat carries sin th, so on the double-Fourier-sphere
    doubled th circle the reflected node holds MINUS Fhat at the partner
    (ph + pi, Ph + pi) (F itself is continued with a plus sign).
  * Th: d_Th(sin Th Fhat) taken as sin Th D_Th Fhat + cos Th P Fhat, with D_Th on
    the odd continuation (minus Fhat at the partner Ph + pi) and P the removal
    of the Nyquist bin of the doubled Th circle (the reading the 2-D
    conservative variant takes for its Theta term: its Fejer integral then
    vanishes for every Fhat).
  * Ph: the flux itself is differentiated, D_Ph(sin Ph Fhat) (periodic, Nyquist
    bin zeroed); the trapezoid sum of a periodic derivative is zero.
  * Collision: J CT(F) at F = Fhat / J.
  * Boundaries: the plain form's Tau rows (an inflow node's rate of Fhat is J
    times that of F, so both vanish together); inflow data are values of Fhat.
  * Quadrature of N: Clenshaw-Curtis in r; int_0^pi h dth of h = sin th g by
    Fejer's first rule on h / sin th (and the same in Th); trapezoid in ph, Ph.
  * Time: classical RK4 or the paper's AB2 (as in the plain form).
Discrete balance: the r term integrates to J_R2 - J_R1 exactly (Clenshaw-
Curtis integrates the degree N_r - 2 derivative exactly), the ph and Ph terms to
zero (trapezoid sums of periodic derivatives), the Th term to zero (the
projection), the scattering gain to its loss (the same quadrature); the th term
is left: the odd continuation's derivative is a cosine series for Fourier modes
with m + M even, and the Fejer-based rule does not integrate those exactly, so
the balance error is the th term's integral, spectrally small for resolved data.
"""
from __future__ import annotations

import numpy as np

from .transport import AX_PH, AX_R, AX_TH, AX_TPH, AX_TTH, Grid, Problem


def jacobian(g):
    """r^2 sin(th) sin(Th), broadcastable against [G][Nr][Nth][Nph][NTh][NPh]."""
    r = g.r.reshape(1, -1, 1, 1, 1, 1)
    th = g.theta.reshape(1, 1, -1, 1, 1, 1)
    Th = g.Theta.reshape(1, 1, 1, 1, -1, 1)
    return r ** 2 * np.sin(th) * np.sin(Th)


def d_th_odd(g, Fh):
    """d/dth on the doubled th circle, the reflected node carrying -Fhat at the
    partner (ph + pi, Ph + pi)."""
    ext = g._extend(Fh, AX_TH, -g._partner_th(Fh))
    return np.take(g._fourier_deriv(ext, AX_TH), np.arange(g.Nt), axis=AX_TH)


def d_Th_odd(g, Fh):
    """d/dTh on the doubled Th circle, the reflected node carrying -Fhat at Ph + pi."""
    ext = g._extend(Fh, AX_TTH, -g._partner_Th(Fh))
    return np.take(g._fourier_deriv(ext, AX_TTH), np.arange(g.NT), axis=AX_TTH)


def nyquist_free_Th(g, Fh):
    """Fhat without the Nyquist bin of its odd continuation on the doubled Th circle."""
    ext = g._extend(Fh, AX_TTH, -g._partner_Th(Fh))
    c = np.fft.fft(ext, axis=AX_TTH)
    idx = [slice(None)] * c.ndim
    idx[AX_TTH] = g.NT
    c[tuple(idx)] = 0.0
    return np.take(np.real(np.fft.ifft(c, axis=AX_TTH)), np.arange(g.NT), axis=AX_TTH)


def liouville_terms(g, Fh):
    """The five flux derivatives of Eq. Cohercons, in the order r, th, ph, Th, Ph."""
    r = g.r.reshape(1, -1, 1, 1, 1, 1)
    th = g.theta.reshape(1, 1, -1, 1, 1, 1)
    Th = g.Theta.reshape(1, 1, 1, 1, -1, 1)
    Ph = g.Phi.reshape(1, 1, 1, 1, 1, -1)
    sT, cT = np.sin(Th), np.cos(Th)
    t_r = cT * g.d_r(Fh)
    t_th = sT * np.cos(Ph) / r * d_th_odd(g, Fh)
    t_ph = sT * np.sin(Ph) / (r * np.sin(th)) * g.d_ph(Fh)
    t_Th = -(sT * d_Th_odd(g, Fh) + cT * nyquist_free_Th(g, Fh)) / r
    t_Ph = -sT * np.cos(th) / (np.sin(th) * r) * g.d_Ph(np.sin(Ph) * Fh)
    return t_r, t_th, t_ph, t_Th, t_Ph


def liouville_hat(g, Fh):
    """The flux-form streaming operator applied to Fhat (the sum of the five terms)."""
    return sum(liouville_terms(g, Fh))


def hat_weights(g):
    """Weights W with N = sum W Fhat over [Nr][Nth][Nph][NTh][NPh] (Eq. Npho on
    Fhat), and the surface weights w_s with J_R = sum w_s cos Th Fhat(R) over
    [Nth][Nph][NTh][NPh] (Eq. Flux)."""
    wr = g.clenshaw_curtis_r(np.eye(g.Nr), axis=1)
    wt = g.fejer_integral(np.eye(g.Nt), 1) / np.sin(g.theta)
    wT = g.fejer_integral(np.eye(g.NT), 1) / np.sin(g.Theta)
    wp = np.full(g.Np, 2 * np.pi / g.Np)
    wP = np.full(g.NP, 2 * np.pi / g.NP)
    ws = np.einsum("j,l,k,m->jlkm", wt, wp, wT, wP)
    return np.einsum("i,jlkm->ijlkm", wr, ws), ws


class ConservativeProblem(Problem):
    """The flux form on the Chebyshev grid; state Fhat. Same coefficients,
    kernels, inflow handling and schemes (RK4, AB2) as the plain Problem."""

    def __init__(self, grid, *args, **kw):
        if type(grid) is not Grid:
            raise ValueError("the conservative form runs on the Chebyshev radial grid")
        super().__init__(grid, *args, **kw)
        if self.scheme not in ("rk4", "ab2") or self.filter_on:
            raise ValueError("the conservative form steps with RK4 or AB2, unfiltered")
        self.jac = jacobian(grid)

    def to_hat(self, F):
        return self.jac * F

    def from_hat(self, Fh):
        return Fh / self.jac

    def collision(self, Fh):
        """J CT(F) at F = Fhat / J (the last line of Eq. Cohercons, with the
        absorption and emission of the plain form)."""
        return self.jac * Problem.collision(self, Fh / self.jac)

    def rhs(self, Fh, streaming_only=False):
        K = -liouville_hat(self.g, Fh)
        if not streaming_only:
            K = K + self.collision(Fh)
        if self.bc == "tau":
            K = self.g.tau(K)
        return K

    # ---------------------------------------------------------- number balance
    def number(self, Fh):
        W, _ = hat_weights(self.g)
        return np.einsum("gijlkm,ijlkm->g", Fh, W)

    def fluxes(self, Fh):
        _, ws = hat_weights(self.g)
        cT = np.cos(self.g.Theta)[None, None, :, None]
        J1 = np.einsum("gjlkm,jlkm->g", Fh[:, 0], ws * cT)
        J2 = np.einsum("gjlkm,jlkm->g", Fh[:, -1], ws * cT)
        return J1, J2

    def source(self, Fh):
        """S = int J (eta - kappa F): the non-conservative part of the collision."""
        return self.number(self.jac * self._c(self.eta) - self._c(self.kappa) * Fh)

    def balance(self, Fh):
        """(N, J_R1, J_R2, dN/dt, S) per group, dN/dt from the operator without
        Tau rows."""
        saved, self.bc = self.bc, "none"
        try:
            K = self.rhs(Fh)
        finally:
            self.bc = saved
        J1, J2 = self.fluxes(Fh)
        return self.number(Fh), J1, J2, self.number(K), self.source(Fh)

    def balance_residual(self, Fh):
        N, J1, J2, dN, S = self.balance(Fh)
        return dN + J2 - J1 - S


def plain_balance(pr, F):
    """(N, J_R1, J_R2, dN/dt, S) of the plain form with the plain quadrature
    (ts_moments' rules: r^2 dr, Fejer in cos th and cos Th), dN/dt from the
    operator without Tau rows."""
    g = pr.g
    saved, pr.bc = pr.bc, "none"
    try:
        K = pr.rhs(F)
    finally:
        pr.bc = saved
    _, _, N, J1, J2 = g.moments(F)
    dN = g.moments(K)[2]
    S = g.moments(pr._c(pr.eta) - pr._c(pr.kappa) * F)[2]
    return N, J1, J2, dN, S
