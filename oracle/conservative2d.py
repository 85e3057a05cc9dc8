"""Plain FP64 CPU oracle of the conservative 2-D (r, Theta) formulation of App. B.

TEST INFRASTRUCTURE ONLY. The tests and the benchmark's CPU leg are the only
callers; the CUDA library never calls this module and this module imports
nothing from the library.

What it computes (Bonazzola, Vasset & Peres 2011, App. A and App. B): the
spherically symmetric problem F(r, Theta, t) with coherent scattering, written
for the conservative variable (Eq. flux of App. B)
    Fhat(r, Theta, t) = r^2 sin(Theta) F(r, Theta, t),
    dFhat/dt = - cos(Th) dFhat/dr + (1/r) ( sin(Th) dFhat/dTh + cos(Th) Fhat )
               + kappa_s [ - Fhat + sin(Th) int_0^pi k_c(Th, Th') Fhat(Th') dTh' ]   (Eq. speccons)
where k_c is the Phi'-average of the scattering kernel (kappa_s/4pi)(1 + c (mu^2 - 1/3)):
    k_c(Th, Th') = (1/2) (1 + c (cos^2 Th cos^2 Th' + (1/2) sin^2 Th sin^2 Th' - 1/3)),
which for Thomson scattering (c = 3/4) is the (3/8)(1 + (cos Th cos Th')^2 +
(1/2)(sin Th sin Th')^2) of Eq. speccons; c = 0 is isotropic scattering.
Alongside, the plain form of the same problem (the 2-D reduction of the
Liouville operator, Eq. Sphersy, with the same source):
    dF/dt = - cos(Th) dF/dr + (sin(Th)/r) dF/dTh + kappa_s [ - F + int_0^pi k_c F(Th') sin Th' dTh' ].

Number and fluxes of a spherically symmetric F (App. A, Eqs. Npho and Flux,
the theta, phi and Phi integrals done: 4 pi x 2 pi):
    N = 8 pi^2 int dr int dTh Fhat = 8 pi^2 int r^2 dr int sin Th dTh F,
    J_R = 8 pi^2 int cos Th Fhat(R, Th) dTh,    dN/dt + J_R2 - J_R1 = 0 (Eq. Cons).

Readings (the same as the 5-D oracle where they overlap):
  * r: Chebyshev-Gauss-Lobatto nodes; d/dr in coefficient space (values ->
    coefficients -> derivative recurrence -> values).
  * Theta: pole-free nodes pi (k+1/2)/N, N even. F is even under the
    reflection Th -> -Th of the doubled circle, Fhat (with its sin Th factor)
    odd: the reflected node carries +F, respectively -Fhat. Fourier derivative
    on the doubled circle, Nyquist mode zeroed.
  * int_0^pi g(Th) sin Th dTh by Fejer's first rule (weights w_k); int_0^pi h dTh
    of an odd-extended h = sin(Th) g by the same rule applied to h / sin Th.
    Radial integrals: Clenshaw-Curtis.
  * Conservative Theta term: sin(Th) dFhat/dTh + cos(Th) Fhat with the
    Nyquist sine mode of Fhat left out of the second product (the derivative
    zeroes it in the first). The Fejer integral of that term then vanishes for
    every Fhat, and with the radial flux (Clenshaw-Curtis integrates dFhat/dr
    exactly) and the scattering term (its gain integrates to its loss) the
    discrete number balance holds to rounding. Without the projection the
    balance error is the Nyquist mode's, small for resolved data -- the paper
    reports a Theta balance error that falls exponentially with N_Theta.
  * Boundaries: Tau inflow rows on every stage derivative (inflow at R1 where
    cos Th > 0, at R2 where cos Th < 0) or none (operator and balance tests).
  * Time: classical RK4.
  * Three-zone radial grid (App. B, optional): the r derivative and radial
    integrals of the 5-D oracle's three-zone grid (first-order upwind edge
    zones, a Chebyshev central zone joined by the interface Tau correction,
    trapezoid + Clenshaw-Curtis); the outer inflow nodes hold their data (zero
    rate) in place of the Tau rows. The number balance is then exact only up to
    the edge zones' first-order differences.
The paper's own 2-D solver advances the radial term implicitly with a per-angle
optimal step; that time scheme is out of scope here (the conservative variable
and its discrete balance are built).
"""
from __future__ import annotations

import numpy as np

from .transport import Grid as _Grid5, GridZonedR as _GridZ5


def _fejer(N):
    """Fejer's first rule for int_0^pi g(t) sin t dt on t_k = pi (k+1/2)/N."""
    t = np.pi * (np.arange(N) + 0.5) / N
    m = np.arange(1, N // 2 + 1)
    s = (np.cos(2.0 * np.outer(t, m)) / (4.0 * m * m - 1.0)).sum(axis=1)
    return 2.0 / N * (1.0 - 2.0 * s)


class Grid2D:
    """Nodes, derivatives and quadratures of the (r, Theta) grid."""

    def __init__(self, R1, R2, Nr, NTheta, zone_nodes=0, zone_width=0.0):
        if Nr < 3 or NTheta % 2 or NTheta < 2:
            raise ValueError("need Nr >= 3 and an even NTheta")
        # the radial machinery of the 5-D oracle (coefficient-space Chebyshev)
        self._g5 = _Grid5(R1, R2, Nr, 2, 2, NTheta, 2)
        self.R1, self.R2, self.Nr, self.NT = float(R1), float(R2), Nr, NTheta
        self.r = self._g5.r
        # three-zone radial grid: the 5-D oracle's zoned grid on the same Theta nodes
        self.zoned = zone_nodes > 0
        self._gz = (_GridZ5(R1, R2, Nr, 2, 2, NTheta, 2, zone_nodes=zone_nodes,
                            zone_width=zone_width) if self.zoned else None)
        self.Theta = np.pi * (np.arange(NTheta) + 0.5) / NTheta
        self.wF = _fejer(NTheta)                      # int g sin Th dTh
        # Clenshaw-Curtis weights on the Gauss-Lobatto nodes (int dr): the
        # integral of the Chebyshev interpolant, c_k int T_k
        k = np.arange(Nr)
        ints = np.zeros(Nr)
        ev = k % 2 == 0
        ints[ev] = 2.0 / (1.0 - k[ev].astype(float) ** 2)   # int_{-1}^{1} T_k dx
        self.wr = (ints @ self._g5.cheb_S) * 0.5 * (R2 - R1)
        if self.zoned:
            self.r = self._gz.r
            self.wr = self._gz.clenshaw_curtis_r(np.eye(Nr), axis=1)

    # -------------------------------------------------------------- derivatives
    def d_r(self, F):
        """d/dr along axis 1 of [P][Nr][NT] (on the three-zone grid: per
        direction, each zone's rate taken from the direction's upstream side)."""
        if self.zoned:
            F6 = np.ascontiguousarray(np.broadcast_to(F[:, :, None, None, :, None],
                                                      (F.shape[0], self.Nr, 2, 2, self.NT, 2)))
            return self._gz.d_r_zoned(F6)[:, :, 0, 0, :, 0]
        c = np.tensordot(self._g5.cheb_S, F, axes=([1], [1]))
        c = np.tensordot(self._g5.cheb_C, c, axes=([1], [0]))
        return np.moveaxis(np.tensordot(self._g5.cheb_V, c, axes=([1], [0])), 0, 1)

    def d_Theta(self, F, parity):
        """d/dTh along axis 2 on the doubled circle: the node 2N-1-k carries
        parity * F(Th_k) (+1: even functions such as F, -1: odd ones such as Fhat)."""
        ext = np.concatenate([F, parity * np.flip(F, axis=2)], axis=2)
        M = ext.shape[2]
        kk = np.fft.fftfreq(M, d=1.0 / M)
        mult = 1j * kk
        mult[M // 2] = 0.0
        d = np.real(np.fft.ifft(np.fft.fft(ext, axis=2) * mult, axis=2))
        return d[:, :, :self.NT]

    def nyquist_free(self, Fh):
        """Fhat without its Nyquist component sin(NT Th) (on the doubled circle
        of an odd function: the alternating pattern of the Nyquist bin)."""
        ext = np.concatenate([Fh, -np.flip(Fh, axis=2)], axis=2)
        c = np.fft.fft(ext, axis=2)
        c[:, :, self.NT] = 0.0
        return np.real(np.fft.ifft(c, axis=2))[:, :, :self.NT]

    # -------------------------------------------------------------- quadratures
    def int_Theta_sin(self, g):
        """int_0^pi g sin Th dTh along the last axis (Fejer)."""
        return np.tensordot(g, self.wF, axes=([-1], [0]))

    def int_Theta_hat(self, h):
        """int_0^pi h dTh of an odd-extended h = sin Th g (Fejer on h / sin Th)."""
        return np.tensordot(h, self.wF / np.sin(self.Theta), axes=([-1], [0]))

    def int_r(self, f):
        """int_R1^R2 f dr along axis 1 (Clenshaw-Curtis)."""
        return np.tensordot(f, self.wr, axes=([1], [0]))

    def inflow_node(self):
        """Radial index of the inflow node of each Theta (R1 where cos Th > 0)."""
        return np.where(np.cos(self.Theta) > 0, 0, self.Nr - 1)


class Problem2D:
    """The conservative (form="hat", unknown Fhat) or plain (form="plain",
    unknown F) 2-D problem with scattering coefficient kappa_s(r) per problem
    ([P][Nr]) and kernel parameter c; bc "tau" or "none"."""

    def __init__(self, grid, kappa_s, c=0.75, form="hat", bc="tau"):
        if form not in ("hat", "plain") or bc not in ("tau", "none"):
            raise ValueError((form, bc))
        self.g, self.form, self.bc, self.c = grid, form, bc, float(c)
        self.ks = np.asarray(kappa_s, dtype=np.float64)[:, :, None]

    def _kernel(self):
        """k_c(Th_k, Th_k') as an [NT][NT] matrix."""
        ct, st = np.cos(self.g.Theta), np.sin(self.g.Theta)
        return 0.5 * (1.0 + self.c * (np.outer(ct ** 2, ct ** 2) + 0.5 * np.outer(st ** 2, st ** 2)
                                      - 1.0 / 3.0))

    def streaming(self, X):
        g = self.g
        r = g.r[None, :, None]
        ct, st = np.cos(g.Theta)[None, None, :], np.sin(g.Theta)[None, None, :]
        if self.form == "hat":
            # the Theta term on the Nyquist-free band (the derivative drops the
            # Nyquist mode already; the cos(Th) Fhat term drops it here), so that
            # its Fejer integral vanishes for every Fhat
            return -ct * g.d_r(X) + (st * g.d_Theta(X, -1.0) + ct * g.nyquist_free(X)) / r
        return -ct * g.d_r(X) + st / r * g.d_Theta(X, +1.0)

    def scattering(self, X):
        g = self.g
        K = self._kernel()
        st = np.sin(g.Theta)
        if self.form == "hat":
            # int_0^pi k_c(Th, Th') Fhat(Th') dTh' (Fhat / sin Th' under Fejer)
            gain = st[None, None, :] * np.tensordot(X / st, K * g.wF[None, :], axes=([2], [1]))
        else:
            gain = np.tensordot(X, K * g.wF[None, :], axes=([2], [1]))
        return self.ks * (gain - X)

    def tau(self, K, gdot=0.0):
        """Replace the top Chebyshev coefficient of each Theta column so that the
        rate at its inflow node is gdot (zero for static inflow data)."""
        g = self.g
        if self.bc == "none":
            return K
        if g.zoned:   # three-zone grid: the outer inflow nodes hold their data
            out = K.copy()
            b = g.inflow_node()
            for k in range(g.NT):
                out[:, b[k], k] = gdot
            return out
        N = g.Nr - 1
        tN = np.cos(np.pi * (N - np.arange(g.Nr)))     # T_N(x_i) on the Gauss-Lobatto nodes
        b = g.inflow_node()
        out = K.copy()
        for k in range(g.NT):
            alpha = (gdot - K[:, b[k], k]) / tN[b[k]]
            out[:, :, k] += alpha[:, None] * tN[None, :]
        return out

    def rhs(self, X):
        return self.tau(self.streaming(X) + self.scattering(X))

    def rk4_step(self, X, dt, stages=None):
        K1 = self.rhs(X)
        K2 = self.rhs(X + 0.5 * dt * K1)
        K3 = self.rhs(X + 0.5 * dt * K2)
        U4 = X + dt * K3
        K4 = self.rhs(U4)
        if stages is not None:
            stages.extend([X, X + 0.5 * dt * K1, X + 0.5 * dt * K2, U4])
        return X + dt / 6.0 * (K1 + 2 * K2 + 2 * K3 + K4)

    def run(self, X, dt, nsteps):
        for _ in range(nsteps):
            X = self.rk4_step(X, dt)
        return X

    # ------------------------------------------------------------- balances
    def number(self, X):
        """N per problem (Eq. Npho)."""
        g = self.g
        if self.form == "hat":
            return 8 * np.pi ** 2 * g.int_r(g.int_Theta_hat(X))
        return 8 * np.pi ** 2 * g.int_r(g.r[None, :] ** 2 * g.int_Theta_sin(X))

    def fluxes(self, X):
        """(J_R1, J_R2) per problem (Eq. Flux)."""
        g = self.g
        ct = np.cos(g.Theta)
        if self.form == "hat":
            J = [8 * np.pi ** 2 * g.int_Theta_hat(ct * X[:, i]) for i in (0, -1)]
        else:
            J = [8 * np.pi ** 2 * R ** 2 * g.int_Theta_sin(ct * X[:, i])
                 for i, R in ((0, g.R1), (-1, g.R2))]
        return J[0], J[1]

    def balance_residual(self, X):
        """dN/dt + J_R2 - J_R1 of the semi-discrete operator (no boundary rows),
        per problem: the discrete form of Eq. Cons."""
        g = self.g
        K = self.streaming(X) + self.scattering(X)
        if self.form == "hat":
            dN = 8 * np.pi ** 2 * g.int_r(g.int_Theta_hat(K))
        else:
            dN = 8 * np.pi ** 2 * g.int_r(g.r[None, :] ** 2 * g.int_Theta_sin(K))
        J1, J2 = self.fluxes(X)
        return dN + J2 - J1


def to_hat(grid, F):
    """Fhat = r^2 sin(Th) F."""
    return F * (grid.r[None, :, None] ** 2) * np.sin(grid.Theta)[None, None, :]


def from_hat(grid, Fh):
    return Fh / ((grid.r[None, :, None] ** 2) * np.sin(grid.Theta)[None, None, :])
