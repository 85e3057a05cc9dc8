"""Plain FP64 CPU oracle for one time step of the 6-D spectral transport method.

TEST INFRASTRUCTURE ONLY. The tests, the smoke check and the bench's CPU
baseline leg are the only callers; the CUDA library never calls this module and
this module imports nothing from the library.

What it computes (Bonazzola, Vasset & Peres 2011):
  dF/dt = -L_sph F + CT,
  L_sph = cos(Th) d_r + (1/r)[ sin(Th)cos(Ph) d_th + sin(Th)sin(Ph)/sin(th) d_ph
                               - sin(Th) d_Th - sin(Th)sin(Ph) cot(th) d_Ph ]   (Eq. Liouvsph, Sect. 4.1)
  CT = eta - kappa F + kappa_s (J + b omega.H + c omega.M~.omega - F),     (Eq. Transp, Sect. 2.2)
  J = (1/4pi) int F dOmega, H = (1/4pi) int omega F dOmega, M~ = M - J I/3 with
  M = (1/4pi) int omega omega F dOmega, from the scattering kernel
  (kappa_s/4pi)(1 + b mu + c (mu^2 - 1/3)), mu = omega.omega' (Eqs. sigmadif,
  sigmatot; b: the neutrino-nucleon kernels, Eqs. crossnun, crossnup; c = 3/4,
  b = 0: Thomson, Eq. sigmaTh); b = c = 0 is isotropic scattering
on the phase-space grid (r, th, ph, Th, Ph) with energy groups as independent
slices. Every per-axis derivative follows the paper's coefficient-space route
(Sect. 5.1): nodal values -> spectral coefficients -> derivative in coefficient
space -> back to nodal values.

Readings of the paper taken here (the paper is silent or garbled on these):
  * State: nodal values; coefficients are formed per line when needed.
  * r: Chebyshev-Gauss-Lobatto nodes r_i = (R1+R2)/2 - (R2-R1)/2 cos(pi i/(Nr-1)).
  * th, Th: pole-free nodes pi (j+1/2)/N with a double-Fourier-sphere (DFS)
    parity basis: on the doubled circle F(-th, ph, Th, Ph) = F(th, ph+pi, Th, Ph+pi)
    and F(-Th, Ph) = F(Th, Ph+pi); both maps leave position and direction unchanged.
  * ph, Ph: Fourier on 2 pi l/N. Nyquist modes of first derivatives are zeroed.
  * Boundaries: Tau method (Sect. 5.1) on every stage derivative: for each
    direction node the inflow node is r = R1 when cos(Th) > 0 and r = R2
    otherwise; the top Chebyshev coefficient of dF/dt is replaced so that
    dF/dt at the inflow node equals the (static, hence zero) rate of the
    inflow data. Inflow data enter by setting F = g at the inflow nodes once
    (``apply_inflow``).
  * Time: classical RK4 by default; the paper's second-order Adams-Bashforth
    (Sect. 5.1) as scheme "ab2": F_{n+1} = F_n + dt (3/2 K_n - 1/2 K_{n-1}),
    K = Tau(-L F + CT); the paper does not say how the first step is taken:
    here K_{-1} = K_0 (one forward-Euler step), and the history restarts when
    asked (``reset_history``).
  * Quadrature: Fejer's first rule in cos(th), cos(Th) (integral of the
    polynomial interpolant); trapezoid in ph, Ph; Clenshaw-Curtis in r.
  * Split variant: one streaming-only RK4 step, then a backward-Euler
    collision step solved in closed form, then F = g again at inflow nodes
    (model: the implicit first-order source step of App. B).
  * Filter (off unless asked): sigma(k) = exp(-alpha (k/k_max)^order) per axis
    in coefficient space.

Layout: F[g][r][th][ph][Th][Ph] (numpy, float64, Ph fastest); coefficient
fields kappa, eta, kappa_s are [g][r][th][ph]; inflow data g_R1 is
[g][th][ph][NTh/2][Ph] (directions with cos Th > 0), g_R2 the other half.
"""
from __future__ import annotations

import numpy as np

AX_R, AX_TH, AX_PH, AX_TTH, AX_TPH = 1, 2, 3, 4, 5   # axes of F (axis 0 = group)


def _along(M, F, axis):
    """Apply the matrix M (n_out x n_in) along one axis of F."""
    return np.moveaxis(np.tensordot(M, F, axes=([1], [axis])), 0, axis)


class Grid:
    """Nodes and per-axis spectral machinery of one phase-space grid."""

    def __init__(self, R1, R2, Nr, Ntheta, Nphi, NTheta, NPhi, groups=1, summation="matrix"):
        """summation: "matrix" forms Chebyshev coefficients by the transform
        matrices and Fourier derivatives by numpy's FFT; "library" uses scipy's
        DCT-I for the Chebyshev transforms and explicit DFT matrices for the
        Fourier axes. Both compute the same chain in a different summation
        order; their difference measures the oracle's own rounding floor."""
        if Nr < 3 or Nphi % 2 or NPhi % 2 or NTheta % 2:
            raise ValueError("need Nr >= 3 and even N_phi, N_Phi, N_Theta")
        if summation not in ("matrix", "library"):
            raise ValueError(summation)
        self.summation = summation
        self.R1, self.R2 = float(R1), float(R2)
        self.Nr, self.Nt, self.Np, self.NT, self.NP = Nr, Ntheta, Nphi, NTheta, NPhi
        self.G = groups
        N = Nr - 1
        i = np.arange(Nr)
        self.xr = -np.cos(np.pi * i / N)                 # Chebyshev variable, ascending
        self.r = 0.5 * (R1 + R2) + 0.5 * (R2 - R1) * self.xr
        self.theta = np.pi * (np.arange(Ntheta) + 0.5) / Ntheta
        self.phi = 2 * np.pi * np.arange(Nphi) / Nphi
        self.Theta = np.pi * (np.arange(NTheta) + 0.5) / NTheta
        self.Phi = 2 * np.pi * np.arange(NPhi) / NPhi
        # Chebyshev transform pair on the Gauss-Lobatto nodes.
        # V[i][k] = T_k(x_i);  x_i = cos(pi (N - i)/N).
        k = np.arange(Nr)
        self.cheb_V = np.cos(np.pi * np.outer(N - i, k) / N)
        cbar = np.ones(Nr)
        cbar[0] = cbar[-1] = 2.0
        # c_k = 2/(N cbar_k) sum_i f_i T_k(x_i)/cbar_i   (discrete orthogonality)
        self.cheb_S = (2.0 / N) * self.cheb_V.T / cbar[:, None] / cbar[None, :]
        # derivative in coefficient space by the backward recurrence
        # b_{k-1} = b_{k+1} + 2 k a_k, b_0 halved; columns = unit coefficient vectors
        C = np.zeros((Nr, Nr))
        for col in range(Nr):
            a = np.zeros(Nr)
            a[col] = 1.0
            C[:, col] = self._cheb_deriv_coef(a)
        self.cheb_C = C * (2.0 / (R2 - R1))              # d/dr = 2/(R2-R1) d/dx
        self.shape = (groups, Nr, Ntheta, Nphi, NTheta, NPhi)

    @property
    def points(self):
        return int(np.prod(self.shape))

    @staticmethod
    def _cheb_deriv_coef(a):
        N = len(a) - 1
        b = np.zeros(N + 2)
        for kk in range(N, 0, -1):
            b[kk - 1] = b[kk + 1] + 2 * kk * a[kk]
        b[0] *= 0.5
        return b[:N + 1]

    # ------------------------------------------------------------------ r axis
    def cheb_coeffs(self, F, axis=AX_R):
        if self.summation == "library":
            # scipy's DCT-I y_k = x_0 + (-1)^k x_N + 2 sum_inner x_n cos(pi k n/N);
            # with T_k(x_i) = (-1)^k cos(pi k i/N): c_k = (-1)^k y_k/(N cbar_k)
            import scipy.fft
            N = self.Nr - 1
            y = scipy.fft.dct(F, type=1, axis=axis)
            scale = (-1.0) ** np.arange(self.Nr) / N
            scale[0] *= 0.5
            scale[-1] *= 0.5
            shp = [1] * F.ndim
            shp[axis] = self.Nr
            return y * scale.reshape(shp)
        return _along(self.cheb_S, F, axis)

    def cheb_values(self, c, axis=AX_R):
        if self.summation == "library":
            # f_i = sum_k d_k cos(pi k i/N), d_k = (-1)^k c_k: half of (DCT-I(d) + d_0 + (-1)^i d_N)
            import scipy.fft
            shp = [1] * c.ndim
            shp[axis] = self.Nr
            sgn = ((-1.0) ** np.arange(self.Nr)).reshape(shp)
            d = c * sgn
            y = scipy.fft.dct(d, type=1, axis=axis)
            d0 = np.take(d, [0], axis=axis)
            dN = np.take(d, [self.Nr - 1], axis=axis)
            return 0.5 * (y + d0 + sgn * dN)
        return _along(self.cheb_V, c, axis)

    def d_r(self, F):
        """d/dr: values -> Chebyshev coefficients -> recurrence -> values."""
        c = self.cheb_coeffs(F)
        c = _along(self.cheb_C, c, AX_R)
        return self.cheb_values(c)

    def d_r_T(self, mu):
        """Transpose of d_r (explicit transposes of the three factors)."""
        m = _along(self.cheb_V.T, mu, AX_R)
        m = _along(self.cheb_C.T, m, AX_R)
        return _along(self.cheb_S.T, m, AX_R)

    # -------------------------------------------------------- Fourier machinery
    def _fourier_deriv(self, f, axis):
        """Periodic spectral derivative along `axis` (period 2 pi, equispaced),
        Nyquist mode zeroed: coefficients, multiply by i k, back."""
        M = f.shape[axis]
        kk = np.fft.fftfreq(M, d=1.0 / M)
        mult = 1j * kk
        if M % 2 == 0:
            mult[M // 2] = 0.0
        shp = [1] * f.ndim
        shp[axis] = M
        if self.summation == "library":
            n = np.arange(M)
            E = np.exp(-2j * np.pi * np.outer(kk, n) / M)      # forward DFT, rows = modes
            c = _along(E, f.astype(complex), axis)
            return np.real(_along(np.conj(E).T / M, c * mult.reshape(shp), axis))
        c = np.fft.fft(f, axis=axis)
        return np.real(np.fft.ifft(c * mult.reshape(shp), axis=axis))

    @staticmethod
    def _fourier_filter(f, axis, sigma_of_k):
        M = f.shape[axis]
        c = np.fft.fft(f, axis=axis)
        kk = np.abs(np.fft.fftfreq(M, d=1.0 / M))
        shp = [1] * f.ndim
        shp[axis] = M
        return np.real(np.fft.ifft(c * sigma_of_k(kk).reshape(shp), axis=axis))

    def _partner_th(self, F):
        """F at the DFS partner of (th, ph, Th, Ph): (ph + pi, Ph + pi)."""
        return np.roll(np.roll(F, -self.Np // 2, axis=AX_PH), -self.NP // 2, axis=AX_TPH)

    def _partner_Th(self, F):
        """F at the DFS partner of (Th, Ph): (Ph + pi)."""
        return np.roll(F, -self.NP // 2, axis=AX_TPH)

    def _extend(self, F, axis, partner):
        """Doubled circle of 2N nodes: node n < N is th_n; node 2N-1-j carries
        the reflected angle 2 pi - th_j whose value is F at the partner."""
        return np.concatenate([F, np.flip(partner, axis=axis)], axis=axis)

    def _restrict_T(self, mu, axis):
        """Transpose of 'take the first N nodes of the doubled circle'."""
        return np.concatenate([mu, np.zeros_like(mu)], axis=axis)

    def _extend_T(self, e, axis, partner_T):
        N = e.shape[axis] // 2
        first = np.take(e, np.arange(N), axis=axis)
        second = np.flip(np.take(e, np.arange(N, 2 * N), axis=axis), axis=axis)
        return first + partner_T(second)

    def d_th(self, F):
        ext = self._extend(F, AX_TH, self._partner_th(F))
        return np.take(self._fourier_deriv(ext, AX_TH), np.arange(self.Nt), axis=AX_TH)

    def d_Th(self, F):
        ext = self._extend(F, AX_TTH, self._partner_Th(F))
        return np.take(self._fourier_deriv(ext, AX_TTH), np.arange(self.NT), axis=AX_TTH)

    def d_ph(self, F):
        return self._fourier_deriv(F, AX_PH)

    def d_Ph(self, F):
        return self._fourier_deriv(F, AX_TPH)

    # Transposes: the Nyquist-zeroed periodic derivative is antisymmetric.
    def d_ph_T(self, mu):
        return -self._fourier_deriv(mu, AX_PH)

    def d_Ph_T(self, mu):
        return -self._fourier_deriv(mu, AX_TPH)

    def _partner_th_inv(self, F):
        return np.roll(np.roll(F, self.Np // 2, axis=AX_PH), self.NP // 2, axis=AX_TPH)

    def _partner_Th_inv(self, F):
        return np.roll(F, self.NP // 2, axis=AX_TPH)

    def d_th_T(self, mu):
        e = -self._fourier_deriv(self._restrict_T(mu, AX_TH), AX_TH)
        return self._extend_T(e, AX_TH, self._partner_th_inv)

    def d_Th_T(self, mu):
        e = -self._fourier_deriv(self._restrict_T(mu, AX_TTH), AX_TTH)
        return self._extend_T(e, AX_TTH, self._partner_Th_inv)

    # ------------------------------------------------------ geometric factors
    def coefficients(self):
        """The five factors of Eq. (Liouvsph), broadcastable against F."""
        r = self.r.reshape(1, -1, 1, 1, 1, 1)
        th = self.theta.reshape(1, 1, -1, 1, 1, 1)
        Th = self.Theta.reshape(1, 1, 1, 1, -1, 1)
        Ph = self.Phi.reshape(1, 1, 1, 1, 1, -1)
        a_r = np.cos(Th)
        a_th = np.sin(Th) * np.cos(Ph) / r
        a_ph = np.sin(Th) * np.sin(Ph) / (r * np.sin(th))
        a_Th = -np.sin(Th) / r
        a_Ph = -np.sin(Th) * np.sin(Ph) * np.cos(th) / (r * np.sin(th))
        return a_r, a_th, a_ph, a_Th, a_Ph

    def liouville(self, F):
        """L_sph F (Eq. Liouvsph)."""
        a_r, a_th, a_ph, a_Th, a_Ph = self.coefficients()
        return (a_r * self.d_r(F) + a_th * self.d_th(F) + a_ph * self.d_ph(F)
                + a_Th * self.d_Th(F) + a_Ph * self.d_Ph(F))

    def liouville_T(self, mu):
        """Transpose of liouville: sum_ax D_ax^T (a_ax mu)."""
        a_r, a_th, a_ph, a_Th, a_Ph = self.coefficients()
        return (self.d_r_T(a_r * mu) + self.d_th_T(a_th * mu) + self.d_ph_T(a_ph * mu)
                + self.d_Th_T(a_Th * mu) + self.d_Ph_T(a_Ph * mu))

    # ---------------------------------------------------------- quadratures
    @staticmethod
    def fejer_integral(g, axis):
        """int_0^pi g(t) sin t dt from values at t_k = pi (k+1/2)/N: integrate
        the interpolating polynomial in cos t exactly (Fejer's first rule)."""
        N = g.shape[axis]
        t = np.pi * (np.arange(N) + 0.5) / N
        n = np.arange(N)
        Tm = np.cos(np.outer(n, t))                       # T_n(cos t_k)
        a = _along(Tm * (2.0 / N), g, axis)
        a0 = np.take(a, [0], axis=axis) * 0.5
        a = np.concatenate([a0, np.take(a, n[1:], axis=axis)], axis=axis)
        In = np.zeros(N)
        In[0::2] = 2.0 / (1.0 - n[0::2].astype(float) ** 2)
        return np.tensordot(a, In, axes=([axis], [0]))

    @staticmethod
    def trapezoid_periodic(g, axis):
        """int_0^{2 pi} g: 2 pi x the mean of the equispaced samples."""
        return 2 * np.pi * np.mean(g, axis=axis)

    def clenshaw_curtis_r(self, h, axis=AX_R):
        """int_{R1}^{R2} h dr: integrate the Chebyshev interpolant exactly."""
        c = _along(self.cheb_S, h, axis)
        k = np.arange(self.Nr)
        Ik = np.zeros(self.Nr)
        Ik[0::2] = 2.0 / (1.0 - k[0::2].astype(float) ** 2)
        return 0.5 * (self.R2 - self.R1) * np.tensordot(c, Ik, axes=([axis], [0]))

    def sphere_integral(self, F):
        """int F dOmega = int_0^pi sin Th dTh int_0^{2pi} dPh F  over the last two axes."""
        return self.fejer_integral(self.trapezoid_periodic(F, -1), -1)

    def scattering_mean(self, F):
        """J = (1/4pi) int F dOmega, shape [g][r][th][ph]."""
        return self.sphere_integral(F) / (4 * np.pi)

    def quadrature_weights_direction(self):
        """q[k][m] with J = sum q F: obtained by applying scattering_mean to
        unit vectors (the functional's own coefficients)."""
        q = np.zeros((self.NT, self.NP))
        for kk in range(self.NT):
            for m in range(self.NP):
                e = np.zeros((self.NT, self.NP))
                e[kk, m] = 1.0
                q[kk, m] = self.sphere_integral(e) / (4 * np.pi)
        return q

    # ------------------------------------------------------------ boundaries
    def inflow_mask(self):
        """True at (r, Th) inflow nodes: r = R1 for cos Th > 0, r = R2 otherwise (Sect. 4.2)."""
        m = np.zeros((self.Nr, self.NT), dtype=bool)
        h = self.NT // 2
        m[0, :h] = np.cos(self.Theta[:h]) > 0
        m[-1, h:] = np.cos(self.Theta[h:]) < 0
        return m

    def apply_inflow(self, F, g_R1=None, g_R2=None):
        F = F.copy()
        h = self.NT // 2
        F[:, 0, :, :, :h, :] = 0.0 if g_R1 is None else g_R1
        F[:, -1, :, :, h:, :] = 0.0 if g_R2 is None else g_R2
        return F

    def _inflow_node_index(self):
        return np.where(np.cos(self.Theta) > 0, 0, self.Nr - 1)

    def tau(self, K, gdot=0.0):
        """Tau boundary condition (Sect. 5.1): per r-line replace the top
        Chebyshev coefficient of K so that K at the inflow node = gdot."""
        c = self.cheb_coeffs(K)
        out_c = c.copy()
        N = self.Nr - 1
        b_of_k = self._inflow_node_index()
        for kk in range(self.NT):
            b = b_of_k[kk]
            Tb = self.cheb_V[b, :]                         # T_k(x_b)
            cl = c[:, :, :, :, kk, :]                      # [g][k][th][ph][Ph]
            val = np.tensordot(Tb, cl, axes=([0], [1]))    # K at x_b
            out_c[:, N, :, :, kk, :] += (gdot - val) / Tb[N]
        return self.cheb_values(out_c)

    def tau_T(self, mu):
        """Transpose of the linear part of tau."""
        N = self.Nr - 1
        m = _along(self.cheb_V.T, mu, AX_R)                # adjoint in coefficient space
        b_of_k = self._inflow_node_index()
        out = m.copy()
        for kk in range(self.NT):
            b = b_of_k[kk]
            Tb = self.cheb_V[b, :]
            top = m[:, N, :, :, kk, :] / Tb[N]             # [g][th][ph][Ph]
            out[:, :, :, :, kk, :] -= Tb.reshape(1, -1, 1, 1, 1) * top[:, None]
        return _along(self.cheb_S.T, out, AX_R)

    # ---------------------------------------------------------- filter
    def filter(self, F, alpha=36.0, order=16):
        """Exponential filter sigma(k) = exp(-alpha (k/k_max)^order) applied
        per axis in coefficient space (r, th, ph, Th, Ph)."""
        F = self._filter_r(F, alpha, order)
        def circ(f, axis, kmax):
            return self._fourier_filter(f, axis, lambda k: np.exp(-alpha * (k / kmax) ** order))
        ext = self._extend(F, AX_TH, self._partner_th(F))
        F = np.take(circ(ext, AX_TH, self.Nt), np.arange(self.Nt), axis=AX_TH)
        F = circ(F, AX_PH, self.Np // 2)
        ext = self._extend(F, AX_TTH, self._partner_Th(F))
        F = np.take(circ(ext, AX_TTH, self.NT), np.arange(self.NT), axis=AX_TTH)
        F = circ(F, AX_TPH, self.NP // 2)
        return F

    def _filter_r(self, F, alpha, order):
        N = self.Nr - 1
        sig_r = np.exp(-alpha * (np.arange(self.Nr) / N) ** order)
        c = self.cheb_coeffs(F)
        return self.cheb_values(c * sig_r.reshape(1, -1, 1, 1, 1, 1))

    # ------------------------------------------------------------- moments
    def direction_cartesian(self):
        """Cartesian components (ox, oy, oz) of the momentum direction omega at
        every (th, ph, Th, Ph) node, Eqs. omegax-omegaz: omega = cos Th e_r +
        sin Th cos Ph e_th + sin Th sin Ph e_ph. Shapes [th][ph][Th][Ph]."""
        th = self.theta.reshape(-1, 1, 1, 1)
        ph = self.phi.reshape(1, -1, 1, 1)
        Th = self.Theta.reshape(1, 1, -1, 1)
        Ph = self.Phi.reshape(1, 1, 1, -1)
        ox = (np.cos(Th) * np.sin(th) * np.cos(ph) + np.sin(Th) * np.cos(Ph) * np.cos(th) * np.cos(ph)
              - np.sin(Th) * np.sin(Ph) * np.sin(ph))
        oy = (np.cos(Th) * np.sin(th) * np.sin(ph) + np.sin(Th) * np.cos(Ph) * np.cos(th) * np.sin(ph)
              + np.sin(Th) * np.sin(Ph) * np.cos(ph))
        oz = np.cos(Th) * np.cos(th) - np.sin(Th) * np.cos(Ph) * np.sin(th)
        shape = (self.Nt, self.Np, self.NT, self.NP)
        return tuple(np.ascontiguousarray(np.broadcast_to(o, shape)) for o in (ox, oy, oz))

    def first_moment(self, F):
        """H = (1/4pi) int F omega dOmega, Cartesian components, [3][g][r][th][ph]."""
        return np.stack([self.scattering_mean(F * o) for o in self.direction_cartesian()])

    def second_moment(self, F):
        """M = (1/4pi) int F omega omega dOmega, Cartesian, [3][3][g][r][th][ph]."""
        o = self.direction_cartesian()
        return np.stack([np.stack([self.scattering_mean(F * o[i] * o[j]) for j in range(3)])
                         for i in range(3)])

    def moments(self, F):
        """F0 = J, F1 = (1/4pi) int F omega dOmega (Cartesian components,
        Eqs. omegax-omegaz and Fmom0), particle number N (Eq. Npho, with the
        missing dTheta restored) and the radial fluxes J_R1, J_R2 (Eq. Flux)."""
        F0 = self.scattering_mean(F)
        F1 = self.first_moment(F)
        n_dir = self.sphere_integral(F)                                  # [g][r][th][ph]
        n_pos = self.fejer_integral(self.trapezoid_periodic(n_dir, -1), -1)   # [g][r]
        r2 = (self.r ** 2)[None, :]
        Nnum = self.clenshaw_curtis_r(r2 * n_pos, axis=1)
        cosTh = np.cos(self.Theta).reshape(1, 1, 1, -1, 1)
        def flux(i, R):
            f = self.sphere_integral(F[:, i] * cosTh)                    # [g][th][ph]
            return R ** 2 * self.fejer_integral(self.trapezoid_periodic(f, -1), -1)
        return F0, F1, Nnum, flux(0, self.R1), flux(-1, self.R2)

    def outgoing_flux_weights(self):
        """w such that J_R2 = sum over [th][ph][Th][Ph] of w * F(R2, ...):
        the functional's coefficients, from unit vectors."""
        Nt, Np, NT, NP = self.Nt, self.Np, self.NT, self.NP
        w = np.zeros((Nt, Np, NT, NP))
        # separable: R2^2 * q_th[j] * (2pi/Np) * q_Th[k] cos Th_k * (2pi/NP)
        qt = np.array([self.fejer_integral(np.eye(Nt)[j], 0) for j in range(Nt)])
        qT = np.array([self.fejer_integral(np.eye(NT)[k], 0) for k in range(NT)])
        w = (self.R2 ** 2 * qt[:, None, None, None] * (2 * np.pi / Np)
             * (qT * np.cos(self.Theta))[None, None, :, None] * (2 * np.pi / NP)
             * np.ones((Nt, Np, NT, NP)))
        return w


class GridUpwindR(Grid):
    """The hybrid grid of Sect. 5.3: spectral in (th, ph, Th, Ph) as in Grid,
    first-order finite differences in r on N_r uniform nodes r_i = R1 + i dr.
    Readings: the paper's "simple first order finite-difference scheme" in r is
    taken upwind along the propagation (cos Th > 0: (F_i - F_{i-1})/dr; cos Th < 0:
    (F_{i+1} - F_i)/dr), and the inflow node (no upstream neighbour) holds the
    inflow data: its rate is zero instead of the Tau row. Radial integrals use the
    trapezoid rule; the radial filter is the identity. No adjoint."""

    def __init__(self, R1, R2, Nr, Ntheta, Nphi, NTheta, NPhi, groups=1):
        super().__init__(R1, R2, Nr, Ntheta, Nphi, NTheta, NPhi, groups)
        self.dr = (self.R2 - self.R1) / (Nr - 1)
        self.r = self.R1 + self.dr * np.arange(Nr)

    def d_r_upwind(self, F):
        """One-sided differences upstream of each direction; zero at the inflow node."""
        back = np.zeros_like(F)
        back[:, 1:] = (F[:, 1:] - F[:, :-1]) / self.dr
        fwd = np.zeros_like(F)
        fwd[:, :-1] = (F[:, 1:] - F[:, :-1]) / self.dr
        out = (np.cos(self.Theta) > 0).reshape(1, 1, 1, 1, -1, 1)
        return np.where(out, back, fwd)

    def liouville(self, F):
        a_r, a_th, a_ph, a_Th, a_Ph = self.coefficients()
        return (a_r * self.d_r_upwind(F) + a_th * self.d_th(F) + a_ph * self.d_ph(F)
                + a_Th * self.d_Th(F) + a_Ph * self.d_Ph(F))

    def tau(self, K, gdot=0.0):
        """The inflow nodes hold the static inflow data: their rate is gdot (= 0)."""
        K = K.copy()
        b_of_k = self._inflow_node_index()
        for kk in range(self.NT):
            K[:, b_of_k[kk], :, :, kk, :] = gdot
        return K

    def clenshaw_curtis_r(self, h, axis=AX_R):
        """int_{R1}^{R2} h dr by the trapezoid rule on the uniform nodes."""
        w = np.full(self.Nr, self.dr)
        w[0] = w[-1] = 0.5 * self.dr
        return np.tensordot(h, w, axes=([axis], [0]))

    def _filter_r(self, F, alpha, order):
        return F

    def d_r(self, F):
        raise NotImplementedError("the upwind radial derivative depends on the direction")

    def liouville_T(self, mu):
        raise NotImplementedError("no adjoint on the finite-difference radial grid")

    def tau_T(self, mu):
        raise NotImplementedError("no adjoint on the finite-difference radial grid")


class GridZonedR(Grid):
    """The three-zone radial grid of App. B: first-order upwind finite differences
    on n_fd uniform nodes in each edge zone of width w = zone_width (R2 - R1), and
    Chebyshev-Gauss-Lobatto differentiation on the n_sp = Nr - 2 (n_fd - 1) nodes
    of the central zone [R1 + w, R2 - w]; neighbouring zones share their interface
    node. Readings (the paper solves the central zone with its implicit radial
    update; here every zone is explicit, RK4 as elsewhere):
      * the rate at an interface node is the upstream zone's (the zone the
        direction comes from), so the value stays continuous;
      * the central zone takes that rate at its inflow interface by the Tau
        method: its top Chebyshev coefficient is replaced so that its rate there
        equals the upstream one. The non-radial parts of the rate are the same at
        the node, so this is a correction of the radial derivative alone:
          d(i) = dB(i) + (dFD(b) - dB(b)) T_N(x_i) / T_N(x_b)   (i in the central zone),
        b the inflow interface, dB the Chebyshev derivative, dFD the upstream
        zone's one-sided difference at b;
      * the outer inflow nodes hold their data (zero rate), as on the hybrid grid;
      * radial integrals: trapezoid in the edge zones, Clenshaw-Curtis in the
        central one. No adjoint, no radial filter."""

    def __init__(self, R1, R2, Nr, Ntheta, Nphi, NTheta, NPhi, groups=1, zone_nodes=30,
                 zone_width=0.1):
        super().__init__(R1, R2, Nr, Ntheta, Nphi, NTheta, NPhi, groups)
        nA = zone_nodes
        nB = Nr - 2 * (nA - 1)
        if nA < 2 or nB < 3 or not (0.0 < zone_width < 0.5):
            raise ValueError("need zone_nodes >= 2, Nr - 2 (zone_nodes - 1) >= 3, 0 < width < 1/2")
        w = zone_width * (self.R2 - self.R1)
        self.nA, self.nB, self.w = nA, nB, w
        self.iB0, self.iB1 = nA - 1, nA - 1 + nB - 1          # interface nodes (global)
        self.hA = w / (nA - 1)
        self._gB = Grid(self.R1 + w, self.R2 - w, nB, 2, 2, NTheta, 2)
        self.r = np.concatenate([self.R1 + self.hA * np.arange(nA), self._gB.r[1:-1],
                                 self.R2 - w + self.hA * np.arange(nA)])

    def _dB(self, F):
        """Chebyshev derivative of the central zone (coefficient space, its own nodes)."""
        FB = F[:, self.iB0:self.iB1 + 1]
        gB = self._gB
        c = _along(gB.cheb_S, FB, AX_R)
        c = _along(gB.cheb_C, c, AX_R)
        return _along(gB.cheb_V, c, AX_R)

    def _outward(self):
        """Directions whose inflow is at R1 (cos Theta > 0)."""
        return np.cos(self.Theta) > 0

    def _tau_profile(self, b):
        """T_N(x_i) / T_N(x_b) on the central nodes: the shape of the Tau
        correction (the top Chebyshev mode, normalised at the interface b)."""
        nB = self.nB
        tN = np.cos(np.pi * (nB - 1 - np.arange(nB)))    # T_N on the central nodes (ascending)
        return tN / tN[b]

    def d_r_zoned(self, F):
        """The radial derivative of every direction (see the class notes)."""
        h = self.hA
        nA, iB0, iB1, N = self.nA, self.iB0, self.iB1, self.Nr - 1
        back = np.zeros_like(F)
        back[:, 1:] = (F[:, 1:] - F[:, :-1]) / h       # valid inside the edge zones
        fwd = np.zeros_like(F)
        fwd[:, :-1] = (F[:, 1:] - F[:, :-1]) / h
        dB = self._dB(F)
        nB = self.nB
        out = np.zeros_like(F)
        outward = self._outward()
        for kk in range(self.NT):
            sl = (slice(None), slice(None), slice(None), slice(None), kk)
            if outward[kk]:   # from R1: zone A backward, inflow interface iB0
                out[sl][:, :iB0 + 1] = back[sl][:, :iB0 + 1]
                b, dfd = 0, back[sl][:, iB0]
                dz = dB[sl] + (dfd - dB[sl][:, b])[:, None] * self._tau_profile(b)[None, :, None, None, None]
                out[sl][:, iB0:iB1 + 1] = dz
                out[sl][:, iB0] = dfd
                out[sl][:, iB1 + 1:] = back[sl][:, iB1 + 1:]
            else:             # from R2: zone C forward, inflow interface iB1
                out[sl][:, iB1:] = fwd[sl][:, iB1:]
                b, dfd = nB - 1, fwd[sl][:, iB1]
                dz = dB[sl] + (dfd - dB[sl][:, b])[:, None] * self._tau_profile(b)[None, :, None, None, None]
                out[sl][:, iB0:iB1 + 1] = dz
                out[sl][:, iB1] = dfd
                out[sl][:, :iB0] = fwd[sl][:, :iB0]
        return out

    def liouville(self, F):
        a_r, a_th, a_ph, a_Th, a_Ph = self.coefficients()
        return (a_r * self.d_r_zoned(F) + a_th * self.d_th(F) + a_ph * self.d_ph(F)
                + a_Th * self.d_Th(F) + a_Ph * self.d_Ph(F))

    def tau(self, K, gdot=0.0):
        """The outer inflow nodes hold the static inflow data: their rate is gdot."""
        K = K.copy()
        b_of_k = self._inflow_node_index()
        for kk in range(self.NT):
            K[:, b_of_k[kk], :, :, kk, :] = gdot
        return K

    def clenshaw_curtis_r(self, h, axis=AX_R):
        """Trapezoid in the edge zones, Clenshaw-Curtis in the central one."""
        wts = np.zeros(self.Nr)
        tr = np.full(self.nA, self.hA)
        tr[0] = tr[-1] = 0.5 * self.hA
        wts[:self.nA] += tr
        wts[self.iB1:] += tr
        gB = self._gB
        k = np.arange(self.nB)
        ints = np.zeros(self.nB)
        ev = k % 2 == 0
        ints[ev] = 2.0 / (1.0 - k[ev].astype(float) ** 2)
        wts[self.iB0:self.iB1 + 1] += (ints @ gB.cheb_S) * 0.5 * (gB.R2 - gB.R1)
        return np.tensordot(h, wts, axes=([axis], [0]))

    def _filter_r(self, F, alpha, order):
        return F

    def d_r(self, F):
        raise NotImplementedError("the zoned radial derivative depends on the direction")

    def liouville_T(self, mu):
        raise NotImplementedError("no adjoint on the zoned radial grid")

    def tau_T(self, mu):
        raise NotImplementedError("no adjoint on the zoned radial grid")


class Problem:
    """Grid + coefficient fields + boundary data + scheme options."""

    def __init__(self, grid, kappa=None, eta=None, kappa_s=None, g_R1=None, g_R2=None,
                 bc="tau", scheme="rk4", filter_on=False, filter_alpha=36.0, filter_order=16,
                 scatter_b=None, scatter_c=None):
        """scatter_b, scatter_c: the coefficients of the scattering kernel
        (kappa_s/4pi)(1 + b mu + c (mu^2 - 1/3)), mu = omega.omega', each a
        [g][r][th][ph] field or a scalar; None or 0 drops the term. b = B/A of
        the neutrino-nucleon kernels A (1 + b mu) (Eqs. crossnun, crossnup);
        c = 3/4 with b = 0 is the Thomson kernel (3/16pi)(1 + mu^2) (Eq. sigmaTh)."""
        self.g = grid
        z = np.zeros((grid.G, grid.Nr, grid.Nt, grid.Np))
        self.kappa = z if kappa is None else np.asarray(kappa, dtype=np.float64)
        self.eta = z if eta is None else np.asarray(eta, dtype=np.float64)
        self.kappa_s = z if kappa_s is None else np.asarray(kappa_s, dtype=np.float64)
        self.scatter_b = z if scatter_b is None else np.broadcast_to(
            np.asarray(scatter_b, dtype=np.float64), z.shape)
        self.scatter_c = z if scatter_c is None else np.broadcast_to(
            np.asarray(scatter_c, dtype=np.float64), z.shape)
        self.g_R1, self.g_R2 = g_R1, g_R2
        self.bc, self.scheme = bc, scheme
        self._K_prev = None   # AB2 history: K of the previous step
        self.filter_on, self.filter_alpha, self.filter_order = filter_on, filter_alpha, filter_order

    def _c(self, a):
        return a[..., None, None]

    def collision(self, F):
        """CT = eta - kappa F - sigma_t F + int sigma_d(omega.omega') F(omega') dOmega'
        with sigma_d = (kappa_s/4pi)(1 + b mu + c (mu^2 - 1/3)) and kappa_s = sigma_t
        (the mu^2 - 1/3 term integrates to zero):
        CT = eta - kappa F + kappa_s (J + b omega.H + c omega.M~.omega - F), since
        (1/4pi) int (omega.omega')^2 F' dOmega' = omega.M.omega and omega.I.omega = 1."""
        J = self.g.scattering_mean(F)[..., None, None]
        CT = self._c(self.eta) - self._c(self.kappa) * F + self._c(self.kappa_s) * (J - F)
        o = self.g.direction_cartesian()
        if np.any(self.scatter_b != 0):
            H = self.g.first_moment(F)
            wH = sum(oi * h[..., None, None] for oi, h in zip(o, H))
            CT = CT + self._c(self.kappa_s * self.scatter_b) * wH
        if np.any(self.scatter_c != 0):
            M = self.g.second_moment(F)
            wMw = sum(o[i] * o[j] * M[i, j][..., None, None] for i in range(3) for j in range(3))
            CT = CT + self._c(self.kappa_s * self.scatter_c) * (wMw - J / 3.0)
        return CT

    def rhs(self, F, streaming_only=False):
        """One stage derivative K = Tau(-L F + CT) (Eq. Transpfpsph)."""
        K = -self.g.liouville(F)
        if not streaming_only:
            K = K + self.collision(F)
        if self.bc == "tau":
            K = self.g.tau(K)
        return K

    def apply_inflow(self, F):
        return self.g.apply_inflow(F, self.g_R1, self.g_R2)

    def rk4_step(self, F, dt, streaming_only=False, keep_stages=False):
        """Classical RK4: U1 = F, U2 = F + dt/2 K1, U3 = F + dt/2 K2, U4 = F + dt K3,
        F_new = F + dt/6 (K1 + 2 K2 + 2 K3 + K4)."""
        U1 = F
        K1 = self.rhs(U1, streaming_only)
        U2 = F + 0.5 * dt * K1
        K2 = self.rhs(U2, streaming_only)
        U3 = F + 0.5 * dt * K2
        K3 = self.rhs(U3, streaming_only)
        U4 = F + dt * K3
        K4 = self.rhs(U4, streaming_only)
        Fn = F + (dt / 6.0) * (K1 + 2 * K2 + 2 * K3 + K4)
        if keep_stages:
            return Fn, (U1, U2, U3, U4)
        return Fn

    def implicit_collision(self, Fs, dt):
        """Backward Euler F+ = F* + dt CT(F+), solved exactly. CT couples the
        directions only through the moments l_a(F) = (1/4pi) int phi_a F dOmega
        of phi = (1, ox, oy, oz, ox^2, oy^2, oz^2, ox oy, ox oz, oy oz): its gain
        term is kappa_s sum_a w_a phi_a l_a(F) with w = (1 - c/3, b, b, b, c, c, c,
        2c, 2c, 2c). So
          (1 + dt (kappa + kappa_s)) F+ = F* + dt eta + dt kappa_s sum_a w_a phi_a L_a,
        L_a = l_a(F+). Applying l_b gives, per position, the 10 x 10 system
          (1 + dt (kappa + kappa_s)) L_b - dt kappa_s sum_a w_a G_ba L_a = l_b(F* + dt eta),
        G_ba = l_b(phi_a) (the quadrature's own Gram matrix); then F+ from L.
        Isotropic case (b = c = 0): J+ = (J* + dt eta)/(1 + dt kappa)."""
        g = self.g
        o = g.direction_cartesian()
        phi = ((np.ones_like(o[0]),) + o + tuple(o[i] * o[i] for i in range(3))
               + (o[0] * o[1], o[0] * o[2], o[1] * o[2]))
        Gm = np.stack([np.stack([g.scattering_mean(pb * pa) for pa in phi], -1) for pb in phi], -2)
        rhs_F = Fs + dt * self._c(self.eta)
        rhs = np.stack([g.scattering_mean(rhs_F * pb) for pb in phi], -1)      # [g][r][th][ph][10]
        den = 1.0 + dt * (self.kappa + self.kappa_s)
        b, c = self.scatter_b, self.scatter_c
        w = np.stack([1.0 - c / 3.0, b, b, b, c, c, c, 2 * c, 2 * c, 2 * c], -1)
        M = (den[..., None, None] * np.eye(len(phi))
             - dt * self.kappa_s[..., None, None] * Gm[None, None] * w[..., None, :])
        L = np.linalg.solve(M, rhs[..., None])[..., 0]
        src = sum(phi[a] * (w[..., a] * L[..., a])[..., None, None] for a in range(len(phi)))
        return (rhs_F + dt * self._c(self.kappa_s) * src) / self._c(den)

    def reset_history(self):
        """Forget the AB2 history: the next step starts with forward Euler."""
        self._K_prev = None

    def ab2_step(self, F, dt):
        """Second-order Adams-Bashforth (Sect. 5.1): F + dt (3/2 K_n - 1/2 K_{n-1});
        the first step after a restart is F + dt K_0."""
        K = self.rhs(F)
        Kp = K if self._K_prev is None else self._K_prev
        self._K_prev = K
        return F + dt * (1.5 * K - 0.5 * Kp)

    def step(self, F, dt):
        if self.scheme == "rk4":
            Fn = self.rk4_step(F, dt)
        elif self.scheme == "ab2":
            Fn = self.ab2_step(F, dt)
        elif self.scheme == "split":
            Fs = self.rk4_step(F, dt, streaming_only=True)
            Fn = self.implicit_collision(Fs, dt)
            if self.bc == "tau":
                Fn = self.apply_inflow(Fn)
        else:
            raise ValueError(self.scheme)
        if self.filter_on:
            Fn = self.g.filter(Fn, self.filter_alpha, self.filter_order)
        return Fn

    def run(self, F, dt, nsteps):
        for _ in range(nsteps):
            F = self.step(F, dt)
        return F

    # ------------------------------------------------------ time-step limit
    def spectral_radius(self, x0, iters=60):
        """Power-iteration estimate of the spectral radius of the linear part of
        the stage operator, A x = rhs(x) - rhs(0) (the stage derivative with
        eta = 0 and homogeneous inflow rows), from the start field x0: x <- A x,
        renormalised each iteration; the estimate is the geometric mean of the
        growth factors ||A x|| / ||x|| over the second half of the iterations
        (their product over m iterations tends to rho^m: Gelfand's formula; the
        single factor oscillates when the largest eigenvalues are a complex
        pair, their geometric mean does not)."""
        K0 = self.rhs(np.zeros_like(x0))
        x = x0 / np.linalg.norm(x0)
        logs = []
        for _ in range(iters):
            y = self.rhs(x) - K0
            ny = np.linalg.norm(y)
            logs.append(np.log(ny))
            x = y / ny
        half = logs[len(logs) // 2:]
        return float(np.exp(np.mean(half)))

    def stable_dt(self, x0, iters=60, limit=2.6):
        """Largest dt with dt rho(A) <= limit (RK4: its stability region reaches
        2 sqrt(2) on the imaginary axis and 2.79 on the negative real axis; 2.6
        keeps a margin for the estimate) -- the explicit scheme's Courant limit
        (Sect. 5.4) from the discrete operator itself, every axis included."""
        return limit / self.spectral_radius(x0, iters)

    # ------------------------------------------------------------- adjoint
    def _A_T(self, lam):
        """Transpose of the linear stage operator
        U -> -L U - kappa U + kappa_s (J(U) + b omega.H(U) + c omega.M~(U).omega - U),
        with J(U) = sum q U, H(U) = sum q omega U, M(U) = sum q omega omega U: the
        scattering part transposes to q (sum kappa_s lam) + q omega.(sum kappa_s b
        omega lam) + q omega.(sum kappa_s c omega omega lam).omega - q (sum kappa_s c lam)/3."""
        q = self._q
        s = np.sum(self._c(self.kappa_s) * lam, axis=(-2, -1), keepdims=True)
        out = (-self.g.liouville_T(lam) - self._c(self.kappa) * lam
               + q * s - self._c(self.kappa_s) * lam)
        o = self.g.direction_cartesian()
        if np.any(self.scatter_b != 0):
            kb = self._c(self.kappa_s * self.scatter_b)
            for oi in o:
                out = out + q * oi * np.sum(kb * oi * lam, axis=(-2, -1), keepdims=True)
        if np.any(self.scatter_c != 0):
            # U -> kappa_s c (sum_ij o_i o_j M_ij(U) - J(U)/3), M_ij(U) = sum q o_i o_j U
            kc = self._c(self.kappa_s * self.scatter_c)
            for i in range(3):
                for j in range(3):
                    out = out + q * o[i] * o[j] * np.sum(kc * o[i] * o[j] * lam, axis=(-2, -1),
                                                         keepdims=True)
            out = out - q * np.sum(kc * lam, axis=(-2, -1), keepdims=True) / 3.0
        return out

    def adjoint_step(self, F_n, lam, dt):
        """Discrete adjoint of one RK4 step (plain RK4 scheme, filter off).

        Given F_n and lam = dObj/dF_{n+1}, returns (lam_n, g_kappa, g_eta) where
        lam_n = (dF_{n+1}/dF_n)^T lam and g_kappa, g_eta ([g][r][th][ph]) are the
        contributions of this step to dObj/dkappa and dObj/deta."""
        if self.scheme != "rk4" or self.filter_on:
            raise NotImplementedError("adjoint covers the plain RK4 step")
        self._q = self.g.quadrature_weights_direction()
        _, U = self.rk4_step(F_n, dt, keep_stages=True)
        w = np.array([1.0, 2.0, 2.0, 1.0]) * dt / 6.0
        gk = np.zeros_like(self.kappa)
        ge = np.zeros_like(self.eta)
        lam_n = lam.copy()
        Ubar_next = None
        for s in (3, 2, 1, 0):
            Kbar = w[s] * lam
            if s == 3:
                pass
            elif s == 2:
                Kbar = Kbar + dt * Ubar_next
            else:
                Kbar = Kbar + 0.5 * dt * Ubar_next
            lt = self.g.tau_T(Kbar) if self.bc == "tau" else Kbar
            ge += lt.sum(axis=(-2, -1))
            gk -= (lt * U[s]).sum(axis=(-2, -1))
            Ubar = self._A_T(lt)
            lam_n = lam_n + Ubar
            Ubar_next = Ubar
        return lam_n, gk, ge


    def _ab2_adjoint_weights(self, first):
        """Weights of dObj/dF_{n+1} and dObj/dF_{n+2} in the stage-derivative
        adjoint mu_n: K_n enters step n with dt (the start) or 3/2 dt, and step
        n+1 with -1/2 dt."""
        return (1.0 if first else 1.5), -0.5

    def adjoint_step_ab2(self, F_n, lam, lam_prev, dt, first):
        """Discrete adjoint of one AB2 step (filter off). The forward marching
        F_{n+1} = F_n + dt (3/2 K_n - 1/2 K_{n-1}) (n >= 1) and F_1 = F_0 + dt K_0
        uses K_n = K(F_n) in step n (weight 3/2 dt, or dt in the starting step) and
        in step n+1 (weight -1/2 dt). So with lam = dObj/dF_{n+1} and lam_prev =
        dObj/dF_{n+2} (zero for the last step), the stage-derivative adjoint is
        mu_n = dt (w lam - lam_prev/2), w = 1 if `first` (n = 0) else 3/2, and
          dObj/dF_n = lam + A^T Tau^T mu_n,
          g_kappa = -sum_(Th,Ph) (Tau^T mu_n) F_n,   g_eta = sum_(Th,Ph) Tau^T mu_n.
        Returns (dObj/dF_n, g_kappa, g_eta); the caller then passes (dObj/dF_n,
        lam) as (lam, lam_prev) of the step before."""
        if self.filter_on:
            raise NotImplementedError("adjoint covers steps without the filter")
        self._q = self.g.quadrature_weights_direction()
        w, w_prev = self._ab2_adjoint_weights(first)
        mu = dt * (w * lam + w_prev * lam_prev)
        lt = self.g.tau_T(mu) if self.bc == "tau" else mu
        ge = lt.sum(axis=(-2, -1))
        gk = -(lt * F_n).sum(axis=(-2, -1))
        return lam + self._A_T(lt), gk, ge


def nucleon_scattering(A_n, A_p):
    """Scattering of neutrinos on neutrons and protons (Eqs. cross, crossnun,
    crossnup, Sect. 6): sigma^D = A_n (1 - omega.omega'/3) + A_p (1 - omega.omega'/10).
    Returns (kappa_s, b) of the single kernel (kappa_s/4pi)(1 + b omega.omega'):
    kappa_s = 4 pi (A_n + A_p), b = -(A_n/3 + A_p/10)/(A_n + A_p)."""
    A_n = np.asarray(A_n, dtype=np.float64)
    A_p = np.asarray(A_p, dtype=np.float64)
    A = A_n + A_p
    return 4 * np.pi * A, -(A_n / 3.0 + A_p / 10.0) / A


def exact_free_streaming(grid, F0_of, t):
    """Exact vacuum solution with zero inflow (rays are straight lines, Eq. Tra1):
    F(t, x, omega) = F0(x - t omega, omega) if the segment {x - s omega, 0<=s<=t}
    stays inside R1 <= |.| <= R2, else 0. F0_of(r, cosTheta) must be independent
    of theta, phi, Phi. Returns [Nr][NTheta]."""
    r = grid.r[:, None]
    mu = np.cos(grid.Theta)[None, :]
    rp2 = r ** 2 - 2 * r * t * mu + t ** 2
    rp = np.sqrt(np.maximum(rp2, 0.0))
    mup = (r * mu - t) / np.where(rp > 0, rp, 1.0)
    # closest approach to the origin along the back-traced segment
    s_star = r * mu                                    # parameter of closest approach
    inside_seg = (s_star > 0) & (s_star < t)
    dmin = np.where(inside_seg, r * np.sqrt(np.maximum(1 - mu ** 2, 0.0)), np.minimum(r, rp))
    ok = (rp <= grid.R2 * (1 + 1e-14)) & (dmin >= grid.R1 * (1 - 1e-14))
    return np.where(ok, F0_of(rp, mup), 0.0)
