"""Pins of the conservative 2-D (r, Theta) oracle (App. A and App. B):

* the plain 2-D form equals the 5-D oracle (itself pinned) on spherically
  symmetric data, boundary rows included (Eq. Sphersy is the reduction);
* the conservative form of band-limited data equals r^2 sin(Th) times the
  plain form (the change of variable of Eq. flux, App. B);
* number conservation (Eq. Cons): the conservative operator's discrete
  balance dN/dt + J_R2 - J_R1 vanishes to rounding on data without a Theta
  Nyquist mode, term by term (radial flux, Theta term, scattering), and the
  fully discrete RK4 balance with the stage fluxes holds to rounding; the
  plain form's balance error is at the truncation level instead;
* isotropic radiation is a steady state, and planted mistakes fail a pin.
"""
import numpy as np
import pytest

from oracle.conservative2d import Grid2D, Problem2D, from_hat, to_hat
from oracle.transport import Grid as Grid5, Problem as Problem5

R1, R2 = 0.2, 1.0


def _smooth(g, P, seed, rdeg, tdeg):
    """Band-limited data: a polynomial of degree rdeg in r times a polynomial of
    degree tdeg in cos(Th) per problem (F: even on the doubled Theta circle)."""
    rng = np.random.default_rng(seed)
    x = (2 * g.r - R1 - R2) / (R2 - R1)
    out = np.zeros((P, g.Nr, g.NT))
    for p in range(P):
        a = rng.standard_normal((rdeg + 1, tdeg + 1))
        for i in range(rdeg + 1):
            for k in range(tdeg + 1):
                out[p] += a[i, k] * np.polynomial.chebyshev.chebval(x, np.eye(rdeg + 1)[i])[:, None] \
                    * np.cos(g.Theta)[None, :] ** k
    return out


def _ks(g, P, seed=3):
    rng = np.random.default_rng(seed)
    return 0.5 + rng.uniform(0, 1, (P, 1)) * (1 + 0.3 * np.sin(3 * g.r))[None, :]


@pytest.mark.parametrize("bc", ["none", "tau"])
@pytest.mark.parametrize("c", [0.0, 0.75])
def test_plain_form_is_the_5d_oracle_on_spherically_symmetric_data(bc, c):
    g = Grid2D(R1, R2, 9, 8)
    P = 2
    F = _smooth(g, P, 1, 6, 5)
    ks = _ks(g, P)
    K2 = Problem2D(g, ks, c=c, form="plain", bc=bc).rhs(F)
    g5 = Grid5(R1, R2, 9, 4, 4, 8, 6, groups=P)
    F5 = np.ascontiguousarray(np.broadcast_to(F[:, :, None, None, :, None], g5.shape))
    ks5 = np.ascontiguousarray(np.broadcast_to(ks[:, :, None, None], (P, 9, 4, 4)))
    gin = F5[:, 0, :, :, :4] * 0 + F5[:, 0, :, :, :4]      # static inflow = data at the inflow nodes
    pr5 = Problem5(g5, None, None, ks5, F5[:, 0, :, :, :4], F5[:, -1, :, :, 4:],
                   bc=bc, scatter_c=c if c else None)
    K5 = pr5.rhs(F5)
    assert np.abs(K5 - K5[:, :, :1, :1, :, :1]).max() < 1e-12 * np.abs(K5).max()
    assert np.abs(K5[:, :, 0, 0, :, 0] - K2).max() < 1e-12 * np.abs(K2).max()


@pytest.mark.parametrize("bc", ["none", "tau"])
@pytest.mark.parametrize("form", ["plain", "hat"])
def test_three_zone_2d_is_the_5d_three_zone_oracle_on_spherically_symmetric_data(bc, form):
    """On the three-zone radial grid of App. B, the plain 2-D form equals the 5-D
    oracle's three-zone grid (itself pinned) on spherically symmetric data, held
    inflow nodes included; the conservative form's radial term is the same zoned
    derivative of Fhat (its Theta and scattering terms are the Chebyshev grid's)."""
    from oracle.transport import GridZonedR
    nA, nB = 5, 9
    Nr = 2 * (nA - 1) + nB
    g = Grid2D(R1, R2, Nr, 8, zone_nodes=nA, zone_width=0.1)
    gc = Grid2D(R1, R2, Nr, 8)
    P = 2
    F = _smooth(g, P, 1, 6, 5)
    ks = _ks(g, P)
    if form == "plain":
        K2 = Problem2D(g, ks, c=0.75, form="plain", bc=bc).rhs(F)
        g5 = GridZonedR(R1, R2, Nr, 4, 4, 8, 6, groups=P, zone_nodes=nA, zone_width=0.1)
        F5 = np.ascontiguousarray(np.broadcast_to(F[:, :, None, None, :, None], g5.shape))
        ks5 = np.ascontiguousarray(np.broadcast_to(ks[:, :, None, None], (P, Nr, 4, 4)))
        pr5 = Problem5(g5, None, None, ks5, F5[:, 0, :, :, :4], F5[:, -1, :, :, 4:], bc=bc,
                       scatter_c=0.75)
        K5 = pr5.rhs(F5)
        assert np.abs(K5[:, :, 0, 0, :, 0] - K2).max() < 1e-12 * np.abs(K2).max()
    else:
        # the zoned conservative operator minus the Chebyshev one on the same nodes is
        # -cos(Th) times the difference of their r derivatives (Tau/hold rows aside)
        Kz = Problem2D(g, ks, form="hat", bc="none").rhs(F)
        gc.r = g.r   # the same nodes for the non-radial terms
        pc = Problem2D(gc, ks, form="hat", bc="none")
        diff = Kz - pc.rhs(F)
        ct = np.cos(g.Theta)[None, None, :]
        expect = -ct * (g.d_r(F) - gc.d_r(F))
        assert np.abs(diff - expect).max() < 1e-12 * np.abs(Kz).max()


@pytest.mark.parametrize("c", [0.0, 0.75])
def test_conservative_form_is_the_plain_form_times_the_jacobian(c):
    g = Grid2D(R1, R2, 11, 12)
    F = _smooth(g, 3, 2, 7, 8)             # r^2 F: degree 9 <= Nr - 1; sin(Th) F: sine degree 9 < 12
    ks = _ks(g, 3)
    Kp = Problem2D(g, ks, c=c, form="plain", bc="none").rhs(F)
    Kh = Problem2D(g, ks, c=c, form="hat", bc="none").rhs(to_hat(g, F))
    assert np.abs(Kh - to_hat(g, Kp)).max() < 1e-12 * np.abs(Kh).max()
    assert np.abs(from_hat(g, to_hat(g, F)) - F).max() < 1e-14 * np.abs(F).max()


def test_number_and_fluxes_agree_between_forms():
    g = Grid2D(R1, R2, 9, 8)
    F = _smooth(g, 2, 4, 5, 5)
    pp = Problem2D(g, _ks(g, 2), form="plain")
    ph = Problem2D(g, _ks(g, 2), form="hat")
    Nh, Np = ph.number(to_hat(g, F)), pp.number(F)
    assert np.abs(Nh - Np).max() < 1e-13 * np.abs(Np).max()
    for a, b in zip(ph.fluxes(to_hat(g, F)), pp.fluxes(F)):
        assert np.abs(a - b).max() < 1e-13 * np.abs(b).max()
    # N of F = 1: 8 pi^2 (R2^3 - R1^3)/3 * 2
    one = np.ones((1, g.Nr, g.NT))
    assert abs(pp.number(one)[0] - 16 * np.pi ** 2 * (R2 ** 3 - R1 ** 3) / 3) < 1e-12


def _random_hat(g, P, seed):
    """Random conservative data of full radial degree with no Theta Nyquist mode:
    Fhat = sum_{m < NT} b_m(r) sin(m Th)."""
    rng = np.random.default_rng(seed)
    m = np.arange(1, g.NT)
    b = rng.standard_normal((P, g.Nr, g.NT - 1))
    return np.einsum("pim,km->pik", b, np.sin(np.outer(g.Theta, m)))


@pytest.mark.parametrize("c", [0.0, 0.75])
def test_conservative_balance_is_exact_and_the_plain_one_is_not(c):
    """N_r = 10: with an odd number N of Chebyshev intervals the Clenshaw-Curtis
    rule is exact to degree N only, so the plain form's r^2 dF/dr (degree N+1)
    leaves a radial balance error; the conservative form's dFhat/dr has degree
    N-1 and balances exactly for every N_r. (With N even both radial terms are
    integrated exactly; in Theta both forms balance on data without the Nyquist
    sine mode of Fhat.)"""
    g = Grid2D(R1, R2, 10, 8)
    X = _random_hat(g, 3, 5)
    ks = _ks(g, 3)
    ph = Problem2D(g, ks, c=c, form="hat", bc="none")
    scale = np.abs(ph.fluxes(X)[1]).max() + np.abs(ph.number(X)).max()
    res = ph.balance_residual(X)
    assert np.abs(res).max() < 1e-13 * scale
    # term by term: radial flux, Theta term, scattering
    r = g.r[None, :, None]
    ct, st = np.cos(g.Theta), np.sin(g.Theta)
    rad = 8 * np.pi ** 2 * g.int_r(g.int_Theta_hat(-ct * g.d_r(X)))
    J1, J2 = ph.fluxes(X)
    assert np.abs(rad + J2 - J1).max() < 1e-13 * scale
    th = 8 * np.pi ** 2 * g.int_r(g.int_Theta_hat((st * g.d_Theta(X, -1.0) +
                                                   ct * g.nyquist_free(X)) / r))
    assert np.abs(th).max() < 1e-13 * scale
    # a Nyquist sine mode in Fhat: exact with the projection, not without it
    Xn = X + np.sin(g.NT * g.Theta)[None, None, :] * g.r[None, :, None]
    assert np.abs(ph.balance_residual(Xn)).max() < 1e-13 * scale
    th_raw = 8 * np.pi ** 2 * g.int_r(g.int_Theta_hat((st * g.d_Theta(Xn, -1.0) + ct * Xn) / r))
    assert np.abs(th_raw).max() > 1e-6 * scale
    assert np.abs(8 * np.pi ** 2 * g.int_r(g.int_Theta_hat(ph.scattering(X)))).max() < 1e-13 * scale
    # the plain form of the same data: balance error at the truncation level
    pp = Problem2D(g, ks, c=c, form="plain", bc="none")
    assert np.abs(pp.balance_residual(from_hat(g, X))).max() > 1e-6 * scale
    # with an even number of intervals the plain radial term balances too
    g9 = Grid2D(R1, R2, 9, 8)
    X9 = _random_hat(g9, 3, 5)
    p9 = Problem2D(g9, _ks(g9, 3), c=c, form="plain", bc="none")
    assert np.abs(p9.balance_residual(from_hat(g9, X9))).max() < 1e-12 * scale


def test_rk4_number_balance_with_stage_fluxes():
    """N_n - N_0 + dt sum_steps sum_s b_s (J_R2 - J_R1)(U_s) = 0 to rounding."""
    g = Grid2D(R1, R2, 9, 8)
    X = _random_hat(g, 2, 6) * 0.1
    ph = Problem2D(g, _ks(g, 2), form="hat", bc="none")
    dt = 2e-3
    N0 = ph.number(X)
    flux = 0.0
    for _ in range(20):
        st = []
        X = ph.rk4_step(X, dt, stages=st)
        for b, U in zip((1 / 6, 1 / 3, 1 / 3, 1 / 6), st):
            J1, J2 = ph.fluxes(U)
            flux = flux + dt * b * (J2 - J1)
    assert np.abs(ph.number(X) - N0 + flux).max() < 1e-13 * np.abs(N0).max()


def test_isotropic_radiation_is_steady():
    g = Grid2D(R1, R2, 9, 8)
    X = to_hat(g, 2.5 * np.ones((1, g.Nr, g.NT)))
    for c in (0.0, 0.75):
        ph = Problem2D(g, _ks(g, 1), c=c, form="hat", bc="tau")
        assert np.abs(ph.rhs(X)).max() < 1e-13


def test_planted_mistakes_fail_a_pin():
    g = Grid2D(R1, R2, 9, 8)
    X = _random_hat(g, 2, 7)
    F = _smooth(g, 2, 8, 5, 5)
    ks = _ks(g, 2)

    class NoCos(Problem2D):          # the cos(Th) Fhat / r term dropped
        def streaming(self, Y):
            ct, st = np.cos(self.g.Theta), np.sin(self.g.Theta)
            return -ct * self.g.d_r(Y) + st * self.g.d_Theta(Y, -1.0) / self.g.r[None, :, None]

    class EvenHat(Problem2D):        # Fhat extended as even on the doubled circle
        def streaming(self, Y):
            ct, st = np.cos(self.g.Theta), np.sin(self.g.Theta)
            r = self.g.r[None, :, None]
            return -ct * self.g.d_r(Y) + (st * self.g.d_Theta(Y, +1.0) +
                                          ct * self.g.nyquist_free(Y)) / r

    class HalfKernel(Problem2D):     # the kernel without its Phi'-average factor 1/2
        def _kernel(self):
            return 2.0 * super()._kernel()

    for bad in (NoCos, EvenHat, HalfKernel):
        pb = bad(g, ks, form="hat", bc="none")
        scale = np.abs(pb.fluxes(X)[1]).max() + np.abs(pb.number(X)).max()
        balance_ok = np.abs(pb.balance_residual(X)).max() < 1e-13 * scale
        Kp = Problem2D(g, ks, form="plain", bc="none").rhs(F)
        jac_ok = np.abs(pb.rhs(to_hat(g, F)) - to_hat(g, Kp)).max() < 1e-12 * np.abs(Kp).max()
        assert not (balance_ok and jac_ok), bad.__name__
